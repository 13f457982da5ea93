"""Full-field parity of the benchmark's own path at 2048^2 against the FP64 oracle.

The benchmark step runs, for a batch of 2048^2 complex64 fields with mixed distances in one call:
the RS forward that saves the input's 2D spectrum (row-major intermediate, bulk-copy column
gather), the row-major CZT forward onto the 512^2 window, the CZT adjoint, and the RS adjoint that
reads the saved spectrum and returns the distance gradient. Here the same calls, on three fields
at z = 0.5, 2 and 10 mm in ONE batched call (so the per-element spectra and chirp tables of the
mixed-distance launches are exercised), are compared pixel by pixel with the oracle's FFT
realisation of the RS convolution and its direct separable CZT sums. The vectorial workload
(VRS and VCZT at 2048^2, z = 5 mm, radially polarised Gaussian and a random Jones field) is
compared the same way, and so is one whole gradient step of the benchmark (its own step object)
against the oracle's composition. Paper passages: Methods, "Features and performance" (RS, VRS,
CZT on 2048^2 grids; the propagation benchmark of the Introduction's speed-up figure).

Bars: relative L2 over every pixel <= 2e-5 for fields; <= 1e-3 relative for distance gradients.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

W = inputs.WORKLOADS["rs2048"]
LAM = W["wavelength"]
ZS = list(W["zs"])  # 0.5, 2, 10 mm: one field each, one batched call


def _rs2048_fields():
    g = inputs.Grid.centred(W["n"], W["pitch"])
    win = inputs.Window.centred(W["window_m"], W["window_w"])
    u = np.stack([inputs.gaussian_random_phase(g, W["w0"], W["seed"] + b) for b in range(len(ZS))]
                 ).astype(np.complex64)
    GA = inputs.random_unit(7, (len(ZS), g.ny, g.nx)).astype(np.complex64)
    GC = inputs.random_unit(8, (len(ZS), win.my, win.mx)).astype(np.complex64)
    return g, win, u, GA, GC


@pytest.fixture(scope="module")
def gpu_step():
    """The benchmark step's library calls on the three fields (one batched call each)."""
    xl = lib()
    g, win, u, GA, GC = _rs2048_fields()
    U = to_dev(u, np.complex64)
    S = xl.save_buffer(U)
    A = to_np(xl.rs_propagate(U, g, LAM, ZS, saved=S))
    C = to_np(xl.czt_propagate(U, g, win, LAM, ZS))
    gc = to_np(xl.czt_propagate_backward(to_dev(GC, np.complex64), g, win, LAM, ZS))
    ga, gz = xl.rs_propagate_backward(to_dev(GA, np.complex64), None, g, LAM, ZS, want_field=True,
                                      want_dz=True, saved=S)
    xl.device_status()
    return dict(g=g, win=win, u=u, GA=GA, GC=GC, A=A, C=C, gc=gc, ga=to_np(ga), gz=to_np(gz))


@pytest.mark.parametrize("b", range(len(ZS)))
def test_rs_forward_adjoint_dz_full_field_2048(gpu_step, b):
    s = gpu_step
    g, z = s["g"], ZS[b]
    u0 = s["u"][b].astype(np.complex128)
    ref = oracle.rs_conv(u0, g.dx, g.dy, LAM, z)
    assert rel(s["A"][b], ref) < TOL_C64
    G = s["GA"][b].astype(np.complex128)
    ref_g = oracle.rs_conv(G, g.dx, g.dy, LAM, z, oracle.K_H, adjoint=True)
    assert rel(s["ga"][b], ref_g) < TOL_C64
    # dL/dz = Re sum conj(G) dA/dz, with dA/dz the convolution with dh/dz
    dz = float(np.real(np.vdot(G, oracle.rs_conv(u0, g.dx, g.dy, LAM, z, oracle.K_DH))))
    assert abs(s["gz"][b] - dz) <= 1e-3 * abs(dz), (b, s["gz"][b], dz)


@pytest.mark.parametrize("b", range(len(ZS)))
def test_czt_forward_adjoint_full_window_2048_to_512(gpu_step, b):
    s = gpu_step
    g, win, z = s["g"], s["win"], ZS[b]
    u0 = s["u"][b].astype(np.complex128)
    ref = oracle.czt_conv(u0, g.astuple(), win.astuple(), LAM, z)
    assert rel(s["C"][b], ref) < TOL_C64
    ref_g = oracle.czt_conv(s["GC"][b].astype(np.complex128), g.astuple(), win.astuple(), LAM, z,
                            adjoint=True)
    assert rel(s["gc"][b], ref_g) < TOL_C64


def _vrs_inputs():
    w = inputs.WORKLOADS["vrs2048"]
    g = inputs.Grid.centred(w["n"], w["pitch"])
    exy = np.stack([inputs.radial_gaussian(g, w["w0"]),
                    inputs.random_jones(g, w["w0"], w["seed"])]).astype(np.complex64)
    return w, g, exy


def test_vrs_2048_full_field_forward_adjoint_dz():
    """VRS at 2048^2 (z = 5 mm), the saved-spectrum forward and adjoint the optimiser uses."""
    xl = lib()
    w, g, exy = _vrs_inputs()
    lam, z = w["wavelength"], w["z"]
    B = exy.shape[0]
    E = to_dev(exy, np.complex64)
    S = xl.save_buffer(E, 2)
    out = to_np(xl.vrs_propagate(E, g, lam, [z] * B, saved=S))
    Gh = inputs.random_unit(23, (B, 3, g.ny, g.nx)).astype(np.complex64)
    gi, gz = xl.vrs_propagate_backward(to_dev(Gh, np.complex64), None, g, lam, [z] * B,
                                       want_field=True, want_dz=True, saved=S)
    gi, gz = to_np(gi), to_np(gz)
    xl.device_status()
    for b in range(B):
        e = exy[b].astype(np.complex128)
        assert rel(out[b], oracle.vrs(e, g.dx, g.dy, lam, z)) < TOL_C64, b
        G = Gh[b].astype(np.complex128)
        assert rel(gi[b], oracle.vrs_adjoint(G, g.dx, g.dy, lam, z)) < TOL_C64, b
        dz = float(np.real(np.vdot(G, oracle.vrs_dz(e, g.dx, g.dy, lam, z))))
        assert abs(gz[b] - dz) <= 1e-3 * abs(dz), (b, gz[b], dz)


def test_vczt_2048_to_512_full_window_forward_adjoint():
    xl = lib()
    w, g, exy = _vrs_inputs()
    win = inputs.Window.centred(w["window_m"], w["window_w"])
    lam, z = w["wavelength"], w["z"]
    B = exy.shape[0]
    out = to_np(xl.czt_propagate(to_dev(exy, np.complex64), g, win, lam, [z] * B, vectorial=1))
    Gh = inputs.random_unit(24, (B, 3, win.my, win.mx)).astype(np.complex64)
    gi = to_np(xl.czt_propagate_backward(to_dev(Gh, np.complex64), g, win, lam, [z] * B,
                                         vectorial=1))
    xl.device_status()
    for b in range(B):
        e = exy[b].astype(np.complex128)
        assert rel(out[b], oracle.vczt(e, g.astuple(), win.astuple(), lam, z)) < TOL_C64, b
        ref = oracle.vczt_adjoint(Gh[b].astype(np.complex128), g.astuple(), win.astuple(), lam, z)
        assert rel(gi[b], ref) < TOL_C64, b


def test_benchmark_gradient_step_against_oracle_composition():
    """One step of the benchmark's gradient evaluation (SLM -> RS and CZT -> spot-size losses ->
    adjoints with dL/dz -> mask gradient -> Adam) on the three fields at 0.5, 2 and 10 mm, run by
    the benchmark's own step object, against the same composition in FP64 by the oracle: the two
    losses (1e-4), the phase-invariant dL/dz (1e-3) and the mask gradient (relative L2 1e-3)."""
    import torch
    import bench
    xl = lib()
    g, win, u, _, _ = _rs2048_fields()
    step = bench.GpuStep(xl, torch, g, win, to_dev(u, np.complex64), ZS)
    lA, lC, gz, gphi = (to_np(t) for t in step.run())
    xl.device_status()
    for b in range(len(ZS)):
        st = (np.zeros((g.ny, g.nx)), np.zeros((g.ny, g.nx)), 0)
        _, _, ref = bench.oracle_step(u[b], np.zeros((g.ny, g.nx)), g, win, ZS[b], st)
        assert abs(lA[b] - ref["loss_a"]) <= 1e-4 * abs(ref["loss_a"]), b
        assert abs(lC[b] - ref["loss_c"]) <= 1e-4 * abs(ref["loss_c"]), b
        assert abs(gz[b] - ref["dz"]) <= 1e-3 * abs(ref["dz"]), (b, gz[b], ref["dz"])
        assert rel(gphi[b], ref["gphi"]) < 1e-3, b
