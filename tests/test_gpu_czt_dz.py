"""Segmented Bluestein CZT and the CZT distance gradient against the FP64 oracle.

- Segment plans (the grid side of an axis cut into S segments whose spectra are summed before
  one inverse transform): full-window parity of the forward and the adjoint, scalar and
  vectorial, complex64 and complex128, on sizes where S > 1, the last segment is ragged and the
  two axes take different plans.
- dL/dz = Re sum conj(G) du_out/dz (Methods, "Features and performance": the CZT propagator; the
  paper trains distances by reverse-mode gradients) against the oracle's sum with the derivative
  kernel dK/dz (kind 3; kinds 4 and 5 for the Ez kernel of VCZT), which the oracle tests pin by
  finite differences; with the forward's saved sums and with the sums formed in the adjoint
  call; host and device distances; the phase-invariant form; the autograd wrapper.
Bars: fields 2e-5 (complex64) / 1e-10 (complex128) relative L2; g_z 1e-3 (complex64) /
1e-8 (complex128) relative.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C64, TOL_C128, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

LAM = 0.6328


def _case(nx, ny, mx, my, seed):
    g = inputs.Grid(nx, ny, 0.5, 0.6, -(nx // 2) * 0.5 + 0.1, -(ny // 2) * 0.6 - 0.2)
    win = inputs.Window(mx, my, 0.3, 0.25, -mx * 0.15 + 0.05, -my * 0.125 - 0.07)
    u = inputs.gaussian_random_phase(g, 0.15 * min(nx, ny), seed)
    return g, win, u


def _tol(dtype):
    return TOL_C64 if dtype == np.complex64 else TOL_C128


# (nx, ny, mx, my): S > 1 on both axes (ragged last segments), different plans per axis,
# and a plain one-segment case
SIZES = [(300, 256, 40, 64), (1000, 523, 100, 31), (96, 80, 90, 70)]


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("size", SIZES)
def test_segmented_forward_and_adjoint_full_window(size, dtype):
    xl = lib()
    nx, ny, mx, my = size
    g, win, u = _case(nx, ny, mx, my, 5100 + nx)
    zs = [700.0, 2500.0]
    U = np.stack([u, np.roll(u, 7, axis=1)]).astype(dtype)
    out = to_np(xl.czt_propagate(to_dev(U, dtype), g, win, LAM, zs))
    G = inputs.random_unit(5101, (2, my, mx)).astype(dtype)
    gi = to_np(xl.czt_propagate_backward(to_dev(G, dtype), g, win, LAM, zs))
    for b in range(2):
        ref = oracle.czt_conv(U[b].astype(np.complex128), g.astuple(), win.astuple(), LAM, zs[b])
        assert rel(out[b], ref) < _tol(dtype), b
        ref = oracle.czt_conv(G[b].astype(np.complex128), g.astuple(), win.astuple(), LAM, zs[b],
                              adjoint=True)
        assert rel(gi[b], ref) < _tol(dtype), b


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_segmented_vectorial_forward_and_adjoint(dtype):
    xl = lib()
    g, win, _ = _case(512, 300, 64, 48, 5200)
    exy = np.stack([inputs.radial_gaussian(g, 60.0), inputs.random_jones(g, 60.0, 5201)]).astype(dtype)
    z = 900.0
    out = to_np(xl.czt_propagate(to_dev(exy, dtype), g, win, LAM, [z, z], vectorial=1))
    G = inputs.random_unit(5202, (2, 3, win.my, win.mx)).astype(dtype)
    gi = to_np(xl.czt_propagate_backward(to_dev(G, dtype), g, win, LAM, [z, z], vectorial=1))
    for b in range(2):
        e = exy[b].astype(np.complex128)
        assert rel(out[b], oracle.vczt(e, g.astuple(), win.astuple(), LAM, z)) < _tol(dtype)
        ref = oracle.vczt_adjoint(G[b].astype(np.complex128), g.astuple(), win.astuple(), LAM, z)
        assert rel(gi[b], ref) < _tol(dtype)


def _dz_ref(u, G, g, win, z, kind=3):
    d = oracle.czt_conv(u.astype(np.complex128), g.astuple(), win.astuple(), LAM, z, kind)
    return float(np.real(np.vdot(G.astype(np.complex128), d)))


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("size", SIZES[:2])
def test_czt_distance_gradient_saved_and_recomputed(size, dtype):
    import torch
    xl = lib()
    nx, ny, mx, my = size
    g, win, u = _case(nx, ny, mx, my, 5300 + nx)
    zs = [600.0, 1800.0, 5000.0]
    U = np.stack([u, np.roll(u, 5, axis=0), np.conj(u)]).astype(dtype)
    G = inputs.random_unit(5301, (3, my, mx)).astype(dtype)
    Ud, Gd = to_dev(U, dtype), to_dev(G, dtype)
    S = xl.czt_save_buffer(Ud, g, win)
    out_s = xl.czt_propagate(Ud, g, win, LAM, zs, saved=S)
    assert torch.equal(out_s, xl.czt_propagate(Ud, g, win, LAM, zs)) or \
        rel(to_np(out_s), to_np(xl.czt_propagate(Ud, g, win, LAM, zs))) < _tol(dtype)
    gi_s, gz_s = xl.czt_propagate_backward(Gd, g, win, LAM, zs, u_in=Ud, want_dz=True, saved=S)
    gi_r, gz_r = xl.czt_propagate_backward(Gd, g, win, LAM, zs, u_in=Ud, want_dz=True)
    gi_p = xl.czt_propagate_backward(Gd, g, win, LAM, zs)
    xl.device_status()
    tol_z = 1e-3 if dtype == np.complex64 else 1e-8
    for b in range(3):
        ref = _dz_ref(U[b], G[b], g, win, zs[b])
        assert abs(float(gz_s[b]) - ref) <= tol_z * abs(ref), (b, float(gz_s[b]), ref)
        assert abs(float(gz_r[b]) - ref) <= tol_z * abs(ref), (b, float(gz_r[b]), ref)
    # the distance-gradient form of the adjoint gives the same field gradient
    assert rel(to_np(gi_s), to_np(gi_p)) < _tol(dtype)
    assert rel(to_np(gi_r), to_np(gi_p)) < _tol(dtype)
    # g_z alone (no field gradient requested)
    _, gz_only = xl.czt_propagate_backward(Gd, g, win, LAM, zs, u_in=Ud, want_dz=True,
                                           want_field=False, saved=S)
    assert torch.allclose(gz_only, gz_s, rtol=1e-6 if dtype == np.complex64 else 1e-12, atol=0)


def test_czt_distance_gradient_phase_invariant_and_device_z():
    """XL_PHASE_INVARIANT leaves out Re(ik <G, u_out>); device distances give the host results."""
    import torch
    xl = lib()
    g, win, u = _case(300, 256, 40, 64, 5400)
    zs = [800.0, 3000.0]
    U = np.stack([u, np.roll(u, 3, axis=1)]).astype(np.complex128)
    G = inputs.random_unit(5401, (2, 64, 40)).astype(np.complex128)
    Ud, Gd = to_dev(U, np.complex128), to_dev(G, np.complex128)
    _, gz = xl.czt_propagate_backward(Gd, g, win, LAM, zs, u_in=Ud, want_dz=True,
                                      phase_invariant=True)
    k = 2 * np.pi / LAM
    for b in range(2):
        out = oracle.czt_conv(U[b], g.astuple(), win.astuple(), LAM, zs[b])
        rot = float(np.real(1j * k * np.vdot(G[b], out)))  # the term the flag leaves out
        ref = _dz_ref(U[b], G[b], g, win, zs[b]) - rot
        # the reference is a difference of two sums each about 1e4 times larger than it: its own
        # double-precision rounding is relative to those sums
        assert abs(float(gz[b]) - ref) <= 1e-8 * (abs(ref) + abs(rot)), (b, float(gz[b]), ref, rot)
    zd = torch.tensor(zs, dtype=torch.float64, device="cuda")
    _, gz_h = xl.czt_propagate_backward(Gd, g, win, LAM, zs, u_in=Ud, want_dz=True)
    _, gz_d = xl.czt_propagate_backward(Gd, g, win, LAM, zd, u_in=Ud, want_dz=True)
    assert torch.allclose(gz_h, gz_d, rtol=1e-12, atol=0)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_vczt_distance_gradient(dtype):
    xl = lib()
    g, win, _ = _case(512, 300, 64, 48, 5500)
    exy = np.stack([inputs.radial_gaussian(g, 60.0), inputs.random_jones(g, 60.0, 5501)]).astype(dtype)
    z = 1200.0
    Ed = to_dev(exy, dtype)
    G = inputs.random_unit(5502, (2, 3, win.my, win.mx)).astype(dtype)
    Gd = to_dev(G, dtype)
    S = xl.czt_save_buffer(Ed, g, win, vectorial=1)
    xl.czt_propagate(Ed, g, win, LAM, [z, z], vectorial=1, saved=S)
    gi, gz = xl.czt_propagate_backward(Gd, g, win, LAM, [z, z], vectorial=1, u_in=Ed,
                                       want_dz=True, saved=S)
    _, gz_r = xl.czt_propagate_backward(Gd, g, win, LAM, [z, z], vectorial=1, u_in=Ed, want_dz=True)
    gi_p = xl.czt_propagate_backward(Gd, g, win, LAM, [z, z], vectorial=1)
    assert rel(to_np(gi), to_np(gi_p)) < _tol(dtype)
    tol_z = 1e-3 if dtype == np.complex64 else 1e-8
    for b in range(2):
        d = oracle.vczt_dz(exy[b].astype(np.complex128), g.astuple(), win.astuple(), LAM, z)
        ref = float(np.real(np.vdot(G[b].astype(np.complex128), d)))
        assert abs(float(gz[b]) - ref) <= tol_z * abs(ref), (b, float(gz[b]), ref)
        assert abs(float(gz_r[b]) - ref) <= tol_z * abs(ref)


def test_czt_autograd_distance_gradient():
    import torch
    xl = lib()
    from paper_2310_08408_gb300 import autograd
    g, win, u = _case(300, 256, 40, 64, 5600)
    U = to_dev(np.stack([u, np.roll(u, 9, axis=0)]).astype(np.complex64), np.complex64)
    z = torch.tensor([900.0, 2000.0], dtype=torch.float64, device="cuda", requires_grad=True)
    Ur = U.clone().requires_grad_(True)
    out = autograd.CZTPropagate.apply(Ur, z, g, win, LAM, 0)
    W = to_dev(inputs.random_unit(5601, (2, 64, 40)).astype(np.complex64), np.complex64)
    (out * W.conj()).real.sum().backward()
    gi, gz = xl.czt_propagate_backward(W, g, win, LAM, z.detach(), u_in=U, want_dz=True)
    assert torch.equal(Ur.grad, gi)
    assert torch.allclose(z.grad, gz, rtol=1e-5, atol=0)


def test_czt_distance_gradient_2048_to_512_three_distances():
    """The benchmark's CZT (2048^2 -> 512^2 over 64 um, one batched call over z = 0.5, 2 and
    10 mm) with saved sums: forward and adjoint full-window parity and g_z."""
    xl = lib()
    w = inputs.WORKLOADS["rs2048"]
    g = inputs.Grid.centred(w["n"], w["pitch"])
    win = inputs.Window.centred(w["window_m"], w["window_w"])
    zs = list(w["zs"])
    u = np.stack([inputs.gaussian_random_phase(g, w["w0"], w["seed"] + b) for b in range(3)]
                 ).astype(np.complex64)
    G = inputs.random_unit(8, (3, win.my, win.mx)).astype(np.complex64)
    Ud = to_dev(u, np.complex64)
    S = xl.czt_save_buffer(Ud, g, win)
    out = to_np(xl.czt_propagate(Ud, g, win, w["wavelength"], zs, saved=S))
    gi, gz = xl.czt_propagate_backward(to_dev(G, np.complex64), g, win, w["wavelength"], zs, u_in=Ud,
                                       want_dz=True, saved=S)
    gi, gz = to_np(gi), to_np(gz)
    xl.device_status()
    for b in range(3):
        u0 = u[b].astype(np.complex128)
        assert rel(out[b], oracle.czt_conv(u0, g.astuple(), win.astuple(), w["wavelength"], zs[b])) < TOL_C64
        ref = oracle.czt_conv(G[b].astype(np.complex128), g.astuple(), win.astuple(), w["wavelength"],
                              zs[b], adjoint=True)
        assert rel(gi[b], ref) < TOL_C64
        d = oracle.czt_conv(u0, g.astuple(), win.astuple(), w["wavelength"], zs[b], 3)
        ref = float(np.real(np.vdot(G[b].astype(np.complex128), d)))
        assert abs(gz[b] - ref) <= 1e-3 * abs(ref), (b, gz[b], ref)
