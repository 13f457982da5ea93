"""GPU parity of CZT / VCZT propagation and adjoints against the FP64 oracle.

Reading (Methods, "Features and performance"; Bluestein method of the cited Hu et al.): CZT is
the Fresnel form of the RS integral evaluated on an explicit output window; VCZT applies the VRS
kernel ratio -(offset / z) for Ez. The oracle evaluates the sums directly (separable), the GPU by
Bluestein chirp convolutions, so agreement checks the factorisation as well as the kernels.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C128, TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu
LAM = 0.633


CASES = [
    # nx, ny, pitch, mx, my, window width x, window width y, z
    (64, 64, 0.5, 48, 40, 12.0, 10.0, 200.0),
    (37, 53, 0.7, 29, 61, 20.0, 25.0, 150.0),      # ragged, non powers of two
    (256, 256, 0.5, 64, 64, 16.0, 16.0, 500.0),
    (100, 80, 1.0, 300, 200, 200.0, 150.0, 1000.0),  # window larger than the input
]


def _case(nx, ny, pitch, mx, my, wx, wy):
    g = inputs.Grid(nx, ny, pitch, pitch, -(nx // 2) * pitch, -(ny // 2) * pitch + 0.3)
    w = inputs.Window(mx, my, wx / mx, wy / my, -wx / 2 + 1.1, -wy / 2 - 0.7)
    return g, w


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("dtype,tol", [(np.complex64, TOL_C64), (np.complex128, TOL_C128)])
def test_czt_forward_and_adjoint(case, dtype, tol):
    xl = lib()
    nx, ny, pitch, mx, my, wx, wy, z = case
    g, w = _case(nx, ny, pitch, mx, my, wx, wy)
    u = inputs.gaussian_random_phase(g, 0.3 * nx * pitch, 70 + nx).astype(dtype)
    out = to_np(xl.czt_propagate(to_dev(u, dtype), g, w, LAM, z))
    ref = oracle.czt_conv(u.astype(np.complex128), g.astuple(), w.astuple(), LAM, z)
    assert rel(out, ref) < tol
    G = inputs.random_unit(71 + nx, (my, mx)).astype(dtype)
    gin = to_np(xl.czt_propagate_backward(to_dev(G, dtype), g, w, LAM, z))
    refb = oracle.czt_conv(G.astype(np.complex128), g.astuple(), w.astuple(), LAM, z, adjoint=True)
    assert rel(gin, refb) < tol


@pytest.mark.parametrize("case", CASES[:3])
@pytest.mark.parametrize("dtype,tol", [(np.complex64, TOL_C64), (np.complex128, TOL_C128)])
def test_vczt_forward_and_adjoint(case, dtype, tol):
    xl = lib()
    nx, ny, pitch, mx, my, wx, wy, z = case
    g, w = _case(nx, ny, pitch, mx, my, wx, wy)
    exy = inputs.random_jones(g, 0.3 * nx * pitch, 80 + nx).astype(dtype)
    out = to_np(xl.czt_propagate(to_dev(exy, dtype), g, w, LAM, z, vectorial=True))
    ref = oracle.vczt(exy.astype(np.complex128), g.astuple(), w.astuple(), LAM, z)
    assert rel(out, ref) < tol
    G = inputs.random_unit(81 + nx, (3, my, mx)).astype(dtype)
    gin = to_np(xl.czt_propagate_backward(to_dev(G, dtype), g, w, LAM, z, vectorial=True))
    refb = oracle.vczt_adjoint(G.astype(np.complex128), g.astuple(), w.astuple(), LAM, z)
    assert rel(gin, refb) < tol


def test_czt_batch_device_z_and_full_size_points():
    """2048^2 -> 512^2 over 64 um (the benchmark workload) at the three distances, batch 3 with
    device-resident z; sampled window pixels against the oracle's direct sum."""
    import torch
    xl = lib()
    wl = inputs.WORKLOADS["rs2048"]
    g = inputs.Grid.centred(wl["n"], wl["pitch"])
    w = inputs.Window.centred(wl["window_m"], wl["window_w"])
    us = np.stack([inputs.gaussian_random_phase(g, wl["w0"], wl["seed"] + i) for i in range(3)]
                  ).astype(np.complex64)
    zs = list(wl["zs"])
    ud = to_dev(us, np.complex64)
    out_h = to_np(xl.czt_propagate(ud, g, w, wl["wavelength"], zs))
    out_d = to_np(xl.czt_propagate(ud, g, w, wl["wavelength"],
                                   torch.tensor(zs, dtype=torch.float64, device="cuda")))
    assert rel(out_d, out_h) < 1e-6
    rng = np.random.default_rng(11)
    pts = np.concatenate([rng.integers(0, 512, (24, 2)), [[0, 0], [511, 511], [256, 256]]])
    for i, z in enumerate(zs):
        ref = oracle.czt_points(us[i].astype(np.complex128), g.astuple(), w.astuple(),
                                wl["wavelength"], z, pts)
        got = np.array([out_h[i][q, p] for p, q in pts])
        assert rel(got, ref) < TOL_C64


def test_czt_argument_errors():
    import torch
    xl = lib()
    u = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(xl.XLError) as e:
        xl.czt_propagate(u, (64, 64, 1.0, 1.0, 0.0, 0.0), (8200, 8, 1.0, 1.0, 0.0, 0.0), LAM, 10.0)
    assert e.value.status == xl.ERR_UNSUPPORTED
    with pytest.raises(xl.XLError) as e:
        xl.czt_propagate(u, (64, 64, 1.0, 1.0, 0.0, 0.0), (8, 8, 0.0, 1.0, 0.0, 0.0), LAM, 10.0)
    assert e.value.status == xl.ERR_ARG


@pytest.mark.parametrize("vectorial", [0, 1])
def test_mixed_distance_batch_one_launch(vectorial):
    """A batch whose elements have different distances runs in one launch per pass, each element
    with its own chirp tables: every element matches the oracle and, bit for bit, the same
    element propagated alone."""
    import torch
    xl = lib()
    g, w = _case(64, 48, 0.5, 40, 36, 12.0, 10.0)
    zs = [150.0, 150.0, 300.0, 80.0, 80.0]
    B = len(zs)
    if vectorial:
        u = np.stack([inputs.random_jones(g, 10.0, 90 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(96, (B, 3, w.my, w.mx)).astype(np.complex64)
    else:
        u = np.stack([inputs.gaussian_random_phase(g, 10.0, 90 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(96, (B, w.my, w.mx)).astype(np.complex64)
    U, Gd = to_dev(u, np.complex64), to_dev(G, np.complex64)
    out = xl.czt_propagate(U, g, w, LAM, zs, vectorial=vectorial)
    gin = xl.czt_propagate_backward(Gd, g, w, LAM, zs, vectorial=vectorial)
    for i, z in enumerate(zs):
        one = xl.czt_propagate(U[i:i + 1], g, w, LAM, [z], vectorial=vectorial)
        assert torch.equal(one[0], out[i]), i
        oneb = xl.czt_propagate_backward(Gd[i:i + 1], g, w, LAM, [z], vectorial=vectorial)
        assert torch.equal(oneb[0], gin[i]), i
        ui, Gi = u[i].astype(np.complex128), G[i].astype(np.complex128)
        if vectorial:
            ref = oracle.vczt(ui, g.astuple(), w.astuple(), LAM, z)
            refb = oracle.vczt_adjoint(Gi, g.astuple(), w.astuple(), LAM, z)
        else:
            ref = oracle.czt_conv(ui, g.astuple(), w.astuple(), LAM, z)
            refb = oracle.czt_conv(Gi, g.astuple(), w.astuple(), LAM, z, adjoint=True)
        assert rel(to_np(out[i]), ref) < TOL_C64, i
        assert rel(to_np(gin[i]), refb) < TOL_C64, i


@pytest.mark.parametrize("case", [
    (200, 150, 0.5, 120, 90, 40.0, 30.0, 400.0),    # one column tile of 150 rows per copy
    (180, 300, 0.5, 96, 100, 30.0, 40.0, 600.0),    # 300 rows: two copies, the second ragged
    (300, 260, 0.7, 702, 40, 400.0, 20.0, 900.0),   # wide window: several column blocks
    (160, 700, 0.5, 64, 400, 30.0, 300.0, 800.0),   # y length 2048: three copies, the last ragged
])
def test_row_major_forward_matches_transposed(case, monkeypatch):
    """The scalar complex64 forward stores the x transforms row-major and gathers the y pass's
    columns with bulk tensor copies; the transposing x pass (XL_CZT_RM=0) gives bit-identical
    windows, and both match the oracle, for a batch of mixed distances."""
    import torch
    xl = lib()
    nx, ny, pitch, mx, my, wx, wy, z = case
    g, w = _case(nx, ny, pitch, mx, my, wx, wy)
    zs = [z, 0.7 * z, z]
    u = np.stack([inputs.gaussian_random_phase(g, 20.0, 300 + i) for i in range(len(zs))]).astype(np.complex64)
    U = to_dev(u, np.complex64)
    rm = xl.czt_propagate(U, g, w, LAM, zs)
    torch.cuda.synchronize()
    monkeypatch.setenv("XL_CZT_RM", "0")
    tr = xl.czt_propagate(U, g, w, LAM, zs)
    torch.cuda.synchronize()
    xl.device_status()
    assert torch.equal(rm, tr)
    for i, zi in enumerate(zs):
        ref = oracle.czt_conv(u[i].astype(np.complex128), g.astuple(), w.astuple(), LAM, zi)
        assert rel(to_np(rm[i]), ref) < TOL_C64, i
