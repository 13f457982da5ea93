"""GPU parity of the angular-spectrum CZT (forward, adjoint and distance gradient) against the FP64
oracle, element by element on the same seeded inputs: square and rectangular grids, windows off
the grid (shifted, finer, coarser, rectangular), runs of equal and different distances,
device-resident distances, a strongly evanescent spectrum, and a 1024^2 -> 256^2 case."""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C128, TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu
LAM = 0.6328


def _grid(nx, ny, d):
    return inputs.Grid(nx, ny, d, d, -(nx // 2) * d, -(ny // 2) * d)


def _src(g, seed):
    return inputs.gaussian_random_phase(g, 0.25 * g.nx * g.dx, seed)


CASES = [
    # nx, ny, pitch, window (mx, my, dxo, dyo, xo0, yo0), distances
    (64, 64, 0.5, (40, 36, 0.3, 0.25, -6.0, -4.5), [30.0, 30.0, 80.0]),
    (128, 64, 0.4, (128, 64, 0.4, 0.4, -25.6, -12.8), [15.0]),          # native grid
    (64, 128, 0.6, (100, 30, 0.45, 1.1, -20.0, -16.0), [50.0, 120.0]),
    (64, 64, 0.2, (48, 48, 0.15, 0.15, -3.6, -3.6), [1.5]),             # mostly evanescent spectrum
]


@pytest.mark.parametrize("dtype,tol", [(np.complex64, TOL_C64), (np.complex128, TOL_C128)])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_forward_adjoint_dz(dtype, tol, case):
    import torch
    xl = lib()
    nx, ny, d, w, zs = CASES[case]
    g = _grid(nx, ny, d)
    B = len(zs)
    u = np.stack([_src(g, 5400 + 10 * case + b) for b in range(B)]).astype(dtype)
    G = inputs.random_unit(5500 + case, (B, w[1], w[0])).astype(dtype)
    U, Gd = to_dev(u, dtype), to_dev(G, dtype)
    out = to_np(xl.asczt_propagate(U, g, w, LAM, zs))
    gi, gz = xl.asczt_propagate_backward(Gd, U, g, w, LAM, zs, want_field=True, want_dz=True)
    gi, gz = to_np(gi), to_np(gz)
    ga = g.astuple()
    for b in range(B):
        ub = u[b].astype(np.complex128)
        Gb = G[b].astype(np.complex128)
        assert rel(out[b], oracle.asczt(ub, ga, w, LAM, zs[b])) < tol
        assert rel(gi[b], oracle.asczt(Gb, ga, w, LAM, zs[b], adjoint=True)) < tol
        dz = float(np.real(np.vdot(Gb, oracle.asczt(ub, ga, w, LAM, zs[b], oracle.AS_DH))))
        assert abs(gz[b] - dz) < (1e-3 if dtype == np.complex64 else 1e-9) * max(abs(dz), 1e-30)


def test_device_distances_match_host():
    import torch
    xl = lib()
    g = _grid(64, 64, 0.5)
    w = (32, 32, 0.5, 0.5, -8.0, -8.0)
    zs = [20.0, 45.0]
    u = np.stack([_src(g, 5600 + b) for b in range(2)]).astype(np.complex64)
    U = to_dev(u, np.complex64)
    zd = torch.tensor(zs, dtype=torch.float64, device="cuda")
    a = xl.asczt_propagate(U, g, w, LAM, zs)
    b = xl.asczt_propagate(U, g, w, LAM, zd)
    assert torch.equal(a, b)
    G = to_dev(inputs.random_unit(5610, (2, 32, 32)).astype(np.complex64), np.complex64)
    g1, z1 = xl.asczt_propagate_backward(G, U, g, w, LAM, zs, want_dz=True)
    g2, z2 = xl.asczt_propagate_backward(G, U, g, w, LAM, zd, want_dz=True)
    assert torch.equal(g1, g2) and torch.equal(z1, z2)


def test_1024_to_256_window():
    xl = lib()
    g = _grid(1024, 1024, 1.0)
    w = (256, 256, 0.25, 0.25, -32.0, -32.0)
    u = _src(g, 5700).astype(np.complex64)
    out = to_np(xl.asczt_propagate(to_dev(u[None], np.complex64), g, w, LAM, [5000.0]))[0]
    ref = oracle.asczt(u.astype(np.complex128), g.astuple(), w, LAM, 5000.0)
    assert rel(out, ref) < TOL_C64


def test_argument_errors():
    import torch
    xl = lib()
    U = torch.zeros((1, 32, 32), dtype=torch.complex64, device="cuda")
    with pytest.raises(xl.XLError):
        xl.asczt_propagate(U, _grid(32, 32, 1.0), (8, 8, 1.0, 1.0, 0.0, 0.0), LAM, [10.0])
    U = torch.zeros((1, 64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(xl.XLError):
        xl.asczt_propagate(U, _grid(64, 64, 1.0), (8, 8, 1.0, 1.0, 0.0, 0.0), LAM, [-1.0])


def test_mixed_distance_batch_matches_single_element_calls():
    """A batch of different distances runs in one launch per pass, each element reading the
    transfer tables of its own distance: bit-identical to propagating each element alone, forward
    and adjoint with the distance gradient."""
    import torch
    xl = lib()
    g = _grid(64, 64, 0.5)
    w = (40, 36, 0.3, 0.25, -6.0, -4.5)
    zs = [30.0, 80.0, 80.0, 15.0]
    B = len(zs)
    u = np.stack([_src(g, 5800 + b) for b in range(B)]).astype(np.complex64)
    G = inputs.random_unit(5810, (B, w[1], w[0])).astype(np.complex64)
    U, Gd = to_dev(u, np.complex64), to_dev(G, np.complex64)
    out = xl.asczt_propagate(U, g, w, LAM, zs)
    gi, gz = xl.asczt_propagate_backward(Gd, U, g, w, LAM, zs, want_field=True, want_dz=True)
    for i, z in enumerate(zs):
        o1 = xl.asczt_propagate(U[i:i + 1], g, w, LAM, [z])
        g1, z1 = xl.asczt_propagate_backward(Gd[i:i + 1], U[i:i + 1], g, w, LAM, [z], want_field=True,
                                             want_dz=True)
        assert torch.equal(o1[0], out[i]) and torch.equal(g1[0], gi[i]) and torch.equal(z1[0], gz[i]), i
        assert rel(to_np(out[i]), oracle.asczt(u[i].astype(np.complex128), g.astuple(), w, LAM, z)) < TOL_C64
