"""Parity at the full workload sizes, in the launch configuration the benchmark uses, on outputs
the FP64 oracle can compute one by one:
- vectorial RS at 2048^2 (radially polarised Gaussian, then a random Jones field; z = 5 mm): the
  three output components and the adjoint's two at sampled pixels (direct sums), and the distance
  gradient for a cotangent that is non-zero only at those pixels (so the oracle's direct sums of
  the distance-derivative kernels give it exactly);
- vectorial CZT 2048^2 -> 512^2 over 64 um at z = 5 mm, sampled window pixels;
- the 256-setup batched optimiser of mixed grids 512^2 / 1024^2 / 2048^2 (one step of the whole
  batch), with the loss and every gradient of sampled setups checked against the oracle's table.
"""
import numpy as np
import pytest

import oracle
import oracle.table as otable
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C64, TOL_LOSS, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def _vrs_inputs():
    w = inputs.WORKLOADS["vrs2048"]
    g = inputs.Grid.centred(w["n"], w["pitch"])
    exy = np.stack([inputs.radial_gaussian(g, w["w0"]),
                    inputs.random_jones(g, w["w0"], w["seed"])]).astype(np.complex64)
    return w, g, exy


def _points(n, seed, k=20):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.integers(0, n, (k, 2)), [[0, 0], [n - 1, n - 1], [n // 2, n // 2]]])


def test_vrs_2048_forward_adjoint_dz_sampled():
    import torch
    xl = lib()
    w, g, exy = _vrs_inputs()
    lam, z = w["wavelength"], w["z"]
    E = to_dev(exy, np.complex64)
    S = xl.save_buffer(E, 2)
    out = to_np(xl.vrs_propagate(E, g, lam, [z, z], saved=S))
    pts = _points(g.nx, 21)
    for b in range(2):
        ex, ey = (exy[b, c].astype(np.complex128) for c in range(2))
        rp = lambda u, kind, adj=False: oracle.rs_points(u, g.dx, g.dy, lam, z, pts, kind, adj)
        ref = [rp(ex, oracle.K_H), rp(ey, oracle.K_H), rp(ex, oracle.K_HX) + rp(ey, oracle.K_HY)]
        for c in range(3):
            got = np.array([out[b, c][q, p] for p, q in pts])
            assert rel(got, ref[c]) < TOL_C64, (b, c)
    # adjoint field and distance gradient for a cotangent supported on the sampled pixels
    Gh = np.zeros((2, 3, g.ny, g.nx), np.complex64)
    vals = inputs.random_unit(22, (2, 3, len(pts))).astype(np.complex64)
    for i, (p, q) in enumerate(pts):
        Gh[:, :, q, p] += vals[:, :, i]
    G = to_dev(Gh, np.complex64)
    gi, gz = xl.vrs_propagate_backward(G, None, g, lam, [z, z], want_field=True, want_dz=True,
                                       saved=S)
    gi, gz = to_np(gi), to_np(gz)
    for b in range(2):
        ex, ey = (exy[b, c].astype(np.complex128) for c in range(2))
        Gb = Gh[b].astype(np.complex128)
        # adjoint at sampled pixels: g_ex = P_h^H gx + P_hx^H gz, g_ey = P_h^H gy + P_hy^H gz
        adj = lambda u, kind: oracle.rs_points(u, g.dx, g.dy, lam, z, pts, kind, True)
        ref_x = adj(Gb[0], oracle.K_H) + adj(Gb[2], oracle.K_HX)
        ref_y = adj(Gb[1], oracle.K_H) + adj(Gb[2], oracle.K_HY)
        assert rel(np.array([gi[b, 0][q, p] for p, q in pts]), ref_x) < TOL_C64
        assert rel(np.array([gi[b, 1][q, p] for p, q in pts]), ref_y) < TOL_C64
        # dz = Re sum conj(G) d out/dz over the support of G
        rp = lambda u, kind: oracle.rs_points(u, g.dx, g.dy, lam, z, pts, kind)
        # merge repeated pixels: G holds their sum once
        uniq, idx = np.unique(pts, axis=0, return_index=True)
        d = [rp(ex, oracle.K_DH), rp(ey, oracle.K_DH), rp(ex, oracle.K_DHX) + rp(ey, oracle.K_DHY)]
        dz = sum(float(np.real(np.vdot(Gb[c][pts[idx, 1], pts[idx, 0]], d[c][idx]))) for c in range(3))
        assert abs(gz[b] - dz) < 1e-3 * abs(dz)


def test_vczt_2048_to_512_sampled():
    xl = lib()
    w, g, exy = _vrs_inputs()
    win = inputs.Window.centred(w["window_m"], w["window_w"])
    lam, z = w["wavelength"], w["z"]
    out = to_np(xl.czt_propagate(to_dev(exy, np.complex64), g, win, lam, [z, z], vectorial=1))
    pts = _points(win.mx, 31)
    for b in range(2):
        ex, ey = (exy[b, c].astype(np.complex128) for c in range(2))
        cp = lambda u, kind: oracle.czt_points(u, g.astuple(), win.astuple(), lam, z, pts, kind)
        ref = [cp(ex, 0), cp(ey, 0), cp(ex, 1) + cp(ey, 2)]
        for c in range(3):
            assert rel(np.array([out[b, c][q, p] for p, q in pts]), ref[c]) < TOL_C64, (b, c)


def test_batch_256_mixed_grids_sampled_setups():
    """The benchmark's optimiser batch (256 setups, grids drawn from 512^2 / 1024^2 / 2048^2,
    one CUDA-graph step of all of them); sampled setups against the oracle's table."""
    xl = lib()
    cfg = dict(wavelength=0.6328, extent=1024.0, w0=200.0, f=5000.0, cam_m=256, cam_width=64.0,
               lr=0.01, lr_z=1.0)
    seed = inputs.SEED0 + 5
    grid_n = [512 * (2 ** int(3 * x)) for x in inputs.uniform(seed, 256)]
    init = [[0.3, 20_000.0, 20_000.0] for _ in grid_n]
    b = xl.Batch(cfg, grid_n, init, seed)
    picks = [i for i, n in enumerate(grid_n) if n == 512][:2] + [grid_n.index(1024)]
    phis = {s: (b.read(xl.BATCH_PHI1, s).astype(np.float64), b.read(xl.BATCH_PHI2, s).astype(np.float64))
            for s in picks}
    b.step(use_graph=True)
    for s in picks:
        n = grid_n[s]
        g = inputs.Grid.centred(n, cfg["extent"] / n)
        win = inputs.Window.centred(cfg["cam_m"], cfg["cam_width"])
        t = otable.Table(g.astuple(), win.astuple(), cfg["wavelength"], cfg["f"])
        src = inputs.x_polarised_gaussian(g, cfg["w0"]).astype(np.complex64).astype(np.complex128)
        th, z1, z2 = init[s]
        L, planes = otable.forward(t, src, *phis[s], th, z1, z2)
        gr = otable.backward(t, src, *phis[s], th, z1, z2, planes)
        assert abs(b.read(xl.BATCH_LOSS, s)[0] - L) / L < TOL_LOSS, s
        assert rel(b.read(xl.BATCH_GRAD_PHI1, s), gr["phi1"]) < 1e-3, s
        assert rel(b.read(xl.BATCH_GRAD_PHI2, s), gr["phi2"]) < 1e-3, s
        gs = b.read(xl.BATCH_GRAD_SCALARS, s)
        errs = [abs(a - r) / abs(r) for a, r in zip(gs, (gr["theta"], gr["z1"], gr["z2"]))]
        assert max(errs) < 1e-3, (s, errs)
    b.close()


def test_maximum_transform_length_4096_grid_sampled():
    """The largest transform length the kernels build (8192): RS forward and adjoint of a 4096^2
    complex64 field (padded to 8192^2, both through the row-major intermediate) and CZT 4096^2 ->
    1024^2 (Bluestein length 8192, row-major forward pair), at sampled pixels against the
    oracle's direct sums."""
    xl = lib()
    g = inputs.Grid.centred(4096, 0.5)
    lam, z = 0.6328, 3000.0
    u = inputs.gaussian_random_phase(g, 400.0, 4242).astype(np.complex64)[None]
    U = to_dev(u, np.complex64)
    pts = _points(4096, 43, k=12)
    u0 = u[0].astype(np.complex128)
    out = to_np(xl.rs_propagate(U, g, lam, [z]))[0]
    ref = oracle.rs_points(u0, g.dx, g.dy, lam, z, pts)
    assert rel(np.array([out[q, p] for p, q in pts]), ref) < TOL_C64
    gi = to_np(xl.rs_propagate_backward(U, None, g, lam, [z], want_field=True)[0])[0]
    ref = oracle.rs_points(u0, g.dx, g.dy, lam, z, pts, oracle.K_H, True)
    assert rel(np.array([gi[q, p] for p, q in pts]), ref) < TOL_C64
    w = inputs.Window(1024, 1024, 0.25, 0.25, -128.0 + 0.3, -128.0 - 0.2)
    c = to_np(xl.czt_propagate(U, g, w, lam, [z]))[0]
    wp = _points(1024, 44, k=12)
    ref = oracle.czt_points(u0, g.astuple(), w.astuple(), lam, z, wp)
    assert rel(np.array([c[q, p] for p, q in wp]), ref) < TOL_C64
    lib().device_status()
