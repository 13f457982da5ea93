"""GPU parity of scalar and vectorial RS propagation (and adjoints) against the FP64 oracle.

Reading (Methods, "Features and performance"): RS is the rectangle-rule first RS integral on the
input grid, realised by a zero-padded 2D FFT convolution; VRS adds Ez' = h_x * Ex + h_y * Ey.
Inputs are the seeded synthetic sources of paper_2310_08408_gb300.inputs; the oracle receives the
complex64 (complex128) rounding of the same values in float64.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C128, TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu
LAM = 0.6328


def _src(n, pitch, w0, seed, nyx=None):
    ny, nx = nyx or (n, n)
    g = inputs.Grid(nx, ny, pitch, pitch, -(nx // 2) * pitch, -(ny // 2) * pitch)
    return g, inputs.gaussian_random_phase(g, w0, seed)


@pytest.mark.parametrize("nx,ny,pitch,z", [(32, 32, 1.0, 50.0), (64, 64, 0.5, 200.0),
                                           (64, 128, 0.75, 120.0), (256, 256, 1.0, 10_000.0),
                                           (512, 256, 1.0, 3000.0)])
def test_rs_forward_c64(nx, ny, pitch, z):
    xl = lib()
    g, u = _src(nx, pitch, 0.3 * nx * pitch, 100 + nx + ny, (ny, nx))
    u64 = u.astype(np.complex64)
    out = to_np(xl.rs_propagate(to_dev(u64, np.complex64), g, LAM, z))
    ref = oracle.rs_conv(u64.astype(np.complex128), g.dx, g.dy, LAM, z)
    assert rel(out, ref) < TOL_C64


def test_rs_forward_c128_256():
    xl = lib()
    g, u = _src(256, 1.0, 40.0, inputs.SEED0 + 1)
    out = to_np(xl.rs_propagate(to_dev(u, np.complex128), g, LAM, 10_000.0))
    ref = oracle.rs_conv(u, 1.0, 1.0, LAM, 10_000.0)
    assert rel(out, ref) < TOL_C128


def test_rs_batch_mixed_distances_and_chunks():
    xl = lib()
    g = inputs.Grid.centred(128, 0.5)
    zs = [300.0, 300.0, 300.0, 80.0, 300.0]
    us = np.stack([inputs.gaussian_random_phase(g, 20.0, 7 + i) for i in range(5)]).astype(np.complex64)
    out = to_np(xl.rs_propagate(to_dev(us, np.complex64), g, LAM, zs))
    for i, z in enumerate(zs):
        ref = oracle.rs_conv(us[i].astype(np.complex128), 0.5, 0.5, LAM, z)
        assert rel(out[i], ref) < TOL_C64


def test_rs_device_z_matches_host_z():
    import torch
    xl = lib()
    g, u = _src(128, 0.5, 20.0, 31)
    ud = to_dev(np.stack([u, u]), np.complex64)
    zs = [150.0, 900.0]
    a = to_np(xl.rs_propagate(ud, g, LAM, zs))
    b = to_np(xl.rs_propagate(ud, g, LAM, torch.tensor(zs, dtype=torch.float64, device="cuda")))
    assert rel(b, a) < 1e-6


@pytest.mark.parametrize("dtype,tol", [(np.complex64, TOL_C64), (np.complex128, TOL_C128)])
def test_rs_backward_field_and_dz(dtype, tol):
    xl = lib()
    g, u = _src(64, 0.5, 10.0, 41)
    G = inputs.random_unit(42, (2, 64, 64))
    u2 = np.stack([u, np.conj(u)]).astype(dtype)
    G = G.astype(dtype)
    zs = [40.0, 95.0]
    g_in, g_z = xl.rs_propagate_backward(to_dev(G, dtype), to_dev(u2, dtype), g, LAM, zs,
                                         want_field=True, want_dz=True)
    g_in, g_z = to_np(g_in), to_np(g_z)
    for i, z in enumerate(zs):
        Gi = G[i].astype(np.complex128)
        ui = u2[i].astype(np.complex128)
        ref = oracle.rs_conv(Gi, 0.5, 0.5, LAM, z, oracle.K_H, adjoint=True)
        assert rel(g_in[i], ref) < tol
        dz = np.real(np.vdot(Gi, oracle.rs_conv(ui, 0.5, 0.5, LAM, z, oracle.K_DH)))
        assert abs(g_z[i] - dz) / abs(dz) < (1e-4 if dtype == np.complex64 else 1e-10)


@pytest.mark.parametrize("dtype,tol", [(np.complex64, TOL_C64), (np.complex128, TOL_C128)])
def test_vrs_forward_and_backward(dtype, tol):
    xl = lib()
    g = inputs.Grid.centred(64, 0.5)
    exy = inputs.random_jones(g, 12.0, 51).astype(dtype)
    z = 60.0
    out = to_np(xl.vrs_propagate(to_dev(exy, dtype), g, LAM, z))
    ref = oracle.vrs(exy.astype(np.complex128), 0.5, 0.5, LAM, z)
    assert rel(out, ref) < tol
    G = inputs.random_unit(52, (3, 64, 64)).astype(dtype)
    g_exy, g_z = xl.vrs_propagate_backward(to_dev(G, dtype), to_dev(exy, dtype), g, LAM, z,
                                           want_field=True, want_dz=True)
    refb = oracle.vrs_adjoint(G.astype(np.complex128), 0.5, 0.5, LAM, z)
    assert rel(to_np(g_exy), refb) < tol
    dz = np.real(np.vdot(G.astype(np.complex128), oracle.vrs_dz(exy.astype(np.complex128), 0.5, 0.5, LAM, z)))
    assert abs(to_np(g_z)[0] - dz) / abs(dz) < (1e-4 if dtype == np.complex64 else 1e-10)


def test_rs_full_size_2048_sampled_points():
    """2048^2 complex64 at the benchmark's distances, batch of 2, checked at sampled output pixels
    (including the ragged edges) against the oracle's direct sum."""
    xl = lib()
    w = inputs.WORKLOADS["rs2048"]
    g = inputs.Grid.centred(w["n"], w["pitch"])
    us = np.stack([inputs.gaussian_random_phase(g, w["w0"], w["seed"] + i) for i in range(2)]
                  ).astype(np.complex64)
    zs = [w["zs"][0], w["zs"][2]]
    out = to_np(xl.rs_propagate(to_dev(us, np.complex64), g, w["wavelength"], zs))
    rng = np.random.default_rng(5)
    pts = np.concatenate([rng.integers(0, 2048, (40, 2)),
                          [[0, 0], [2047, 2047], [0, 2047], [2047, 0], [1024, 1024]]])
    for i, z in enumerate(zs):
        ref = oracle.rs_points(us[i].astype(np.complex128), g.dx, g.dy, w["wavelength"], z, pts)
        got = np.array([out[i][q, p] for p, q in pts])
        assert rel(got, ref) < TOL_C64


def test_rs_argument_errors():
    import torch
    xl = lib()
    u = torch.zeros((48, 48), dtype=torch.complex64, device="cuda")
    with pytest.raises(xl.XLError) as e:
        xl.rs_propagate(u, (48, 48, 1.0, 1.0, 0.0, 0.0), LAM, 10.0)
    assert e.value.status == xl.ERR_UNSUPPORTED
    u = torch.zeros((64, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(xl.XLError) as e:
        xl.rs_propagate(u, (64, 64, 1.0, 1.0, 0.0, 0.0), LAM, -1.0)
    assert e.value.status == xl.ERR_ARG
    with pytest.raises(xl.XLError):
        xl.rs_propagate(u, (64, 64, 1.0, 1.0, 0.0, 0.0), LAM, 5.0, out=u)
    # empty batch is a no-op
    e0 = torch.zeros((0, 64, 64), dtype=torch.complex64, device="cuda")
    assert xl.rs_propagate(e0, (64, 64, 1.0, 1.0, 0.0, 0.0), LAM, []).shape == (0, 64, 64)


@pytest.mark.parametrize("vectorial", [False, True])
def test_phase_invariant_distance_gradient(vectorial):
    """XL_PHASE_INVARIANT drops Re(ik <g, u_out>) from dL/dz: on a random cotangent the two
    results differ by exactly that term (oracle), in complex128."""
    xl = lib()
    g = inputs.Grid.centred(64, 0.5)
    z = 45.0
    k = 2 * np.pi / LAM
    if vectorial:
        u = inputs.random_jones(g, 10.0, 61)
        G = inputs.random_unit(62, (3, 64, 64))
        out = oracle.vrs(u, 0.5, 0.5, LAM, z)
        fb = xl.vrs_propagate_backward
    else:
        u = inputs.gaussian_random_phase(g, 10.0, 61)
        G = inputs.random_unit(62, (64, 64))
        out = oracle.rs_conv(u, 0.5, 0.5, LAM, z)
        fb = xl.rs_propagate_backward
    ud, Gd = to_dev(u[None], np.complex128), to_dev(G[None], np.complex128)
    _, gz = fb(Gd, ud, g, LAM, z, want_field=False, want_dz=True)
    _, gzp = fb(Gd, ud, g, LAM, z, want_field=False, want_dz=True, phase_invariant=True)
    term = np.real(1j * k * np.vdot(G, out))
    assert abs((to_np(gz)[0] - to_np(gzp)[0]) - term) / abs(term) < 1e-9


@pytest.mark.parametrize("vectorial", [False, True])
def test_row_pass_chunks_do_not_change_results(vectorial, monkeypatch):
    """The row passes run over chunks of the batch whatever the distances (pass 2 once per run of
    equal distances): a one-element chunk budget and the default give bit-identical fields and
    distance gradients, forward, adjoint and adjoint from saved spectra."""
    import torch
    xl = lib()
    g = inputs.Grid.centred(64, 0.5)
    zs = [60.0, 60.0, 25.0, 90.0, 90.0]
    B = len(zs)
    if vectorial:
        u = np.stack([inputs.random_jones(g, 12.0, 500 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(510, (B, 3, 64, 64)).astype(np.complex64)
        fwd, bwd = xl.vrs_propagate, xl.vrs_propagate_backward
    else:
        u = np.stack([inputs.gaussian_random_phase(g, 12.0, 500 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(510, (B, 64, 64)).astype(np.complex64)
        fwd, bwd = xl.rs_propagate, xl.rs_propagate_backward
    U, Gd = to_dev(u, np.complex64), to_dev(G, np.complex64)

    def run():
        S = xl.save_buffer(U, 2 if vectorial else 1)
        out = fwd(U, g, LAM, zs, saved=S)
        gi, gz = bwd(Gd, U, g, LAM, zs, want_field=True, want_dz=True)
        gs, gzs = bwd(Gd, None, g, LAM, zs, want_field=True, want_dz=True, saved=S)
        torch.cuda.synchronize()
        return out, gi, gz, gs, gzs

    monkeypatch.setenv("XL_RS_CHUNK_MB", "1")
    small = run()
    monkeypatch.delenv("XL_RS_CHUNK_MB")
    big = run()
    for a, b in zip(small, big):
        assert torch.equal(a, b)
    out = to_np(big[0])
    for i, z in enumerate(zs):
        ui = u[i].astype(np.complex128)
        ref = oracle.vrs(ui, 0.5, 0.5, LAM, z) if vectorial else oracle.rs_conv(ui, 0.5, 0.5, LAM, z)
        assert rel(out[i], ref) < TOL_C64, i


@pytest.mark.parametrize("vectorial", [False, True])
def test_device_distances_chunked_match_host(vectorial, monkeypatch):
    """Device-resident distances run the batch in chunks whose spectra one launch pair generates
    (element e reading z[e]): forward, adjoint with distance gradient, saved and phase-invariant
    variants agree with host distances (spectra from the cache) for a one-element chunk budget and
    the default, and with the oracle."""
    import torch
    xl = lib()
    g = inputs.Grid.centred(64, 0.5)
    zs = [60.0, 25.0, 25.0, 90.0, 40.0]
    B = len(zs)
    zd = torch.tensor(zs, dtype=torch.float64, device="cuda")
    if vectorial:
        u = np.stack([inputs.random_jones(g, 12.0, 700 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(710, (B, 3, 64, 64)).astype(np.complex64)
        fwd, bwd, comps = xl.vrs_propagate, xl.vrs_propagate_backward, 2
    else:
        u = np.stack([inputs.gaussian_random_phase(g, 12.0, 700 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(710, (B, 64, 64)).astype(np.complex64)
        fwd, bwd, comps = xl.rs_propagate, xl.rs_propagate_backward, 1
    U, Gd = to_dev(u, np.complex64), to_dev(G, np.complex64)

    def run(z):
        S = xl.save_buffer(U, comps)
        out = fwd(U, g, LAM, z, saved=S)
        gi, gz = bwd(Gd, None, g, LAM, z, want_field=True, want_dz=True, saved=S)
        gp, gzp = bwd(Gd, U, g, LAM, z, want_field=True, want_dz=True, phase_invariant=True)
        torch.cuda.synchronize()
        return [to_np(x) for x in (out, gi, gz, gp, gzp)]

    host = run(zs)
    dev = run(zd)
    monkeypatch.setenv("XL_RS_CHUNK_MB", "1")
    dev1 = run(zd)
    for h, d, d1 in zip(host, dev, dev1):
        assert np.array_equal(d, d1)
        assert rel(d, h) < 1e-6
    for i, z in enumerate(zs):
        ui = u[i].astype(np.complex128)
        ref = oracle.vrs(ui, 0.5, 0.5, LAM, z) if vectorial else oracle.rs_conv(ui, 0.5, 0.5, LAM, z)
        assert rel(dev[0][i], ref) < TOL_C64, i


@pytest.mark.parametrize("vectorial", [False, True])
def test_pass3_bulk_copy_gather_matches_async_gather(vectorial, monkeypatch):
    """Pass 3 of complex64 grids gathers its rows with tiled bulk tensor copies; the per-thread
    asynchronous-copy gather (XL_P3_TMA=0) gives bit-identical fields, forward and adjoint."""
    import torch
    xl = lib()
    g = inputs.Grid.centred(256, 0.5)
    zs = [80.0, 30.0, 30.0]
    B = len(zs)
    if vectorial:
        u = np.stack([inputs.random_jones(g, 30.0, 800 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(810, (B, 3, 256, 256)).astype(np.complex64)
        fwd, bwd = xl.vrs_propagate, xl.vrs_propagate_backward
    else:
        u = np.stack([inputs.gaussian_random_phase(g, 30.0, 800 + i) for i in range(B)]).astype(np.complex64)
        G = inputs.random_unit(810, (B, 256, 256)).astype(np.complex64)
        fwd, bwd = xl.rs_propagate, xl.rs_propagate_backward
    U, Gd = to_dev(u, np.complex64), to_dev(G, np.complex64)

    def run():
        out = fwd(U, g, LAM, zs)
        gi, gz = bwd(Gd, U, g, LAM, zs, want_field=True, want_dz=True)
        torch.cuda.synchronize()
        return out, gi, gz

    tma = run()
    monkeypatch.setenv("XL_P3_TMA", "0")
    cp = run()
    for a, b in zip(tma, cp):
        assert torch.equal(a, b)
    xl.device_status()  # no bulk-copy wait gave up
    ref = oracle.vrs(u[0].astype(np.complex128), 0.5, 0.5, LAM, zs[0]) if vectorial else \
        oracle.rs_conv(u[0].astype(np.complex128), 0.5, 0.5, LAM, zs[0])
    assert rel(to_np(tma[0])[0], ref) < TOL_C64


def test_row_major_intermediate_matches_transposed(monkeypatch):
    """The scalar forward and the saved-spectrum adjoint of complex64 grids store the row
    transforms row-major and gather pass 2's columns with bulk tensor copies; the transposing
    pass 1 (XL_RS_RM=0) gives bit-identical fields, saved spectra and distance gradients."""
    import torch
    xl = lib()
    g = inputs.Grid.centred(128, 0.5)
    zs = [50.0, 20.0, 20.0, 75.0]
    B = len(zs)
    u = np.stack([inputs.gaussian_random_phase(g, 15.0, 900 + i) for i in range(B)]).astype(np.complex64)
    G = inputs.random_unit(910, (B, 128, 128)).astype(np.complex64)
    U, Gd = to_dev(u, np.complex64), to_dev(G, np.complex64)

    def run():
        S = xl.save_buffer(U)
        out = xl.rs_propagate(U, g, LAM, zs, saved=S)
        gi, gz = xl.rs_propagate_backward(Gd, None, g, LAM, zs, want_field=True, want_dz=True, saved=S)
        torch.cuda.synchronize()
        return out, S, gi, gz

    rm = run()
    monkeypatch.setenv("XL_RS_RM", "0")
    tr = run()
    for a, b in zip(rm, tr):
        assert torch.equal(a, b)
    xl.device_status()
    for i, z in enumerate(zs):
        assert rel(to_np(rm[0])[i], oracle.rs_conv(u[i].astype(np.complex128), 0.5, 0.5, LAM, z)) < TOL_C64
