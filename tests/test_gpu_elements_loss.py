"""GPU parity of the fused element chains, camera losses and Adam against the FP64 oracle.

Elements (Methods, "Features and performance"; readings: SLM / super-SLM phases, thin lens
exp(-ik rho^2 / 2f), Jones polariser R(-a) diag(1,0) R(a), wave plate R(-t) diag(1, e^{i eta}) R(t),
to-vector (u, 0)); losses (Methods, "Loss function"; second-moment reading); Adam (Kingma & Ba).
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C128, TOL_C64, TOL_LOSS, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu
LAM = 0.6328


# SLM -> lens -> to-vector -> wave plate -> super-SLM -> polariser (the wave plate gives Ey a
# non-zero value before the super-SLM so that both of its masks receive a gradient)
def _chain(ph, px, py):
    return [dict(kind=0, phi_x=ph), dict(kind=2, f=3000.0), dict(kind=5),
            dict(kind=4, eta=2.1, theta=0.35), dict(kind=1, phi_x=px, phi_y=py),
            dict(kind=3, alpha=-0.4)]


def _oracle_chain(ph, px, py):
    return [dict(kind=oracle.SLM, phi_x=ph), dict(kind=oracle.LENS, f=3000.0),
            dict(kind=oracle.TO_VECTOR), dict(kind=oracle.WAVEPLATE, eta=2.1, theta=0.35),
            dict(kind=oracle.SSLM, phi_x=px, phi_y=py), dict(kind=oracle.POLARIZER, alpha=-0.4)]


@pytest.mark.parametrize("dtype,rdtype,tol", [(np.complex64, np.float32, TOL_C64),
                                              (np.complex128, np.float64, TOL_C128)])
@pytest.mark.parametrize("shared", [False, True])
def test_element_chain_forward_backward(dtype, rdtype, tol, shared):
    import torch
    xl = lib()
    g = inputs.Grid(96, 80, 1.0, 1.0, -48.0, -40.0)
    B = 2
    u = np.stack([inputs.gaussian_random_phase(g, 30.0, 5 + b) for b in range(B)])[:, None].astype(dtype)
    nm = 1 if shared else B
    phs = [np.stack([inputs.random_phase(g, 10 * k + b) for b in range(nm)]).astype(rdtype) for k in range(3)]
    dev = [to_dev(p[0] if shared else p, rdtype) for p in phs]
    out = to_np(xl.apply_elements(to_dev(u, dtype), g, LAM, _chain(*dev), comps_in=1))
    G = inputs.random_unit(77, (B, 2, 80, 96)).astype(dtype)
    g_in, gpx, gpy, gp = xl.apply_elements_backward(to_dev(G, dtype), to_dev(u, dtype), g, LAM,
                                                    _chain(*dev), comps_in=1)
    gsum = [np.zeros((80, 96)) for _ in range(3)]
    for b in range(B):
        sel = [p[0] if shared else p[b] for p in phs]
        och = _oracle_chain(*[s.astype(np.float64) for s in sel])
        ref = oracle.apply_elements(u[b].astype(np.complex128), g.astuple(), LAM, och)
        assert rel(out[b], ref) < tol
        rg, rpx, rpy, rp = oracle.apply_elements_backward(G[b].astype(np.complex128),
                                                          u[b].astype(np.complex128), g.astuple(),
                                                          LAM, och)
        assert rel(to_np(g_in)[b], rg) < tol
        for k, (arr, idx) in enumerate(((gpx, 0), (gpx, 4), (gpy, 4))):
            got = to_np(arr[idx])
            rr = (rpx if arr is gpx else rpy)[idx]
            if shared:
                gsum[k] += rr
            else:
                assert rel(got[b], rr) < 10 * tol
        gpn = to_np(gp)[b]
        for e, j in ((1, 0), (3, 2), (3, 3), (5, 1)):
            assert abs(gpn[e, j] - rp[e, j]) <= 1e-5 * max(1.0, abs(rp[e, j])) if dtype == np.complex64 \
                else abs(gpn[e, j] - rp[e, j]) <= 1e-10 * max(1.0, abs(rp[e, j]))
    if shared:
        for k, (arr, idx) in enumerate(((gpx, 0), (gpx, 4), (gpy, 4))):
            assert rel(to_np(arr[idx]), gsum[k]) < 10 * tol


@pytest.mark.parametrize("dtype,rdtype,tol", [(np.complex64, np.float32, TOL_C64),
                                              (np.complex128, np.float64, TOL_C128)])
@pytest.mark.parametrize("kind,comps", [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3)])
@pytest.mark.parametrize("want_field", [True, False])
def test_single_mask_backward(dtype, rdtype, tol, kind, comps, want_field):
    """A chain of one SLM (kind 0) or super-SLM (kind 1) with masks per batch element: the
    adjoint that reads only the input, the cotangent and the masks, on a plane that is not a
    multiple of the pixels a block takes (37 x 53), against the oracle."""
    xl = lib()
    g = inputs.Grid(53, 37, 1.0, 1.0, -26.0, -18.0)
    B = 3
    u = inputs.random_unit(91, (B, comps, 37, 53)).astype(dtype)
    G = inputs.random_unit(92, (B, comps, 37, 53)).astype(dtype)
    px = np.stack([inputs.random_phase(g, 930 + b) for b in range(B)]).astype(rdtype)
    py = np.stack([inputs.random_phase(g, 940 + b) for b in range(B)]).astype(rdtype)
    el = dict(kind=kind, phi_x=to_dev(px, rdtype))
    if kind == 1:
        el["phi_y"] = to_dev(py, rdtype)
    xl.profile_enable(True)
    g_in, gpx, gpy, gp = xl.apply_elements_backward(to_dev(G, dtype), to_dev(u, dtype), g, LAM, [el],
                                                    comps_in=comps, want_field=want_field,
                                                    want_params=False)
    launched = xl.profile_report()
    xl.profile_enable(False)
    assert "elements_bwd_mask" in launched and "elements_bwd" not in launched
    for b in range(B):
        oe = dict(kind=oracle.SLM if kind == 0 else oracle.SSLM, phi_x=px[b].astype(np.float64))
        if kind == 1:
            oe["phi_y"] = py[b].astype(np.float64)
        Gb, ub = G[b].astype(np.complex128), u[b].astype(np.complex128)
        if comps == 3:
            # the oracle's chains take 1 or 2 components; the masks act on each component on its
            # own (an SLM on all three, a super-SLM on Ex and Ey with Ez passed through), so the
            # 3-component adjoint is the per-component (SLM) or (Ex, Ey) (super-SLM) one
            if kind == 0:
                parts = [oracle.apply_elements_backward(Gb[c], ub[c], g.astuple(), LAM, [oe])
                         for c in range(3)]
                rg = np.stack([p[0][0] for p in parts])
                rpx = [sum(p[1][0] for p in parts)]
            else:
                rg2, rpx, rpy, _ = oracle.apply_elements_backward(Gb[:2], ub[:2], g.astuple(), LAM, [oe])
                rg = np.concatenate([rg2, Gb[2:]])
        else:
            rg, rpx, rpy, _ = oracle.apply_elements_backward(Gb, ub, g.astuple(), LAM, [oe])
        if want_field:
            assert rel(to_np(g_in)[b], rg) < tol
        assert rel(to_np(gpx[0])[b], rpx[0]) < 10 * tol
        if kind == 1:
            assert rel(to_np(gpy[0])[b], rpy[0]) < 10 * tol
    assert (g_in is None) == (not want_field)


def test_elements_device_parameters_match_host():
    import torch
    xl = lib()
    g = inputs.Grid.centred(64, 0.5)
    u = inputs.random_jones(g, 10.0, 3)[None].astype(np.complex64)
    els = [dict(kind=4, eta=np.pi, theta=0.3), dict(kind=2, f=900.0), dict(kind=3, alpha=0.2)]
    a = to_np(xl.apply_elements(to_dev(u, np.complex64), g, LAM, els, comps_in=2))
    prm = torch.tensor([[[0, 0, np.pi, 0.3], [900.0, 0, 0, 0], [0, 0.2, 0, 0]]], dtype=torch.float64,
                       device="cuda")
    b = to_np(xl.apply_elements(to_dev(u, np.complex64), g, LAM, els, comps_in=2, params=prm))
    assert rel(b, a) < 1e-6


@pytest.mark.parametrize("dtype,tol", [(np.complex64, TOL_LOSS), (np.complex128, 1e-10)])
@pytest.mark.parametrize("mask", [0b011, 0b100, 0b111])
def test_second_moment_loss_and_gradient(dtype, tol, mask):
    xl = lib()
    g = inputs.Grid(200, 150, 0.25, 0.3, -20.0, -25.0)
    E = np.stack([inputs.random_jones(g, 6.0, 9 + b) for b in range(3)])
    E = np.concatenate([E, 0.3 * E[:, :1]], axis=1).astype(dtype)  # 3 components
    loss, inten = xl.intensity_loss(to_dev(E, dtype), g, mask, xl.SECOND_MOMENT, want_intensity=True)
    gf = to_np(xl.intensity_loss_backward(to_dev(E, dtype), g, mask, xl.SECOND_MOMENT))
    for b in range(3):
        L, I = oracle.intensity_loss(E[b].astype(np.complex128), g.astuple(), mask)
        assert abs(to_np(loss)[b] - L) / L < tol
        assert rel(to_np(inten)[b], I) < (1e-6 if dtype == np.complex64 else 1e-13)
        rg = oracle.intensity_loss_backward(E[b].astype(np.complex128), g.astuple(), mask)
        assert rel(gf[b], rg) < (1e-4 if dtype == np.complex64 else 1e-10)


def test_density_loss_and_gradient():
    import torch
    xl = lib()
    g = inputs.Grid.centred(128, 0.5)
    E = inputs.random_jones(g, 12.0, 21)[None].astype(np.complex64)
    eps = 0.5
    # both sides decide "I > eps * i_max" from the same complex64 values; check the margin so the
    # selection cannot differ between float32 and float64 intensities
    I = np.sum(np.abs(E[0].astype(np.complex128)) ** 2, axis=0)
    assert np.min(np.abs(I - eps * I.max())) > 1e-5 * I.max()
    loss, _ = xl.intensity_loss(to_dev(E, np.complex64), g, 0b11, xl.DENSITY, eps)
    L, _ = oracle.intensity_loss(E[0].astype(np.complex128), g.astuple(), 0b11, oracle.DENSITY, eps)
    assert abs(to_np(loss)[0] - L) / L < TOL_LOSS
    gl = torch.tensor([2.5], dtype=torch.float64, device="cuda")
    gf = to_np(xl.intensity_loss_backward(to_dev(E, np.complex64), g, 0b11, xl.DENSITY, eps, g_loss=gl))
    rg = oracle.intensity_loss_backward(E[0].astype(np.complex128), g.astuple(), 0b11, oracle.DENSITY,
                                        eps, g_loss=2.5)
    assert rel(gf[0], rg) < 1e-4


def test_nonfinite_loss_sets_device_status():
    import torch
    xl = lib()
    g = inputs.Grid.centred(32, 1.0)
    E = torch.zeros((1, 1, 32, 32), dtype=torch.complex64, device="cuda")
    xl.device_status()  # clear
    xl.intensity_loss(E, g, 1, xl.SECOND_MOMENT)  # 0 / 0
    with pytest.raises(xl.XLError) as e:
        xl.device_status()
    assert e.value.status == xl.ERR_NONFINITE
    xl.device_status()  # cleared


@pytest.mark.parametrize("rdtype", [np.float32, np.float64])
def test_adam_matches_oracle_over_steps(rdtype):
    import torch
    xl = lib()
    n = 1000
    p0 = inputs.uniform(1, n) * 4 - 2
    grads = [inputs.uniform(10 + k, n) - 0.5 for k in range(4)]
    p = to_dev(p0.astype(rdtype), rdtype)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    t = torch.ones(1, dtype=torch.int32, device="cuda")
    pr, mr, vr = p0.astype(rdtype).astype(np.float64), np.zeros(n), np.zeros(n)
    for k, gk in enumerate(grads):
        gk = gk.astype(rdtype)
        xl.adam_step(p, m, v, to_dev(gk, rdtype), lr=0.01, t=t)
        xl.step_advance(t)
        oracle.adam(pr, mr, vr, gk.astype(np.float64), 0.01, k + 1)
    tol = 1e-6 if rdtype == np.float32 else 1e-14
    assert np.max(np.abs(to_np(p) - pr)) < tol
    assert int(to_np(t)[0]) == 5


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("comps,mask", [(1, 1), (3, 0b111), (3, 0b100)])
def test_loss_and_grad_in_one_call(mode, comps, mask):
    """xl_intensity_loss_and_grad equals the two calls it replaces (same statistics and kernels:
    bit for bit) and the oracle (loss 1e-4, gradient relative L2 1e-3... at complex64)."""
    import torch
    xl = lib()
    g = inputs.Grid(96, 80, 0.7, 0.6, -33.6, -24.0)
    f = np.stack([inputs.random_unit(6100 + c, (80, 96)) * inputs.gaussian(g, 15.0)
                  for c in range(comps)])[None].astype(np.complex64)
    F = to_dev(f, np.complex64)
    l1, _ = xl.intensity_loss(F, g, mask, mode, 0.4)
    g1 = xl.intensity_loss_backward(F, g, mask, mode, 0.4)
    l2, g2 = xl.intensity_loss_and_grad(F, g, mask, mode, 0.4)
    assert torch.equal(l1, l2) and torch.equal(g1, g2)
    L, _ = oracle.intensity_loss(f[0].astype(np.complex128), g.astuple(), mask, mode, 0.4)
    G = oracle.intensity_loss_backward(f[0].astype(np.complex128), g.astuple(), mask, mode, 0.4)
    assert abs(float(l2.cpu()[0]) - L) <= TOL_LOSS * abs(L)
    assert rel(to_np(g2)[0], G) < 1e-3
