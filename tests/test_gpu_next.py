"""GPU parity of the STED effective-intensity losses, MSE, softmin over detectors and AdamW
against the oracle (Methods: "Stimulated emission depletion model", "Loss function",
"Rediscovery through exploration of optical topologies"; Results: "Data-driven rediscovery")."""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_LOSS, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def _I(E, mask):
    return sum(np.abs(E[c]) ** 2 for c in range(E.shape[0]) if mask & (1 << c))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("beta", [1.0, 0.5])
def test_sted_loss_and_gradient(mode, beta):
    xl = lib()
    g = inputs.Grid.centred(96, 0.5)
    Ex = np.stack([inputs.random_jones(g, 9.0, 30 + b) for b in range(2)]).astype(np.complex64)
    Ed = np.stack([inputs.random_jones(g, 12.0, 40 + b) for b in range(2)]).astype(np.complex64)
    mask, eps = 0b11, 0.4
    loss, ieff = xl.intensity_loss_ex(to_dev(Ex, np.complex64), g, mask, mode, eps,
                                      field_dep=to_dev(Ed, np.complex64), beta=beta,
                                      want_intensity=True)
    gx, gd = xl.intensity_loss_ex_backward(to_dev(Ex, np.complex64), g, mask, mode, eps,
                                           field_dep=to_dev(Ed, np.complex64), beta=beta)
    for b in range(2):
        ie = _I(Ex[b].astype(np.complex128), mask)
        idp = _I(Ed[b].astype(np.complex128), mask)
        I = oracle.sted(ie, idp, beta)
        if mode == 1:  # the selection is decided in float32 on the GPU: keep a clear margin
            assert np.min(np.abs(I - eps * I.max())) > 1e-5 * I.max()
        L, dI = oracle.loss_from_intensity(I, g.astuple(), mode, eps, want_grad=True)
        assert abs(to_np(loss)[b] - L) / L < TOL_LOSS
        assert rel(to_np(ieff)[b], I) < 1e-5
        ge, gdd = oracle.sted_backward(ie, idp, beta, dI)
        assert rel(to_np(gx)[b], 2 * ge * Ex[b].astype(np.complex128)) < 1e-4
        assert rel(to_np(gd)[b], 2 * gdd * Ed[b].astype(np.complex128)) < 1e-4


def test_mse_loss_and_gradient():
    xl = lib()
    g = inputs.Grid.centred(64, 1.0)
    E = np.stack([inputs.random_jones(g, 15.0, 50 + b) for b in range(3)]).astype(np.complex64)
    T = np.stack([np.abs(inputs.random_jones(g, 10.0, 60 + b)).sum(0) ** 2 for b in range(3)]
                 ).astype(np.float32)
    loss, _ = xl.intensity_loss_ex(to_dev(E, np.complex64), g, 0b11, xl.MSE,
                                   target=to_dev(T, np.float32))
    gf, _ = xl.intensity_loss_ex_backward(to_dev(E, np.complex64), g, 0b11, xl.MSE,
                                          target=to_dev(T, np.float32))
    for b in range(3):
        I = _I(E[b].astype(np.complex128), 0b11)
        L, dI = oracle.mse(I, T[b].astype(np.float64), want_grad=True)
        assert abs(to_np(loss)[b] - L) / L < TOL_LOSS
        assert rel(to_np(gf)[b], 2 * dI * E[b].astype(np.complex128)) < 1e-4


def test_softmin_matches_oracle():
    xl = lib()
    l = (inputs.uniform(70, 5 * 6) * 10).reshape(5, 6)
    out, w = xl.softmin(to_dev(l, np.float64), beta=1.7)
    ro, rw = oracle.softmin(l, 1.7)
    assert np.allclose(to_np(out), ro, rtol=1e-13, atol=0)
    assert np.allclose(to_np(w), rw, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("rdtype", [np.float32, np.float64])
def test_adamw_matches_oracle(rdtype):
    import torch
    xl = lib()
    n = 500
    p0 = inputs.uniform(80, n) * 4 - 2
    p = to_dev(p0.astype(rdtype), rdtype)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    pr, mr, vr = p0.astype(rdtype).astype(np.float64), np.zeros(n), np.zeros(n)
    for t in range(1, 4):
        gk = (inputs.uniform(90 + t, n) - 0.5).astype(rdtype)
        xl.adamw_step(p, m, v, to_dev(gk, rdtype), lr=0.01, t=t, weight_decay=1e-4)
        oracle.adamw(pr, mr, vr, gk.astype(np.float64), 0.01, t, 1e-4)
    assert np.max(np.abs(to_np(p) - pr)) < (1e-6 if rdtype == np.float32 else 1e-14)
