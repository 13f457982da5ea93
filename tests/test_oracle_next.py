"""Pins of the oracle's STED derivative, intensity-image losses, softmin over detectors, AdamW
and MSE (Methods: "Stimulated emission depletion model", "Loss function", "Rediscovery through
exploration of optical topologies"; Results: "Data-driven rediscovery").

- STED derivative: central finite differences of the STED intensity (itself pinned by the
  paper's worked values in test_oracle_elements_loss.py), and its stated I_ex = 0 limit.
- Loss of an intensity image: equal to the field version on |E|^2, gradient by finite differences.
- Softmin: closed forms (n equal losses give l - log(n)/beta; a large beta gives the minimum; a
  small beta the mean minus log(n)/beta), weights sum to one and match finite differences.
- AdamW: first step p - lr (g/(|g|+eps) + wd p); wd = 0 reduces to Adam.
- MSE: closed form and finite-difference gradient.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs


def _fd(f, h):
    return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)


@pytest.mark.parametrize("beta", [1.0, 0.5, 0.0, 0.8])
def test_sted_derivative_by_fd(beta):
    ie = 0.2 + inputs.uniform(1, 50) * 3
    idp = inputs.uniform(2, 50) * 4
    ones = np.ones(50)
    ge, gd = oracle.sted_backward(ie, idp, beta, ones)
    fe = _fd(lambda t: oracle.sted(ie + t, idp, beta), 1e-4)
    fdp = _fd(lambda t: oracle.sted(ie, idp + t, beta), 1e-4)
    assert np.max(np.abs(ge - fe)) < 1e-9 and np.max(np.abs(gd - fdp)) < 1e-9
    # I_ex = 0: I_eff = 0 and the I_dep > 0 limit of the derivative
    ge0, gd0 = oracle.sted_backward(np.zeros(1), np.ones(1), beta, np.ones(1))
    assert ge0[0] == pytest.approx(1 - beta) and gd0[0] == 0.0


@pytest.mark.parametrize("mode", [oracle.SECOND_MOMENT, oracle.DENSITY])
def test_loss_from_intensity_matches_field_version_and_fd(mode):
    g = inputs.Grid.centred(24, 0.5)
    E = inputs.random_jones(g, 4.0, 3)
    L1, I = oracle.intensity_loss(E, g.astuple(), 0b11, mode, 0.4)
    L2, dI = oracle.loss_from_intensity(I, g.astuple(), mode, 0.4, want_grad=True)
    assert L1 == pytest.approx(L2, rel=1e-14)
    D = inputs.uniform(4, I.size).reshape(I.shape) - 0.5
    if mode == oracle.DENSITY:
        D[np.unravel_index(np.argmax(I), I.shape)] = 0
        h = 1e-8
    else:
        h = 1e-4
    fd = _fd(lambda t: oracle.loss_from_intensity(I + t * D, g.astuple(), mode, 0.4)[0], h)
    assert abs(np.sum(dI * D) - fd) / abs(fd) < 1e-6


def test_softmin_closed_forms_and_gradient():
    out, w = oracle.softmin(np.full((1, 6), 2.5), beta=3.0)
    assert out[0] == pytest.approx(2.5 - np.log(6) / 3.0, rel=1e-15)
    assert np.allclose(w, 1 / 6)
    l = np.array([[3.0, 1.2, 5.0, 1.25]])
    assert oracle.softmin(l, 1e4)[0][0] == pytest.approx(1.2, abs=1e-4)
    small = oracle.softmin(l, 1e-6)[0][0]
    assert small == pytest.approx(l.mean() - np.log(4) / 1e-6, rel=1e-6)
    _, w = oracle.softmin(l, 2.0)
    assert w.sum() == pytest.approx(1.0, rel=1e-15)
    for d in range(4):
        e = np.zeros_like(l)
        e[0, d] = 1
        fd = _fd(lambda t: oracle.softmin(l + t * e, 2.0)[0][0], 1e-4)
        assert w[0, d] == pytest.approx(fd, rel=1e-8)


def test_adamw_first_step_and_reduction_to_adam():
    g = np.array([0.3, -2.0, 0.5])
    p0 = np.array([1.0, -2.0, 3.0])
    p, m, v = p0.copy(), np.zeros(3), np.zeros(3)
    oracle.adamw(p, m, v, g, lr=0.01, t=1, wd=1e-4)
    assert np.allclose(p, p0 - 0.01 * (g / (np.abs(g) + 1e-8) + 1e-4 * p0), rtol=0, atol=1e-15)
    a, ma, va = p0.copy(), np.zeros(3), np.zeros(3)
    b, mb, vb = p0.copy(), np.zeros(3), np.zeros(3)
    for t in range(1, 4):
        oracle.adam(a, ma, va, g * t, 0.02, t)
        oracle.adamw(b, mb, vb, g * t, 0.02, t, wd=0.0)
    assert np.array_equal(a, b)


def test_mse_closed_form_and_fd():
    I = np.array([[1.0, 2.0], [3.0, 4.0]])
    T = np.array([[1.5, 2.0], [2.0, 6.0]])
    L, dI = oracle.mse(I, T, want_grad=True)
    assert L == pytest.approx((0.25 + 0 + 1 + 4) / 4, rel=1e-15)
    assert np.allclose(dI, 2 * (I - T) / 4)
