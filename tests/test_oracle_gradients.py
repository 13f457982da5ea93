"""Pins of the oracle's adjoints and gradients.

- Dot-product test <P u, v> = <u, P^H v> for RS (every kernel kind), VRS, CZT and VCZT.
- Central finite differences (float64) along seeded random directions for the loss gradient
  (second moment; density with the selection frozen), the element gradients (phase masks,
  lens f, polariser angle, wave-plate eta and theta, the input field), the distance
  derivatives, and the whole optical table (masks, theta, z1, z2).
Gradients follow the convention g = dL/dRe u + i dL/dIm u, so dL = Re sum conj(g) du.
"""
import numpy as np
import pytest

import oracle
import oracle.table as otable
from paper_2310_08408_gb300 import inputs

LAM = 0.6328


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def inner(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


@pytest.mark.parametrize("kind", range(6))
def test_rs_adjoint_dot_product(kind):
    u = inputs.random_unit(1, (16, 32))
    v = inputs.random_unit(2, (16, 32))
    Pu = oracle.rs_conv(u, 0.5, 0.6, LAM, 20.0, kind)
    PHv = oracle.rs_conv(v, 0.5, 0.6, LAM, 20.0, kind, adjoint=True)
    assert abs(inner(v, Pu) - inner(PHv, u)) / abs(inner(v, Pu)) < 1e-12


def test_vrs_vczt_czt_adjoint_dot_products():
    u = inputs.random_unit(3, (2, 16, 16))
    v = inputs.random_unit(4, (3, 16, 16))
    a = inner(v, oracle.vrs(u, 0.5, 0.5, LAM, 20.0))
    b = inner(oracle.vrs_adjoint(v, 0.5, 0.5, LAM, 20.0), u)
    assert abs(a - b) / abs(a) < 1e-12
    grid = (16, 16, 0.5, 0.5, -4.0, -4.0)
    win = (12, 10, 0.4, 0.3, -2.0, -1.0)
    w = inputs.random_unit(5, (3, 10, 12))
    a = inner(w, oracle.vczt(u, grid, win, LAM, 30.0))
    b = inner(oracle.vczt_adjoint(w, grid, win, LAM, 30.0), u)
    assert abs(a - b) / abs(a) < 1e-12
    for kind in range(6):
        a = inner(w[0], oracle.czt_conv(u[0], grid, win, LAM, 30.0, kind))
        b = inner(oracle.czt_conv(w[0], grid, win, LAM, 30.0, kind, adjoint=True), u[0])
        assert abs(a - b) / abs(a) < 1e-12


def _fd(fun, h):
    return (-fun(2 * h) + 8 * fun(h) - 8 * fun(-h) + fun(-2 * h)) / (12 * h)


@pytest.mark.parametrize("mask", [0b011, 0b100, 0b111])
def test_second_moment_gradient_fd(mask):
    g = inputs.Grid.centred(24, 0.5)
    E = inputs.random_unit(6, (3, 24, 24))
    D = inputs.random_unit(7, (3, 24, 24))
    grad = oracle.intensity_loss_backward(E, g.astuple(), mask, oracle.SECOND_MOMENT)
    L = lambda t: oracle.intensity_loss(E + t * D, g.astuple(), mask, oracle.SECOND_MOMENT)[0]
    fd = _fd(L, 1e-4)
    assert abs(np.real(inner(grad, D)) - fd) / abs(fd) < 1e-8


def test_density_gradient_fd_with_frozen_selection():
    g = inputs.Grid.centred(24, 0.5)
    E = inputs.random_unit(8, (1, 24, 24))
    D = inputs.random_unit(9, (1, 24, 24))
    eps = 0.4
    grad = oracle.intensity_loss_backward(E, g.astuple(), 1, oracle.DENSITY, eps)
    # the step is small enough that no pixel crosses the threshold
    _, I = oracle.intensity_loss(E, g.astuple(), 1, oracle.DENSITY, eps)
    margin = np.min(np.abs(I - eps * I.max()))
    h = 1e-7
    assert margin > 100 * h
    L = lambda t: oracle.intensity_loss(E + t * D, g.astuple(), 1, oracle.DENSITY, eps)[0]
    # the threshold moves with i_max, which has no gradient (as with a where-based selection):
    # freeze it by perturbing away from the brightest pixel
    imax = np.unravel_index(np.argmax(I), I.shape)
    D[0][imax] = 0
    fd = _fd(L, h)
    assert abs(np.real(inner(grad, D)) - fd) / abs(fd) < 1e-6


def test_element_gradients_fd():
    g = inputs.Grid.centred(12, 0.5)
    gt = g.astuple()
    u = inputs.random_unit(10, (1, 12, 12))
    phi = 2 * np.pi * inputs.uniform(11, 144).reshape(12, 12)
    phx = 2 * np.pi * inputs.uniform(12, 144).reshape(12, 12)
    phy = 2 * np.pi * inputs.uniform(13, 144).reshape(12, 12)
    prm = dict(f=400.0, alpha=0.4, eta=1.3, theta=0.25)

    def chain(uu, ph, px, py, p):
        return [dict(kind=oracle.SLM, phi_x=ph), dict(kind=oracle.LENS, f=p["f"]),
                dict(kind=oracle.TO_VECTOR), dict(kind=oracle.SSLM, phi_x=px, phi_y=py),
                dict(kind=oracle.WAVEPLATE, eta=p["eta"], theta=p["theta"]),
                dict(kind=oracle.POLARIZER, alpha=p["alpha"])]

    W = inputs.random_unit(14, (2, 12, 12))

    def L(uu=u, ph=phi, px=phx, py=phy, p=prm):
        out = oracle.apply_elements(uu, gt, LAM, chain(uu, ph, px, py, p))
        return float(np.real(inner(W, out)))

    els = chain(u, phi, phx, phy, prm)
    g_in, gpx, gpy, gp = oracle.apply_elements_backward(W, u, gt, LAM, els)
    Du = inputs.random_unit(15, (1, 12, 12))
    assert abs(np.real(inner(g_in, Du)) - _fd(lambda t: L(uu=u + t * Du), 1e-5)) < 1e-9
    Dp = inputs.uniform(16, 144).reshape(12, 12) - 0.5
    assert abs(np.sum(gpx[0] * Dp) - _fd(lambda t: L(ph=phi + t * Dp), 1e-5)) < 1e-9
    assert abs(np.sum(gpx[3] * Dp) - _fd(lambda t: L(px=phx + t * Dp), 1e-5)) < 1e-9
    assert abs(np.sum(gpy[3] * Dp) - _fd(lambda t: L(py=phy + t * Dp), 1e-5)) < 1e-9
    for idx, (name, h) in [(1, ("f", 1e-3)), (4, ("eta", 1e-5)), (4, ("theta", 1e-5)),
                           (5, ("alpha", 1e-5))]:
        col = {"f": 0, "alpha": 1, "eta": 2, "theta": 3}[name]
        fd = _fd(lambda t: L(p={**prm, name: prm[name] + t}), h)
        assert abs(gp[idx, col] - fd) < 1e-8 * max(1.0, abs(fd)), name


@pytest.mark.parametrize("which", ["rs", "vrs", "czt"])
def test_distance_derivative_fd(which):
    z = 25.0
    if which == "rs":
        u = inputs.random_unit(17, (16, 16))
        W = inputs.random_unit(18, (16, 16))
        L = lambda zz: np.real(inner(W, oracle.rs_conv(u, 0.5, 0.5, LAM, zz)))
        d = np.real(inner(W, oracle.rs_conv(u, 0.5, 0.5, LAM, z, oracle.K_DH)))
    elif which == "vrs":
        u = inputs.random_unit(19, (2, 16, 16))
        W = inputs.random_unit(20, (3, 16, 16))
        L = lambda zz: np.real(inner(W, oracle.vrs(u, 0.5, 0.5, LAM, zz)))
        d = np.real(inner(W, oracle.vrs_dz(u, 0.5, 0.5, LAM, z)))
    else:
        grid = (16, 16, 0.5, 0.5, -4.0, -4.0)
        win = (12, 10, 0.4, 0.3, -2.0, -1.0)
        u = inputs.random_unit(21, (2, 16, 16))
        W = inputs.random_unit(22, (3, 10, 12))
        L = lambda zz: np.real(inner(W, oracle.vczt(u, grid, win, LAM, zz)))
        d = np.real(inner(W, oracle.vczt_dz(u, grid, win, LAM, z)))
    fd = _fd(lambda t: L(z + t), 1e-4)
    assert abs(d - fd) / abs(fd) < 1e-8


def test_optical_table_gradient_fd():
    n, pitch = 32, 1.0
    g = inputs.Grid.centred(n, pitch)
    win = inputs.Window.centred(24, 40.0)
    t = otable.Table(g.astuple(), win.astuple(), LAM, f=600.0)
    src = inputs.x_polarised_gaussian(g, 8.0)
    phi1 = 0.3 * inputs.random_phase(g, 23)
    phi2 = 0.3 * inputs.random_phase(g, 24)
    theta, z1, z2 = 0.3, 150.0, 120.0
    loss, planes = otable.forward(t, src, phi1, phi2, theta, z1, z2)
    grads = otable.backward(t, src, phi1, phi2, theta, z1, z2, planes)
    D1 = inputs.uniform(25, n * n).reshape(n, n) - 0.5
    D2 = inputs.uniform(26, n * n).reshape(n, n) - 0.5
    F = lambda **kw: otable.forward(t, src, kw.get("phi1", phi1), kw.get("phi2", phi2),
                                    kw.get("theta", theta), kw.get("z1", z1), kw.get("z2", z2))[0]
    checks = [
        # steps balance the 4th-order truncation against round-off of a loss of O(100 um^2)
        (np.sum(grads["phi1"] * D1), _fd(lambda s: F(phi1=phi1 + s * D1), 1e-2)),
        (np.sum(grads["phi2"] * D2), _fd(lambda s: F(phi2=phi2 + s * D2), 1e-2)),
        (grads["theta"], _fd(lambda s: F(theta=theta + s), 1e-3)),
        (grads["z1"], _fd(lambda s: F(z1=z1 + s), 1e-1)),
        (grads["z2"], _fd(lambda s: F(z2=z2 + s), 1e-1)),
    ]
    for got, fd in checks:
        assert abs(got - fd) / abs(fd) < 1e-6, (got, fd)
