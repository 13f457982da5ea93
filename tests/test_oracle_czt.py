"""Pins of the oracle's CZT / VCZT (reading: Fresnel form of the RS integral evaluated on an
explicit output window, amplitude exp(ikz)/(i lambda z); Methods, "Features and performance").

- The separable two-pass sum equals the brute-force sum over the full, non-factored kernel
  (every kernel kind, including the Ez and z-derivative kinds).
- Dirichlet closed form: a thin lens of focal length f followed by CZT over z = f turns a
  K x K aperture into prefactor x product of sin(K beta/2)/sin(beta/2).
- With output pitch lambda z / (N dx) and M = N the CZT is chirp x plain DFT (numpy FFT).
- A sampled Gaussian propagates to the closed-form Fresnel Gaussian.
- Energy is conserved when the window covers the beam.
- VCZT identity Ez' = -(1/z)[X Ex' + Y Ey' - C(x Ex + y Ey)].
- The kernel z-derivatives agree with finite differences.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs

LAM = 0.633
K = 2 * np.pi / LAM


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


GRID = (12, 10, 0.7, 0.9, -4.0, -3.5)
WIN = (9, 7, 0.3, 0.45, -1.2, -0.8)


@pytest.mark.parametrize("kind", range(6))
def test_czt_separable_equals_brute(kind):
    u = inputs.random_unit(40 + kind, (10, 12))
    a = oracle.czt_conv(u, GRID, WIN, LAM, 50.0, kind)
    b = oracle.czt_conv(u, GRID, WIN, LAM, 50.0, kind, method="brute")
    assert rel(a, b) < 1e-12
    pts = [(0, 0), (8, 6), (3, 2)]
    got = oracle.czt_points(u, GRID, WIN, LAM, 50.0, pts, kind)
    assert rel(got, np.array([b[q, p] for p, q in pts])) < 1e-12


def test_czt_dirichlet_closed_form_lens_then_focus():
    n, pitch, Kap, f = 64, 1.0, 21, 2000.0
    g = inputs.Grid.centred(n, pitch)
    x, y = g.coords()
    ap = np.zeros((n, n), complex)
    s = n // 2 - Kap // 2
    ap[s:s + Kap, s:s + Kap] = 1.0
    lensed = oracle.apply_elements(ap[None], g.astuple(), LAM, [dict(kind=oracle.LENS, f=f)])[0]
    win = inputs.Window.centred(48, 240.0)
    out = oracle.czt_conv(lensed, g.astuple(), win.astuple(), LAM, f)
    X = win.xo0 + np.arange(win.mx) * win.dxo
    Y = win.yo0 + np.arange(win.my) * win.dyo
    xs = x[s]

    def axis(Xv):
        beta = K * Xv * pitch / f
        with np.errstate(invalid="ignore", divide="ignore"):
            d = np.where(np.abs(np.sin(beta / 2)) < 1e-15, Kap,
                         np.sin(Kap * beta / 2) / np.sin(beta / 2))
        return np.exp(-1j * K * Xv * xs / f) * np.exp(-1j * beta * (Kap - 1) / 2) * d

    pref = np.exp(1j * K * f) / (1j * LAM * f) * pitch * pitch
    exact = (pref * np.exp(1j * K * (X[None, :] ** 2 + Y[:, None] ** 2) / (2 * f))
             * axis(Y)[:, None] * axis(X)[None, :])
    assert rel(out, exact) < 1e-12


def test_czt_reduces_to_dft():
    n, pitch, z = 32, 0.5, 300.0
    g = inputs.Grid.centred(n, pitch)
    x, _ = g.coords()
    d = LAM * z / (n * pitch)
    win = inputs.Window(n, n, d, d, -7.0, 3.0)
    u = inputs.random_unit(9, (n, n))
    out = oracle.czt_conv(u, g.astuple(), win.astuple(), LAM, z)
    X = win.xo0 + np.arange(n) * d
    Y = win.yo0 + np.arange(n) * d
    ax = np.exp(1j * K * x ** 2 / (2 * z)) * np.exp(-1j * K * win.xo0 * (x - x[0]) / z)
    ay = np.exp(1j * K * x ** 2 / (2 * z)) * np.exp(-1j * K * win.yo0 * (x - x[0]) / z)
    F = np.fft.fft2(u * ay[:, None] * ax[None, :])
    post_x = np.exp(1j * K * X ** 2 / (2 * z)) * np.exp(-1j * K * X * x[0] / z)
    post_y = np.exp(1j * K * Y ** 2 / (2 * z)) * np.exp(-1j * K * Y * x[0] / z)
    pref = np.exp(1j * K * z) / (1j * LAM * z) * pitch * pitch
    assert rel(out, pref * post_y[:, None] * post_x[None, :] * F) < 1e-12


def test_czt_gaussian_fresnel_closed_form_and_energy():
    n, pitch, w0, z = 128, 0.5, 6.0, 150.0
    g = inputs.Grid.centred(n, pitch)
    u0 = inputs.gaussian(g, w0).astype(complex)
    win = inputs.Window.centred(96, 60.0)
    out = oracle.czt_conv(u0, g.astuple(), win.astuple(), LAM, z)
    X = win.xo0 + np.arange(win.mx) * win.dxo
    zr = K * w0 * w0 / 2
    q0, q = -1j * zr, z - 1j * zr
    rho2 = X[None, :] ** 2 + X[:, None] ** 2
    exact = np.exp(1j * K * z) * (q0 / q) * np.exp(1j * K * rho2 / (2 * q))
    assert rel(out, exact) < 1e-8
    e_in = np.sum(abs(u0) ** 2) * pitch ** 2
    e_out = np.sum(abs(out) ** 2) * win.dxo * win.dyo
    assert abs(e_out / e_in - 1) < 1e-6


def test_vczt_ez_identity_and_adjoint_kinds():
    u = inputs.random_unit(50, (2, 10, 12))
    z = 40.0
    out = oracle.vczt(u, GRID, WIN, LAM, z)
    nx, ny, dx, dy, x0, y0 = GRID
    mx, my, dxo, dyo, xo0, yo0 = WIN
    x = x0 + np.arange(nx) * dx
    y = y0 + np.arange(ny) * dy
    X = xo0 + np.arange(mx) * dxo
    Y = yo0 + np.arange(my) * dyo
    s = x[None, :] * u[0] + y[:, None] * u[1]
    rhs = -(1 / z) * (X[None, :] * out[0] + Y[:, None] * out[1]
                      - oracle.czt_conv(s, GRID, WIN, LAM, z))
    assert rel(out[2], rhs) < 1e-12


@pytest.mark.parametrize("kind,dkind", [(0, 3), (1, 4), (2, 5)])
def test_czt_z_derivative_kinds_by_fd(kind, dkind):
    u = inputs.random_unit(60, (10, 12))
    z, h = 50.0, 1e-3
    c = lambda zz: oracle.czt_conv(u, GRID, WIN, LAM, zz, kind)
    fd = (-c(z + 2 * h) + 8 * c(z + h) - 8 * c(z - h) + c(z - 2 * h)) / (12 * h)
    assert rel(oracle.czt_conv(u, GRID, WIN, LAM, z, dkind), fd) < 1e-8
