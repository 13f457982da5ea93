"""Pins of the oracle's angular-spectrum CZT (the exact-RS reading of the CZT propagator: Methods,
"Features and performance", CZT of Hu et al.).

Reading: the angular spectrum of the sampled field (the n-point DFT, signed frequencies
f = j / (n dx), j in [-n/2, n/2)), times the transfer function exp(i z sqrt(k^2 - kx^2 - ky^2))
(evanescent decay beyond the light cone), summed back onto an arbitrary window and divided by
nx ny. Pins, none of which retypes that formula:
- on the native grid it is the angular-spectrum method, ifft2(fft2(u) H) (library routine);
- a sum of plane waves on the DFT frequencies is propagated exactly, at any output point: each
  wave picks up exp(i z kz) (a propagating one) or decays by exp(-z kappa) (an evanescent one),
  the trigonometric interpolation of such a band-limited field being exact;
- z = 0 on the native grid is the identity;
- the adjoint identity <A u, G> = <u, A^H G>;
- the distance derivative (kind AS_DH) against central differences in z.
"""
import numpy as np

import oracle
from paper_2310_08408_gb300 import inputs

LAM = 0.6328
K = 2 * np.pi / LAM


def _grid(n, d):
    return (n, n, d, d, -(n // 2) * d, -(n // 2) * d)


def _transfer_fft_order(n, d, z):
    f = np.fft.fftfreq(n, d)
    FX, FY = np.meshgrid(f, f)
    a = K * K - (2 * np.pi) ** 2 * (FX ** 2 + FY ** 2)
    kz = np.where(a >= 0, np.sqrt(np.abs(a)) + 0j, 1j * np.sqrt(np.abs(a)))
    return np.exp(1j * kz * z)


def test_native_grid_is_angular_spectrum_method():
    n, d, z = 64, 0.5, 40.0
    g = _grid(n, d)
    u = inputs.random_unit(5300, (n, n))
    out = oracle.asczt(u, g, g, LAM, z)
    ref = np.fft.ifft2(np.fft.fft2(u) * _transfer_fft_order(n, d, z))
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))


def test_plane_waves_propagate_exactly_at_any_point():
    n, d, z = 32, 0.25, 2.0
    g = _grid(n, d)
    x = g[4] + d * np.arange(n)
    X, Y = np.meshgrid(x, x)
    # (j, l, amplitude): propagating waves and one evanescent wave (|f| > 1 / lambda)
    waves = [(0, 0, 1.0), (3, -2, 0.5 - 0.2j), (-7, 5, 0.3j), (13, 0, 0.25)]
    u = np.zeros((n, n), complex)
    for j, l, c in waves:
        u += c * np.exp(2j * np.pi * (j / (n * d) * X + l / (n * d) * Y))
    assert 13 / (n * d) > 1 / LAM  # the last wave is evanescent
    # an off-grid window: shifted, finer and rectangular
    w = (24, 20, 0.13, 0.21, -1.7, 0.9)
    out = oracle.asczt(u, g, w, LAM, z)
    Xp = w[4] + w[2] * np.arange(w[0])
    Yq = w[5] + w[3] * np.arange(w[1])
    XP, YQ = np.meshgrid(Xp, Yq)
    ref = np.zeros_like(out)
    for j, l, c in waves:
        f, gg = j / (n * d), l / (n * d)
        a = K * K - (2 * np.pi) ** 2 * (f * f + gg * gg)
        kz = np.sqrt(a) if a >= 0 else 1j * np.sqrt(-a)
        ref += c * np.exp(1j * kz * z) * np.exp(2j * np.pi * (f * XP + gg * YQ))
    assert np.max(np.abs(out - ref)) < 1e-12
    # the evanescent wave alone has decayed by exp(-z kappa)
    j, l, c = waves[-1]
    f = j / (n * d)
    kappa = np.sqrt((2 * np.pi * f) ** 2 - K * K)
    ue = c * np.exp(2j * np.pi * f * X)
    oe = oracle.asczt(ue, g, w, LAM, z)
    assert abs(np.max(np.abs(oe)) - abs(c) * np.exp(-z * kappa)) < 1e-12


def test_zero_distance_is_identity_on_native_grid():
    n, d = 32, 0.7
    g = _grid(n, d)
    u = inputs.random_unit(5310, (n, n))
    out = oracle.asczt(u, g, g, LAM, 0.0)
    assert np.max(np.abs(out - u)) < 1e-13


def test_adjoint_identity():
    n, d, z = 32, 0.5, 60.0
    g = _grid(n, d)
    w = (20, 24, 0.3, 0.25, -2.0, -3.0)
    u = inputs.random_unit(5320, (n, n))
    G = inputs.random_unit(5330, (w[1], w[0]))
    for kind in (oracle.AS_H, oracle.AS_DH):
        Au = oracle.asczt(u, g, w, LAM, z, kind)
        AhG = oracle.asczt(G, g, w, LAM, z, kind, adjoint=True)
        lhs, rhs = np.vdot(G, Au), np.vdot(AhG, u)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_distance_derivative_finite_differences():
    n, d, z = 32, 0.5, 80.0
    g = _grid(n, d)
    w = (16, 16, 0.4, 0.4, -3.2, -3.2)
    u = inputs.gaussian_random_phase(inputs.Grid(n, n, d, d, g[4], g[5]), 5.0, 5340)
    dA = oracle.asczt(u, g, w, LAM, z, oracle.AS_DH)
    h = 1e-3
    fd = (-oracle.asczt(u, g, w, LAM, z + 2 * h) + 8 * oracle.asczt(u, g, w, LAM, z + h)
          - 8 * oracle.asczt(u, g, w, LAM, z - h) + oracle.asczt(u, g, w, LAM, z - 2 * h)) / (12 * h)
    assert np.max(np.abs(dA - fd)) < 1e-8 * np.max(np.abs(dA))
