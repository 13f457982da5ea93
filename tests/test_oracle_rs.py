"""Pins of the oracle's FFT, RS and VRS against things other than itself.

- FFT: the direct DFT definition and numpy's FFT (a library routine).
- RS (Methods, "Features and performance"; reading: rectangle-rule first RS integral on the
  input grid): the FFT realisation equals the brute-force O(N^4) direct sum; the kernel equals
  -(dx dy / 2 pi) d/dz [exp(ikr)/r] by finite differences of the Green's function; a
  complex-source-point beam (an exact outgoing Helmholtz solution, Deschamps 1971) is
  reproduced; 90-degree rotation and flip equivariance; energy conservation for a beam well
  inside the window; paraxial Gaussian width.
- VRS (reading: Ez' = sum Ex h_x + Ey h_y, h_x = -(a dx/z) h): the exact discrete identity
  Ez' = -(1/z)[x Ex' + y Ey' - RS(x Ex + y Ey)], the h_x kernel against d/dx of the Green's
  function, and the divergence of the propagated field.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs

LAM = 0.6328
K = 2 * np.pi / LAM


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32, 64, 256])
def test_fft_matches_direct_dft_and_numpy(n):
    x = inputs.random_unit(11 + n, (n,))
    for sign in (-1, 1):
        f = oracle.fft(x, sign)
        assert rel(f, oracle.dft(x, sign)) < 1e-13 if n > 1 else np.allclose(f, x)
    assert rel(oracle.fft(x, -1), np.fft.fft(x)) < 1e-13 if n > 1 else True
    assert rel(oracle.fft(x, +1), n * np.fft.ifft(x)) < 1e-13 if n > 1 else True


def test_fft2_matches_numpy():
    x = inputs.random_unit(5, (64, 128))
    assert rel(oracle.fft2(x), np.fft.fft2(x)) < 1e-13


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12, complex))


@pytest.mark.parametrize("kind", range(6))
@pytest.mark.parametrize("adjoint", [False, True])
def test_rs_fft_equals_direct_sum(kind, adjoint):
    # rectangular grid so x/y mix-ups fail
    u = inputs.random_unit(100 + kind, (32, 64))
    a = oracle.rs_conv(u, 0.5, 0.75, LAM, 40.0, kind, adjoint, "fft")
    b = oracle.rs_conv(u, 0.5, 0.75, LAM, 40.0, kind, adjoint, "direct")
    assert rel(a, b) < 1e-12


def test_rs_direct_points_match_direct():
    u = inputs.random_unit(7, (16, 16))
    full = oracle.rs_conv(u, 1.0, 1.0, LAM, 30.0, 0, False, "direct")
    pts = [(0, 0), (15, 3), (7, 15), (9, 9)]
    got = oracle.rs_points(u, 1.0, 1.0, LAM, 30.0, pts)
    assert rel(got, np.array([full[q, p] for p, q in pts])) < 1e-13


def _green(x, y, z):
    r = np.sqrt(x * x + y * y + z * z)
    return np.exp(1j * K * r) / r


def test_rs_kernel_is_minus_dz_green_over_2pi():
    dx, dy, z, n = 0.7, 1.1, 25.0, 6
    tab = oracle.rs_kernel_table(0, n, n, dx, dy, LAM, z)
    a = np.arange(-(n - 1), n)
    X, Y = a[None, :] * dx, a[:, None] * dy
    hstep = 1e-3
    d4 = lambda f: (-f(2 * hstep) + 8 * f(hstep) - 8 * f(-hstep) + f(-2 * hstep)) / (12 * hstep)
    dG = d4(lambda t: _green(X, Y, z + t))
    assert rel(tab, -(dx * dy / (2 * np.pi)) * dG) < 1e-9
    # h_x = (dx dy / 2 pi) dG/dX: the transverse derivative of the Green's function
    tabx = oracle.rs_kernel_table(1, n, n, dx, dy, LAM, z)
    dGx = d4(lambda t: _green(X + t, Y, z))
    assert rel(tabx, (dx * dy / (2 * np.pi)) * dGx) < 1e-9
    taby = oracle.rs_kernel_table(2, n, n, dx, dy, LAM, z)
    dGy = d4(lambda t: _green(X, Y + t, z))
    assert rel(taby, (dx * dy / (2 * np.pi)) * dGy) < 1e-9


@pytest.mark.parametrize("kind,dkind", [(0, 3), (1, 4), (2, 5)])
def test_rs_kernel_z_derivatives_by_fd(kind, dkind):
    dx, dy, z, n = 0.5, 0.5, 30.0, 5
    hz = 1e-3
    t = lambda s: oracle.rs_kernel_table(kind, n, n, dx, dy, LAM, z + s)
    fd = (-t(2 * hz) + 8 * t(hz) - 8 * t(-hz) + t(-2 * hz)) / (12 * hz)
    assert rel(oracle.rs_kernel_table(dkind, n, n, dx, dy, LAM, z), fd) < 1e-9


def _csp_beam(x, y, z, b, d):
    """Complex-source-point beam exp(ik(R + ib)) / R, R = sqrt(rho^2 + (z + d - ib)^2),
    principal branch (continuous from R = z + d - ib on the axis for z + d > 0)."""
    R = np.sqrt(x * x + y * y + (z + d - 1j * b) ** 2 + 0j)
    return np.exp(1j * K * (R + 1j * b)) / R


def test_rs_reproduces_complex_source_point_beam():
    n, pitch, w0, d, z = 512, 1.0, 40.0, 1000.0, 10_000.0
    g = inputs.Grid.centred(n, pitch)
    x, y = g.coords()
    b = K * w0 * w0 / 2
    u0 = _csp_beam(x[None, :], y[:, None], 0.0, b, d)
    u1 = oracle.rs_conv(u0, pitch, pitch, LAM, z)
    exact = _csp_beam(x[None, :], y[:, None], z, b, d)
    c = slice(n // 4, 3 * n // 4)
    assert rel(u1[c, c], exact[c, c]) < 1e-4


def test_rs_rotation_and_flip_equivariance():
    u = inputs.random_unit(3, (32, 32))
    f = lambda a: oracle.rs_conv(a, 0.8, 0.8, LAM, 20.0)
    out = f(u)
    assert rel(f(np.rot90(u)), np.rot90(out)) < 1e-12
    assert rel(f(u[:, ::-1]), out[:, ::-1]) < 1e-12
    assert rel(f(u[::-1, :]), out[::-1, :]) < 1e-12
    # linearity
    v = inputs.random_unit(4, (32, 32))
    assert rel(f(2.0 * u - 1j * v), 2.0 * out - 1j * f(v)) < 1e-12


def test_rs_energy_conservation_and_paraxial_width():
    n, pitch, w0, z = 256, 1.0, 20.0, 2000.0
    g = inputs.Grid.centred(n, pitch)
    u0 = inputs.gaussian(g, w0).astype(complex)
    u1 = oracle.rs_conv(u0, pitch, pitch, LAM, z)
    e0, e1 = np.sum(abs(u0) ** 2), np.sum(abs(u1) ** 2)
    assert abs(e1 / e0 - 1) < 1e-3
    # second moment of |u|^2 = exp(-2 rho^2/w^2) gives sigma_x^2 = w^2/4
    x, y = g.coords()
    I = abs(u1) ** 2
    sx2 = np.sum(I * (x[None, :] ** 2)) / np.sum(I)
    zr = np.pi * w0 * w0 / LAM
    w = w0 * np.sqrt(1 + (z / zr) ** 2)
    assert abs(sx2 / (w * w / 4) - 1) < 2e-3


def test_vrs_ez_identity():
    n, pitch, z = 32, 0.5, 15.0
    g = inputs.Grid.centred(n, pitch)
    x, y = g.coords()
    exy = inputs.random_unit(21, (2, n, n))
    out = oracle.vrs(exy, pitch, pitch, LAM, z)
    s = x[None, :] * exy[0] + y[:, None] * exy[1]
    rhs = -(1 / z) * (x[None, :] * out[0] + y[:, None] * out[1] - oracle.rs_conv(s, pitch, pitch, LAM, z))
    assert rel(out[2], rhs) < 1e-12
    assert rel(oracle.vrs(exy, pitch, pitch, LAM, z, "direct"), out) < 1e-12


def test_vrs_field_is_divergence_free():
    # transverse derivatives spectrally (the propagated beam stays well inside the window),
    # the z derivative by a 4th-order central difference
    n, pitch, w0, z, dz = 128, 0.25, 4.0, 30.0, 0.02
    g = inputs.Grid.centred(n, pitch)
    ex = inputs.gaussian(g, w0).astype(complex)
    exy = np.stack([ex, 0.3j * ex])
    E = lambda zz: oracle.vrs(exy, pitch, pitch, LAM, zz)
    e0, ep, em, ep2, em2 = E(z), E(z + dz), E(z - dz), E(z + 2 * dz), E(z - 2 * dz)
    kx = 2 * np.pi * np.fft.fftfreq(n, pitch)
    dxEx = np.fft.ifft(1j * kx[None, :] * np.fft.fft(e0[0], axis=1), axis=1)
    dyEy = np.fft.ifft(1j * kx[:, None] * np.fft.fft(e0[1], axis=0), axis=0)
    dzEz = (-ep2[2] + 8 * ep[2] - 8 * em[2] + em2[2]) / (12 * dz)
    c = slice(n // 4, 3 * n // 4)
    div = dxEx + dyEy + dzEz
    assert np.linalg.norm(div[c, c]) / np.linalg.norm(dxEx[c, c]) < 1e-4
    # without Ez the divergence would not vanish
    assert np.linalg.norm((dxEx + dyEy)[c, c]) / np.linalg.norm(dxEx[c, c]) > 1e-2
