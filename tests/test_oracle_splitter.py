"""Pins of the oracle's beam splitter (Results, "Towards large-scale discovery"; Methods, "The
large-scale search space": beam splitters with a continuous ratio connect the paths of the table).

Reading: a lossless, non-polarising splitter of reflectance R, amplitudes t = sqrt(1 - R),
r = sqrt(R), the reflected amplitude carrying the factor i. The pins are properties any such
splitter must have, not the formula retyped: energy conservation for every R, the limits R = 0
(straight through) and R = 1 (ports exchanged), the 50:50 split, a balanced Mach-Zehnder
interferometer sending all light to one port, the adjoint identity, and the R-gradient by finite
differences.
"""
import numpy as np

import oracle
from paper_2310_08408_gb300 import inputs


def _pair(seed, n=257):
    a = inputs.random_unit(seed, (n,)) * (0.5 + inputs.uniform(seed + 1, n))
    b = inputs.random_unit(seed + 2, (n,)) * (0.5 + inputs.uniform(seed + 3, n))
    return a.astype(np.complex128), b.astype(np.complex128)


def _energy(*fs):
    return sum(float(np.sum(np.abs(f) ** 2)) for f in fs)


def test_energy_conserved_every_ratio():
    a, b = _pair(5100)
    for R in (0.0, 0.1, 0.37, 0.5, 0.9, 1.0):
        ot, orr = oracle.beam_splitter(a, b, R)
        assert abs(_energy(ot, orr) - _energy(a, b)) < 1e-12 * _energy(a, b)


def test_limits():
    a, b = _pair(5110)
    ot, orr = oracle.beam_splitter(a, b, 0.0)
    assert np.array_equal(ot, a) and np.array_equal(orr, b)
    ot, orr = oracle.beam_splitter(a, b, 1.0)
    assert np.allclose(ot, 1j * b, atol=1e-15) and np.allclose(orr, 1j * a, atol=1e-15)


def test_fifty_fifty_split():
    a, _ = _pair(5120)
    ot, orr = oracle.beam_splitter(a, None, 0.5)
    assert np.allclose(np.abs(ot) ** 2, np.abs(a) ** 2 / 2, rtol=1e-14)
    assert np.allclose(orr, 1j * ot, atol=1e-15)  # quarter-wave phase of the reflected port


def test_balanced_mach_zehnder_sends_all_light_to_one_port():
    """Two 50:50 splitters with equal arms: the transmitted-port amplitudes of the two paths
    cancel, so every photon leaves through the other port (the textbook interferometer)."""
    a, _ = _pair(5130)
    u1, u2 = oracle.beam_splitter(a, None, 0.5)
    ot, orr = oracle.beam_splitter(u1, u2, 0.5)
    assert np.max(np.abs(ot)) < 1e-15
    assert np.allclose(orr, 1j * a, atol=1e-15)
    # a phase pi on one arm swaps the dark port
    ot, orr = oracle.beam_splitter(u1, -u2, 0.5)
    assert np.max(np.abs(orr)) < 1e-15 and np.allclose(ot, a, atol=1e-15)


def test_adjoint_identity():
    a, b = _pair(5140)
    gt, gr = _pair(5150)
    for R in (0.2, 0.75):
        ot, orr = oracle.beam_splitter(a, b, R)
        ga, gb, _ = oracle.beam_splitter_backward(gt, gr, a, b, R)
        lhs = np.vdot(gt, ot) + np.vdot(gr, orr)
        rhs = np.vdot(ga, a) + np.vdot(gb, b)
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_ratio_gradient_finite_differences():
    """L = sum |out_t|^2 w_t + Re(conj(c) out_r): dL/dR by 4th-order central differences."""
    a, b = _pair(5160)
    w = inputs.uniform(5170, a.size)
    c = inputs.random_unit(5180, a.shape)

    def loss(R):
        ot, orr = oracle.beam_splitter(a, b, R)
        return float(np.sum(w * np.abs(ot) ** 2) + np.real(np.vdot(c, orr)))

    for R in (0.15, 0.5, 0.8):
        ot, _ = oracle.beam_splitter(a, b, R)
        g_t = 2 * w * ot  # dL/dRe + i dL/dIm of sum w |o|^2
        g_r = c           # of Re(conj(c) o)
        _, _, gR = oracle.beam_splitter_backward(g_t, g_r, a, b, R)
        h = 1e-4
        fd = (-loss(R + 2 * h) + 8 * loss(R + h) - 8 * loss(R - h) + loss(R - 2 * h)) / (12 * h)
        assert abs(gR - fd) < 1e-7 * max(1.0, abs(fd))
