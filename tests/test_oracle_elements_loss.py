"""Pins of the oracle's optical elements, camera losses, STED model and Adam.

Elements (Methods, "Features and performance"; readings: Jones matrices R(-t) D R(t),
R(t) = [[cos t, sin t], [-sin t, cos t]]): a polariser is idempotent; a wave plate is unitary;
eta = 0 is the identity; two quarter-wave plates at one angle equal a half-wave plate; a
half-wave plate at theta turns x into polarisation angle 2 theta; an SLM of constant phase c
multiplies by exp(ic); a super-SLM acts per component; to-vector yields (u, 0).
Losses (Methods, "Loss function"; second-moment reading): a sampled Gaussian of intensity
exp(-2 rho^2 / w^2) has sigma_x^2 = sigma_y^2 = w^2/4; a uniform disk of intensity i0 has density
loss exactly 1/i0; the threshold is strict.
STED (Methods, "Stimulated emission depletion model"): the worked values printed in the paper
(tests/golden/sted_worked_values.txt).
Adam (Kingma & Ba): the first bias-corrected step is lr g / (|g| + eps).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs

LAM = 0.6328
G = inputs.Grid.centred(16, 0.5)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def vec_field(seed):
    return inputs.random_unit(seed, (2, G.ny, G.nx))


def app(field, *els):
    return oracle.apply_elements(field, G.astuple(), LAM, list(els))


def test_polariser_idempotent_and_projects():
    f = vec_field(1)
    p = dict(kind=oracle.POLARIZER, alpha=0.37)
    once = app(f, p)
    assert rel(app(once, p), once) < 1e-14
    # the output is along (cos a, sin a)
    c, s = np.cos(0.37), np.sin(0.37)
    assert np.max(np.abs(once[0] * s - once[1] * c)) < 1e-14


def test_waveplate_unitary_identity_and_composition():
    f = vec_field(2)
    w = dict(kind=oracle.WAVEPLATE, eta=1.1, theta=0.6)
    out = app(f, w)
    assert abs(np.sum(abs(out) ** 2) / np.sum(abs(f) ** 2) - 1) < 1e-14
    assert rel(app(f, dict(kind=oracle.WAVEPLATE, eta=0.0, theta=0.6)), f) < 1e-15
    q = dict(kind=oracle.WAVEPLATE, eta=np.pi / 2, theta=0.6)
    h = dict(kind=oracle.WAVEPLATE, eta=np.pi, theta=0.6)
    assert rel(app(f, q, q), app(f, h)) < 1e-14


@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0, -0.7])
def test_half_wave_plate_rotates_x_to_two_theta(theta):
    u = np.ones((1, G.ny, G.nx), complex)
    out = app(u, dict(kind=oracle.TO_VECTOR), dict(kind=oracle.WAVEPLATE, eta=np.pi, theta=theta))
    assert np.allclose(out[0], np.cos(2 * theta), atol=1e-15)
    assert np.allclose(out[1], np.sin(2 * theta), atol=1e-15)


def test_slm_and_super_slm():
    f = vec_field(3)
    c = np.full((G.ny, G.nx), 0.9)
    out = app(f, dict(kind=oracle.SLM, phi_x=c))
    assert rel(out, np.exp(0.9j) * f) < 1e-15
    out = app(f, dict(kind=oracle.SSLM, phi_x=c, phi_y=-2 * c))
    assert rel(out[0], np.exp(0.9j) * f[0]) < 1e-15
    assert rel(out[1], np.exp(-1.8j) * f[1]) < 1e-15
    # pi phase negates
    u = inputs.random_unit(4, (1, G.ny, G.nx))
    assert rel(app(u, dict(kind=oracle.SLM, phi_x=np.full((G.ny, G.nx), np.pi))), -u) < 1e-15


def test_to_vector_and_lens_limit():
    u = inputs.random_unit(5, (1, G.ny, G.nx))
    out = app(u, dict(kind=oracle.TO_VECTOR))
    assert out.shape == (2, G.ny, G.nx) and rel(out[0], u[0]) == 0 and np.all(out[1] == 0)
    # a very long focal length is (nearly) the identity and never changes |u|
    out = app(u, dict(kind=oracle.LENS, f=1e15))
    assert rel(out, u) < 1e-12
    out = app(u, dict(kind=oracle.LENS, f=300.0))
    assert np.allclose(abs(out), abs(u), rtol=1e-15)


def test_second_moment_of_gaussian():
    g = inputs.Grid.centred(256, 0.25)
    w = 6.0
    amp = np.sqrt(np.exp(-2 * ((g.coords()[0][None, :] - 1.5) ** 2
                               + (g.coords()[1][:, None] + 2.0) ** 2) / (w * w)))
    field = np.stack([amp * 0.6, amp * 0.8j, amp * 5.0]).astype(complex)
    loss, inten = oracle.intensity_loss(field, g.astuple(), 0b011, oracle.SECOND_MOMENT)
    assert abs(loss / (w * w / 2) - 1) < 1e-12
    assert np.allclose(inten, amp ** 2)
    # the Ez component alone: same shape, same spot size
    loss_z, _ = oracle.intensity_loss(field, g.astuple(), 0b100, oracle.SECOND_MOMENT)
    assert abs(loss_z / (w * w / 2) - 1) < 1e-12


def test_density_loss_disk_and_strict_threshold():
    g = inputs.Grid.centred(64, 1.0)
    x, y = g.coords()
    disk = ((x[None, :] ** 2 + y[:, None] ** 2) < 15 ** 2).astype(float)
    i0 = 2.5
    field = (np.sqrt(i0) * disk)[None].astype(complex)
    loss, _ = oracle.intensity_loss(field, g.astuple(), 1, oracle.DENSITY, eps=0.5)
    assert loss == pytest.approx(1 / i0, rel=1e-15)
    # a pixel exactly at eps * i_max is excluded (strict ">")
    inten = np.zeros((4, 4))
    inten[0, 0], inten[1, 1], inten[2, 2] = 16.0, 4.0, 9.0  # exact squares; 4 = 0.25 * 16
    loss, _ = oracle.intensity_loss(np.sqrt(inten)[None].astype(complex),
                                    inputs.Grid.centred(4, 1.0).astuple(), 1, oracle.DENSITY,
                                    eps=0.25)
    assert loss == pytest.approx(2 / 25.0, rel=1e-15)


def _golden_sted():
    path = os.path.join(os.path.dirname(__file__), "golden", "sted_worked_values.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            beta, ratio, closed, approx, tol = line.split()
            rows.append((float(beta), float(ratio), closed, float(approx), float(tol)))
    return rows


def test_sted_worked_values_from_paper():
    for beta, ratio, closed, approx, tol in _golden_sted():
        i_ex = np.array([1.0, 3.0])
        out = oracle.sted(i_ex, ratio * i_ex, beta) / i_ex
        exact = eval(closed, {"exp": np.exp})
        assert np.allclose(out, exact, rtol=1e-15)
        assert abs(out[0] - approx) < tol
    i = np.array([0.0, 2.0, 2.0])
    assert np.allclose(oracle.sted(i, np.array([1.0, 0.0, 5.0]), 0.0), [0.0, 2.0, 2.0])
    assert oracle.sted(np.array([2.0]), np.array([0.0]), 1.0)[0] == 2.0


def test_adam_first_step_closed_form_and_second_step():
    g = np.array([0.3, -2.0, 1e-9, 0.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    m, v = np.zeros(4), np.zeros(4)
    p0 = p.copy()
    oracle.adam(p, m, v, g, lr=0.01, t=1)
    assert np.allclose(p, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    p1 = p.copy()
    oracle.adam(p, m, v, g, lr=0.01, t=2)
    assert np.allclose(p, p1 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-14)
