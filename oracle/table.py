"""Oracle composition of the differentiable optical table (test infrastructure only).

The table follows the paper's virtual optical tables (Results, "Towards large-scale
discovery"; Methods, "Rediscovery through exploration within fixed topologies": light source,
SLMs, wave plate, free-space propagation, lens, camera): an x-polarised source goes through
    SLM1 (phi1) -> RS over z1 -> SLM2 (phi2) -> to-vector -> half-wave plate (theta)
    -> VRS over z2 -> thin lens (f) -> VCZT over f onto the camera window
    -> second-moment spot size of the total intensity.
``forward`` returns the loss and the per-plane fields; ``backward`` applies the adjoint of
every step in reverse (the oracle's own adjoints), giving dL/dphi1, dL/dphi2, dL/dtheta,
dL/dz1, dL/dz2. Everything is float64 / complex128.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle


@dataclasses.dataclass
class Table:
    grid: tuple          # (nx, ny, dx, dy, x0, y0)
    window: tuple        # (mx, my, dxo, dyo, xo0, yo0)
    wavelength: float
    f: float             # lens focal length = CZT distance
    comp_mask: int = 0b111


def _inner_re(a, b):
    """Re <a, b> = Re sum conj(a) b."""
    return float(np.real(np.vdot(np.ravel(a), np.ravel(b))))


def forward(t: Table, src, phi1, phi2, theta, z1, z2):
    g = t.grid
    nx, ny, dx, dy = g[0], g[1], g[2], g[3]
    lam = t.wavelength
    a0 = oracle.apply_elements(np.asarray(src)[None], g, lam, [dict(kind=oracle.SLM, phi_x=phi1)])
    a1 = oracle.rs_conv(a0[0], dx, dy, lam, z1)[None]
    vec_els = [dict(kind=oracle.SLM, phi_x=phi2), dict(kind=oracle.TO_VECTOR),
               dict(kind=oracle.WAVEPLATE, eta=np.pi, theta=theta)]
    a2 = oracle.apply_elements(a1, g, lam, vec_els)
    a3 = oracle.vrs(a2, dx, dy, lam, z2)
    a4 = oracle.apply_elements(a3[:2], g, lam, [dict(kind=oracle.LENS, f=t.f)])
    # the lens acts on the transverse components; VCZT re-forms Ez from them
    a5 = oracle.vczt(a4, g, t.window, lam, t.f)
    win_grid = t.window
    loss, _ = oracle.intensity_loss(a5, win_grid, t.comp_mask, oracle.SECOND_MOMENT)
    planes = dict(a0=a0, a1=a1, a2=a2, a3=a3, a4=a4, a5=a5, vec_els=vec_els)
    return loss, planes


def backward(t: Table, src, phi1, phi2, theta, z1, z2, planes):
    g = t.grid
    nx, ny, dx, dy = g[0], g[1], g[2], g[3]
    lam = t.wavelength
    g5 = oracle.intensity_loss_backward(planes["a5"], t.window, t.comp_mask, oracle.SECOND_MOMENT)
    g4 = oracle.vczt_adjoint(g5, g, t.window, lam, t.f)
    g3t, _, _, _ = oracle.apply_elements_backward(g4, planes["a3"][:2], g, lam,
                                                  [dict(kind=oracle.LENS, f=t.f)])
    g3 = np.stack([g3t[0], g3t[1], np.zeros_like(g3t[0])])
    # the lens output dropped Ez of the VRS plane (VCZT rebuilds it), so its gradient is 0
    g2 = oracle.vrs_adjoint(g3, dx, dy, lam, z2)
    dz2 = _inner_re(g3, oracle.vrs_dz(planes["a2"], dx, dy, lam, z2))
    g1, gpx, _, gp = oracle.apply_elements_backward(g2, planes["a1"], g, lam, planes["vec_els"])
    dphi2 = gpx[0]
    dtheta = gp[2, 3]
    dz1 = _inner_re(g1[0], oracle.rs_conv(planes["a0"][0], dx, dy, lam, z1, oracle.K_DH))
    g0 = oracle.rs_conv(g1[0], dx, dy, lam, z1, oracle.K_H, adjoint=True)
    _, gpx0, _, _ = oracle.apply_elements_backward(g0[None], np.asarray(src)[None], g, lam,
                                                   [dict(kind=oracle.SLM, phi_x=phi1)])
    return dict(phi1=gpx0[0], phi2=dphi2, theta=dtheta, z1=dz1, z2=dz2)
