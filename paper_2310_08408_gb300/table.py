"""Differentiable optical table on the GPU (the virtual tables of the paper's discovery runs:
Results, "Towards large-scale discovery", and Methods, "Rediscovery through exploration within
fixed topologies": source, SLMs, wave plate, free-space propagation, lens, camera).

    x-polarised source -> SLM1 (phi1) -> RS over z1 -> SLM2 (phi2) -> to-vector
    -> half-wave plate (theta) -> VRS over z2 -> thin lens (f) -> VCZT over f onto the camera
    window -> second-moment spot size of the total intensity |Ex|^2 + |Ey|^2 + |Ez|^2

Each stage is a torch.autograd.Function over one C-ABI call (forward and adjoint in the CUDA
library); torch autograd only chains them and keeps the per-plane fields (one checkpoint per
optical plane). The batch dimension holds independent setups: every setup has its own masks,
angle and distances.
"""
from __future__ import annotations

import dataclasses
import math

import torch

from . import autograd as A
from . import xl


@dataclasses.dataclass
class TableGeometry:
    grid: tuple          # (nx, ny, dx, dy, x0, y0)
    window: tuple        # (mx, my, dxo, dyo, xo0, yo0)
    wavelength: float
    f: float             # lens focal length = VCZT distance


def table_loss(geo: TableGeometry, src, phi1, phi2, theta, z1, z2, checkpoint=False):
    """src [B][1][ny][nx] complex; phi1, phi2 [B][ny][nx] real; theta, z1, z2 float64 [B].
    Returns the loss per setup [B] (float64). checkpoint: the RS and VRS stages keep their input
    fields for the distance gradients instead of their input spectra (three planes a setup
    instead of twelve; the adjoints transform the inputs again)."""
    B = src.shape[0]
    dev = src.device
    zero = torch.zeros(B, dtype=torch.float64, device=dev)
    g, lam = geo.grid, geo.wavelength
    # SLM1 on the scalar field
    p1 = torch.zeros((B, 1, 4), dtype=torch.float64, device=dev)
    a0 = A.elements(src, g, lam, [xl.SLM], [(phi1, None)], p1, 1)
    # RS over z1
    # the camera loss ignores a constant phase on every plane (phase_invariant distance gradients)
    a1 = A.RSPropagate.apply(a0[:, 0], z1, g, lam, True, checkpoint)[:, None]
    # SLM2, to-vector, half-wave plate (eta = pi) at theta
    wp = torch.stack([zero, zero, zero + math.pi, theta], dim=1)
    p2 = torch.stack([torch.zeros_like(wp), torch.zeros_like(wp), wp], dim=1).contiguous()
    a2 = A.elements(a1, g, lam, [xl.SLM, xl.TO_VECTOR, xl.WAVEPLATE], [(phi2, None), (None, None),
                                                                       (None, None)], p2, 1)
    # VRS over z2 (Ex, Ey, Ez); the lens acts on all three components; VCZT propagates the
    # transverse ones and re-forms Ez on the camera window (the input Ez plane is not used)
    a3 = A.VRSPropagate.apply(a2, z2, g, lam, True, checkpoint)
    pl = torch.zeros((B, 1, 4), dtype=torch.float64, device=dev)
    pl[:, 0, 0] = geo.f
    a4 = A.elements(a3, g, lam, [xl.LENS], [(None, None)], pl, 3)
    zf = torch.full((B,), geo.f, dtype=torch.float64, device=dev)
    a5 = A.CZTPropagate.apply(a4, zf, g, geo.window, lam, 2)
    return A.IntensityLoss.apply(a5, geo.window, 0b111, xl.SECOND_MOMENT, 0.0)
