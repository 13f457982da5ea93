"""Seeded synthetic inputs shared by the GPU path's tests/benchmark and the CPU oracle.

This module holds no propagation, element or loss arithmetic: it only draws random numbers and
samples source beams, so that both sides receive bit-identical inputs. The GPU path gets the
complex64 (or complex128) rounding of each field; the oracle gets the same rounded values
promoted to float64.

Random numbers: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state_i = seed + (i + 1) * 0x9E3779B97F4A7C15, output
mix(state_i); a double in [0, 1) is (x >> 11) * 2^-53.

Sources follow the paper's simulations (Methods, "Features and performance": Gaussian beams
defined in larger computational windows, 1024^2 or 2048^2 pixels); the grids and sizes are
those of the synthetic workloads listed in ``WORKLOADS``.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs (uint64) for the given seed."""
    with np.errstate(over="ignore"):
        s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (np.arange(1, n + 1, dtype=np.uint64) * _GAMMA)
        z = s
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """n doubles uniform in [0, 1)."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclasses.dataclass(frozen=True)
class Grid:
    """Sampling grid x_m = x0 + m dx, y_n = y0 + n dy (micrometres)."""
    nx: int
    ny: int
    dx: float
    dy: float
    x0: float
    y0: float

    @staticmethod
    def centred(n: int, pitch: float) -> "Grid":
        return Grid(n, n, pitch, pitch, -(n // 2) * pitch, -(n // 2) * pitch)

    def coords(self):
        x = self.x0 + np.arange(self.nx) * self.dx
        y = self.y0 + np.arange(self.ny) * self.dy
        return x, y

    def astuple(self):
        return (self.nx, self.ny, self.dx, self.dy, self.x0, self.y0)


@dataclasses.dataclass(frozen=True)
class Window:
    """Output window X_p = xo0 + p dxo, Y_q = yo0 + q dyo (micrometres)."""
    mx: int
    my: int
    dxo: float
    dyo: float
    xo0: float
    yo0: float

    @staticmethod
    def centred(m: int, width: float) -> "Window":
        d = width / m
        return Window(m, m, d, d, -width / 2, -width / 2)

    def astuple(self):
        return (self.mx, self.my, self.dxo, self.dyo, self.xo0, self.yo0)


def gaussian(grid: Grid, w0: float) -> np.ndarray:
    """Real amplitude exp(-rho^2 / w0^2), peak 1, [ny, nx] float64."""
    x, y = grid.coords()
    return np.exp(-(y[:, None] ** 2 + x[None, :] ** 2) / (w0 * w0))


def random_phase(grid: Grid, seed: int) -> np.ndarray:
    """Phase uniform in [0, 2 pi), [ny, nx] float64."""
    return (2.0 * np.pi) * uniform(seed, grid.nx * grid.ny).reshape(grid.ny, grid.nx)


def gaussian_random_phase(grid: Grid, w0: float, seed: int) -> np.ndarray:
    """Scalar source: Gaussian times exp(i phi) with phi ~ U[0, 2 pi)."""
    return gaussian(grid, w0) * np.exp(1j * random_phase(grid, seed))


def radial_gaussian(grid: Grid, w0: float) -> np.ndarray:
    """Radially polarised source (Ex, Ey) = (x / w0, y / w0) G, [2, ny, nx]."""
    x, y = grid.coords()
    g = gaussian(grid, w0)
    return np.stack([x[None, :] / w0 * g, y[:, None] / w0 * g]).astype(np.complex128)


def random_jones(grid: Grid, w0: float, seed: int) -> np.ndarray:
    """Random Jones field (cos chi e^{i phi1}, sin chi e^{i phi2}) G with chi ~ U[0, pi/2),
    phi1, phi2 ~ U[0, 2 pi); [2, ny, nx]."""
    n = grid.nx * grid.ny
    u = uniform(seed, 3 * n).reshape(3, grid.ny, grid.nx)
    chi = 0.5 * np.pi * u[0]
    g = gaussian(grid, w0)
    return np.stack([np.cos(chi) * np.exp(2j * np.pi * u[1]) * g,
                     np.sin(chi) * np.exp(2j * np.pi * u[2]) * g])


def x_polarised_gaussian(grid: Grid, w0: float) -> np.ndarray:
    """Scalar Gaussian field (the x component of an x-polarised source), [ny, nx] complex."""
    return gaussian(grid, w0).astype(np.complex128)


def random_unit(seed: int, shape) -> np.ndarray:
    """Complex field with independent U(-1, 1) real and imaginary parts (test vectors)."""
    n = int(np.prod(shape))
    u = uniform(seed, 2 * n)
    return ((2 * u[:n] - 1) + 1j * (2 * u[n:] - 1)).reshape(shape)


def rounded(a: np.ndarray, dtype) -> np.ndarray:
    """The field as the GPU receives it (complex64 / complex128)."""
    return np.ascontiguousarray(a, dtype=dtype)


# Synthetic workloads (micrometres). Seeds: 20231012 + index.
SEED0 = 20231012
WORKLOADS = {
    # RS, complex128, 256^2 at 1 um, lambda 0.6328, G(w0=40) x lens(f=10 mm) x random phase, z=10 mm
    "rs256_c128": dict(n=256, pitch=1.0, wavelength=0.6328, w0=40.0, f=10_000.0, z=10_000.0,
                       seed=SEED0 + 1),
    # RS and CZT at 2048^2, 0.5 um, lambda 0.633, G(w0=200) x random phase; CZT onto 512^2 over 64 um
    "rs2048": dict(n=2048, pitch=0.5, wavelength=0.633, w0=200.0, zs=(500.0, 2000.0, 10_000.0),
                   window_m=512, window_w=64.0, seed=SEED0 + 2),
    # VRS / VCZT at 2048^2, z = 5 mm
    "vrs2048": dict(n=2048, pitch=0.5, wavelength=0.633, w0=200.0, z=5000.0, window_m=512,
                    window_w=64.0, seed=SEED0 + 3),
    # optical table at 1024^2: SLM1 -> RS z1 -> SLM2 -> HWP(0.3) -> VRS z2 -> lens f -> VCZT f
    "table1024": dict(n=1024, pitch=1.0, wavelength=0.6328, w0=200.0, z1=20_000.0, z2=20_000.0,
                      theta=0.3, f=5000.0, window_m=256, window_w=64.0, seed=SEED0 + 4),
}
