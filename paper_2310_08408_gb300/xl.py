"""Thin ctypes binding of the C-ABI library ``libxl.so`` (argument marshalling only).

Every function takes torch CUDA tensors (complex64 or complex128, contiguous) and enqueues the
library call on torch's current stream; all arithmetic runs in the library's CUDA kernels.
There is no fallback: if the library is missing or a call fails, an exception is raised.
Names follow the C ABI (``include/xl.h``) without the ``xl_`` prefix.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libxl.so")

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_NONFINITE = range(7)
C64, C128 = 0, 1
Z_DEVICE = 1

_lock = threading.Lock()
_lib = None


class XLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"xl status {status}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    """xl_grid: x_m = x0 + m dx, y_n = y0 + n dy."""
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double)]

    @staticmethod
    def of(g) -> "Grid":
        if isinstance(g, Grid):
            return g
        t = g.astuple() if hasattr(g, "astuple") else tuple(g)
        return Grid(int(t[0]), int(t[1]), *map(float, t[2:6]))


class Window(ctypes.Structure):
    """xl_window: X_p = xo0 + p dxo, Y_q = yo0 + q dyo."""
    _fields_ = [("mx", ctypes.c_int32), ("my", ctypes.c_int32), ("dxo", ctypes.c_double),
                ("dyo", ctypes.c_double), ("xo0", ctypes.c_double), ("yo0", ctypes.c_double)]

    @staticmethod
    def of(w) -> "Window":
        if isinstance(w, Window):
            return w
        t = w.astuple() if hasattr(w, "astuple") else tuple(w)
        return Window(int(t[0]), int(t[1]), *map(float, t[2:6]))


_P = ctypes.c_void_p
_I = ctypes.c_int32
_D = ctypes.c_double
_GP = ctypes.POINTER(Grid)
_WP = ctypes.POINTER(Window)

# C signatures (argtypes) of every exported entry point, in header order.
SIGNATURES = {
    "xl_version": ([], ctypes.c_char_p),
    "xl_last_error": ([], ctypes.c_char_p),
    "xl_cache_clear": ([], _I),
    "xl_cache_bytes": ([], ctypes.c_int64),
    "xl_rs_propagate": ([_P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_rs_propagate_backward": ([_P, _P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_vrs_propagate": ([_P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_vrs_propagate_backward": ([_P, _P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
}


def load(path: str = LIB_PATH):
    """Loads the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"xl CUDA library not found at {path}: build it first "
                                   "(python -m paper_2310_08408_gb300.build)")
            lib = ctypes.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _check(status: int) -> None:
    if status != OK:
        raise XLError(status, load().xl_last_error().decode())


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dtype(t: torch.Tensor) -> int:
    if t.dtype == torch.complex64:
        return C64
    if t.dtype == torch.complex128:
        return C128
    raise TypeError(f"expected complex64 or complex128, got {t.dtype}")


def _dev(t: torch.Tensor, name: str) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class _Z:
    """Distances: a host array (float / sequence / numpy / CPU tensor) or a CUDA float64 tensor
    (read by the kernels at run time)."""

    def __init__(self, z, batch: int):
        if isinstance(z, torch.Tensor) and z.is_cuda:
            if z.dtype != torch.float64 or z.numel() != batch or not z.is_contiguous():
                raise ValueError("device z must be a contiguous float64 tensor with one entry per batch element")
            self.keep = z
            self.ptr = z.data_ptr()
            self.flags = Z_DEVICE
        else:
            a = np.asarray(z.cpu() if isinstance(z, torch.Tensor) else z, dtype=np.float64).ravel()
            if a.size == 1 and batch > 1:
                a = np.repeat(a, batch)
            if a.size != batch:
                raise ValueError("z must have one entry per batch element")
            self.keep = np.ascontiguousarray(a)
            self.ptr = self.keep.ctypes.data
            self.flags = 0


def version() -> str:
    return load().xl_version().decode()


def cache_clear() -> None:
    _check(load().xl_cache_clear())


def cache_bytes() -> int:
    return int(load().xl_cache_bytes())


def _planes(u: torch.Tensor, comps: int, name: str):
    """Returns (batch, ny, nx) of a [B][comps][ny][nx] (or [comps][ny][nx] / [ny][nx]) tensor."""
    if comps == 1:
        if u.dim() == 2:
            return 1, u.shape[0], u.shape[1]
        if u.dim() == 3:
            return u.shape[0], u.shape[1], u.shape[2]
    else:
        if u.dim() == 3 and u.shape[0] == comps:
            return 1, u.shape[1], u.shape[2]
        if u.dim() == 4 and u.shape[1] == comps:
            return u.shape[0], u.shape[2], u.shape[3]
    raise ValueError(f"{name}: bad shape {tuple(u.shape)} for {comps} component(s)")


def rs_propagate(u: torch.Tensor, grid, wavelength: float, z, out: torch.Tensor | None = None):
    """Scalar RS propagation of [B][ny][nx] (or [ny][nx]) planes; returns the same shape."""
    _dev(u, "u")
    B, ny, nx = _planes(u, 1, "u")
    g = Grid.of(grid)
    if out is None:
        out = torch.empty_like(u)
    zz = _Z(z, B)
    _check(load().xl_rs_propagate(u.data_ptr(), _dev(out, "out").data_ptr(), B, ctypes.byref(g),
                                  float(wavelength), zz.ptr, zz.flags, _dtype(u), _stream()))
    return out


def rs_propagate_backward(g_out: torch.Tensor, u_in: torch.Tensor | None, grid, wavelength: float,
                          z, want_field: bool = True, want_dz: bool = False):
    """Adjoint of rs_propagate: returns (g_in or None, g_z [B] float64 or None)."""
    _dev(g_out, "g_out")
    B, ny, nx = _planes(g_out, 1, "g_out")
    g = Grid.of(grid)
    g_in = torch.empty_like(g_out) if want_field else None
    g_z = torch.empty(B, dtype=torch.float64, device=g_out.device) if want_dz else None
    zz = _Z(z, B)
    _check(load().xl_rs_propagate_backward(
        g_out.data_ptr(), _dev(u_in, "u_in").data_ptr() if u_in is not None else None,
        g_in.data_ptr() if g_in is not None else None, g_z.data_ptr() if g_z is not None else None,
        B, ctypes.byref(g), float(wavelength), zz.ptr, zz.flags, _dtype(g_out), _stream()))
    return g_in, g_z


def vrs_propagate(exy: torch.Tensor, grid, wavelength: float, z, out: torch.Tensor | None = None):
    """Vectorial RS: [B][2][ny][nx] -> [B][3][ny][nx] (also [2][ny][nx] -> [3][ny][nx])."""
    _dev(exy, "exy")
    B, ny, nx = _planes(exy, 2, "exy")
    g = Grid.of(grid)
    if out is None:
        shape = (3, ny, nx) if exy.dim() == 3 else (B, 3, ny, nx)
        out = torch.empty(shape, dtype=exy.dtype, device=exy.device)
    zz = _Z(z, B)
    _check(load().xl_vrs_propagate(exy.data_ptr(), _dev(out, "out").data_ptr(), B, ctypes.byref(g),
                                   float(wavelength), zz.ptr, zz.flags, _dtype(exy), _stream()))
    return out


def vrs_propagate_backward(g_exyz: torch.Tensor, exy_in: torch.Tensor | None, grid,
                           wavelength: float, z, want_field: bool = True, want_dz: bool = False):
    """Adjoint of vrs_propagate: returns (g_exy or None, g_z or None)."""
    _dev(g_exyz, "g_exyz")
    B, ny, nx = _planes(g_exyz, 3, "g_exyz")
    g = Grid.of(grid)
    g_exy = None
    if want_field:
        shape = (2, ny, nx) if g_exyz.dim() == 3 else (B, 2, ny, nx)
        g_exy = torch.empty(shape, dtype=g_exyz.dtype, device=g_exyz.device)
    g_z = torch.empty(B, dtype=torch.float64, device=g_exyz.device) if want_dz else None
    zz = _Z(z, B)
    _check(load().xl_vrs_propagate_backward(
        g_exyz.data_ptr(), _dev(exy_in, "exy_in").data_ptr() if exy_in is not None else None,
        g_exy.data_ptr() if g_exy is not None else None,
        g_z.data_ptr() if g_z is not None else None, B, ctypes.byref(g), float(wavelength),
        zz.ptr, zz.flags, _dtype(g_exyz), _stream()))
    return g_exy, g_z
