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
PHASE_INVARIANT = 2
ACCUMULATE = 4

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


class Element(ctypes.Structure):
    """xl_element: one optical element of a chain (kind, masks, host parameters)."""
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("phi_x", ctypes.c_void_p), ("phi_y", ctypes.c_void_p),
                ("phi_stride", ctypes.c_int64), ("f", ctypes.c_double), ("alpha", ctypes.c_double),
                ("eta", ctypes.c_double), ("theta", ctypes.c_double)]


SLM, SSLM, LENS, POLARIZER, WAVEPLATE, TO_VECTOR = range(6)
SECOND_MOMENT, DENSITY, MSE = 0, 1, 2

class TableConfig(ctypes.Structure):
    """xl_table_config of the batched optical-table optimiser."""
    _fields_ = [("wavelength", ctypes.c_double), ("extent", ctypes.c_double), ("w0", ctypes.c_double),
                ("f", ctypes.c_double), ("cam_width", ctypes.c_double), ("lr", ctypes.c_double),
                ("lr_z", ctypes.c_double), ("cam_m", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("checkpoint", ctypes.c_int32), ("memory_budget", ctypes.c_int64)]

CHECKPOINT_AUTO = 2


BATCH_LOSS, BATCH_SCALARS, BATCH_GRAD_SCALARS, BATCH_PHI1, BATCH_PHI2, BATCH_GRAD_PHI1, BATCH_GRAD_PHI2 = range(7)

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
    "xl_launch_count": ([], ctypes.c_int64),
    "xl_profile_enable": ([_I], _I),
    "xl_profile_report": ([ctypes.c_char_p, _I], _I),
    "xl_rs_propagate": ([_P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_rs_propagate_backward": ([_P, _P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_rs_propagate_static": ([_P, _P, _I, _GP, _D, _P, _P], _I),
    "xl_vrs_propagate": ([_P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_vrs_propagate_backward": ([_P, _P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_rs_propagate_save": ([_P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_rs_propagate_backward_saved": ([_P, _P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_vrs_propagate_save": ([_P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_vrs_propagate_backward_saved": ([_P, _P, _P, _P, _I, _GP, _D, _P, _I, _I, _P], _I),
    "xl_czt_propagate": ([_P, _P, _I, _I, _GP, _WP, _D, _P, _I, _I, _P], _I),
    "xl_apply_elements": ([_P, _P, _I, _I, _GP, _D, ctypes.POINTER(Element), _I, _P, _I, _I, _P], _I),
    "xl_apply_elements_backward": ([_P, _P, _P, _I, _I, _GP, _D, ctypes.POINTER(Element), _I, _P,
                                    _I, _P, _P, _P, _I, _P], _I),
    "xl_intensity_loss": ([_P, _I, _I, ctypes.c_uint32, _GP, _I, _D, _P, _P, _I, _P], _I),
    "xl_intensity_loss_backward": ([_P, _I, _I, ctypes.c_uint32, _GP, _I, _D, _P, _P, _I, _P], _I),
    "xl_intensity_loss_ex": ([_P, _P, _P, _I, _I, ctypes.c_uint32, _GP, _I, _D, _D, _P, _P, _I, _P], _I),
    "xl_intensity_loss_ex_backward": ([_P, _P, _P, _I, _I, ctypes.c_uint32, _GP, _I, _D, _D, _P, _P,
                                       _P, _I, _P], _I),
    "xl_intensity_loss_and_grad": ([_P, _P, _P, _I, _I, ctypes.c_uint32, _GP, _I, _D, _D, _P, _P, _P,
                                    _I, _P], _I),
    "xl_softmin": ([_P, _I, _I, _D, _P, _P, _P], _I),
    "xl_device_status": ([_P], _I),
    "xl_asczt_propagate": ([_P, _P, _I, _GP, _WP, _D, _P, _I, _I, _P], _I),
    "xl_asczt_propagate_backward": ([_P, _P, _P, _P, _I, _GP, _WP, _D, _P, _I, _I, _P], _I),
    "xl_autotune": ([_GP, _WP, _I, _I, _P], _I),
    "xl_tune_get": ([_I, _I, _I], _I),
    "xl_tune_set": ([_I, _I, _I, _I], _I),
    "xl_tune_clear": ([], _I),
    "xl_tune_save": ([ctypes.c_char_p], _I),
    "xl_tune_load": ([ctypes.c_char_p], _I),
    "xl_beam_splitter": ([_P, _P, _P, _P, _I, ctypes.c_int64, _P, _I, _P], _I),
    "xl_beam_splitter_backward": ([_P, _P, _P, _P, _P, _P, _P, _I, ctypes.c_int64, _P, _I, _P], _I),
    "xl_adam_step": ([_P, _P, _P, _P, ctypes.c_int64, _I, _D, _D, _D, _D, _P, _I, _P], _I),
    "xl_adamw_step": ([_P, _P, _P, _P, ctypes.c_int64, _I, _D, _D, _D, _D, _D, _P, _I, _P], _I),
    "xl_step_advance": ([_P, _P], _I),
    "xl_batch_create": ([ctypes.POINTER(TableConfig), _I, _P, _P, ctypes.c_uint64,
                         ctypes.POINTER(ctypes.c_void_p), _P], _I),
    "xl_batch_plan_memory": ([ctypes.POINTER(TableConfig), _I, _P, ctypes.POINTER(_I)], ctypes.c_int64),
    "xl_batch_step": ([_P, _I, _P], _I),
    "xl_batch_read": ([_P, _I, _I, _P, _P], _I),
    "xl_batch_grid": ([_P, _I], _I),
    "xl_batch_memory": ([_P], ctypes.c_int64),
    "xl_batch_destroy": ([_P], _I),
    "xl_czt_propagate_backward": ([_P, _P, _P, _P, _I, _I, _GP, _WP, _D, _P, _I, _I, _P], _I),
    "xl_czt_save_elems": ([_GP, _WP, _I, _I], ctypes.c_int64),
    "xl_czt_propagate_save": ([_P, _P, _P, _I, _I, _GP, _WP, _D, _P, _I, _I, _P], _I),
    "xl_czt_propagate_backward_saved": ([_P, _P, _P, _P, _P, _I, _I, _GP, _WP, _D, _P, _I, _I, _P], _I),
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


def launch_count() -> int:
    """Kernels launched by the library so far (host counter)."""
    return int(load().xl_launch_count())


def profile_enable(on: bool) -> None:
    _check(load().xl_profile_enable(int(bool(on))))


def profile_report() -> dict:
    """{kernel family: (launches, total_ms)} of the launches recorded since profiling was
    enabled (synchronises on their events); clears the records."""
    buf = ctypes.create_string_buffer(1 << 16)
    load().xl_profile_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.rsplit(" ", 2)
        out[name] = (int(n), float(ms))
    return out


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


def rs_propagate(u: torch.Tensor, grid, wavelength: float, z, out: torch.Tensor | None = None,
                 saved: torch.Tensor | None = None):
    """Scalar RS propagation of [B][ny][nx] (or [ny][nx]) planes; returns the same shape.
    saved: optional [B][2nx][2ny] tensor that receives the 2D spectra of the zero-padded input
    for rs_propagate_backward(..., saved=...) (xl_rs_propagate_save); see save_buffer()."""
    _dev(u, "u")
    B, ny, nx = _planes(u, 1, "u")
    g = Grid.of(grid)
    if out is None:
        out = torch.empty_like(u)
    zz = _Z(z, B)
    if saved is not None:
        _check(load().xl_rs_propagate_save(u.data_ptr(), _dev(out, "out").data_ptr(),
                                           _dev(saved, "saved").data_ptr(), B, ctypes.byref(g),
                                           float(wavelength), zz.ptr, zz.flags, _dtype(u),
                                           _stream()))
        return out
    _check(load().xl_rs_propagate(u.data_ptr(), _dev(out, "out").data_ptr(), B, ctypes.byref(g),
                                  float(wavelength), zz.ptr, zz.flags, _dtype(u), _stream()))
    return out


def save_buffer(field: torch.Tensor, comps: int = 1) -> torch.Tensor:
    """Buffer for the spectra a forward RS (comps 1) or VRS (comps 2) call saves for its
    adjoint: [B][comps][2nx][2ny] of the field's dtype."""
    B, ny, nx = _planes(field, comps, "field")
    return torch.empty((B, comps, 2 * nx, 2 * ny), dtype=field.dtype, device=field.device)


def rs_propagate_static(u: torch.Tensor, grid, wavelength: float, z,
                        out: torch.Tensor | None = None):
    """xl_rs_propagate_static: RS for complex64 grids up to 256 x 256 using the library's fixed
    static scratch (no device allocation by the library); host distances only."""
    _dev(u, "u")
    B, ny, nx = _planes(u, 1, "u")
    g = Grid.of(grid)
    if out is None:
        out = torch.empty_like(u)
    zz = _Z(z, B)
    if zz.flags:
        raise ValueError("rs_propagate_static takes host distances")
    _check(load().xl_rs_propagate_static(u.data_ptr(), _dev(out, "out").data_ptr(), B,
                                         ctypes.byref(g), float(wavelength), zz.ptr, _stream()))
    return out


def rs_propagate_backward(g_out: torch.Tensor, u_in: torch.Tensor | None, grid, wavelength: float,
                          z, want_field: bool = True, want_dz: bool = False,
                          phase_invariant: bool = False, saved: torch.Tensor | None = None):
    """Adjoint of rs_propagate: returns (g_in or None, g_z [B] float64 or None).
    phase_invariant: the loss ignores a constant phase on the output (XL_PHASE_INVARIANT).
    saved: the spectra a forward call saved; used in place of u_in."""
    _dev(g_out, "g_out")
    B, ny, nx = _planes(g_out, 1, "g_out")
    g = Grid.of(grid)
    g_in = torch.empty_like(g_out) if want_field else None
    g_z = torch.empty(B, dtype=torch.float64, device=g_out.device) if want_dz else None
    zz = _Z(z, B)
    fn = load().xl_rs_propagate_backward
    if saved is not None:
        fn, u_in = load().xl_rs_propagate_backward_saved, saved
    _check(fn(
        g_out.data_ptr(), _dev(u_in, "u_in").data_ptr() if u_in is not None else None,
        g_in.data_ptr() if g_in is not None else None, g_z.data_ptr() if g_z is not None else None,
        B, ctypes.byref(g), float(wavelength), zz.ptr,
        zz.flags | (PHASE_INVARIANT if phase_invariant else 0), _dtype(g_out), _stream()))
    return g_in, g_z


def vrs_propagate(exy: torch.Tensor, grid, wavelength: float, z, out: torch.Tensor | None = None,
                  saved: torch.Tensor | None = None):
    """Vectorial RS: [B][2][ny][nx] -> [B][3][ny][nx] (also [2][ny][nx] -> [3][ny][nx]).
    saved: optional [B][2][2nx][2ny] tensor for vrs_propagate_backward(..., saved=...)."""
    _dev(exy, "exy")
    B, ny, nx = _planes(exy, 2, "exy")
    g = Grid.of(grid)
    if out is None:
        shape = (3, ny, nx) if exy.dim() == 3 else (B, 3, ny, nx)
        out = torch.empty(shape, dtype=exy.dtype, device=exy.device)
    zz = _Z(z, B)
    if saved is not None:
        _check(load().xl_vrs_propagate_save(exy.data_ptr(), _dev(out, "out").data_ptr(),
                                            _dev(saved, "saved").data_ptr(), B, ctypes.byref(g),
                                            float(wavelength), zz.ptr, zz.flags, _dtype(exy),
                                            _stream()))
        return out
    _check(load().xl_vrs_propagate(exy.data_ptr(), _dev(out, "out").data_ptr(), B, ctypes.byref(g),
                                   float(wavelength), zz.ptr, zz.flags, _dtype(exy), _stream()))
    return out


def vrs_propagate_backward(g_exyz: torch.Tensor, exy_in: torch.Tensor | None, grid,
                           wavelength: float, z, want_field: bool = True, want_dz: bool = False,
                           phase_invariant: bool = False, saved: torch.Tensor | None = None):
    """Adjoint of vrs_propagate: returns (g_exy or None, g_z or None); saved as in
    rs_propagate_backward."""
    _dev(g_exyz, "g_exyz")
    B, ny, nx = _planes(g_exyz, 3, "g_exyz")
    g = Grid.of(grid)
    g_exy = None
    if want_field:
        shape = (2, ny, nx) if g_exyz.dim() == 3 else (B, 2, ny, nx)
        g_exy = torch.empty(shape, dtype=g_exyz.dtype, device=g_exyz.device)
    g_z = torch.empty(B, dtype=torch.float64, device=g_exyz.device) if want_dz else None
    zz = _Z(z, B)
    fn = load().xl_vrs_propagate_backward
    if saved is not None:
        fn, exy_in = load().xl_vrs_propagate_backward_saved, saved
    _check(fn(
        g_exyz.data_ptr(), _dev(exy_in, "exy_in").data_ptr() if exy_in is not None else None,
        g_exy.data_ptr() if g_exy is not None else None,
        g_z.data_ptr() if g_z is not None else None, B, ctypes.byref(g), float(wavelength),
        zz.ptr, zz.flags | (PHASE_INVARIANT if phase_invariant else 0), _dtype(g_exyz), _stream()))
    return g_exy, g_z


def czt_propagate(u: torch.Tensor, grid, window, wavelength: float, z, vectorial=False,
                  out: torch.Tensor | None = None, saved: torch.Tensor | None = None):
    """CZT onto a window: [B][ny][nx] -> [B][my][mx]; vectorial (1): [B][2][ny][nx] ->
    [B][3][my][mx]; vectorial 2: [B][3][ny][nx] (Ez unused) -> [B][3][my][mx].
    saved: optional buffer (czt_save_buffer) that receives what the adjoint's distance gradient
    needs (xl_czt_propagate_save)."""
    _dev(u, "u")
    vectorial = int(vectorial)
    comps = {0: 1, 1: 2, 2: 3}[vectorial]
    B, ny, nx = _planes(u, comps, "u")
    g, w = Grid.of(grid), Window.of(window)
    if out is None:
        lead = u.shape[:-2] if not vectorial else (u.shape[:-3] + (3,))
        out = torch.empty(tuple(lead) + (w.my, w.mx), dtype=u.dtype, device=u.device)
    zz = _Z(z, B)
    if saved is not None:
        _check(load().xl_czt_propagate_save(u.data_ptr(), _dev(out, "out").data_ptr(),
                                            _dev(saved, "saved").data_ptr(), B, int(vectorial),
                                            ctypes.byref(g), ctypes.byref(w), float(wavelength),
                                            zz.ptr, zz.flags, _dtype(u), _stream()))
        return out
    _check(load().xl_czt_propagate(u.data_ptr(), _dev(out, "out").data_ptr(), B, int(vectorial),
                                   ctypes.byref(g), ctypes.byref(w), float(wavelength), zz.ptr,
                                   zz.flags, _dtype(u), _stream()))
    return out


def czt_save_buffer(u: torch.Tensor, grid, window, vectorial=False) -> torch.Tensor:
    """Buffer for what a forward CZT saves for its adjoint's distance gradient:
    [B][xl_czt_save_elems] of the field's dtype."""
    vectorial = int(vectorial)
    comps = {0: 1, 1: 2, 2: 3}[vectorial]
    B, ny, nx = _planes(u, comps, "u")
    g, w = Grid.of(grid), Window.of(window)
    n = int(load().xl_czt_save_elems(ctypes.byref(g), ctypes.byref(w), vectorial, _dtype(u)))
    if n < 0:
        raise XLError(ERR_UNSUPPORTED, "czt_save_buffer: unsupported sizes")
    return torch.empty((B, n), dtype=u.dtype, device=u.device)


def czt_propagate_backward(g_out: torch.Tensor, grid, window, wavelength: float, z,
                           vectorial=False, u_in: torch.Tensor | None = None,
                           want_dz: bool = False, want_field: bool = True,
                           phase_invariant: bool = False, saved: torch.Tensor | None = None,
                           g_in: torch.Tensor | None = None, g_z: torch.Tensor | None = None,
                           accumulate: bool = False):
    """Adjoint of czt_propagate: window gradient -> input-grid gradient. With want_dz (needs
    u_in, the forward's input) returns (g_in or None, g_z [B] float64); otherwise g_in.
    saved: the buffer a czt_propagate(..., saved=...) call filled (else the sums are formed
    here, at the cost of one forward). g_in / g_z: output tensors to use; accumulate: add the
    results to them (XL_ACCUMULATE)."""
    _dev(g_out, "g_out")
    vectorial = int(vectorial)
    comps = 3 if vectorial else 1
    B, my, mx = _planes(g_out, comps, "g_out")
    g, w = Grid.of(grid), Window.of(window)
    lead = g_out.shape[:-2] if not vectorial else (g_out.shape[:-3] + ({1: 2, 2: 3}[vectorial],))
    if accumulate and ((want_field or not want_dz) and g_in is None or want_dz and g_z is None):
        raise ValueError("czt_propagate_backward: accumulate needs the output tensors")
    if (want_field or not want_dz) and g_in is None:
        g_in = torch.empty(tuple(lead) + (g.ny, g.nx), dtype=g_out.dtype, device=g_out.device)
    if not (want_field or not want_dz):
        g_in = None
    if want_dz and g_z is None:
        g_z = torch.empty(B, dtype=torch.float64, device=g_out.device)
    if not want_dz:
        g_z = None
    if want_dz and u_in is None:
        raise ValueError("czt_propagate_backward: want_dz needs u_in")
    zz = _Z(z, B)
    flags = zz.flags | (PHASE_INVARIANT if phase_invariant else 0) | (ACCUMULATE if accumulate else 0)
    uptr = _dev(u_in, "u_in").data_ptr() if u_in is not None else None
    gin_ptr = g_in.data_ptr() if g_in is not None else None
    gz_ptr = g_z.data_ptr() if g_z is not None else None
    if saved is not None:
        _check(load().xl_czt_propagate_backward_saved(
            g_out.data_ptr(), uptr, _dev(saved, "saved").data_ptr(), gin_ptr, gz_ptr, B,
            int(vectorial), ctypes.byref(g), ctypes.byref(w), float(wavelength), zz.ptr, flags,
            _dtype(g_out), _stream()))
    else:
        _check(load().xl_czt_propagate_backward(
            g_out.data_ptr(), uptr, gin_ptr, gz_ptr, B, int(vectorial), ctypes.byref(g),
            ctypes.byref(w), float(wavelength), zz.ptr, flags, _dtype(g_out), _stream()))
    return (g_in, g_z) if want_dz else g_in


# ----------------------------------------------------------------------------- elements
def _real_dtype(field: torch.Tensor):
    return torch.float32 if field.dtype == torch.complex64 else torch.float64


def _elements(elements: Sequence[dict], field: torch.Tensor, batch: int, ny: int, nx: int):
    """ctypes array of xl_element from dicts {kind, phi_x, phi_y, f, alpha, eta, theta}.
    Masks are CUDA real tensors [ny][nx] (shared by the batch) or [B][ny][nx]."""
    n = len(elements)
    arr = (Element * max(n, 1))()
    keep = []
    rd = _real_dtype(field)
    for i, e in enumerate(elements):
        arr[i].kind = int(e["kind"])
        stride = None
        for key in ("phi_x", "phi_y"):
            ph = e.get(key)
            if ph is None:
                continue
            if not isinstance(ph, torch.Tensor) or not ph.is_cuda or ph.dtype != rd or not ph.is_contiguous():
                raise ValueError(f"element {i}: {key} must be a contiguous CUDA {rd} tensor")
            if ph.shape[-2:] != (ny, nx) or ph.dim() not in (2, 3):
                raise ValueError(f"element {i}: {key} must be [ny][nx] or [B][ny][nx]")
            st = 0 if ph.dim() == 2 else ny * nx
            if ph.dim() == 3 and ph.shape[0] != batch:
                raise ValueError(f"element {i}: {key} batch mismatch")
            stride = st if stride is None else stride
            setattr(arr[i], key, ph.data_ptr())
            keep.append(ph)
        arr[i].phi_stride = stride or 0
        for key in ("f", "alpha", "eta", "theta"):
            v = e.get(key, 0.0)
            setattr(arr[i], key, float(v) if not isinstance(v, torch.Tensor) else 0.0)
    return arr, keep


def _params(params, batch: int, n: int):
    """Device parameters [B][n][4] (float64 CUDA) or None for host values."""
    if params is None:
        return None, 0
    if (not isinstance(params, torch.Tensor) or not params.is_cuda or params.dtype != torch.float64
            or params.numel() != batch * n * 4 or not params.is_contiguous()):
        raise ValueError("params must be a contiguous CUDA float64 tensor [B][n_elem][4]")
    return params.data_ptr(), Z_DEVICE


def _comps_out(comps_in: int, elements) -> int:
    return 2 if any(int(e["kind"]) == TO_VECTOR for e in elements) else comps_in


def apply_elements(field: torch.Tensor, grid, wavelength: float, elements: Sequence[dict],
                   comps_in: int = 1, params: torch.Tensor | None = None,
                   out: torch.Tensor | None = None):
    """field [B][comps_in][ny][nx] -> [B][comps_out][ny][nx] through the element chain."""
    _dev(field, "field")
    B, C, ny, nx = field.shape
    assert C == comps_in
    g = Grid.of(grid)
    arr, keep = _elements(elements, field, B, ny, nx)
    pp, flags = _params(params, B, len(elements))
    co = _comps_out(comps_in, elements)
    if out is None:
        out = torch.empty((B, co, ny, nx), dtype=field.dtype, device=field.device)
    _check(load().xl_apply_elements(field.data_ptr(), _dev(out, "out").data_ptr(), B, comps_in,
                                    ctypes.byref(g), float(wavelength), arr, len(elements), pp,
                                    flags, _dtype(field), _stream()))
    return out


def apply_elements_backward(g_out: torch.Tensor, field: torch.Tensor, grid, wavelength: float,
                            elements: Sequence[dict], comps_in: int = 1,
                            params: torch.Tensor | None = None, want_field: bool = True,
                            want_phi: bool = True, want_params: bool = True):
    """Adjoint of apply_elements at the forward input `field`. Returns (g_in, g_phi_x list,
    g_phi_y list, g_params [B][n][4])."""
    _dev(g_out, "g_out")
    _dev(field, "field")
    B, C, ny, nx = field.shape
    g = Grid.of(grid)
    arr, keep = _elements(elements, field, B, ny, nx)
    pp, flags = _params(params, B, len(elements))
    n = len(elements)
    g_in = torch.empty_like(field) if want_field else None
    gpx, gpy = [], []
    cpx = (ctypes.c_void_p * max(n, 1))()
    cpy = (ctypes.c_void_p * max(n, 1))()
    for i, e in enumerate(elements):
        for key, lst, carr in (("phi_x", gpx, cpx), ("phi_y", gpy, cpy)):
            ph = e.get(key)
            if ph is not None and want_phi:
                t = torch.empty_like(ph)
                lst.append(t)
                carr[i] = t.data_ptr()
            else:
                lst.append(None)
    g_params = torch.empty((B, n, 4), dtype=torch.float64, device=field.device) if want_params and n else None
    _check(load().xl_apply_elements_backward(
        g_out.data_ptr(), field.data_ptr(), g_in.data_ptr() if g_in is not None else None, B,
        comps_in, ctypes.byref(g), float(wavelength), arr, n, pp, flags, cpx, cpy,
        g_params.data_ptr() if g_params is not None else None, _dtype(field), _stream()))
    return g_in, gpx, gpy, g_params


# ----------------------------------------------------------------------------- losses
def intensity_loss(field: torch.Tensor, grid, comp_mask: int, mode: int = SECOND_MOMENT,
                   eps: float = 0.5, want_intensity: bool = False):
    """field [B][C][ny][nx] -> (loss [B] float64, intensity [B][ny][nx] or None)."""
    _dev(field, "field")
    B, C, ny, nx = field.shape
    g = Grid.of(grid)
    loss = torch.empty(B, dtype=torch.float64, device=field.device)
    inten = torch.empty((B, ny, nx), dtype=_real_dtype(field), device=field.device) if want_intensity else None
    _check(load().xl_intensity_loss(field.data_ptr(), B, C, comp_mask, ctypes.byref(g), mode,
                                    float(eps), loss.data_ptr(),
                                    inten.data_ptr() if inten is not None else None,
                                    _dtype(field), _stream()))
    return loss, inten


def intensity_loss_backward(field: torch.Tensor, grid, comp_mask: int, mode: int = SECOND_MOMENT,
                            eps: float = 0.5, g_loss: torch.Tensor | None = None,
                            out: torch.Tensor | None = None):
    """dL/dE (torch convention) of intensity_loss; g_loss [B] float64 CUDA or None (= 1)."""
    _dev(field, "field")
    B, C, ny, nx = field.shape
    g = Grid.of(grid)
    if out is None:
        out = torch.empty_like(field)
    if g_loss is not None:
        g_loss = _dev(g_loss.to(torch.float64), "g_loss")
    _check(load().xl_intensity_loss_backward(field.data_ptr(), B, C, comp_mask, ctypes.byref(g),
                                             mode, float(eps),
                                             g_loss.data_ptr() if g_loss is not None else None,
                                             out.data_ptr(), _dtype(field), _stream()))
    return out


def intensity_loss_and_grad(field: torch.Tensor, grid, comp_mask: int, mode: int = SECOND_MOMENT,
                            eps: float = 0.5, out: torch.Tensor | None = None,
                            loss: torch.Tensor | None = None):
    """(loss [B] float64, dL/dE) of intensity_loss in one call (xl_intensity_loss_and_grad)."""
    _dev(field, "field")
    B, C, ny, nx = field.shape
    g = Grid.of(grid)
    if loss is None:
        loss = torch.empty(B, dtype=torch.float64, device=field.device)
    if out is None:
        out = torch.empty_like(field)
    _check(load().xl_intensity_loss_and_grad(field.data_ptr(), None, None, B, C, comp_mask,
                                             ctypes.byref(g), mode, float(eps), 0.0,
                                             _dev(loss, "loss").data_ptr(),
                                             _dev(out, "out").data_ptr(), None, _dtype(field),
                                             _stream()))
    return loss, out


def intensity_loss_ex(field: torch.Tensor, grid, comp_mask: int, mode: int = SECOND_MOMENT,
                      eps: float = 0.5, field_dep: torch.Tensor | None = None, beta: float = 1.0,
                      target: torch.Tensor | None = None, want_intensity: bool = False):
    """Camera loss of |E|^2, of the STED effective intensity (field_dep given) or the MSE to a
    target intensity (mode MSE). Returns (loss [B], intensity or None)."""
    _dev(field, "field")
    B, C, ny, nx = field.shape
    g = Grid.of(grid)
    loss = torch.empty(B, dtype=torch.float64, device=field.device)
    inten = torch.empty((B, ny, nx), dtype=_real_dtype(field), device=field.device) if want_intensity else None
    _check(load().xl_intensity_loss_ex(
        field.data_ptr(), _dev(field_dep, "field_dep").data_ptr() if field_dep is not None else None,
        _dev(target, "target").data_ptr() if target is not None else None, B, C, comp_mask,
        ctypes.byref(g), mode, float(eps), float(beta), loss.data_ptr(),
        inten.data_ptr() if inten is not None else None, _dtype(field), _stream()))
    return loss, inten


def intensity_loss_ex_backward(field: torch.Tensor, grid, comp_mask: int, mode: int = SECOND_MOMENT,
                               eps: float = 0.5, field_dep: torch.Tensor | None = None,
                               beta: float = 1.0, target: torch.Tensor | None = None,
                               g_loss: torch.Tensor | None = None):
    """Returns (g_field, g_field_dep or None)."""
    _dev(field, "field")
    B, C, ny, nx = field.shape
    g = Grid.of(grid)
    gf = torch.empty_like(field)
    gd = torch.empty_like(field_dep) if field_dep is not None else None
    _check(load().xl_intensity_loss_ex_backward(
        field.data_ptr(), field_dep.data_ptr() if field_dep is not None else None,
        _dev(target, "target").data_ptr() if target is not None else None, B, C, comp_mask,
        ctypes.byref(g), mode, float(eps), float(beta),
        _dev(g_loss, "g_loss").data_ptr() if g_loss is not None else None, gf.data_ptr(),
        gd.data_ptr() if gd is not None else None, _dtype(field), _stream()))
    return gf, gd


def softmin(losses: torch.Tensor, beta: float, want_weights: bool = True):
    """losses [B][n_det] float64 CUDA -> (softmin [B], weights [B][n_det] or None)."""
    _dev(losses, "losses")
    B, n = losses.shape
    out = torch.empty(B, dtype=torch.float64, device=losses.device)
    w = torch.empty_like(losses) if want_weights else None
    _check(load().xl_softmin(losses.data_ptr(), B, n, float(beta), out.data_ptr(),
                             w.data_ptr() if w is not None else None, _stream()))
    return out, w


def device_status() -> None:
    """Raises XLError(ERR_NONFINITE) if a loss became non-finite since the last check."""
    _check(load().xl_device_status(_stream()))


# ----------------------------------------------------------------------------- angular-spectrum CZT
def asczt_propagate(u: torch.Tensor, grid, window, wavelength: float, z,
                    out: torch.Tensor | None = None):
    """Angular-spectrum CZT: [B][ny][nx] (or [ny][nx]) -> [B][my][mx] on the window."""
    _dev(u, "u")
    B, ny, nx = _planes(u, 1, "u")
    g, w = Grid.of(grid), Window.of(window)
    if out is None:
        shape = (w.my, w.mx) if u.dim() == 2 else (B, w.my, w.mx)
        out = torch.empty(shape, dtype=u.dtype, device=u.device)
    zz = _Z(z, B)
    _check(load().xl_asczt_propagate(u.data_ptr(), _dev(out, "out").data_ptr(), B, ctypes.byref(g),
                                     ctypes.byref(w), float(wavelength), zz.ptr, zz.flags,
                                     _dtype(u), _stream()))
    return out


def asczt_propagate_backward(g_out: torch.Tensor, u_in: torch.Tensor | None, grid, window,
                             wavelength: float, z, want_field: bool = True, want_dz: bool = False):
    """Adjoint of asczt_propagate: returns (g_in [B][ny][nx] or None, g_z [B] or None)."""
    _dev(g_out, "g_out")
    g, w = Grid.of(grid), Window.of(window)
    B = g_out.shape[0] if g_out.dim() == 3 else 1
    g_in = None
    if want_field:
        shape = (g.ny, g.nx) if g_out.dim() == 2 else (B, g.ny, g.nx)
        g_in = torch.empty(shape, dtype=g_out.dtype, device=g_out.device)
    g_z = torch.empty(B, dtype=torch.float64, device=g_out.device) if want_dz else None
    zz = _Z(z, B)
    _check(load().xl_asczt_propagate_backward(
        g_out.data_ptr(), _dev(u_in, "u_in").data_ptr() if u_in is not None else None,
        g_in.data_ptr() if g_in is not None else None, g_z.data_ptr() if g_z is not None else None,
        B, ctypes.byref(g), ctypes.byref(w), float(wavelength), zz.ptr, zz.flags, _dtype(g_out),
        _stream()))
    return g_in, g_z


# ----------------------------------------------------------------------------- autotuner
TUNE_RS_PASS1, TUNE_RS_PASS3, TUNE_CZT_FWD_X, TUNE_CZT_FWD_Y, TUNE_CZT_ADJ_X, TUNE_CZT_ADJ_Y = range(6)


def autotune(grid, window=None, dtype: int = C64, reps: int = 5) -> None:
    """Times the launch variants of the passes `grid` (and a CZT onto `window`) uses and keeps
    the fastest for this process (xl_autotune)."""
    g = Grid.of(grid)
    w = Window.of(window) if window is not None else None
    _check(load().xl_autotune(ctypes.byref(g), ctypes.byref(w) if w is not None else None,
                              int(dtype), int(reps), _stream()))


def tune_get(family: int, L: int, dtype: int = C64) -> int:
    return int(load().xl_tune_get(int(family), int(L), int(dtype)))


def tune_set(family: int, L: int, dtype: int, variant: int) -> None:
    _check(load().xl_tune_set(int(family), int(L), int(dtype), int(variant)))


def tune_clear() -> None:
    _check(load().xl_tune_clear())


def tune_save(path: str) -> None:
    _check(load().xl_tune_save(os.fsencode(path)))


def tune_load(path: str) -> None:
    _check(load().xl_tune_load(os.fsencode(path)))


# ----------------------------------------------------------------------------- beam splitters
def _ptr_or_none(t, name):
    return _dev(t, name).data_ptr() if t is not None else None


def beam_splitter(a: torch.Tensor | None, b: torch.Tensor | None, R: torch.Tensor,
                  out_t: torch.Tensor | None = None, out_r: torch.Tensor | None = None):
    """Lossless beam splitter of reflectance R [B] (float64 CUDA): returns (out_t, out_r) =
    (t a + i r b, i r a + t b) for fields [B][...] (a or b None: a zero input)."""
    ref = a if a is not None else b
    if ref is None:
        raise ValueError("beam_splitter needs at least one input")
    B = ref.shape[0]
    elems = ref[0].numel()
    out_t = torch.empty_like(ref) if out_t is None else out_t
    out_r = torch.empty_like(ref) if out_r is None else out_r
    _check(load().xl_beam_splitter(_ptr_or_none(a, "a"), _ptr_or_none(b, "b"),
                                   _dev(out_t, "out_t").data_ptr(), _dev(out_r, "out_r").data_ptr(),
                                   B, elems, _dev(R, "R").data_ptr(), _dtype(ref), _stream()))
    return out_t, out_r


def beam_splitter_backward(g_t, g_r, a, b, R: torch.Tensor, want_a: bool = True,
                           want_b: bool = True, want_R: bool = True):
    """Adjoint of beam_splitter: returns (g_a or None, g_b or None, g_R [B] float64 or None)."""
    ref = next(x for x in (g_t, g_r, a, b) if x is not None)
    B = ref.shape[0]
    elems = ref[0].numel()
    g_a = torch.empty_like(ref) if want_a else None
    g_b = torch.empty_like(ref) if want_b else None
    g_R = torch.empty(B, dtype=torch.float64, device=ref.device) if want_R else None
    _check(load().xl_beam_splitter_backward(
        _ptr_or_none(g_t, "g_t"), _ptr_or_none(g_r, "g_r"), _ptr_or_none(a, "a"),
        _ptr_or_none(b, "b"), g_a.data_ptr() if g_a is not None else None,
        g_b.data_ptr() if g_b is not None else None, g_R.data_ptr() if g_R is not None else None,
        B, elems, _dev(R, "R").data_ptr(), _dtype(ref), _stream()))
    return g_a, g_b, g_R


# ----------------------------------------------------------------------------- Adam
def adam_step(p: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, lr: float,
              t, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
    """In-place Adam step on float32 / float64 CUDA tensors. t: int step (>= 1) or a CUDA int32
    tensor holding it (read at run time)."""
    for name, a in (("p", p), ("m", m), ("v", v), ("grad", grad)):
        _dev(a, name)
        if a.dtype != p.dtype or a.numel() != p.numel():
            raise ValueError(f"{name} must match p in dtype and size")
    rd = {torch.float32: 0, torch.float64: 1}[p.dtype]
    if isinstance(t, torch.Tensor):
        t_dev, t_host = _dev(t, "t").data_ptr(), 0
    else:
        t_dev, t_host = None, int(t)
    _check(load().xl_adam_step(p.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(), p.numel(),
                               rd, float(lr), float(beta1), float(beta2), float(eps), t_dev, t_host,
                               _stream()))


def adamw_step(p: torch.Tensor, m: torch.Tensor, v: torch.Tensor, grad: torch.Tensor, lr: float,
               t, weight_decay: float, beta1: float = 0.9, beta2: float = 0.999,
               eps: float = 1e-8) -> None:
    """In-place AdamW step (decoupled weight decay)."""
    for name, a in (("p", p), ("m", m), ("v", v), ("grad", grad)):
        _dev(a, name)
    rd = {torch.float32: 0, torch.float64: 1}[p.dtype]
    t_dev, t_host = (t.data_ptr(), 0) if isinstance(t, torch.Tensor) else (None, int(t))
    _check(load().xl_adamw_step(p.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(),
                                p.numel(), rd, float(lr), float(beta1), float(beta2), float(eps),
                                float(weight_decay), t_dev, t_host, _stream()))


def step_advance(t: torch.Tensor) -> None:
    _check(load().xl_step_advance(_dev(t, "t").data_ptr(), _stream()))


# ----------------------------------------------------------------------------- batched tables
def table_config(cfg: dict) -> TableConfig:
    """The xl_table_config of a Batch configuration dict (see Batch)."""
    return TableConfig(float(cfg["wavelength"]), float(cfg["extent"]), float(cfg["w0"]),
                       float(cfg["f"]), float(cfg["cam_width"]), float(cfg["lr"]),
                       float(cfg["lr_z"]), int(cfg["cam_m"]),
                       C128 if cfg.get("dtype", "c64") == "c128" else C64,
                       int(cfg.get("checkpoint", 0)), int(cfg.get("memory_budget", 0)))


def batch_plan_memory(cfg: dict, grid_n) -> tuple:
    """(bytes, checkpoint mode) that a Batch of these setups allocates (xl_batch_plan_memory:
    host arithmetic, no device call)."""
    c = table_config(cfg)
    gn = np.ascontiguousarray(grid_n, dtype=np.int32)
    mode = ctypes.c_int32(-1)
    nb = int(load().xl_batch_plan_memory(ctypes.byref(c), len(gn), gn.ctypes.data, ctypes.byref(mode)))
    if nb < 0:
        raise XLError(ERR_ARG, "xl_batch_plan_memory: invalid configuration")
    return nb, int(mode.value)


class Batch:
    """Many optical-table setups optimised together (xl_batch_*). cfg: dict with wavelength,
    extent, w0, f, cam_m, cam_width, lr, lr_z, dtype ("c64" / "c128"), checkpoint (0: the RS /
    VRS adjoints read spectra the forwards keep; 1: only the plane fields are kept and the
    adjoints transform their inputs again; CHECKPOINT_AUTO: 0 if it fits in memory_budget),
    memory_budget (bytes, 0 = no limit); grid_n: list of N per setup; init: [n][3] =
    (theta, z1, z2)."""

    def __init__(self, cfg: dict, grid_n, init, seed: int):
        self.cfg = table_config(cfg)
        self.n = len(grid_n)
        gn = np.ascontiguousarray(grid_n, dtype=np.int32)
        ini = np.ascontiguousarray(init, dtype=np.float64).reshape(self.n, 3)
        h = ctypes.c_void_p()
        _check(load().xl_batch_create(ctypes.byref(self.cfg), self.n, gn.ctypes.data,
                                      ini.ctypes.data, int(seed) & (2 ** 64 - 1), ctypes.byref(h),
                                      _stream()))
        self.h = h

    def step(self, use_graph: bool = True) -> None:
        _check(load().xl_batch_step(self.h, int(use_graph), _stream()))

    def grid(self, setup: int) -> int:
        return int(load().xl_batch_grid(self.h, setup))

    def memory(self) -> int:
        """Device bytes the batch's own buffers hold."""
        return int(load().xl_batch_memory(self.h))

    def read(self, what: int, setup: int) -> np.ndarray:
        n = self.grid(setup)
        rd = np.float64 if self.cfg.dtype == C128 else np.float32
        if what == BATCH_LOSS:
            out = np.zeros(1)
        elif what in (BATCH_SCALARS, BATCH_GRAD_SCALARS):
            out = np.zeros(3)
        else:
            out = np.zeros((n, n), rd)
        _check(load().xl_batch_read(self.h, what, setup, out.ctypes.data, _stream()))
        return out

    def close(self) -> None:
        if getattr(self, "h", None):
            _check(load().xl_batch_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
