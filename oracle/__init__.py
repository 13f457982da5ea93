"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. It is a plain, slow, double-precision restatement of what the GPU library
computes, written from the paper's description of the method (XLuminA, arXiv 2310.08408,
Methods, "Features and performance": RS / VRS / CZT / VCZT propagation, SLM and super-SLM
phase masks, polarisers, wave plates, lenses; "Loss function"; "Stimulated emission depletion
model"; Adam). It shares no code with the CUDA path. The C++ source is ``xl_oracle.cpp``;
``build()`` compiles it with g++ into ``oracle/_build/liboracle.so``.

Every function takes and returns numpy arrays: complex128 fields laid out [..., ny, nx] and
float64 masks. Each pinned function is checked by ``tests/test_oracle_*.py`` against brute
force, closed forms, invariants or finite differences (see the docstrings there).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xl_oracle.cpp")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

SLM, SSLM, LENS, POLARIZER, WAVEPLATE, TO_VECTOR = range(6)
K_H, K_HX, K_HY, K_DH, K_DHX, K_DHY = range(6)
SECOND_MOMENT, DENSITY = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle (plain -O2, no fast-math) if missing or older than its source."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _sig(_lib)
    return _lib


_D = ctypes.c_double
_I64 = ctypes.c_int64
_I32 = ctypes.c_int
_P = ctypes.c_void_p


def _sig(lib):
    lib.orc_set_threads.argtypes = [_I32]
    lib.orc_get_threads.restype = _I32
    lib.orc_fft.argtypes = [_P, _I64, _I32]
    lib.orc_fft2.argtypes = [_P, _I64, _I64, _I32]
    lib.orc_dft.argtypes = [_P, _P, _I64, _I32]
    lib.orc_rs_kernel_table.argtypes = [_I32, _I64, _I64, _D, _D, _D, _D, _P]
    for f in (lib.orc_rs_fft, lib.orc_rs_direct):
        f.argtypes = [_P, _P, _I64, _I64, _D, _D, _D, _D, _I32, _I32]
    lib.orc_rs_direct_points.argtypes = [_P, _I64, _I64, _D, _D, _D, _D, _I32, _I32, _P, _I64, _P]
    lib.orc_czt_direct.argtypes = [_P, _P, _I64, _I64, _D, _D, _D, _D, _I64, _I64, _D, _D, _D, _D,
                                   _D, _D, _I32, _I32]
    lib.orc_czt_brute.argtypes = [_P, _P, _I64, _I64, _D, _D, _D, _D, _I64, _I64, _D, _D, _D, _D,
                                  _D, _D, _I32]
    lib.orc_czt_points.argtypes = [_P, _I64, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _I32,
                                   _P, _I64, _P]
    lib.orc_elements_forward.argtypes = [_P, _P, _I32, _I64, _I64, _D, _D, _D, _D, _D, _I32, _P,
                                         _P, _P, _P]
    lib.orc_elements_backward.argtypes = [_P, _P, _P, _I32, _I64, _I64, _D, _D, _D, _D, _D, _I32,
                                          _P, _P, _P, _P, _P, _P, _P]
    lib.orc_intensity_loss.argtypes = [_P, _I32, ctypes.c_uint32, _I64, _I64, _D, _D, _D, _D, _I32,
                                       _D, _P, _P]
    lib.orc_intensity_loss_backward.argtypes = [_P, _I32, ctypes.c_uint32, _I64, _I64, _D, _D, _D,
                                                _D, _I32, _D, _D, _P]
    lib.orc_sted.argtypes = [_P, _P, _D, _I64, _P]
    lib.orc_adam.argtypes = [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _I64]
    lib.orc_loss_from_intensity.argtypes = [_P, _I64, _I64, _D, _D, _D, _D, _I32, _D, _P, _P]
    lib.orc_loss_from_intensity.restype = _I32
    lib.orc_sted_backward.argtypes = [_P, _P, _D, _P, _I64, _P, _P]
    lib.orc_softmin.argtypes = [_P, _I64, _I64, _D, _P, _P]
    lib.orc_adamw.argtypes = [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _D, _I64]
    lib.orc_mse.argtypes = [_P, _P, _I64, _P]
    lib.orc_mse.restype = _D
    lib.orc_beam_splitter.argtypes = [_P, _P, _I64, _D, _P, _P]
    lib.orc_asczt.argtypes = [_P, _P, _I64, _I64, _D, _D, _D, _D, _I64, _I64, _D, _D, _D, _D, _D,
                              _D, _I32, _I32]
    lib.orc_asczt.restype = _I32
    lib.orc_beam_splitter_backward.argtypes = [_P, _P, _P, _P, _I64, _D, _P, _P, _P]
    for name in ("orc_fft", "orc_fft2", "orc_rs_fft", "orc_rs_direct", "orc_rs_direct_points",
                 "orc_czt_direct", "orc_czt_brute", "orc_czt_points", "orc_elements_forward",
                 "orc_elements_backward", "orc_intensity_loss", "orc_intensity_loss_backward"):
        getattr(lib, name).restype = _I32


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid arguments")


def set_threads(n: int) -> None:
    """Number of host threads the oracle uses (0 = all hardware threads)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


# ---------------------------------------------------------------- transforms
def fft(x, sign=-1):
    """Unnormalised 1D DFT (own radix-2 FFT), exp(sign 2 pi i j k / n)."""
    a = _c(x, np.complex128).copy()
    _check(_load().orc_fft(_ptr(a), a.size, sign), "fft")
    return a


def fft2(x, sign=-1):
    a = _c(x, np.complex128).copy()
    _check(_load().orc_fft2(_ptr(a), a.shape[0], a.shape[1], sign), "fft2")
    return a


def dft(x, sign=-1):
    """Direct O(n^2) DFT."""
    a = _c(x, np.complex128)
    y = np.empty_like(a)
    _load().orc_dft(_ptr(a), _ptr(y), a.size, sign)
    return y


# ---------------------------------------------------------------- Rayleigh-Sommerfeld
def rs_kernel_table(kind, nx, ny, dx, dy, wavelength, z):
    out = np.empty((2 * ny - 1, 2 * nx - 1), np.complex128)
    _load().orc_rs_kernel_table(kind, nx, ny, dx, dy, wavelength, z, _ptr(out))
    return out


def rs_conv(u, dx, dy, wavelength, z, kind=K_H, adjoint=False, method="fft"):
    """Discrete RS convolution u_out[q,p] = sum u[n,m] K[p-m, q-n] of one [ny, nx] plane."""
    u = _c(u, np.complex128)
    ny, nx = u.shape
    out = np.empty_like(u)
    fn = _load().orc_rs_fft if method == "fft" else _load().orc_rs_direct
    _check(fn(_ptr(u), _ptr(out), nx, ny, dx, dy, wavelength, z, kind, int(adjoint)), "rs")
    return out


def rs_points(u, dx, dy, wavelength, z, pts, kind=K_H, adjoint=False):
    """Direct RS sum at output pixels pts = [(p, q), ...] (p along x)."""
    u = _c(u, np.complex128)
    ny, nx = u.shape
    pts = _c(pts, np.int32).reshape(-1, 2)
    out = np.empty(len(pts), np.complex128)
    _check(_load().orc_rs_direct_points(_ptr(u), nx, ny, dx, dy, wavelength, z, kind,
                                        int(adjoint), _ptr(pts), len(pts), _ptr(out)), "rs_points")
    return out


def rs(u, dx, dy, wavelength, z, method="fft"):
    """Scalar RS propagation of [..., ny, nx] planes."""
    u = np.asarray(u, np.complex128)
    flat = u.reshape(-1, *u.shape[-2:])
    return np.stack([rs_conv(p, dx, dy, wavelength, z, K_H, False, method) for p in flat]
                    ).reshape(u.shape)


def vrs(exy, dx, dy, wavelength, z, method="fft"):
    """Vectorial RS: exy [2, ny, nx] -> [3, ny, nx] (Ex', Ey', Ez')."""
    ex, ey = np.asarray(exy, np.complex128)
    exo = rs_conv(ex, dx, dy, wavelength, z, K_H, False, method)
    eyo = rs_conv(ey, dx, dy, wavelength, z, K_H, False, method)
    ezo = (rs_conv(ex, dx, dy, wavelength, z, K_HX, False, method)
           + rs_conv(ey, dx, dy, wavelength, z, K_HY, False, method))
    return np.stack([exo, eyo, ezo])


def vrs_adjoint(g, dx, dy, wavelength, z, method="fft"):
    """Adjoint of vrs: g [3, ny, nx] -> [2, ny, nx]."""
    gx, gy, gz = np.asarray(g, np.complex128)
    ax = (rs_conv(gx, dx, dy, wavelength, z, K_H, True, method)
          + rs_conv(gz, dx, dy, wavelength, z, K_HX, True, method))
    ay = (rs_conv(gy, dx, dy, wavelength, z, K_H, True, method)
          + rs_conv(gz, dx, dy, wavelength, z, K_HY, True, method))
    return np.stack([ax, ay])


def vrs_dz(exy, dx, dy, wavelength, z):
    """d/dz of vrs(exy) at fixed input."""
    ex, ey = np.asarray(exy, np.complex128)
    return np.stack([rs_conv(ex, dx, dy, wavelength, z, K_DH),
                     rs_conv(ey, dx, dy, wavelength, z, K_DH),
                     rs_conv(ex, dx, dy, wavelength, z, K_DHX)
                     + rs_conv(ey, dx, dy, wavelength, z, K_DHY)])


# ---------------------------------------------------------------- chirped z-transform
def _cz_args(grid, window):
    nx, ny, dx, dy, x0, y0 = grid
    mx, my, dxo, dyo, xo0, yo0 = window
    return nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo, xo0, yo0


def czt_conv(u, grid, window, wavelength, z, kind=0, adjoint=False, method="direct"):
    """CZT sum of one plane. grid = (nx, ny, dx, dy, x0, y0); window = (mx, my, dxo, dyo,
    xo0, yo0). Forward: [ny, nx] -> [my, mx]; adjoint: [my, mx] -> [ny, nx]."""
    nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo, xo0, yo0 = _cz_args(grid, window)
    u = _c(u, np.complex128)
    if method == "brute":
        assert not adjoint
        out = np.empty((my, mx), np.complex128)
        _check(_load().orc_czt_brute(_ptr(u), _ptr(out), nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo,
                                     xo0, yo0, wavelength, z, kind), "czt_brute")
        return out
    out = np.empty((ny, nx) if adjoint else (my, mx), np.complex128)
    _check(_load().orc_czt_direct(_ptr(u), _ptr(out), nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo,
                                  xo0, yo0, wavelength, z, kind, int(adjoint)), "czt")
    return out


def czt_points(u, grid, window, wavelength, z, pts, kind=0):
    nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo, xo0, yo0 = _cz_args(grid, window)
    u = _c(u, np.complex128)
    pts = _c(pts, np.int32).reshape(-1, 2)
    out = np.empty(len(pts), np.complex128)
    _check(_load().orc_czt_points(_ptr(u), nx, ny, dx, dy, x0, y0, dxo, dyo, xo0, yo0, wavelength,
                                  z, kind, _ptr(pts), len(pts), _ptr(out)), "czt_points")
    return out


def czt(u, grid, window, wavelength, z):
    u = np.asarray(u, np.complex128)
    flat = u.reshape(-1, *u.shape[-2:])
    out = [czt_conv(p, grid, window, wavelength, z) for p in flat]
    return np.stack(out).reshape(*u.shape[:-2], window[1], window[0])


def vczt(exy, grid, window, wavelength, z):
    """Vectorial CZT: [2, ny, nx] -> [3, my, mx]."""
    ex, ey = np.asarray(exy, np.complex128)
    return np.stack([czt_conv(ex, grid, window, wavelength, z, 0),
                     czt_conv(ey, grid, window, wavelength, z, 0),
                     czt_conv(ex, grid, window, wavelength, z, 1)
                     + czt_conv(ey, grid, window, wavelength, z, 2)])


def vczt_adjoint(g, grid, window, wavelength, z):
    gx, gy, gz = np.asarray(g, np.complex128)
    c = lambda a, kd: czt_conv(a, grid, window, wavelength, z, kd, adjoint=True)
    return np.stack([c(gx, 0) + c(gz, 1), c(gy, 0) + c(gz, 2)])


def vczt_dz(exy, grid, window, wavelength, z):
    ex, ey = np.asarray(exy, np.complex128)
    c = lambda a, kd: czt_conv(a, grid, window, wavelength, z, kd)
    return np.stack([c(ex, 3), c(ey, 3), c(ex, 4) + c(ey, 5)])


# ---------------------------------------------------------------- elements
def _elem_arrays(elements, ny, nx):
    n = len(elements)
    kinds = np.array([e["kind"] for e in elements], np.int32)
    params = np.zeros((max(n, 1), 4), np.float64)
    keep = []
    px = (ctypes.c_void_p * max(n, 1))()
    py = (ctypes.c_void_p * max(n, 1))()
    for i, e in enumerate(elements):
        params[i] = [e.get("f", 0.0), e.get("alpha", 0.0), e.get("eta", 0.0), e.get("theta", 0.0)]
        for key, arr in (("phi_x", px), ("phi_y", py)):
            if e.get(key) is not None:
                a = _c(e[key], np.float64).reshape(ny, nx)
                keep.append(a)
                arr[i] = a.ctypes.data
    return kinds, params, px, py, keep


def apply_elements(field, grid, wavelength, elements):
    """field [C, ny, nx] (C = 1 or 2); elements = list of dicts with 'kind' and the fields
    f, alpha, eta, theta, phi_x, phi_y as needed. Returns [C_out, ny, nx]."""
    nx, ny, dx, dy, x0, y0 = grid
    f = _c(field, np.complex128).reshape(-1, ny, nx)
    kinds, params, px, py, keep = _elem_arrays(elements, ny, nx)
    co = 2 if (f.shape[0] == 2 or TO_VECTOR in kinds.tolist()) else 1
    out = np.empty((co, ny, nx), np.complex128)
    _check(_load().orc_elements_forward(_ptr(f), _ptr(out), f.shape[0], nx, ny, dx, dy, x0, y0,
                                        wavelength, len(elements), _ptr(kinds), _ptr(params), px,
                                        py), "elements")
    return out


def apply_elements_backward(g_out, field, grid, wavelength, elements):
    """Returns (g_in [C, ny, nx], g_phi_x list, g_phi_y list, g_params [n_el, 4])."""
    nx, ny, dx, dy, x0, y0 = grid
    f = _c(field, np.complex128).reshape(-1, ny, nx)
    kinds, params, px, py, keep = _elem_arrays(elements, ny, nx)
    g = _c(g_out, np.complex128)
    n = len(elements)
    gpx = [np.zeros((ny, nx)) if e.get("phi_x") is not None else None for e in elements]
    gpy = [np.zeros((ny, nx)) if e.get("phi_y") is not None else None for e in elements]
    cpx = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data if a is not None else None for a in gpx])
    cpy = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data if a is not None else None for a in gpy])
    gp = np.zeros((max(n, 1), 4))
    g_in = np.empty_like(f)
    _check(_load().orc_elements_backward(_ptr(g), _ptr(f), _ptr(g_in), f.shape[0], nx, ny, dx, dy,
                                         x0, y0, wavelength, n, _ptr(kinds), _ptr(params), px, py,
                                         cpx, cpy, _ptr(gp)), "elements_backward")
    return g_in, gpx, gpy, gp[:n]


# ---------------------------------------------------------------- losses, STED, Adam
def intensity_loss(field, grid, comp_mask, mode=SECOND_MOMENT, eps=0.5):
    """Returns (loss, intensity [ny, nx])."""
    nx, ny, dx, dy, x0, y0 = grid
    f = _c(field, np.complex128).reshape(-1, ny, nx)
    loss = np.zeros(1)
    inten = np.empty((ny, nx))
    _check(_load().orc_intensity_loss(_ptr(f), f.shape[0], comp_mask, nx, ny, dx, dy, x0, y0, mode,
                                      eps, _ptr(loss), _ptr(inten)), "intensity_loss")
    return float(loss[0]), inten


def intensity_loss_backward(field, grid, comp_mask, mode=SECOND_MOMENT, eps=0.5, g_loss=1.0):
    nx, ny, dx, dy, x0, y0 = grid
    f = _c(field, np.complex128).reshape(-1, ny, nx)
    g = np.empty_like(f)
    _check(_load().orc_intensity_loss_backward(_ptr(f), f.shape[0], comp_mask, nx, ny, dx, dy, x0,
                                               y0, mode, eps, g_loss, _ptr(g)), "loss_backward")
    return g


def sted(i_ex, i_dep, beta):
    a = _c(i_ex, np.float64).ravel()
    b = _c(i_dep, np.float64).ravel()
    out = np.empty_like(a)
    _load().orc_sted(_ptr(a), _ptr(b), beta, a.size, _ptr(out))
    return out.reshape(np.shape(i_ex))


def adam(p, m, v, g, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on float64 arrays p, m, v with gradient g; t >= 1."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c(g, np.float64)
    _load().orc_adam(_ptr(p), _ptr(m), _ptr(v), _ptr(g), p.size, lr, b1, b2, eps, t)


def loss_from_intensity(I, grid, mode=SECOND_MOMENT, eps=0.5, want_grad=False):
    """Loss of an intensity image [ny, nx]; returns (loss, dL/dI or None)."""
    nx, ny, dx, dy, x0, y0 = grid
    I = _c(I, np.float64)
    loss = np.zeros(1)
    dI = np.empty_like(I) if want_grad else None
    _check(_load().orc_loss_from_intensity(_ptr(I), nx, ny, dx, dy, x0, y0, mode, eps, _ptr(loss),
                                           _ptr(dI)), "loss_from_intensity")
    return float(loss[0]), dI


def sted_backward(i_ex, i_dep, beta, g_eff):
    """(dL/dI_ex, dL/dI_dep) from dL/dI_eff."""
    a, b, g = (_c(x, np.float64).ravel() for x in (i_ex, i_dep, g_eff))
    ge, gd = np.empty_like(a), np.empty_like(a)
    _load().orc_sted_backward(_ptr(a), _ptr(b), beta, _ptr(g), a.size, _ptr(ge), _ptr(gd))
    sh = np.shape(i_ex)
    return ge.reshape(sh), gd.reshape(sh)


def softmin(losses, beta):
    """losses [batch, n_det] -> (softmin [batch], weights [batch, n_det])."""
    l = _c(np.atleast_2d(losses), np.float64)
    out = np.empty(l.shape[0])
    w = np.empty_like(l)
    _load().orc_softmin(_ptr(l), l.shape[0], l.shape[1], beta, _ptr(out), _ptr(w))
    return out, w


def adamw(p, m, v, g, lr, t, wd, b1=0.9, b2=0.999, eps=1e-8):
    """One AdamW step in place (float64 arrays)."""
    g = _c(g, np.float64)
    _load().orc_adamw(_ptr(p), _ptr(m), _ptr(v), _ptr(g), p.size, lr, b1, b2, eps, wd, t)


def mse(I, target, want_grad=False):
    I = _c(I, np.float64)
    t = _c(target, np.float64)
    dI = np.empty_like(I) if want_grad else None
    L = _load().orc_mse(_ptr(I), _ptr(t), I.size, _ptr(dI))
    return float(L), dI


def beam_splitter(a, b, R):
    """Lossless beam splitter of reflectance R: (out_t, out_r) = (t a + i r b, i r a + t b);
    a or b None is a zero input."""
    ref = a if a is not None else b
    a = _c(a, np.complex128).ravel() if a is not None else None
    b = _c(b, np.complex128).ravel() if b is not None else None
    n = (a if a is not None else b).size
    ot, orr = np.empty(n, np.complex128), np.empty(n, np.complex128)
    _load().orc_beam_splitter(_ptr(a), _ptr(b), n, float(R), _ptr(ot), _ptr(orr))
    sh = np.shape(ref)
    return ot.reshape(sh), orr.reshape(sh)


def beam_splitter_backward(g_t, g_r, a, b, R):
    """(g_a, g_b, dL/dR) of beam_splitter from the output gradients (None = zero)."""
    arrs = [_c(x, np.complex128).ravel() if x is not None else None for x in (g_t, g_r, a, b)]
    ref = next(x for x in (g_t, g_r, a, b) if x is not None)
    n = next(x for x in arrs if x is not None).size
    ga, gb = np.empty(n, np.complex128), np.empty(n, np.complex128)
    gR = np.zeros(1)
    _load().orc_beam_splitter_backward(*[_ptr(x) for x in arrs], n, float(R), _ptr(ga), _ptr(gb),
                                       _ptr(gR))
    sh = np.shape(ref)
    return ga.reshape(sh), gb.reshape(sh), float(gR[0])


AS_H, AS_DH = 0, 1


def asczt(u, grid, window, wavelength, z, kind=AS_H, adjoint=False):
    """Angular-spectrum CZT: u [ny][nx] -> [my][mx] on the window (adjoint: window -> grid).
    grid = (nx, ny, dx, dy, x0, y0), window = (mx, my, dxo, dyo, xo0, yo0); kind AS_DH gives the
    distance derivative of the forward map."""
    nx, ny, dx, dy, x0, y0 = grid
    mx, my, dxo, dyo, xo0, yo0 = window
    src = _c(u, np.complex128)
    shape = (ny, nx) if adjoint else (my, mx)
    out = np.empty(shape, np.complex128)
    st = _load().orc_asczt(_ptr(src), _ptr(out), nx, ny, dx, dy, x0, y0, mx, my, dxo, dyo, xo0, yo0,
                           wavelength, z, kind, int(bool(adjoint)))
    if st != 0:
        raise ValueError("orc_asczt: bad arguments")
    return out
