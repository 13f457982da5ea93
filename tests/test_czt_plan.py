"""Segment plans of the CZT window passes (host logic, no GPU): the size of the buffer a forward
with saved sums fills (xl_czt_save_elems) encodes each axis's transform length L, so it pins the
plan the library picks: among S = 1, 2, 4, ... segments of the grid side, the one with the least
(S + 1) L log2 L transform work, L = 2^ceil(log2(ceil(N / S) + M - 1))."""
import ctypes
import math

import pytest

from paper_2310_08408_gb300 import build, xl


def plan(N, M):
    best, cost = None, math.inf
    S = 1
    while S <= 64 and S <= N:
        seg = -(-N // S)
        if (S - 1) * seg < N:
            L = 64
            while L < seg + M - 1:
                L *= 2
            if L <= 8192:
                c = (S + 1) * L * math.log2(L) + 4 * S * L
                if c < cost * (1 - 1e-9):
                    best, cost = (L, S, seg), c
        S *= 2
    return best


def save_elems(nx, ny, mx, my, cT, Lx, Ly):
    return cT * (mx * ny + ny * Lx + mx * Ly + my * mx)


@pytest.mark.parametrize("nx,ny,mx,my", [(2048, 2048, 512, 512), (1024, 1024, 256, 256),
                                         (512, 512, 256, 256), (2048, 2048, 256, 256),
                                         (4096, 4096, 1024, 1024), (300, 256, 40, 64),
                                         (1000, 523, 100, 31), (96, 80, 90, 70)])
@pytest.mark.parametrize("vectorial", [0, 1])
def test_save_size_follows_the_least_work_plan(nx, ny, mx, my, vectorial):
    lib = xl.load(build.build())
    g = xl.Grid(nx, ny, 0.5, 0.5, 0.0, 0.0)
    w = xl.Window(mx, my, 0.1, 0.1, 0.0, 0.0)
    Lx, Sx, _ = plan(nx, mx)
    Ly, Sy, _ = plan(ny, my)
    got = lib.xl_czt_save_elems(ctypes.byref(g), ctypes.byref(w), vectorial, xl.C64)
    assert got == save_elems(nx, ny, mx, my, 3 if vectorial else 1, Lx, Ly)


def test_bench_workload_plan():
    # 2048 -> 512: four segments of 512 and transforms of 1024 (five transforms of 1024 per row
    # instead of two of 4096)
    assert plan(2048, 512) == (1024, 4, 512)
    assert plan(1024, 256) == (512, 4, 256)


def test_save_size_rejects_unsupported():
    lib = xl.load(build.build())
    g = xl.Grid(8000, 16, 0.5, 0.5, 0.0, 0.0)
    w = xl.Window(400, 16, 0.1, 0.1, 0.0, 0.0)
    assert lib.xl_czt_save_elems(ctypes.byref(g), ctypes.byref(w), 0, xl.C64) == -1
