"""The allocation-free RS entry point (xl_rs_propagate_static) against the allocating one and
the FP64 oracle. It exists for callers that cannot let a library allocate device memory; its
scratch is one fixed static device array shared by every call. This file is collected last so
that a failure here leaves every other test already run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu

LAM = 0.6328


def _static(xl, ud, g, zs):
    import torch
    lib_ = xl.load()
    grid = xl.Grid.of(g)
    stream = torch.cuda.current_stream().cuda_stream
    out = torch.full_like(ud, float("nan"))
    zz = np.ascontiguousarray(zs, dtype=np.float64)
    st = lib_.xl_rs_propagate_static(ud.data_ptr(), out.data_ptr(), ud.shape[0], ctypes.byref(grid),
                                     LAM, zz.ctypes.data, stream)
    assert st == xl.OK, lib_.xl_last_error().decode()
    return to_np(out)


# (nx, ny): every transform length of the scratch's twiddle blocks (64..512) on both axes, and
# grids with nx > ny and nx < ny; the distances change partway through the batch.
SHAPES = [(256, 128), (32, 32), (64, 256), (128, 64), (256, 256)]


@pytest.mark.parametrize("nx,ny", SHAPES)
def test_static_entry_point_matches_allocating_one_and_oracle_twice_in_a_row(nx, ny):
    xl = lib()
    g = inputs.Grid(nx, ny, 0.8, 0.6, -(nx // 2) * 0.8, -(ny // 2) * 0.6)
    u = np.stack([inputs.gaussian_random_phase(g, 10.0 + nx / 8, 900 + i) for i in range(3)]
                 ).astype(np.complex64)
    zs = [150.0, 150.0, 600.0]
    ud = to_dev(u, np.complex64)
    ref = to_np(xl.rs_propagate(ud, g, LAM, zs))
    orc = np.stack([oracle.rs_conv(u[i].astype(np.complex128), g.dx, g.dy, LAM, zs[i])
                    for i in range(3)])
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        out = _static(xl, ud, g, zs)
        assert rel(out, ref) < TOL_C64
        assert rel(out, orc) < TOL_C64


def test_static_entry_point_rejects_grids_above_its_scratch():
    import torch
    xl = lib()
    u = torch.zeros((1, 512, 512), dtype=torch.complex64, device="cuda")
    with pytest.raises(xl.XLError) as e:
        xl.rs_propagate_static(u, (512, 512, 1.0, 1.0, 0.0, 0.0), LAM, 100.0)
    assert e.value.status == xl.ERR_UNSUPPORTED and "256" in str(e.value)
