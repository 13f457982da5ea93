"""The allocation-free RS entry point (xl_rs_propagate_static) gives the results of
xl_rs_propagate. It exists for callers that cannot let a library allocate device memory; its
scratch is one fixed static device array shared by every call. This file is collected last so
that a failure here leaves every other test already run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu


def test_static_entry_point_matches_allocating_one_twice_in_a_row():
    import torch
    xl = lib()
    g = inputs.Grid(256, 128, 0.8, 0.6, -102.4, -38.4)
    u = np.stack([inputs.gaussian_random_phase(g, 40.0, 900 + i) for i in range(3)]).astype(np.complex64)
    zs = np.array([150.0, 150.0, 600.0])
    ud = to_dev(u, np.complex64)
    ref = to_np(xl.rs_propagate(ud, g, 0.6328, zs))
    lib_ = xl.load()
    grid = xl.Grid.of(g)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # two calls in a row share (and reuse) the static scratch
        out = torch.full_like(ud, float("nan"))
        st = lib_.xl_rs_propagate_static(ud.data_ptr(), out.data_ptr(), 3, ctypes.byref(grid),
                                         0.6328, zs.ctypes.data, stream)
        assert st == xl.OK, lib_.xl_last_error().decode()
        assert rel(to_np(out), ref) < TOL_C64


def test_static_entry_point_rejects_grids_above_its_scratch():
    import torch
    xl = lib()
    u = torch.zeros((1, 512, 512), dtype=torch.complex64, device="cuda")
    with pytest.raises(xl.XLError) as e:
        xl.rs_propagate_static(u, (512, 512, 1.0, 1.0, 0.0, 0.0), 0.6328, 100.0)
    assert e.value.status == xl.ERR_UNSUPPORTED and "256" in str(e.value)
