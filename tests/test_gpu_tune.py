"""The autotuner on the device: xl_autotune picks a variant for every pass a grid and window use.
Rows-per-block variants (0-2) give bit-identical fields; the radix-plan variants of the CZT
passes (3, 4: the FFT's radix-4 stage first or second instead of last) give the same fields
within rounding, checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_C64, lib, rel, to_dev, to_np

pytestmark = pytest.mark.gpu
LAM = 0.633


def test_autotune_variants_and_radix_plans():
    import torch
    xl = lib()
    n, m = 2048, 512
    g = inputs.Grid(n, n, 0.5, 0.5, -n / 4, -n / 4)
    w = inputs.Window(m, m, 0.125, 0.125, -32.0, -32.0)
    u0 = inputs.gaussian_random_phase(g, 200.0, 5800).astype(np.complex64)
    u = to_dev(u0[None], np.complex64)
    G0 = inputs.random_unit(5810, (m, m)).astype(np.complex64)
    G = to_dev(G0[None], np.complex64)
    z = 3000.0
    xl.tune_clear()
    ref_rs = xl.rs_propagate(u, g, LAM, [z])
    ref_czt = xl.czt_propagate(u, g, w, LAM, [z])
    ref_adj = xl.czt_propagate_backward(G, g, w, LAM, [z])
    xl.autotune(g, w, xl.C64, reps=3)
    Lrs, Lczt = 2 * n, 1024  # CZT 2048 -> 512: four segments, transforms of 1024
    rs_fams = [(xl.TUNE_RS_PASS1, Lrs), (xl.TUNE_RS_PASS3, Lrs)]
    czt_fams = [(f, Lczt) for f in (xl.TUNE_CZT_FWD_X, xl.TUNE_CZT_FWD_Y, xl.TUNE_CZT_ADJ_X,
                                    xl.TUNE_CZT_ADJ_Y)]
    for f, L in rs_fams:
        assert xl.tune_get(f, L, xl.C64) in (0, 1, 2)
    for f, L in czt_fams:
        assert xl.tune_get(f, L, xl.C64) in (0, 1, 2, 3, 4)
    orc = oracle.czt_conv(u0.astype(np.complex128), g.astuple(), w.astuple(), LAM, z)
    orc_adj = oracle.czt_conv(G0.astype(np.complex128), g.astuple(), w.astuple(), LAM, z, adjoint=True)
    # under the tuned choice and under every forced variant
    for v in (None, 0, 1, 2, 3, 4):
        if v is not None:
            for f, L in rs_fams:
                xl.tune_set(f, L, xl.C64, min(v, 2))
            for f, L in czt_fams:
                xl.tune_set(f, L, xl.C64, v)
        assert torch.equal(xl.rs_propagate(u, g, LAM, [z]), ref_rs)
        c = xl.czt_propagate(u, g, w, LAM, [z])
        a = xl.czt_propagate_backward(G, g, w, LAM, [z])
        if v is not None and v < 3:
            assert torch.equal(c, ref_czt) and torch.equal(a, ref_adj), v
        assert rel(to_np(c)[0], orc) < TOL_C64, v
        assert rel(to_np(a)[0], orc_adj) < TOL_C64, v
    xl.tune_clear()


def test_tune_set_rejects_plan_variants_for_rs_families():
    xl = lib()
    with pytest.raises(xl.XLError):
        xl.tune_set(xl.TUNE_RS_PASS1, 4096, xl.C64, 3)
    xl.tune_set(xl.TUNE_CZT_FWD_X, 1024, xl.C64, 4)
    assert xl.tune_get(xl.TUNE_CZT_FWD_X, 1024, xl.C64) == 4
    xl.tune_clear()
