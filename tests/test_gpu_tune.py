"""The autotuner on the device: xl_autotune picks a variant for every pass a grid and window use,
and every variant of every tunable pass gives bit-identical fields (they differ only in how many
rows a block holds)."""
import numpy as np
import pytest

from paper_2310_08408_gb300 import inputs
from gpu_util import lib, to_dev

pytestmark = pytest.mark.gpu
LAM = 0.633


def test_autotune_and_variants_bit_identical():
    import torch
    xl = lib()
    n, m = 1024, 256
    g = inputs.Grid(n, n, 1.0, 1.0, -n / 2, -n / 2)
    w = (m, m, 0.25, 0.25, -32.0, -32.0)
    u = to_dev(inputs.gaussian_random_phase(g, 200.0, 5800)[None].astype(np.complex64), np.complex64)
    G = to_dev(inputs.random_unit(5810, (1, m, m)).astype(np.complex64), np.complex64)
    xl.tune_clear()
    ref_rs = xl.rs_propagate(u, g, LAM, [3000.0])
    ref_czt = xl.czt_propagate(u, g, w, LAM, [3000.0])
    ref_adj = xl.czt_propagate_backward(G, g, w, LAM, [3000.0])
    xl.autotune(g, w, xl.C64, reps=3)
    Lrs, Lczt = 2 * n, 2048  # czt: next power of two >= n + m - 1
    fams = [(xl.TUNE_RS_PASS1, Lrs), (xl.TUNE_RS_PASS3, Lrs), (xl.TUNE_CZT_FWD_X, Lczt),
            (xl.TUNE_CZT_FWD_Y, Lczt), (xl.TUNE_CZT_ADJ_X, Lczt), (xl.TUNE_CZT_ADJ_Y, Lczt)]
    for f, L in fams:
        assert xl.tune_get(f, L, xl.C64) in (0, 1, 2)
    # results under the tuned choice and under every forced variant
    for v in (None, 0, 1, 2):
        if v is not None:
            for f, L in fams:
                xl.tune_set(f, L, xl.C64, v)
        assert torch.equal(xl.rs_propagate(u, g, LAM, [3000.0]), ref_rs)
        assert torch.equal(xl.czt_propagate(u, g, w, LAM, [3000.0]), ref_czt)
        assert torch.equal(xl.czt_propagate_backward(G, g, w, LAM, [3000.0]), ref_adj)
    xl.tune_clear()
