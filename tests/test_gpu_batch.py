"""Batched optical-table optimiser (native runner, CUDA-graph replay) against the oracle's table.

Each setup: x-polarised Gaussian -> SLM1 -> RS z1 -> SLM2 -> half-wave plate (theta) -> VRS z2 ->
lens f -> VCZT f -> second-moment spot size (Results / Methods virtual tables, batched as with the
paper's vmap). Masks start from SplitMix64 draws, which the test regenerates independently.
"""
import numpy as np
import pytest

import oracle
import oracle.table as otable
from paper_2310_08408_gb300 import inputs
from gpu_util import TOL_LOSS, lib, rel

pytestmark = pytest.mark.gpu

CFG = dict(wavelength=0.6328, extent=64.0, w0=12.0, f=800.0, cam_m=40, cam_width=48.0, lr=0.01,
           lr_z=1.0)
GRIDS = [64, 128, 64]
INIT = [[0.3, 300.0, 250.0], [0.5, 280.0, 260.0], [0.1, 320.0, 240.0]]
SEED = 1234


def _oracle(setup, phi1, phi2, dtype):
    n = GRIDS[setup]
    g = inputs.Grid.centred(n, CFG["extent"] / n)
    win = inputs.Window.centred(CFG["cam_m"], CFG["cam_width"])
    t = otable.Table(g.astuple(), win.astuple(), CFG["wavelength"], CFG["f"])
    src = inputs.x_polarised_gaussian(g, CFG["w0"])
    if dtype == "c64":
        src = src.astype(np.complex64).astype(np.complex128)
    th, z1, z2 = INIT[setup]
    L, planes = otable.forward(t, src, phi1, phi2, th, z1, z2)
    return L, otable.backward(t, src, phi1, phi2, th, z1, z2, planes)


@pytest.mark.parametrize("checkpoint", [0, 1])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_batch_step_matches_oracle_table(dtype, checkpoint):
    """Both checkpointing modes: spectra kept by the forwards (0), plane fields only (1)."""
    xl = lib()
    b = xl.Batch(dict(CFG, dtype=dtype, checkpoint=checkpoint), GRIDS, INIT, SEED)
    tol_l, tol_g = (TOL_LOSS, 1e-3) if dtype == "c64" else (1e-10, 1e-8)
    phis = []
    for s in range(len(GRIDS)):
        p1, p2 = b.read(xl.BATCH_PHI1, s), b.read(xl.BATCH_PHI2, s)
        n = GRIDS[s]
        # the device SplitMix64 draws equal the published generator's
        e1 = (2 * np.pi * inputs.uniform(SEED + s, n * n)).reshape(n, n)
        e2 = (2 * np.pi * inputs.uniform(SEED + s + 0x10000, n * n)).reshape(n, n)
        assert np.max(np.abs(p1 - e1.astype(p1.dtype))) == 0
        assert np.max(np.abs(p2 - e2.astype(p2.dtype))) == 0
        phis.append((p1.astype(np.float64), p2.astype(np.float64)))
    b.step(use_graph=False)
    for s in range(len(GRIDS)):
        L, gr = _oracle(s, *phis[s], dtype)
        assert abs(b.read(xl.BATCH_LOSS, s)[0] - L) / L < tol_l
        assert rel(b.read(xl.BATCH_GRAD_PHI1, s), gr["phi1"]) < tol_g
        assert rel(b.read(xl.BATCH_GRAD_PHI2, s), gr["phi2"]) < tol_g
        gs = b.read(xl.BATCH_GRAD_SCALARS, s)
        errs = [abs(a - ref) / abs(ref) for a, ref in zip(gs, (gr["theta"], gr["z1"], gr["z2"]))]
        assert max(errs) < tol_g, (s, errs)
        # first Adam step: p - lr g / (|g| + eps)
        sc = b.read(xl.BATCH_SCALARS, s)
        for k, (lr, g0) in enumerate(((CFG["lr"], gs[0]), (CFG["lr_z"], gs[1]), (CFG["lr_z"], gs[2]))):
            assert abs(sc[k] - (INIT[s][k] - lr * g0 / (abs(g0) + 1e-8))) < 1e-12 * max(1, abs(sc[k]))
    b.close()


def test_batch_graph_replay_equals_eager_steps():
    xl = lib()
    eager = xl.Batch(CFG, GRIDS, INIT, SEED)
    graph = xl.Batch(CFG, GRIDS, INIT, SEED)
    for _ in range(4):
        eager.step(use_graph=False)
        graph.step(use_graph=True)
    for s in range(len(GRIDS)):
        assert np.array_equal(eager.read(xl.BATCH_SCALARS, s), graph.read(xl.BATCH_SCALARS, s))
        assert np.array_equal(eager.read(xl.BATCH_PHI1, s), graph.read(xl.BATCH_PHI1, s))
        assert eager.read(xl.BATCH_LOSS, s)[0] == graph.read(xl.BATCH_LOSS, s)[0]
    eager.close()
    graph.close()


def test_batch_checkpoint_mode_memory_and_steps():
    """Plane-field checkpointing holds 0.6 of the spectra mode's memory per pixel (14 complex
    field planes and 8 real mask / moment planes a setup against 26 and 8; the camera buffers add
    a little at these small grids) and steps to the same optimiser state within the complex64
    gradient tolerance after several steps."""
    xl = lib()
    a = xl.Batch(dict(CFG, checkpoint=0), GRIDS, INIT, SEED)
    c = xl.Batch(dict(CFG, checkpoint=1), GRIDS, INIT, SEED)
    assert c.memory() < 0.65 * a.memory(), (c.memory(), a.memory())
    for _ in range(3):
        a.step(use_graph=True)
        c.step(use_graph=True)
    for s in range(len(GRIDS)):
        assert abs(a.read(xl.BATCH_LOSS, s)[0] - c.read(xl.BATCH_LOSS, s)[0]) <= TOL_LOSS * a.read(xl.BATCH_LOSS, s)[0]
        assert rel(c.read(xl.BATCH_GRAD_PHI1, s), a.read(xl.BATCH_GRAD_PHI1, s)) < 1e-3
        assert np.allclose(c.read(xl.BATCH_SCALARS, s), a.read(xl.BATCH_SCALARS, s), rtol=1e-6, atol=1e-9)
    a.close()
    c.close()


def test_batch_memory_budget():
    """The batch allocates exactly the planned bytes in both modes; XL_CHECKPOINT_AUTO keeps the
    spectra while they fit in memory_budget and checkpoints the plane fields when they do not;
    a budget below the checkpointed need fails with XL_ERR_NOMEM before any allocation."""
    xl = lib()
    plan0, _ = xl.batch_plan_memory(dict(CFG, checkpoint=0), GRIDS)
    plan1, _ = xl.batch_plan_memory(dict(CFG, checkpoint=1), GRIDS)
    auto = dict(CFG, checkpoint=xl.CHECKPOINT_AUTO)
    a = xl.Batch(dict(auto, memory_budget=plan0), GRIDS, INIT, SEED)
    assert a.memory() == plan0
    c = xl.Batch(dict(auto, memory_budget=plan0 - 1), GRIDS, INIT, SEED)
    assert c.memory() == plan1
    c.step(use_graph=True)
    assert np.isfinite(c.read(xl.BATCH_LOSS, 0)[0])
    a.close()
    c.close()
    with pytest.raises(xl.XLError) as e:
        xl.Batch(dict(auto, memory_budget=plan1 - 1), GRIDS, INIT, SEED)
    assert e.value.status == xl.ERR_NOMEM
