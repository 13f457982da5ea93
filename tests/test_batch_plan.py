"""The batch runner's memory plan (xl_batch_plan_memory: host arithmetic, no device call): the
bytes a batch of optical-table setups allocates in each checkpoint mode, and the automatic mode
choice under a memory budget."""
import pytest

from paper_2310_08408_gb300 import build, xl

CFG = dict(wavelength=0.6328, extent=1024.0, w0=200.0, f=5000.0, cam_m=256, cam_width=64.0,
           lr=0.01, lr_z=1.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    xl.load(build.build())


def per_setup(n, cam_m, mode, cs=8, rs=4):
    """Bytes of one setup of side n, counted from the table's planes: 8 complex field planes (the
    source, after SLM1, after RS, the 2-component field after SLM2, the 3-component field after
    the wave plate), two 3-component gradient buffers, 12 complex spectrum planes in mode 0 (the
    RS input's 4 and the VRS input's 8: zero-padded 2n x 2n), 8 real planes (two masks, their
    gradients, their Adam moments), the camera field and its gradient (3 components each), 43
    doubles of parameters, gradients, moments and loss, and one int of the setup table."""
    p = n * n
    cplx_planes = 8 + 6 + (12 if mode == 0 else 0)
    return cplx_planes * p * cs + 8 * p * rs + 2 * 3 * cam_m * cam_m * cs + 43 * 8 + 4


@pytest.mark.parametrize("dtype,cs,rs", [("c64", 8, 4), ("c128", 16, 8)])
@pytest.mark.parametrize("mode", [0, 1])
def test_plan_counts_every_plane(dtype, cs, rs, mode):
    grid_n = [512, 1024, 512, 2048, 64]
    nb, m = xl.batch_plan_memory(dict(CFG, dtype=dtype, checkpoint=mode), grid_n)
    assert m == mode
    assert nb == 4 + sum(per_setup(n, 256, mode, cs, rs) for n in grid_n)


def test_checkpointing_takes_0_6_of_the_memory_per_pixel():
    a, _ = xl.batch_plan_memory(dict(CFG, checkpoint=0), [2048])
    c, _ = xl.batch_plan_memory(dict(CFG, checkpoint=1), [2048])
    assert abs(c / a - 144 / 240) < 0.01
    assert c < 0.61e9 and a > 1.0e9


def test_auto_mode_follows_the_budget():
    grid_n = [2048] * 8
    a, _ = xl.batch_plan_memory(dict(CFG, checkpoint=0), grid_n)
    c, _ = xl.batch_plan_memory(dict(CFG, checkpoint=1), grid_n)
    auto = dict(CFG, checkpoint=xl.CHECKPOINT_AUTO)
    assert xl.batch_plan_memory(dict(auto, memory_budget=0), grid_n) == (a, 0)
    assert xl.batch_plan_memory(dict(auto, memory_budget=a), grid_n) == (a, 0)
    assert xl.batch_plan_memory(dict(auto, memory_budget=a - 1), grid_n) == (c, 1)
    # below the checkpointed need the mode is still 1: xl_batch_create then fails without
    # allocating
    assert xl.batch_plan_memory(dict(auto, memory_budget=c - 1), grid_n) == (c, 1)


def test_budget_of_n_spectra_setups_holds_1_6_n_checkpointed():
    n = 10
    budget, _ = xl.batch_plan_memory(dict(CFG, checkpoint=0), [2048] * n)
    auto = dict(CFG, checkpoint=xl.CHECKPOINT_AUTO, memory_budget=budget)
    m = n
    while xl.batch_plan_memory(auto, [2048] * (m + 1))[0] <= budget:
        m += 1
    assert m == 16 and xl.batch_plan_memory(auto, [2048] * m)[1] == 1


@pytest.mark.parametrize("bad", [dict(checkpoint=3), dict(checkpoint=-1), dict(memory_budget=-5),
                                 dict(cam_m=0)])
def test_plan_rejects_bad_configurations(bad):
    with pytest.raises(xl.XLError):
        xl.batch_plan_memory(dict(CFG, **bad), [512])
    with pytest.raises(xl.XLError):
        xl.batch_plan_memory(CFG, [500])
