"""Host-staged pipeline: chunked, stream-overlapped runs give the same results as one device
pass over the whole batch (ragged last chunk, more chunks than staging slots)."""
import numpy as np
import pytest

from paper_2310_08408_gb300 import inputs
from gpu_util import lib, to_dev

pytestmark = pytest.mark.gpu
LAM = 0.6328


@pytest.mark.parametrize("chunk,depth", [(2, 2), (3, 1), (7, 2)])
def test_pipeline_matches_direct(chunk, depth):
    import torch
    xl = lib()
    from paper_2310_08408_gb300.pipeline import HostPipeline
    n, B = 64, 7
    g = inputs.Grid(n, n, 1.0, 1.0, -n / 2, -n / 2)
    u = np.stack([inputs.gaussian_random_phase(g, 20.0, 4600 + b) for b in range(B)]).astype(np.complex64)
    zs = [300.0 + 100.0 * (b % 3) for b in range(B)]
    U = to_dev(u, np.complex64)
    ref_out = xl.rs_propagate(U, g, LAM, zs)
    ref_i = xl.intensity_loss(ref_out.unsqueeze(1), (n, n, 1.0, 1.0, -n / 2, -n / 2), 1)[0]
    U_h = torch.from_numpy(u).pin_memory()
    out_h = torch.empty((B, n, n), dtype=torch.complex64).pin_memory()
    loss_h = torch.empty((B,), dtype=torch.float64).pin_memory()
    pipe = HostPipeline([((n, n), torch.complex64)], [((n, n), torch.complex64), ((), torch.float64)],
                        chunk=chunk, depth=depth)

    def fn(ins, outs, lo, k):
        xl.rs_propagate(ins[0], g, LAM, zs[lo:lo + k], out=outs[0])
        loss, _ = xl.intensity_loss(outs[0].unsqueeze(1), (n, n, 1.0, 1.0, -n / 2, -n / 2), 1)
        outs[1].copy_(loss)

    for _ in range(2):  # the second run reuses the staging slots and events
        pipe.run([U_h], [out_h, loss_h], fn)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(out_h, ref_out.cpu())
        assert torch.equal(loss_h, ref_i.cpu())


@pytest.mark.parametrize("chunk,depth", [(2, 4), (3, 3), (7, 1)])
def test_overlapped_passes_keep_each_pass_apart(chunk, depth):
    """prime / run_overlapped / finish: every pass's chunks carry that pass's values (a pass
    counter is added to the outputs), the last chunk's values arrive one pass late (during the
    next pass, or with finish), and the ahead-of-time upload of the next pass's first chunk never
    overwrites an input the current pass still reads."""
    import torch
    xl = lib()
    from paper_2310_08408_gb300.pipeline import HostPipeline
    n, B = 64, 7
    g = inputs.Grid(n, n, 1.0, 1.0, -n / 2, -n / 2)
    u = np.stack([inputs.gaussian_random_phase(g, 20.0, 4700 + b) for b in range(B)]).astype(np.complex64)
    zs = [300.0 + 100.0 * (b % 3) for b in range(B)]
    ref = xl.rs_propagate(to_dev(u, np.complex64), g, LAM, zs).cpu()
    U_h = torch.from_numpy(u).pin_memory()
    out_h = torch.zeros((B, n, n), dtype=torch.complex64).pin_memory()
    pipe = HostPipeline([((n, n), torch.complex64)], [((n, n), torch.complex64)], chunk=chunk, depth=depth)
    count = torch.zeros((), dtype=torch.float32, device="cuda")

    def fn(ins, outs, lo, k):
        if lo == 0:
            count.add_(1.0)
        xl.rs_propagate(ins[0], g, LAM, zs[lo:lo + k], out=outs[0])
        outs[0].add_(count)

    last_lo = ((B - 1) // chunk) * chunk
    pipe.prime([U_h])
    for p in range(1, 4):
        pipe.run_overlapped([U_h], [out_h], fn)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(out_h[:last_lo], ref[:last_lo] + p) or last_lo == 0
        if p > 1:
            assert torch.equal(out_h[last_lo:], ref[last_lo:] + (p - 1))
    pipe.finish()
    torch.cuda.current_stream().synchronize()
    assert torch.equal(out_h, ref + 3)


def test_alternating_passes_keep_each_pass_apart():
    """prime_alternating / run_alternating / finish: the whole batch in one chunk, passes
    alternating between two staging slots; each pass's results arrive during the next pass (or
    with finish) and carry that pass's values, and the upload of the next pass's input never
    overwrites the input the current pass reads. tail_due re-arms the last download after passes
    replayed from CUDA graphs."""
    import torch
    xl = lib()
    from paper_2310_08408_gb300.pipeline import HostPipeline
    n, B = 64, 5
    g = inputs.Grid(n, n, 1.0, 1.0, -n / 2, -n / 2)
    u = np.stack([inputs.gaussian_random_phase(g, 20.0, 4800 + b) for b in range(B)]).astype(np.complex64)
    zs = [300.0 + 100.0 * (b % 3) for b in range(B)]
    ref = xl.rs_propagate(to_dev(u, np.complex64), g, LAM, zs).cpu()
    U_h = torch.from_numpy(u).pin_memory()
    out_h = torch.zeros((B, n, n), dtype=torch.complex64).pin_memory()
    pipe = HostPipeline([((n, n), torch.complex64)], [((n, n), torch.complex64)], chunk=B, depth=2)
    count = torch.zeros((), dtype=torch.float32, device="cuda")

    def fn(ins, outs, lo, k):
        count.add_(1.0)
        xl.rs_propagate(ins[0], g, LAM, zs[lo:lo + k], out=outs[0])
        outs[0].add_(count)

    pipe.prime_alternating([U_h], 0)
    for p in range(1, 5):
        pipe.run_alternating([U_h], [out_h], fn, (p - 1) % 2)
        torch.cuda.current_stream().synchronize()
        if p > 1:
            assert torch.equal(out_h, ref + (p - 1))
    pipe.tail_due([out_h], B, 1)
    pipe.finish()
    torch.cuda.current_stream().synchronize()
    assert torch.equal(out_h, ref + 4)
