"""Replica bookkeeping for runs on several GPUs of one node (one process per GPU).

The hot path shards over independent units (fields of a batch, setups of the optimiser batch)
with no exchange between ranks: each rank works on its own units, and the only collective
operations are the barrier around the timed region and the maximum of the ranks' times. The
functions here take any torch.distributed backend (NCCL on GPUs, gloo for the host-side tests) and
degrade to single-process behaviour when no process group is initialised.
"""
from __future__ import annotations

import torch


def world_and_rank() -> tuple[int, int]:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def contiguous_shard(n_items: int, rank: int, world: int) -> range:
    """The contiguous slice of n_items units of `rank`: sizes differ by at most one, the slices
    are disjoint, ordered by rank and cover all units."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, n_items >= 0")
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's synthetic inputs (independent streams per rank for weak scaling)."""
    return int(base) + 1000 * int(rank)


def barrier(device=None) -> None:
    """Waits for every rank; with a CUDA device also for its queued work."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
    if device is not None and torch.device(device).type == "cuda":
        torch.cuda.synchronize(device)


def max_over_ranks(value: float, device="cpu") -> float:
    """The maximum of a per-rank value (the slowest rank's time) over all ranks."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, repeats: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    if max_ms <= 0:
        raise ValueError("max_ms must be positive")
    return units_per_rank * world * repeats / (max_ms / 1000.0)
