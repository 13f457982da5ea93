"""Replica bookkeeping of multi-GPU runs, exercised on the host with two gloo ranks: sharding
partitions the units, the timing is the slowest rank's, the whole-job rate counts every rank's
units, and the ranks draw independent inputs (no GPU needed)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2310_08408_gb300 import replicas


def test_contiguous_shard_partitions():
    for n in (0, 1, 5, 256, 257):
        for world in (1, 2, 3, 8):
            parts = [replicas.contiguous_shard(n, r, world) for r in range(world)]
            flat = [i for p in parts for i in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.contiguous_shard(4, 2, 2)


def test_single_process_fallbacks():
    assert replicas.world_and_rank() == (1, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    replicas.barrier()
    assert replicas.whole_job_rate(64, 1, 10, 100.0) == 6400.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert replicas.world_and_rank() == (world, rank)
        shard = replicas.contiguous_shard(256, rank, world)
        replicas.barrier()
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        m = replicas.max_over_ranks(ms)
        rate = replicas.whole_job_rate(len(shard), world, 3, m)
        out[rank] = (shard.start, shard.stop, m, rate, replicas.rank_seed(100, rank))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    (a0, b0, m0, r0, s0), (a1, b1, m1, r1, s1) = res[0], res[1]
    assert (a0, b0, a1, b1) == (0, 128, 128, 256)
    assert m0 == m1 == 15.0                       # the slowest rank's time on every rank
    assert r0 == r1 == pytest.approx(128 * 2 * 3 / 0.015)
    assert s0 != s1                               # independent input streams
