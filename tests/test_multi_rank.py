"""The benchmark's multi-rank logic on the CPU with two gloo ranks: every
rank answers its own batch (replicas, no collective on the data path); the
job time is the slowest rank's, the value counts all ranks' queries."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took (r + 1) * 100 ms for 4 steps of 1,000 queries each
        total = bench.max_over_ranks((rank + 1) * 100.0, dist, "cpu")
        ms, value = bench.job_rate(total, 4, 1000, world)
        dist.barrier()
        out[rank] = (total, ms, value)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_sum_the_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        total, ms, value = out[r]
        assert total == 200.0               # the slower rank
        assert ms == 50.0
        assert value == pytest.approx(2 * 1000 / 0.05)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    ms, v = bench.job_rate(100.0, 10, 500, 1)
    assert ms == 10.0 and v == pytest.approx(50_000)
