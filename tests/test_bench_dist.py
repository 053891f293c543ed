"""The multi-process path of bench.py on the CPU: two gloo ranks, each an
independent replica, combine their step times (max) and work (sum)."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    assert bench.dist_env() == (rank, world, rank)
    ms, units = bench.aggregate(100.0 + 50.0 * rank, 7.0 + rank, world)
    bench.barrier(world)
    out.put((rank, ms, units))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in res:
        assert ms == 150.0  # max over ranks
        assert units == 15.0  # sum over ranks


def test_single_rank_aggregation_is_identity():
    import bench

    assert bench.aggregate(12.5, 3.0, 1) == (12.5, 3.0)
