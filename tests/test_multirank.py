"""Multi-rank path of bench.py on CPU: gloo, world size 2 (no GPU).

Every rank renders its own replica; the only cross-rank steps are the barrier
and the reduction of the timing (max over ranks) and of the work (sum).
"""
from __future__ import annotations

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_env() == (world, rank, rank)
    bench.barrier()
    ms, units = bench.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1))
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_aggregate_takes_max_time_and_sums_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units in out:
        assert ms == 15.0
        assert units == 300.0


def test_aggregate_is_identity_without_process_group():
    import bench
    assert bench.aggregate(3.0, 7.0) == (3.0, 7.0)
