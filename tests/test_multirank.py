"""Replica aggregation of bench.py across ranks (world size 2, gloo on CPU).

The path shards as independent replicas: each rank solves its own problem and
the only exchange is the max of the times and the sum of the work after the
timed region.  This checks that reduction on two CPU ranks."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, REPO)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs, units = bench.aggregate_over_ranks(1.5 + rank, 100.0 * (rank + 1), world, "cpu")
    out[rank] = (secs, units)
    dist.destroy_process_group()


def test_max_time_and_summed_work_over_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        for r in range(world):
            assert out[r] == (2.5, 300.0)


def test_single_rank_is_identity():
    sys.path.insert(0, REPO)
    import bench
    assert bench.aggregate_over_ranks(2.0, 7, 1, "cpu") == (2.0, 7.0)
