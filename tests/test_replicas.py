"""The multi-GPU form is independent replicas (one per rank, no data exchange): the bench's
whole-job figures are the slowest rank's time and the sum of the ranks' updates.  Checked with
two gloo ranks on the CPU."""
from __future__ import annotations

import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 13.25][rank]
    upd = [1000, 1500][rank]
    t, n = bench.replica_totals(ms, upd, dist, "cpu")
    out[rank] = (t, n)
    dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (13.25, 2500)


def test_replica_totals_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(7.0, 42) == (7.0, 42)
