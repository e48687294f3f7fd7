"""bench.py's multi-GPU form runs independent replicas (the row update is a
sequential insertion and the path has no exchange step on one GPU's
families); its aggregation -- the slowest rank's times, every rank's cells --
is checked here with two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, e2e, cells = bench.replica_totals(10.0 + rank, 20.0 - rank, 1000.0 * (rank + 1), dist, "cpu")
        out[rank] = (ms, e2e, cells)
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (11.0, 20.0, 3000.0)
