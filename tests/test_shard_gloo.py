"""The sharded tree's exchange over two and three gloo ranks on the CPU.

Each rank computes the minimum spanning forest of its rows (here with the
oracle, so that no GPU is needed), one all-gather exchanges the forests, and
every rank builds the whole family's tree from the union.  Every rank's tree
must equal the oracle's tree of the whole family.  The GPU form runs the same
code with the library's famsa_msf_rows / famsa_tree_from_edges
(tests/test_gpu_shard.py covers those on one GPU).
"""
import os
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, fam, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    import synth
    from paper_1603_06958_gb300.shard import sharded_tree
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res, off = synth.family(**fam)
        t = sharded_tree(res, off,
                         local_msf=lambda b, e: oracle.msf_rows(res, off, b, e),
                         merge=lambda k, edges: oracle.tree_from_edges(k, edges), device="cpu")
        out[rank] = {n: np.asarray(v).tolist() for n, v in t.items()}
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,fam", [
    (2, dict(k=90, seed=5, root_len=30, alphabet=3, dup_frac=0.2)),
    (3, dict(k=61, seed=8, root_len=50)),
])
def test_sharded_tree_over_gloo_ranks(world, fam):
    pytest.importorskip("torch.distributed")
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    res, off = synth.family(**fam)
    want = oracle.tree(res, off)
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29600 + (os.getpid() % 1500) + world
    procs = [ctx.Process(target=_rank, args=(r, world, port, fam, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    for r in range(world):
        for name, v in want.items():
            assert np.array_equal(np.asarray(out[r][name]).reshape(np.asarray(v).shape), v), (r, name)


def test_shard_rows_cover_every_row_once():
    sys.path.insert(0, ROOT)
    from paper_1603_06958_gb300.shard import shard_rows
    for k in (1, 2, 3, 10, 61, 1000, 20000):
        for world in (1, 2, 3, 4, 8):
            ranges = shard_rows(k, world)
            assert len(ranges) == world
            rows = [i for b, e in ranges for i in range(b, e)]
            assert rows == list(range(1, k))
    # about equal pair counts
    ranges = shard_rows(20000, 4)
    pairs = [(e * (e - 1) - b * (b - 1)) // 2 for b, e in ranges]
    assert max(pairs) < 1.01 * min(pairs)
