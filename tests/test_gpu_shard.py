"""Sharded pair set on one GPU: famsa_msf_rows per shard of rows, the union
of the shards' trees through famsa_tree_from_edges, against the oracle.

Any partition of the rows must give exactly the oracle's tree of the whole
family (and famsa_slink_tree's).  Each shard's tree is checked against the
oracle's Kruskal forest of the same pairs (the family's internal row order
is its (length, index) order): same edge count, and the same sorted edge
weights -- unique for every minimum spanning tree, ties or not.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    from paper_1603_06958_gb300 import build
    build.build()
    import paper_1603_06958_gb300 as m
    m.load()
    return m


def _same(got, want):
    for key in ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den", "sizes"):
        g, w = np.asarray(got[key]), np.asarray(want[key])
        assert np.array_equal(g.reshape(w.shape), w), key


def _weights(e):
    return sorted((int(n), int(d)) for n, d in zip(e["h_num"], e["h_den"]))


FAMS = [dict(k=2, seed=1, root_len=30),
        dict(k=60, seed=4, root_len=12, alphabet=2, dup_frac=0.3),
        dict(k=300, seed=8, root_len=8, alphabet=2, indel_rate=0.1, dup_frac=0.05),
        dict(k=700, seed=41, root_len=60, alphabet=3, sub_rate=0.1),
        dict(k=1500, seed=3, root_len=250)]


@pytest.mark.parametrize("fam", range(len(FAMS)))
def test_shards_union_gives_the_whole_tree(fg, fam):
    from paper_1603_06958_gb300.shard import shard_rows
    res, off = synth.family(**FAMS[fam])
    k = len(off) - 1
    want = oracle.tree(res, off)
    order = np.lexsort((np.arange(k), np.diff(off))).astype(np.int32)
    f = fg.pack_peq(res, off)
    try:
        _same(fg.slink_tree(f), want)
        rng = np.random.default_rng(fam)
        parts = [shard_rows(k, w) for w in (1, 2, 3, 5)]
        if k > 8:
            cuts = sorted({1, k, *rng.integers(2, k - 1, 4).tolist()})
            parts.append(list(zip(cuts[:-1], cuts[1:])))
        for ranges in parts:
            edges = []
            for b, e in ranges:
                if e <= b:
                    continue
                got = fg.msf_rows(f, b, e)
                assert len(got["edge_a"]) == e - 1
                assert (got["edge_a"] < got["edge_b"]).all()
                if k <= 700:
                    ref = oracle.msf_rows(res, off, b, e, order=order)
                    assert _weights(got) == _weights(ref)
                edges.append(got)
            union = {n: np.concatenate([x[n] for x in edges]) for n in edges[0]}
            _same(fg.tree_from_edges(k, union), want)
    finally:
        f.free()


def test_shard_outputs_on_the_device_and_sharded_tree(fg):
    import torch
    from paper_1603_06958_gb300.shard import sharded_tree
    res, off = synth.family(400, 11, root_len=150, alphabet=4, dup_frac=0.05)
    k = len(off) - 1
    want = oracle.tree(res, off)
    f = fg.pack_peq(torch.from_numpy(res).cuda(), torch.from_numpy(off).cuda())
    try:
        e1 = fg.msf_rows(f, 1, 200, device=True)
        e2 = fg.msf_rows(f, 200, k, device=True)
        union = {n: torch.cat([e1[n], e2[n]]) for n in e1}
        t = fg.tree_from_edges(k, union, device=True)
        torch.cuda.synchronize()
        _same({n: v.cpu().numpy() for n, v in t.items()}, want)
    finally:
        f.free()
    # one process: the orchestration with the library's calls
    t = sharded_tree(torch.from_numpy(res).cuda(), torch.from_numpy(off).cuda())
    torch.cuda.synchronize()
    _same({n: v.cpu().numpy() for n, v in t.items()}, want)


def test_shard_errors(fg):
    res, off = synth.family(50, 6, root_len=40)
    k = len(off) - 1
    f = fg.pack_peq(res, off)
    lib = fg.load()
    try:
        a = np.zeros(k, np.int32)
        n = np.zeros(k, np.uint64)
        d = np.zeros(k, np.uint32)
        for b, e in ((0, 5), (5, 5), (10, 9), (1, k + 1)):
            assert lib.famsa_msf_rows(f.handle, b, e, a.ctypes.data, a.ctypes.data, n.ctypes.data,
                                      d.ctypes.data, 0, None) == fg.FAMSA_EINVAL
        full = fg.msf_rows(f, 1, k)
    finally:
        f.free()
    # too few edges, a repeated edge (so not all points joined), a self loop,
    # a point out of range, a denominator beyond the exact keys' range
    bad = []
    bad.append({n: v[1:] for n, v in full.items()})
    dup = {n: v.copy() for n, v in full.items()}
    for n in dup:
        dup[n][1] = dup[n][0]
    bad.append(dup)
    loop = {n: v.copy() for n, v in full.items()}
    loop["edge_b"][3] = loop["edge_a"][3]
    bad.append(loop)
    out = {n: v.copy() for n, v in full.items()}
    out["edge_b"][4] = k
    bad.append(out)
    big = {n: v.copy() for n, v in full.items()}
    big["h_den"][5] = 40000
    bad.append(big)
    for edges in bad:
        with pytest.raises(fg.FamsaError) as ei:
            fg.tree_from_edges(k, edges)
        assert ei.value.status == fg.FAMSA_EINVAL
    # the exact keys of this path need lengths <= 32767
    seqs = [np.arange(20, dtype=np.uint8)] * 3 + [np.zeros(33000, np.uint8)]
    wres = np.concatenate(seqs)
    woff = np.concatenate([[0], np.cumsum([len(x) for x in seqs])]).astype(np.int64)
    f = fg.pack_peq(wres, woff)
    try:
        with pytest.raises(fg.FamsaError) as ei:
            fg.msf_rows(f, 1, 4)
        assert ei.value.status == fg.FAMSA_ERANGE
    finally:
        f.free()
