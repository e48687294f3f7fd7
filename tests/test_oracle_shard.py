"""Pins for the oracle's sharded-pair-set routines (CPU only).

msf_rows is Kruskal's minimum spanning forest of a range of rows; it is
pinned by the cut property checked by brute force (every forest edge is the
lightest pair across the cut it makes, among the shard's pairs), by its
edge count (a spanning tree of points 0..r1-1), and against SciPy's minimum
spanning tree on families whose keys are all distinct.  slink_edges is SLINK
over an edge list alone; with every pair it equals the matrix SLINK, and --
the fact the sharded tree rests on -- with only a minimum spanning tree, or
the union of the forests of any partition of the rows, it still does.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _frac(n, d):
    return Fraction(10 ** 30) if d == 0 else Fraction(int(n), int(d))


def _same(got, want):
    for key in ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den", "sizes"):
        assert np.array_equal(np.asarray(got[key]), np.asarray(want[key])), key


FAMS = [dict(k=40, seed=4, root_len=12, alphabet=2, dup_frac=0.3),
        dict(k=90, seed=5, root_len=30, alphabet=3, dup_frac=0.2),
        dict(k=120, seed=7, root_len=60)]


@pytest.mark.parametrize("fam", range(len(FAMS)))
def test_msf_rows_cut_property_and_size(fam):
    res, off = synth.family(**FAMS[fam])
    k = len(off) - 1
    lens = np.diff(off)
    tri = oracle.lcs_allpairs(res, off)
    sq = oracle.tri_to_square(tri, k)

    def key(i, j):
        L = int(sq[i, j])
        d = int(lens[i] + lens[j] - 2 * L)
        return _frac(d * d, L)

    rng = np.random.default_rng(fam)
    order = rng.permutation(k).astype(np.int32)
    for r0, r1 in ((1, k), (k // 3, 2 * k // 3), (k - 5, k)):
        e = oracle.msf_rows(res, off, r0, r1, order=order)
        assert len(e["edge_a"]) == r1 - 1
        pairs = [(order[i], order[j]) for i in range(r0, r1) for j in range(i)]
        for a, b, n, d in zip(e["edge_a"], e["edge_b"], e["h_num"], e["h_den"]):
            assert a < b and _frac(n, d) == key(a, b)
        # cut property: removing edge t splits the forest; it is a lightest shard pair across
        for t in range(len(e["edge_a"])):
            comp = {int(order[i]): int(order[i]) for i in range(r1)}

            def find(x):
                while comp[x] != x:
                    x = comp[x]
                return x
            for u in range(len(e["edge_a"])):
                if u != t:
                    comp[find(int(e["edge_a"][u]))] = find(int(e["edge_b"][u]))
            side = find(int(e["edge_a"][t]))
            best = min(key(a, b) for a, b in pairs if (find(a) == side) != (find(b) == side))
            assert _frac(e["h_num"][t], e["h_den"][t]) == best


def test_msf_rows_matches_scipy_tree_weights():
    # the sorted edge weights of a minimum spanning tree are the same for
    # every minimum spanning tree, ties or not
    scipy_mst = pytest.importorskip("scipy.sparse.csgraph").minimum_spanning_tree
    res, off = synth.family(60, 9, root_len=200, sub_rate=0.15)
    k = len(off) - 1
    lens = np.diff(off).astype(np.float64)
    sq = oracle.tri_to_square(oracle.lcs_allpairs(res, off), k).astype(np.float64)
    iu = np.triu_indices(k, 1)
    assert (sq[iu] > 0).all()
    d = lens[:, None] + lens[None, :] - 2 * sq
    w = d * d / np.where(sq > 0, sq, 1) + 1.0  # +1: SciPy reads a zero weight as no edge
    m = scipy_mst(np.triu(w, 1)).tocoo()
    want = sorted(m.data.tolist())
    e = oracle.msf_rows(res, off, 1, k)
    got = sorted((int(n) / int(dd) + 1.0) for n, dd in zip(e["h_num"], e["h_den"]))
    assert len(got) == len(want) == k - 1
    assert np.allclose(got, want, rtol=0, atol=1e-9)


@pytest.mark.parametrize("fam", range(len(FAMS)))
def test_slink_edges_from_all_pairs_tree_and_shards(fam):
    res, off = synth.family(**FAMS[fam])
    k = len(off) - 1
    want = oracle.tree(res, off)
    # every pair
    iu = np.triu_indices(k, 1)
    tri = oracle.lcs_allpairs(res, off)
    lens = np.diff(off).astype(np.int64)
    L = tri.astype(np.int64)
    indel = lens[iu[0]] + lens[iu[1]] - 2 * L
    num = np.where(L == 0, 1, indel * indel).astype(np.uint64)
    den = L.astype(np.uint32)
    full = {"edge_a": iu[0], "edge_b": iu[1], "h_num": num, "h_den": den}
    _same(oracle.tree_from_edges(k, full), want)
    # a minimum spanning tree alone
    _same(oracle.tree_from_edges(k, oracle.msf_rows(res, off, 1, k)), want)
    # the union of the forests of a partition of the rows, in any row order
    rng = np.random.default_rng(10 + fam)
    order = rng.permutation(k).astype(np.int32)
    cuts = sorted({1, k, *rng.integers(2, k - 1, 3).tolist()})
    parts = [oracle.msf_rows(res, off, a, b, order=order) for a, b in zip(cuts[:-1], cuts[1:])]
    union = {n: np.concatenate([p[n] for p in parts]) for n in parts[0]}
    _same(oracle.tree_from_edges(k, union), want)
    # a proper subset of a spanning tree is not enough: lambda changes
    cut = {n: v[1:] for n, v in oracle.msf_rows(res, off, 1, k).items()}
    got = oracle.tree_from_edges(k, cut)
    assert not all(np.array_equal(got[x], want[x]) for x in ("lambda_num", "lambda_den"))
