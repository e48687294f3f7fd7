"""Pins for the oracle's UPGMA (CPU only): a textbook worked example (five
taxa with the merges at 17, 22, 28 and 33), SciPy's average linkage (an
independent implementation of UPGMA) on matrices with distinct distances,
and the invariants: heights never decrease, sizes add up, ids are fresh."""
import numpy as np
import pytest

import oracle
import synth


def test_textbook_five_taxa():
    # the classic worked example of UPGMA (a..e), merges (a,b), (ab,e), (c,d), (abe,cd)
    names = "abcde"
    d = {("a", "b"): 17, ("a", "c"): 21, ("a", "d"): 31, ("a", "e"): 23, ("b", "c"): 30,
         ("b", "d"): 34, ("b", "e"): 21, ("c", "d"): 28, ("c", "e"): 39, ("d", "e"): 43}
    D = np.zeros((5, 5))
    for (x, y), v in d.items():
        D[names.index(x), names.index(y)] = D[names.index(y), names.index(x)] = v
    u = oracle.upgma(D)
    assert u["merges"].tolist() == [[0, 1], [4, 5], [2, 3], [6, 7]]
    assert u["heights"].tolist() == [17.0, 22.0, 28.0, 33.0]
    assert u["sizes"].tolist() == [2, 3, 2, 5]


def test_scipy_average_linkage():
    hier = pytest.importorskip("scipy.cluster.hierarchy")
    dist = pytest.importorskip("scipy.spatial.distance")
    # random distinct distances (sequence families tie too often for a unique tree)
    rng = np.random.default_rng(3)
    k = 90
    D = np.zeros((k, k))
    iu = np.triu_indices(k, 1)
    D[iu] = rng.permutation(len(iu[0])) + rng.random(len(iu[0]))
    D = D + D.T
    assert len(set(D[iu].tolist())) == len(D[iu])
    u = oracle.upgma(D)
    Z = hier.linkage(dist.squareform(D, checks=False), method="average")
    assert np.allclose(u["heights"], Z[:, 2], rtol=1e-12, atol=0)
    assert np.array_equal(u["merges"], np.sort(Z[:, :2].astype(np.int32), axis=1))
    assert np.array_equal(u["sizes"], Z[:, 3].astype(np.int32))


@pytest.mark.parametrize("kw", [dict(k=60, seed=4, root_len=12, alphabet=2, dup_frac=0.3),
                                dict(k=120, seed=7, root_len=60)])
def test_invariants_and_distances(kw):
    res, off = synth.family(**kw)
    k = len(off) - 1
    D = oracle.distance_matrix(res, off)
    lens = np.diff(off).astype(np.int64)
    tri = oracle.lcs_allpairs(res, off).astype(np.int64)
    iu = np.triu_indices(k, 1)
    indel = lens[iu[0]] + lens[iu[1]] - 2 * tri
    want = np.where(tri == 0, np.inf, (indel * indel) / np.where(tri == 0, 1, tri))
    assert np.array_equal(D[iu], want) and np.array_equal(D, D.T)
    u = oracle.upgma(D)
    assert (np.diff(u["heights"]) >= 0).all()
    size = np.ones(2 * k - 1, np.int64)
    used = np.zeros(2 * k - 1, bool)
    for t, (a, b) in enumerate(u["merges"]):
        assert a < b < k + t and not used[a] and not used[b]
        used[a] = used[b] = True
        size[k + t] = size[a] + size[b]
    assert np.array_equal(size[k:], u["sizes"]) and u["sizes"][-1] == k
