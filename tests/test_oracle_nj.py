"""Pins for the oracle's neighbour joining (CPU only).

NJ is exact on additive (tree) metrics: given the path lengths between the
leaves of a tree with positive edges it rejoins that tree, and its branch
lengths are the tree's edge lengths (Saitou & Nei; Studier & Keppler).  With
integer edge lengths every quantity NJ forms is exactly representable, so
the recovered topology (as a set of leaf bipartitions) and every edge length
are checked for equality.  A wrong Q criterion, a wrong sign or factor in the
branch formula or in the distance update breaks one of them.  Also pinned:
the three-point formula for k = 3, the tie order, the invariants of the merge
list, and the refusal of infinite distances.
"""
import numpy as np
import pytest

import oracle
import synth


def random_tree(k, rng, max_len=20):
    """A random rooted binary tree on leaves 0..k-1 by random joins: its
    children lists, integer edge lengths (to the parent) and the leaf distances."""
    nodes = list(range(k))
    children, elen = {}, {}
    nxt = k
    while len(nodes) > 1:
        i, j = sorted(rng.choice(len(nodes), 2, replace=False))
        a, b = nodes[i], nodes[j]
        children[nxt] = (a, b)
        elen[a] = int(rng.integers(1, max_len + 1))
        elen[b] = int(rng.integers(1, max_len + 1))
        nodes = [x for t, x in enumerate(nodes) if t not in (i, j)] + [nxt]
        nxt += 1
    root = nodes[0]
    # depth of every node, then leaf distances through the lowest common ancestor
    parent = {c: p for p, cs in children.items() for c in cs}
    def path(x):
        out = [x]
        while x in parent:
            x = parent[x]
            out.append(x)
        return out
    D = np.zeros((k, k))
    for a in range(k):
        pa = path(a)
        da = {x: sum(elen[y] for y in pa[:i]) for i, x in enumerate(pa)}
        for b in range(k):
            if a == b:
                continue
            pb = path(b)
            for i, x in enumerate(pb):
                if x in da:
                    D[a, b] = da[x] + sum(elen[y] for y in pb[:i])
                    break
    return children, elen, root, D


def splits_from_tree(k, children, elen, root):
    """{frozenset(side without leaf 0): length} of an unrooted view of a rooted
    binary tree (the root's two edges are one edge)."""
    leaves = {}
    def below(x):
        if x < k:
            return frozenset([x])
        if x not in leaves:
            a, b = children[x]
            leaves[x] = below(a) | below(b)
        return leaves[x]
    full = frozenset(range(k))
    out = {}
    for x in list(children) + list(range(k)):
        if x == root:
            continue
        s = below(x)
        side = s if 0 not in s else full - s
        out[side] = out.get(side, 0) + elen[x]
    return out


def splits_from_nj(k, nj):
    children, elen = {}, {}
    for t, ((a, b), (la, lb)) in enumerate(zip(nj["merges"], nj["lengths"])):
        children[k + t] = (int(a), int(b))
        elen[int(a)] = float(la)
        elen[int(b)] = float(lb)
    return splits_from_tree(k, children, elen, 2 * k - 2)


@pytest.mark.parametrize("k,seed", [(4, 1), (5, 2), (8, 3), (13, 4), (25, 5), (40, 6), (64, 7)])
def test_additive_metric_is_rejoined_exactly(k, seed):
    rng = np.random.default_rng(seed)
    children, elen, root, D = random_tree(k, rng)
    want = splits_from_tree(k, children, elen, root)
    got = splits_from_nj(k, oracle.nj(D))
    assert set(got) == set(want)
    for s, v in want.items():
        assert got[s] == v, (sorted(s), got[s], v)


def test_three_points():
    D = np.array([[0.0, 7.0, 11.0], [7.0, 0.0, 8.0], [11.0, 8.0, 0.0]])
    u = oracle.nj(D)
    # every Q ties at k = 3, so slots (0, 1) join first, on the three-point formula
    assert u["merges"].tolist() == [[0, 1], [2, 3]]
    d0 = (7.0 + 11.0 - 8.0) / 2
    assert u["lengths"][0].tolist() == [d0, 7.0 - d0]
    root = (11.0 + 8.0 - 7.0) / 2  # d(new node, 2), split evenly at the root
    assert u["lengths"][1].tolist() == [root / 2, root / 2]
    assert u["sizes"].tolist() == [2, 3]


def test_ties_take_the_lowest_slots():
    # four equidistant points: every Q is equal, so slots (0, 1) join (id 4
    # takes slot 0, at distance (6 + 6 - 6) / 2 = 3 from 2 and 3); at r = 3
    # all Q tie again and slots (0, 2) join, i.e. ids (2, 4); the root joins 3
    D = np.full((4, 4), 6.0)
    np.fill_diagonal(D, 0.0)
    u = oracle.nj(D)
    assert u["merges"].tolist() == [[0, 1], [2, 4], [3, 5]]
    assert u["sizes"].tolist() == [2, 3, 4]
    assert u["lengths"].tolist() == [[3.0, 3.0], [3.0, 0.0], [1.5, 1.5]]


@pytest.mark.parametrize("kw", [dict(k=60, seed=4, root_len=12, alphabet=4, dup_frac=0.3),
                                dict(k=150, seed=7, root_len=60)])
def test_invariants_on_families(kw):
    res, off = synth.family(**kw)
    k = len(off) - 1
    u = oracle.nj(oracle.distance_matrix(res, off))
    size = np.ones(2 * k - 1, np.int64)
    used = np.zeros(2 * k - 1, bool)
    for t, (a, b) in enumerate(u["merges"]):
        assert a < b < k + t and not used[a] and not used[b]
        used[a] = used[b] = True
        size[k + t] = size[a] + size[b]
        assert u["sizes"][t] == size[k + t]
    assert u["sizes"][-1] == k
    assert np.isfinite(u["lengths"]).all()
    # the root's two branches are equal halves
    assert u["lengths"][-1, 0] == u["lengths"][-1, 1]


def test_infinite_distance_is_refused():
    D = np.array([[0.0, np.inf, 3.0], [np.inf, 0.0, 4.0], [3.0, 4.0, 0.0]])
    with pytest.raises(RuntimeError, match="code -3"):
        oracle.nj(D)


def test_small_k():
    assert len(oracle.nj(np.zeros((1, 1)))["merges"]) == 0
    u = oracle.nj(np.array([[0.0, 5.0], [5.0, 0.0]]))
    assert u["merges"].tolist() == [[0, 1]] and u["lengths"].tolist() == [[2.5, 2.5]]
