"""Pins for the oracle's progressive-stage schedule (CPU only).

Constructed trees with known levels (a caterpillar: one level per merge; a
balanced tree of 2^m sequences: m levels of halving width), a recursive
height computed independently in Python on the oracle's own trees, and the
invariants the schedule promises: children sit on lower levels, each merge
has a child exactly one level down, a level never uses its own merges, the
order is sorted by (level, index) and level_start delimits it, and kind
counts the profiles among the two children.
"""
import numpy as np
import pytest

import oracle
import synth


def test_caterpillar():
    k = 9
    mg = [(0, 1)] + [(i + 1, k + i - 1) for i in range(1, k - 1)]
    s = oracle.schedule(np.array(mg), np.arange(2, k + 1))
    assert s["level"].tolist() == list(range(1, k))
    assert s["order"].tolist() == list(range(k - 1))
    assert s["level_start"].tolist() == list(range(k))
    assert s["kind"].tolist() == [0] + [1] * (k - 2)


def test_balanced_tree():
    m = 4
    k = 1 << m
    mg, sizes, ids = [], [], list(range(k))
    nxt = k
    while len(ids) > 1:
        new = []
        for a, b in zip(ids[::2], ids[1::2]):
            mg.append((a, b))
            sizes.append((sizes[a - k] if a >= k else 1) + (sizes[b - k] if b >= k else 1))
            new.append(nxt)
            nxt += 1
        ids = new
    s = oracle.schedule(np.array(mg), np.array(sizes))
    assert s["n_levels"] == m
    widths = np.diff(s["level_start"]).tolist()
    assert widths == [k >> (l + 1) for l in range(m)]
    assert (s["kind"][: k // 2] == 0).all() and (s["kind"][k // 2:] == 2).all()


def _height(mg, k):
    memo = {}

    def h(node):
        if node < k:
            return 0
        if node not in memo:
            a, b = mg[node - k]
            memo[node] = 1 + max(h(a), h(b))
        return memo[node]
    return [h(k + t) for t in range(len(mg))]


@pytest.mark.parametrize("kw", [dict(k=300, seed=8, root_len=8, alphabet=2, indel_rate=0.1, dup_frac=0.05),
                                dict(k=400, seed=11, root_len=150, alphabet=4, dup_frac=0.05),
                                dict(k=250, seed=3, root_len=200)])
def test_oracle_trees(kw):
    res, off = synth.family(**kw)
    t = oracle.tree(res, off)
    k = len(off) - 1
    mg = t["merges"].tolist()
    s = oracle.schedule(t["merges"], t["sizes"])
    lev = s["level"]
    assert lev.tolist() == _height(mg, k)
    size = lambda x: 1 if x < k else int(t["sizes"][x - k])  # noqa: E731
    for tt, (a, b) in enumerate(mg):
        la = 0 if a < k else lev[a - k]
        lb = 0 if b < k else lev[b - k]
        assert max(la, lb) == lev[tt] - 1
        assert s["kind"][tt] == (size(a) > 1) + (size(b) > 1)
    order = s["order"].tolist()
    assert sorted(order) == list(range(k - 1))
    assert order == sorted(order, key=lambda x: (lev[x], x))
    st = s["level_start"]
    assert st[0] == 0 and st[-1] == k - 1 and len(st) == s["n_levels"] + 1
    for l in range(1, s["n_levels"] + 1):
        block = order[st[l - 1]:st[l]]
        assert block and all(lev[x] == l for x in block)
        ids = {k + x for x in block}
        assert not any(a in ids or b in ids for x in block for a, b in [mg[x]])


def test_bad_merge_list():
    with pytest.raises(RuntimeError):
        oracle.schedule(np.array([[0, 1], [2, 5]]), np.array([2, 3]))
