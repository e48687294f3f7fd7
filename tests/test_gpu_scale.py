"""Scale recipe (k=400,000 family, 25-letter alphabet with X/B/Z ambiguity codes).

A k=2,500 family from the same recipe is checked exactly against the oracle
on every row update.  Prefixes of the k=400,000 family (its first n
sequences) are checked bit-exactly against oracle tree digests stored by
tests/golden/make_scale_golden.py, whose SLINK runs on the oracle's own
bit-parallel LCS.  At the full k=400,000 (global-memory row update,
about 8e10 pairs streamed in row blocks), LCS rows sampled from the start, the
middle and the end are checked against the oracle's DP, and the tree against
properties that hold at any size:
  * pi(j) > j, the last point is its own pointer with lambda = +inf;
  * lambda(j) < lambda(pi(j)) unless both are +inf (Sibson's canonical form);
  * lambda(j) <= d(j, r) for every j < r of a sampled row r, because the
    single-link distance never exceeds the direct one;
  * merge heights non-decreasing, ids and sizes consistent, one final cluster.
"""
import hashlib
import json
import os

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
    yield m
    m.debug_set_update_path(0)


def _same(got, want):
    for key in ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den", "sizes"):
        g, w = np.asarray(got[key]), np.asarray(want[key])
        assert np.array_equal(g.reshape(w.shape), w), key


def test_scale_recipe_family_exact_both_paths(fg):
    res, off = synth.scale400k(2, k=2500)
    assert int(res.max()) >= 20  # ambiguity codes present
    want = oracle.tree(res, off)
    for path in (1, 2, 3):
        fg.debug_set_update_path(path)
        try:
            fam = fg.pack_peq(res, off)
            got = fg.slink_tree(fam)
            st = fam.stats()
            fam.free()
        finally:
            fg.debug_set_update_path(0)
        assert st["update_path"] == path
        _same(got, want)


@pytest.fixture(scope="module")
def full(fg):
    import torch
    res, off = synth.scale400k(1)
    fam = fg.pack_peq(torch.from_numpy(res).cuda(), torch.from_numpy(off).cuda())
    tree = fg.slink_tree(fam)
    st = fam.stats()
    yield res, off, fam, tree, st
    fam.free()


SAMPLED_ROWS = (1, 2, 1234, 200001, 399999)


@pytest.fixture(scope="module")
def oracle_rows(full):
    res, off = full[0], full[1]
    return {r: oracle.lcs_rows(res, off, r, r + 1) for r in SAMPLED_ROWS}


def test_scale400k_sampled_rows_against_oracle(fg, full, oracle_rows):
    res, off, fam, _, st = full
    k = len(off) - 1
    assert k == 400000 and st["update_path"] == 3 and st["pairs"] == k * (k - 1) // 2
    for r in SAMPLED_ROWS:
        got = np.asarray(fg.lcs_rows(fam, r, r + 1))
        assert np.array_equal(got, oracle_rows[r]), r


def _le(an, ad, bn, bd):
    """a <= b for exact fractions num/den (den 0 = +inf), elementwise."""
    an, ad, bn, bd = (np.asarray(x, dtype=np.int64) for x in (an, ad, bn, bd))
    a_inf, b_inf = ad == 0, bd == 0
    return np.where(b_inf, True, np.where(a_inf, False, an * bd <= bn * ad))


def test_scale400k_tree_properties(fg, full, oracle_rows):
    res, off, fam, t, _ = full
    k = len(off) - 1
    pi = np.asarray(t["pi"], dtype=np.int64)
    ln = np.asarray(t["lambda_num"], dtype=np.int64)
    ld = np.asarray(t["lambda_den"], dtype=np.int64)
    j = np.arange(k - 1)
    assert (pi[:-1] > j).all() and pi[-1] == k - 1 and ld[-1] == 0
    # canonical: lambda(j) < lambda(pi(j)), or both +inf
    p = pi[:-1]
    both_inf = (ld[:-1] == 0) & (ld[p] == 0)
    strict = _le(ln[:-1], ld[:-1], ln[p], ld[p]) & ~_le(ln[p], ld[p], ln[:-1], ld[:-1])
    assert (both_inf | strict).all()
    # lambda(j) <= d(j, r) for every j < r of the sampled rows
    lens = np.diff(off).astype(np.int64)
    for r in SAMPLED_ROWS:
        L = oracle_rows[r].astype(np.int64)
        indel = lens[:r] + lens[r] - 2 * L
        dn, dd = indel * indel, L
        assert _le(ln[:r], ld[:r], dn, dd).all(), r
    # merge list: heights non-decreasing, ids valid, sizes add up, one cluster
    mg = np.asarray(t["merges"], dtype=np.int64).reshape(k - 1, 2)
    hn = np.asarray(t["h_num"], dtype=np.int64)
    hd = np.asarray(t["h_den"], dtype=np.int64)
    assert _le(hn[:-1], hd[:-1], hn[1:], hd[1:]).all()
    ids = k + np.arange(k - 1)
    assert (mg[:, 0] < mg[:, 1]).all() and (mg[:, 1] < ids).all()
    size = np.ones(2 * k - 1, dtype=np.int64)
    sizes = np.asarray(t["sizes"], dtype=np.int64)
    used = np.zeros(2 * k - 1, dtype=bool)
    for tt in range(k - 1):  # plain loop: every cluster id is merged at most once
        a, b = mg[tt]
        assert not used[a] and not used[b]
        used[a] = used[b] = True
        size[k + tt] = size[a] + size[b]
    assert np.array_equal(size[k:], sizes) and sizes[-1] == k


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_trees.json")
PREFIX = "scale400k_seed1_prefix"


def _digest(t):
    h1 = hashlib.sha256()
    for a, dt in ((t["pi"], "<i4"), (t["lambda_num"], "<u8"), (t["lambda_den"], "<u4")):
        h1.update(np.ascontiguousarray(a).astype(dt).tobytes())
    h2 = hashlib.sha256()
    for a, dt in ((t["merges"], "<i4"), (t["h_num"], "<u8"), (t["h_den"], "<u4"),
                  (t["sizes"], "<i4")):
        h2.update(np.ascontiguousarray(a).astype(dt).tobytes())
    return h1.hexdigest(), h2.hexdigest()


def test_scale400k_prefix_trees_against_oracle_digests(fg, full):
    gold = json.load(open(GOLDEN)) if os.path.exists(GOLDEN) else {}
    ns = sorted(int(name[len(PREFIX):]) for name in gold if name.startswith(PREFIX))
    if not ns:
        pytest.skip("no oracle digest of a k=400,000 prefix stored yet")
    res, off = full[0], full[1]
    for n in ns:
        want = gold[PREFIX + str(n)]
        if n == len(off) - 1:
            got, st = full[3], full[4]
        else:
            fam = fg.pack_peq(res[:off[n]], off[:n + 1])
            got = fg.slink_tree(fam)
            st = fam.stats()
            fam.free()
        assert st["update_path"] == 3
        assert _digest(got) == (want["pi_lambda_sha256"], want["merges_sha256"]), n
