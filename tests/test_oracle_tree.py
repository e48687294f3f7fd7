"""Pins for the oracle's single-linkage tree and merge list (CPU only).

FAMSA builds its guide tree by single linkage with SLINK (Methods,
"Determination of the guide tree").  The oracle computes the pointer
representation three independent ways (Sibson's insertion, naive
agglomeration, the minimax definition); here they are checked against each
other on tie-heavy families, against SciPy's single-linkage routine, against
closed-form special cases and against the invariants of the representation.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def fam_case(k, seed, **kw):
    res, off = synth.family(k, seed, **kw)
    lens = np.diff(off).astype(np.int32)
    return res, off, lens, oracle.lcs_allpairs(res, off)


TIE_CASES = [
    dict(k=1, seed=1, root_len=10),
    dict(k=2, seed=2, root_len=10),
    dict(k=3, seed=3, root_len=5, alphabet=2),
    dict(k=25, seed=4, root_len=12, alphabet=2, dup_frac=0.3),
    dict(k=80, seed=5, root_len=30, alphabet=3, dup_frac=0.2),
    dict(k=150, seed=6, root_len=20, alphabet=4, sub_rate=0.2),
    dict(k=200, seed=7, root_len=60),
    dict(k=300, seed=8, root_len=8, alphabet=2, indel_rate=0.1, dup_frac=0.05),
]


def as_frac(n, d):
    return None if d == 0 else Fraction(int(n), int(d))


@pytest.mark.parametrize("case", TIE_CASES, ids=lambda c: "k%d_s%d" % (c["k"], c["seed"]))
def test_three_routes_agree(case):
    case = dict(case)
    res, off, lens, tri = fam_case(case.pop("k"), case.pop("seed"), **case)
    a = oracle.slink_matrix(tri, lens)
    b = oracle.slink_naive(tri, lens)
    c = oracle.slink_definition(tri, lens)
    d = oracle.slink_streamed(res, off)
    for other in (b, c, d):
        for x, y in zip(a, other):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("case", TIE_CASES[2:], ids=lambda c: "k%d_s%d" % (c["k"], c["seed"]))
def test_pointer_invariants_and_ultrametric(case):
    case = dict(case)
    res, off, lens, tri = fam_case(case.pop("k"), case.pop("seed"), **case)
    k = len(lens)
    pi, ln, ld = oracle.slink_matrix(tri, lens)
    assert pi[k - 1] == k - 1 and ld[k - 1] == 0
    lam = [as_frac(ln[j], ld[j]) for j in range(k)]
    for j in range(k - 1):
        assert pi[j] > j
        p = pi[j]
        if p != k - 1:
            assert lam[j] is not None and (lam[p] is None or lam[j] < lam[p])
    # cophenetic distance from the merge list equals the minimax closure
    un, ud = oracle.minimax(tri, lens)
    pairs, hn, hd, sz = oracle.merges(pi, ln, ld)
    members = {i: [i] for i in range(k)}
    coph = [[None] * k for _ in range(k)]
    prev = Fraction(-1)
    for t in range(k - 1):
        h = as_frac(hn[t], hd[t])
        hh = Fraction(10 ** 30) if h is None else h
        assert hh >= prev
        prev = hh
        A, B = members.pop(int(pairs[t, 0])), members.pop(int(pairs[t, 1]))
        for x in A:
            for y in B:
                coph[x][y] = coph[y][x] = h
        members[k + t] = A + B
        assert sz[t] == len(A) + len(B)
    for x in range(k):
        for y in range(k):
            if x != y:
                assert coph[x][y] == as_frac(un[x, y], ud[x, y])
    # ultrametric inequality on a sample of triples
    rng = np.random.default_rng(1)
    big = Fraction(10 ** 30)
    for _ in range(2000):
        x, y, z = rng.integers(0, k, 3)
        if len({x, y, z}) < 3:
            continue
        f = lambda a, b: big if coph[a][b] is None else coph[a][b]  # noqa: E731
        assert f(x, z) <= max(f(x, y), f(y, z))


def test_special_cases():
    # k = 1: root only, no merges
    res, off, lens, tri = fam_case(1, 1, root_len=7)
    pi, ln, ld = oracle.slink_matrix(tri, lens)
    assert list(pi) == [0] and (ln[0], ld[0]) == (1, 0)
    assert len(oracle.merges(pi, ln, ld)[0]) == 0
    # all identical sequences: every lambda is 0 and pi(j) = k - 1
    k = 17
    seq = np.arange(20, dtype=np.uint8)
    res = np.tile(seq, k)
    off = np.arange(k + 1, dtype=np.int64) * 20
    tri = oracle.lcs_allpairs(res, off)
    pi, ln, ld = oracle.slink_matrix(tri, np.diff(off).astype(np.int32))
    assert (pi[:-1] == k - 1).all() and (ln[:-1] == 0).all() and (ld[:-1] == 1).all()
    pairs, hn, hd, sz = oracle.merges(pi, ln, ld)
    # fixed lowest-index order: j = 0, 1, 2, ... join the cluster of k-1 in turn
    assert pairs[0].tolist() == [0, k - 1] and pairs[1].tolist() == [1, k]
    assert sz.tolist() == list(range(2, k + 1))
    # disjoint alphabets: LCS 0 everywhere, all distances +inf
    res = np.concatenate([np.full(5, c, np.uint8) for c in range(6)])
    off = np.arange(7, dtype=np.int64) * 5
    tri = oracle.lcs_allpairs(res, off)
    assert (tri == 0).all()
    pi, ln, ld = oracle.slink_matrix(tri, np.diff(off).astype(np.int32))
    assert (pi == 5).all() and (ld == 0).all() and (ln == 1).all()
    # k = 2: one merge at the pair's distance, reduced
    res = np.array([0, 1, 2, 3, 0, 1, 9, 9, 3], np.uint8)
    off = np.array([0, 4, 9], np.int64)
    L = oracle.lcs(res[:4], res[4:])
    assert L == 3
    pi, ln, ld = oracle.slink_matrix(np.array([L], np.int32), np.array([4, 5], np.int32))
    indel = 4 + 5 - 2 * 3
    f = Fraction(indel * indel, L)
    assert pi.tolist() == [1, 1] and (ln[0], ld[0]) == (f.numerator, f.denominator)


def _scipy_linkage(tri, lens):
    hier = pytest.importorskip("scipy.cluster.hierarchy")
    k = len(lens)
    iu = np.triu_indices(k, 1)
    la, lb = lens[iu[0]].astype(np.int64), lens[iu[1]].astype(np.int64)
    indel = la + lb - 2 * tri.astype(np.int64)
    with np.errstate(divide="ignore"):
        d = np.where(tri > 0, (indel * indel).astype(np.float64) / np.maximum(tri, 1), np.inf)
    d = np.where(np.isinf(d), 1e300, d)
    return hier.linkage(d, method="single"), hier


@pytest.mark.parametrize("seed", [21, 22, 23])
def test_matches_scipy_single_linkage(seed):
    # Real-valued distances indel^2/LCS; distinct rationals of this size are
    # distinct, order-preserving doubles, so SciPy's heights must equal ours.
    res, off, lens, tri = fam_case(120, seed, root_len=80)
    Z, hier = _scipy_linkage(tri, lens)
    pi, ln, ld = oracle.slink_matrix(tri, lens)
    pairs, hn, hd, sz = oracle.merges(pi, ln, ld)
    ours = np.where(hd > 0, hn.astype(np.float64) / np.maximum(hd, 1), 1e300)
    assert np.array_equal(np.sort(ours), np.sort(Z[:, 2]))
    # flat clusters at every height agree
    k = len(lens)
    for t in np.unique(ours)[:: max(1, len(np.unique(ours)) // 25)]:
        sc = hier.fcluster(Z, t, criterion="distance")
        parent = list(range(k))

        def find(x):
            while parent[x] != x:
                x = parent[x]
            return x
        for j in range(k - 1):
            if ours_lam(ln[j], ld[j]) <= t:
                parent[find(j)] = find(int(pi[j]))
        mine = np.array([find(x) for x in range(k)])
        assert same_partition(mine, sc)
    # with distinct heights the merge sequence itself is unique: compare to SciPy's
    if len(np.unique(ours)) == k - 1:
        assert np.array_equal(np.sort(Z[:, :2].astype(np.int64), axis=1), pairs)
        assert np.array_equal(Z[:, 3].astype(np.int64), sz)


def ours_lam(n, d):
    return 1e300 if d == 0 else float(n) / float(d)


def same_partition(a, b):
    m1, m2 = {}, {}
    for x, y in zip(a, b):
        if m1.setdefault(x, y) != y or m2.setdefault(y, x) != x:
            return False
    return True


def test_distinct_heights_case_is_exercised():
    # a family with all-distinct pair keys so the strict merge-order comparison above runs
    found = False
    for seed in range(30, 60):
        res, off, lens, tri = fam_case(40, seed, root_len=400, sub_rate=0.3)
        pi, ln, ld = oracle.slink_matrix(tri, lens)
        h = ln.astype(np.float64)[:-1] / np.maximum(ld[:-1], 1)
        if len(np.unique(h)) == len(h):
            Z, _ = _scipy_linkage(tri, lens)
            pairs, hn, hd, sz = oracle.merges(pi, ln, ld)
            assert np.array_equal(np.sort(Z[:, :2].astype(np.int64), axis=1), pairs)
            found = True
            break
    assert found


def test_merges_fixed_tie_break():
    # three identical sequences and one far one: ties at height 0 resolve by index
    res = np.array([1, 2, 3, 1, 2, 3, 1, 2, 3, 9, 9, 9], np.uint8)
    off = np.array([0, 3, 6, 9, 12], np.int64)
    tri = oracle.lcs_allpairs(res, off)
    pi, ln, ld = oracle.slink_matrix(tri, np.diff(off).astype(np.int32))
    assert pi.tolist() == [2, 2, 3, 3]
    pairs, hn, hd, sz = oracle.merges(pi, ln, ld)
    assert pairs.tolist() == [[0, 2], [1, 4], [3, 5]]
    assert hn[:2].tolist() == [0, 0] and (hn[2], hd[2]) == (1, 0)
    assert sz.tolist() == [2, 3, 4]
