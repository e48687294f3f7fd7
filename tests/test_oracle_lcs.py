"""Pins for the oracle's LCS and distance keys (CPU only).

The oracle's DP LCS (FAMSA Methods, "Pairwise similarities calculation") is
checked against brute-force subsequence enumeration, a textbook worked
example, closed forms and invariants; the distance key indel^2/LCS against
exact Fraction arithmetic.
"""
import itertools
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CODE = {c: i for i, c in enumerate(synth.ALPHABET)}


def enc(s):
    return np.array([CODE[c] for c in s], dtype=np.uint8)


def is_subseq(sub, s):
    it = iter(s)
    return all(c in it for c in sub)


def brute_lcs(a, b):
    """Longest subsequence of a (by enumeration of all index subsets) that is a subsequence of b."""
    a, b = list(a), list(b)
    best = 0
    for mask in range(1 << len(a)):
        n = bin(mask).count("1")
        if n <= best:
            continue
        sub = [a[i] for i in range(len(a)) if mask >> i & 1]
        if is_subseq(sub, b):
            best = n
    return best


def test_textbook_examples():
    with open(os.path.join(GOLDEN, "lcs_textbook.txt")) as f:
        rows = [ln.split(None, 3) for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 5
    for a, b, n, _note in rows:
        assert oracle.lcs(enc(a), enc(b)) == int(n), (a, b)


def test_brute_force_all_binary_strings():
    # every pair of strings over {0,1} with lengths 0..5
    strings = [s for n in range(6) for s in itertools.product((0, 1), repeat=n)]
    for a in strings:
        for b in strings:
            assert oracle.lcs(np.array(a, np.uint8), np.array(b, np.uint8)) == brute_lcs(a, b)


@pytest.mark.parametrize("alpha", [2, 3, 4, 25])
def test_brute_force_random_up_to_12(alpha):
    rng = random.Random(1000 + alpha)
    for _ in range(60):
        la, lb = rng.randint(0, 12), rng.randint(0, 12)
        a = [rng.randrange(alpha) for _ in range(la)]
        b = [rng.randrange(alpha) for _ in range(lb)]
        assert oracle.lcs(np.array(a, np.uint8), np.array(b, np.uint8)) == brute_lcs(a, b), (a, b)


def test_closed_forms_subsequence_and_foreign_insertions():
    rng = np.random.default_rng(7)
    for _ in range(50):
        n = int(rng.integers(1, 400))
        a = rng.integers(0, 20, n).astype(np.uint8)
        keep = rng.random(n) < rng.random()
        b = a[keep]
        assert oracle.lcs(a, b) == len(b)           # b is a subsequence of a
        # insert symbols that a does not use (codes 20..24): LCS stays |a|
        ins = rng.integers(20, 25, int(rng.integers(0, 50))).astype(np.uint8)
        pos = np.sort(rng.integers(0, n + 1, len(ins)))
        c = np.insert(a, pos, ins)
        assert oracle.lcs(a, c) == n
        assert oracle.lcs(c, a) == n


def test_invariants_on_families():
    res, off = synth.family(40, 11, root_len=60, alphabet=4, dup_frac=0.1)
    k = len(off) - 1
    lens = np.diff(off)
    tri = oracle.lcs_allpairs(res, off)
    m = oracle.tri_to_square(tri, k)
    for i in range(k):
        si = res[off[i]:off[i + 1]]
        assert oracle.lcs(si, si) == lens[i]
        m[i, i] = lens[i]
    assert (m == m.T).all()
    assert (m <= np.minimum.outer(lens, lens)).all()
    assert (m >= 0).all()
    # indel distance is a metric (triangle inequality)
    indel = lens[:, None] + lens[None, :] - 2 * m
    assert (indel >= 0).all() and (np.diag(indel) == 0).all()
    for j in range(k):
        assert (indel <= indel[:, [j]] + indel[[j], :]).all()


def test_superadditivity_and_disjoint():
    rng = np.random.default_rng(3)
    for _ in range(40):
        a1, a2, b1, b2 = (rng.integers(0, 4, int(rng.integers(0, 30))).astype(np.uint8)
                          for _ in range(4))
        lhs = oracle.lcs(np.concatenate([a1, a2]), np.concatenate([b1, b2]))
        assert lhs >= oracle.lcs(a1, b1) + oracle.lcs(a2, b2)
        c = rng.integers(0, 10, 50).astype(np.uint8)
        d = rng.integers(10, 25, 50).astype(np.uint8)
        assert oracle.lcs(c, d) == 0


def test_pairs_rows_allpairs_agree():
    res, off = synth.family(30, 5, root_len=70)
    k = len(off) - 1
    tri = oracle.lcs_allpairs(res, off)
    iu = np.triu_indices(k, 1)
    assert (oracle.lcs_pairs(res, off, iu[0], iu[1]) == tri).all()
    m = oracle.tri_to_square(tri, k)
    rows = oracle.lcs_rows(res, off, 7, 19)
    t = 0
    for i in range(7, 19):
        assert (rows[t:t + i] == m[i, :i]).all()
        t += i
    assert t == len(rows)
    for i in range(k):
        for j in range(k):
            if i != j:
                assert m[i, j] == oracle.lcs(res[off[i]:off[i + 1]], res[off[j]:off[j + 1]])


# ------------------------------------------------------------------ keys
def frac_key(lcs_len, la, lb):
    indel = la + lb - 2 * lcs_len
    return None if lcs_len == 0 else Fraction(indel * indel, lcs_len)  # None = +inf


def cmp_frac(x, y):
    if x is None and y is None:
        return 0
    if x is None:
        return 1
    if y is None:
        return -1
    return (x > y) - (x < y)


def test_key_order_matches_fractions():
    rng = random.Random(5)
    cases = []
    for _ in range(3000):
        la, lb = rng.randint(1, 65535), rng.randint(1, 65535)
        if rng.random() < 0.3:
            la, lb = rng.randint(1, 40), rng.randint(1, 40)
        cases.append((rng.randint(0, min(la, lb)), la, lb))
    cases += [(0, 5, 7), (3, 3, 3), (1, 65535, 65535), (0, 65535, 65535), (65535, 65535, 65535)]
    for i in range(len(cases) - 1):
        a, b = cases[i], cases[i + 1]
        want = cmp_frac(frac_key(*a), frac_key(*b))
        got = oracle.key_cmp(oracle.key(*a), oracle.key(*b))
        assert got == want, (a, b)


def test_key_special_values():
    inf = oracle.key(0, 10, 12)
    zero = oracle.key(10, 10, 10)          # identical sequences: indel 0
    assert inf == (1, 0) and zero == (0, 10)
    assert oracle.key_cmp(inf, oracle.key(0, 3, 4)) == 0      # +inf == +inf
    assert oracle.key_cmp(zero, oracle.key(5, 5, 5)) == 0     # 0/10 == 0/5
    assert oracle.key_cmp((4, 2), (2, 1)) == 0                # equal values, different forms
    assert oracle.key_cmp((36, 12), (9, 3)) == 0
    assert oracle.key_cmp(zero, (1, 65535)) == -1
    assert oracle.key_cmp(inf, (131070 ** 2, 1)) == 1
    big = 131070 ** 2
    assert oracle.key_cmp((big, 65535), (big - 1, 65535)) == 1
    assert oracle.key_cmp((big, 65534), (big, 65535)) == 1
    # similarity = LCS/indel^2 orders the opposite way to the key
    assert oracle.key_cmp(oracle.key(50, 60, 60), oracle.key(40, 60, 60)) == -1
