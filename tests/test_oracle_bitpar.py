"""Pins for the oracle's bit-parallel LCS and its streamed SLINK (CPU only).

The bit-parallel recurrence (FAMSA Methods, "Pairwise similarities
calculation") is a second, independent way to the LCS length; it serves the
oracle's trees of families too large for the DP.  It is pinned here against
the DP (itself pinned by brute force in test_oracle_lcs.py):
  * every pair of binary strings up to length 5, and random short strings;
  * every pair of the k=1,000 family;
  * lengths on both sides of every 64-bit word boundary up to 3,000, with
    2-, 4- and 25-letter alphabets and arbitrary byte codes;
and its trees against the DP-fed trees, including resumed runs and prefixes.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def test_all_binary_strings_up_to_5():
    strings = [s for n in range(6) for s in itertools.product((0, 1), repeat=n)]
    for a in strings:
        for b in strings:
            a8, b8 = np.array(a, np.uint8), np.array(b, np.uint8)
            assert oracle.lcs_bitpar(a8, b8) == oracle.lcs(a8, b8), (a, b)


def test_random_short_strings_many_alphabets():
    rng = np.random.default_rng(3)
    for sigma in (2, 3, 4, 25, 256):
        for _ in range(400):
            a = rng.integers(0, sigma, rng.integers(0, 14), dtype=np.uint8)
            b = rng.integers(0, sigma, rng.integers(0, 14), dtype=np.uint8)
            assert oracle.lcs_bitpar(a, b) == oracle.lcs(a, b)


def test_every_pair_of_the_1k_family():
    res, off = synth.plain1k(1)
    k = len(off) - 1
    iu = np.triu_indices(k, 1)
    want = oracle.lcs_allpairs(res, off)
    got = oracle.lcs_pairs_bitpar(res, off, iu[0], iu[1])
    assert np.array_equal(got, want)
    # the Peq side does not matter
    assert np.array_equal(oracle.lcs_pairs_bitpar(res, off, iu[1], iu[0]), want)


BOUNDARY_LENGTHS = sorted({n for w in range(1, 48) for n in (64 * w - 1, 64 * w, 64 * w + 1)
                           if n <= 3000} | {1, 2, 3000})


@pytest.mark.parametrize("sigma", [2, 4, 25])
def test_word_boundaries_up_to_3000(sigma):
    rng = np.random.default_rng(sigma)
    seqs = []
    for n in BOUNDARY_LENGTHS:
        seqs.append(rng.integers(0, sigma, n, dtype=np.uint8))
        # a mutated copy keeps long common runs, so carries travel across words
        m = seqs[-1].copy()
        flip = rng.random(n) < 0.05
        m[flip] = rng.integers(0, sigma, int(flip.sum()), dtype=np.uint8)
        seqs.append(m)
    off = np.zeros(len(seqs) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    res = np.concatenate(seqs)
    k = len(seqs)
    # every sequence against its mutated copy, its neighbours and a random partner
    pa, pb = [], []
    for i in range(0, k, 2):
        for j in (i + 1, min(i + 2, k - 1), min(i + 3, k - 1), int(rng.integers(0, k))):
            pa.append(i)
            pb.append(j)
    pa, pb = np.array(pa), np.array(pb)
    want = oracle.lcs_pairs(res, off, pa, pb)
    assert np.array_equal(oracle.lcs_pairs_bitpar(res, off, pa, pb), want)
    assert np.array_equal(oracle.lcs_pairs_bitpar(res, off, pb, pa), want)


def test_all_ones_carry_runs():
    # A = all the same letter: V + (V & Peq) carries through whole words at once
    for n in (63, 64, 65, 128, 129, 200, 640):
        a = np.zeros(n, np.uint8)
        for m in (1, 63, 64, 65, 300):
            b = np.zeros(m, np.uint8)
            assert oracle.lcs_bitpar(a, b) == min(n, m)
            b[::2] = 1
            assert oracle.lcs_bitpar(a, b) == oracle.lcs(a, b)


def _same(got, want):
    for key in ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den", "sizes"):
        assert np.array_equal(np.asarray(got[key]), np.asarray(want[key])), key


def test_tree_bitpar_equals_dp_tree():
    res, off = synth.plain1k(1)
    _same(oracle.tree_bitpar(res, off), oracle.tree(res, off))
    for kw in (dict(k=25, seed=4, root_len=12, alphabet=2, dup_frac=0.3),
               dict(k=80, seed=5, root_len=30, alphabet=3, dup_frac=0.2),
               dict(k=150, seed=6, root_len=20, alphabet=4, sub_rate=0.2),
               dict(k=60, seed=9, root_len=400, alphabet=2, sub_rate=0.1)):
        res, off = synth.family(**kw)
        _same(oracle.tree_bitpar(res, off), oracle.tree(res, off))


def test_resumed_ranges_and_prefixes():
    res, off = synth.plain1k(2)
    k = len(off) - 1
    one = oracle.slink_state(k)
    oracle.slink_bitpar_range(res, off, one, 0, k)
    parts = oracle.slink_state(k)
    for n0, n1 in ((0, 1), (1, 333), (333, 334), (334, 1000)):
        oracle.slink_bitpar_range(res, off, parts, n0, n1)
        if n1 == 333:
            # after n insertions the state is the tree of the first n sequences
            pre = {name: a[:333].copy() for name, a in parts.items()}
            _same(oracle.tree_from_state(pre), oracle.tree(res[:off[333]], off[:334]))
    for name in one:
        assert np.array_equal(one[name], parts[name])
    _same(oracle.tree_from_state(one), oracle.tree(res, off))
