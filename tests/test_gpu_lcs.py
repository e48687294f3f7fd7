"""GPU parity of the LCS kernels against the oracle's DP (bit-exact, int32).

Covers thread-per-pair, sliced and warp-per-pair kernels at every word boundary,
ragged tails, tie-heavy small alphabets, ambiguity codes, host and device
buffers, row bands, query scoring and the error paths of the C ABI.
"""
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
    m.debug_set_tpp_max_w(32)
    m.debug_set_slices(24, 0)


def family_from(seqs):
    off = np.zeros(len(seqs) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    res = np.concatenate([np.asarray(s, np.uint8) for s in seqs]) if seqs else np.zeros(0, np.uint8)
    return res, off


def boundary_family(seed, alphabet=25, extra=()):
    rng = np.random.default_rng(seed)
    lens = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 191, 192, 193, 255, 256, 257, 511, 512,
            513, 1023, 1024, 1025, 2047, 2048, 2049, 3000] + list(extra)
    seqs = [rng.integers(0, alphabet, n).astype(np.uint8) for n in lens]
    # related sequences so LCS values are large, not just random-level
    for n in (64, 300, 1100, 2100):
        base = rng.integers(0, alphabet, n).astype(np.uint8)
        for _ in range(3):
            s = base.copy()
            idx = rng.random(n) < 0.1
            s[idx] = rng.integers(0, alphabet, idx.sum())
            keep = rng.random(n) > 0.05
            seqs.append(s[keep])
    return family_from(seqs)


def check_allpairs(fg, res, off, device=False):
    fam = fg.pack_peq(res, off)
    got = fg.lcs_allpairs(fam, device=device)
    if device:
        got = got.cpu().numpy()
    want = oracle.lcs_allpairs(res, off)
    assert got.shape == want.shape
    bad = np.nonzero(got != want)[0]
    assert len(bad) == 0, (bad[:10], got[bad[:10]], want[bad[:10]])
    fam.free()


@pytest.mark.parametrize("alphabet", [25, 4, 2])
def test_allpairs_word_boundaries(fg, alphabet):
    res, off = boundary_family(1 + alphabet, alphabet)
    check_allpairs(fg, res, off)


@pytest.mark.parametrize("tmax", [0, 1, 2, 5])
def test_warp_per_pair_matches(fg, tmax):
    # with slices off, rows wider than tmax words go through the warp-per-pair kernel
    fg.debug_set_tpp_max_w(tmax)
    fg.debug_set_slices(0)
    try:
        res, off = boundary_family(40 + tmax)
        check_allpairs(fg, res, off)
    finally:
        fg.debug_set_tpp_max_w(32)
        fg.debug_set_slices(24, 0)


@pytest.mark.parametrize("min_w,words", [(1, 1), (1, 2), (2, 3), (1, 5), (1, 16), (24, 0)])
def test_sliced_matches(fg, min_w, words):
    # rows of at least min_w words split over warps of at most `words` words:
    # one slice (W <= words), two, and up to 16 (W = 47 in slices of 3); the
    # carries cross slices at every word boundary of the family's lengths
    fg.debug_set_slices(min_w, words)
    try:
        for alphabet in (25, 2):
            res, off = boundary_family(60 + min_w + words + alphabet, alphabet, extra=(1300, 1344, 1345))
            check_allpairs(fg, res, off)
    finally:
        fg.debug_set_slices(24, 0)


@pytest.mark.parametrize("rows", [1, 2, 4])
def test_rows_per_tile_choices(fg, rows):
    # every (width, rows per tile) kernel the autotuner may pick gives the same LCS
    try:
        for w in range(1, 33):
            fg.debug_set_tpp_rows(w, rows if rows * w <= 32 else 0)
        assert fg.debug_tpp_rows(8) == rows and fg.debug_tpp_rows(16) == (rows if rows * 16 <= 32 else 1)
        res, off = boundary_family(77, extra=(700, 900, 1500))
        check_allpairs(fg, res, off)
    finally:
        for w in range(1, 33):
            fg.debug_set_tpp_rows(w, 0)


def test_long_sequences_default_kernels(fg):
    # rows of 33..141 words take the sliced kernel (2 to 9 slices), the one of
    # 16,385 residues (257 words) warp-per-pair
    rng = np.random.default_rng(9)
    seqs = [rng.integers(0, 20, n).astype(np.uint8) for n in (2100, 4096, 4097, 6000, 100, 9000, 16385)]
    seqs.append(seqs[3][::2].copy())
    seqs.append(np.concatenate([seqs[5], seqs[3][:7385]]))  # shares 9,000 + residues with two rows
    res, off = family_from(seqs)
    check_allpairs(fg, res, off)


def test_small_k_and_identical(fg):
    for seqs in ([[3]], [[3], [3]], [[1, 2], [2, 1], [1, 2]], [[5] * 70] * 5,
                 [[0] * 10, [1] * 10, [2] * 10]):
        res, off = family_from(seqs)
        if len(seqs) == 1:
            fam = fg.pack_peq(res, off)
            assert len(fg.lcs_allpairs(fam)) == 0
            fam.free()
        else:
            check_allpairs(fg, res, off)


def test_plain1k_full_and_device_buffers(fg):
    import torch
    res, off = synth.plain1k(1)
    want = oracle.lcs_allpairs(res, off)
    fam = fg.pack_peq(torch.from_numpy(res).cuda(), torch.from_numpy(off).cuda())
    got = fg.lcs_allpairs(fam, device=True)
    torch.cuda.synchronize()
    assert np.array_equal(got.cpu().numpy(), want)
    fam2 = fg.pack_peq(res, off)
    assert np.array_equal(fg.lcs_allpairs(fam2), want)


def test_ambiguity_and_scale_alphabet(fg):
    res, off = synth.scale400k(1, k=300)
    check_allpairs(fg, res, off)


@pytest.mark.parametrize("k,root_len", [(400, 120), (120, 1800)])
def test_rows_band(fg, k, root_len):
    # short rows (thread-per-pair) and rows of 24-32 words (sliced kernel)
    res, off = synth.family(k, 3, root_len=root_len, alphabet=0, ext_frac=0.2)
    fam = fg.pack_peq(res, off)
    for r0, r1 in ((0, 1), (0, 5), (37, 61), (k - 10, k), (0, k)):
        got = fg.lcs_rows(fam, r0, r1)
        want = oracle.lcs_rows(res, off, r0, r1)
        assert np.array_equal(got, want), (r0, r1)


@pytest.mark.parametrize("qlen", [180, 2000])
def test_query(fg, qlen):
    # queries of 3 words (thread-per-pair) and of about 32 words (sliced)
    res, off = synth.family(300, 4, root_len=200)
    q, qoff = synth.family(17, 5, root_len=qlen)
    fam = fg.pack_peq(res, off)
    got = fg.lcs_query(fam, q, qoff)
    k, nq = len(off) - 1, len(qoff) - 1
    allres = np.concatenate([q, res])
    alloff = np.concatenate([qoff, off[1:] + qoff[-1]])
    pa = np.repeat(np.arange(nq), k)
    pb = np.tile(np.arange(k), nq) + nq
    want = oracle.lcs_pairs(allres, alloff, pa, pb).reshape(nq, k)
    assert np.array_equal(got, want)


def test_error_paths(fg):
    res, off = family_from([[1, 2, 3], [4, 25, 6]])       # code 25 is invalid
    with pytest.raises(fg.FamsaError) as e:
        fg.pack_peq(res, off)
    assert e.value.status == fg.FAMSA_EINVAL
    import torch
    dres = torch.from_numpy(np.zeros(70000, np.uint8)).cuda()
    doff = torch.tensor([0, 70000], dtype=torch.int64).cuda()
    with pytest.raises(fg.FamsaError) as e:
        fg.pack_peq(dres, doff)                            # device input, too long
    assert e.value.status == fg.FAMSA_ERANGE
    doff = torch.tensor([0, 5, 5, 9], dtype=torch.int64).cuda()
    with pytest.raises(fg.FamsaError) as e:
        fg.pack_peq(dres[:9].contiguous(), doff)           # device input, empty sequence
    assert e.value.status == fg.FAMSA_EINVAL
    res, off = family_from([[1, 2, 3], [4, 5, 6]])
    fam = fg.pack_peq(res, off)
    with pytest.raises(fg.FamsaError):
        fg.lcs_rows(fam, 1, 3)                             # row_end > k
    fam.free()
    # allocation failure while packing leaves nothing behind and reports ENOMEM
    fg.debug_fail_alloc_after(2)
    try:
        with pytest.raises(fg.FamsaError) as e:
            fg.pack_peq(res, off)
        assert e.value.status == fg.FAMSA_ENOMEM
    finally:
        fg.debug_fail_alloc_after(-1)
    fam = fg.pack_peq(res, off)                            # and the library still works
    assert fg.lcs_allpairs(fam).tolist() == [0]


def test_plain20k_sampled_pairs(fg):
    # full-size family of the benchmark; all 2e8 pairs on the GPU, a seeded
    # sample of them recomputed by the oracle's DP
    import torch
    res, off = synth.plain20k(1)
    fam = fg.pack_peq(res, off)
    got = fg.lcs_allpairs(fam, device=True)
    k = len(off) - 1
    rng = np.random.default_rng(20)
    i = rng.integers(0, k, 3000)
    j = rng.integers(0, k, 3000)
    keep = i != j
    a, b = np.minimum(i, j)[keep], np.maximum(i, j)[keep]
    idx = a.astype(np.int64) * k - a.astype(np.int64) * (a + 1) // 2 + (b - a - 1)
    sample = got[torch.from_numpy(idx).cuda()].cpu().numpy()
    want = oracle.lcs_pairs(res, off, a, b)
    assert np.array_equal(sample, want)


@pytest.mark.parametrize("slices", [24, 0])
def test_wide_rows_sliced_or_whole(fg, slices):
    # rows of 23..29 words: from 24 words on they run sliced by default, with
    # slices off thread-per-pair takes them whole; both forms equal the oracle
    rng = np.random.default_rng(77)
    base = rng.integers(0, 20, 1900).astype(np.uint8)
    seqs = []
    for n in range(1450, 1880, 24):
        s = base[:n].copy()
        flip = rng.random(n) < 0.15
        s[flip] = rng.integers(0, 20, int(flip.sum()))
        seqs.append(s)
    res, off = family_from(seqs)
    fg.debug_set_slices(slices)
    try:
        fam = fg.pack_peq(res, off)
        got = np.asarray(fg.lcs_allpairs(fam))
        fam.free()
    finally:
        fg.debug_set_slices(24, 0)
    assert np.array_equal(got, oracle.lcs_allpairs(res, off))
