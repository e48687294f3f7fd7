"""famsa_nj_tree on the GPU against the oracle's neighbour joining over the
oracle's distance matrix: merges, sizes and branch lengths bit-exact (both
sides round each operation on its own, in the same order), on tie-heavy and
plain families, host and device outputs, and the refusal of an infinite
distance."""
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


@pytest.mark.parametrize("kw", [dict(k=2, seed=1, root_len=30),
                                dict(k=3, seed=2, root_len=5, alphabet=2),
                                dict(k=4, seed=3, root_len=40),
                                dict(k=60, seed=4, root_len=12, alphabet=2, dup_frac=0.3),
                                dict(k=300, seed=8, root_len=20, alphabet=3, indel_rate=0.1, dup_frac=0.05),
                                dict(k=700, seed=41, root_len=60, alphabet=4, sub_rate=0.1),
                                dict(k=1000, seed=1, root_len=250)])
def test_nj_matches_oracle(fg, kw):
    res, off = synth.family(**kw)
    want = oracle.nj(oracle.distance_matrix(res, off))
    f = fg.pack_peq(res, off)
    try:
        got = fg.nj_tree(f)
    finally:
        f.free()
    assert np.array_equal(got["merges"], want["merges"])
    assert np.array_equal(got["sizes"], want["sizes"])
    assert np.array_equal(got["lengths"], want["lengths"])


def test_nj_device_outputs_and_long_rows(fg):
    import torch
    # rows of up to 2,600 residues (sliced LCS) and one duplicate pair
    res, off = synth.family(120, 11, root_len=2400, clip_hi=2600, dup_frac=0.03)
    want = oracle.nj(oracle.distance_matrix(res, off))
    f = fg.pack_peq(torch.from_numpy(res).cuda(), torch.from_numpy(off).cuda())
    try:
        got = fg.nj_tree(f, device=True)
        torch.cuda.synchronize()
    finally:
        f.free()
    for n in ("merges", "lengths", "sizes"):
        assert np.array_equal(got[n].cpu().numpy(), want[n]), n


def test_nj_infinite_distance_is_refused(fg):
    # two sequences over disjoint letters: LCS 0, an infinite distance
    res = np.array([0, 0, 0, 1, 1, 1, 0, 1], np.uint8)
    off = np.array([0, 3, 6, 8], np.int64)
    f = fg.pack_peq(res, off)
    try:
        with pytest.raises(fg.FamsaError) as e:
            fg.nj_tree(f)
        assert e.value.status == fg.FAMSA_ERANGE
    finally:
        f.free()
