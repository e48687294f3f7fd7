"""famsa_upgma_tree on the GPU against the oracle's UPGMA over the oracle's
distance matrix: merges, sizes and heights bit-exact (both sides round
each operation on its own, in the same order), on tie-heavy and plain
families, host and device outputs."""
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
                                dict(k=60, seed=4, root_len=12, alphabet=2, dup_frac=0.3),
                                dict(k=300, seed=8, root_len=8, alphabet=2, indel_rate=0.1, dup_frac=0.05),
                                dict(k=700, seed=41, root_len=60, alphabet=3, sub_rate=0.1),
                                dict(k=1000, seed=1, root_len=250)])
def test_upgma_matches_oracle(fg, kw):
    res, off = synth.family(**kw)
    want = oracle.upgma(oracle.distance_matrix(res, off))
    f = fg.pack_peq(res, off)
    try:
        got = fg.upgma_tree(f)
    finally:
        f.free()
    assert np.array_equal(got["merges"], want["merges"])
    assert np.array_equal(got["sizes"], want["sizes"])
    assert np.array_equal(got["heights"], want["heights"])


def test_upgma_disjoint_and_device(fg):
    import torch
    # every distance +inf: merges by lowest slots, heights +inf
    res = np.concatenate([np.full(7, c, np.uint8) for c in range(25)])
    off = np.arange(26, dtype=np.int64) * 7
    want = oracle.upgma(oracle.distance_matrix(res, off))
    f = fg.pack_peq(torch.from_numpy(res).cuda(), torch.from_numpy(off).cuda())
    try:
        got = fg.upgma_tree(f, device=True)
        torch.cuda.synchronize()
    finally:
        f.free()
    assert np.isinf(want["heights"]).all()
    for n in ("merges", "heights", "sizes"):
        assert np.array_equal(got[n].cpu().numpy(), want[n]), n
