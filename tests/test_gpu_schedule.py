"""famsa_progressive_schedule on the GPU against the oracle's schedule, on
the trees the GPU builds (exactly the oracle's), host and device buffers,
the degenerate sizes and a bad merge list."""
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


def _same(got, want):
    for key in ("level", "order", "level_start", "kind"):
        assert np.array_equal(np.asarray(got[key]), np.asarray(want[key])), key
    assert got["n_levels"] == want["n_levels"]


@pytest.mark.parametrize("kw", [dict(k=2, seed=1, root_len=30),
                                dict(k=300, seed=8, root_len=8, alphabet=2, indel_rate=0.1, dup_frac=0.05),
                                dict(k=1000, seed=1, root_len=250),
                                dict(k=3000, seed=5, root_len=120, alphabet=4)])
def test_schedule_matches_oracle(fg, kw):
    res, off = synth.family(**kw)
    f = fg.pack_peq(res, off)
    t = fg.slink_tree(f)
    f.free()
    want = oracle.schedule(t["merges"], t["sizes"])
    _same(fg.progressive_schedule(t), want)


def test_schedule_large_tree_and_device_buffers(fg):
    # 60,000 merges: the levels no longer fit shared memory
    import torch
    res, off = synth.plain20k(3, k=60001)
    f = fg.pack_peq(torch.from_numpy(res).cuda(), torch.from_numpy(off).cuda())
    t = fg.slink_tree(f, device=True)
    f.free()
    got = fg.progressive_schedule(t, device=True)
    torch.cuda.synchronize()
    host = {n: (v.cpu().numpy() if hasattr(v, "cpu") else v) for n, v in got.items()}
    want = oracle.schedule(t["merges"].cpu().numpy(), t["sizes"].cpu().numpy())
    _same(host, want)
    # at least half the merges of a large family are degenerate (a single sequence)
    assert (want["kind"] < 2).mean() >= 0.5


def test_schedule_single_point_and_bad_list(fg):
    s = fg.progressive_schedule({"merges": np.zeros((0, 2), np.int32), "sizes": np.zeros(0, np.int32)})
    assert s["n_levels"] == 0
    with pytest.raises(fg.FamsaError) as ei:
        fg.progressive_schedule({"merges": np.array([[0, 1], [2, 5]], np.int32),
                                 "sizes": np.array([2, 3], np.int32)})
    assert ei.value.status == fg.FAMSA_EINVAL
