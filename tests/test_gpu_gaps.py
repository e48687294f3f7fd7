"""famsa_gap_types, famsa_gap_insert and famsa_gap_cost on the GPU against
the oracle on random alignments (exact for the byte outputs; the scaled
costs within 1e-14 relative: the device and host logarithms may differ in
the last bit, and the rest of the arithmetic is exact sums of small integer
multiples rounded once)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    from paper_1603_06958_gb300 import build
    build.build()
    import paper_1603_06958_gb300 as m
    m.load()
    return m


def _aln(rng, m, n, p_gap):
    a = rng.integers(0, 25, (m, n)).astype(np.uint8)
    runs = rng.random((m, n)) < p_gap
    a[runs] = oracle.GAP
    a[: max(1, m // 50)] = oracle.GAP  # a few rows of gaps only
    return a


@pytest.mark.parametrize("m,n,p", [(1, 1, 0.5), (7, 3, 0.3), (1000, 300, 0.3), (5000, 64, 0.6)])
def test_types_insert_and_cost_match_oracle(fg, m, n, p):
    import torch
    rng = np.random.default_rng(m + n)
    a = _aln(rng, m, n, p)
    da = torch.from_numpy(a).cuda()
    t = fg.gap_types(da)
    want_t = oracle.gap_types(a)
    assert np.array_equal(t.cpu().numpy(), want_t)
    for c in (0, 1, 5, 40):
        pos = np.sort(rng.integers(0, n + 1, c)).astype(np.int32)
        ao, to = fg.gap_insert(da, t, pos)
        wa, wt = oracle.gap_insert(a, want_t, pos)
        assert np.array_equal(ao.cpu().numpy(), wa) and np.array_equal(to.cpu().numpy(), wt)
    for k in (10, 45, 20000, 400000):
        got = fg.gap_cost(t, k, [10.0, 1.0, 5.0, 0.5]).cpu().numpy()
        want = oracle.gap_cost(want_t, k, [10.0, 1.0, 5.0, 0.5])
        assert np.allclose(got, want, rtol=1e-14, atol=0)
        assert fg.gap_scale(k) == pytest.approx(oracle.gap_scale(k), rel=1e-15)


def test_gap_insert_rejects_bad_positions(fg):
    import torch
    a = torch.zeros((2, 5), dtype=torch.uint8, device="cuda")
    t = fg.gap_types(a)
    for pos in ([3, 1], [6], [-1]):
        with pytest.raises(fg.FamsaError) as ei:
            fg.gap_insert(a, t, pos)
        assert ei.value.status == fg.FAMSA_EINVAL
