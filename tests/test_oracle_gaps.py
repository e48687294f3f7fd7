"""Pins for the oracle's gap helpers (CPU only): the four gap types, the six
insertion corrections S1..S6 and the set-size scaling ("Gap types and costs
determination").

Worked rows classify as the type definitions say; each case S1..S6 is built
on a row that shows it, with the outcome the paper states; and, on random
rows and insertion sets, the corrections give exactly the classification of
the new row (the reading that the corrections keep the types consistent).
g_scale is 1 at k = g_l and grows by 1 for every factor e^g_d (natural log).
"""
import math

import numpy as np
import pytest

import oracle

G = oracle.GAP
TO, TE, GO, GE = 1, 2, 3, 4


def row(s):
    return np.array([[G if c == "-" else 1 for c in s]], np.uint8)


@pytest.mark.parametrize("s,want", [
    ("--AB-C--", [TO, TE, 0, 0, GO, 0, TO, TE]),
    ("A--B---C", [0, GO, GE, 0, GO, GE, GE, 0]),
    ("---", [TO, TE, TE]),
    ("ABC", [0, 0, 0]),
    ("-A-", [TO, 0, TO]),
])
def test_worked_rows(s, want):
    assert oracle.gap_types(row(s))[0].tolist() == want


def _insert(s, pos):
    a = row(s)
    return oracle.gap_insert(a, oracle.gap_types(a), [pos])[1][0].tolist()


def test_the_six_cases():
    # S1: a T_o right of the new gap -> the new gap is T_o and the old one T_e
    assert _insert("AB--", 2) == [0, 0, TO, TE, TE]
    assert _insert("--AB", 0) == [TO, TE, TE, 0, 0]
    # S2: a T_e left of it -> T_e
    assert _insert("A---", 4) == [0, TO, TE, TE, TE]
    # S3: inside a run of gaps -> G_e
    assert _insert("A--B", 2) == [0, GO, GE, GE, 0]
    # S4: a G_o right of it -> G_o, and the old G_o becomes G_e
    assert _insert("A--B", 1) == [0, GO, GE, GE, 0]
    assert _insert("AB-C", 2) == [0, 0, GO, GE, 0]
    # S5: alone between residues -> G_o
    assert _insert("ABC", 1) == [0, GO, 0, 0]
    # S6: a T_o left of it -> T_e
    assert _insert("A-", 2) == [0, TO, TE]
    assert _insert("-A", 1) == [TO, TE, 0]
    # a new run at an end of the row is terminal
    assert _insert("AB", 0) == [TO, 0, 0] and _insert("AB", 2) == [0, 0, TO]


def test_corrections_keep_the_classification():
    rng = np.random.default_rng(5)
    for _ in range(300):
        m, n = int(rng.integers(1, 6)), int(rng.integers(0, 25))
        a = np.where(rng.random((m, n)) < rng.random(), G, rng.integers(0, 25, (m, n))).astype(np.uint8)
        c = int(rng.integers(0, 8))
        pos = np.sort(rng.integers(0, n + 1, c)).astype(np.int32)
        ao, to = oracle.gap_insert(a, oracle.gap_types(a), pos)
        assert np.array_equal(to, oracle.gap_types(ao))
        # the residues keep their order, and exactly c gap columns were added
        for r in range(m):
            assert ao[r][ao[r] != G].tolist() == a[r][a[r] != G].tolist()
        assert ao.shape == (m, n + c) and ((ao == G).sum() - (a == G).sum()) == m * c


def test_gap_scale_and_cost():
    assert oracle.gap_scale(45) == 1.0
    assert abs(oracle.gap_scale(round(45 * math.exp(7))) - 2.0) < 1e-4
    ks = [1, 10, 45, 100, 1000, 10 ** 5, 4 * 10 ** 5]
    sc = [oracle.gap_scale(k) for k in ks]
    assert sc == sorted(sc)
    t = oracle.gap_types(row("--AB-C--A---B"))
    # 1 T_o, 1 T_e (the leading run), then internal runs of 1, 2 and 3: 3 G_o, 3 G_e
    assert t[0].tolist().count(TO) == 1 and t[0].tolist().count(GO) == 3
    got = oracle.gap_cost(t, 1000, [10.0, 1.0, 5.0, 0.5])[0]
    assert got == pytest.approx(oracle.gap_scale(1000) * (1 * 10 + 1 * 1 + 3 * 5 + 3 * 0.5), rel=1e-15)
