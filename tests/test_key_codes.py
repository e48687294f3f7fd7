"""Exact order codes of the row update's distances (CPU only, host arithmetic).

The shared-memory row update compares distances indel^2 / LCS (lengths up to
32767) through the integer code floor(num * 2^30 / den).  Checked here against
Python's exact fractions: the code is that floor, codes order exactly as the
fractions do (equal fractions, equal codes), and decoding gives the reduced
fraction back.
"""
import math
import random
from fractions import Fraction

import pytest

import paper_1603_06958_gb300 as fg
from paper_1603_06958_gb300 import build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fg.load()


def random_keys(rng, n):
    """Distances the row update meets: indel^2 / L with 1 <= L <= 32767 and
    indel = la + lb - 2L for lengths <= 32767, plus extremes and near-ties."""
    keys = [(0, 1), (0, 32767), (1, 32767), (1, 32766), (4, 2), (2 ** 32 - 1, 1), (65534 ** 2, 1),
            (65534 ** 2, 32767), (65533 ** 2, 32767), (1, 1), (9, 3), (16, 8), (36, 18)]
    for _ in range(n):
        L = rng.choice([rng.randint(1, 40), rng.randint(1, 32767), 32767 - rng.randint(0, 5)])
        la = rng.randint(L, 32767)
        lb = rng.randint(L, 32767)
        indel = la + lb - 2 * L
        keys.append((indel * indel, L))
    # neighbours in the Farey sense: a/b and c/d with cb - ad = 1, both dens near 32767
    for _ in range(n // 10):
        b = rng.randint(30000, 32767)
        a = rng.randint(0, 4 * b)
        d = rng.randint(30000, 32767)
        c = (a * d + 1) // b if (a * d + 1) % b == 0 else None
        if c is not None:
            keys.append((c, d))
        keys.append((a, b))
    return keys


def test_code_is_the_scaled_floor_and_decodes(lib):
    rng = random.Random(7)
    for num, den in random_keys(rng, 4000):
        code = fg.debug_order_code(num, den)
        assert code == (num << 30) // den, (num, den)
        p, q = fg.debug_code_fraction(code)
        g = math.gcd(num, den)
        assert (p, q) == (num // g, den // g), (num, den, code)


def test_codes_order_exactly_like_the_fractions(lib):
    rng = random.Random(11)
    keys = random_keys(rng, 3000)
    # close values: dense small-denominator neighbourhoods of a few points
    for _ in range(300):
        x = Fraction(rng.randint(0, 10 ** 6), rng.randint(1, 32767))
        for den in (32767, 32766, 32765, 16384, 3):
            num = math.floor(x * den)
            if 0 <= num < 2 ** 32:
                keys.append((num, den))
                if num + 1 < 2 ** 32:
                    keys.append((num + 1, den))
    vals = [(Fraction(n, d), fg.debug_order_code(n, d)) for n, d in keys]
    vals.sort(key=lambda t: t[0])
    for (fa, ca), (fb, cb) in zip(vals, vals[1:]):
        if fa == fb:
            assert ca == cb, (fa, fb)
        else:
            assert ca < cb, (fa, fb, ca, cb)


def test_code_argument_errors(lib):
    import ctypes
    out = ctypes.c_uint64()
    assert lib.famsa_debug_order_code(1, 0, ctypes.byref(out)) == fg.FAMSA_EINVAL
    assert lib.famsa_debug_order_code(1, 32768, ctypes.byref(out)) == fg.FAMSA_EINVAL
    assert lib.famsa_debug_order_code(1, 1, None) == fg.FAMSA_EINVAL


def test_code_sweep_over_denominators(lib):
    # every 7th denominator 1..32767, numerators at and around multiples of
    # it across the 32-bit range: code = floor(num * 2^30 / den) and decoding
    # gives the reduced fraction back
    rng = random.Random(5)
    for den in range(1, 32768, 7):
        qmax = (2 ** 32 - 1) // den
        for q in (0, 1, qmax // 3, qmax // 2, qmax - 1, qmax, rng.randint(0, qmax)):
            for delta in (0, 1, den - 1):
                num = q * den + delta
                if num >= 2 ** 32:
                    continue
                code = fg.debug_order_code(num, den)
                assert code == (num << 30) // den, (num, den)
                g = math.gcd(num, den)
                assert fg.debug_code_fraction(code) == (num // g, den // g), (num, den)
