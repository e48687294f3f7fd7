"""The seeded input generator: determinism, recipe properties, golden hashes."""
import hashlib
import json
import os
import sys

import numpy as np

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_synth_hashes  # noqa: E402


def test_golden_hashes_reproduce():
    with open(os.path.join(HERE, "golden", "synth_sha256.json")) as f:
        want = json.load(f)
    got = make_synth_hashes.compute()
    for name, h in got.items():
        assert want[name] == h, name
    assert want["batch512_params_seed1"] == hashlib.sha256(
        json.dumps(synth.batch_params()).encode()).hexdigest()


def test_deterministic_and_seeded():
    a = synth.family(300, 5, root_len=120)
    b = synth.family(300, 5, root_len=120)
    c = synth.family(300, 6, root_len=120)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0][:1000], c[0][:1000])


def test_preset_properties():
    res, off = synth.plain1k(1)
    L = np.diff(off)
    assert len(L) == 1000 and L.min() >= 50 and L.max() <= 400 and res.max() < 20
    res, off = synth.plain20k(1, k=3000)
    L = np.diff(off)
    assert L.min() >= 30 and L.max() <= 1500 and res.max() < 20
    res, off = synth.scale400k(1, k=3000)
    L = np.diff(off)
    assert L.min() >= 30 and L.max() <= 3000
    frac = np.isin(res, [20, 21, 22]).mean()
    assert 0.005 < frac < 0.02          # 1 % X/B/Z
    ks, ls = synth.batch_params()
    assert len(ks) == 512 and min(ks) >= 50 and max(ks) <= 5000
    assert min(ls) >= 30 and max(ls) <= 2000


def test_small_alphabet_and_duplicates():
    res, off = synth.family(200, 3, root_len=30, alphabet=2, dup_frac=0.5)
    assert res.max() <= 1
    seqs = {res[off[i]:off[i + 1]].tobytes() for i in range(200)}
    assert len(seqs) < 150                # duplicates present


def test_terminal_extension_fraction():
    base = synth.family(4000, 9, root_len=300, clip_lo=1, clip_hi=65535)
    ext = synth.family(4000, 9, root_len=300, clip_lo=1, clip_hi=65535, ext_frac=0.05)
    assert np.diff(ext[1]).mean() > np.diff(base[1]).mean()
