"""The Peq packing on its own, bit by bit (the LCS parity tests only see it
through the LCS values): for every sequence and 64-position word, exactly
one of the 25 codes has each valid position's bit set, the code slots
25..31 and the bits past the sequence's end are zero, and reading the set
bits back gives the residues.  Lengths sit on both sides of word
boundaries, with ambiguity codes and sequences of a single letter."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    from paper_1603_06958_gb300 import build
    build.build()
    import paper_1603_06958_gb300 as m
    m.load()
    return m


def _family():
    rng = np.random.default_rng(17)
    seqs = []
    for n in (1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 1000, 2047, 2048, 2049, 4100):
        seqs.append(rng.integers(0, 25, n).astype(np.uint8))
    seqs.append(np.full(130, 22, np.uint8))    # all X
    seqs.append(np.full(64, 24, np.uint8))     # all O, exactly one word
    res, off = synth.scale400k(3, k=40)
    seqs += [res[off[i]:off[i + 1]] for i in range(40)]
    off = np.concatenate([[0], np.cumsum([len(x) for x in seqs])]).astype(np.int64)
    return np.concatenate(seqs), off


def test_peq_bits(fg):
    res, off = _family()
    k = len(off) - 1
    fam = fg.pack_peq(res, off)
    try:
        d = fg.debug_peq(fam)
    finally:
        fam.free()
    peq, woff, perm = d["peq"], d["word_off"], d["perm"]
    lens = np.diff(off)
    assert np.array_equal(perm, np.lexsort((np.arange(k), lens)))
    assert woff[0] == 0 and woff[-1] == len(peq)
    for s in range(k):
        seq = res[off[perm[s]]:off[perm[s] + 1]]
        W = (len(seq) + 63) // 64
        assert woff[s + 1] - woff[s] == W
        words = peq[woff[s]:woff[s + 1]].astype(np.uint64)
        masks = words[:, :32] | (words[:, 32:] << np.uint64(32))   # (W, 32 code slots)
        assert (masks[:, 25:] == 0).all()
        bits = ((masks[:, :25, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)).astype(np.int64)
        bits = bits.transpose(0, 2, 1).reshape(W * 64, 25)        # position x code
        n = len(seq)
        assert (bits[n:] == 0).all()                              # padding bits
        assert (bits[:n].sum(axis=1) == 1).all()                  # one code per position
        assert np.array_equal(bits[:n].argmax(axis=1), seq)       # decodes to the residues
