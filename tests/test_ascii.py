"""The ASCII helper of the C ABI (host only): letters of either case map to
the residue codes 0..24 in the order A C D E F G H I K L M N P Q R S T V W Y B
Z X U O; gaps, stops, digits, J and whitespace are rejected with their
position.  Also the float convenience view of merge heights."""
import numpy as np
import pytest

import paper_1603_06958_gb300 as fg
import synth
from paper_1603_06958_gb300 import build

ORDER = "ACDEFGHIKLMNPQRSTVWYBZXUO"


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fg.load()


def test_every_letter_both_cases(lib):
    assert fg.encode_ascii(ORDER).tolist() == list(range(25))
    assert fg.encode_ascii(ORDER.lower()).tolist() == list(range(25))
    assert fg.encode_ascii(b"MkVlA").tolist() == [ORDER.index(c) for c in "MKVLA"]
    assert fg.encode_ascii("").size == 0
    # the synthetic generator uses the same alphabet
    assert synth.ALPHABET == ORDER


@pytest.mark.parametrize("text,pos", [("ACD-E", 3), ("*", 0), ("ACJ", 2), ("AC D", 2), ("A1", 1),
                                      ("ACDE\n", 4), ("Z\x00", 1), ("\xff".encode("latin-1"), 0)])
def test_rejected_bytes_name_their_position(lib, text, pos):
    with pytest.raises(fg.FamsaError) as ei:
        fg.encode_ascii(text)
    assert ei.value.status == fg.FAMSA_EINVAL
    assert "byte %d" % pos in str(ei.value)


def test_encode_null_and_negative_length(lib):
    import ctypes
    out = np.zeros(4, np.uint8)
    assert lib.famsa_encode_ascii(None, 4, out.ctypes.data, None) == fg.FAMSA_EINVAL
    assert lib.famsa_encode_ascii(b"ACDE", -1, out.ctypes.data, None) == fg.FAMSA_EINVAL
    assert lib.famsa_encode_ascii(b"ACDE", 4, None, None) == fg.FAMSA_EINVAL
