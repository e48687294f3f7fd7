"""Seeded synthetic protein families (input generator shared by tests and benches).

Holds no LCS or single-linkage arithmetic.  The C source ``synth.c`` does the
work; this module builds it (gcc, in-tree) and exposes presets for the five
workloads below.  Each preset stands in for the extHomFam-scale families that
the paper evaluates on (extHomFam section, Table S1): those datasets are not
available, so families are evolved down random trees instead.

Presets (residues are uint8 codes 0..24, lengths >= 1):

* ``plain1k``   -- k=1,000; root length 250; clip 50..400; 20 amino acids.
* ``plain20k``  -- k=20,000; root length log-normal (median 300, sigma 0.4);
                   clip 30..1,500; 5 % of sequences get a 20..80-residue
                   terminal extension.
* ``batch512``  -- 512 families; k log-uniform 50..5,000; root length
                   log-uniform 30..2,000; clip 20..3,000.
* ``scale400k`` -- k=400,000; root length log-normal (median 250, sigma 0.5)
                   clamped to 30..3,000; 1 % of residues become X/B/Z.
* serving streams draw families with the ``plain20k`` length model.

All presets: 0.02 substitutions per site per branch, 0.01 indel events per
site per branch (Geometric lengths, mean 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

ALPHABET = "ACDEFGHIKLMNPQRSTVWYBZXUO"


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("k", ctypes.c_int32),
        ("root_len", ctypes.c_int32),
        ("root_median", ctypes.c_double),
        ("root_sigma", ctypes.c_double),
        ("root_lo", ctypes.c_int32),
        ("root_hi", ctypes.c_int32),
        ("sub_rate", ctypes.c_double),
        ("indel_rate", ctypes.c_double),
        ("clip_lo", ctypes.c_int32),
        ("clip_hi", ctypes.c_int32),
        ("ext_frac", ctypes.c_double),
        ("ext_lo", ctypes.c_int32),
        ("ext_hi", ctypes.c_int32),
        ("ambig_frac", ctypes.c_double),
        ("alphabet", ctypes.c_int32),
        ("dup_frac", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (gcc, -ffp-contract=off)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + ".tmp%d" % os.getpid()
            subprocess.check_call(
                ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                 "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_family.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.c_void_p]
        lib.synth_family.restype = ctypes.c_int
        lib.synth_free.argtypes = [ctypes.c_void_p]
        lib.synth_uniform_ints.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                           ctypes.c_void_p]
        lib.synth_uniform_ints.restype = ctypes.c_int
        lib.synth_log_uniform_ints.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int64, ctypes.c_void_p]
        lib.synth_log_uniform_ints.restype = ctypes.c_int
        _lib = lib
    return _lib


def family(k: int, seed: int = 1, *, root_len: int = 250, root_median: float = 300.0,
           root_sigma: float = 0.0, root_lo: int = 0, root_hi: int = 0,
           sub_rate: float = 0.02, indel_rate: float = 0.01, clip_lo: int = 1,
           clip_hi: int = 65535, ext_frac: float = 0.0, ext_lo: int = 20, ext_hi: int = 80,
           ambig_frac: float = 0.0, alphabet: int = 0, dup_frac: float = 0.0):
    """One family: returns (residues uint8[sum len], offsets int64[k+1]).

    ``root_len > 0`` fixes the root length; otherwise it is drawn from a
    log-normal with the given median and sigma.  ``alphabet=a > 0`` replaces
    the amino-acid background by a uniform draw over codes 0..a-1 (small
    alphabets force ties); ``dup_frac`` makes exact duplicate sequences.
    """
    lib = _load()
    p = _Params(seed, k, root_len, root_median, root_sigma, root_lo, root_hi, sub_rate,
                indel_rate, clip_lo, clip_hi, ext_frac, ext_lo, ext_hi, ambig_frac, alphabet,
                dup_frac)
    offsets = np.zeros(k + 1, dtype=np.int64)
    ptr = ctypes.c_void_p()
    rc = lib.synth_family(ctypes.byref(p), ctypes.byref(ptr), offsets.ctypes.data)
    if rc != 0:
        raise ValueError("synth_family failed with code %d" % rc)
    total = int(offsets[-1])
    res = np.empty(total, dtype=np.uint8)
    ctypes.memmove(res.ctypes.data, ptr.value, total)
    lib.synth_free(ptr)
    return res, offsets


def uniform_ints(seed: int, n_below: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint32)
    if lib.synth_uniform_ints(seed, n_below, count, out.ctypes.data) != 0:
        raise ValueError("bad arguments")
    return out


# ----------------------------------------------------------------- presets
def plain1k(seed: int = 1):
    return family(1000, seed, root_len=250, clip_lo=50, clip_hi=400)


def plain20k(seed: int = 1, k: int = 20000):
    return family(k, seed, root_len=0, root_median=300.0, root_sigma=0.4, clip_lo=30,
                  clip_hi=1500, ext_frac=0.05, ext_lo=20, ext_hi=80)


def scale400k(seed: int = 1, k: int = 400000):
    return family(k, seed, root_len=0, root_median=250.0, root_sigma=0.5, root_lo=30,
                  root_hi=3000, clip_lo=30, clip_hi=3000, ambig_frac=0.01)


def log_uniform_ints(seed: int, lo: float, hi: float, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.int32)
    if lib.synth_log_uniform_ints(seed, lo, hi, count, out.ctypes.data) != 0:
        raise ValueError("bad arguments")
    return out


def batch_params(n_families: int = 512, seed: int = 1):
    """(k, root_len) per family of the batched workload, log-uniform draws."""
    ks = log_uniform_ints(seed * 7919 + 17, 50.0, 5000.0, n_families)
    ls = log_uniform_ints(seed * 7919 + 18, 30.0, 2000.0, n_families)
    return [int(x) for x in ks], [int(x) for x in ls]


def batch_family(f: int, k: int, root_len: int, seed: int = 1):
    return family(k, seed * 1000003 + f, root_len=root_len, clip_lo=20, clip_hi=3000)


def batch512(seed: int = 1, n_families: int = 512):
    ks, ls = batch_params(n_families, seed)
    return [batch_family(f, ks[f], ls[f], seed) for f in range(n_families)]


PRESETS = {"plain1k": plain1k, "plain20k": plain20k, "scale400k": scale400k}


def to_text(residues: np.ndarray, offsets: np.ndarray):
    """Decode codes back to one-letter strings (for fixtures and debugging)."""
    return ["".join(ALPHABET[c] for c in residues[offsets[i]:offsets[i + 1]])
            for i in range(len(offsets) - 1)]
