"""CPU oracle for FAMSA stages I+II -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
arms of ``bench.py`` may import this package.  The GPU library never calls
it, and it imports nothing from the GPU package: the two share no code.

``oracle.c`` holds the arithmetic (plain C, OpenMP over independent pairs
only); this module compiles it with gcc and wraps it with numpy.

Functions and the paper passages they follow (FAMSA, Methods):

* :func:`lcs`, :func:`lcs_pairs`, :func:`lcs_allpairs`, :func:`lcs_rows` --
  LCS length by the textbook DP rule ("Pairwise similarities calculation").
* :func:`lcs_bitpar`, :func:`lcs_pairs_bitpar` -- the same LCS length by
  the bit-parallel recurrence the paper applies in stage I, as plain scalar
  64-bit C; pinned against the DP.
* :func:`key` -- the exact rational distance indel^2 / LCS used to order
  pairs; indel = |A| + |B| - 2 LCS and similarity = LCS / indel^2 are the
  two displayed equations of the same subsection.
* :func:`slink_matrix`, :func:`slink_streamed` -- Sibson's SLINK pointer
  representation ("Determination of the guide tree").
* :func:`slink_naive` -- naive single-linkage agglomeration, then the
  pointer representation read off the merges.
* :func:`slink_definition` -- the pointer representation evaluated from its
  definition via the minimax (single-link ultrametric) closure.
* :func:`slink_bitpar_range`, :func:`tree_bitpar` -- Sibson's SLINK fed by
  bit-parallel rows, resumable over ranges of points, for families too large
  for the DP (the k=400,000 digest).
* :func:`merges` -- the merge list with the fixed (lambda, index) order.
* :func:`gap_types`, :func:`gap_insert`, :func:`gap_scale`, :func:`gap_cost`
  -- the four gap types, gap-column insertion with the six corrections, and
  the set-size gap-cost scaling ("Gap types and costs determination").
* :func:`distance_matrix`, :func:`upgma`, :func:`nj` -- UPGMA and neighbour
  joining, the O(k^2)-memory guide trees the paper names beside single
  linkage, over indel^2 / LCS as doubles.
* :func:`schedule` -- the merge list as the progressive stage's schedule
  (levels of independent merges, their order, and which merges align a
  single sequence) ("Progressive construction of the alignment").
* :func:`msf_rows`, :func:`slink_edges`, :func:`tree_from_edges` -- the
  sharded pair set: Kruskal's minimum spanning forest of a range of rows, and
  SLINK over an edge list alone (single linkage depends only on a minimum
  spanning tree).

Every function here is pinned by ``tests/test_oracle_*.py`` against brute
force, closed forms, invariants, textbook examples or library routines.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2 -fopenmp, no SIMD intrinsics)."""
    with _lock:
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            tmp = _LIB_PATH + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC,
                   "-lm"]
            try:
                subprocess.check_call(cmd)
            except subprocess.CalledProcessError:
                subprocess.check_call([c for c in cmd if c != "-fopenmp"])
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i32, i64, u64, u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32
        sig = {
            "oracle_key_cmp": ([u64, u32, u64, u32], ctypes.c_int),
            "oracle_lcs": ([_P, i32, _P, i32], i32),
            "oracle_num_threads": ([], ctypes.c_int),
            "oracle_lcs_pairs": ([_P, _P, i32, _P, _P, i64, _P, ctypes.c_int], ctypes.c_int),
            "oracle_lcs_bitpar": ([_P, i32, _P, i32], i32),
            "oracle_lcs_pairs_bitpar": ([_P, _P, i32, _P, _P, i64, _P, ctypes.c_int],
                                        ctypes.c_int),
            "oracle_slink_bitpar_range": ([_P, _P, i32, i32, i32, _P, _P, _P, ctypes.c_int],
                                          ctypes.c_int),
            "oracle_reduce_keys": ([_P, _P, i64, _P, _P], ctypes.c_int),
            "oracle_msf_rows": ([_P, _P, i32, _P, i32, i32, _P, _P, _P, _P, ctypes.c_int], i64),
            "oracle_slink_edges": ([i32, i64, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
            "oracle_schedule": ([i32, _P, _P, _P, _P, _P, _P], i32),
            "oracle_gap_types": ([_P, i64, i32, _P], ctypes.c_int),
            "oracle_distance_matrix": ([_P, _P, i32, _P, ctypes.c_int], ctypes.c_int),
            "oracle_upgma": ([i32, _P, _P, _P, _P], ctypes.c_int),
            "oracle_nj": ([i32, _P, _P, _P, _P], ctypes.c_int),
            "oracle_gap_insert": ([_P, _P, i64, i32, _P, i32, _P, _P], ctypes.c_int),
            "oracle_gap_scale": ([i64, ctypes.c_double, ctypes.c_double], ctypes.c_double),
            "oracle_gap_cost": ([_P, i64, i32, i64, _P, ctypes.c_double, ctypes.c_double, _P], ctypes.c_int),
            "oracle_lcs_allpairs": ([_P, _P, i32, _P, ctypes.c_int], ctypes.c_int),
            "oracle_lcs_rows": ([_P, _P, i32, i32, i32, _P, ctypes.c_int], ctypes.c_int),
            "oracle_slink_matrix": ([_P, _P, i32, _P, _P, _P], ctypes.c_int),
            "oracle_slink_streamed": ([_P, _P, i32, _P, _P, _P, ctypes.c_int], ctypes.c_int),
            "oracle_slink_naive": ([_P, _P, i32, _P, _P, _P], ctypes.c_int),
            "oracle_slink_definition": ([_P, _P, i32, _P, _P, _P], ctypes.c_int),
            "oracle_minimax": ([_P, _P, i32, _P, _P], ctypes.c_int),
            "oracle_merges": ([_P, _P, _P, i32, _P, _P, _P, _P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (what, rc))


def _prep(residues, offsets):
    res = np.ascontiguousarray(residues, dtype=np.uint8)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    return res, off, len(off) - 1


def num_threads() -> int:
    return int(_load().oracle_num_threads())


# --------------------------------------------------------------------- LCS
def lcs(a, b) -> int:
    """LCS length of two code sequences by the DP rule."""
    a = np.ascontiguousarray(a, dtype=np.uint8)
    b = np.ascontiguousarray(b, dtype=np.uint8)
    r = _load().oracle_lcs(_ptr(a), len(a), _ptr(b), len(b))
    _check(0 if r >= 0 else r, "oracle_lcs")
    return int(r)


def lcs_pairs(residues, offsets, pa, pb, nthreads: int = 0) -> np.ndarray:
    res, off, k = _prep(residues, offsets)
    pa = np.ascontiguousarray(pa, dtype=np.int32)
    pb = np.ascontiguousarray(pb, dtype=np.int32)
    out = np.empty(len(pa), dtype=np.int32)
    _check(_load().oracle_lcs_pairs(_ptr(res), _ptr(off), k, _ptr(pa), _ptr(pb), len(pa),
                                    _ptr(out), nthreads), "oracle_lcs_pairs")
    return out


def lcs_bitpar(a, b) -> int:
    """LCS length of two code sequences by the bit-parallel recurrence (A = a is the Peq side)."""
    a = np.ascontiguousarray(a, dtype=np.uint8)
    b = np.ascontiguousarray(b, dtype=np.uint8)
    r = _load().oracle_lcs_bitpar(_ptr(a), len(a), _ptr(b), len(b))
    _check(0 if r >= 0 else r, "oracle_lcs_bitpar")
    return int(r)


def lcs_pairs_bitpar(residues, offsets, pa, pb, nthreads: int = 0) -> np.ndarray:
    """Bit-parallel LCS of the pairs (pa[t], pb[t]); pa[t] is the Peq side."""
    res, off, k = _prep(residues, offsets)
    pa = np.ascontiguousarray(pa, dtype=np.int32)
    pb = np.ascontiguousarray(pb, dtype=np.int32)
    out = np.empty(len(pa), dtype=np.int32)
    _check(_load().oracle_lcs_pairs_bitpar(_ptr(res), _ptr(off), k, _ptr(pa), _ptr(pb), len(pa),
                                           _ptr(out), nthreads), "oracle_lcs_pairs_bitpar")
    return out


def lcs_allpairs(residues, offsets, nthreads: int = 0) -> np.ndarray:
    """LCS of all pairs i < j, row-major (length k(k-1)/2)."""
    res, off, k = _prep(residues, offsets)
    out = np.empty(k * (k - 1) // 2, dtype=np.int32)
    _check(_load().oracle_lcs_allpairs(_ptr(res), _ptr(off), k, _ptr(out), nthreads),
           "oracle_lcs_allpairs")
    return out


def lcs_rows(residues, offsets, r0: int, r1: int, nthreads: int = 0) -> np.ndarray:
    """Rows r0..r1-1 of the lower triangle: row i lists LCS(i, j) for j = 0..i-1."""
    res, off, k = _prep(residues, offsets)
    n = (r1 * (r1 - 1) - r0 * (r0 - 1)) // 2
    out = np.empty(n, dtype=np.int32)
    _check(_load().oracle_lcs_rows(_ptr(res), _ptr(off), k, r0, r1, _ptr(out), nthreads),
           "oracle_lcs_rows")
    return out


def tri_to_square(tri: np.ndarray, k: int, diag=0) -> np.ndarray:
    m = np.full((k, k), diag, dtype=tri.dtype)
    iu = np.triu_indices(k, 1)
    m[iu] = tri
    m[(iu[1], iu[0])] = tri
    return m


# --------------------------------------------------------------------- keys
def key(lcs_len: int, la: int, lb: int):
    """Exact distance indel^2 / LCS as an unreduced (num, den); den 0 = +inf."""
    indel = la + lb - 2 * lcs_len
    if lcs_len == 0:
        return (1, 0)
    return (indel * indel, lcs_len)


def key_cmp(a, b) -> int:
    r = _load().oracle_key_cmp(a[0], a[1], b[0], b[1])
    if r == -2:
        raise ValueError("0/0 is not a key")
    return int(r)


# --------------------------------------------------------------------- trees
def _tree_out(k):
    return (np.empty(k, dtype=np.int32), np.empty(k, dtype=np.uint64), np.empty(k, dtype=np.uint32))


def _lens(offsets):
    return np.ascontiguousarray(np.diff(np.asarray(offsets, dtype=np.int64)), dtype=np.int32)


def slink_matrix(lcs_tri, lens):
    """Sibson's SLINK over a precomputed triangle; returns (pi, lambda_num, lambda_den)."""
    tri = np.ascontiguousarray(lcs_tri, dtype=np.int32)
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    k = len(lens)
    pi, ln, ld = _tree_out(k)
    _check(_load().oracle_slink_matrix(_ptr(tri), _ptr(lens), k, _ptr(pi), _ptr(ln), _ptr(ld)),
           "oracle_slink_matrix")
    return pi, ln, ld


def slink_streamed(residues, offsets, nthreads: int = 0):
    """SLINK with row n computed by DP when point n is inserted (no k x k storage)."""
    res, off, k = _prep(residues, offsets)
    pi, ln, ld = _tree_out(k)
    _check(_load().oracle_slink_streamed(_ptr(res), _ptr(off), k, _ptr(pi), _ptr(ln), _ptr(ld),
                                         nthreads), "oracle_slink_streamed")
    return pi, ln, ld


def slink_state(k: int):
    """Empty pointer state for :func:`slink_bitpar_range`: pi, lambda num, lambda den (unreduced)."""
    return {"pi": np.zeros(k, dtype=np.int32), "lam_num": np.zeros(k, dtype=np.uint64),
            "lam_den": np.zeros(k, dtype=np.uint32)}


def slink_bitpar_range(residues, offsets, state, n0: int, n1: int, nthreads: int = 0):
    """Insert points n0..n1-1 into ``state`` (from :func:`slink_state`), rows by bit-parallel LCS."""
    res, off, k = _prep(residues, offsets)
    for name, dt in (("pi", np.int32), ("lam_num", np.uint64), ("lam_den", np.uint32)):
        a = state[name]
        if a.dtype != dt or a.shape != (k,) or not a.flags.c_contiguous:
            raise ValueError("bad state array " + name)
    _check(_load().oracle_slink_bitpar_range(_ptr(res), _ptr(off), k, n0, n1, _ptr(state["pi"]),
                                             _ptr(state["lam_num"]), _ptr(state["lam_den"]),
                                             nthreads), "oracle_slink_bitpar_range")
    return state


def reduce_keys(num, den):
    """Keys num/den in lowest terms (+inf = 1/0, zero = 0/1)."""
    num = np.ascontiguousarray(num, dtype=np.uint64)
    den = np.ascontiguousarray(den, dtype=np.uint32)
    rn = np.empty_like(num)
    rd = np.empty_like(den)
    _check(_load().oracle_reduce_keys(_ptr(num), _ptr(den), len(num), _ptr(rn), _ptr(rd)),
           "oracle_reduce_keys")
    return rn, rd


def tree_from_state(state):
    """Full tree result (pi, reduced lambda, merge list) from a completed pointer state."""
    pi = state["pi"].copy()
    ln, ld = reduce_keys(state["lam_num"], state["lam_den"])
    pairs, hn, hd, sz = merges(pi, ln, ld)
    return {"pi": pi, "lambda_num": ln, "lambda_den": ld, "merges": pairs, "h_num": hn,
            "h_den": hd, "sizes": sz}


def tree_bitpar(residues, offsets, nthreads: int = 0):
    """Like :func:`tree`, but the SLINK rows come from the bit-parallel LCS."""
    res, off, k = _prep(residues, offsets)
    st = slink_state(k)
    slink_bitpar_range(res, off, st, 0, k, nthreads)
    return tree_from_state(st)


def slink_naive(lcs_tri, lens):
    tri = np.ascontiguousarray(lcs_tri, dtype=np.int32)
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    k = len(lens)
    pi, ln, ld = _tree_out(k)
    _check(_load().oracle_slink_naive(_ptr(tri), _ptr(lens), k, _ptr(pi), _ptr(ln), _ptr(ld)),
           "oracle_slink_naive")
    return pi, ln, ld


def slink_definition(lcs_tri, lens):
    tri = np.ascontiguousarray(lcs_tri, dtype=np.int32)
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    k = len(lens)
    pi, ln, ld = _tree_out(k)
    _check(_load().oracle_slink_definition(_ptr(tri), _ptr(lens), k, _ptr(pi), _ptr(ln),
                                           _ptr(ld)), "oracle_slink_definition")
    return pi, ln, ld


def minimax(lcs_tri, lens):
    """Single-link ultrametric u (k x k) as reduced (num, den) arrays."""
    tri = np.ascontiguousarray(lcs_tri, dtype=np.int32)
    lens = np.ascontiguousarray(lens, dtype=np.int32)
    k = len(lens)
    un = np.empty((k, k), dtype=np.uint64)
    ud = np.empty((k, k), dtype=np.uint32)
    _check(_load().oracle_minimax(_ptr(tri), _ptr(lens), k, _ptr(un), _ptr(ud)), "oracle_minimax")
    return un, ud


def merges(pi, lnum, lden):
    """Merge list: (pairs int32[k-1,2], h_num, h_den, sizes)."""
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    lnum = np.ascontiguousarray(lnum, dtype=np.uint64)
    lden = np.ascontiguousarray(lden, dtype=np.uint32)
    k = len(pi)
    m = max(k - 1, 0)
    pairs = np.empty((m, 2), dtype=np.int32)
    hn = np.empty(m, dtype=np.uint64)
    hd = np.empty(m, dtype=np.uint32)
    sz = np.empty(m, dtype=np.int32)
    _check(_load().oracle_merges(_ptr(pi), _ptr(lnum), _ptr(lden), k, _ptr(pairs), _ptr(hn),
                                 _ptr(hd), _ptr(sz)), "oracle_merges")
    return pairs, hn, hd, sz


def tree(residues, offsets, nthreads: int = 0):
    """Full oracle result for a family: dict with pi, lambda, merges (streamed SLINK)."""
    pi, ln, ld = slink_streamed(residues, offsets, nthreads)
    pairs, hn, hd, sz = merges(pi, ln, ld)
    return {"pi": pi, "lambda_num": ln, "lambda_den": ld, "merges": pairs, "h_num": hn,
            "h_den": hd, "sizes": sz}


# --------------------------------------------------------------------- shards
def msf_rows(residues, offsets, r0: int, r1: int, order=None, nthreads: int = 0):
    """Kruskal's minimum spanning forest of the pairs (order[i], order[j]), r0 <= i < r1,
    j < i: dict of edge_a < edge_b (labels), h_num / h_den (reduced keys)."""
    res, off, k = _prep(residues, offsets)
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    n = max(r1 - 1, 0) if r1 > 0 else 0
    ea = np.empty(max(n, 1), np.int32)
    eb = np.empty(max(n, 1), np.int32)
    en = np.empty(max(n, 1), np.uint64)
    ed = np.empty(max(n, 1), np.uint32)
    got = _load().oracle_msf_rows(_ptr(res), _ptr(off), k, None if o is None else _ptr(o), r0, r1,
                                  _ptr(ea), _ptr(eb), _ptr(en), _ptr(ed), nthreads)
    _check(0 if got >= 0 else got, "oracle_msf_rows")
    return {"edge_a": ea[:got], "edge_b": eb[:got], "h_num": en[:got], "h_den": ed[:got]}


def slink_edges(k: int, edges: dict):
    """SLINK over an edge list alone (+inf for absent pairs): (pi, lambda_num, lambda_den)."""
    ea = np.ascontiguousarray(edges["edge_a"], dtype=np.int32)
    eb = np.ascontiguousarray(edges["edge_b"], dtype=np.int32)
    en = np.ascontiguousarray(edges["h_num"], dtype=np.uint64)
    ed = np.ascontiguousarray(edges["h_den"], dtype=np.uint32)
    pi, ln, ld = _tree_out(k)
    _check(_load().oracle_slink_edges(k, len(ea), _ptr(ea), _ptr(eb), _ptr(en), _ptr(ed), _ptr(pi),
                                      _ptr(ln), _ptr(ld)), "oracle_slink_edges")
    return pi, ln, ld


def tree_from_edges(k: int, edges: dict):
    """Full tree result (pi, lambda, merge list) from an edge list alone."""
    pi, ln, ld = slink_edges(k, edges)
    pairs, hn, hd, sz = merges(pi, ln, ld)
    return {"pi": pi, "lambda_num": ln, "lambda_den": ld, "merges": pairs, "h_num": hn,
            "h_den": hd, "sizes": sz}


# --------------------------------------------------------------------- schedule
def schedule(merges, sizes):
    """Progressive-stage schedule of a merge list: dict of level, order, level_start, kind."""
    mg = np.ascontiguousarray(np.asarray(merges).reshape(-1), dtype=np.int32)
    sz = np.ascontiguousarray(sizes, dtype=np.int32)
    n = len(sz)
    k = n + 1
    level = np.empty(max(n, 1), np.int32)
    order = np.empty(max(n, 1), np.int32)
    start = np.empty(max(n, 1) + 1, np.int32)
    kind = np.empty(max(n, 1), np.int32)
    top = _load().oracle_schedule(k, _ptr(mg), _ptr(sz), _ptr(level), _ptr(order), _ptr(start),
                                  _ptr(kind))
    _check(0 if top >= 0 else top, "oracle_schedule")
    return {"level": level[:n], "order": order[:n], "level_start": start[:top + 1], "kind": kind[:n],
            "n_levels": int(top)}


# --------------------------------------------------------------------- gaps
GAP = 255


def gap_types(aln):
    """Per-cell gap types of an m x n alignment (0 residue, 1 T_o, 2 T_e, 3 G_o, 4 G_e)."""
    a = np.ascontiguousarray(aln, dtype=np.uint8)
    t = np.empty_like(a)
    _check(_load().oracle_gap_types(_ptr(a), a.shape[0], a.shape[1], _ptr(t)), "oracle_gap_types")
    return t


def gap_insert(aln, types, positions):
    """Insert gap columns before original columns positions (ascending) with the
    S1..S6 corrections: (aln_out, types_out)."""
    a = np.ascontiguousarray(aln, dtype=np.uint8)
    t = np.ascontiguousarray(types, dtype=np.uint8)
    p = np.ascontiguousarray(positions, dtype=np.int32)
    m, n = a.shape
    ao = np.empty((m, n + len(p)), np.uint8)
    to = np.empty((m, n + len(p)), np.uint8)
    _check(_load().oracle_gap_insert(_ptr(a), _ptr(t), m, n, _ptr(p), len(p), _ptr(ao), _ptr(to)),
           "oracle_gap_insert")
    return ao, to


def gap_scale(k: int, g_l: float = 45.0, g_d: float = 7.0) -> float:
    return float(_load().oracle_gap_scale(k, g_l, g_d))


def gap_cost(types, k: int, costs, g_l: float = 45.0, g_d: float = 7.0):
    t = np.ascontiguousarray(types, dtype=np.uint8)
    c = np.ascontiguousarray(costs, dtype=np.float64)
    out = np.empty(t.shape[0], np.float64)
    _check(_load().oracle_gap_cost(_ptr(t), t.shape[0], t.shape[1], k, _ptr(c), g_l, g_d, _ptr(out)),
           "oracle_gap_cost")
    return out


# --------------------------------------------------------------------- UPGMA
def distance_matrix(residues, offsets, nthreads: int = 0) -> np.ndarray:
    """k x k doubles indel^2 / LCS (+inf for LCS 0, 0 on the diagonal)."""
    res, off, k = _prep(residues, offsets)
    D = np.empty((k, k), np.float64)
    _check(_load().oracle_distance_matrix(_ptr(res), _ptr(off), k, _ptr(D), nthreads),
           "oracle_distance_matrix")
    return D


def upgma(D):
    """Plain UPGMA over a distance matrix: dict of merges (k-1, 2), heights, sizes."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    k = D.shape[0]
    m = max(k - 1, 0)
    mg = np.empty((max(m, 1), 2), np.int32)
    h = np.empty(max(m, 1), np.float64)
    sz = np.empty(max(m, 1), np.int32)
    _check(_load().oracle_upgma(k, _ptr(D), _ptr(mg), _ptr(h), _ptr(sz)), "oracle_upgma")
    return {"merges": mg[:m], "heights": h[:m], "sizes": sz[:m]}


def nj(D):
    """Plain neighbour joining over a distance matrix: dict of merges (k-1, 2),
    lengths (k-1, 2) (the branch to each id of the merge), sizes.  Raises
    RuntimeError (code -3) for an infinite distance."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    k = D.shape[0]
    m = max(k - 1, 0)
    mg = np.empty((max(m, 1), 2), np.int32)
    ln = np.empty((max(m, 1), 2), np.float64)
    sz = np.empty(max(m, 1), np.int32)
    _check(_load().oracle_nj(k, _ptr(D), _ptr(mg), _ptr(ln), _ptr(sz)), "oracle_nj")
    return {"merges": mg[:m], "lengths": ln[:m], "sizes": sz[:m]}
