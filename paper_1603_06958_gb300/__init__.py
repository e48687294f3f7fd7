"""GB300 (sm_103a) FAMSA stages I+II: all-pairs bit-parallel LCS and the
single-linkage guide tree -- thin Python binding over the C ABI in
``include/famsa_gpu.h`` (``libfamsa_gpu.so``).

This module only marshals arguments: every step runs in the CUDA library.
Inputs and outputs may be numpy arrays (host) or torch tensors (host or
CUDA); PyTorch is used for device memory and streams only.  If the compiled
library is missing the import of the functions fails loudly -- there is no
CPU fallback.

Paper: Deorowicz, Debudaj-Grabysz, Gudys, "Aligning 415 519 proteins in less
than two hours on PC" (FAMSA), Methods: "Pairwise similarities calculation"
and "Determination of the guide tree".
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FAMSA_CHECKED=1 selects the checked build (kernels count failed invariants;
# python -m paper_1603_06958_gb300.build --checked)
LIB_PATH = os.path.join(_HERE, "libfamsa_gpu_checked.so" if os.environ.get("FAMSA_CHECKED") == "1"
                        else "libfamsa_gpu.so")
INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
HEADERS = [os.path.join(INCLUDE, h) for h in ("famsa_gpu.h", "famsa_gpu_debug.h")]

FAMSA_OK, FAMSA_EINVAL, FAMSA_ERANGE, FAMSA_ENOMEM, FAMSA_ECUDA, FAMSA_ETIMEOUT, FAMSA_EBUSY, \
    FAMSA_ELIMIT, FAMSA_ECANCELED = range(9)
NOALLOC_MAX_QUERIES, NOALLOC_MAX_LEN = 64, 4096

_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p


class FamsaError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, strerror(status), status))


def declared_functions():
    """Names of the entry points declared in the headers under include/."""
    names = set()
    for h in HEADERS:
        with open(h) as f:
            text = f.read()
        names.update(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s*]+(famsa_[a-z0-9_]+)\s*\(",
                                text, re.M))
    return sorted(names)


def load(path: str = LIB_PATH):
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError("%s not built: run python -m paper_1603_06958_gb300.build%s"
                              % (os.path.basename(path), " --checked" if "checked" in path else ""))
        lib = ctypes.CDLL(path)
        i32, u64p = ctypes.c_int32, _P
        sig = {
            "famsa_strerror": ([ctypes.c_int], ctypes.c_char_p),
            "famsa_version": ([], ctypes.c_int),
            "famsa_encode_ascii": ([ctypes.c_char_p, ctypes.c_int64, _P, _P], ctypes.c_int),
            "famsa_pack_peq": ([_P, _P, i32, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
            "famsa_family_size": ([_P], i32),
            "famsa_lcs_allpairs": ([_P, _P, ctypes.c_int, _P], ctypes.c_int),
            "famsa_lcs_rows": ([_P, i32, i32, _P, ctypes.c_int, _P], ctypes.c_int),
            "famsa_slink_tree": ([_P, _P, u64p, _P, _P, u64p, _P, _P, ctypes.c_int, _P], ctypes.c_int),
            "famsa_lcs_query": ([_P, _P, _P, i32, ctypes.c_int, _P, ctypes.c_int, _P], ctypes.c_int),
            "famsa_lcs_query_noalloc": ([_P, _P, _P, i32, i32, _P, _P], ctypes.c_int),
            "famsa_batch_pack": ([_P, _P, ctypes.c_int64, _P, i32, ctypes.c_int, _P, ctypes.POINTER(_P)],
                                 ctypes.c_int),
            "famsa_batch_tree": ([_P, _P, u64p, _P, _P, u64p, _P, _P, ctypes.c_int, _P], ctypes.c_int),
            "famsa_batch_stats": ([_P, _P], ctypes.c_int),
            "famsa_batch_free": ([_P], None),
            "famsa_server_create": ([ctypes.c_int64, i32, ctypes.POINTER(_P)], ctypes.c_int),
            "famsa_server_submit_tree": ([_P, _P, _P, i32, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
                                         ctypes.c_int),
            "famsa_server_submit_query": ([_P, ctypes.c_int64, _P, _P, i32,
                                           ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
            "famsa_server_wait": ([_P, ctypes.c_int64, ctypes.c_int64], ctypes.c_int),
            "famsa_server_tree_result": ([_P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
            "famsa_server_query_result": ([_P, ctypes.c_int64, _P], ctypes.c_int),
            "famsa_server_request_info": ([_P, ctypes.c_int64, _P], ctypes.c_int),
            "famsa_server_release": ([_P, ctypes.c_int64], ctypes.c_int),
            "famsa_server_stats": ([_P, _P], ctypes.c_int),
            "famsa_server_cancel": ([_P, ctypes.c_int64], ctypes.c_int),
            "famsa_server_destroy": ([_P], None),
            "famsa_free": ([_P], None),
            "famsa_last_stats": ([_P, _P], ctypes.c_int),
            "famsa_debug_fail_alloc_after": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_set_tpp_max_w": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_set_cluster": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_set_update_path": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_set_row_block": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_alloc_count": ([], ctypes.c_int64),
            "famsa_debug_set_slices": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "famsa_debug_check_count": ([_P], ctypes.c_int64),
            "famsa_debug_check_selftest": ([], ctypes.c_int),
            "famsa_debug_peq": ([_P, _P, _P, _P, _P], ctypes.c_int),
            "famsa_merge_similarity": ([_P, _P, ctypes.c_int64, _P, _P], ctypes.c_int),
            "famsa_msf_rows": ([_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int, _P],
                               ctypes.c_int),
            "famsa_tree_from_edges": ([ctypes.c_int32, ctypes.c_int64] + [_P] * 11 + [ctypes.c_int, _P],
                                      ctypes.c_int),
            "famsa_progressive_schedule": ([ctypes.c_int32] + [_P] * 7 + [ctypes.c_int, _P], ctypes.c_int),
            "famsa_gap_types": ([_P, ctypes.c_int64, ctypes.c_int32, _P, _P], ctypes.c_int),
            "famsa_upgma_tree": ([_P, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
            "famsa_nj_tree": ([_P, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
            "famsa_gap_scale": ([ctypes.c_int64, ctypes.c_double, ctypes.c_double], ctypes.c_double),
            "famsa_gap_cost": ([_P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P, ctypes.c_double,
                                ctypes.c_double, _P, _P], ctypes.c_int),
            "famsa_gap_insert": ([_P, _P, ctypes.c_int64, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P],
                                 ctypes.c_int),
            "famsa_debug_set_serial": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_set_update_threads": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_sub_kcycles": ([_P, _P], ctypes.c_int),
            "famsa_debug_set_global_variant": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_set_fin_small": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_order_code": ([ctypes.c_uint32, ctypes.c_uint32, _P], ctypes.c_int),
            "famsa_debug_code_fraction": ([ctypes.c_uint64, _P, _P], ctypes.c_int),
            "famsa_debug_set_tpp_rows": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
            "famsa_debug_tpp_rows": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_set_autotune": ([ctypes.c_int], ctypes.c_int),
            "famsa_debug_insertion_state": ([_P, _P, _P, _P, _P], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def strerror(status: int) -> str:
    try:
        return load().famsa_strerror(status).decode()
    except ImportError:
        return "status %d" % status


def _check(rc: int, what: str):
    if rc != FAMSA_OK:
        raise FamsaError(rc, what)


# ------------------------------------------------------------ marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a contiguous numpy array or torch tensor."""
    if x is None:
        return None, False
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), bool(x.is_cuda)
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data, False


_TORCH_DT = {"uint8": "uint8", "int32": "int32", "int64": "int64", "uint32": "uint32",
             "uint64": "uint64"}


def _require(x, dtype, name, count=None, at_least=None):
    """Refuse a buffer of the wrong element type or size before the library sees
    its pointer (the library trusts the sizes it is given)."""
    want = np.dtype(dtype).name
    if _is_torch(x):
        got, n = str(x.dtype).replace("torch.", ""), x.numel()
    else:
        got, n = np.asarray(x).dtype.name, np.asarray(x).size
    if got != _TORCH_DT[want]:
        raise ValueError("%s must be %s, not %s" % (name, want, got))
    if count is not None and n != count:
        raise ValueError("%s must have %d elements, not %d" % (name, count, n))
    if at_least is not None and n < at_least:
        raise ValueError("%s needs at least %d elements, has %d" % (name, at_least, n))


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _empty(n, dtype, device):
    if device:
        import torch
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint64: torch.uint64,
               np.uint32: torch.uint32}[dtype]
        return torch.empty(n, dtype=tdt, device="cuda")
    return np.empty(n, dtype=dtype)


class Family:
    """A packed family resident on the device (owns the C handle)."""

    def __init__(self, handle: int, k: int):
        self.handle = handle
        self.k = k

    def free(self):
        if self.handle:
            load().famsa_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        s = np.zeros(24, dtype=np.int64)
        _check(load().famsa_last_stats(self.handle, s.ctypes.data), "famsa_last_stats")
        keys = ["launches", "cells", "word_steps", "pairs", "relayout_merges", "merge_rounds", "rows",
                "lcs_ns", "update_ns", "finalize_ns", "lcs_launches", "pack_launches",
                "update_path", "update_cluster", "phaseA_kcycles", "phaseB_kcycles",
                "phaseC_kcycles", "phaseD_kcycles", "narrow_keys",
                "fast_merges", "fast_merge_runs"]
        return {k: int(v) for k, v in zip(keys, s)}


# ------------------------------------------------------------ entry points
def famsa_pack_peq(residues, offsets, stream=None) -> Family:
    """Validate a family, copy it to the device and build its Peq tables."""
    lib = load()
    _require(residues, np.uint8, "residues")
    _require(offsets, np.int64, "offsets")
    rp, rdev = _ptr(residues)
    op, odev = _ptr(offsets)
    if rdev != odev:
        raise ValueError("residues and offsets must both be on the host or both on the device")
    k = len(offsets) - 1
    h = _P()
    _check(lib.famsa_pack_peq(rp, op, k, int(rdev), _stream_ptr(stream), ctypes.byref(h)),
           "famsa_pack_peq")
    return Family(h.value, k)


pack_peq = famsa_pack_peq


def famsa_lcs_allpairs(fam: Family, out=None, device: bool = False, stream=None):
    """LCS of all pairs i < j, row-major (k(k-1)/2 int32)."""
    n = fam.k * (fam.k - 1) // 2
    if out is None:
        out = _empty(n, np.int32, device)
    _require(out, np.int32, "out", at_least=n)
    p, dev = _ptr(out)
    _check(load().famsa_lcs_allpairs(fam.handle, p, int(dev), _stream_ptr(stream)),
           "famsa_lcs_allpairs")
    return out


lcs_allpairs = famsa_lcs_allpairs


def famsa_lcs_rows(fam: Family, row_begin: int, row_end: int, out=None, device: bool = False,
                   stream=None):
    """Rows row_begin..row_end-1 of the lower triangle, concatenated."""
    n = (row_end * (row_end - 1) - row_begin * (row_begin - 1)) // 2
    if out is None:
        out = _empty(max(n, 0), np.int32, device)
    _require(out, np.int32, "out", at_least=max(n, 0))
    p, dev = _ptr(out)
    _check(load().famsa_lcs_rows(fam.handle, row_begin, row_end, p, int(dev), _stream_ptr(stream)),
           "famsa_lcs_rows")
    return out


lcs_rows = famsa_lcs_rows


def famsa_encode_ascii(text) -> np.ndarray:
    """Protein letters (str or bytes, either case) -> residue codes 0..24; any
    other byte raises FamsaError naming its position."""
    data = text.encode("ascii", "strict") if isinstance(text, str) else bytes(text)
    out = np.empty(len(data), dtype=np.uint8)
    bad = ctypes.c_int64(-1)
    st = load().famsa_encode_ascii(data, len(data), out.ctypes.data, ctypes.byref(bad))
    if st != FAMSA_OK:
        raise FamsaError(st, "famsa_encode_ascii (byte %d)" % bad.value)
    return out


encode_ascii = famsa_encode_ascii


def famsa_merge_similarity(tree: dict, stream=None):
    """The merge heights as the paper's similarity LCS / indel^2 (= h_den / h_num),
    computed by the library on the device: +inf for height 0, 0 for +inf.
    Device tensors in give a device tensor out; host arrays are copied over and back."""
    import torch
    num, den = tree["h_num"], tree["h_den"]
    on_host = not _is_torch(num)
    if on_host:
        num = torch.from_numpy(np.ascontiguousarray(num, dtype=np.uint64)).cuda()
        den = torch.from_numpy(np.ascontiguousarray(den, dtype=np.uint32)).cuda()
    _require(num, np.uint64, "h_num")
    _require(den, np.uint32, "h_den", count=num.numel())
    out = torch.empty(num.numel(), dtype=torch.float64, device=num.device)
    _check(load().famsa_merge_similarity(num.data_ptr(), den.data_ptr(), num.numel(), out.data_ptr(),
                                         _stream_ptr(stream)), "famsa_merge_similarity")
    if on_host:
        return out.cpu().numpy()
    return out


merge_similarity = famsa_merge_similarity


def famsa_slink_tree(fam: Family, device: bool = False, stream=None) -> dict:
    """Single-linkage tree: pointer representation and merge list (see the C header)."""
    k = fam.k
    m = max(k - 1, 0)
    out = {
        "pi": _empty(k, np.int32, device),
        "lambda_num": _empty(k, np.uint64, device),
        "lambda_den": _empty(k, np.uint32, device),
        "merges": _empty(2 * m, np.int32, device),
        "h_num": _empty(m, np.uint64, device),
        "h_den": _empty(m, np.uint32, device),
        "sizes": _empty(m, np.int32, device),
    }
    ptrs = [_ptr(out[n])[0] for n in ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den",
                                      "sizes")]
    _check(load().famsa_slink_tree(fam.handle, *ptrs, int(device), _stream_ptr(stream)),
           "famsa_slink_tree")
    out["merges"] = out["merges"].reshape(m, 2)
    return out


slink_tree = famsa_slink_tree


def famsa_msf_rows(fam: Family, row_begin: int, row_end: int, device: bool = False,
                   stream=None) -> dict:
    """Minimum spanning tree of the pairs of rows [row_begin, row_end) (one shard of
    the pair set): row_end - 1 edges, dict of edge_a < edge_b, h_num / h_den."""
    n = max(row_end - 1, 0)
    out = {"edge_a": _empty(n, np.int32, device), "edge_b": _empty(n, np.int32, device),
           "h_num": _empty(n, np.uint64, device), "h_den": _empty(n, np.uint32, device)}
    _check(load().famsa_msf_rows(fam.handle, row_begin, row_end, _ptr(out["edge_a"])[0],
                                 _ptr(out["edge_b"])[0], _ptr(out["h_num"])[0], _ptr(out["h_den"])[0],
                                 int(device), _stream_ptr(stream)), "famsa_msf_rows")
    return out


msf_rows = famsa_msf_rows


def famsa_tree_from_edges(k: int, edges: dict, device: bool = False, stream=None) -> dict:
    """The single-linkage tree of k points from an edge list that contains a minimum
    spanning tree (e.g. the union of famsa_msf_rows forests of all shards)."""
    m = len(edges["edge_a"])
    _require(edges["edge_a"], np.int32, "edge_a")
    _require(edges["edge_b"], np.int32, "edge_b", count=m)
    _require(edges["h_num"], np.uint64, "h_num", count=m)
    _require(edges["h_den"], np.uint32, "h_den", count=m)
    sides = {_ptr(edges[n])[1] for n in ("edge_a", "edge_b", "h_num", "h_den")}
    if sides != {bool(device)}:
        raise ValueError("edges must be on the %s" % ("device" if device else "host"))
    km = max(k - 1, 0)
    out = {"pi": _empty(k, np.int32, device), "lambda_num": _empty(k, np.uint64, device),
           "lambda_den": _empty(k, np.uint32, device), "merges": _empty(2 * km, np.int32, device),
           "h_num": _empty(km, np.uint64, device), "h_den": _empty(km, np.uint32, device),
           "sizes": _empty(km, np.int32, device)}
    ins = [_ptr(edges[n])[0] for n in ("edge_a", "edge_b", "h_num", "h_den")]
    outs = [_ptr(out[n])[0] for n in ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den",
                                      "sizes")]
    _check(load().famsa_tree_from_edges(k, m, *ins, *outs, int(device), _stream_ptr(stream)),
           "famsa_tree_from_edges")
    out["merges"] = out["merges"].reshape(km, 2)
    return out


tree_from_edges = famsa_tree_from_edges


def famsa_progressive_schedule(tree: dict, device: bool = False, stream=None) -> dict:
    """The merge list as the progressive stage's schedule: level, order (by level,
    index), level_start (n_levels + 1 offsets into order) and kind per merge."""
    merges, sizes = tree["merges"], tree["sizes"]
    n = len(sizes)
    k = n + 1
    _require(merges, np.int32, "merges", count=2 * n)
    _require(sizes, np.int32, "sizes")
    out = {"level": _empty(n, np.int32, device), "order": _empty(n, np.int32, device),
           "level_start": _empty(k, np.int32, device), "kind": _empty(n, np.int32, device)}
    top = ctypes.c_int32()
    _check(load().famsa_progressive_schedule(k, _ptr(merges)[0], _ptr(sizes)[0], _ptr(out["level"])[0],
                                             _ptr(out["order"])[0], _ptr(out["level_start"])[0],
                                             _ptr(out["kind"])[0], ctypes.byref(top), int(device),
                                             _stream_ptr(stream)), "famsa_progressive_schedule")
    out["level_start"] = out["level_start"][:top.value + 1]
    out["n_levels"] = top.value
    return out


progressive_schedule = famsa_progressive_schedule


def famsa_upgma_tree(fam: Family, device: bool = False, stream=None) -> dict:
    """UPGMA over the family's distances indel^2 / LCS: merges (k-1, 2), heights, sizes."""
    m = max(fam.k - 1, 0)
    out = {"merges": _empty(2 * m, np.int32, device), "sizes": _empty(m, np.int32, device)}
    if device:
        import torch
        out["heights"] = torch.empty(m, dtype=torch.float64, device="cuda")
    else:
        out["heights"] = np.empty(m, np.float64)
    _check(load().famsa_upgma_tree(fam.handle, _ptr(out["merges"])[0], _ptr(out["heights"])[0],
                                   _ptr(out["sizes"])[0], int(device), _stream_ptr(stream)),
           "famsa_upgma_tree")
    out["merges"] = out["merges"].reshape(m, 2)
    return out


upgma_tree = famsa_upgma_tree


def famsa_nj_tree(fam: Family, device: bool = False, stream=None) -> dict:
    """Neighbour joining over the family's distances indel^2 / LCS: merges
    (k-1, 2), lengths (k-1, 2) (the branch to each id of a merge), sizes."""
    m = max(fam.k - 1, 0)
    out = {"merges": _empty(2 * m, np.int32, device), "sizes": _empty(m, np.int32, device)}
    if device:
        import torch
        out["lengths"] = torch.empty(2 * m, dtype=torch.float64, device="cuda")
    else:
        out["lengths"] = np.empty(2 * m, np.float64)
    _check(load().famsa_nj_tree(fam.handle, _ptr(out["merges"])[0], _ptr(out["lengths"])[0],
                                _ptr(out["sizes"])[0], int(device), _stream_ptr(stream)),
           "famsa_nj_tree")
    out["merges"] = out["merges"].reshape(m, 2)
    out["lengths"] = out["lengths"].reshape(m, 2)
    return out


nj_tree = famsa_nj_tree

GAP = 255  # FAMSA_GAP: a gap in alignment rows


def famsa_gap_types(aln, stream=None):
    """Gap types of every cell of an m x n uint8 alignment on the device (torch)."""
    import torch
    _require(aln, np.uint8, "aln")
    m, n = aln.shape
    out = torch.empty((m, n), dtype=torch.uint8, device=aln.device)
    _check(load().famsa_gap_types(aln.data_ptr(), m, n, out.data_ptr(), _stream_ptr(stream)),
           "famsa_gap_types")
    return out


def famsa_gap_scale(k: int, g_l: float = 45.0, g_d: float = 7.0) -> float:
    """g_scale = 1 + log(k / g_l) / g_d."""
    return float(load().famsa_gap_scale(k, g_l, g_d))


def famsa_gap_cost(types, k: int, costs, g_l: float = 45.0, g_d: float = 7.0, stream=None):
    """Per row: g_scale(k) x sum of gap counts x costs (T_o, T_e, G_o, G_e); device in, device out."""
    import torch
    _require(types, np.uint8, "types")
    m, n = types.shape
    c = np.ascontiguousarray(costs, dtype=np.float64)
    if c.shape != (4,):
        raise ValueError("costs must hold T_o, T_e, G_o, G_e")
    out = torch.empty(m, dtype=torch.float64, device=types.device)
    _check(load().famsa_gap_cost(types.data_ptr(), m, n, k, c.ctypes.data, g_l, g_d, out.data_ptr(),
                                 _stream_ptr(stream)), "famsa_gap_cost")
    return out


def famsa_gap_insert(aln, types, positions, stream=None):
    """Insert gap columns before original columns positions (ascending) into every
    row, types corrected by S1..S6: (aln_out, types_out) on the device."""
    import torch
    _require(aln, np.uint8, "aln")
    _require(types, np.uint8, "types", count=aln.numel())
    m, n = aln.shape
    p = np.ascontiguousarray(positions, dtype=np.int32)
    ao = torch.empty((m, n + len(p)), dtype=torch.uint8, device=aln.device)
    to = torch.empty((m, n + len(p)), dtype=torch.uint8, device=aln.device)
    _check(load().famsa_gap_insert(aln.data_ptr(), types.data_ptr(), m, n, p.ctypes.data, len(p),
                                   ao.data_ptr(), to.data_ptr(), _stream_ptr(stream)), "famsa_gap_insert")
    return ao, to


gap_types = famsa_gap_types
gap_scale = famsa_gap_scale
gap_cost = famsa_gap_cost
gap_insert = famsa_gap_insert


class Batch:
    """Packed families resident on the device (owns the C batch handle)."""

    def __init__(self, handle: int, family_offsets: np.ndarray):
        self.handle = handle
        self.family_offsets = family_offsets
        self.n_seqs = int(family_offsets[-1])
        self.n_families = len(family_offsets) - 1

    def free(self):
        if self.handle:
            load().famsa_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self) -> dict:
        s = np.zeros(16, dtype=np.int64)
        _check(load().famsa_batch_stats(self.handle, s.ctypes.data), "famsa_batch_stats")
        keys = ["cells", "word_steps", "pairs", "lcs_items", "graph_launches", "lcs_widths",
                "global_update_families", "lcs_ns", "update_ns", "finalize_ns", "tuned_widths",
                "tune_ns", "plan_host_ns", "capture_ns", "instantiate_ns", "graph_nodes"]
        return {k: int(v) for k, v in zip(keys, s)}


def famsa_batch_pack(residues, offsets, family_offsets, stream=None) -> Batch:
    """Pack many families (one sequence list split by host family_offsets)."""
    _require(residues, np.uint8, "residues")
    _require(offsets, np.int64, "offsets")
    rp, rdev = _ptr(residues)
    op, odev = _ptr(offsets)
    if rdev != odev:
        raise ValueError("residues and offsets must be on the same side")
    fo = np.ascontiguousarray(np.asarray(family_offsets, dtype=np.int64))
    n_seqs = len(offsets) - 1
    h = _P()
    _check(load().famsa_batch_pack(rp, op, n_seqs, fo.ctypes.data, len(fo) - 1, int(rdev),
                                   _stream_ptr(stream), ctypes.byref(h)), "famsa_batch_pack")
    return Batch(h.value, fo)


batch_pack = famsa_batch_pack


def famsa_batch_tree(b: Batch, device: bool = False, stream=None) -> dict:
    """Every family's tree, concatenated (see the C header): pi/lambda per
    sequence, merges per family at merge offset family_offsets[f] - f."""
    n, m = b.n_seqs, b.n_seqs - b.n_families
    out = {
        "pi": _empty(n, np.int32, device),
        "lambda_num": _empty(n, np.uint64, device),
        "lambda_den": _empty(n, np.uint32, device),
        "merges": _empty(2 * m, np.int32, device),
        "h_num": _empty(m, np.uint64, device),
        "h_den": _empty(m, np.uint32, device),
        "sizes": _empty(m, np.int32, device),
    }
    ptrs = [_ptr(out[k])[0] for k in ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den",
                                      "sizes")]
    _check(load().famsa_batch_tree(b.handle, *ptrs, int(device), _stream_ptr(stream)),
           "famsa_batch_tree")
    out["merges"] = out["merges"].reshape(m, 2)
    return out


batch_tree = famsa_batch_tree


class Server:
    """The library's serving loop (see famsa_server_* in the C header): host
    inputs and outputs, admission by an HBM budget, `slots` concurrent requests."""

    def __init__(self, hbm_budget_bytes: int, slots: int):
        h = _P()
        _check(load().famsa_server_create(int(hbm_budget_bytes), int(slots), ctypes.byref(h)),
               "famsa_server_create")
        self.handle = h.value
        self.sizes = {}

    def submit_tree(self, residues, offsets, keep: bool = False) -> int:
        r = np.ascontiguousarray(residues, dtype=np.uint8)
        o = np.ascontiguousarray(offsets, dtype=np.int64)
        rid = ctypes.c_int64()
        _check(load().famsa_server_submit_tree(self.handle, r.ctypes.data, o.ctypes.data, len(o) - 1,
                                               int(keep), ctypes.byref(rid)), "famsa_server_submit_tree")
        self.sizes[rid.value] = ("tree", len(o) - 1, None)
        return rid.value

    def submit_query(self, family_request: int, q, q_offsets) -> int:
        r = np.ascontiguousarray(q, dtype=np.uint8)
        o = np.ascontiguousarray(q_offsets, dtype=np.int64)
        rid = ctypes.c_int64()
        _check(load().famsa_server_submit_query(self.handle, int(family_request), r.ctypes.data,
                                                o.ctypes.data, len(o) - 1, ctypes.byref(rid)),
               "famsa_server_submit_query")
        self.sizes[rid.value] = ("query", len(o) - 1, self.sizes[family_request][1])
        return rid.value

    def wait(self, request_id: int, timeout_ms: int = -1) -> int:
        return load().famsa_server_wait(self.handle, int(request_id), int(timeout_ms))

    def tree_result(self, request_id: int) -> dict:
        k = self.sizes[request_id][1]
        m = max(k - 1, 0)
        out = {"pi": np.empty(k, np.int32), "lambda_num": np.empty(k, np.uint64),
               "lambda_den": np.empty(k, np.uint32), "merges": np.empty(2 * m, np.int32),
               "h_num": np.empty(m, np.uint64), "h_den": np.empty(m, np.uint32),
               "sizes": np.empty(m, np.int32)}
        ptrs = [out[n].ctypes.data for n in ("pi", "lambda_num", "lambda_den", "merges", "h_num",
                                             "h_den", "sizes")]
        _check(load().famsa_server_tree_result(self.handle, int(request_id), *ptrs),
               "famsa_server_tree_result")
        out["merges"] = out["merges"].reshape(m, 2)
        return out

    def query_result(self, request_id: int) -> np.ndarray:
        _, nq, k = self.sizes[request_id]
        out = np.empty(nq * k, np.int32)
        _check(load().famsa_server_query_result(self.handle, int(request_id), out.ctypes.data),
               "famsa_server_query_result")
        return out.reshape(nq, k)

    def info(self, request_id: int) -> dict:
        a = np.zeros(7, np.int64)
        _check(load().famsa_server_request_info(self.handle, int(request_id), a.ctypes.data),
               "famsa_server_request_info")
        return dict(zip(["status", "kind", "n", "queue_ns", "latency_ns", "cells", "reserved"],
                        [int(x) for x in a]))

    def release(self, request_id: int):
        _check(load().famsa_server_release(self.handle, int(request_id)), "famsa_server_release")

    def cancel(self, request_id: int) -> int:
        """Cancel a queued request: FAMSA_OK; FAMSA_EBUSY while it runs; FAMSA_EINVAL if
        unknown or finished."""
        return int(load().famsa_server_cancel(self.handle, int(request_id)))

    def stats(self) -> dict:
        a = np.zeros(8, np.int64)
        _check(load().famsa_server_stats(self.handle, a.ctypes.data), "famsa_server_stats")
        return dict(zip(["submitted", "done", "failed", "queued", "running", "peak_running",
                         "reserved", "peak_reserved"], [int(x) for x in a]))

    def close(self):
        if self.handle:
            load().famsa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_family_tree(out: dict, b: Batch, f: int) -> dict:
    """Family f's slice of a famsa_batch_tree result."""
    a, z = int(b.family_offsets[f]), int(b.family_offsets[f + 1])
    ma, mz = a - f, z - f - 1
    return {"pi": out["pi"][a:z], "lambda_num": out["lambda_num"][a:z],
            "lambda_den": out["lambda_den"][a:z], "merges": out["merges"][ma:mz],
            "h_num": out["h_num"][ma:mz], "h_den": out["h_den"][ma:mz], "sizes": out["sizes"][ma:mz]}


def famsa_lcs_query(fam: Family, q_residues, q_offsets, out=None, device: bool = False,
                    stream=None):
    """LCS of each query against every member: (nq, k) int32."""
    nq = len(q_offsets) - 1
    _require(q_residues, np.uint8, "q_residues")
    _require(q_offsets, np.int64, "q_offsets", count=nq + 1)
    if out is not None:
        _require(out, np.int32, "out", at_least=nq * fam.k)
    qp, qdev = _ptr(q_residues)
    op, odev = _ptr(q_offsets)
    if qdev != odev:
        raise ValueError("query residues and offsets must be on the same side")
    if out is None:
        out = _empty(nq * fam.k, np.int32, device)
    p, dev = _ptr(out)
    _check(load().famsa_lcs_query(fam.handle, qp, op, nq, int(qdev), p, int(dev),
                                  _stream_ptr(stream)), "famsa_lcs_query")
    return out.reshape(nq, fam.k)


lcs_query = famsa_lcs_query


def famsa_lcs_query_noalloc(fam: Family, q_residues, q_offsets, max_len: int, out=None,
                            stream=None):
    """famsa_lcs_query with no device allocation inside the call: device inputs
    and output only, at most NOALLOC_MAX_QUERIES queries of at most
    NOALLOC_MAX_LEN residues (max_len bounds them all); (nq, k) int32."""
    nq = len(q_offsets) - 1
    _require(q_residues, np.uint8, "q_residues")
    _require(q_offsets, np.int64, "q_offsets", count=nq + 1)
    if out is not None:
        _require(out, np.int32, "out", at_least=nq * fam.k)
    qp, qdev = _ptr(q_residues)
    op, odev = _ptr(q_offsets)
    if not (qdev and odev):
        raise ValueError("famsa_lcs_query_noalloc takes device inputs")
    if out is None:
        out = _empty(nq * fam.k, np.int32, True)
    p, dev = _ptr(out)
    if not dev:
        raise ValueError("famsa_lcs_query_noalloc writes a device output")
    _check(load().famsa_lcs_query_noalloc(fam.handle, qp, op, nq, int(max_len), p,
                                          _stream_ptr(stream)), "famsa_lcs_query_noalloc")
    return out.reshape(nq, fam.k)


lcs_query_noalloc = famsa_lcs_query_noalloc


def famsa_free(fam: Family):
    fam.free()


def debug_fail_alloc_after(n: int):
    """Make the n-th next device allocation of a pack fail (n < 0 disables)."""
    load().famsa_debug_fail_alloc_after(n)


def debug_set_tpp_max_w(w: int):
    """Rows wider than w words leave thread-per-pair (32 = default) for the
    sliced kernel where it is on for their width, else warp-per-pair."""
    _check(load().famsa_debug_set_tpp_max_w(w), "famsa_debug_set_tpp_max_w")


def debug_set_slices(min_w: int, words: int = 0):
    """Rows of at least min_w words run sliced (0 = off; default 24), slices of
    at most `words` words (0 = 16)."""
    _check(load().famsa_debug_set_slices(min_w, words), "famsa_debug_set_slices")


def debug_set_update_path(path: int):
    """0 automatic, 1/2 insertion row update (cluster shared / global memory), 3 tree rebuild."""
    _check(load().famsa_debug_set_update_path(path), "famsa_debug_set_update_path")


def debug_insertion_state(fam: Family) -> dict:
    """Pointer representation of the last tree build, in insertion labels."""
    k = fam.k
    out = {"perm": np.empty(k, np.int32), "pi": np.empty(k, np.int32),
           "lambda_num": np.empty(k, np.uint64), "lambda_den": np.empty(k, np.uint32)}
    _check(load().famsa_debug_insertion_state(fam.handle, *[out[n].ctypes.data for n in
                                                            ("perm", "pi", "lambda_num", "lambda_den")]),
           "famsa_debug_insertion_state")
    return out


def debug_peq(fam: Family) -> dict:
    """The packed Peq tables of a family (host copies): peq (words, 64) uint32,
    word_off (k + 1), perm (k) in the family's sorted order."""
    n = ctypes.c_int64()
    _check(load().famsa_debug_peq(fam.handle, None, None, None, ctypes.byref(n)), "famsa_debug_peq")
    peq = np.empty((n.value, 64), np.uint32)
    off = np.empty(fam.k + 1, np.int64)
    perm = np.empty(fam.k, np.int32)
    _check(load().famsa_debug_peq(fam.handle, peq.ctypes.data, off.ctypes.data, perm.ctypes.data, None),
           "famsa_debug_peq")
    return {"peq": peq, "word_off": off, "perm": perm}


def debug_check_count():
    """(failed kernel checks so far, source line of the first) from the checked
    build; (-1, 0) from the normal one."""
    line = ctypes.c_int64()
    n = load().famsa_debug_check_count(ctypes.byref(line))
    return int(n), int(line.value)


def debug_check_selftest() -> int:
    """Checked build: one kernel check fails on purpose (the count grows by one)."""
    return int(load().famsa_debug_check_selftest())


def debug_alloc_count() -> int:
    """Device allocations made by the library in this process so far."""
    return int(load().famsa_debug_alloc_count())


def debug_set_row_block(rows: int):
    """Rows per row block of the tree build (0 = automatic)."""
    _check(load().famsa_debug_set_row_block(rows), "famsa_debug_set_row_block")


def debug_set_update_threads(threads: int):
    """Threads per CTA of the shared-memory row update (0 = default)."""
    _check(load().famsa_debug_set_update_threads(threads), "famsa_debug_set_update_threads")


def debug_set_serial(on: bool):
    load().famsa_debug_set_serial(int(on))


def debug_sub_kcycles(fam: Family):
    out = np.zeros(16, np.int64)
    _check(load().famsa_debug_sub_kcycles(fam.handle, out.ctypes.data), "famsa_debug_sub_kcycles")
    return out.tolist()


_probe_lib = None
PROBE_LIB_PATH = os.path.join(_HERE, "libfamsa_probe.so")
PROBE_HEADER = os.path.join(INCLUDE, "famsa_probe.h")


def load_probes(path: str = PROBE_LIB_PATH):
    """The benchmark's microbenchmark library (libfamsa_probe.so), separate from the product."""
    global _probe_lib
    with _lock:
        if _probe_lib is None:
            if not os.path.exists(path):
                raise ImportError("libfamsa_probe.so not built: run python -m paper_1603_06958_gb300.build")
            lib = ctypes.CDLL(path)
            lib.famsa_probe_int_pipe_rate.argtypes = [ctypes.c_int, _P]
            lib.famsa_probe_int_pipe_rate.restype = ctypes.c_int
            lib.famsa_probe_cluster.argtypes = [ctypes.c_int, ctypes.c_int, _P]
            lib.famsa_probe_cluster.restype = ctypes.c_int
            _probe_lib = lib
    return _probe_lib


def probe_int_pipe_rate(kind: int) -> float:
    """Thread-instructions/s of independent LOP3 (0), IADD3 (1), IMAD (2) or
    LOP3+IMAD (3) chains over the whole device."""
    out = ctypes.c_double()
    _check(load_probes().famsa_probe_int_pipe_rate(kind, ctypes.byref(out)), "famsa_probe_int_pipe_rate")
    return out.value


def probe_cluster(kind: int, cluster_ctas: int = 16) -> float:
    """SM clocks per repetition of a row-update building block (see famsa_probe.h)."""
    out = ctypes.c_double()
    _check(load_probes().famsa_probe_cluster(int(kind), int(cluster_ctas), ctypes.byref(out)),
           "famsa_probe_cluster")
    return out.value


def debug_set_tpp_rows(w: int, r: int):
    """Rows per thread-per-pair tile for width w (0 = default)."""
    _check(load().famsa_debug_set_tpp_rows(int(w), int(r)), "famsa_debug_set_tpp_rows")


def debug_tpp_rows(w: int) -> int:
    return int(load().famsa_debug_tpp_rows(int(w)))


def debug_set_autotune(on: bool):
    _check(load().famsa_debug_set_autotune(int(on)), "famsa_debug_set_autotune")


def debug_set_global_variant(v: int):
    """Global-memory row update: -1 = by size (default), 0 = 1,024 threads a CTA, 1 = 512."""
    _check(load().famsa_debug_set_global_variant(int(v)), "famsa_debug_set_global_variant")


def debug_order_code(num: int, den: int) -> int:
    """The row update's exact order code of the distance num / den (host arithmetic)."""
    out = ctypes.c_uint64()
    _check(load().famsa_debug_order_code(int(num), int(den), ctypes.byref(out)), "famsa_debug_order_code")
    return int(out.value)


def debug_code_fraction(code: int) -> tuple:
    """The reduced fraction (num, den) an order code came from (host arithmetic)."""
    num, den = ctypes.c_uint64(), ctypes.c_uint32()
    _check(load().famsa_debug_code_fraction(int(code), ctypes.byref(num), ctypes.byref(den)),
           "famsa_debug_code_fraction")
    return int(num.value), int(den.value)


def debug_set_fin_small(on: bool):
    """True (default): one-launch finalisation up to 4,096 points; False: multi-kernel always."""
    _check(load().famsa_debug_set_fin_small(int(on)), "famsa_debug_set_fin_small")


def debug_set_cluster(ctas: int):
    """Force the row-update cluster size (0 = automatic)."""
    _check(load().famsa_debug_set_cluster(ctas), "famsa_debug_set_cluster")
