"""The C-ABI library builds, loads and exports every declared entry point (CPU only).

No compute calls here: there is no GPU in this environment.  Argument checks
that fail before any device work are exercised too.
"""
import ctypes
import re
import subprocess

import numpy as np
import pytest

import paper_1603_06958_gb300 as fg
from paper_1603_06958_gb300 import build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return fg.load()


def test_exports_every_declared_symbol(lib):
    declared = fg.declared_functions()
    assert {"famsa_pack_peq", "famsa_lcs_allpairs", "famsa_lcs_rows", "famsa_slink_tree",
            "famsa_lcs_query", "famsa_free", "famsa_strerror"} <= set(declared)
    out = subprocess.check_output(["nm", "-D", "--defined-only", fg.LIB_PATH], text=True)
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in declared:
        assert name in exported, name
        assert getattr(lib, name) is not None


def test_probes_live_in_their_own_library(lib):
    # the roofline microbenchmarks are not part of the product ABI
    out = subprocess.check_output(["nm", "-D", "--defined-only", fg.LIB_PATH], text=True)
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert not any("probe" in name for name in exported)
    text = open(fg.PROBE_HEADER).read()
    names = set(re.findall(r"^int\s+(famsa_probe_[a-z0-9_]+)\s*\(", text, re.M))
    assert names == {"famsa_probe_int_pipe_rate", "famsa_probe_cluster"}
    out = subprocess.check_output(["nm", "-D", "--defined-only", fg.PROBE_LIB_PATH], text=True)
    pexported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert names <= pexported


def test_strerror_and_version(lib):
    for s in range(9):
        assert len(fg.strerror(s)) > 3 and "unknown" not in fg.strerror(s)
    assert "unknown" in fg.strerror(99)
    assert lib.famsa_version() >= 10000


def test_argument_errors_without_device_work(lib):
    h = ctypes.c_void_p()
    res = np.zeros(4, np.uint8)
    off = np.array([0, 2, 4], np.int64)
    # NULL out-pointer, NULL inputs, k < 1: rejected before touching CUDA
    assert lib.famsa_pack_peq(res.ctypes.data, off.ctypes.data, 2, 0, None, None) == fg.FAMSA_EINVAL
    assert lib.famsa_pack_peq(None, off.ctypes.data, 2, 0, None, ctypes.byref(h)) == fg.FAMSA_EINVAL
    assert lib.famsa_pack_peq(res.ctypes.data, off.ctypes.data, 0, 0, None, ctypes.byref(h)) == fg.FAMSA_EINVAL
    # host offsets not increasing (an empty sequence), sequence longer than 65535
    bad = np.array([0, 2, 2], np.int64)
    assert lib.famsa_pack_peq(res.ctypes.data, bad.ctypes.data, 2, 0, None, ctypes.byref(h)) == fg.FAMSA_EINVAL
    big = np.array([0, 70000], np.int64)
    assert lib.famsa_pack_peq(res.ctypes.data, big.ctypes.data, 1, 0, None, ctypes.byref(h)) == fg.FAMSA_ERANGE
    assert h.value is None
    # NULL handles
    out = np.zeros(1, np.int32)
    assert lib.famsa_lcs_allpairs(None, out.ctypes.data, 0, None) == fg.FAMSA_EINVAL
    assert lib.famsa_lcs_rows(None, 0, 1, out.ctypes.data, 0, None) == fg.FAMSA_EINVAL
    assert lib.famsa_slink_tree(None, *([None] * 7), 0, None) == fg.FAMSA_EINVAL
    assert lib.famsa_lcs_query(None, res.ctypes.data, off.ctypes.data, 2, 0, out.ctypes.data, 0, None) == fg.FAMSA_EINVAL
    assert lib.famsa_family_size(None) == -1
    lib.famsa_free(None)
    assert lib.famsa_debug_set_tpp_max_w(99) == fg.FAMSA_EINVAL
    assert lib.famsa_debug_set_slices(-1, 0) == fg.FAMSA_EINVAL
    assert lib.famsa_debug_set_slices(1, 17) == fg.FAMSA_EINVAL
    assert lib.famsa_debug_set_cluster(3) == fg.FAMSA_EINVAL
    assert lib.famsa_server_cancel(None, 0) == fg.FAMSA_EINVAL


def test_no_cpu_fallback_when_library_missing(tmp_path):
    with pytest.raises(ImportError):
        fg.load.__wrapped__ if hasattr(fg.load, "__wrapped__") else None
        import importlib
        mod = importlib.import_module("paper_1603_06958_gb300")
        saved = mod._lib
        try:
            mod._lib = None
            mod.load(str(tmp_path / "missing.so"))
        finally:
            mod._lib = saved


def test_binding_refuses_wrong_types_and_sizes(lib):
    # the library trusts the sizes it is given, so the binding checks types
    # and lengths before a pointer crosses the boundary
    res = np.zeros(4, np.uint8)
    with pytest.raises(ValueError):
        fg.pack_peq(res.astype(np.int32), np.array([0, 2, 4], np.int64))
    with pytest.raises(ValueError):
        fg.pack_peq(res, np.array([0, 2, 4], np.int32))
    fam = fg.Family.__new__(fg.Family)
    fam.handle, fam.k = None, 10
    q, qo = np.zeros(6, np.uint8), np.array([0, 3, 6], np.int64)
    with pytest.raises(ValueError):
        fg.lcs_query(fam, q, qo.astype(np.int32))
    with pytest.raises(ValueError):
        fg.lcs_query(fam, q, qo, out=np.zeros(19, np.int32))
    with pytest.raises(ValueError):
        fg.lcs_query(fam, q, qo, out=np.zeros(20, np.int64))
    with pytest.raises(ValueError):
        fg.lcs_query_noalloc(fam, q, qo.astype(np.int32), 3)
    with pytest.raises(ValueError):
        fg.lcs_allpairs(fam, out=np.zeros(44, np.int32))
    with pytest.raises(ValueError):
        fg.lcs_rows(fam, 2, 4, out=np.zeros(4, np.int32))
