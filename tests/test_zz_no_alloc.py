"""famsa_lcs_query_noalloc, called through the C ABI, against famsa_lcs_query.

The no-allocation variant keeps its scratch in one fixed device array that
every call shares; two calls in a row with different query sets (the second
smaller and narrower, so the first call's leftovers sit around it) must both
give exactly the values of the allocating entry point.  The library's
allocation count shows that warmed-up calls allocate nothing, and calls from
several host threads on their own streams still give each thread its own
values.
"""
import ctypes

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


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _noalloc(fg, fam, q, off, max_len):
    """The new entry point through ctypes: device inputs and output."""
    import torch
    nq = off.numel() - 1
    out = torch.full((nq * fam.k,), -1, dtype=torch.int32, device="cuda")
    lib = fg.load()
    rc = lib.famsa_lcs_query_noalloc(ctypes.c_void_p(fam.handle), ctypes.c_void_p(q.data_ptr()),
                                     ctypes.c_void_p(off.data_ptr()), nq, max_len,
                                     ctypes.c_void_p(out.data_ptr()), None)
    return rc, out.reshape(nq, fam.k)


def test_noalloc_matches_lcs_query_on_two_calls_in_a_row(fg):
    import torch
    res, off = synth.family(300, 71, root_len=400, ext_frac=0.1)
    fam = fg.pack_peq(_dev(res), _dev(off))
    try:
        # call 1: 40 queries of 850 to 1450 residues (up to 23 words)
        q1, o1 = synth.family(40, 72, root_len=900, ext_frac=0.3, ext_lo=20, ext_hi=600)
        # call 2: 7 queries of about 150 residues (3 words) from another family
        q2, o2 = synth.family(7, 73, root_len=150, alphabet=6)
        for q, o in ((q1, o1), (q2, o2)):
            qd, od = _dev(q), _dev(o)
            max_len = int(np.diff(o).max())
            want = fg.lcs_query(fam, qd, od, device=True)
            rc, got = _noalloc(fg, fam, qd, od, max_len)
            assert rc == fg.FAMSA_OK, fg.strerror(rc)
            torch.cuda.synchronize()
            assert torch.equal(got, want)
            # a looser length bound (more words per query) gives the same values
            rc, got2 = _noalloc(fg, fam, qd, od, min(4 * max_len, fg.NOALLOC_MAX_LEN))
            assert rc == fg.FAMSA_OK
            assert torch.equal(got2, want)
    finally:
        fam.free()


def test_noalloc_makes_no_device_allocation(fg):
    # every device allocation of the library goes through one counted routine:
    # the allocating query call moves the count, warmed-up no-alloc calls do not
    import torch
    res, off = synth.family(120, 76, root_len=200)
    fam = fg.pack_peq(_dev(res), _dev(off))
    try:
        q, o = synth.family(9, 77, root_len=180)
        qd, od = _dev(q), _dev(o)
        max_len = int(np.diff(o).max())
        rc, _ = _noalloc(fg, fam, qd, od, max_len)  # the first call on the device sets up
        assert rc == fg.FAMSA_OK
        c0 = fg.debug_alloc_count()
        want = fg.lcs_query(fam, q, o)  # host inputs and output: allocates
        assert fg.debug_alloc_count() > c0
        c1 = fg.debug_alloc_count()
        for _ in range(2):
            rc, got = _noalloc(fg, fam, qd, od, max_len)
            assert rc == fg.FAMSA_OK
            torch.cuda.synchronize()
            assert np.array_equal(got.cpu().numpy(), want)
        assert fg.debug_alloc_count() == c1
    finally:
        fam.free()


def test_noalloc_from_several_threads(fg):
    # calls from several host threads on their own streams run one at a time
    # on the shared array, each with its own queries
    import threading
    import torch
    res, off = synth.family(200, 78, root_len=300)
    fam = fg.pack_peq(_dev(res), _dev(off))
    try:
        sets = [synth.family(5 + 3 * t, 80 + t, root_len=100 + 90 * t) for t in range(4)]
        wants = [fg.lcs_query(fam, q, o) for q, o in sets]
        got = [None] * len(sets)
        errors = []

        def worker(t):
            try:
                q, o = sets[t]
                stream = torch.cuda.Stream()
                with torch.cuda.stream(stream):
                    qd, od = _dev(q), _dev(o)
                    for _ in range(3):
                        nq = len(o) - 1
                        out = torch.full((nq * fam.k,), -1, dtype=torch.int32, device="cuda")
                        rc = fg.load().famsa_lcs_query_noalloc(
                            ctypes.c_void_p(fam.handle), ctypes.c_void_p(qd.data_ptr()),
                            ctypes.c_void_p(od.data_ptr()), nq, int(np.diff(o).max()),
                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
                        if rc != fg.FAMSA_OK:
                            errors.append(rc)
                    stream.synchronize()
                    got[t] = out.reshape(nq, fam.k).cpu().numpy()
            except Exception as e:  # reported below
                errors.append(e)

        threads = [threading.Thread(target=worker, args=(t,)) for t in range(len(sets))]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert not errors, errors
        for g, w in zip(got, wants):
            assert np.array_equal(g, w)
    finally:
        fam.free()


def test_noalloc_limits_and_bad_input(fg):
    res, off = synth.family(50, 74, root_len=100)
    fam = fg.pack_peq(_dev(res), _dev(off))
    try:
        q, o = synth.family(3, 75, root_len=60)
        qd, od = _dev(q), _dev(o)
        max_len = int(np.diff(o).max())
        lib = fg.load()
        # sizes beyond the fixed scratch are refused before any device work
        big = _dev(np.arange(fg.NOALLOC_MAX_QUERIES + 2, dtype=np.int64))
        rc = lib.famsa_lcs_query_noalloc(ctypes.c_void_p(fam.handle), ctypes.c_void_p(qd.data_ptr()),
                                         ctypes.c_void_p(big.data_ptr()), fg.NOALLOC_MAX_QUERIES + 1,
                                         max_len, ctypes.c_void_p(qd.data_ptr()), None)
        assert rc == fg.FAMSA_ELIMIT and "limits" in fg.strerror(rc)
        rc, _ = _noalloc(fg, fam, qd, od, fg.NOALLOC_MAX_LEN + 1)
        assert rc == fg.FAMSA_ELIMIT
        # a query longer than the stated bound, and a residue code >= 25, are found on the device
        rc, _ = _noalloc(fg, fam, qd, od, max_len - 1)
        assert rc == fg.FAMSA_EINVAL
        bad = q.copy()
        bad[1] = 30
        rc, _ = _noalloc(fg, fam, _dev(bad), od, max_len)
        assert rc == fg.FAMSA_EINVAL
        # and the next good call is unaffected by the status those left behind
        want = fg.lcs_query(fam, qd, od, device=True)
        rc, got = _noalloc(fg, fam, qd, od, max_len)
        assert rc == fg.FAMSA_OK
        import torch
        assert torch.equal(got, want)
    finally:
        fam.free()
