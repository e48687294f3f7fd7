"""The serving loop: results in a concurrent mix equal the single-request calls.

Tree requests of several families and query batches against the resident
families are submitted together to a server with several slots (their work
overlaps on the device); each result must equal famsa_slink_tree /
famsa_lcs_query run alone on the same input, and the oracle's for the small
families.  Admission by budget: with a budget smaller than any request the
server runs them one at a time, still exactly.  Failures stay per request.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

KEYS = ("pi", "lambda_num", "lambda_den", "merges", "h_num", "h_den", "sizes")


@pytest.fixture(scope="module")
def fg():
    from paper_1603_06958_gb300 import build
    build.build()
    import paper_1603_06958_gb300 as m
    m.load()
    return m


def alone_tree(fg, r, o):
    fam = fg.pack_peq(r, o)
    t = fg.slink_tree(fam)
    fam.free()
    return t


def alone_query(fg, r, o, q, qo):
    fam = fg.pack_peq(r, o)
    out = np.asarray(fg.lcs_query(fam, q, qo))
    fam.free()
    return out


def same_tree(a, b, tag):
    for key in KEYS:
        x, y = np.asarray(a[key]), np.asarray(b[key])
        assert np.array_equal(x.reshape(y.shape), y), (tag, key)


FAMS = [dict(k=300, seed=31, root_len=120), dict(k=60, seed=32, root_len=40, alphabet=4),
        dict(k=1200, seed=33, root_len=200, ext_frac=0.1), dict(k=2, seed=34, root_len=25),
        dict(k=4000, seed=35, root_len=90), dict(k=700, seed=36, root_len=2200, indel_rate=0.002)]


def make(c):
    c = dict(c)
    return synth.family(c.pop("k"), c.pop("seed"), **c)


@pytest.mark.parametrize("slots,budget", [(6, 16 << 30), (1, 1 << 20)])
def test_mix_equals_alone(fg, slots, budget):
    fams = [make(c) for c in FAMS]
    queries = [synth.family(n, 40 + n, root_len=150) for n in (1, 7, 64)]
    srv = fg.Server(budget, slots)
    try:
        tids = [srv.submit_tree(r, o, keep=True) for r, o in fams]
        qids = []
        for j, (q, qo) in enumerate(queries):
            for fi in (0, 2, 5):
                qids.append((srv.submit_query(tids[fi], q, qo), fi, j))
        for t in tids:
            assert srv.wait(t) == fg.FAMSA_OK
        for qid, _, _ in qids:
            assert srv.wait(qid) == fg.FAMSA_OK
        for i, (r, o) in enumerate(fams):
            got = srv.tree_result(tids[i])
            same_tree(got, alone_tree(fg, r, o), ("alone", i))
            if len(o) - 1 <= 1200:
                same_tree(got, oracle.tree(r, o), ("oracle", i))
            info = srv.info(tids[i])
            assert info["status"] == 0 and info["latency_ns"] >= info["queue_ns"] >= 0
        for qid, fi, j in qids:
            r, o = fams[fi]
            q, qo = queries[j]
            assert np.array_equal(srv.query_result(qid), alone_query(fg, r, o, q, qo)), (fi, j)
        st = srv.stats()
        assert st["done"] == len(tids) + len(qids) and st["failed"] == 0
        if slots == 1:
            assert st["peak_running"] == 1
        for t in tids:
            srv.release(t)
        assert srv.stats()["reserved"] == 0
    finally:
        srv.close()


def test_concurrent_calls_of_every_size(fg):
    # many tree requests of different sizes at once on 8 slots: their kernels
    # that size their shared memory by the family (the leaf-order join, the
    # sliced LCS) run side by side on different streams, and every call must
    # still succeed and equal the call alone (a per-launch shared-memory cap
    # set by one call must never be lowered under another's launch)
    ks = [int(x) for x in np.geomspace(30, 16000, 24)]
    fams = [synth.family(k, 500 + i, root_len=60 if i % 3 else 1700, indel_rate=0.002)
            for i, k in enumerate(ks)]
    want = [alone_tree(fg, r, o) for r, o in fams]
    srv = fg.Server(32 << 30, 8)
    try:
        for rep in range(2):
            tids = [srv.submit_tree(r, o) for r, o in fams]
            for i, t in enumerate(tids):
                assert srv.wait(t) == fg.FAMSA_OK, (rep, ks[i])
                same_tree(srv.tree_result(t), want[i], (rep, ks[i]))
                srv.release(t)
    finally:
        srv.close()


def test_failures_stay_per_request(fg):
    srv = fg.Server(8 << 30, 3)
    try:
        r, o = make(FAMS[1])
        bad = r.copy()
        bad[5] = 27                                      # residue code out of range
        t_bad = srv.submit_tree(bad, o, keep=True)
        t_ok = srv.submit_tree(r, o, keep=False)         # not kept: queries cannot use it
        q, qo = synth.family(3, 50, root_len=30)
        q_bad = srv.submit_query(t_bad, q, qo)           # its family fails
        assert srv.wait(t_bad) == fg.FAMSA_EINVAL
        assert srv.wait(q_bad) == fg.FAMSA_EINVAL
        assert srv.wait(t_ok) == fg.FAMSA_OK
        same_tree(srv.tree_result(t_ok), oracle.tree(r, o), "ok")
        with pytest.raises(fg.FamsaError):
            srv.submit_query(t_ok, q, qo)
        with pytest.raises(fg.FamsaError):
            srv.tree_result(t_bad)
        assert srv.stats()["failed"] == 2
    finally:
        srv.close()


def test_cancel_queued_requests(fg):
    # one slot: a large tree request runs while the others wait in the queue
    import time
    srv = fg.Server(64 << 30, 1)
    try:
        big_r, big_o = synth.plain20k(5, k=30000)
        b_r, b_o = make(FAMS[0])
        c_r, c_o = make(FAMS[1])
        a = srv.submit_tree(big_r, big_o)
        b = srv.submit_tree(b_r, b_o, keep=True)
        c = srv.submit_tree(c_r, c_o)
        q, qo = synth.family(5, 51, root_len=60)
        d = srv.submit_query(b, q, qo)
        assert srv.cancel(b) == fg.FAMSA_OK          # queued: taken out
        assert srv.wait(b) == fg.FAMSA_ECANCELED
        assert srv.cancel(b) == fg.FAMSA_EINVAL       # no longer queued
        t0 = time.time()
        while srv.info(a)["status"] == -1 and time.time() - t0 < 30:
            time.sleep(0.001)
        if srv.info(a)["status"] == -2:               # running: it cannot be stopped
            assert srv.cancel(a) == fg.FAMSA_EBUSY
        assert srv.wait(d) == fg.FAMSA_EINVAL         # its family was cancelled
        assert srv.wait(c) == fg.FAMSA_OK
        same_tree(srv.tree_result(c), oracle.tree(c_r, c_o), "after cancel")
        assert srv.wait(a) == fg.FAMSA_OK
        assert srv.cancel(a) == fg.FAMSA_EINVAL and srv.cancel(12345) == fg.FAMSA_EINVAL
        with pytest.raises(fg.FamsaError):
            srv.tree_result(b)
    finally:
        srv.close()
