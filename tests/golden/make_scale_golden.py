"""Oracle tree digests for prefixes of the k=400,000 scale family (seed 1).

Calls only the oracle and the seeded input generator.  The oracle's streamed
SLINK inserts the points of ``synth.scale400k(1)`` in index order with every
row computed by its plain scalar bit-parallel LCS (itself pinned against the
DP in tests/test_oracle_bitpar.py).  After n insertions the pointer state is
exactly the single-linkage tree of the first n sequences, so one pass yields
the tree of every prefix on the way; the digest of each milestone prefix is
stored in tests/golden/oracle_trees.json as ``scale400k_seed1_prefix<n>``.

The whole family is about 1.7e14 word steps, about 12 hours on 8 host
threads, so the run saves its pointer state every chunk of rows and resumes
from it when started again with the same state file.

Run: python tests/golden/make_scale_golden.py STATE_FILE [threads]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from make_oracle_golden import tree_digest  # noqa: E402

MILESTONES = (60000, 120000, 160000, 200000, 250000, 300000, 350000, 400000)
CHUNK = 1000


def _save_state(path, st, done, seconds):
    tmp = path + ".tmp.npz"
    np.savez(tmp, pi=st["pi"], lam_num=st["lam_num"], lam_den=st["lam_den"], done=done,
             seconds=seconds)
    os.replace(tmp, path)


def _load_state(path, k):
    if not os.path.exists(path):
        return oracle.slink_state(k), 0, 0.0
    z = np.load(path)
    st = {"pi": z["pi"].copy(), "lam_num": z["lam_num"].copy(), "lam_den": z["lam_den"].copy()}
    return st, int(z["done"]), float(z["seconds"])


def _record(n, st, lens, seconds, threads):
    prefix = {name: a[:n].copy() for name, a in st.items()}
    t = oracle.tree_from_state(prefix)
    pl, mg = tree_digest(t)
    ln = lens[:n].astype(np.float64)
    path = os.path.join(HERE, "oracle_trees.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    out["scale400k_seed1_prefix%d" % n] = {
        "k": int(n), "cells": int((ln.sum() ** 2 - (ln ** 2).sum()) / 2),
        "pi_lambda_sha256": pl, "merges_sha256": mg,
        "zero_lambdas": int((t["lambda_num"][:-1] == 0).sum()),
        "root_children": int((t["pi"][:-1] == n - 1).sum()),
        "oracle_seconds": round(seconds, 1), "oracle_threads": threads,
        "lcs": "bit-parallel",
    }
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print("milestone", n, pl, mg, flush=True)


def main(state_path, threads=0):
    res, off = synth.scale400k(1)
    k = len(off) - 1
    lens = np.diff(off)
    st, done, before = _load_state(state_path, k)
    nt = threads or oracle.num_threads()
    t0 = time.time()
    while done < k:
        n1 = min(k, done + CHUNK)
        nxt = [m for m in MILESTONES if done < m <= n1]
        if nxt:
            n1 = nxt[0]
        oracle.slink_bitpar_range(res, off, st, done, n1, threads)
        done = n1
        _save_state(state_path, st, done, before + time.time() - t0)
        print("rows %d / %d  %.0f s" % (done, k, before + time.time() - t0), flush=True)
        if done in MILESTONES:
            _record(done, st, lens, before + time.time() - t0, nt)


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else 0)
