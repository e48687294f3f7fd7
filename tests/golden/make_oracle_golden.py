"""Write tests/golden/oracle_trees.json: oracle tree digests for full-size families.

Calls only the oracle (and the seeded input generator).  The plain k=20,000
family needs ~2e8 DP LCS computations (~3e13 cells): about an hour and a half
on 8 cores, so its result is stored here rather than recomputed in a test.
Run: python tests/golden/make_oracle_golden.py [threads]
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def tree_digest(t):
    h1 = hashlib.sha256()
    for a, dt in ((t["pi"], "<i4"), (t["lambda_num"], "<u8"), (t["lambda_den"], "<u4")):
        h1.update(np.ascontiguousarray(a).astype(dt).tobytes())
    h2 = hashlib.sha256()
    for a, dt in ((t["merges"], "<i4"), (t["h_num"], "<u8"), (t["h_den"], "<u4"),
                  (t["sizes"], "<i4")):
        h2.update(np.ascontiguousarray(a).astype(dt).tobytes())
    return h1.hexdigest(), h2.hexdigest()


def main(threads=0):
    path = os.path.join(HERE, "oracle_trees.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    res, off = synth.plain20k(1)
    t0 = time.time()
    t = oracle.tree(res, off, nthreads=threads)
    dt = time.time() - t0
    pl, mg = tree_digest(t)
    lens = np.diff(off)
    out["plain20k_seed1"] = {
        "k": int(len(lens)), "cells": int((lens.astype(np.float64).sum() ** 2 -
                                           (lens.astype(np.float64) ** 2).sum()) / 2),
        "pi_lambda_sha256": pl, "merges_sha256": mg,
        "zero_lambdas": int((t["lambda_num"][:-1] == 0).sum()),
        "root_children": int((t["pi"][:-1] == len(lens) - 1).sum()),
        "oracle_seconds": round(dt, 1), "oracle_threads": oracle.num_threads(),
    }
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
