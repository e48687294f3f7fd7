"""Oracle tree digests for a subset of the 512-family batch (seed 1): every
family with k <= 500 and 16 seeded others, stored in
tests/golden/oracle_trees.json as ``batch512_seed1`` (family index -> digests).

Calls only the oracle and the seeded input generator; the trees come from the
oracle's streamed SLINK over its bit-parallel LCS (pinned against the DP), about
2e11 word steps in all, a minute or two on 8 host threads.
Run: python tests/golden/make_batch_golden.py [threads]
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


def subset(fams):
    ks = np.array([len(o) - 1 for _, o in fams])
    small = np.flatnonzero(ks <= 500)
    rng = np.random.default_rng(16)
    others = rng.choice(np.flatnonzero(ks > 500), 16, replace=False)
    return sorted(int(f) for f in np.concatenate([small, others]))


def main(threads=0):
    fams = synth.batch512(1)
    pick = subset(fams)
    t0 = time.time()
    out = {}
    for f in pick:
        r, o = fams[f]
        pl, mg = tree_digest(oracle.tree_bitpar(r, o, nthreads=threads))
        out[str(f)] = {"k": int(len(o) - 1), "pi_lambda_sha256": pl, "merges_sha256": mg}
    path = os.path.join(HERE, "oracle_trees.json")
    gold = json.load(open(path)) if os.path.exists(path) else {}
    gold["batch512_seed1"] = {"families": out, "oracle_seconds": round(time.time() - t0, 1),
                              "oracle_threads": oracle.num_threads(), "lcs": "bit-parallel",
                              "selection": "every family with k <= 500, and 16 others drawn with seed 16"}
    with open(path, "w") as fh:
        json.dump(gold, fh, indent=1, sort_keys=True)
    print(len(out), "families", round(time.time() - t0, 1), "s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 0)
