"""Write tests/golden/synth_sha256.json: SHA-256 of the seeded generator's output.

The generator must give identical bytes on every machine (x86-64 here,
AArch64 on the GPU host); the GPU-side tests regenerate the same inputs and
compare trees against stored oracle results, so a drift in the generator
would show up here first.  Run: python tests/golden/make_synth_hashes.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402


def digest(res, off):
    h = hashlib.sha256()
    h.update(off.astype("<i8").tobytes())
    h.update(res.tobytes())
    return h.hexdigest()


CASES = {
    "plain1k_seed1": lambda: synth.plain1k(1),
    "plain20k_seed1": lambda: synth.plain20k(1),
    "scale400k_shape_k5000_seed1": lambda: synth.scale400k(1, k=5000),
    "batch512_family7_seed1": lambda: synth.batch_family(7, *[p[7] for p in synth.batch_params()]),
}


def compute():
    return {name: digest(*fn()) for name, fn in CASES.items()}


if __name__ == "__main__":
    out = compute()
    out["batch512_params_seed1"] = hashlib.sha256(
        json.dumps(synth.batch_params()).encode()).hexdigest()
    with open(os.path.join(HERE, "synth_sha256.json"), "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(json.dumps(out, indent=1))
