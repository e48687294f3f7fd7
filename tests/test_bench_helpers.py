"""bench.py's host-side helpers (CPU only): the algorithmic counts behind
GCUPS and pairs/s, the CPU baseline's pair sample, the validity check of the
committed DRAM-traffic record, and the clock sampler's parsing of nvidia-smi
lines (including a throttle reason)."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_cells_and_pairs_brute_force():
    rng = np.random.default_rng(3)
    lens = rng.integers(1, 50, 37)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cells, pairs = bench.cells_and_pairs(off)
    want = sum(int(lens[i]) * int(lens[j]) for i in range(len(lens)) for j in range(i + 1, len(lens)))
    assert cells == want
    assert pairs == len(lens) * (len(lens) - 1) / 2


def test_random_pairs_are_distinct_in_range_and_seeded():
    i, j = bench.random_pairs(10, 5000, 7)
    assert i.dtype == np.int32 and j.dtype == np.int32
    assert (i != j).all() and (i >= 0).all() and (i < 10).all() and (j >= 0).all() and (j < 10).all()
    # every ordered pair turns up, none favoured by more than noise
    counts = np.zeros((10, 10), np.int64)
    np.add.at(counts, (i, j), 1)
    assert (counts[~np.eye(10, dtype=bool)] > 20).all()
    i2, j2 = bench.random_pairs(10, 5000, 7)
    assert np.array_equal(i, i2) and np.array_equal(j, j2)


def test_traffic_record_is_current_and_checked_against_sources(tmp_path, monkeypatch):
    rec = bench.recorded_traffic()
    assert rec is not None, "profiles/lcs_traffic.json no longer matches the LCS sources"
    assert rec["launches"] == len(rec["per_launch"]) and rec["passes"] == 1
    # the captured launches' DRAM bytes per ns, times the step's mean LCS launch time
    got = sum(x["dram_read"] + x["dram_write"] for x in rec["per_launch"])
    ns = sum(x["ns"] for x in rec["per_launch"])
    assert got == rec["dram_bytes_captured"] and ns == rec["ns_captured"]
    per = got / ns * rec["mean_lcs_launch_ns"]
    assert abs(per - rec["dram_bytes_per_launch"]) < 1
    # a copy of the tree with one source changed: the record no longer applies
    for f in rec["sources"] + ["profiles/lcs_traffic.json"]:
        dst = tmp_path / f
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, f), "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic() is not None
    with open(tmp_path / rec["sources"][0], "ab") as fh:
        fh.write(b"\n// changed\n")
    assert bench.recorded_traffic() is None


def test_clock_sampler_parses_lines_and_reasons():
    s = bench.ClockSampler(0)
    s.proc = type("P", (), {"terminate": lambda self: None, "wait": lambda self, timeout=None: 0})()
    s.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    out = s.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    json.dumps(out)
