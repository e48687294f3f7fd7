"""Benchmark: all-pairs LCS + single-linkage guide tree (FAMSA stages I+II) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload plain20k|plain1k|scale400k]
                [--impl ours|reference]

A step is one pass of the whole hot path over one synthetic family with its
residues already in HBM: validate + length sort + Peq packing
(famsa_pack_peq), every pairwise LCS by the bit-parallel kernels, streamed
row block by row block into the on-device SLINK row update, and the
canonical pointer representation + merge list (famsa_slink_tree).

Metric: cell updates per second of the whole step in GCUPS, where cells =
sum over pairs of |A||B| (pairs/s is reported beside it).  The roofline of
the dominant kernel (thread-per-pair LCS) is integer-ALU bound: 6 INT32 ops
per 64-cell word step (LOP3 and 32-bit adds with carry, which issue on the
ALU pipe only) against 152 SMs x 64 ALU-pipe lanes x 2.07 GHz; the figure
for all 128 INT32 lanes (ALU + FMA pipes) is reported beside it.

python bench.py --int-peaks measures the integer pipe widths the roofline
uses (independent LOP3 / IADD3 / IMAD chains over the whole device).

N > 1 (torchrun) runs independent replicas, one family per GPU (the path
does not shard); value is the total cells of all ranks / the slowest rank.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "all-pairs LCS GCUPS + pairs/s on 1 GB300 vs plain; INT32 roofline fraction"
SMS, SM_MAX_GHZ = 152, 2.07
ALU_LANES = 64      # LOP3 / IADD3 lanes per SM per clock (ALU pipe; --int-peaks)
INT32_LANES = 128   # ALU + FMA pipes together
OPS_PER_WORD_STEP = 6
WORKLOADS = {
    "plain20k": "plain large family: k=20,000, root length log-normal (median 300, sigma 0.4), "
                "clip 30-1,500, 5% terminal extensions of 20-80 residues, 0.02 subs/site and "
                "0.01 indels/site per branch of a random coalescent tree, seed 1",
    "plain1k": "plain family: k=1,000, root length 250, clip 50-400, seed 1",
    "scale400k": "scale family: k=400,000, root length log-normal (median 250, sigma 0.5) "
                 "clamped 30-3,000, 1% X/B/Z ambiguity residues, 25-letter alphabet, seed 1",
    "serve": "serving: seeded Poisson stream of 120 requests, 70% new families (k log-uniform "
             "100-50,000, plain20k length model) and 30% batches of 1-256 query sequences "
             "scored against a resident family; admission by an HBM budget (64 GB), 8 slots",
    "batch512": "batched: 512 independent families, k log-uniform 50-5,000, root length "
                "log-uniform 30-2,000, 0.02 subs/site and 0.01 indels/site per branch, seed 1; "
                "one famsa_batch_pack + famsa_batch_tree (one CUDA graph) per step",
}


def make_family(workload: str, seed: int, k: int | None):
    import synth
    if workload == "plain20k":
        return synth.plain20k(seed, **({"k": k} if k else {}))
    if workload == "plain1k":
        return synth.plain1k(seed)
    if workload == "scale400k":
        return synth.scale400k(seed, **({"k": k} if k else {}))
    if workload == "serve":  # the largest family of the stream stands for it
        fams = [(r[1], r[2]) for r in serve_requests(seed) if r[0] == "tree"]
        return max(fams, key=lambda t: cells_and_pairs(t[1])[0])
    if workload == "batch512":  # one family stands for the batch (the oracle arm samples its rows)
        fams = synth.batch512(seed)
        return max(fams, key=lambda t: cells_and_pairs(t[1])[0])
    raise SystemExit("unknown workload %s" % workload)


def cells_and_pairs(off):
    lens = np.diff(off).astype(np.float64)
    cells = (lens.sum() ** 2 - (lens ** 2).sum()) / 2
    k = len(lens)
    return cells, k * (k - 1) / 2


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ traffic
def recorded_traffic():
    """DRAM bytes per LCS launch from the committed ncu summary, if the kernel source
    it was taken from is unchanged; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "lcs_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    for f in rec.get("sources", []):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != rec.get("sources_sha256"):
        return None
    return rec


# ------------------------------------------------------------------ CPU baseline
def random_pairs(k: int, n: int, seed: int):
    """n seeded uniform random pairs i != j of a family of k sequences."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, k, n)
    j = rng.integers(0, k - 1, n)
    j = np.where(j >= i, j + 1, j)
    return i.astype(np.int32), j.astype(np.int32)


def cpu_baseline(res, off, budget_s=15.0):
    """The oracle's DP LCS, as it stands, on a bounded sample of the workload's
    pairs: seeded uniform random pairs (the oracle spreads pairs over all host
    threads), grown until one run takes at least half the budget."""
    import oracle
    k = len(off) - 1
    lens = np.diff(off).astype(np.float64)
    n = 256
    while True:
        pa, pb = random_pairs(k, n, 12345)
        t0 = time.perf_counter()
        oracle.lcs_pairs(res, off, pa, pb)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * budget_s or n >= (1 << 26):
            break
        n = int(min(1 << 26, n * max(2.0, 0.75 * budget_s / max(dt, 1e-3))))
    cells = float((lens[pa] * lens[pb]).sum())
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "DP LCS of %d seeded uniform random pairs of the family (%.3g cells, %.1f s); "
                      "the O(k) per-row SLINK update is not part of the sample" % (n, cells, dt)}


# ------------------------------------------------------------------ arms
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle
    res, off = make_family(args.workload, args.seed, args.k)
    k = len(off) - 1
    lens = np.diff(off).astype(np.int64)
    # each step: a fresh seeded sample of uniform random pairs, about 2 s of
    # host work (sized once from a calibration run); the oracle spreads pairs
    # over all host threads
    n = 512
    while True:
        pa, pb = random_pairs(k, n, 999)
        t0 = time.perf_counter()
        oracle.lcs_pairs(res, off, pa, pb)
        dt = time.perf_counter() - t0
        if dt >= 0.25 or n >= (1 << 24):
            break
        n *= 4
    n = int(max(512, min(1 << 24, n * args.ref_seconds / max(dt, 1e-6))))
    vals, tot_cells, tot_t = [], 0.0, 0.0
    for s in range(args.warmup + args.steps):
        pa, pb = random_pairs(k, n, 1000 + s)
        t0 = time.perf_counter()
        oracle.lcs_pairs(res, off, pa, pb)
        dt = time.perf_counter() - t0
        cells = float((lens[pa].astype(np.float64) * lens[pb]).sum())
        if s >= args.warmup:
            vals.append(cells / dt / 1e9)
            tot_cells += cells
            tot_t += dt
    value = tot_cells / tot_t / 1e9
    cells_all, pairs_all = cells_and_pairs(off)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GCUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_t / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "k": k, "cells": cells_all,
                   "pairs": pairs_all,
                   "sample_per_step": "DP LCS of %d seeded uniform random pairs" % n},
        "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "per step: DP LCS of %d seeded uniform random pairs of the family" % n},
        "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def replica_totals(ms_step, e2e_ms, cells, dist, device):
    """Replicas (one family per GPU): the slowest rank's step and end-to-end
    times, and the cells of all ranks."""
    import torch
    vals = torch.tensor([ms_step, e2e_ms, cells], dtype=torch.float64, device=device)
    mx = vals.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = vals.clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(mx[1]), float(tot[2])


def concat_families(fams):
    res = np.concatenate([r for r, _ in fams])
    offs, fo, base = [np.zeros(1, np.int64)], [0], 0
    for r, o in fams:
        offs.append(o[1:] + base)
        base += int(o[-1])
        fo.append(fo[-1] + len(o) - 1)
    return res, np.concatenate(offs), np.array(fo, np.int64)


def run_batch(args, rank, world, local_rank):
    """Batched families: every step packs the whole batch and builds every tree
    through one CUDA graph; the same families one plain pack + tree at a time
    are timed beside it."""
    import torch
    import paper_1603_06958_gb300 as fg
    import synth

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    fg.load()
    fams = synth.batch512(args.seed + rank)
    res, off, fo = concat_families(fams)
    cells = sum(cells_and_pairs(o)[0] for _, o in fams)
    pairs = sum(cells_and_pairs(o)[1] for _, o in fams)
    dres = torch.from_numpy(res).cuda()
    doff = torch.from_numpy(off).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step():
        b = fg.batch_pack(dres, doff, fo)
        t = fg.batch_tree(b, device=True)
        return b, t

    tune = None
    for _ in range(args.warmup):
        b, _ = step()
        s0 = b.stats()
        if tune is None:  # the first plan of the process runs the autotuner
            tune = {"widths_timed": s0["tuned_widths"], "seconds": s0["tune_ns"] / 1e9,
                    "rows_per_tile": {w: fg.debug_tpp_rows(w) for w in range(1, 33)}}
        b.free()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ms, graph_ms, pack_ms, stats = [], [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0, ep, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e0.record()
        b = fg.batch_pack(dres, doff, fo)
        ep.record()
        fg.batch_tree(b, device=True)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        pack_ms.append(e0.elapsed_time(ep))
        stats.append(b.stats())
        # the same graph again: the steady state of a resident batch
        flush.zero_()
        e1.record()
        fg.batch_tree(b, device=True)
        e2.record()
        e2.synchronize()
        graph_ms.append(e1.elapsed_time(e2))
        b.free()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_step = float(np.mean(ms))
    st = stats[-1]
    lcs_ms = float(np.mean([s["lcs_ns"] for s in stats])) / 1e6

    # plain: the same families, one famsa_pack_peq + famsa_slink_tree each
    plain_ms = None
    if not args.no_plain:
        fams_dev = [(torch.from_numpy(r).cuda(), torch.from_numpy(o).cuda()) for r, o in fams]
        for r, o in fams_dev[:8]:
            fam = fg.pack_peq(r, o)
            fg.slink_tree(fam, device=True)
            fam.free()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for r, o in fams_dev:
            fam = fg.pack_peq(r, o)
            fg.slink_tree(fam, device=True)
            fam.free()
        e1.record()
        e1.synchronize()
        plain_ms = e0.elapsed_time(e1)

    # end to end through the public API with pinned host buffers
    pres = torch.from_numpy(res).pin_memory()
    poff = torch.from_numpy(off).pin_memory()
    e2e_ms = []
    for i in range(1 + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = fg.batch_pack(pres, poff, fo)
        t = fg.batch_tree(b, device=False)
        b.free()
        dt = time.perf_counter() - t0
        if i >= 1:
            e2e_ms.append(1e3 * dt)
    d2h = sum(v.nbytes for v in t.values())
    h2d = res.nbytes + off.nbytes
    if dist is not None:
        ms_max, e2e_max, cells_total = replica_totals(ms_step, float(np.mean(e2e_ms)), cells, dist, "cuda")
    else:
        ms_max, e2e_max, cells_total = ms_step, float(np.mean(e2e_ms)), cells
    if rank != 0:
        return 0
    achieved = OPS_PER_WORD_STEP * st["word_steps"] / (lcs_ms * 1e-3) / 1e12
    peak = SMS * ALU_LANES * SM_MAX_GHZ * 1e9 / 1e12
    line = {
        "metric": METRIC, "value": cells_total / (ms_max * 1e-3) / 1e9, "unit": "GCUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["batch512"], "families": len(fams), "sequences": int(fo[-1]),
                   "cells": cells, "pairs": pairs, "pairs_per_s": pairs * world / (ms_max * 1e-3),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between timed steps (L2 flush)",
                   "inputs": "residues and offsets resident in HBM before each timed step",
                   "breakdown_ms": {"lcs_kernels": lcs_ms,
                                    "row_update_kernels": float(np.mean([s["update_ns"] for s in stats])) / 1e6,
                                    "finalise": float(np.mean([s["finalize_ns"] for s in stats])) / 1e6,
                                    "graph_only": float(np.mean(graph_ms)),
                                    "pack": float(np.mean(pack_ms)),
                                    "plan_and_capture": ms_step - float(np.mean(pack_ms)) - float(np.mean(graph_ms)),
                                    "plan_host": float(np.mean([s["plan_host_ns"] for s in stats])) / 1e6,
                                    "capture": float(np.mean([s["capture_ns"] for s in stats])) / 1e6,
                                    "instantiate": float(np.mean([s["instantiate_ns"] for s in stats])) / 1e6},
                   "graph_nodes": int(stats[-1]["graph_nodes"]),
                   "graph_only_gcups": cells / (float(np.mean(graph_ms)) * 1e-3) / 1e9,
                   "plain_ms": plain_ms,
                   "plain_gcups": (cells / (plain_ms * 1e-3) / 1e9) if plain_ms else None,
                   "speedup_vs_plain": (plain_ms / ms_step) if plain_ms else None,
                   "lcs_items": st["lcs_items"], "lcs_widths": st["lcs_widths"],
                   "autotuner": tune},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOPS",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "k_lcs_tpp / k_lcs_wpp over the batch work lists",
                     "peak_note": "152 SMs x 64 ALU-pipe lanes x 2.07 GHz (bench.py --int-peaks)",
                     "achieved_note": "6 INT32 ops per word step x word steps / LCS span of the graph "
                                      "(CUDA events recorded inside the graph)"},
        "e2e": {"value": cells_total / (e2e_max * 1e-3) / 1e9, "unit": "GCUPS",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(st["graph_launches"]) + 40,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_families(fams, args.cpu_budget)
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_families(fams, budget_s=15.0):
    """The oracle's DP LCS over whole families of the batch, smallest first, until
    about the budget is spent."""
    import oracle
    order = sorted(range(len(fams)), key=lambda f: cells_and_pairs(fams[f][1])[0])
    done_cells, t_used, n = 0.0, 0.0, 0
    for f in order:
        r, o = fams[f]
        c = cells_and_pairs(o)[0]
        if n > 0 and t_used > 0 and (t_used + c * t_used / done_cells) > budget_s:
            break
        t0 = time.perf_counter()
        oracle.lcs_allpairs(r, o)
        t_used += time.perf_counter() - t0
        done_cells += c
        n += 1
    return {"value": done_cells / t_used / 1e9, "unit": "GCUPS", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "DP LCS of all pairs of the %d smallest families of the batch (%.3g cells, %.1f s)"
                      % (n, done_cells, t_used)}


def serve_requests(seed: int, n: int = 120):
    """The seeded request stream: (kind, family index or arrays, arrival gap in
    units of the mean gap)."""
    import synth
    rng = np.random.default_rng(seed)
    reqs, n_trees = [], 0
    for i in range(n):
        gap = float(rng.exponential(1.0))
        if i == 0 or rng.random() < 0.7 or n_trees == 0:
            k = int(np.exp(rng.uniform(np.log(100), np.log(50000))))
            res, off = synth.plain20k(seed * 100003 + i, k=k)
            reqs.append(("tree", res, off, gap))
            n_trees += 1
        else:
            nq = int(rng.integers(1, 257))
            q, qo = synth.plain20k(seed * 100003 + i, k=nq)
            target = int(rng.integers(0, n_trees))  # the target-th tree request so far
            reqs.append(("query", q, qo, gap, target))
    return reqs


def run_serve(args, rank, world, local_rank):
    """Serving: the request stream through famsa_server_* -- serially (one slot,
    all submitted at once: plain launches one after another), as a burst with 8
    slots (capacity), and as Poisson arrivals at 75% of that capacity (latency)."""
    import torch
    import paper_1603_06958_gb300 as fg

    torch.cuda.set_device(local_rank)
    fg.load()
    reqs = serve_requests(args.seed + rank)
    budget = 64 << 30

    def run(slots, rate=None):
        srv = fg.Server(budget, slots)
        ids, trees = [], []
        t0 = time.perf_counter()
        clk_next = t0
        for r in reqs:
            if rate is not None:
                clk_next += r[3] / rate
                d = clk_next - time.perf_counter()
                if d > 0:
                    time.sleep(d)
            if r[0] == "tree":
                rid = srv.submit_tree(r[1], r[2], keep=True)
                trees.append(rid)
            else:
                rid = srv.submit_query(trees[r[4]], r[1], r[2])
            ids.append(rid)
        for rid in ids:
            rc = srv.wait(rid)
            if rc != fg.FAMSA_OK:
                raise RuntimeError("request %d failed: %s" % (rid, fg.strerror(rc)))
        makespan = time.perf_counter() - t0
        infos = [srv.info(i) for i in ids]
        st = srv.stats()
        srv.close()
        return makespan, infos, st

    run(8)  # warm-up: kernels loaded, memory pools grown
    clocks = ClockSampler(local_rank)
    clocks.start()
    t_serial, inf_serial, _ = run(1)
    t_burst, inf_burst, st_burst = run(8)
    rate = 0.75 * len(reqs) / t_burst
    t_pois, inf_pois, st_pois = run(8, rate)
    clk = clocks.stop()
    cells = float(sum(i["cells"] for i in inf_burst))

    def lat(infos, kind=None):
        v = np.array([i["latency_ns"] for i in infos if kind is None or i["kind"] == kind]) / 1e6
        return {"p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99)),
                "mean_ms": float(v.mean()), "n": int(len(v))}

    n_tree = sum(1 for r in reqs if r[0] == "tree")
    line = {
        "metric": METRIC, "value": cells / t_burst / 1e9, "unit": "GCUPS", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * t_burst, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOADS["serve"], "requests": len(reqs), "tree_requests": n_tree,
                   "query_requests": len(reqs) - n_tree, "cells": cells,
                   "serial_one_slot_s": t_serial, "serial_gcups": cells / t_serial / 1e9,
                   "burst_8_slots_s": t_burst, "speedup_vs_serial": t_serial / t_burst,
                   "peak_running": st_burst["peak_running"],
                   "peak_reserved_gb": st_burst["peak_reserved"] / 2 ** 30,
                   "poisson_rate_per_s": rate, "poisson_makespan_s": t_pois,
                   "poisson_gcups": cells / t_pois / 1e9,
                   "latency_poisson": {"all": lat(inf_pois), "tree": lat(inf_pois, 0),
                                       "query": lat(inf_pois, 1)},
                   "latency_burst": lat(inf_burst), "latency_serial": lat(inf_serial),
                   "inputs": "host buffers copied at submission; results copied back to the host",
                   "l2": "inputs larger than L2 across the stream"},
        "roofline": None,
        "e2e": {"value": cells / t_burst / 1e9, "unit": "GCUPS",
                "h2d_bytes_per_step": int(sum(r[1].nbytes + r[2].nbytes for r in reqs)),
                "d2h_bytes_per_step": 0},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_1603_06958_gb300 as fg

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    fg.load()
    fg.debug_set_update_path(args.update_path)
    fg.debug_set_global_variant(args.global_variant)
    res, off = make_family(args.workload, args.seed + rank, args.k)
    k = len(off) - 1
    cells, pairs = cells_and_pairs(off)
    dres = torch.from_numpy(res).cuda()
    doff = torch.from_numpy(off).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def step(mid=None):
        fam = fg.pack_peq(dres, doff)
        if mid is not None:
            mid.record()
        t = fg.slink_tree(fam, device=True)
        st = fam.stats()
        fam.free()
        return t, st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    barrier()
    clocks.start()
    ms, pack_ms, stats = [], [], []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        em = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, st = step(em)
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        pack_ms.append(e0.elapsed_time(em))
        stats.append(st)
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    ms_step = float(np.mean(ms))
    lcs_ms = float(np.mean([s["lcs_ns"] for s in stats])) / 1e6
    upd_ms = float(np.mean([s["update_ns"] for s in stats])) / 1e6
    fin_ms = float(np.mean([s["finalize_ns"] for s in stats])) / 1e6
    launches = int(sum(s["launches"] + s["pack_launches"] for s in stats))
    word_steps = stats[-1]["word_steps"]

    # end to end through the public API with pinned host buffers
    pres = torch.from_numpy(res).pin_memory()
    poff = torch.from_numpy(off).pin_memory()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fam = fg.pack_peq(pres, poff)
        t = fg.slink_tree(fam, device=False)
        fam.free()
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_ms.append(1e3 * dt)
    d2h = sum(v.nbytes for v in t.values())
    h2d = res.nbytes + off.nbytes

    if dist is not None:
        ms_step_max, e2e_max, cells_total = replica_totals(ms_step, float(np.mean(e2e_ms)), cells, dist,
                                                          "cuda")
    else:
        ms_step_max, e2e_max, cells_total = ms_step, float(np.mean(e2e_ms)), cells
    if rank != 0:
        return 0
    achieved = OPS_PER_WORD_STEP * word_steps / (lcs_ms * 1e-3) / 1e12
    peak = SMS * ALU_LANES * SM_MAX_GHZ * 1e9 / 1e12
    peak_all = SMS * INT32_LANES * SM_MAX_GHZ * 1e9 / 1e12
    # the DRAM record is of the plain k=20,000 family's LCS launches: it
    # applies to that workload only
    tr = recorded_traffic() if args.workload == "plain20k" and args.k is None and args.seed == 1 else None
    line = {
        "metric": METRIC,
        "value": cells_total / (ms_step_max * 1e-3) / 1e9,
        "unit": "GCUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "k": k, "cells": cells, "pairs": pairs,
                   "pairs_per_s": pairs * world / (ms_step_max * 1e-3),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between timed steps (L2 flush)",
                   "inputs": "residues and offsets resident in HBM before each timed step",
                   "breakdown_ms": {"pack": float(np.mean(pack_ms)), "lcs_kernels": lcs_ms,
                                    "row_update_kernels": upd_ms, "finalise": fin_ms},
                   "lcs_only_gcups": cells / (lcs_ms * 1e-3) / 1e9,
                   "wall_s_timed_region": wall},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOPS",
                     "frac": achieved / peak,
                     "traffic": (tr["dram_bytes_per_launch"] if tr else None),
                     "kernel": "k_lcs_tpp (thread-per-pair bit-parallel LCS)",
                     "peak_note": "derived: 152 SMs x 64 ALU-pipe lanes x 2.07 GHz max SM "
                                  "clock; LOP3 and IADD3 issue on the ALU pipe only, 64 lanes "
                                  "per SM per clock as measured by bench.py --int-peaks "
                                  "(MEASURED_PEAKS.json has no integer peak)",
                     "peak_all_int32_lanes": peak_all,
                     "frac_all_int32_lanes": achieved / peak_all,
                     "achieved_note": "6 INT32 ops per 64-cell word step x word steps / summed "
                                      "CUDA-event time of the LCS launches of the step"},
        "e2e": {"value": cells_total / (e2e_max * 1e-3) / 1e9, "unit": "GCUPS",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(res, off, args.cpu_budget)
    if world == 1 and args.workload == "plain20k" and not args.no_extra and not args.k:
        # the other configurations of the metric, measured in the same run:
        # the largest single-GPU one (k=400,000) and batched against plain
        line["config"]["batch512"] = measure_batch512(fg, args, flush)
        line["config"]["scale400k"] = measure_scale400k(fg, args, flush)
    print(json.dumps(line), flush=True)
    return 0


def measure_scale400k(fg, args, flush):
    """The largest single-GPU configuration (k=400,000), measured after the
    headline steps: one step through the public API with pinned host buffers
    (the e2e figure; it also warms every kernel and allocation pool at this
    size), then one step with the inputs resident in HBM, timed with CUDA
    events on the launching stream and with the clocks sampled."""
    import torch
    res, off = make_family("scale400k", args.seed, None)
    k = len(off) - 1
    cells, pairs = cells_and_pairs(off)
    pres = torch.from_numpy(res).pin_memory()
    poff = torch.from_numpy(off).pin_memory()
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fam = fg.pack_peq(pres, poff)
    t = fg.slink_tree(fam, device=False)
    fam.free()
    e2e_ms = 1e3 * (time.perf_counter() - t0)
    d2h = sum(v.nbytes for v in t.values())
    dres = torch.from_numpy(res).cuda()
    doff = torch.from_numpy(off).cuda()
    flush.zero_()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fam = fg.pack_peq(dres, doff)
    fg.slink_tree(fam, device=True)
    e1.record()
    e1.synchronize()
    st = fam.stats()
    fam.free()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    lcs_ms = st["lcs_ns"] / 1e6
    achieved = OPS_PER_WORD_STEP * st["word_steps"] / (lcs_ms * 1e-3) / 1e12
    peak = SMS * ALU_LANES * SM_MAX_GHZ * 1e9 / 1e12
    del dres, doff
    return {"workload": WORKLOADS["scale400k"], "k": k, "cells": cells, "pairs": pairs,
            "steps": 1, "warmup": "one e2e step of the same family first (and the headline steps "
                                  "before it, with the same kernels)",
            "ms_per_step": ms, "gcups": cells / (ms * 1e-3) / 1e9, "pairs_per_s": pairs / (ms * 1e-3),
            "breakdown_ms": {"lcs_kernels": lcs_ms, "row_update_kernels": st["update_ns"] / 1e6,
                             "finalise": st["finalize_ns"] / 1e6},
            "gpu_launches": int(st["launches"] + st["pack_launches"]),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TOPS",
                         "frac": achieved / peak, "kernel": "k_lcs_tpp / k_lcs_wpp",
                         "frac_all_int32_lanes": achieved / (SMS * INT32_LANES * SM_MAX_GHZ * 1e9 / 1e12)},
            "e2e": {"value": cells / (e2e_ms * 1e-3) / 1e9, "unit": "GCUPS", "ms": e2e_ms,
                    "h2d_bytes_per_step": int(res.nbytes + off.nbytes), "d2h_bytes_per_step": int(d2h)},
            "clocks": clk,
            "l2": "256 MB buffer written before the step; inputs and working set far above L2"}


def measure_batch512(fg, args, flush):
    """Batched against plain on the 512-family workload: one warm-up batch step
    (it runs the autotuner), one timed batch step (pack + plan + graph capture +
    graph), then the same families one plain pack + tree at a time."""
    import torch
    import synth
    fams = synth.batch512(args.seed)
    res, off, fo = concat_families(fams)
    cells = sum(cells_and_pairs(o)[0] for _, o in fams)
    dres = torch.from_numpy(res).cuda()
    doff = torch.from_numpy(off).cuda()
    b = fg.batch_pack(dres, doff, fo)
    fg.batch_tree(b, device=True)
    b.free()
    flush.zero_()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    b = fg.batch_pack(dres, doff, fo)
    fg.batch_tree(b, device=True)
    e1.record()
    e1.synchronize()
    st = b.stats()
    b.free()
    batch_ms = e0.elapsed_time(e1)
    fams_dev = [(torch.from_numpy(r).cuda(), torch.from_numpy(o).cuda()) for r, o in fams]
    flush.zero_()
    torch.cuda.synchronize()
    e0.record()
    for r, o in fams_dev:
        fam = fg.pack_peq(r, o)
        fg.slink_tree(fam, device=True)
        fam.free()
    e1.record()
    e1.synchronize()
    plain_ms = e0.elapsed_time(e1)
    lcs_ms = st["lcs_ns"] / 1e6
    achieved = OPS_PER_WORD_STEP * st["word_steps"] / (lcs_ms * 1e-3) / 1e12
    peak = SMS * ALU_LANES * SM_MAX_GHZ * 1e9 / 1e12
    return {"workload": WORKLOADS["batch512"], "families": len(fams), "cells": cells,
            "batch_ms": batch_ms, "batch_gcups": cells / (batch_ms * 1e-3) / 1e9,
            "plain_ms": plain_ms, "plain_gcups": cells / (plain_ms * 1e-3) / 1e9,
            "speedup_vs_plain": plain_ms / batch_ms,
            "lcs_roofline_frac": achieved / peak,
            "note": "batched: famsa_batch_pack + famsa_batch_tree (one CUDA graph) per step; plain: "
                    "famsa_pack_peq + famsa_slink_tree per family, one after another on one stream; "
                    "trees bit-exact either way (tests/test_gpu_batch.py)"}


def run_int_peaks():
    """Instruction rates of independent LOP3 / IADD3 / IMAD chains, as lanes per SM per clock."""
    import torch
    import paper_1603_06958_gb300 as fg
    fg.load()
    torch.cuda.init()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = {"sms": sms, "kinds": {}}
    for kind, name in enumerate(["lop3", "iadd3", "imad", "lop3+imad"]):
        fg.probe_int_pipe_rate(kind)  # warm-up
        clk = ClockSampler(0)
        clk.start()
        rates = [fg.probe_int_pipe_rate(kind) for _ in range(20)]
        c = clk.stop()
        rate = float(np.median(rates))
        mhz = c.get("sm_mhz") or SM_MAX_GHZ * 1e3
        out["kinds"][name] = {"inst_per_s": rate, "sm_mhz": mhz,
                              "lanes_per_sm_per_clk": rate / (sms * mhz * 1e6),
                              "clock_reasons": c.get("reasons")}
    print(json.dumps(out), flush=True)
    return 0


def run_lcs_widths(widths=None, modes=None, reps=3):
    """LCS rate per row width on families of one length: thread-per-pair, the
    sliced kernel and warp-per-pair, as fractions of the ALU-pipe peak, from
    the library's own LCS timers."""
    import torch
    import paper_1603_06958_gb300 as fg
    import synth
    fg.load()
    torch.cuda.init()
    peak = SMS * ALU_LANES * SM_MAX_GHZ * 1e9
    out = []
    # (name, thread-per-pair limit, slice minimum width, words per slice)
    modes_all = [("tpp", 32, 0, 0), ("sliced", 32, 1, 16), ("wpp", 0, 0, 0)]
    for W in widths or (4, 8, 12, 17, 20, 21, 22, 23, 24, 26, 28, 30, 32, 33, 40, 47, 55, 64, 100, 128, 200):
        L = 64 * W - 20
        k = max(1000 if W > 100 else 1500, int(120000 / W))
        res, off = synth.family(k, 300 + W, root_len=L, clip_lo=L, clip_hi=L, indel_rate=0.0)
        fam = fg.pack_peq(res, off)
        row = {"W": W, "len": L, "k": k}
        for name, tmax, smin, words in modes_all:
            if name == "tpp" and W > 32 or modes and name not in modes:
                continue
            fg.debug_set_tpp_max_w(tmax)
            fg.debug_set_slices(smin, words)
            best = None
            for _ in range(reps):
                fg.slink_tree(fam)
                st = fam.stats()
                best = st["lcs_ns"] if best is None else min(best, st["lcs_ns"])
            row[name] = round(OPS_PER_WORD_STEP * st["word_steps"] / (best * 1e-9) / peak, 4)
        fg.debug_set_tpp_max_w(32)
        fg.debug_set_slices(24, 0)
        fam.free()
        out.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"lcs_widths": out}), flush=True)
    return 0


def run_cluster_probe():
    """SM clocks of the row update's building blocks on 1- and 16-CTA clusters."""
    import paper_1603_06958_gb300 as fg
    fg.load()
    names = ["block_scan_order_codes", "block_scan_cross_multiplied", "cluster_barrier",
             "push_to_every_cta_and_barrier", "dependent_local_smem_load", "dependent_dsmem_load"]
    out = {}
    for cl in (1, 16):
        row = {}
        for kind, name in enumerate(names):
            fg.probe_cluster(kind, cl)  # warm-up
            row[name] = float(np.median([fg.probe_cluster(kind, cl) for _ in range(5)]))
        out["cluster_%d" % cl] = row
    print(json.dumps({"unit": "SM clocks per repetition", "threads_per_cta": 512, **out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="plain20k", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--k", type=int, default=None, help="override family size (testing)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="plain20k: skip the k=400,000 step and the batched-vs-plain run that "
                         "follow the headline steps")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=2.0,
                    help="--impl reference: host seconds of oracle work per step")
    ap.add_argument("--update-path", type=int, default=0, choices=[0, 1, 2, 3],
                    help="row-update kernel: 0 automatic, 1 cluster shared memory, 2 global memory "
                         "(profiling; the default picks by family size)")
    ap.add_argument("--global-variant", type=int, default=-1, choices=[-1, 0, 1],
                    help="global-memory row update: -1 by size (default), 0 = 1,024 threads a CTA, 1 = 512")
    ap.add_argument("--no-plain", action="store_true",
                    help="batch512: skip timing the one-family-at-a-time comparator")
    ap.add_argument("--cluster-probe", action="store_true",
                    help="time the row update's building blocks (scans, barriers, DSMEM) and exit")
    ap.add_argument("--lcs-widths", action="store_true",
                    help="LCS rate per row width: thread-per-pair, sliced and warp-per-pair kernels")
    ap.add_argument("--widths", default="",
                    help="with --lcs-widths: comma-separated row widths in 64-bit words (default: the sweep)")
    ap.add_argument("--modes", default="",
                    help="with --lcs-widths: comma-separated kernels among tpp, sliced, wpp (default: all)")
    ap.add_argument("--reps", type=int, default=3, help="with --lcs-widths: tree calls per kernel")
    ap.add_argument("--int-peaks", action="store_true",
                    help="measure the integer pipe widths used by the roofline, then exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.int_peaks:
        return run_int_peaks()
    if args.cluster_probe:
        return run_cluster_probe()
    if args.lcs_widths:
        return run_lcs_widths([int(w) for w in args.widths.split(",") if w] or None,
                              [m for m in args.modes.split(",") if m] or None, args.reps)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    arm = {"batch512": run_batch, "serve": run_serve}.get(args.workload, run_ours)
    rc = arm(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
