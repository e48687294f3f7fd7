"""Build libfamsa_gpu.so in-tree for sm_103a (nvcc, parallel translation units).

With --checked (or build(checked=True)) it also builds
libfamsa_gpu_checked.so: the same sources with -DFAMSA_CHECKED, whose kernels
count every failed invariant (an index outside its buffer, a row wider than
its kernel) instead of trusting it.  The binding loads that library when
FAMSA_CHECKED=1 is set in the environment.

Usage: python -m paper_1603_06958_gb300.build [--force] [--checked]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfamsa_gpu.so")
OBJ_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libfamsa_gpu_checked.so")
ROOT = os.path.dirname(HERE)

SOURCES = ["api.cu", "pack.cu", "lcs.cu", "lcs_tpp_a.cu", "lcs_tpp_b.cu", "lcs_tpp_c.cu", "lcs_tpp_d.cu",
           "lcs_slice_a.cu", "lcs_slice_b.cu", "lcs_wpp.cu", "slink.cu", "slink_global.cu", "slink_smem.cu", "slink_msf.cu", "shard.cu", "schedule.cu", "gaps.cu", "upgma.cu", "finalize.cu",
           "noalloc.cu", "batch.cu", "server.cu"]
# microbenchmarks behind the roofline figures: a separate library that only
# bench.py loads (--int-peaks, --cluster-probe), not part of the product ABI
PROBE_SOURCES = ["probes/int_peak.cu", "probes/cluster_probe.cu"]
PROBE_LIB = os.path.join(HERE, "libfamsa_probe.so")
HEADERS = [os.path.join(ROOT, "include", "famsa_probe.h"), "famsa_internal.cuh", "lcs_kernels.cuh", "lcs_step.inc", "slink_common.cuh", "slink_msf.cuh",
           "slink_merge.cuh", os.path.join(ROOT, "include", "famsa_gpu_debug.h"),
           os.path.join(ROOT, "include", "famsa_gpu.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _mtime(p):
    return os.path.getmtime(p) if os.path.exists(p) else 0.0


def _gen_step():
    gen = os.path.join(CSRC, "gen_lcs_step.py")
    inc = os.path.join(CSRC, "lcs_step.inc")
    if _mtime(inc) < _mtime(gen):
        out = subprocess.check_output([sys.executable, gen])
        with open(inc + ".tmp", "wb") as f:
            f.write(out)
        os.replace(inc + ".tmp", inc)


def _build_lib(sources, lib, force, verbose, ptxas_v, obj_dir=OBJ, extra=()):
    os.makedirs(obj_dir, exist_ok=True)
    hdr = max(_mtime(h if os.path.isabs(h) else os.path.join(CSRC, h)) for h in HEADERS)
    jobs = []
    objs = []
    for s in sources:
        src = os.path.join(CSRC, s)
        obj = os.path.join(obj_dir, s.replace("/", "_").replace(".cu", ".o"))
        objs.append(obj)
        if force or _mtime(obj) < max(_mtime(src), hdr):
            cmd = [nvcc()] + ARCH + FLAGS + list(extra) + (["-Xptxas", "-v"] if ptxas_v else []) + \
                ["-c", src, "-o", obj]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = [ex.submit(subprocess.run, j, capture_output=True, text=True) for j in jobs]
            for j, fu in zip(jobs, futs):
                r = fu.result()
                if verbose or ptxas_v:
                    sys.stderr.write(r.stderr)
                if r.returncode != 0:
                    sys.stderr.write(" ".join(j) + "\n" + r.stdout + r.stderr)
                    raise RuntimeError("nvcc failed for %s" % j[-3])
    if force or jobs or _mtime(lib) < max(_mtime(o) for o in objs):
        tmp = lib + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, lib)
    return lib


def build(force: bool = False, verbose: bool = False, ptxas_v: bool = False, checked: bool = False) -> str:
    """Build libfamsa_gpu.so (and the benchmark's probe library beside it);
    with checked=True also libfamsa_gpu_checked.so."""
    _gen_step()
    _build_lib(SOURCES, LIB, force, verbose, ptxas_v)
    _build_lib(PROBE_SOURCES, PROBE_LIB, force, verbose, ptxas_v)
    if checked:
        _build_lib(SOURCES, LIB_CHECKED, force, verbose, ptxas_v, OBJ_CHECKED, ["-DFAMSA_CHECKED"])
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_v="--ptxas-v" in sys.argv,
          checked="--checked" in sys.argv)
