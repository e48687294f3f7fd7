"""The checked build: libfamsa_gpu_checked.so, the same sources compiled with
-DFAMSA_CHECKED, whose kernels test the invariants their indexing relies on
(indices inside their buffers, rows inside their kernel's width, component
ids inside their range) and count each failure, skipping the access it
guards, instead of trusting it.  No memory checker runs on this GPU pool, so
this build stands in for one: the parity tests of every path run against it
in a child process, and after each test the library's count of failed checks
must not have moved (tests/conftest.py).  The file is collected after the
other GPU parity files, so that a stop at the first failure has run them."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# every GPU parity file but the k = 400,000 runs (minutes, and the same
# kernels as the smaller families here) and this file
FILES = ["test_gpu_pack.py", "test_gpu_lcs.py", "test_gpu_tree.py", "test_gpu_batch.py", "test_gpu_shard.py",
         "test_gpu_schedule.py", "test_gpu_gaps.py", "test_gpu_upgma.py", "test_gpu_nj.py", "test_gpu_serve.py",
         "test_zz_no_alloc.py"]


IN_CHECKED = os.environ.get("FAMSA_CHECKED") == "1"


@pytest.mark.skipif(IN_CHECKED, reason="already running the checked build")
def test_parity_tests_pass_the_checked_build_without_a_failed_check():
    from paper_1603_06958_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, FAMSA_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider"]
    cmd += [os.path.join("tests", f) for f in FILES]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout.splitlines()[-1]


@pytest.mark.skipif(IN_CHECKED, reason="this process runs the checked build")
def test_the_checked_build_counts_and_the_normal_one_does_not():
    import paper_1603_06958_gb300 as fg
    from paper_1603_06958_gb300 import build
    fg.load()
    assert fg.debug_check_count() == (-1, 0)  # this process runs the normal build
    assert fg.debug_check_selftest() == -1
    # in the checked build a failing check is counted, with its source line
    build.build(checked=True)
    code = ("import paper_1603_06958_gb300 as fg; fg.load(); n0, _ = fg.debug_check_count(); "
            "assert fg.debug_check_selftest() == 0; n1, line = fg.debug_check_count(); print(n1 - n0, line)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, FAMSA_CHECKED="1"),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    moved, line = (int(x) for x in r.stdout.split())
    assert moved == 1 and line > 0
