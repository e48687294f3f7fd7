import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(autouse=True)
def no_failed_kernel_check(request):
    """Under FAMSA_CHECKED=1 (the checked build), every GPU test must leave
    the library's count of failed kernel checks where it found it."""
    if os.environ.get("FAMSA_CHECKED") != "1" or "gpu" not in request.keywords:
        yield
        return
    import paper_1603_06958_gb300 as fg
    fg.load()
    before, _ = fg.debug_check_count()
    assert before >= 0, "FAMSA_CHECKED=1 but the normal library was loaded"
    yield
    import torch
    torch.cuda.synchronize()
    after, line = fg.debug_check_count()
    assert after == before, "%d failed kernel checks (the first at source line %d)" % (after - before, line)
