"""The row update's building blocks as the library's microbenchmark times
them: order-code keys make the block clamp scan cheaper than cross-multiplied
ones, and a load from another CTA's shared memory costs more than a local one."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fg():
    from paper_1603_06958_gb300 import build
    build.build()
    import paper_1603_06958_gb300 as m
    m.load()
    return m


def test_cluster_building_blocks(fg):
    codes = fg.debug_cluster_probe(0, 16)
    cross = fg.debug_cluster_probe(1, 16)
    local = fg.debug_cluster_probe(4, 16)
    remote = fg.debug_cluster_probe(5, 16)
    barrier = fg.debug_cluster_probe(2, 16)
    assert 0 < codes < cross
    assert 0 < local < remote
    assert barrier > 0
    with pytest.raises(fg.FamsaError):
        fg.debug_cluster_probe(0, 3)
