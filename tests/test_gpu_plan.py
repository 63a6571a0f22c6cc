"""The M4RM tile-height and K-split choices on this GPU (152 SMs), pinned at
the shapes where they were measured (`bench.py --workload sweep`): tall
tensor-memory tiles wherever their partly empty last wave still costs less
than shorter tiles, 256-row tiles for ragged 2111-row leaves, and a K split
only when two splits of every tile fit in one wave."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0811_1714_gb300 as g  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("tile choices pinned for a 152-SM GB300")
    g.build()
    g.lib()
    yield


def fields(m, l, n, **kw):
    p = g.gf2_describe_plan(m, l, n, g.opts(base=g.GF2_BASE_M4RM, peel=0, **kw))
    return dict(x.split("=", 1) for x in p.split() if "=" in x)


@pytest.mark.parametrize("m,l,n,depth,rows,ksplit", [
    (32768, 32768, 32768, 4, "2048", "1"),     # the headline: 2401 leaves of 2048^3
    (16384, 16384, 16384, 0, "2048", "1"),     # 128 tiles: one partly empty wave of tall tiles
    (8192, 8192, 8192, 2, "2048", "1"),        # 49 leaves of 2048^3
    (1024, 1024, 1024, 0, "64", "10"),         # config 1: 16 tiles, K split ten ways
    (33768, 33768, 33768, 4, "256", "1"),      # padded leaves of 2111 rows
])
def test_tile_height_and_k_split(m, l, n, depth, rows, ksplit):
    f = fields(m, l, n, depth=depth)
    assert (f["tile_rows"], f["ksplit"]) == (rows, ksplit), f


def test_requested_k_keeps_its_own_tile():
    """A k whose tables do not fit the tall tiles falls back to 1024-row tiles."""
    f = fields(16384, 16384, 16384, depth=0, k=7)
    assert (f["m4rm_k"], f["tile_rows"]) == ("7", "1024"), f
