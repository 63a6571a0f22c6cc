"""Peeling (Section 4) instead of padding for sizes that do not halve evenly:
Strassen-Winograd on the core, the leftover rows, columns and K entries by
base-case products.  Bit-exact against the CPU oracle, and on the
rectangular 20000x12000 . 12000x28000 case by sampled oracle blocks and
Freivalds' test."""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_same_bits, to_dev, to_host, valid_words

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0811_1714_gb300 as g  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g.build()
    g.lib()
    yield
    torch.cuda.synchronize()


@pytest.mark.parametrize("base,depth,m,l,n", [
    (g.GF2_BASE_M4RM, 1, 1301, 1500, 1100), (g.GF2_BASE_M4RM, 2, 1300, 1700, 2100),
    (g.GF2_BASE_TC_FP8, 1, 1025, 1100, 1300), (g.GF2_BASE_TC_FP8, 2, 2047, 2049, 2050),
    (g.GF2_BASE_M4RM, 2, 4095, 4095, 4095), (g.GF2_BASE_M4RM, 3, 4100, 4300, 4200),
    (g.GF2_BASE_M4RM, 1, 300, 100, 300)])
@pytest.mark.parametrize("acc", [0, 1])
def test_peeled_product_parity(base, depth, m, l, n, acc):
    A = synth.random_packed(m, l, 3 + m)
    B = synth.random_packed(l, n, 4 + n)
    C0 = synth.random_packed(m, n, 5) if acc else None
    ref = oracle.mul_packed(A, B, m, l, n)
    if acc:
        ref = ref ^ C0
    Ad, Bd = to_dev(A), to_dev(B)
    Cd = to_dev(C0) if acc else g.empty(m, n)
    if not acc:
        Cd.fill_(-1)
    g.gf2_mul(g.mat(Cd, n), g.mat(Ad, l), g.mat(Bd, n), g.opts(base=base, depth=depth, peel=1, accumulate=acc))
    g.gf2_device_status()
    assert_same_bits(to_host(Cd), ref, n, "peel %s" % ((base, depth, m, l, n, acc),))


def test_peeled_rectangular_20000_12000_28000():
    m, l, n = 20000, 12000, 28000
    A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
    MA, MB, MC = g.mat(A, l), g.mat(B, n), g.mat(C, n)
    g.gf2_random(MA, 5)
    g.gf2_random(MB, 6)
    o = g.opts(base=g.GF2_BASE_M4RM, depth=2, peel=1)
    assert "peel core=" in g.gf2_describe_plan(m, l, n, o)
    g.gf2_mul(MC, MA, MB, o)
    g.gf2_device_status()
    assert g.gf2_freivalds(MC, MA, MB, synth.SEED_FREIVALDS) == 0
    rng = np.random.default_rng(77)
    # blocks inside the core, in the leftover columns and touching the last row
    for r0, c0 in ((int(rng.integers(0, 19000)), 64 * int(rng.integers(0, 400))), (19936, 27648), (5000, 27904)):
        Ar = synth.random_packed(64, l, 5, row0=r0)
        Bc = synth.random_packed_cols(l, n, 6, c0, min(c0 + 64, n))
        cols = min(64, n - c0)
        ref = oracle.mul_packed(Ar, Bc, 64, l, cols)
        got = np.ascontiguousarray(to_host(C[r0:r0 + 64, c0 // 64:c0 // 64 + 1].contiguous()))
        assert np.array_equal(valid_words(got, cols), valid_words(ref, cols)), (r0, c0)


@pytest.mark.parametrize("n,expect_peel", [(33768, True), (32767, False)])
def test_autotuner_chooses_padding_or_peeling(n, expect_peel):
    """peel = -1 (the default): the first call for a shape times both and keeps
    the faster.  Just above 2^15 the padded leaves (2176 rows) fit the tiles
    badly and peeling wins by a wide margin; just below it padding wins."""
    A, B, C = g.empty(n, n), g.empty(n, n), g.empty(n, n)
    MA, MB, MC = g.mat(A, n), g.mat(B, n), g.mat(C, n)
    g.gf2_random(MA, 91)
    g.gf2_random(MB, 92)
    o = g.opts(base=g.GF2_BASE_M4RM, depth=4)
    g.gf2_mul(MC, MA, MB, o)                 # chooses (and leaves C = A B)
    assert g.gf2_freivalds(MC, MA, MB, 93) == 0
    g.gf2_mul(MC, MA, MB, o)                 # the cached choice
    g.gf2_device_status()
    assert g.gf2_freivalds(MC, MA, MB, 94) == 0
    plan = g.gf2_describe_plan(n, n, n, o)
    assert ("peel core=" in plan) == expect_peel, plan
    del A, B, C
    torch.cuda.empty_cache()
