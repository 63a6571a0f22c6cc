"""Parity of the tcgen05 tensor-core base cases (0/1 FP8 and block-scaled FP4
products on operands expanded once in HBM, parity of exact sums).

Bit-exact against the CPU oracle.  The adversarial inputs for exactness are
all-ones operands, whose dot products all equal the K extent, the largest
sum a chunk can hold, and staircase right factors, whose dot products take
every value up to K (so a lost low bit of any partial sum flips a parity).
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_same_bits, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0811_1714_gb300 as g  # noqa: E402

TCS = [g.GF2_BASE_TC_FP8, g.GF2_BASE_TC_FP4]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g.build()
    g.lib()
    yield
    torch.cuda.synchronize()


def tc_mul(A, B, m, l, n, depth=0, accumulate=0, C0=None, base=g.GF2_BASE_TC_FP8):
    Ad, Bd = to_dev(A), to_dev(B)
    C = to_dev(C0) if C0 is not None else g.empty(m, n)
    g.gf2_mul(g.mat(C, n), g.mat(Ad, l), g.mat(Bd, n), g.opts(base=base, depth=depth, accumulate=accumulate))
    g.gf2_device_status()
    return to_host(C)


@pytest.mark.parametrize("base", TCS)
@pytest.mark.parametrize("m,l,n", [
    (128, 128, 256), (1, 1, 1), (200, 300, 500), (128, 4096, 256), (130, 4097, 300),
    (1024, 1000, 1100), (300, 9000, 700), (4096, 512, 4096), (129, 257, 257)])
def test_tc_base_case_parity(m, l, n, base):
    A = synth.random_packed(m, l, synth.SEED_A)
    B = synth.random_packed(l, n, synth.SEED_B)
    ref = oracle.mul_packed(A, B, m, l, n)
    assert_same_bits(tc_mul(A, B, m, l, n, base=base), ref, n, "tc %d %s" % (base, (m, l, n)))


@pytest.mark.parametrize("base", TCS)
@pytest.mark.parametrize("l", [4095, 4096, 4097, 8191, 8192, 8193, 12345, 16385])
def test_tc_all_ones_at_the_chunk_bound(l, base):
    """K-chunks of 4096 (FP8) and 8192 (FP4) entries: every dot product is
    the chunk's full count, the largest sum an accumulation holds."""
    m, n = 256, 512
    A = synth.pack_bits(np.ones((m, l), np.uint8))
    B = synth.pack_bits(np.ones((l, n), np.uint8))
    expect = synth.pack_bits(np.full((m, n), l & 1, np.uint8))
    assert_same_bits(tc_mul(A, B, m, l, n, base=base), expect, n, "ones l=%d" % l)


@pytest.mark.parametrize("base", TCS)
@pytest.mark.parametrize("l", [4096, 6144, 8192, 9000, 16400])
def test_tc_staircase_sums(l, base):
    """A all ones, column j of B ones in rows 0..c_j - 1 with c_j running over
    0..l: entry (i, j) of C is c_j mod 2.  Every count up to l occurs, so
    every partial sum of a K-chunk has its low bits exercised."""
    m, n = 130, 520
    c = (np.arange(n) * 4099) % (l + 1)
    c[:5] = [l, l - 1, 4095 if l > 4095 else 1, min(l, 8191), min(l, 8193)]
    Bb = (np.arange(l)[:, None] < c[None, :]).astype(np.uint8)
    A = synth.pack_bits(np.ones((m, l), np.uint8))
    B = synth.pack_bits(Bb)
    expect = synth.pack_bits(np.repeat((c & 1)[None, :].astype(np.uint8), m, axis=0))
    assert_same_bits(tc_mul(A, B, m, l, n, base=base), expect, n, "staircase l=%d" % l)


@pytest.mark.parametrize("base", TCS)
def test_tc_density_09(base):
    m, l, n = 640, 5000, 768
    A = synth.random_packed(m, l, 3, p=0.9)
    B = synth.random_packed(l, n, 4, p=0.9)
    assert_same_bits(tc_mul(A, B, m, l, n, base=base), oracle.mul_packed(A, B, m, l, n), n, "p=0.9")


@pytest.mark.parametrize("base", TCS)
@pytest.mark.parametrize("m,l,n,depth", [(1024, 1024, 1024, 1), (1500, 2100, 1300, 2), (2048, 2048, 2048, 3)])
def test_tc_under_strassen_winograd(m, l, n, depth, base):
    A = synth.random_packed(m, l, synth.SEED_A)
    B = synth.random_packed(l, n, synth.SEED_B)
    ref = oracle.mul_packed(A, B, m, l, n)
    assert_same_bits(tc_mul(A, B, m, l, n, depth=depth, base=base), ref, n, "tc depth %d" % depth)


@pytest.mark.parametrize("base", TCS)
def test_tc_accumulate(base):
    m, l, n = 300, 700, 500
    A = synth.random_packed(m, l, 7)
    B = synth.random_packed(l, n, 8)
    C0 = synth.random_packed(m, n, 9)
    ref = oracle.mul_packed(A, B, m, l, n) ^ C0
    assert_same_bits(tc_mul(A, B, m, l, n, accumulate=1, C0=C0, base=base), ref, n, "tc accumulate")


@pytest.mark.parametrize("base", TCS)
def test_tc_matches_m4rm_on_the_same_inputs(base):
    m = l = n = 4096
    A = synth.random_packed(m, l, 21)
    B = synth.random_packed(l, n, 22)
    Ad, Bd = to_dev(A), to_dev(B)
    C1, C2 = g.empty(m, n), g.empty(m, n)
    g.gf2_mul(g.mat(C1, n), g.mat(Ad, l), g.mat(Bd, n), g.opts(base=base, depth=0))
    g.gf2_mul(g.mat(C2, n), g.mat(Ad, l), g.mat(Bd, n), g.opts(base=g.GF2_BASE_M4RM, depth=0))
    g.gf2_device_status()
    assert torch.equal(C1, C2)
    assert g.gf2_freivalds(g.mat(C1, n), g.mat(Ad, l), g.mat(Bd, n), 1000) == 0



@pytest.mark.parametrize("base", TCS)
@pytest.mark.parametrize("m,l,n", [(300, 700, 500), (1024, 1000, 1100), (129, 4097, 260)])
def test_tc_single_cta_tiles(m, l, n, base, monkeypatch):
    """The same products with one CTA per 128-row tile (GF2_TC_PAIRS=0) instead
    of pairs of CTAs that run one M = 256 MMA stream over both."""
    monkeypatch.setenv("GF2_TC_PAIRS", "0")
    A = synth.random_packed(m, l, 31)
    B = synth.random_packed(l, n, 32)
    ref = oracle.mul_packed(A, B, m, l, n)
    assert_same_bits(tc_mul(A, B, m, l, n, base=base), ref, n, "single-CTA tc %d %s" % (base, (m, l, n)))


@pytest.mark.parametrize("n", [32, 96, 223, 224, 225, 447, 448, 449, 673, 1000, 2240])
@pytest.mark.parametrize("accumulate", [0, 1])
def test_fp4_pair_tile_columns(n, accumulate):
    """FP4 pairs run 224-column tiles (two accumulators beside the scale
    factors), which end on 32-bit boundaries of C's words: widths around the
    tile width and its multiples, with and without C ^= A B, and bits past
    the last column of the last word written as zero (or kept, with
    accumulate)."""
    m, l = 300, 1100
    A = synth.random_packed(m, l, 41)
    B = synth.random_packed(l, n, 42)
    ref = oracle.mul_packed(A, B, m, l, n)
    if accumulate:
        C0 = synth.random_packed(m, n, 43)
        ref = ref ^ C0
    else:
        # garbage everywhere, tail bits included: the product must zero them
        C0 = np.full((m, synth.padded_stride(n)), 0xFFFFFFFFFFFFFFFF, np.uint64)
    got = tc_mul(A, B, m, l, n, accumulate=accumulate, C0=C0, base=g.GF2_BASE_TC_FP4)
    assert_same_bits(got, ref, n, "fp4 pair n=%d acc=%d" % (n, accumulate))
