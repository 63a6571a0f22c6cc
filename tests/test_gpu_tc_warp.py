"""Parity of the warp-level tensor-core base cases: 0/1 int8 products and
1-bit AND + popcount on the packed words, both with int32 sums.

Bit-exact against the CPU oracle.  int32 sums are exact for any K below
2^31, so the all-ones operands (every dot product equals K) are checked at a
K far beyond the FP8 form's chunk bound.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_same_bits, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0811_1714_gb300 as g  # noqa: E402

BASES = {"tc_s8": g.GF2_BASE_TC_S8, "tc_b1": g.GF2_BASE_TC_B1}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g.build()
    g.lib()
    yield
    torch.cuda.synchronize()


@pytest.fixture(params=sorted(BASES))
def base(request):
    return request.param


def warp_mul(base, A, B, m, l, n, depth=0, accumulate=0, C0=None):
    Ad, Bd = to_dev(A), to_dev(B)
    C = to_dev(C0) if C0 is not None else g.empty(m, n)
    if C0 is None:
        C.fill_(-1)
    g.gf2_mul(g.mat(C, n), g.mat(Ad, l), g.mat(Bd, n),
              g.opts(base=BASES[base], depth=depth, accumulate=accumulate))
    g.gf2_device_status()
    return to_host(C)


@pytest.mark.parametrize("m,l,n", [
    (128, 256, 128), (1, 1, 1), (200, 300, 500), (130, 4097, 300), (129, 33, 65), (300, 9000, 700),
    (1024, 1000, 1100), (257, 511, 129)])
def test_base_case_parity(base, m, l, n):
    A = synth.random_packed(m, l, synth.SEED_A)
    B = synth.random_packed(l, n, synth.SEED_B)
    assert_same_bits(warp_mul(base, A, B, m, l, n), oracle.mul_packed(A, B, m, l, n), n,
                     "%s %s" % (base, (m, l, n)))


@pytest.mark.parametrize("l", [31, 32, 33, 255, 256, 257, 70001])
def test_all_ones(base, l):
    m, n = 130, 200
    A = synth.pack_bits(np.ones((m, l), np.uint8))
    B = synth.pack_bits(np.ones((l, n), np.uint8))
    expect = synth.pack_bits(np.full((m, n), l & 1, np.uint8))
    assert_same_bits(warp_mul(base, A, B, m, l, n), expect, n, "%s ones l=%d" % (base, l))


def test_garbage_beyond_k_is_ignored(base):
    """Bits of A and B past column l are random: the K tail must be masked."""
    m, l, n = 150, 300, 170
    A = synth.random_packed(m, l, 3)
    B = synth.random_packed(l, n, 4)
    ref = oracle.mul_packed(A, B, m, l, n)
    Ag = A.copy()
    Ag[:, synth.words_for(l) - 1] |= ~synth.tail_mask(l)      # the last word holding entries
    Bg = B.copy()
    Bg[:, synth.words_for(n) - 1] |= ~synth.tail_mask(n)
    assert_same_bits(warp_mul(base, Ag, Bg, m, l, n), ref, n, base + " tail garbage")


@pytest.mark.parametrize("m,l,n,depth", [(1024, 1024, 1024, 1), (1500, 2100, 1300, 2)])
def test_under_strassen_winograd(base, m, l, n, depth):
    A = synth.random_packed(m, l, synth.SEED_A)
    B = synth.random_packed(l, n, synth.SEED_B)
    assert_same_bits(warp_mul(base, A, B, m, l, n, depth=depth), oracle.mul_packed(A, B, m, l, n), n,
                     "%s depth %d" % (base, depth))


def test_accumulate_and_plan(base):
    m, l, n = 300, 700, 500
    assert "base=%s" % base in g.gf2_describe_plan(m, l, n, g.opts(base=BASES[base], depth=0))
    A = synth.random_packed(m, l, 7, p=0.9)
    B = synth.random_packed(l, n, 8, p=0.9)
    C0 = synth.random_packed(m, n, 9)
    ref = oracle.mul_packed(A, B, m, l, n) ^ C0
    assert_same_bits(warp_mul(base, A, B, m, l, n, accumulate=1, C0=C0), ref, n, base + " accumulate")


def test_profile_family(base):
    """The launches are counted under the base case's own family."""
    fam = list(g.PROFILE_FAMILIES).index(base)
    A = synth.random_packed(256, 512, 1)
    B = synth.random_packed(512, 256, 2)
    g.gf2_profile_enable(True)
    warp_mul(base, A, B, 256, 512, 256)
    ms, launches = g.gf2_profile_read(fam)
    g.gf2_profile_enable(False)
    assert launches == 1 and ms > 0
