"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the benchmark times (automatic Strassen depth, each base case).

The oracle cannot multiply these matrices whole, so each run is checked on
sampled 64 x 64 blocks of C that the oracle computes from the same seeded
inputs drawn independently on the host (rows of A, columns of B), and on
every row by Freivalds' test with 64 random vectors (a wrong C passes with
probability at most 2^-64).  The device generator that makes the inputs is
checked bit for bit against the host generator in test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import to_host, valid_words

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


def check_product(m, l, n, base, p=0.5, seeds=(1, 2), blocks=4, depth=-1):
    A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
    MA, MB, MC = g.mat(A, l), g.mat(B, n), g.mat(C, n)
    g.gf2_random(MA, seeds[0], p)
    g.gf2_random(MB, seeds[1], p)
    o = g.opts(base=base, depth=depth)
    plan = g.gf2_describe_plan(m, l, n, o)
    g.gf2_mul(MC, MA, MB, o)
    g.gf2_device_status()
    assert g.gf2_freivalds(MC, MA, MB, synth.SEED_FREIVALDS) == 0, plan
    rng = np.random.default_rng(m ^ (l << 1) ^ (n << 2) ^ base)
    # one 1024 x 1024 block, then smaller 64 x 64 ones, all drawn on the host
    for i in range(blocks):
        h = 1024 if i == 0 else 64
        r0 = int(rng.integers(0, m - h))
        c0 = 64 * int(rng.integers(0, (n - h) // 64))
        Ar = synth.random_packed(h, l, seeds[0], p, row0=r0)
        Bc = synth.random_packed_cols(l, n, seeds[1], c0, c0 + h, p)
        ref = oracle.mul_packed(Ar, Bc, h, l, h)
        got = C[r0:r0 + h, c0 // 64:c0 // 64 + h // 64]
        got = np.ascontiguousarray(to_host(got.contiguous()))
        assert np.array_equal(valid_words(got, h), valid_words(ref, h)), (plan, r0, c0, h)
    del A, B, C
    torch.cuda.empty_cache()


@pytest.mark.parametrize("base", [g.GF2_BASE_M4RM, g.GF2_BASE_TC_FP8, g.GF2_BASE_TC_FP4, g.GF2_BASE_TC_S8,
                                  g.GF2_BASE_TC_B1])
def test_square_32768(base):
    check_product(32768, 32768, 32768, base)


@pytest.mark.parametrize("base", [g.GF2_BASE_M4RM, g.GF2_BASE_TC_FP8, g.GF2_BASE_TC_FP4])
def test_rectangular_20000_12000_28000(base):
    """Widths 12000 and 28000 are not multiples of 64 (padding in every level)."""
    check_product(20000, 12000, 28000, base, seeds=(5, 6))


@pytest.mark.parametrize("base,p", [(g.GF2_BASE_M4RM, 0.5), (g.GF2_BASE_TC_FP8, 0.5), (g.GF2_BASE_TC_FP4, 0.5),
                                    (g.GF2_BASE_M4RM, 0.9), (g.GF2_BASE_TC_FP8, 0.9), (g.GF2_BASE_TC_FP4, 0.9)])
def test_square_65536(base, p):
    check_product(65536, 65536, 65536, base, p=p, seeds=(11, 12), blocks=2)


def test_square_16384_every_depth():
    for d in range(0, 4):
        check_product(16384, 16384, 16384, g.GF2_BASE_M4RM, seeds=(21, 22), blocks=1, depth=d)
