"""Seeded random cases over every base case (50: ten per base case), Strassen-Winograd depths,
accumulate mode and user strides, each bit-exact against the CPU oracle.

Strides are padded beyond the logical width by random even amounts and the
padding words and tail bits of A and B hold random garbage, which the
library must ignore; C's padding words must come back untouched.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_same_bits, to_dev, to_host

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


def with_garbage(X, cols, extra, rng):
    """X (packed) copied into a stride `extra` words wider (rounded up to
    even); padding words and the tail bits of the last word are random."""
    rows = X.shape[0]
    W = synth.words_for(cols)
    stride = W + extra + (W + extra) % 2
    out = rng.integers(0, 2**64, size=(rows, stride), dtype=np.uint64)
    if W:
        out[:, :W] = X[:, :W]
        if cols % 64:
            keep = synth.tail_mask(cols)
            out[:, W - 1] = (X[:, W - 1] & keep) | (rng.integers(0, 2**64, size=rows, dtype=np.uint64) & ~keep)
    return np.ascontiguousarray(out)


CASES = []
_r = np.random.default_rng(20260)
for _i in range(50):
    base = [g.GF2_BASE_M4RM, g.GF2_BASE_TC_FP8, g.GF2_BASE_TC_S8, g.GF2_BASE_TC_B1, g.GF2_BASE_TC_FP4][_i % 5]
    depth = int(_r.integers(0, 3))
    m, l, n = (int(x) for x in _r.integers(1, 2600, size=3))
    if depth:
        m, l, n = m + 256, l + 256, n + 256
    CASES.append((base, depth, m, l, n, int(_r.integers(0, 2)), int(_r.integers(0, 3)) * 2, _i))


@pytest.mark.parametrize("base,depth,m,l,n,acc,extra,seed", CASES)
def test_fuzz_against_oracle(base, depth, m, l, n, acc, extra, seed):
    rng = np.random.default_rng(seed)
    A = synth.random_packed(m, l, 100 + seed, p=float(rng.uniform(0.05, 0.95)))
    B = synth.random_packed(l, n, 200 + seed, p=float(rng.uniform(0.05, 0.95)))
    ref = oracle.mul_packed(A, B, m, l, n)
    Ag, Bg = with_garbage(A, l, extra, rng), with_garbage(B, n, extra, rng)
    Wc = synth.words_for(n)
    C0 = rng.integers(0, 2**64, size=(m, Wc + extra + (Wc + extra) % 2), dtype=np.uint64)
    if Wc and n % 64:
        C0[:, Wc - 1] &= synth.tail_mask(n)          # a valid C: tail bits zero
    Ad, Bd, Cd = to_dev(Ag), to_dev(Bg), to_dev(C0)
    g.gf2_mul(g.mat(Cd, n), g.mat(Ad, l), g.mat(Bd, n), g.opts(base=base, depth=depth, accumulate=acc))
    g.gf2_device_status()
    got = to_host(Cd)
    expect = (ref[:, :Wc] ^ C0[:, :Wc]) if acc else ref[:, :Wc]
    assert_same_bits(np.ascontiguousarray(got[:, :Wc]), np.ascontiguousarray(expect), n,
                     "case %d base %d depth %d %s acc %d" % (seed, base, depth, (m, l, n), acc))
    # words beyond the logical width belong to the caller
    assert np.array_equal(got[:, Wc:], C0[:, Wc:]), "padding words of C changed"
