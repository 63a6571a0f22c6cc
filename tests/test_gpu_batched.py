"""The batched form: many products of uneven shapes in one persistent launch.

Bit-exact against the CPU oracle.  Every tile variant the autotuner can
choose is checked on a ragged batch; the autotuned path is checked through
a graph replay with new contents; the 4096-product batch of log-uniform
shapes in [64, 2048] is checked on sampled sub-blocks (oracle) and on every
product by Freivalds' test.
"""
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


def make_batch(dims, seed0):
    hostA, hostB, dA, dB, dC, MA, MB, MC = [], [], [], [], [], [], [], []
    for i, (m, l, n) in enumerate(dims):
        A = synth.random_packed(m, l, seed0 + 2 * i)
        B = synth.random_packed(l, n, seed0 + 2 * i + 1)
        hostA.append(A)
        hostB.append(B)
        dA.append(to_dev(A))
        dB.append(to_dev(B))
        C = g.empty(m, n)
        C.fill_(-1)
        dC.append(C)
        MA.append(g.mat(dA[-1], l))
        MB.append(g.mat(dB[-1], n))
        MC.append(g.mat(C, n))
    return dict(hostA=hostA, hostB=hostB, dA=dA, dB=dB, dC=dC, arrs=g.MatArrays(MC, MA, MB))


# includes row counts past whole 512-row tall blocks with remainders below,
# between and above the split thresholds (76, 276, 88, 406, 383 rows)
RAGGED = [(1, 1, 1), (64, 64, 64), (65, 63, 129), (300, 700, 100), (1000, 90, 1030),
          (17, 2048, 5), (513, 257, 511), (2048, 300, 2048), (129, 1, 300), (7, 4000, 260),
          (1100, 200, 300), (1300, 65, 700), (1624, 33, 130), (1430, 97, 260), (895, 50, 70)]


NVARIANTS = 16   # 8 one-product-per-tile, 3 slot-packed, 1 tall slot-packed, 4 split variants


@pytest.mark.parametrize("variant", list(range(NVARIANTS)))
def test_every_batched_variant(variant):
    assert g.gf2_batched_variant_count() == NVARIANTS
    bt = make_batch(RAGGED, 500)
    used = g.gf2_mul_batched_ex(bt["arrs"], variant=variant)
    assert used == variant
    torch.cuda.synchronize()
    for i, (m, l, n) in enumerate(RAGGED):
        ref = oracle.mul_packed(bt["hostA"][i], bt["hostB"][i], m, l, n)
        assert_same_bits(to_host(bt["dC"][i]), ref, n, "%s %s" % (g.gf2_batched_variant_name(variant), (m, l, n)))


@pytest.fixture(scope="module")
def ragged_refs():
    bt = make_batch(RAGGED, 500)
    refs = [oracle.mul_packed(bt["hostA"][i], bt["hostB"][i], m, l, n) for i, (m, l, n) in enumerate(RAGGED)]
    return refs


@pytest.mark.parametrize("variant", list(range(NVARIANTS)))
def test_every_batched_variant_accumulates(variant, ragged_refs):
    """C ^= A B through every variant's XOR epilogue (C0 random)."""
    bt = make_batch(RAGGED, 500)
    C0 = []
    for i, (m, l, n) in enumerate(RAGGED):
        c0 = synth.random_packed(m, n, 9100 + i)
        bt["dC"][i].copy_(to_dev(c0))
        C0.append(c0)
    o = g.opts(base=g.GF2_BASE_M4RM, depth=0, accumulate=1)
    used = g.gf2_mul_batched_ex(bt["arrs"], options=o, variant=variant)
    assert used == variant
    torch.cuda.synchronize()
    for i, (m, l, n) in enumerate(RAGGED):
        assert_same_bits(to_host(bt["dC"][i]), ragged_refs[i] ^ C0[i], n,
                         "%s accumulate %s" % (g.gf2_batched_variant_name(variant), (m, l, n)))


def test_autotuned_batch_and_graph_replay():
    dims = synth.batch_dims(60, seed=7, lo=16, hi=900)
    bt = make_batch(dims, 900)
    o = g.opts(base=g.GF2_BASE_M4RM, depth=0)
    v1 = g.gf2_mul_batched_ex(bt["arrs"], options=o)
    assert 0 <= v1 < g.gf2_batched_variant_count()
    torch.cuda.synchronize()
    for i, (m, l, n) in enumerate(dims):
        ref = oracle.mul_packed(bt["hostA"][i], bt["hostB"][i], m, l, n)
        assert_same_bits(to_host(bt["dC"][i]), ref, n, "tuned %s" % ((m, l, n),))
    # new contents in the same buffers: the second call replays the graph
    for i, (m, l, n) in enumerate(dims):
        A2 = synth.random_packed(m, l, 3000 + i)
        bt["dA"][i].copy_(to_dev(A2))
        bt["hostA"][i] = A2
        bt["dC"][i].fill_(-1)
    v2 = g.gf2_mul_batched_ex(bt["arrs"], options=o)
    assert v2 == v1
    torch.cuda.synchronize()
    for i, (m, l, n) in enumerate(dims):
        ref = oracle.mul_packed(bt["hostA"][i], bt["hostB"][i], m, l, n)
        assert_same_bits(to_host(bt["dC"][i]), ref, n, "replay %s" % ((m, l, n),))


def test_batch_of_4096_log_uniform_products():
    """4096 products, every dimension log-uniform in [64, 2048] (seeded)."""
    dims = synth.batch_dims(4096)
    MA, MB, MC, keep = [], [], [], []
    for i, (m, l, n) in enumerate(dims):
        A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
        MA.append(g.mat(A, l)); MB.append(g.mat(B, n)); MC.append(g.mat(C, n))
        g.gf2_random(MA[-1], 10_000 + 2 * i)
        g.gf2_random(MB[-1], 10_001 + 2 * i)
        keep.append((A, B, C))
    arrs = g.MatArrays(MC, MA, MB)
    g.gf2_mul_batched(arrs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(4096)
    # oracle on sampled 128 x 128 blocks of 48 products (inputs drawn on the host)
    for i in rng.choice(len(dims), 48, replace=False):
        m, l, n = dims[i]
        r0 = int(rng.integers(0, max(1, m - 128))) if m > 128 else 0
        c0 = 64 * int(rng.integers(0, max(1, (n - 128) // 64))) if n > 128 else 0
        rows, cols = min(128, m - r0), min(128, n - c0)
        A = synth.random_packed(rows, l, 10_000 + 2 * i, row0=r0)
        Bblk = synth.random_packed_cols(l, n, 10_001 + 2 * i, c0, c0 + cols)
        ref = oracle.mul_packed(A, Bblk, rows, l, cols)
        got = to_host(keep[i][2])[r0:r0 + rows]
        got = np.ascontiguousarray(got[:, c0 // 64:c0 // 64 + synth.words_for(cols)])
        # a sub-block: bits beyond its last column belong to later columns of C
        assert np.array_equal(valid_words(got, cols), valid_words(ref, cols)), (i, r0, c0)
    # Freivalds' test on every product
    bad = [i for i in range(len(dims)) if g.gf2_freivalds(MC[i], MA[i], MB[i], 77 + i) != 0]
    assert not bad, bad[:10]


def test_autotuned_batch_with_accumulate():
    """C ^= A B on a batch whose shape signature has not been tuned yet: the
    autotuner times every variant on the caller's C, which must not leave
    those timing runs' XORs behind (C0 ^ A B after the call, C0 again after
    a second, graph-replayed call)."""
    dims = synth.batch_dims(37, seed=4242, lo=20, hi=700)
    bt = make_batch(dims, 7000)
    C0 = []
    for i, (m, l, n) in enumerate(dims):
        c0 = synth.random_packed(m, n, 8000 + i)
        bt["dC"][i].copy_(to_dev(c0))
        C0.append(c0)
    o = g.opts(base=g.GF2_BASE_M4RM, depth=0, accumulate=1)
    g.gf2_mul_batched_ex(bt["arrs"], options=o)
    torch.cuda.synchronize()
    for i, (m, l, n) in enumerate(dims):
        ref = oracle.mul_packed(bt["hostA"][i], bt["hostB"][i], m, l, n) ^ C0[i]
        assert_same_bits(to_host(bt["dC"][i]), ref, n, "first accumulate %s" % ((m, l, n),))
    g.gf2_mul_batched_ex(bt["arrs"], options=o)
    torch.cuda.synchronize()
    for i, (m, l, n) in enumerate(dims):
        assert_same_bits(to_host(bt["dC"][i]), C0[i], n, "second accumulate %s" % ((m, l, n),))
