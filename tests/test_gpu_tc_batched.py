"""The batched form on the tcgen05 base cases (FP8 and FP4): many products of
uneven shapes in one batched transpose, one batched expansion and one
persistent tensor-core launch.

Bit-exact against the CPU oracle on ragged batches (tails in every
dimension, K extents across the exact-sum chunk bound, accumulate mode,
empty products), through a graph replay with new contents, and on the
4096-product batch of log-uniform shapes in [64, 2048] by sampled blocks
(oracle) plus Freivalds' test on every product.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_same_bits, to_dev, to_host, valid_words

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0811_1714_gb300 as g  # noqa: E402

@pytest.fixture(params=[g.GF2_BASE_TC_FP8, g.GF2_BASE_TC_FP4], ids=["fp8", "fp4"])
def TC0(request):
    return dict(base=request.param, depth=0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g.build()
    g.lib()
    yield
    torch.cuda.synchronize()


def make_batch(dims, seed0, C0_seed=None):
    b = dict(hostA=[], hostB=[], hostC0=[], dA=[], dB=[], dC=[], MA=[], MB=[], MC=[])
    for i, (m, l, n) in enumerate(dims):
        A = synth.random_packed(m, l, seed0 + 2 * i)
        B = synth.random_packed(l, n, seed0 + 2 * i + 1)
        b["hostA"].append(A)
        b["hostB"].append(B)
        b["dA"].append(to_dev(A))
        b["dB"].append(to_dev(B))
        if C0_seed is None:
            C = g.empty(m, n)
            C.fill_(-1)                       # every word is overwritten
            b["hostC0"].append(None)
        else:
            C0 = synth.random_packed(m, n, C0_seed + i)
            C = to_dev(C0)
            b["hostC0"].append(C0)
        b["dC"].append(C)
        b["MA"].append(g.mat(b["dA"][-1], l))
        b["MB"].append(g.mat(b["dB"][-1], n))
        b["MC"].append(g.mat(C, n))
    b["arrs"] = g.MatArrays(b["MC"], b["MA"], b["MB"])
    return b


def check_batch(b, dims, what):
    for i, (m, l, n) in enumerate(dims):
        if m == 0 or n == 0:
            continue
        ref = oracle.mul_packed(b["hostA"][i], b["hostB"][i], m, l, n)
        if b["hostC0"][i] is not None:
            ref = ref ^ b["hostC0"][i]
        assert_same_bits(to_host(b["dC"][i]), ref, n, "%s %s" % (what, (m, l, n)))


RAGGED = [(1, 1, 1), (128, 128, 256), (65, 63, 129), (300, 700, 100), (1000, 90, 1030),
          (17, 2048, 5), (513, 257, 511), (2048, 300, 2048), (129, 1, 300), (7, 4000, 260),
          (130, 4097, 300), (200, 9000, 70)]


def test_tc_batched_ragged(TC0):
    b = make_batch(RAGGED, 700)
    g.gf2_mul_batched(b["arrs"], options=g.opts(**TC0))
    g.gf2_device_status()
    check_batch(b, RAGGED, "tc batched")


def test_tc_batched_accumulate(TC0):
    b = make_batch(RAGGED, 710, C0_seed=9000)
    g.gf2_mul_batched(b["arrs"], options=g.opts(accumulate=1, **TC0))
    g.gf2_device_status()
    check_batch(b, RAGGED, "tc batched accumulate")


def test_tc_batched_all_ones_chunk_bound(TC0):
    """All-ones operands: every dot product equals K, the largest chunk sum."""
    dims = [(256, 4096, 512), (130, 4097, 300), (64, 8192, 64), (64, 8193, 70), (129, 16385, 64)]
    hostA = [synth.pack_bits(np.ones((m, l), np.uint8)) for m, l, n in dims]
    hostB = [synth.pack_bits(np.ones((l, n), np.uint8)) for m, l, n in dims]
    dA, dB, dC = [to_dev(x) for x in hostA], [to_dev(x) for x in hostB], [g.empty(m, n) for m, l, n in dims]
    arrs = g.MatArrays([g.mat(c, n) for c, (m, l, n) in zip(dC, dims)],
                       [g.mat(a, l) for a, (m, l, n) in zip(dA, dims)],
                       [g.mat(x, n) for x, (m, l, n) in zip(dB, dims)])
    g.gf2_mul_batched(arrs, options=g.opts(**TC0))
    g.gf2_device_status()
    for i, (m, l, n) in enumerate(dims):
        expect = synth.pack_bits(np.full((m, n), l & 1, np.uint8))
        assert_same_bits(to_host(dC[i]), expect, n, "ones %s" % ((m, l, n),))


def test_tc_batched_empty_products_and_replay(TC0):
    """Empty products beside real ones; the second call replays the cached
    graph on new contents and must clear the K = 0 products again."""
    dims = [(70, 0, 90), (0, 50, 40), (60, 50, 0), (300, 500, 200), (129, 4100, 257)]
    b = make_batch(dims, 720)
    o = g.opts(**TC0)
    g.gf2_mul_batched(b["arrs"], options=o)
    g.gf2_device_status()
    check_batch(b, dims, "tc empty")
    assert not to_host(b["dC"][0]).any()
    for i, (m, l, n) in enumerate(dims):
        A2 = synth.random_packed(m, l, 4000 + i)
        if A2.size:
            b["dA"][i].copy_(to_dev(A2))
        b["hostA"][i] = A2
        b["dC"][i].fill_(-1)
    before = g.gf2_launch_count()
    g.gf2_mul_batched(b["arrs"], options=o)
    g.gf2_device_status()
    assert g.gf2_launch_count() - before == 3          # batched transpose, expansion, product kernel
    check_batch(b, dims, "tc replay")
    assert not to_host(b["dC"][0]).any()


def test_tc_batched_matches_m4rm_batched(TC0):
    dims = synth.batch_dims(40, seed=11, lo=32, hi=1500)
    bt = make_batch(dims, 800)
    bm = make_batch(dims, 800)
    g.gf2_mul_batched(bt["arrs"], options=g.opts(**TC0))
    g.gf2_mul_batched(bm["arrs"], options=g.opts(base=g.GF2_BASE_M4RM, depth=0))
    g.gf2_device_status()
    for i, (m, l, n) in enumerate(dims):
        assert np.array_equal(valid_words(to_host(bt["dC"][i]), n), valid_words(to_host(bm["dC"][i]), n)), i
    check_batch(bt, dims[:8], "tc vs oracle")


def test_tc_batch_of_4096_log_uniform_products(TC0):
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
    g.gf2_mul_batched(arrs, options=g.opts(**TC0))
    g.gf2_device_status()
    torch.cuda.synchronize()
    rng = np.random.default_rng(4097)
    for i in rng.choice(len(dims), 32, replace=False):
        m, l, n = dims[i]
        r0 = int(rng.integers(0, max(1, m - 128))) if m > 128 else 0
        c0 = 64 * int(rng.integers(0, max(1, (n - 128) // 64))) if n > 128 else 0
        rows, cols = min(128, m - r0), min(128, n - c0)
        A = synth.random_packed(rows, l, 10_000 + 2 * i, row0=r0)
        Bblk = synth.random_packed_cols(l, n, 10_001 + 2 * i, c0, c0 + cols)
        ref = oracle.mul_packed(A, Bblk, rows, l, cols)
        got = to_host(keep[i][2])[r0:r0 + rows]
        got = np.ascontiguousarray(got[:, c0 // 64:c0 // 64 + synth.words_for(cols)])
        assert np.array_equal(valid_words(got, cols), valid_words(ref, cols)), (i, r0, c0)
    bad = [i for i in range(len(dims)) if g.gf2_freivalds(MC[i], MA[i], MB[i], 177 + i) != 0]
    assert not bad, bad[:10]
