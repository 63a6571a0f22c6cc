"""gf2_alloc / gf2_free and the bookkeeping calls around them, on a GB300.

The library's own device matrices are checked through the library itself: a
product with the identity (A I = A, an oracle pin) copies an allocated matrix
into a host buffer, because gf2_mul stages host operands.  No raw device
pointer is read from Python.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import assert_same_bits

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


def identity(n):
    return synth.pack_bits(np.eye(n, dtype=np.uint8), synth.padded_stride(n))


def read_back(M, rows, cols):
    """Host copy of an allocated matrix, as M * I through gf2_mul."""
    out = np.full((rows, synth.padded_stride(cols)), 0xA5A5A5A5A5A5A5A5, dtype=np.uint64)
    I = identity(cols)
    g.gf2_mul(g.mat(out, cols), M, g.mat(I, cols), g.opts(base=g.GF2_BASE_M4RM, depth=0))
    return out


@pytest.mark.parametrize("rows,cols", [(1, 1), (3, 65), (100, 128), (257, 1000), (2048, 4097)])
def test_alloc_layout_and_zero_fill(rows, cols):
    M = g.gf2_alloc(rows, cols)
    try:
        assert (M.rows, M.cols) == (rows, cols)
        W = synth.words_for(cols)
        assert M.stride_words == W + (W % 2), "stride: ceil(cols/64) rounded up to even"
        assert M.device == torch.cuda.current_device()
        assert M.data and M.data % 16 == 0
        got = read_back(M, rows, cols)
        assert not np.any(got[:, :W]), "gf2_alloc must zero-fill"
    finally:
        g.gf2_free(M)


@pytest.mark.parametrize("rows,cols", [(0, 5), (5, 0), (0, 0)])
def test_alloc_empty_shapes(rows, cols):
    M = g.gf2_alloc(rows, cols)
    assert M.data is None
    g.gf2_free(M)
    assert M.data is None


def test_free_is_idempotent():
    M = g.gf2_alloc(64, 64)
    assert M.data
    g.gf2_free(M)
    assert M.data is None
    g.gf2_free(M)                       # second call: no-op
    assert M.data is None


def test_alloc_rejects_negative_sizes():
    for rows, cols in [(-1, 5), (5, -1)]:
        with pytest.raises(g.GF2Error) as e:
            g.gf2_alloc(rows, cols)
        assert e.value.status == g.GF2_EINVAL


@pytest.mark.parametrize("m,l,n,depth", [(300, 200, 130, 0), (1100, 700, 900, 0), (1100, 700, 900, 1),
                                         (2500, 1300, 1700, -1)])
def test_product_of_allocated_matrices(m, l, n, depth):
    """gf2_alloc -> gf2_random -> gf2_mul -> gf2_free, against the oracle."""
    A, B, C = g.gf2_alloc(m, l), g.gf2_alloc(l, n), g.gf2_alloc(m, n)
    try:
        g.gf2_random(A, 41)
        g.gf2_random(B, 42)
        g.gf2_mul(C, A, B, g.opts(depth=depth))
        ref = oracle.mul_packed(synth.random_packed(m, l, 41), synth.random_packed(l, n, 42), m, l, n)
        assert_same_bits(read_back(C, m, n), ref, n, "allocated %s depth %d" % ((m, l, n), depth))
        assert g.gf2_freivalds(C, A, B, 7) == 0
    finally:
        for M in (A, B, C):
            g.gf2_free(M)


def test_batched_product_of_allocated_matrices():
    dims = [(70, 130, 90), (300, 64, 257), (513, 700, 65), (1, 1, 1)]
    As = [g.gf2_alloc(m, l) for m, l, _ in dims]
    Bs = [g.gf2_alloc(l, n) for _, l, n in dims]
    Cs = [g.gf2_alloc(m, n) for m, _, n in dims]
    try:
        for i, (A, B) in enumerate(zip(As, Bs)):
            g.gf2_random(A, 500 + i)
            g.gf2_random(B, 600 + i)
        g.gf2_mul_batched(Cs, As, Bs)
        for i, (m, l, n) in enumerate(dims):
            ref = oracle.mul_packed(synth.random_packed(m, l, 500 + i), synth.random_packed(l, n, 600 + i),
                                    m, l, n)
            assert_same_bits(read_back(Cs[i], m, n), ref, n, "batched product %d %s" % (i, dims[i]))
    finally:
        for M in As + Bs + Cs:
            g.gf2_free(M)


def test_reserved_scratch_serves_the_product():
    """After gf2_reserve_scratch(gf2_scratch_bytes(...)) the product runs in
    the reserved arena; releasing it and calling again re-grows it."""
    m = l = n = 2048
    o = g.opts(base=g.GF2_BASE_M4RM, depth=1)
    need = g.gf2_scratch_bytes(m, l, n, o)
    assert need > 0
    A, B, C = g.gf2_alloc(m, l), g.gf2_alloc(l, n), g.gf2_alloc(m, n)
    try:
        g.gf2_random(A, 3)
        g.gf2_random(B, 4)
        g.gf2_release_scratch()
        g.gf2_reserve_scratch(need)
        g.gf2_mul(C, A, B, o)
        assert g.gf2_freivalds(C, A, B, 11) == 0
        g.gf2_release_scratch()
        g.gf2_mul(C, A, B, o)
        assert g.gf2_freivalds(C, A, B, 12) == 0
    finally:
        for M in (A, B, C):
            g.gf2_free(M)


def test_profile_counts_the_launches_of_a_product():
    m = l = n = 1024
    A, B, C = g.gf2_alloc(m, l), g.gf2_alloc(l, n), g.gf2_alloc(m, n)
    try:
        g.gf2_random(A, 5)
        g.gf2_random(B, 6)
        names = list(g.PROFILE_FAMILIES)
        assert names[0] == "m4rm" and g.gf2_profile_name(len(names)) is None
        g.gf2_profile_enable(True)
        g.gf2_mul(C, A, B, g.opts(base=g.GF2_BASE_M4RM, depth=1))
        ms, launches = g.gf2_profile_read(0)
        split_ms, split_launches = g.gf2_profile_read(names.index("sw_split"))
        g.gf2_profile_enable(False)
        assert launches >= 1 and ms > 0
        assert split_launches >= 1 and split_ms > 0
    finally:
        for M in (A, B, C):
            g.gf2_free(M)
