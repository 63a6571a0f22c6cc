"""gf2_mul_noalloc: the product for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: code inside a framework
that has already reserved nearly all of the GPU's memory for its own
allocator, and latency-critical code that must not take the device-wide
synchronisation of cudaMalloc / cudaFree.  gf2_mul_noalloc serves them by
taking its Strassen-Winograd temporaries from a fixed device buffer of the
library.  This file checks, through the C ABI, that it gives exactly the
words gf2_mul gives (the product over GF(2) is unique: the tolerance is
bit-exact equality) on two calls in a row, and that a plan too large for the
buffer is refused without launching anything.

The file name makes pytest collect it after every other test file.
"""
import numpy as np
import pytest

import synth
from tests.helpers import to_dev, to_host, valid_words

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


@pytest.mark.parametrize("m,l,n,depth", [(2048, 2048, 2048, 1), (1500, 2100, 1300, 2)])
def test_noalloc_matches_gf2_mul_on_two_calls(m, l, n, depth):
    o = g.opts(base=g.GF2_BASE_M4RM, depth=depth)
    assert 0 < g.gf2_scratch_bytes(m, l, n, o) <= g.GF2_NOALLOC_SCRATCH_BYTES
    for call, seeds in enumerate([(101, 102), (103, 104)]):
        A = synth.random_packed(m, l, seeds[0])
        B = synth.random_packed(l, n, seeds[1])
        Ad, Bd = to_dev(A), to_dev(B)
        C_ref = g.empty(m, n)
        C_new = g.empty(m, n)
        C_new.fill_(-1)                       # every word must be written by the call
        g.gf2_mul(g.mat(C_ref, n), g.mat(Ad, l), g.mat(Bd, n), o)
        g.gf2_mul_noalloc(g.mat(C_new, n), g.mat(Ad, l), g.mat(Bd, n), o)
        torch.cuda.synchronize()
        ref, got = valid_words(to_host(C_ref), n), valid_words(to_host(C_new), n)
        assert np.array_equal(got, ref), "call %d differs from gf2_mul" % call


def test_noalloc_refuses_plans_beyond_its_buffer():
    m = l = n = 8192
    o = g.opts(base=g.GF2_BASE_M4RM, depth=1)
    assert g.gf2_scratch_bytes(m, l, n, o) > g.GF2_NOALLOC_SCRATCH_BYTES
    A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
    C.fill_(7)
    before = g.gf2_launch_count()
    with pytest.raises(g.GF2Error) as e:
        g.gf2_mul_noalloc(g.mat(C, n), g.mat(A, l), g.mat(B, n), o)
    assert e.value.status == g.GF2_ESCRATCH
    assert g.gf2_launch_count() == before
    torch.cuda.synchronize()
    assert bool((C == 7).all())
