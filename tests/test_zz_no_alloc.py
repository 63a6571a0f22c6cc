"""gf2_mul_noalloc: the product for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: code inside a framework
that has already reserved nearly all of the GPU's memory for its own
allocator, and latency-critical code that must not take the device-wide
synchronisation of cudaMalloc / cudaFree.  gf2_mul_noalloc serves them by
taking its Strassen-Winograd temporaries (and, for the tensor-core base case,
the transposed right factor) from a fixed device buffer of the library.  This
file checks, through the C ABI, that it gives exactly the words of the CPU
oracle and of gf2_mul (the product over GF(2) is unique: the tolerance is
bit-exact equality) on two calls in a row, with the packed and with the
tensor-core base case, and that what it cannot do is refused without
launching anything.

The file name makes pytest collect it after every other test file.
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


@pytest.mark.parametrize("m,l,n,depth,base", [
    (2048, 2048, 2048, 1, "M4RM"),
    (1500, 2100, 1300, 2, "M4RM"),
    (1500, 2100, 1300, 1, "TC_FP8"),       # B^T of the tensor-core base case in the fixed buffer
])
def test_noalloc_matches_oracle_and_gf2_mul_on_two_calls(m, l, n, depth, base):
    o = g.opts(base=getattr(g, "GF2_BASE_" + base), depth=depth)
    assert 0 < g.gf2_scratch_bytes(m, l, n, o) <= g.GF2_NOALLOC_SCRATCH_BYTES
    for call, seeds in enumerate([(101, 102), (103, 104)]):
        A = synth.random_packed(m, l, seeds[0])
        B = synth.random_packed(l, n, seeds[1])
        ref = oracle.mul_packed(A, B, m, l, n)
        Ad, Bd = to_dev(A), to_dev(B)
        C_lib = g.empty(m, n)
        C_new = g.empty(m, n)
        C_new.fill_(-1)                       # every word must be written by the call
        g.gf2_mul(g.mat(C_lib, n), g.mat(Ad, l), g.mat(Bd, n), o)
        g.gf2_mul_noalloc(g.mat(C_new, n), g.mat(Ad, l), g.mat(Bd, n), o)
        torch.cuda.synchronize()
        got = to_host(C_new)
        assert_same_bits(got, ref, n, "call %d against the oracle" % call)
        assert np.array_equal(valid_words(got, n), valid_words(to_host(C_lib), n)), \
            "call %d differs from gf2_mul" % call


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


def test_noalloc_refuses_peeling():
    """Peeling runs several products with their own plans; the fixed buffer
    serves one plan, so peel = 1 is refused before any launch."""
    m, l, n = 1500, 2100, 1300
    A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
    before = g.gf2_launch_count()
    with pytest.raises(g.GF2Error) as e:
        g.gf2_mul_noalloc(g.mat(C, n), g.mat(A, l), g.mat(B, n), g.opts(base=g.GF2_BASE_M4RM, depth=1, peel=1))
    assert e.value.status == g.GF2_EUNSUPPORTED
    assert g.gf2_launch_count() == before
