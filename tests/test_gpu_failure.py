"""Failure detection without a GPU fault: a device wait that nothing can
satisfy runs out after a short bounded time, the host reads GF2_ETIMEOUT
from the status word, and the context keeps working."""
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


def test_expired_wait_is_reported_and_context_survives():
    g.gf2_device_status()                      # clear anything earlier
    g.gf2_selftest_wait(2_000_000)             # ~1 ms at 2 GHz, then it gives up
    with pytest.raises(g.GF2Error) as e:
        g.gf2_device_status()
    assert e.value.status == g.GF2_ETIMEOUT
    g.gf2_device_status()                      # the word was cleared by the read
    # the context is still usable: a tensor-core product is exact
    m, l, n = 300, 700, 500
    A = synth.random_packed(m, l, 61)
    B = synth.random_packed(l, n, 62)
    Ad, Bd, C = to_dev(A), to_dev(B), g.empty(m, n)
    g.gf2_mul(g.mat(C, n), g.mat(Ad, l), g.mat(Bd, n), g.opts(base=g.GF2_BASE_TC_FP8, depth=0))
    g.gf2_device_status()
    assert_same_bits(to_host(C), oracle.mul_packed(A, B, m, l, n), n, "after timeout")


def test_selftest_rejects_bad_limits():
    for bad in (0, -5, 5_000_000_000):
        with pytest.raises(g.GF2Error) as e:
            g.gf2_selftest_wait(bad)
        assert e.value.status == g.GF2_EINVAL
