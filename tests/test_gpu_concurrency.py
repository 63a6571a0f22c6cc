"""Concurrent use of the library: several streams, several host threads, and
host threads sharing one stream while its scratch arena grows.

Every product is checked by Freivalds' test (64 vectors) and, for the small
ones, bit for bit against the CPU oracle.
"""
import threading

import numpy as np
import pytest

import oracle
import synth

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


def make(m, l, n, seed):
    A, B, C = g.empty(m, l), g.empty(l, n), g.empty(m, n)
    MA, MB, MC = g.mat(A, l), g.mat(B, n), g.mat(C, n)
    g.gf2_random(MA, seed)
    g.gf2_random(MB, seed + 1)
    return (A, B, C), (MA, MB, MC)


def test_two_streams_one_thread():
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    t1, (A1, B1, C1) = make(3000, 2800, 3100, 11)
    t2, (A2, B2, C2) = make(2600, 3300, 2900, 21)
    torch.cuda.synchronize()
    for _ in range(3):
        g.gf2_mul(C1, A1, B1, g.opts(base=g.GF2_BASE_M4RM, depth=2), stream=s1)
        g.gf2_mul(C2, A2, B2, g.opts(base=g.GF2_BASE_TC_FP8, depth=1), stream=s2)
    torch.cuda.synchronize()
    g.gf2_device_status()
    assert g.gf2_freivalds(C1, A1, B1, 5) == 0
    assert g.gf2_freivalds(C2, A2, B2, 6) == 0


def test_host_threads_with_their_own_streams():
    errors = []

    def work(tid):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for it in range(4):
                    m, l, n = 700 + 300 * tid + 50 * it, 900 + 100 * it, 800 + 200 * tid
                    tens, (A, B, C) = make(m, l, n, 1000 * tid + 10 * it)
                    base = [g.GF2_BASE_M4RM, g.GF2_BASE_TC_FP8][(tid + it) % 2]
                    g.gf2_mul(C, A, B, g.opts(base=base, depth=it % 3), stream=s)
                    if g.gf2_freivalds(C, A, B, 77 + it, stream=s) != 0:
                        errors.append((tid, it, "freivalds"))
                s.synchronize()
        except Exception as e:      # reported below
            errors.append((tid, repr(e)))

    th = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    g.gf2_device_status()
    assert not errors, errors


def test_host_threads_sharing_one_stream_while_the_arena_grows():
    """Two threads alternate small and growing products on one stream: each
    call's scratch must stay valid until its own work is queued."""
    s = torch.cuda.Stream()
    errors = []
    results = {}

    def work(tid):
        try:
            with torch.cuda.stream(s):
                for it in range(5):
                    m = l = n = 1024 * (it + 1) + 64 * tid
                    tens, (MA, MB, MC) = make(m, l, n, 500 + 10 * tid + it)
                    g.gf2_mul(MC, MA, MB, g.opts(base=g.GF2_BASE_M4RM, depth=min(it, 2)), stream=s)
                    results[(tid, it)] = (tens, MA, MB, MC, m, l, n)
        except Exception as e:
            errors.append((tid, repr(e)))

    th = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    s.synchronize()
    g.gf2_device_status()
    assert not errors, errors
    for (tid, it), (tens, MA, MB, MC, m, l, n) in results.items():
        assert g.gf2_freivalds(MC, MA, MB, 900 + it) == 0, (tid, it)


def test_host_operands_from_threads():
    errors = []

    def work(tid):
        try:
            m, l, n = 500 + 37 * tid, 600 + 11 * tid, 700 + 5 * tid
            A = synth.random_packed(m, l, 40 + tid)
            B = synth.random_packed(l, n, 50 + tid)
            C = np.zeros((m, synth.padded_stride(n)), np.uint64)
            g.gf2_mul(g.mat(C, n), g.mat(A, l), g.mat(B, n), g.opts(depth=1), stream=torch.cuda.Stream())
            if not np.array_equal(C, oracle.mul_packed(A, B, m, l, n)):
                errors.append((tid, "mismatch"))
        except Exception as e:
            errors.append((tid, repr(e)))

    th = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
