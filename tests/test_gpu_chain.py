"""The large rectangular chain: A (131072 x 65536) . B (65536 x 131072), then
. C (131072 x 8192), in that order, Bernoulli(1/2) bits.

Stage 1 and stage 2 are each checked by Freivalds' test (64 vectors) on the
GPU, and on sampled blocks (1024 x 1024 and 64 x 64 of AB, 1024 x 64 and
64 x 64 of (AB)C) computed by the oracle from the seeded inputs alone: a
block of AB is A[rows] B[:, cols]; a block of (AB)C is A[rows] (B C[:, cols]),
formed with the oracle's packed matrix-vector
product of Section 2.3 (64 vectors at once), never from the GPU's AB.
"""
import numpy as np
import pytest

import oracle
import synth
from tests.helpers import to_host, valid_words

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_0811_1714_gb300 as g  # noqa: E402

M, K1, N1, N2 = 131072, 65536, 131072, 8192
SA, SB, SC = 31, 32, 33


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    g.build()
    g.lib()
    yield
    torch.cuda.synchronize()
    g.gf2_release_scratch()
    torch.cuda.empty_cache()


def test_chain_131072_65536_131072_8192():
    A, B, AB = g.empty(M, K1), g.empty(K1, N1), g.empty(M, N1)
    C, ABC = g.empty(N1, N2), g.empty(M, N2)
    MA, MB, MAB, MC, MABC = g.mat(A, K1), g.mat(B, N1), g.mat(AB, N1), g.mat(C, N2), g.mat(ABC, N2)
    g.gf2_random(MA, SA)
    g.gf2_random(MB, SB)
    g.gf2_random(MC, SC)
    g.gf2_mul(MAB, MA, MB)             # automatic plan (Strassen depth, base case)
    g.gf2_mul(MABC, MAB, MC)
    g.gf2_device_status()
    assert g.gf2_freivalds(MAB, MA, MB, 1000) == 0
    assert g.gf2_freivalds(MABC, MAB, MC, 1001) == 0

    rng = np.random.default_rng(5)
    # stage 1 blocks: A[r0:r0+h] . B[:, c0:c0+h], one 1024 x 1024 and one 64 x 64
    for h in (1024, 64):
        r0 = int(rng.integers(0, M - h))
        c0 = 64 * int(rng.integers(0, (N1 - h) // 64))
        Ar = synth.random_packed(h, K1, SA, row0=r0)
        Bc = synth.random_packed_cols(K1, N1, SB, c0, c0 + h)
        ref = oracle.mul_packed(Ar, Bc, h, K1, h)
        got = np.ascontiguousarray(to_host(AB[r0:r0 + h, c0 // 64:c0 // 64 + h // 64].contiguous()))
        assert np.array_equal(valid_words(got, h), valid_words(ref, h)), ("AB", r0, c0, h)
    # stage 2 blocks: A[r0:r0+64] . (B . C[:, c0:c0+64])
    Bfull = synth.random_packed(K1, N1, SB)             # 1 GiB on the host
    for rows in (1024, 64):
        r0 = int(rng.integers(0, M - rows))
        c0 = 64 * int(rng.integers(0, N2 // 64))
        Cc = synth.random_packed_cols(N1, N2, SC, c0, c0 + 64).reshape(-1)
        Y = oracle.matvec64(Bfull, K1, N1, Cc)           # B . C[:, cols]: one word per row of B
        Ar = synth.random_packed(rows, K1, SA, row0=r0)
        Z = oracle.matvec64(Ar, rows, K1, Y)             # A[rows] . (B . C[:, cols])
        got = np.ascontiguousarray(to_host(ABC[r0:r0 + rows, c0 // 64:c0 // 64 + 1].contiguous()))
        assert np.array_equal(valid_words(got, 64)[:, 0], Z), ("ABC", r0, c0, rows)
