"""The large rectangular chain: A (131072 x 65536) . B (65536 x 131072), then
. C (131072 x 8192), in that order, Bernoulli(1/2) bits.

Stage 1 and stage 2 are each checked by Freivalds' test (64 vectors) on the
GPU, and on sampled 64 x 64 blocks computed by the oracle from the seeded
inputs alone: a block of AB is A[rows] B[:, cols]; a block of (AB)C is
A[rows] (B C[:, cols]), formed with the oracle's packed matrix-vector
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


def block_of(t, r0, c0):
    got = t[r0:r0 + 64, c0 // 64:c0 // 64 + 1].contiguous()
    return valid_words(to_host(got), 64)


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
    # stage 1 blocks: A[r0:r0+64] . B[:, c0:c0+64]
    for _ in range(2):
        r0 = int(rng.integers(0, M - 64))
        c0 = 64 * int(rng.integers(0, N1 // 64))
        Ar = synth.random_packed(64, K1, SA, row0=r0)
        Bc = synth.random_packed_cols(K1, N1, SB, c0, c0 + 64)
        ref = oracle.mul_packed(Ar, Bc, 64, K1, 64)
        assert np.array_equal(block_of(AB, r0, c0), valid_words(ref, 64)), ("AB", r0, c0)
    # stage 2 blocks: A[r0:r0+64] . (B . C[:, c0:c0+64])
    Bfull = synth.random_packed(K1, N1, SB)             # 1 GiB on the host
    for _ in range(2):
        r0 = int(rng.integers(0, M - 64))
        c0 = 64 * int(rng.integers(0, N2 // 64))
        Cc = synth.random_packed_cols(N1, N2, SC, c0, c0 + 64).reshape(-1)
        Y = oracle.matvec64(Bfull, K1, N1, Cc)           # B . C[:, cols]: one word per row of B
        Ar = synth.random_packed(64, K1, SA, row0=r0)
        Z = oracle.matvec64(Ar, 64, K1, Y)               # A[rows] . (B . C[:, cols])
        assert np.array_equal(block_of(ABC, r0, c0)[:, 0], Z), ("ABC", r0, c0)
