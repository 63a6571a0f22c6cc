"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: values printed in
the paper, brute force over every small operand, a library routine that
reduces to the same product (numpy integer matmul mod 2), or an algebraic
identity that the product over a field must satisfy.
"""
import itertools
import os
import re

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore")


def np_mod2(A, B):
    """numpy's integer matrix product, reduced mod 2 (library special case)."""
    return (A.astype(np.int64) @ B.astype(np.int64) % 2).astype(np.uint8)


def rand_bits(rng, r, c, p=0.5):
    return (rng.random((r, c)) < p).astype(np.uint8)


# ---------------------------------------------------------------- Section 3.1

def read_gray_fixture(golden_dir):
    out, cur = {}, None
    for line in open(os.path.join(golden_dir, "gray_codes.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        m = re.fullmatch(r"\[(\d+)\]", line)
        if m:
            cur = int(m.group(1))
            out[cur] = []
        else:
            out[cur].append(tuple(int(ch) for ch in line))
    return out


def test_gray_code_matches_figure(golden_dir):
    fig = read_gray_fixture(golden_dir)
    assert sorted(fig) == [2, 3, 4]
    for k, codes in fig.items():
        assert oracle.gray_code(k) == codes


def test_gray_code_is_reflected_binary():
    # textbook closed form: the i-th reflected Gray code is i XOR (i >> 1)
    for k in range(1, 11):
        codes = oracle.gray_code(k)
        assert len(codes) == 1 << k
        for i, bits in enumerate(codes):
            v = int("".join(map(str, bits)), 2)
            assert v == i ^ (i >> 1)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_make_table_cost_and_entries(k):
    # Section 3.1: all 2^k - 1 non-zero combinations in exactly 2^k - 1 additions.
    rng = np.random.default_rng(10 + k)
    B = rand_bits(rng, k + 3, 37)
    T, adds = oracle.make_table(B, 2, 0, k)
    assert adds == (1 << k) - 1
    for x in range(1 << k):
        # ReadBits weights the first row as the most significant bit
        expect = np.zeros(37, dtype=np.uint8)
        for j in range(k):
            if (x >> (k - 1 - j)) & 1:
                expect ^= B[2 + j]
        assert np.array_equal(T[x], expect), x


def test_read_bits_msb_first():
    A = np.array([[1, 0, 1, 1, 0]], dtype=np.uint8)
    assert oracle.read_bits(A, 0, 0, 3) == 0b101
    assert oracle.read_bits(A, 0, 1, 4) == 0b0110


# ------------------------------------------------------ Section 3, worked example

def _eval_formula(expr, env):
    total = 0
    for term in expr.split("+"):
        v = 1
        for f in term.strip().split("*"):
            v &= env[f.strip()]
        total ^= v
    return total


def read_worked_example(golden_dir):
    rows = []
    for line in open(os.path.join(golden_dir, "worked_example_k1.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        lhs, rhs = line.split("=")
        name, i, j = lhs.split()
        rows.append((name, int(i), int(j), rhs.strip()))
    return rows


def test_worked_example_all_2x2_pairs(golden_dir):
    """All 2^8 operand pairs against the formulas printed for k = 1."""
    fx = read_worked_example(golden_dir)
    assert len(fx) == 12
    for bits in itertools.product((0, 1), repeat=8):
        a = bits[:4]
        b = bits[4:]
        env = {f"a{i}": a[i] for i in range(4)}
        env.update({f"b{i}": b[i] for i in range(4)})
        A = np.array(a, dtype=np.uint8).reshape(2, 2)
        B = np.array(b, dtype=np.uint8).reshape(2, 2)
        got = {
            "C": oracle.mul(A, B),
            "A0B0": oracle.mul(A[:, :1], B[:1, :]),
            "A1B1": oracle.mul(A[:, 1:], B[1:, :]),
        }
        for name, i, j, expr in fx:
            assert got[name][i, j] == _eval_formula(expr, env)
        assert np.array_equal(oracle.m4rm(A, B, 1), got["C"])
        assert np.array_equal(oracle.strassen_winograd(A, B, 1), got["C"])


# ------------------------------------------------------------ brute force

def test_brute_force_all_3x3_pairs():
    """Every pair of 3x3 matrices (2^18 pairs) against numpy's product mod 2."""
    allm = np.array(list(itertools.product((0, 1), repeat=9)), dtype=np.uint8).reshape(-1, 3, 3)
    # numpy side: all pairs in one einsum
    ref = (np.einsum("aij,bjk->abik", allm.astype(np.int32), allm.astype(np.int32)) & 1).astype(np.uint8)
    # oracle side: stack all left operands into one tall matrix per right operand
    Atall = allm.reshape(-1, 3)
    for bi in range(allm.shape[0]):
        C = oracle.mul(Atall, allm[bi]).reshape(-1, 3, 3)
        assert np.array_equal(C, ref[:, bi]), bi


def test_packed_matches_numpy_random_shapes():
    rng = np.random.default_rng(1)
    shapes = [(0, 5, 3), (4, 0, 6), (3, 7, 0), (1, 1, 1), (5, 64, 3), (65, 63, 129),
              (7, 128, 200), (64, 65, 64)]
    shapes += [tuple(int(x) for x in rng.integers(1, 140, 3)) for _ in range(20)]
    for (m, l, n) in shapes:
        A = rand_bits(rng, m, l)
        B = rand_bits(rng, l, n)
        ref = np_mod2(A, B)
        C = oracle.mul_packed(synth.pack_bits(A), synth.pack_bits(B), m, l, n)
        assert C.shape == (m, synth.padded_stride(n))
        assert np.array_equal(synth.unpack_bits(C, n), ref), (m, l, n)
        assert np.array_equal(oracle.mul(A, B), ref)


def test_pack_unpack_roundtrip_and_layout():
    rng = np.random.default_rng(2)
    bits = rand_bits(rng, 5, 130)
    P = oracle.pack(bits, 4)
    # Section 2.1 layout: column c is bit c % 64 of word c // 64
    for r in range(5):
        for c in range(130):
            assert ((int(P[r, c // 64]) >> (c % 64)) & 1) == bits[r, c]
    assert np.all(P[:, 3] == 0)
    assert np.array_equal(oracle.unpack(P, 5, 130), bits)
    assert np.array_equal(P, synth.pack_bits(bits, 4))


def test_input_tail_bits_are_ignored_output_tail_zero():
    rng = np.random.default_rng(3)
    m, l, n = 9, 70, 100
    A = synth.pack_bits(rand_bits(rng, m, l))
    B = synth.pack_bits(rand_bits(rng, l, n))
    ref = oracle.mul_packed(A, B, m, l, n)
    A2, B2 = A.copy(), B.copy()
    A2[:, 1] |= np.uint64(0xFFFFFFFFFFFFFFFF) ^ synth.tail_mask(l)
    A2[:, 2:] = np.uint64(0x5A5A5A5A5A5A5A5A)
    B2[:, 1] |= np.uint64(0xFFFFFFFFFFFFFFFF) ^ synth.tail_mask(n)
    C = oracle.mul_packed(A2, B2, m, l, n)
    assert np.array_equal(C, ref)
    assert np.all((C[:, 1] & ~synth.tail_mask(n)) == 0)


# ------------------------------------------------------------ identities

def test_identities():
    rng = np.random.default_rng(4)
    m, l, n, q = 37, 70, 45, 29
    A = rand_bits(rng, m, l)
    A2 = rand_bits(rng, m, l)
    B = rand_bits(rng, l, n)
    B2 = rand_bits(rng, l, n)
    Cm = rand_bits(rng, n, q)
    I_l = np.eye(l, dtype=np.uint8)
    I_m = np.eye(m, dtype=np.uint8)
    assert np.array_equal(oracle.mul(A, I_l), A)
    assert np.array_equal(oracle.mul(I_m, A), A)
    AB = oracle.mul(A, B)
    assert np.array_equal(oracle.mul(AB, Cm), oracle.mul(A, oracle.mul(B, Cm)))
    assert np.array_equal(AB.T, oracle.mul(B.T.copy(), A.T.copy()))
    assert np.array_equal(oracle.mul(A, B ^ B2), AB ^ oracle.mul(A, B2))
    assert np.array_equal(oracle.mul(A ^ A2, B), AB ^ oracle.mul(A2, B))
    # all-ones operands: every entry is the parity of the inner dimension
    ones = oracle.mul(np.ones((5, l), np.uint8), np.ones((l, 7), np.uint8))
    assert np.all(ones == (l & 1))


# ------------------------------------------------------------ Algorithms 1, 3, 4

@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 8])
def test_m4rm_equals_definition(k):
    rng = np.random.default_rng(20 + k)
    m, l, n = 23, 41, 33      # l mod k != 0 for most k: the tail stripe is exercised
    A = rand_bits(rng, m, l)
    B = rand_bits(rng, l, n)
    assert np.array_equal(oracle.m4rm(A, B, k), np_mod2(A, B))


@pytest.mark.parametrize("k,t", [(2, 2), (3, 2), (4, 8), (5, 3)])
def test_m4rm_t_tables_equals_definition(k, t):
    rng = np.random.default_rng(30 + k * t)
    m, l, n = 19, 53, 27
    A = rand_bits(rng, m, l)
    B = rand_bits(rng, l, n)
    assert np.array_equal(oracle.m4rm_tables(A, B, k, t), np_mod2(A, B))


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_strassen_winograd_equals_definition(depth):
    rng = np.random.default_rng(40 + depth)
    for (m, l, n) in [(16, 16, 16), (24, 40, 8), (17, 33, 9), (31, 30, 29)]:
        A = rand_bits(rng, m, l)
        B = rand_bits(rng, l, n)
        assert np.array_equal(oracle.strassen_winograd(A, B, depth), np_mod2(A, B)), (m, l, n)


def test_strassen_operands_one_level():
    """The 7 products of Algorithm 4 recombine to the cubic product."""
    rng = np.random.default_rng(5)
    A = rand_bits(rng, 10, 14)
    B = rand_bits(rng, 14, 6)
    lhs, rhs = oracle.sw_operands(A, B)
    P = [np_mod2(x, y) for x, y in zip(lhs, rhs)]
    assert np.array_equal(oracle.sw_combine(P), np_mod2(A, B))
    # S3 and T3 are the sums of all four quadrants
    q = oracle.quadrants(A)
    assert np.array_equal(lhs[2], q[0] ^ q[1] ^ q[2] ^ q[3])
    qb = oracle.quadrants(B)
    assert np.array_equal(rhs[3], qb[0] ^ qb[1] ^ qb[2] ^ qb[3])


# ------------------------------------------------------------ Section 2.3 matvec

def test_matvec64_matches_definition():
    rng = np.random.default_rng(6)
    for (r, c) in [(1, 1), (13, 64), (50, 130), (7, 200)]:
        M = rand_bits(rng, r, c)
        Xbits = rand_bits(rng, c, 64)
        X = synth.pack_bits(Xbits, 1).reshape(-1)
        Y = oracle.matvec64(synth.pack_bits(M), r, c, X)
        ref = np_mod2(M, Xbits)
        assert np.array_equal(synth.unpack_bits(Y.reshape(-1, 1), 64), ref)


def test_mul_packed_column_block():
    rng = np.random.default_rng(7)
    m, l, n = 12, 90, 300
    A = synth.pack_bits(rand_bits(rng, m, l))
    Bb = rand_bits(rng, l, n)
    B = synth.pack_bits(Bb)
    full = synth.unpack_bits(oracle.mul_packed(A, B, m, l, n), n)
    blk = oracle.mul_packed(A, B, m, l, 100, b_col0=128)
    assert np.array_equal(synth.unpack_bits(blk, 100), full[:, 128:228])


# ------------------------------------------------------------ input generator

def test_splitmix64_reference_vector(golden_dir):
    vals = [int(x) for x in open(os.path.join(golden_dir, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    got = synth.splitmix64(1234567, np.arange(1, 6, dtype=np.uint64))
    assert [int(v) for v in got] == vals


def test_generator_layout_independent_and_row_ranges():
    full = synth.random_packed(40, 200, seed=9)
    wide = synth.random_packed(40, 200, seed=9, stride=8)
    assert np.array_equal(full[:, :4], wide[:, :4]) and np.all(wide[:, 4:] == 0)
    part = synth.random_packed(10, 200, seed=9, row0=25)
    assert np.array_equal(part, full[25:35])
    cols = synth.random_packed_cols(40, 200, 9, 64, 190)
    bits = synth.unpack_bits(full, 200)
    assert np.array_equal(synth.unpack_bits(cols, 126), bits[:, 64:190])
    assert np.all((full[:, 3] & ~synth.tail_mask(200)) == 0)


def test_generator_density():
    for p in (0.5, 0.9, 0.1):
        bits = synth.unpack_bits(synth.random_packed(256, 256, seed=5, p=p), 256)
        assert abs(bits.mean() - p) < 0.01


def test_batch_dims_range():
    dims = synth.batch_dims(4096)
    flat = np.array(dims).reshape(-1)
    assert flat.min() >= 64 and flat.max() <= 2048
    # log-uniform: the mean of log2(size) is near the midpoint 8.5
    assert abs(np.log2(flat).mean() - 8.5) < 0.1
