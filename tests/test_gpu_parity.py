"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every comparison is bit-exact: the product over GF(2) is unique, so the
bar is equality of every packed word (tail bits of the last word must be
zero on output).  Inputs come from the seeded generator in ``synth``.
"""
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
    torch.cuda.synchronize()


def gpu_mul(A, B, m, l, n, **kw):
    Ad, Bd = to_dev(A), to_dev(B)
    C = g.empty(m, n)
    g.gf2_mul(g.mat(C, n), g.mat(Ad, l), g.mat(Bd, n), g.opts(**kw))
    torch.cuda.synchronize()
    return to_host(C)


def inputs(m, l, n, p=0.5, seeds=(synth.SEED_A, synth.SEED_B)):
    return synth.random_packed(m, l, seeds[0], p), synth.random_packed(l, n, seeds[1], p)


# ---------------------------------------------------------------- generator

@pytest.mark.parametrize("rows,cols,p", [(5, 1, 0.5), (37, 200, 0.5), (64, 128, 0.9), (33, 65, 0.1)])
def test_device_generator_matches_host(rows, cols, p):
    M = g.empty(rows, cols)
    M.fill_(-1)
    g.gf2_random(g.mat(M, cols), 77, p)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(M), synth.random_packed(rows, cols, 77, p))


# ---------------------------------------------------------------- M4RM base case

CONFIG1 = (1024, 1024, 1024)


def test_config1_plain_m4rm_k8():
    """m = l = n = 1024, M4RM with k = 8, no Strassen recursion."""
    m, l, n = CONFIG1
    A, B = inputs(m, l, n)
    ref = oracle.mul_packed(A, B, m, l, n)
    got = gpu_mul(A, B, m, l, n, base=g.GF2_BASE_M4RM, depth=0, k=8)
    assert_same_bits(got, ref, n, "config 1")


@pytest.mark.parametrize("m,l,n", [
    (1, 1, 1), (3, 70, 5), (64, 64, 64), (100, 300, 1000), (257, 129, 1025),
    (1023, 1025, 2047), (2100, 700, 1100), (4096, 96, 130)])
def test_m4rm_shapes(m, l, n):
    A, B = inputs(m, l, n)
    ref = oracle.mul_packed(A, B, m, l, n)
    got = gpu_mul(A, B, m, l, n, base=g.GF2_BASE_M4RM, depth=0)
    assert_same_bits(got, ref, n, str((m, l, n)))


@pytest.mark.parametrize("k,t", [(8, 4), (8, 2), (7, 8), (6, 8), (9, 2), (10, 1), (5, 8), (4, 8)])
def test_m4rm_every_table_shape(k, t):
    m, l, n = 2304, 1000, 1500          # ragged in every dimension, several row tiles
    A, B = inputs(m, l, n)
    ref = oracle.mul_packed(A, B, m, l, n)
    got = gpu_mul(A, B, m, l, n, base=g.GF2_BASE_M4RM, depth=0, k=k, t=t)
    assert_same_bits(got, ref, n, "k=%d t=%d" % (k, t))


def test_m4rm_density_09_and_accumulate():
    m, l, n = 700, 900, 800
    A, B = inputs(m, l, n, p=0.9)
    ref = oracle.mul_packed(A, B, m, l, n)
    C0 = synth.random_packed(m, n, 5)
    Cd, Ad, Bd = to_dev(C0), to_dev(A), to_dev(B)     # keep the tensors alive across the call
    g.gf2_mul(g.mat(Cd, n), g.mat(Ad, l), g.mat(Bd, n),
              g.opts(base=g.GF2_BASE_M4RM, depth=0, accumulate=1))
    torch.cuda.synchronize()
    assert_same_bits(to_host(Cd), ref ^ C0, n, "accumulate")


@pytest.mark.parametrize("accumulate", [0, 1])
def test_m4rm_tall_tiles_with_tensor_memory_half(accumulate):
    """2048-row tiles (one half in registers, one in tensor memory): rows
    ragged at the tile end and checked across the half boundary (row 1024),
    columns ragged in the last tile, K not a multiple of the 32-bit pass."""
    m, l, n = 2 * 2048 + 1500, 333, 159 * 1024 + 200
    plan = g.gf2_describe_plan(m, l, n, g.opts(base=g.GF2_BASE_M4RM, depth=0))
    assert "tile_rows=2048" in plan, plan
    A, B = inputs(m, l, n, seeds=(41, 42))
    C0 = synth.random_packed(m, n, 43) if accumulate else None
    Ad, Bd = to_dev(A), to_dev(B)
    Cd = to_dev(C0) if accumulate else g.empty(m, n)
    if not accumulate:
        Cd.fill_(-1)
    g.gf2_mul(g.mat(Cd, n), g.mat(Ad, l), g.mat(Bd, n),
              g.opts(base=g.GF2_BASE_M4RM, depth=0, accumulate=accumulate))
    g.gf2_device_status()
    got = to_host(Cd)
    for r0, r1 in ((0, 40), (1000, 1050), (2030, 2080), (3060, 3090), (5100, 5150), (5560, m)):
        ref = oracle.mul_packed(np.ascontiguousarray(A[r0:r1]), B, r1 - r0, l, n)
        if accumulate:
            ref = ref ^ C0[r0:r1]
        assert_same_bits(got[r0:r1], ref, n, "rows %d..%d" % (r0, r1))


@pytest.mark.parametrize("m,l,n", [(1, 1, 1), (100, 70, 5), (5000, 3000, 63), (777, 4097, 64), (64, 129, 33)])
@pytest.mark.parametrize("acc", [0, 1])
def test_cubic_product_for_narrow_right_factors(m, l, n, acc):
    A, B = inputs(m, l, n, seeds=(81, 82))
    ref = oracle.mul_packed(A, B, m, l, n)
    C0 = synth.random_packed(m, n, 83) if acc else None
    if acc:
        ref = ref ^ C0
    o = g.opts(base=g.GF2_BASE_M4RM, depth=0, accumulate=acc)
    assert "cubic=1" in g.gf2_describe_plan(m, l, n, o)
    Ad, Bd = to_dev(A), to_dev(B)
    Cd = to_dev(C0) if acc else g.empty(m, n)
    if not acc:
        Cd.fill_(-1)
    g.gf2_mul(g.mat(Cd, n), g.mat(Ad, l), g.mat(Bd, n), o)
    torch.cuda.synchronize()
    assert_same_bits(to_host(Cd), ref, n, "cubic %s acc %d" % ((m, l, n), acc))


def test_tail_garbage_is_ignored():
    m, l, n = 300, 200, 333
    A, B = inputs(m, l, n)
    ref = oracle.mul_packed(A, B, m, l, n)
    A2, B2 = A.copy(), B.copy()
    A2[:, 3] |= ~synth.tail_mask(l)
    B2[:, 5] |= ~synth.tail_mask(n)
    for depth in (0, 1):
        got = gpu_mul(A2, B2, m, l, n, depth=depth)
        assert_same_bits(got, ref, n, "depth %d" % depth)


def test_all_ones_closed_form():
    # every entry of ones(m,l) ones(l,n) is l mod 2
    for l in (1023, 1024):
        m, n = 128, 256
        A = synth.pack_bits(np.ones((m, l), np.uint8))
        B = synth.pack_bits(np.ones((l, n), np.uint8))
        got = gpu_mul(A, B, m, l, n, depth=0)
        expect = synth.pack_bits(np.full((m, n), l & 1, np.uint8))
        assert_same_bits(got, expect, n, "ones l=%d" % l)


def test_identity():
    m = n = 777
    A = synth.random_packed(m, n, 11)
    I = synth.pack_bits(np.eye(n, dtype=np.uint8))
    assert_same_bits(gpu_mul(A, I, m, n, n, depth=0), A, n, "A I")
    assert_same_bits(gpu_mul(I, A, n, n, n, depth=0), A, n, "I A")


def test_zero_sizes():
    # l = 0: C is cleared; m = 0 or n = 0: nothing to do
    C = g.empty(5, 70)
    C.fill_(-1)
    A = g.empty(5, 0)
    B = g.empty(0, 70)
    g.gf2_mul(g.mat(C, 70), g.mat(A, 0), g.mat(B, 70))
    torch.cuda.synchronize()
    assert np.all(to_host(C)[:, :2] == 0)
    g.gf2_mul(g.mat(g.empty(0, 70), 70), g.mat(g.empty(0, 9), 9), g.mat(g.empty(9, 70), 70))


# ---------------------------------------------------------------- Strassen-Winograd

@pytest.mark.parametrize("m,l,n,depth", [
    (512, 512, 512, 1), (1024, 1024, 1024, 2), (1000, 1100, 900, 1), (2047, 2049, 1025, 2),
    (2048, 2048, 2048, 3), (300, 5000, 200, 2)])
def test_strassen_winograd_parity(m, l, n, depth):
    A, B = inputs(m, l, n)
    ref = oracle.mul_packed(A, B, m, l, n)
    got = gpu_mul(A, B, m, l, n, base=g.GF2_BASE_M4RM, depth=depth)
    assert_same_bits(got, ref, n, "depth %d" % depth)


@pytest.mark.parametrize("side", [0, 1, 2])
def test_sw_split_matches_algorithm4(side):
    rows, cols = 64, 512
    X = synth.random_packed(rows, cols, 21)
    Xd = to_dev(X)
    cld = cols // 128
    slab = (rows // 2) * cld
    out = torch.zeros(7 * slab, dtype=torch.int64, device="cuda")
    g.gf2_sw_split(out.data_ptr(), slab, g.mat(Xd, cols), side)
    torch.cuda.synchronize()
    outs = to_host(out).reshape(7, rows // 2, cld)
    bits = synth.unpack_bits(X, cols)
    if side == 0:
        ops, _ = oracle.sw_operands(bits, np.zeros((cols, 2), np.uint8))
    elif side == 1:
        _, ops = oracle.sw_operands(np.zeros((2, rows), np.uint8), bits)
    else:
        # X holds B^T: operands are the transposes of the right factors
        _, ops = oracle.sw_operands(np.zeros((2, cols), np.uint8), bits.T.copy())
        ops = [o.T for o in ops]
    for i, o in enumerate(ops):
        assert np.array_equal(synth.unpack_bits(outs[i], cols // 2), o), "operand %d" % i


def test_sw_combine_matches_algorithm4():
    rows, cols = 64, 512
    P = [synth.random_packed(rows // 2, cols // 2, 30 + i) for i in range(7)]
    slab = (rows // 2) * (cols // 128)
    Pd = to_dev(np.concatenate([p.reshape(-1) for p in P]))
    C = g.empty(rows, cols)
    g.gf2_sw_combine(g.mat(C, cols), Pd.data_ptr(), slab)
    torch.cuda.synchronize()
    ref = oracle.sw_combine([synth.unpack_bits(p, cols // 2) for p in P])
    assert np.array_equal(synth.unpack_bits(to_host(C), cols), ref)


# ---------------------------------------------------------------- MakeTable

@pytest.mark.parametrize("k", [1, 3, 4, 8, 10])
def test_make_table_matches_gray_code_table(k):
    rows, cols = 40, 1500
    B = synth.random_packed(rows, cols, 8)
    T = g.empty(1 << k, cols)
    r0 = 35                              # rows beyond B count as zero when k is large
    Bd = to_dev(B)
    g.gf2_make_table(g.mat(T, cols), g.mat(Bd, cols), r0, k)
    torch.cuda.synchronize()
    Tg = synth.unpack_bits(to_host(T), cols)
    bits = synth.unpack_bits(B, cols)
    padded = np.zeros((max(rows, r0 + k), cols), np.uint8)
    padded[:rows] = bits
    Tor, adds = oracle.make_table(padded, r0, 0, k)
    assert adds == (1 << k) - 1
    # the library indexes LSB-first (bit j selects row r0+j); the paper's
    # ReadBits is MSB-first: index x here is the bit reversal of x there
    for x in range(1 << k):
        xr = int(format(x, "0%db" % k)[::-1], 2)
        assert np.array_equal(Tg[x], Tor[xr]), x


# ---------------------------------------------------------------- helpers of the path

@pytest.mark.parametrize("r,c", [(300, 700), (1, 1), (64, 64), (256, 256), (257, 1025), (1000, 64),
                                 (64, 3000), (511, 513), (2048, 300)])
def test_transpose(r, c):
    """The packed transpose (256 x 256-entry warp tiles): every entry, ragged
    tiles on both sides, and the bits past T's last column written as zero."""
    X = synth.random_packed(r, c, 4)
    T = g.empty(c, r)
    T.fill_(-1)
    Xd = to_dev(X)
    g.gf2_transpose(g.mat(T, r), g.mat(Xd, c))
    torch.cuda.synchronize()
    got = to_host(T)
    assert np.array_equal(synth.unpack_bits(got, r), synth.unpack_bits(X, c).T)
    W = synth.words_for(r)
    if r % 64:
        assert np.all((got[:, W - 1] & ~synth.tail_mask(r)) == 0)


def test_freivalds_accepts_and_rejects():
    m, l, n = 1500, 1300, 1700
    A, B = inputs(m, l, n)
    Ad, Bd = to_dev(A), to_dev(B)
    C = g.empty(m, n)
    g.gf2_mul(g.mat(C, n), g.mat(Ad, l), g.mat(Bd, n))
    assert g.gf2_freivalds(g.mat(C, n), g.mat(Ad, l), g.mat(Bd, n), 1000) == 0
    C[17, 3] ^= 1 << 5                   # one wrong entry
    assert g.gf2_freivalds(g.mat(C, n), g.mat(Ad, l), g.mat(Bd, n), 1001) >= 1


def test_host_operands_through_the_abi():
    m, l, n = 500, 600, 700
    A, B = inputs(m, l, n)
    C = np.zeros((m, synth.padded_stride(n)), np.uint64)
    g.gf2_mul(g.mat(C, n), g.mat(A, l), g.mat(B, n), g.opts(depth=1))
    assert_same_bits(C, oracle.mul_packed(A, B, m, l, n), n, "host operands")


@pytest.mark.parametrize("base,depth,l", [(g.GF2_BASE_M4RM, 2, 1500), (g.GF2_BASE_M4RM, 3, 1500),
                                          (g.GF2_BASE_TC_FP8, 2, 1500), (g.GF2_BASE_M4RM, 0, 1500),
                                          (g.GF2_BASE_TC_FP4, 0, 1500), (g.GF2_BASE_TC_FP4, 1, 1500),
                                          (g.GF2_BASE_TC_FP4, 2, 5000), (g.GF2_BASE_TC_S8, 1, 1500)])
def test_host_operands_with_b_copied_beside_a_additions(base, depth, l):
    """Both factors on the host: B's copy runs on a side stream while A's
    Strassen-Winograd additions (and, for the expanded tensor-core base
    cases, A's expansion) run; for the tensor-core base cases B arrives in
    row blocks, each transposed as the next one is copied (ragged last
    block); every call, back to back, with new contents each time (a stale B
    would show)."""
    m, n = 1300, 1100
    for trial in range(3):
        A, B = inputs(m, l, n, seeds=(60 + trial, 70 + trial))
        C = np.full((m, synth.padded_stride(n)), 0xFFFF, np.uint64)
        g.gf2_mul(g.mat(C, n), g.mat(A, l), g.mat(B, n), g.opts(base=base, depth=depth))
        assert_same_bits(C, oracle.mul_packed(A, B, m, l, n), n, "host operands %d %d %d" % (base, depth, trial))


@pytest.mark.parametrize("base,depth,m,l", [(g.GF2_BASE_TC_FP4, 2, 40000, 5000), (g.GF2_BASE_TC_FP4, 1, 20000, 1500),
                                            (g.GF2_BASE_TC_FP8, 2, 20000, 1500), (g.GF2_BASE_M4RM, 1, 40000, 1500),
                                            (g.GF2_BASE_M4RM, 0, 17000, 1500), (g.GF2_BASE_TC_S8, 1, 16500, 1500),
                                            (g.GF2_BASE_TC_FP4, 0, 16400, 700)])
def test_host_operands_in_row_blocks(base, depth, m, l):
    """A, B and C on the host with at least 2 x 8192 rows: A and C go in 2
    row blocks (the last one ragged), block i's product starts once A_i has
    arrived and C_i is copied back while the next block is computed, B's
    transposition, additions and expansion done once for all blocks; two
    calls back to back with new contents (a stale B or block would show)."""
    n = 1100
    for trial in range(2):
        A, B = inputs(m, l, n, seeds=(80 + trial, 90 + trial))
        C = np.full((m, synth.padded_stride(n)), 0xFFFF, np.uint64)
        g.gf2_mul(g.mat(C, n), g.mat(A, l), g.mat(B, n), g.opts(base=base, depth=depth))
        assert_same_bits(C, oracle.mul_packed(A, B, m, l, n), n,
                         "host row blocks %d %d %d %d" % (base, depth, m, trial))


@pytest.mark.parametrize("where", ["hdd", "dhd", "ddh", "hhd", "hdh", "dhh", "hhh"])
@pytest.mark.parametrize("m", [1300, 16500])
@pytest.mark.parametrize("acc", [0, 1])
def test_host_and_device_operands_mixed(where, m, acc):
    """Every mix of host (h) and device (d) operands, in the order A, B, C,
    with C overwritten or accumulated into (a host C is then copied in
    first): all three on the host with m >= 16384 and no accumulation takes
    the row-blocked path, the rest the single-product one."""
    l, n = 1500, 700
    A, B = inputs(m, l, n, seeds=(110 + m % 7, 120 + acc))
    C0 = synth.random_packed(m, n, 130 + acc)
    ref = oracle.mul_packed(A, B, m, l, n) ^ (C0 if acc else 0)
    hA = where[0] == "h"
    hB = where[1] == "h"
    hC = where[2] == "h"
    Ax = A if hA else to_dev(A)
    Bx = B if hB else to_dev(B)
    Cx = C0.copy() if hC else to_dev(C0)
    g.gf2_mul(g.mat(Cx, n), g.mat(Ax, l), g.mat(Bx, n),
              g.opts(base=g.GF2_BASE_TC_FP4, depth=1, accumulate=acc))
    torch.cuda.synchronize()
    got = Cx if hC else to_host(Cx)
    assert_same_bits(got, ref, n, "mixed %s m=%d acc=%d" % (where, m, acc))


def test_launch_count_grows():
    before = g.gf2_launch_count()
    gpu_mul(*inputs(64, 64, 64), 64, 64, 64, depth=0)
    assert g.gf2_launch_count() > before
