"""The arithmetic the tensor-core base cases rest on, checked on the CPU.

The tcgen05 forms encode a 1-bit as FP8 E4M3 0x38 or FP4 E2M1 0x2, both 1.0
(the FP4 one with UE8M0 block scale factors 0x7F = 1.0), so every product is
0 or 1 and a K-chunk of at most 4096 (FP8) or 8192 (FP4) entries sums to an
integer count; the parity is the last mantissa bit of D + 2^23 (Section 2.3:
the GF(2) dot product is the integer dot product mod 2).  The int8 form sums
0/1 products in int32.  These tests decode E4M3, E2M1 and UE8M0 from their
definitions and accumulate in float32 in random orders, and in a model of a
narrower, truncating accumulator.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def e4m3(byte: int) -> float:
    """FP8 E4M3: 1 sign bit, 4 exponent bits with bias 7, 3 mantissa bits;
    exponent 0 is subnormal (m/8 * 2^-6)."""
    s = -1.0 if byte & 0x80 else 1.0
    e = (byte >> 3) & 0xF
    m = byte & 0x7
    if e == 0:
        return s * m * 2.0 ** -9
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


def test_int8_sums_hold_the_parity():
    """The int8 form: 0/1 products summed in int32; the parity is bit 0 for
    any K below 2^31."""
    rng = np.random.default_rng(3)
    for k in (1, 255, 256, 70001, 1 << 20):
        a = rng.integers(0, 2, size=k, dtype=np.int8)
        b = rng.integers(0, 2, size=k, dtype=np.int8)
        s = int(np.sum(a.astype(np.int32) * b.astype(np.int32), dtype=np.int32))
        assert s & 1 == int(np.bitwise_xor.reduce(a & b))


def e2m1(nibble: int) -> float:
    """FP4 E2M1: 1 sign bit, 2 exponent bits with bias 1, 1 mantissa bit;
    exponent 0 is subnormal (m * 0.5)."""
    s = -1.0 if nibble & 0x8 else 1.0
    e = (nibble >> 1) & 0x3
    m = nibble & 0x1
    if e == 0:
        return s * m * 0.5
    return s * (1.0 + m / 2.0) * 2.0 ** (e - 1)


def ue8m0(byte: int) -> float:
    """UE8M0 scale factor: an unsigned 8-bit exponent with bias 127."""
    return 2.0 ** (byte - 127)


def test_expanded_encodings_are_one():
    assert e4m3(0x38) == 1.0 and e4m3(0x00) == 0.0
    assert e2m1(0x2) == 1.0 and e2m1(0x0) == 0.0
    assert ue8m0(0x7F) == 1.0
    # the E2M1 value table from its definition
    assert [e2m1(v) for v in range(8)] == [0.0, 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 6.0]


def test_block_scaled_dot_product_with_unit_scales_is_the_integer_dot_product():
    """kind::mxf4 multiplies each 32-entry block's dot product by the two
    blocks' scale factors; with every scale 1.0 the sum over blocks is the
    plain dot product of the 0/1 vectors."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        a = rng.integers(0, 2, size=256)
        b = rng.integers(0, 2, size=256)
        na = [0x2 if x else 0x0 for x in a]
        nb = [0x2 if x else 0x0 for x in b]
        total = 0.0
        for blk in range(256 // 32):
            part = sum(e2m1(na[i]) * e2m1(nb[i]) for i in range(32 * blk, 32 * blk + 32))
            total += part * ue8m0(0x7F) * ue8m0(0x7F)
        assert total == float(np.dot(a, b))


@pytest.mark.parametrize("seed", range(3))
def test_unit_chunk_sums_to_8192_are_exact_in_float32(seed):
    """Counts up to 8192 of 1.0 products summed in float32 in a random order
    are exact, and the last mantissa bit of D + 2^23 is count mod 2."""
    rng = np.random.default_rng(100 + seed)
    for count in [0, 1, 2, 4095, 4096, 4097, 8191, 8192] + list(rng.integers(0, 8193, size=20)):
        terms = np.zeros(8192, np.float32)
        terms[:count] = 1.0
        rng.shuffle(terms)
        d = np.float32(0.0)
        for t in terms:
            d = np.float32(d + t)
        assert d == np.float32(count)
        f = np.float32(d + np.float32(8388608.0))
        assert int(f.view(np.uint32)) & 1 == count & 1, count


def truncated_sum(terms, bits):
    """Sequential sum in an accumulator that keeps `bits` significant bits
    (each partial sum truncated towards zero to that precision)."""
    acc = 0
    for t in terms:
        acc += int(t)
        if acc:
            drop = max(0, acc.bit_length() - bits)
            acc = (acc >> drop) << drop
    return acc


def test_chunk_bounds_hold_for_narrow_accumulators():
    """The stated bounds: counts <= 2^12 (FP8 chunks) are exact with 12
    significant bits and counts <= 2^13 (FP4 chunks) with 13, in any order of
    0/1 terms; one bit fewer loses the count 2^b - 1."""
    rng = np.random.default_rng(11)
    for bits, bound in ((12, 4096), (13, 8192)):
        for count in [bound, bound - 1, bound // 2 + 1] + list(rng.integers(0, bound + 1, size=10)):
            terms = np.zeros(bound, np.int64)
            terms[:count] = 1
            rng.shuffle(terms)
            assert truncated_sum(terms, bits) == count, (bits, count)
        assert truncated_sum(np.ones(bound - 1, np.int64), bits - 1) != bound - 1
