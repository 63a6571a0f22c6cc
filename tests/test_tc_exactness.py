"""The arithmetic the tensor-core base cases rest on, checked on the CPU.

The FP8 form encodes a 1-bit with K index = i (mod 4) as the E4M3 byte
2^(i-9) in A and 2^(-6-i) in B, so every product of two 1-bits is 2^-15;
a chunk of at most 4096 entries then sums to count * 2^-15, exact in FP32,
and the parity of count is the last mantissa bit of D + 256 (Section 2.3:
the GF(2) dot product is the integer dot product mod 2).  The int8 form sums
0/1 products in int32.  These tests decode E4M3 from its definition (1 sign
bit, 4 exponent bits with bias 7, 3 mantissa bits, subnormals below exponent
1) and accumulate in float32 in random orders.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def e4m3(byte: int) -> float:
    s = -1.0 if byte & 0x80 else 1.0
    e = (byte >> 3) & 0xF
    m = byte & 0x7
    if e == 0:
        return s * m * 2.0 ** -9                    # subnormal: m/8 * 2^(1-7)
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


A_BYTES = [0x01, 0x02, 0x04, 0x08]                  # K index mod 4 = 0, 1, 2, 3
B_BYTES = [0x08, 0x04, 0x02, 0x01]


def test_encodings_are_the_stated_powers_of_two():
    assert [e4m3(b) for b in A_BYTES] == [2.0 ** (i - 9) for i in range(4)]
    assert [e4m3(b) for b in B_BYTES] == [2.0 ** (-6 - i) for i in range(4)]
    assert e4m3(0x00) == 0.0


def test_every_product_of_two_one_bits_is_two_to_the_minus_15():
    for i in range(4):
        assert e4m3(A_BYTES[i]) * e4m3(B_BYTES[i]) == 2.0 ** -15
        # a byte never meets another position's byte: the K index fixes both
        assert np.float32(e4m3(A_BYTES[i])) * np.float32(e4m3(B_BYTES[i])) == np.float32(2.0 ** -15)


@pytest.mark.parametrize("seed", range(4))
def test_chunk_sums_are_exact_and_the_parity_is_the_last_mantissa_bit(seed):
    """Every count 0..4096 of unit products summed in float32 in a random
    order (with zero products interleaved) gives count * 2^-15 exactly, and
    the last mantissa bit of D + 256 is count mod 2."""
    rng = np.random.default_rng(seed)
    unit = np.float32(2.0 ** -15)
    for count in list(range(0, 70)) + list(rng.integers(70, 4097, size=60)) + [4095, 4096]:
        terms = np.zeros(4096, np.float32)
        terms[:count] = unit
        rng.shuffle(terms)
        d = np.float32(0.0)
        for t in terms:                             # sequential float32 accumulation
            d = np.float32(d + t)
        assert d == np.float32(count) * unit
        f = np.float32(d + np.float32(256.0))
        assert int(f.view(np.uint32)) & 1 == count & 1, count


def test_pairwise_float32_sums_are_exact_too():
    """A tree-shaped reduction (another order a tensor core may use) of up
    to 4096 unit products is exact as well: every partial sum is a multiple
    of 2^-15 below 2^-3, representable with 12 significant bits."""
    unit = np.float32(2.0 ** -15)
    rng = np.random.default_rng(9)
    for _ in range(50):
        v = (rng.random(4096) < rng.random()).astype(np.float32) * unit
        while v.size > 1:
            v = (v[0::2] + v[1::2]).astype(np.float32)
        count = int(round(float(v[0]) / float(unit)))
        assert v[0] == np.float32(count) * unit


def test_int8_sums_hold_the_parity():
    """The int8 form: 0/1 products summed in int32; the parity is bit 0 for
    any K below 2^31."""
    rng = np.random.default_rng(3)
    for k in (1, 255, 256, 70001, 1 << 20):
        a = rng.integers(0, 2, size=k, dtype=np.int8)
        b = rng.integers(0, 2, size=k, dtype=np.int8)
        s = int(np.sum(a.astype(np.int32) * b.astype(np.int32), dtype=np.int32))
        assert s & 1 == int(np.bitwise_xor.reduce(a & b))
