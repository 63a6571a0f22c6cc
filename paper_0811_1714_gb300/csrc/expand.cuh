// expand.cuh -- the encoding of packed GF(2) bits as tensor-core operand
// entries: a 1-bit becomes 1.0 (FP8 E4M3 byte 0x38, FP4 E2M1 nibble 0x2), a
// 0-bit 0.  Used by the expansion kernels and by the Strassen-Winograd
// additions that write their last level's operands already expanded.
#pragma once

#include <stdint.h>

namespace gf2 {

// 4 bits -> 4 bytes of 0x00 / 0x38 (E4M3 1.0): the multiply places bit i of
// the nibble at bit 8i (the four shifted copies do not overlap), the mask
// keeps those bits, the second multiply turns each into 0x38.
__device__ __forceinline__ uint32_t f8_of_nibble(uint32_t v)
{
    return ((v * 0x00204081u) & 0x01010101u) * 0x38u;
}

// 8 bits -> 8 nibbles of 0x0 / 0x2 (E2M1 1.0), bit i in nibble i: spread by
// halves, quarters and eighths, then shift each bit to nibble bit 1.
__device__ __forceinline__ uint32_t f4_of_byte(uint32_t v)
{
    v &= 0xFFu;
    v = (v | (v << 12)) & 0x000F000Fu;
    v = (v | (v << 6)) & 0x03030303u;
    v = (v | (v << 3)) & 0x11111111u;
    return v << 1;
}

// Two packed words (128 entries, entry e in bit e % 64 of word e / 64) ->
// their expanded bytes: 8 x 16 bytes (FP8, one byte per entry) or 4 x 16
// bytes (FP4, two entries per byte, entry e in nibble e % 2 of byte e / 2).
template <bool FP8>
__device__ __forceinline__ void expand_words(uint64_t w0, uint64_t w1, uint4 *o)
{
    if (FP8) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const uint32_t h = (uint32_t)((q < 4 ? w0 : w1) >> (16 * (q & 3)));
            o[q] = make_uint4(f8_of_nibble(h & 15u), f8_of_nibble((h >> 4) & 15u), f8_of_nibble((h >> 8) & 15u),
                              f8_of_nibble((h >> 12) & 15u));
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t h = (uint32_t)((q < 2 ? w0 : w1) >> (32 * (q & 1)));
            o[q] = make_uint4(f4_of_byte(h), f4_of_byte(h >> 8), f4_of_byte(h >> 16), f4_of_byte(h >> 24));
        }
    }
}

}  // namespace gf2
