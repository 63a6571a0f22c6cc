// m4rm_dev.cuh -- device building blocks of the Method of the Four Russians
// (Section 3): cp.async staging, 128-bit XOR helpers and the Gray-code table
// build of Section 3.1, for tiles of LPR lanes x 16 bytes per row.
#pragma once

#include "common.cuh"

namespace gf2 {
namespace m4rm_dev {

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int sz = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(sz)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__host__ __device__ constexpr int ctz_c(int s) { return (s & 1) ? 0 : 1 + ctz_c(s >> 1); }

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int sz = valid ? 8 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(sz)
                 : "memory");
}

__device__ __forceinline__ uint4 x4(uint4 a, uint4 b)
{
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}
__device__ __forceinline__ uint4 and4(uint4 a, uint4 m)
{
    return make_uint4(a.x & m.x, a.y & m.y, a.z & m.z, a.w & m.w);
}

// Steps s = S .. 2^LOB - 1 of the Gray-code walk of Section 3.1: entry
// gray(s) = gray(s-1) + (row ctz(s)), one row addition per entry.  A template
// recursion keeps every register index a compile-time constant.
template <int S, int LOB, int LPR>
struct GrayWalk {
    static __device__ __forceinline__ void run(uint4 &v, const uint4 (&lo)[LOB], uint4 *T, int base)
    {
        constexpr int j = ctz_c(S);
        v = x4(v, lo[j]);
        T[(base | (S ^ (S >> 1))) * LPR] = v;
        GrayWalk<S + 1, LOB, LPR>::run(v, lo, T, base);
    }
};
template <int LOB, int LPR>
struct GrayWalk<(1 << LOB), LOB, LPR> {
    static __device__ __forceinline__ void run(uint4 &, const uint4 (&)[LOB], uint4 *, int) {}
};

// Build NT tables of 2^KB rows from KB*NT staged B rows (each LPR x 16
// bytes), one 16-byte column chunk per item (Section 3.1 Gray-code walk over
// the low bits of the index, high bits combined directly).  `cmask` masks
// the thread's column chunk (chunk == tid % LPR for every item of this
// thread, since NTH is a multiple of LPR).
template <int KB, int NT, int NTH, int LPR>
__device__ __forceinline__ void build_tables(uint4 *tab, const uint4 *stg, int tid, uint4 cmask)
{
    constexpr int LOB = KB < 4 ? KB : 4;
    constexpr int HIB = KB - LOB;
    constexpr int TROWS = 1 << KB;
    constexpr int ITEMS = NT * (1 << HIB) * LPR;
    static_assert(NTH % LPR == 0, "");
#pragma unroll 1
    for (int it = tid; it < ITEMS; it += NTH) {
        const int c = it % LPR;
        const int hi = (it / LPR) & ((1 << HIB) - 1);
        const int ti = it / (LPR << HIB);
        const uint4 *S = stg + ti * KB * LPR + c;     // row j of the stripe at S[j*LPR]
        uint4 lo[LOB];
#pragma unroll
        for (int j = 0; j < LOB; ++j) lo[j] = and4(S[j * LPR], cmask);
        uint4 v = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int j = 0; j < HIB; ++j)
            if ((hi >> j) & 1) v = x4(v, and4(S[(LOB + j) * LPR], cmask));
        uint4 *T = tab + ti * TROWS * LPR + c;        // entry x at T[x*LPR]
        const int base = hi << LOB;
        T[base * LPR] = v;
        GrayWalk<1, LOB, LPR>::run(v, lo, T, base);
    }
}


}  // namespace m4rm_dev
}  // namespace gf2
