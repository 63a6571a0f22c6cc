// batched.cu -- many independent products of uneven shapes in ONE persistent
// launch, replayed as a CUDA graph, with the tile shape chosen by an
// autotuner (the batched form of the Method of the Four Russians base case,
// Section 3, Algorithms 1-3).
//
// Device side: a persistent kernel whose CTAs pull tiles from one atomic
// work counter.  Every product has its own A, B, C pointers, strides and
// sizes in a descriptor table.  Two kinds of tile:
//  * one product per tile: (product, first row, first word) of a C block of
//    BM rows x LPR*128 columns (m4rm_batched_kernel);
//  * slot-packed: the 8 sixteen-byte lane chunks of a 1024-column tile are
//    128-column slices of up to 8 different products, each lane working on
//    its own slot's A rows, B rows, masks and C (m4rm_slots_kernel), so that
//    narrow products do not leave most of a tile empty;
//  * tall slot-packed: the same slots over 512 rows with k = 8 tables
//    (m4rm_tall_slots_kernel), for the tall row blocks of a batch.
// Tiles are ordered by decreasing K extent (longest first) so the queue
// drains evenly.  A split variant runs the tall row blocks on the tall
// kernel and the rest on the slot kernel, two kernel nodes of one graph.
//
// Host side (gf2_mul_batched): the first call for a set of operands builds
// the descriptor tables, lets the autotuner time every candidate variant on
// that batch (candidates differ in k, t, tile rows BM and tile width), keeps
// the fastest, and builds a CUDA graph {reset counters, persistent kernel(s)}.
// Later calls with the same operands replay the graph.  The autotuner's
// choices are cached per shape signature, and can be persisted to the JSON
// file named by the GF2_TUNE_CACHE environment variable.
#include "common.cuh"
#include "m4rm_dev.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace gf2 {
namespace {

using namespace m4rm_dev;


struct BProd {
    const uint64_t *A;
    const uint64_t *B;
    uint64_t *C;
    int64_t lda, ldb, ldc;
    int64_t m, l, n;
};

struct BTile {
    int prod;
    int row0;
    int word0;
    int pad;
};

template <int KB, int NT, int LPR, int R, int NW>
__global__ void __launch_bounds__(NW * 32) m4rm_batched_kernel(const BProd *__restrict__ prods,
                                                               const void *__restrict__ tiles_v, int ntiles,
                                                               unsigned int *counter, int accumulate)
{
    const BTile *tiles = static_cast<const BTile *>(tiles_v);
    constexpr int NTH = NW * 32;
    constexpr int KG = KB * NT;
    constexpr int TROWS = 1 << KB;
    constexpr int RPS = 32 / LPR;                 // rows per warp step
    constexpr int BM = NW * RPS * R;
    constexpr int TW = 2 * LPR;                   // words per tile row
    constexpr unsigned IMASK = (1u << KB) - 1u;
    static_assert(KG <= 64, "");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint4 *tab = reinterpret_cast<uint4 *>(smem_raw);   // NT * TROWS * LPR
    uint4 *stg = tab + NT * TROWS * LPR;                  // 2 * KG * LPR
    uint4 *sta = stg + 2 * KG * LPR;                      // 2 * BM
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int chunk = lane % LPR;
    const int trow = warp * RPS * R + lane / LPR;         // tile row of row-group r: trow + RPS*r

    while (true) {
        if (tid == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        const BTile T = tiles[t];
        const BProd P = prods[T.prod];
        const int64_t row0 = T.row0;
        const int64_t w0 = T.word0;
        const int64_t nW = words_of(P.n);
        const int64_t lW = words_of(P.l);
        const int groups = (int)((P.l + KG - 1) / KG);
        const int64_t cw = w0 + 2 * chunk;
        const uint64_t cm0 = word_mask(cw, P.n), cm1 = word_mask(cw + 1, P.n);
        const uint4 cmask = make_uint4((uint32_t)cm0, (uint32_t)(cm0 >> 32), (uint32_t)cm1,
                                       (uint32_t)(cm1 >> 32));
        uint4 acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = make_uint4(0, 0, 0, 0);

        auto issue_stage = [&](int g, int buf) {
#pragma unroll 1
            for (int i = tid; i < KG * LPR; i += NTH) {
                const int rr = i / LPR, cc = i % LPR;
                const int64_t brow = (int64_t)g * KG + rr;
                const int64_t bw = w0 + 2 * cc;
                const bool valid = (brow < P.l) && (bw < nW);
                cp_async16(&stg[buf * KG * LPR + i], valid ? (P.B + brow * P.ldb + bw) : P.B, valid);
            }
            const int64_t kb = (int64_t)g * KG;
            const int64_t wa = kb >> 6;
            const bool two = ((kb & 63) + KG > 64) && (wa + 1 < lW);
#pragma unroll 1
            for (int i = tid; i < BM; i += NTH) {
                const int64_t row = row0 + i;
                const bool valid = row < P.m;
                const uint64_t *src = P.A + (valid ? row * P.lda + wa : 0);
                uint4 *dst = &sta[buf * BM + i];
                cp_async8(dst, src, valid);
                if (two) cp_async8(reinterpret_cast<char *>(dst) + 8, src + 1, valid);
            }
            cp_async_commit();
        };

        if (groups > 0) issue_stage(0, 0);
#pragma unroll 1
        for (int g = 0; g < groups; ++g) {
            const int buf = g & 1;
            cp_async_wait_all();
            __syncthreads();
            if (g + 1 < groups) issue_stage(g + 1, buf ^ 1);
            build_tables<KB, NT, NTH, LPR>(tab, stg + buf * KG * LPR, tid, cmask);
            __syncthreads();
            const int64_t kb = (int64_t)g * KG;
            const int64_t wa = kb >> 6;
            const int sh = (int)(kb & 63);
            const uint64_t mlo = word_mask(wa, P.l);
            const uint64_t mhi = (sh + KG > 64) ? word_mask(wa + 1, P.l) : 0ull;
            const uint4 *arow = sta + buf * BM + trow;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint2 aw = *reinterpret_cast<const uint2 *>(&arow[RPS * r]);
                uint64_t bits = (((uint64_t)aw.y << 32 | aw.x) & mlo) >> sh;
                if (sh + KG > 64) {
                    const uint2 aw2 = reinterpret_cast<const uint2 *>(&arow[RPS * r])[1];
                    bits |= (((uint64_t)aw2.y << 32 | aw2.x) & mhi) << (64 - sh);
                }
                uint4 a = acc[r];
#pragma unroll
                for (int ti = 0; ti < NT; ++ti) {
                    const unsigned x = (unsigned)(bits >> (ti * KB)) & IMASK;
                    a = x4(a, tab[(ti * TROWS + (int)x) * LPR + chunk]);
                }
                acc[r] = a;
                asm volatile("" ::: "memory");
            }
        }

        if (cw < nW) {
            const int64_t first = row0 + trow;
            const int64_t left = P.m - first;
            const int nrows = left <= 0 ? 0 : (left < RPS * R ? (int)left : RPS * R);
            uint64_t *cr = P.C + first * P.ldc + cw;
            const int64_t step = (int64_t)RPS * P.ldc;
            if (!accumulate && cw + 1 < nW) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (RPS * r < nrows) *reinterpret_cast<uint4 *>(cr + r * step) = and4(acc[r], cmask);
            } else {
                const bool two = (cw + 1 < nW);
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
                    if (RPS * r >= nrows) break;
                    uint4 a = make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        if (q == r) a = acc[q];
                    const uint64_t v0 = ((uint64_t)a.y << 32 | a.x) & cm0;
                    const uint64_t v1 = ((uint64_t)a.w << 32 | a.z) & cm1;
                    uint64_t *c = cr + r * step;
                    if (accumulate) {
                        c[0] ^= v0;
                        if (two) c[1] ^= v1;
                    } else {
                        c[0] = v0;
                    }
                }
            }
        }
        (void)TW;
        __syncthreads();    // s_tile and shared buffers are reused by the next tile
    }
}

// Slot-packed tiles: a 1024-column tile whose 8 column chunks (128 columns,
// one per lane of a quarter-warp) come from up to 8 different products.  A
// slot is (product, first row, first word) of a BM x 128 block of that
// product's C; each lane works on its own slot's A rows, B rows and masks,
// so narrow products fill whole tiles.  Table reads stay one full 128-byte
// row per quarter-warp (conflict free).
struct PSlot {
    int prod;     // -1: empty slot
    int row0;
    int word0;
    int pad;
};
struct PTile {
    PSlot slot[8];
    int groups;   // passes: the largest of the slots' ceil(l / (k t))
    int pad[3];
};

template <int KB, int NT, int R, int NW>
__global__ void __launch_bounds__(NW * 32) m4rm_slots_kernel(const BProd *__restrict__ prods,
                                                             const void *__restrict__ tiles_v, int ntiles,
                                                             unsigned int *counter, int accumulate)
{
    constexpr int LPR = 8;
    constexpr int NTH = NW * 32;
    constexpr int KG = KB * NT;
    constexpr int TROWS = 1 << KB;
    constexpr int BM = NW * 4 * R;
    constexpr int PPC = 128 / KG;                         // passes per staged A chunk
    constexpr unsigned IMASK = (1u << KB) - 1u;
    static_assert(128 % KG == 0, "slot tiles stage A in 128-column chunks");
    const PTile *tiles = static_cast<const PTile *>(tiles_v);

    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint4 *tab = reinterpret_cast<uint4 *>(smem_raw);   // NT * TROWS * 8
    uint4 *stg = tab + NT * TROWS * LPR;                  // 2 * KG * 8
    uint4 *sta = stg + 2 * KG * LPR;                      // 2 * BM * 8: A chunk of (row, slot)
    __shared__ BProd sp[8];
    __shared__ PSlot ss[8];
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int c = lane & 7;                               // my slot
    const int trow = warp * 4 * R + (lane >> 3);

    while (true) {
        if (tid == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        if (tid < 8) {
            const PSlot sl = tiles[t].slot[tid];
            ss[tid] = sl;
            if (sl.prod >= 0) sp[tid] = prods[sl.prod];
        }
        const int groups = tiles[t].groups;
        __syncthreads();
        const bool mine = ss[c].prod >= 0;
        const int64_t my_m = mine ? sp[c].m : 0, my_l = mine ? sp[c].l : 0, my_n = mine ? sp[c].n : 0;
        const int64_t my_row0 = ss[c].row0, my_w = ss[c].word0;
        const uint64_t cm0 = mine ? word_mask(my_w, my_n) : 0ull, cm1 = mine ? word_mask(my_w + 1, my_n) : 0ull;
        const uint4 cmask = make_uint4((uint32_t)cm0, (uint32_t)(cm0 >> 32), (uint32_t)cm1, (uint32_t)(cm1 >> 32));
        uint4 acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = make_uint4(0, 0, 0, 0);

        auto issue_stage = [&](int g, int buf, bool a_chunk) {
#pragma unroll 1
            for (int i = tid; i < KG * LPR; i += NTH) {
                const int rr = i >> 3, cc = i & 7;
                const int64_t brow = (int64_t)g * KG + rr;
                const bool valid = ss[cc].prod >= 0 && brow < sp[cc].l && ss[cc].word0 < words_of(sp[cc].n);
                const uint64_t *src = valid ? (sp[cc].B + brow * sp[cc].ldb + ss[cc].word0) : prods[0].B;
                cp_async16(&stg[buf * KG * LPR + i], src, valid);
            }
            if (a_chunk) {
                const int64_t wa = 2 * (int64_t)(g / PPC);
                const int abuf = (g / PPC) & 1;
#pragma unroll 1
                for (int i = tid; i < BM * LPR; i += NTH) {
                    const int row = i >> 3, cc = i & 7;
                    const int64_t grow = (int64_t)ss[cc].row0 + row;
                    const bool valid = ss[cc].prod >= 0 && grow < sp[cc].m && wa < words_of(sp[cc].l);
                    const uint64_t *src = valid ? (sp[cc].A + grow * sp[cc].lda + wa) : prods[0].A;
                    cp_async16(&sta[abuf * BM * LPR + i], src, valid);
                }
            }
            cp_async_commit();
        };

        if (groups > 0) issue_stage(0, 0, true);
#pragma unroll 1
        for (int g = 0; g < groups; ++g) {
            const int buf = g & 1;
            cp_async_wait_all();
            __syncthreads();
            if (g + 1 < groups) issue_stage(g + 1, buf ^ 1, ((g + 1) % PPC) == 0);
            build_tables<KB, NT, NTH, LPR>(tab, stg + buf * KG * LPR, tid, cmask);
            __syncthreads();
            const int64_t kb = (int64_t)g * KG;
            const int64_t wa = kb >> 6;
            const int sh = (int)(kb & 63);
            const uint64_t mlo = mine ? word_mask(wa, my_l) : 0ull;
            const uint4 *arow = sta + ((g / PPC) & 1) * BM * LPR + trow * LPR + c;
            const int aoff = (int)(wa & 1);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const uint2 aw = reinterpret_cast<const uint2 *>(&arow[4 * r * LPR])[aoff];
                const uint64_t bits = ((((uint64_t)aw.y << 32) | aw.x) & mlo) >> sh;
                uint4 a = acc[r];
#pragma unroll
                for (int ti = 0; ti < NT; ++ti) {
                    const unsigned x = (unsigned)(bits >> (ti * KB)) & IMASK;
                    a = x4(a, tab[(ti * TROWS + (int)x) * LPR + c]);
                }
                acc[r] = a;
                asm volatile("" ::: "memory");
            }
        }

        const int64_t nW = words_of(my_n);
        if (mine && my_w < nW) {
            const int64_t first = my_row0 + trow;
            const int64_t left = my_m - first;
            const int nrows = left <= 0 ? 0 : (left < 4 * R ? (int)left : 4 * R);
            uint64_t *cr = sp[c].C + first * sp[c].ldc + my_w;
            const int64_t step = 4 * sp[c].ldc;
            const bool two = my_w + 1 < nW;
            if (!accumulate && two) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (4 * r < nrows) *reinterpret_cast<uint4 *>(cr + r * step) = and4(acc[r], cmask);
            } else {
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
                    if (4 * r >= nrows) break;
                    uint4 a = make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int q = 0; q < R; ++q)
                        if (q == r) a = acc[q];
                    const uint64_t v0 = ((uint64_t)a.y << 32 | a.x) & cm0;
                    const uint64_t v1 = ((uint64_t)a.w << 32 | a.z) & cm1;
                    uint64_t *cc = cr + r * step;
                    if (accumulate) {
                        cc[0] ^= v0;
                        if (two) cc[1] ^= v1;
                    } else {
                        cc[0] = v0;
                    }
                }
            }
        }
        __syncthreads();    // s_tile, slot descriptors and shared buffers are reused
    }
}

// Tall slot-packed tiles for k = 8 tables (Section 3.1; t = 4 tables per
// pass, Section 3.3): the same 8 slots of 128 columns as m4rm_slots_kernel,
// but 512 rows per tile (8 rows per thread), so that one build of the four
// 256-entry tables (128 KB) serves four times as many lookups as a 128-row
// tile.  A is staged in 16-byte chunks per (row, slot) (128 entries of K,
// four passes) by 16-byte copies that bypass L1, into one 64 KB buffer; at
// the start of a chunk every thread moves its rows' chunks into registers,
// and once every thread has done so (the barrier before the lookups) the
// next chunk is copied into the buffer, so it lands during the next four
// passes and no lookup waits on a shared-memory read of A.  Each thread
// stages one slot's rows (its slot is fixed by the thread index).  The
// tile's `rows` field is the largest row count of its slots: warps whose
// rows all lie beyond it skip the lookups.
template <int KB, int NT, int R, int NW>
__global__ void __launch_bounds__(NW * 32, 1) m4rm_tall_slots_kernel(const BProd *__restrict__ prods,
                                                                      const void *__restrict__ tiles_v,
                                                                      int ntiles, unsigned int *counter,
                                                                      int accumulate)
{
    constexpr int LPR = 8;
    constexpr int NTH = NW * 32;
    constexpr int KG = KB * NT;
    constexpr int TROWS = 1 << KB;
    constexpr int PPC = 128 / KG;                         // passes per staged 16-byte A chunk
    constexpr int SROWS = NTH / LPR;                      // rows one staging sweep covers
    constexpr unsigned IMASK = (1u << KB) - 1u;
    static_assert(128 % KG == 0 && KG == 32, "32-bit passes tile the 16-byte A chunks");
    static_assert(NTH % LPR == 0 && KG * LPR <= NTH, "");
    const PTile *tiles = static_cast<const PTile *>(tiles_v);

    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint4 *tab = reinterpret_cast<uint4 *>(smem_raw);     // NT * TROWS * 8
    uint4 *stg = tab + NT * TROWS * LPR;                  // 2 * KG * 8
    uint4 *sta = stg + 2 * KG * LPR;                      // BM * 8: A chunk of (row, slot)
    __shared__ BProd sp[8];
    __shared__ PSlot ss[8];
    __shared__ int s_tile;

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int c = lane & 7;                               // my slot (lookups and output)
    const int trow = warp * 4 * R + (lane >> 3);          // rows trow + 4 r
    const int cs = tid & 7, srow = tid >> 3;              // staging: slot cs, rows srow + SROWS j

    while (true) {
        if (tid == 0) s_tile = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= ntiles) break;
        if (tid < 8) {
            const PSlot sl = tiles[t].slot[tid];
            ss[tid] = sl;
            if (sl.prod >= 0) sp[tid] = prods[sl.prod];
        }
        const int groups = tiles[t].groups;
        const int rows = tiles[t].pad[0];                 // largest row count of the slots
        __syncthreads();
        const bool mine = ss[c].prod >= 0;
        const int64_t my_m = mine ? sp[c].m : 0, my_l = mine ? sp[c].l : 0, my_n = mine ? sp[c].n : 0;
        const int64_t my_row0 = ss[c].row0, my_w = ss[c].word0;
        const uint64_t cm0 = mine ? word_mask(my_w, my_n) : 0ull, cm1 = mine ? word_mask(my_w + 1, my_n) : 0ull;
        const uint4 cmask = make_uint4((uint32_t)cm0, (uint32_t)(cm0 >> 32), (uint32_t)cm1, (uint32_t)(cm1 >> 32));
        const bool active = warp * 4 * R < rows;          // warp-uniform
        // the staging thread's slot: its A rows srow + SROWS j of the slot's
        // row block (below the product's m and below `rows`, at most the
        // tile's 4 R NW rows: the buffer holds no more)
        const bool s_mine = ss[cs].prod >= 0;
        const int64_t s_lda = s_mine ? sp[cs].lda : 0;
        const uint64_t *s_a = s_mine ? sp[cs].A + ((int64_t)ss[cs].row0 + srow) * s_lda : prods[0].A;
        const int64_t s_end = s_mine ? sp[cs].m - ss[cs].row0 : 0;       // rows of the product from row0
        const int64_t s_left = (s_end < rows ? s_end : rows) - srow;
        const int s_nj = s_left <= 0 ? 0 : (int)((s_left + SROWS - 1) / SROWS);
        const int64_t s_lw = s_mine ? words_of(sp[cs].l) : 0;
        uint4 acc[R], areg[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            acc[r] = make_uint4(0, 0, 0, 0);
            areg[r] = make_uint4(0, 0, 0, 0);
        }

        auto issue_b = [&](int g, int buf) {
            if (tid < KG * LPR) {
                const int rr = tid >> 3, cc = tid & 7;
                const int64_t brow = (int64_t)g * KG + rr;
                const bool valid = ss[cc].prod >= 0 && brow < sp[cc].l && ss[cc].word0 < words_of(sp[cc].n);
                const uint64_t *src = valid ? (sp[cc].B + brow * sp[cc].ldb + ss[cc].word0) : prods[0].B;
                cp_async16(&stg[buf * KG * LPR + tid], src, valid);
            }
        };
        // A chunk `ch`: words 2 ch, 2 ch + 1 of every staged row (rows at or
        // past the slot's m are left as they are: their outputs are not stored)
        auto issue_a = [&](int ch) {
            const int64_t wa = 2 * (int64_t)ch;
            const bool kin = wa < s_lw;
#pragma unroll 1
            for (int j = 0; j < s_nj; ++j) {
                const int row = srow + SROWS * j;
                cp_async16(&sta[row * LPR + cs], kin ? s_a + SROWS * j * s_lda + wa : prods[0].A, kin);
            }
        };

        if (groups > 0) {
            issue_a(0);
            issue_b(0, 0);
            cp_async_commit();
        }
#pragma unroll 1
        for (int g = 0; g < groups; ++g) {
            const int buf = g & 1;
            const bool chunk_start = (g % PPC) == 0;
            cp_async_wait_all();
            __syncthreads();                              // B rows of pass g (and A chunk) landed
            if (chunk_start && active) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (warp * 4 * R + 4 * r < rows) areg[r] = sta[(trow + 4 * r) * LPR + c];
            }
            if (g + 1 < groups) issue_b(g + 1, buf ^ 1);
            build_tables<KB, NT, NTH, LPR>(tab, stg + buf * KG * LPR, tid, cmask);
            __syncthreads();                              // tables built, A chunk in registers
            if (chunk_start && g + PPC < groups) issue_a(g / PPC + 1);
            cp_async_commit();
            if (active) {
                const int64_t kb = (int64_t)g * KG;
                const int q = g % PPC;                    // 32-bit word of the chunk
                const uint32_t mlo = mine ? (uint32_t)(word_mask(kb >> 6, my_l) >> (kb & 63)) : 0u;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (warp * 4 * R + 4 * r < rows) {
                        const uint32_t w = q == 0 ? areg[r].x : q == 1 ? areg[r].y : q == 2 ? areg[r].z : areg[r].w;
                        const uint32_t bits = w & mlo;
                        uint4 a = acc[r];
#pragma unroll
                        for (int ti = 0; ti < NT; ++ti) {
                            const unsigned x = (bits >> (ti * KB)) & IMASK;
                            a = x4(a, tab[(ti * TROWS + (int)x) * LPR + c]);
                        }
                        acc[r] = a;
                    }
                }
            }
        }

        const int64_t nW = words_of(my_n);
        if (mine && my_w < nW) {
            const int64_t first = my_row0 + trow;
            const int64_t left = my_m - first;
            const int nrows = left <= 0 ? 0 : (left < 4 * R ? (int)left : 4 * R);
            uint64_t *cr = sp[c].C + first * sp[c].ldc + my_w;
            const int64_t step = 4 * sp[c].ldc;
            const bool two = my_w + 1 < nW;
            if (!accumulate && two) {
#pragma unroll
                for (int r = 0; r < R; ++r)
                    if (4 * r < nrows) *reinterpret_cast<uint4 *>(cr + r * step) = and4(acc[r], cmask);
            } else {
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
                    if (4 * r >= nrows) break;
                    uint4 a = make_uint4(0, 0, 0, 0);
#pragma unroll
                    for (int qq = 0; qq < R; ++qq)
                        if (qq == r) a = acc[qq];
                    const uint64_t v0 = ((uint64_t)a.y << 32 | a.x) & cm0;
                    const uint64_t v1 = ((uint64_t)a.w << 32 | a.z) & cm1;
                    uint64_t *cc = cr + r * step;
                    if (accumulate) {
                        cc[0] ^= v0;
                        if (two) cc[1] ^= v1;
                    } else {
                        cc[0] = v0;
                    }
                }
            }
        }
        __syncthreads();    // s_tile, slot descriptors and shared buffers are reused
    }
}

using BatchedFn = void (*)(const BProd *, const void *, int, unsigned int *, int);

// One kernel of a variant: its function, tile shape and dynamic shared memory.
struct BKernel {
    BatchedFn fn;
    int k, t, lpr, bm, nw, smem;
    int packed;   // 1: slot-packed tiles (PTile), 0: one product per tile (BTile)
};

// A tile variant: one kernel over every tile, or (split > 0) the tall slot
// kernel over the row blocks of at least `split` rows followed by `main`
// over the rest.
struct BVariant {
    const char *name;
    BKernel main;
    int split;
    BKernel tall;
};

template <int KB, int NT, int LPR, int R, int NW>
BKernel one_kernel()
{
    constexpr int BM = NW * (32 / LPR) * R;
    return BKernel{&m4rm_batched_kernel<KB, NT, LPR, R, NW>, KB, NT, LPR, BM, NW,
                   NT * (1 << KB) * LPR * 16 + 2 * KB * NT * LPR * 16 + 2 * BM * 16, 0};
}

template <int KB, int NT, int R, int NW>
BKernel slot_kernel()
{
    constexpr int BM = NW * 4 * R;
    return BKernel{&m4rm_slots_kernel<KB, NT, R, NW>, KB, NT, 8, BM, NW,
                   NT * (1 << KB) * 8 * 16 + 2 * KB * NT * 8 * 16 + 2 * BM * 8 * 16, 1};
}

template <int KB, int NT, int R, int NW>
BKernel tall_kernel()
{
    constexpr int BM = NW * 4 * R;
    return BKernel{&m4rm_tall_slots_kernel<KB, NT, R, NW>, KB, NT, 8, BM, NW,
                   NT * (1 << KB) * 8 * 16 + 2 * KB * NT * 8 * 16 + BM * 8 * 16, 1};
}

const std::vector<BVariant> &bvariants()
{
    static const BKernel none{};
    static const std::vector<BVariant> v = {
        {"k8t4-w1024-bm1024", one_kernel<8, 4, 8, 32, 8>(), 0, none},
        {"k6t8-w1024-bm256", one_kernel<6, 8, 8, 8, 8>(), 0, none},
        {"k6t8-w512-bm512", one_kernel<6, 8, 4, 8, 8>(), 0, none},
        {"k5t8-w512-bm256", one_kernel<5, 8, 4, 4, 8>(), 0, none},
        {"k4t8-w512-bm256", one_kernel<4, 8, 4, 4, 8>(), 0, none},
        {"k6t8-w256-bm512", one_kernel<6, 8, 2, 4, 8>(), 0, none},
        {"k4t8-w256-bm256", one_kernel<4, 8, 2, 2, 8>(), 0, none},
        {"k8t4-w512-bm1024", one_kernel<8, 4, 4, 16, 8>(), 0, none},
        {"slots-k8t4-bm256", slot_kernel<8, 4, 8, 8>(), 0, none},
        {"slots-k4t8-bm256", slot_kernel<4, 8, 8, 8>(), 0, none},
        {"slots-k4t8-bm128", slot_kernel<4, 8, 4, 8>(), 0, none},
        {"tall-k8t4-bm512", tall_kernel<8, 4, 8, 16>(), 0, none},
        {"tall-k8t4-bm512-from256+slots-k4t8-bm128", slot_kernel<4, 8, 4, 8>(), 256, tall_kernel<8, 4, 8, 16>()},
        {"tall-k8t4-bm512-from384+slots-k4t8-bm128", slot_kernel<4, 8, 4, 8>(), 384, tall_kernel<8, 4, 8, 16>()},
        {"tall-k8t4-bm512-from512+slots-k4t8-bm128", slot_kernel<4, 8, 4, 8>(), 512, tall_kernel<8, 4, 8, 16>()},
        {"tall-k8t4-bm512-from256+slots-k4t8-bm256", slot_kernel<4, 8, 8, 8>(), 256, tall_kernel<8, 4, 8, 16>()},
    };
    return v;
}

// ------------------------------------------------------------------ planning

// Tile descriptors of one variant: list 0 for `main`, list 1 for `tall`
// (empty unless split), as bytes of BTile or PTile records.
struct TileLists {
    std::vector<unsigned char> bytes[2];
    int ntiles[2] = {0, 0};
};

// A slot unit: (product, row block, 128-column chunk).
struct Unit { int prod, row0, word0, groups, rows; };

// Slot units grouped 8 per tile among units with similar pass counts and
// row counts; a tile's pad[0] is the largest row count of its slots.
void pack_units(std::vector<Unit> &units, std::vector<unsigned char> &bytes, int *ntiles)
{
    std::stable_sort(units.begin(), units.end(), [](const Unit &a, const Unit &b) {
        return a.groups != b.groups ? a.groups > b.groups : a.rows > b.rows;
    });
    std::vector<PTile> tiles((units.size() + 7) / 8);
    for (size_t t = 0; t < tiles.size(); ++t) {
        PTile &T = tiles[t];
        memset(&T, 0, sizeof T);
        for (int j = 0; j < 8; ++j) {
            const size_t u = t * 8 + j;
            if (u < units.size()) {
                T.slot[j] = PSlot{units[u].prod, units[u].row0, units[u].word0, 0};
                T.groups = std::max(T.groups, units[u].groups);
                T.pad[0] = std::max(T.pad[0], units[u].rows);
            } else {
                T.slot[j] = PSlot{-1, 0, 0, 0};
            }
        }
    }
    bytes.resize(tiles.size() * sizeof(PTile));
    if (!tiles.empty()) memcpy(bytes.data(), tiles.data(), bytes.size());
    *ntiles = (int)tiles.size();
}

// Units of rows [r_lo, m) of product i in row blocks of bm rows.
void add_units(std::vector<Unit> &units, const BProd &p, int i, int64_t r_lo, int bm, int kg)
{
    const int64_t W = words_of(p.n);
    const int groups = (int)((p.l + kg - 1) / kg);
    for (int64_t r = r_lo; r < p.m; r += bm)
        for (int64_t w = 0; w < W; w += 2)
            units.push_back(Unit{i, (int)r, (int)w, groups, (int)std::min<int64_t>(bm, p.m - r)});
}

void build_tiles(const std::vector<BProd> &prods, const BVariant &v, TileLists &out)
{
    out = TileLists{};
    const BKernel &k = v.main;
    if (!k.packed) {
        std::vector<BTile> tiles;
        const int tw = 2 * k.lpr;
        for (size_t i = 0; i < prods.size(); ++i) {
            const BProd &p = prods[i];
            if (p.m <= 0 || p.n <= 0) continue;
            const int64_t W = words_of(p.n);
            for (int64_t r = 0; r < p.m; r += k.bm)
                for (int64_t w = 0; w < W; w += tw) tiles.push_back(BTile{(int)i, (int)r, (int)w, 0});
        }
        // longest K first (the work of a tile grows with the K extent)
        std::stable_sort(tiles.begin(), tiles.end(), [&](const BTile &a, const BTile &b) {
            return prods[a.prod].l > prods[b.prod].l;
        });
        out.bytes[0].resize(tiles.size() * sizeof(BTile));
        if (!tiles.empty()) memcpy(out.bytes[0].data(), tiles.data(), out.bytes[0].size());
        out.ntiles[0] = (int)tiles.size();
        return;
    }
    std::vector<Unit> units, tall;
    for (size_t i = 0; i < prods.size(); ++i) {
        const BProd &p = prods[i];
        if (p.m <= 0 || p.n <= 0) continue;
        int64_t r_lo = 0;
        if (v.split > 0) {
            // rows [0, r_lo) on the tall kernel: its full blocks, and the last
            // block too if it keeps `split` rows
            const int64_t tb = v.tall.bm;
            const int64_t full = p.m / tb * tb;
            r_lo = p.m - full >= v.split ? p.m : full;
            BProd q = p;
            q.m = r_lo;
            add_units(tall, q, (int)i, 0, (int)tb, v.tall.k * v.tall.t);
        }
        add_units(units, p, (int)i, r_lo, k.bm, k.k * k.t);
    }
    pack_units(units, out.bytes[0], &out.ntiles[0]);
    if (v.split > 0) pack_units(tall, out.bytes[1], &out.ntiles[1]);
}

int grid_for(const BKernel &v)
{
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, v.fn, v.nw * 32, v.smem) != cudaSuccess || per < 1) {
        cudaGetLastError();
        per = 1;
    }
    return sms * per;
}

// Shape signature used by the autotuner's cache: the sorted list of shapes.
std::string signature(const std::vector<BProd> &prods, int accumulate)
{
    std::vector<unsigned long long> key;
    key.reserve(prods.size());
    for (const BProd &p : prods)
        key.push_back(((unsigned long long)p.m << 42) ^ ((unsigned long long)p.l << 21) ^ (unsigned long long)p.n);
    std::sort(key.begin(), key.end());
    unsigned long long h = 1469598103934665603ull;
    for (unsigned long long k : key) {
        h ^= k;
        h *= 1099511628211ull;
    }
    char buf[96];
    snprintf(buf, sizeof buf, "batched-%s-n%zu-a%d-%016llx", arch_tag().c_str(), prods.size(), accumulate, h);
    return buf;
}

// ------------------------------------------------------------------ graphs
struct GraphEntry {
    std::vector<unsigned long long> key;    // operand pointers, sizes, strides, stream, options
    int variant = -1;
    void *dev = nullptr;                     // descriptor tables + counters (one cudaMalloc)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int ntiles = 0;                          // over both kernels
    int nkernels = 0;                        // kernel nodes of the graph
};
std::mutex g_mu;
std::list<GraphEntry> g_graphs;             // most recently used first
constexpr size_t kMaxGraphs = 8;

void free_entry(GraphEntry &e)
{
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    if (e.dev) cudaFree(e.dev);
    e.exec = nullptr;
    e.graph = nullptr;
    e.dev = nullptr;
}

// Device copies of the tables: [prods][tiles of main][tiles of tall][2 counters]
struct DevTables {
    void *dev = nullptr;
    BProd *prods = nullptr;
    void *tiles[2] = {nullptr, nullptr};
    unsigned int *counters = nullptr;
};

int upload(const std::vector<BProd> &prods, const TileLists &tl, DevTables *d)
{
    const size_t bp = (prods.size() * sizeof(BProd) + 255) & ~(size_t)255;
    const size_t bt0 = (tl.bytes[0].size() + 255) & ~(size_t)255;
    const size_t bt1 = (tl.bytes[1].size() + 255) & ~(size_t)255;
    void *p = nullptr;
    if (cudaMalloc(&p, bp + bt0 + bt1 + 256) != cudaSuccess) {
        cudaGetLastError();
        return GF2_ENOMEM;
    }
    char *c = static_cast<char *>(p);
    d->dev = p;
    d->prods = reinterpret_cast<BProd *>(c);
    d->tiles[0] = c + bp;
    d->tiles[1] = c + bp + bt0;
    d->counters = reinterpret_cast<unsigned int *>(c + bp + bt0 + bt1);
    GF2_CUDA_TRY(cudaMemcpy(c, prods.data(), prods.size() * sizeof(BProd), cudaMemcpyHostToDevice));
    for (int j = 0; j < 2; ++j)
        if (!tl.bytes[j].empty())
            GF2_CUDA_TRY(cudaMemcpy(d->tiles[j], tl.bytes[j].data(), tl.bytes[j].size(), cudaMemcpyHostToDevice));
    return GF2_OK;
}

// The kernels of a variant in launch order (tall first: its tiles are the
// longest), with their tile lists and counters.
int kernels_of(const BVariant &v, const TileLists &tl, const DevTables &d, const BKernel *ks[2], const void *ts[2],
               int nts[2], unsigned int *cs[2])
{
    int n = 0;
    if (v.split > 0 && tl.ntiles[1] > 0) {
        ks[n] = &v.tall; ts[n] = d.tiles[1]; nts[n] = tl.ntiles[1]; cs[n] = d.counters + 1; ++n;
    }
    if (tl.ntiles[0] > 0) {
        ks[n] = &v.main; ts[n] = d.tiles[0]; nts[n] = tl.ntiles[0]; cs[n] = d.counters; ++n;
    }
    return n;
}

int launch_variant(const BVariant &v, const TileLists &tl, const DevTables &d, int accumulate, cudaStream_t s)
{
    const BKernel *ks[2];
    const void *ts[2];
    int nts[2];
    unsigned int *cs[2];
    const int nk = kernels_of(v, tl, d, ks, ts, nts, cs);
    GF2_CUDA_TRY(cudaMemsetAsync(d.counters, 0, 2 * sizeof(unsigned int), s));
    for (int j = 0; j < nk; ++j) {
        GF2_CUDA_TRY(cudaFuncSetAttribute(ks[j]->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ks[j]->smem));
        ProfScope ps(PF_BATCHED, s);
        ks[j]->fn<<<grid_for(*ks[j]), ks[j]->nw * 32, ks[j]->smem, s>>>(d.prods, ts[j], nts[j], cs[j], accumulate);
        note_launch();
        const int rc = check_launch();
        if (rc) return rc;
    }
    return GF2_OK;
}

int autotune_timed(const std::vector<BProd> &prods, int accumulate, cudaStream_t s);

// Copies of the products' C (words that carry entries, rows packed densely)
// to `buf` (to_buf) or back (!to_buf), one 2-D copy per product.
int copy_cs(const std::vector<BProd> &prods, char *buf, bool to_buf, cudaStream_t s)
{
    size_t off = 0;
    for (const BProd &p : prods) {
        if (p.m <= 0 || p.n <= 0) continue;
        const size_t w = (size_t)words_of(p.n) * 8;
        if (to_buf)
            GF2_CUDA_TRY(cudaMemcpy2DAsync(buf + off, w, p.C, (size_t)p.ldc * 8, w, (size_t)p.m,
                                           cudaMemcpyDeviceToDevice, s));
        else
            GF2_CUDA_TRY(cudaMemcpy2DAsync(p.C, (size_t)p.ldc * 8, buf + off, w, w, (size_t)p.m,
                                           cudaMemcpyDeviceToDevice, s));
        off += w * (size_t)p.m;
    }
    return GF2_OK;
}

// Times every candidate on this batch (two runs each after one warm-up) and
// returns the index of the fastest, or GF2_ECUDA when its timing events
// cannot be created.  Every timed launch writes the products' C; with
// accumulate each one XORs A B into it again, so C is saved first and put
// back afterwards (the caller's launch then sees the C it was given).
int autotune(const std::vector<BProd> &prods, int accumulate, cudaStream_t s)
{
    void *saved = nullptr;
    if (accumulate) {
        size_t bytes = 0;
        for (const BProd &p : prods)
            if (p.m > 0 && p.n > 0) bytes += (size_t)words_of(p.n) * 8 * (size_t)p.m;
        if (bytes) {
            if (cudaMalloc(&saved, bytes) != cudaSuccess) {
                cudaGetLastError();
                return GF2_ENOMEM;
            }
            const int rc = copy_cs(prods, static_cast<char *>(saved), true, s);
            if (rc) {
                cudaFree(saved);
                return rc;
            }
        }
    }
    const int best = autotune_timed(prods, accumulate, s);
    if (saved) {
        const int rc = copy_cs(prods, static_cast<char *>(saved), false, s);
        const cudaError_t e = cudaStreamSynchronize(s);
        cudaFree(saved);
        if (rc) return rc;
        if (e != cudaSuccess) return GF2_ECUDA;
    }
    return best;
}

// The timing loop of autotune.
int autotune_timed(const std::vector<BProd> &prods, int accumulate, cudaStream_t s)
{
    const auto &vs = bvariants();
    int best = 0;
    float best_ms = 1e30f;
    ScopedEvents<2> ev;
    if (ev.create()) return GF2_ECUDA;
    cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
    for (size_t i = 0; i < vs.size(); ++i) {
        TileLists tl;
        build_tiles(prods, vs[i], tl);
        DevTables d;
        if (upload(prods, tl, &d)) {
            if (d.dev) cudaFree(d.dev);
            cudaGetLastError();
            continue;
        }
        float ms = 1e30f;
        bool ok = launch_variant(vs[i], tl, d, accumulate, s) == GF2_OK;
        for (int rep = 0; ok && rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            ok = launch_variant(vs[i], tl, d, accumulate, s) == GF2_OK;
            cudaEventRecord(e1, s);
            float t = 0.f;
            if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
                ms = std::min(ms, t);
        }
        cudaStreamSynchronize(s);
        cudaFree(d.dev);
        cudaGetLastError();
        if (ok && ms < best_ms) {
            best_ms = ms;
            best = (int)i;
        }
    }
    return best;
}

}  // namespace

int batched_variant_count() { return (int)bvariants().size(); }

const char *batched_variant_name(int i)
{
    const auto &vs = bvariants();
    return (i >= 0 && i < (int)vs.size()) ? vs[i].name : nullptr;
}

// C[i] = A[i] B[i] for device operands (arguments already checked).
// `force_variant` >= 0 skips the autotuner.
int batched_mul(gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[], int count,
                int accumulate, int force_variant, cudaStream_t s, int *chosen)
{
    std::vector<BProd> prods;
    prods.reserve(count);
    std::vector<unsigned long long> key;
    key.reserve(9 * (size_t)count + 4);
    for (int i = 0; i < count; ++i) {
        BProd p;
        p.A = A[i]->data; p.B = B[i]->data; p.C = C[i]->data;
        p.lda = A[i]->stride_words; p.ldb = B[i]->stride_words; p.ldc = C[i]->stride_words;
        p.m = A[i]->rows; p.l = A[i]->cols; p.n = B[i]->cols;
        prods.push_back(p);
        key.push_back((unsigned long long)(uintptr_t)p.A);
        key.push_back((unsigned long long)(uintptr_t)p.B);
        key.push_back((unsigned long long)(uintptr_t)p.C);
        key.push_back((unsigned long long)p.lda);
        key.push_back((unsigned long long)p.ldb);
        key.push_back((unsigned long long)p.ldc);
        key.push_back((unsigned long long)p.m);
        key.push_back((unsigned long long)p.l);
        key.push_back((unsigned long long)p.n);
    }
    int dev = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    key.push_back((unsigned long long)(uintptr_t)s);
    key.push_back((unsigned long long)dev);
    key.push_back((unsigned long long)accumulate);
    key.push_back((unsigned long long)(force_variant + 1));

    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
        if (it->key == key) {
            g_graphs.splice(g_graphs.begin(), g_graphs, it);       // most recently used
            if (chosen) *chosen = g_graphs.front().variant;
            if (g_graphs.front().ntiles == 0) return GF2_OK;
            ProfScope ps(PF_BATCHED, s);
            GF2_CUDA_TRY(cudaGraphLaunch(g_graphs.front().exec, s));
            note_launch(g_graphs.front().nkernels);
            return GF2_OK;
        }
    }

    // choose the variant: forced, cached for this shape signature, or tuned now
    const auto &vs = bvariants();
    int vi = force_variant;
    if (vi < 0 || vi >= (int)vs.size()) {
        const std::string sig = signature(prods, accumulate);
        std::string name;
        vi = -1;
        if (tune_get(sig, &name))
            for (size_t i = 0; i < vs.size(); ++i)
                if (name == vs[i].name) vi = (int)i;
        if (vi < 0) {
            vi = autotune(prods, accumulate, s);
            if (vi < 0) return vi;                    // a CUDA error while timing
            tune_put(sig, vs[vi].name);
        }
    }
    const BVariant &v = vs[vi];

    GraphEntry e;
    e.key = key;
    e.variant = vi;
    TileLists tl;
    build_tiles(prods, v, tl);
    e.ntiles = tl.ntiles[0] + tl.ntiles[1];
    if (e.ntiles > 0) {
        DevTables d;
        int rc = upload(prods, tl, &d);
        e.dev = d.dev;
        if (rc) { free_entry(e); return rc; }
        const BKernel *ks[2];
        const void *ts[2];
        int nts[2];
        unsigned int *cs[2];
        const int nk = kernels_of(v, tl, d, ks, ts, nts, cs);
        e.nkernels = nk;
        // graph: reset the work counters, then the persistent kernels in order
        if (cudaGraphCreate(&e.graph, 0) != cudaSuccess) { free_entry(e); return GF2_ECUDA; }
        cudaGraphNode_t prev;
        cudaMemsetParams mp;
        memset(&mp, 0, sizeof mp);
        mp.dst = d.counters;
        mp.value = 0;
        mp.elementSize = sizeof(unsigned int);
        mp.width = 2;
        mp.height = 1;
        mp.pitch = 2 * sizeof(unsigned int);
        if (cudaGraphAddMemsetNode(&prev, e.graph, nullptr, 0, &mp) != cudaSuccess) { free_entry(e); return GF2_ECUDA; }
        for (int j = 0; j < nk; ++j) {
            GF2_CUDA_TRY(cudaFuncSetAttribute(ks[j]->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ks[j]->smem));
            const BProd *dp = d.prods;
            const void *dt = ts[j];
            int nt = nts[j];
            unsigned int *dc = cs[j];
            void *args[5] = {(void *)&dp, (void *)&dt, (void *)&nt, (void *)&dc, (void *)&accumulate};
            cudaKernelNodeParams kp;
            memset(&kp, 0, sizeof kp);
            kp.func = (void *)ks[j]->fn;
            kp.gridDim = dim3((unsigned)grid_for(*ks[j]));
            kp.blockDim = dim3((unsigned)(ks[j]->nw * 32));
            kp.sharedMemBytes = (unsigned)ks[j]->smem;
            kp.kernelParams = args;
            cudaGraphNode_t node;
            if (cudaGraphAddKernelNode(&node, e.graph, &prev, 1, &kp) != cudaSuccess) { free_entry(e); return GF2_ECUDA; }
            prev = node;
        }
        if (cudaGraphInstantiate(&e.exec, e.graph, 0) != cudaSuccess) { free_entry(e); cudaGetLastError(); return GF2_ECUDA; }
        {
            ProfScope ps(PF_BATCHED, s);
            if (cudaGraphLaunch(e.exec, s) != cudaSuccess) { free_entry(e); return GF2_ECUDA; }
        }
        note_launch(nk);
    }
    g_graphs.push_front(std::move(e));
    while (g_graphs.size() > kMaxGraphs) {
        // an older graph may still be running on its stream: wait before freeing
        cudaDeviceSynchronize();
        free_entry(g_graphs.back());
        g_graphs.pop_back();
    }
    if (chosen) *chosen = vi;
    return GF2_OK;
}

void batched_release()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_graphs.empty()) cudaDeviceSynchronize();
    for (GraphEntry &e : g_graphs) free_entry(e);
    g_graphs.clear();
}

}  // namespace gf2
