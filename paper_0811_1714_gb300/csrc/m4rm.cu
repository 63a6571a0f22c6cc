// m4rm.cu -- Method of the Four Russians base case on packed words (sm_103a).
//
// Section 3 (Algorithm 1): split A into stripes of k columns and B into
// stripes of k rows; tabulate all 2^k combinations of the k rows of a B
// stripe (MakeTable), then every row of A reads its k bits of the stripe
// (ReadBits) and adds that table row to its row of C (AddRowFromTable).
// Section 3.2 (Algorithm 2): the table is rebuilt per block of rows so that
// the rows being updated stay in fast memory.  Section 3.3 (Algorithm 3): t
// tables cover t*k rows of B per pass and each row of C receives t table
// rows per pass.
//
// GB300 mapping:
//  * one CTA owns a tile of BM rows x 1024 columns of C, held in REGISTERS
//    for the whole K loop (the analogue of the cache-friendly block);
//  * the t tables of one pass live in SHARED MEMORY, 128 bytes per table row;
//    B rows of the next pass are staged by cp.async while the current pass
//    runs;
//  * a table is built by the Gray-code walk of Section 3.1 in registers: a
//    thread holds the combination of the high bits of the index and walks
//    the low 4 bits in Gray order, one row addition (4 x 32-bit XOR) per new
//    entry; 16 threads fill a k = 8 table chunk in parallel, at 272 row
//    additions against the paper's 2^k - 1 = 255 (the 16 high combinations
//    are formed directly);
//  * lookups: 8 lanes share one C row (16 bytes = 128 columns each), so a
//    warp updates 4 rows per 128-bit shared-memory load; all accesses of a
//    quarter-warp fall in one 128-byte table row (conflict free).
//
// Table index convention: bit j of the index selects row (stripe start + j),
// and the index is read least-significant-bit first from the packed row of A
// (column c is bit c % 64 of its word).  The paper's ReadBits reads the
// stripe most-significant-bit first; the order is internal to a table and
// does not change the product.
#include "common.cuh"
#include "m4rm_dev.cuh"

#include <atomic>
#include <type_traits>

namespace gf2 {
namespace {

using namespace m4rm_dev;

constexpr int LPR = 8;          // lanes per C row
constexpr int TILE_WORDS = 16;  // 64-bit words of C per tile row (1024 columns)

struct Params {
    const uint64_t *A; int64_t lda, bsA;
    const uint64_t *B; int64_t ldb, bsB;
    uint64_t *C; int64_t ldc, bsC;
    int64_t m, l, n;
    int ksplit;
    int64_t groups_per_split;
    int mode;                   // 0: store, 1: C ^= (plain), 2: atomic XOR
};

// Tensor-memory spill of half a tile (Blackwell TMEM, 512 columns x 128
// lanes x 32 bits per SM): 8 row-groups of a thread = 32 columns of its lane.
__device__ __forceinline__ void tm_st32(uint32_t taddr, const uint4 (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
                 ::"r"(taddr), "r"(v[0].x), "r"(v[0].y), "r"(v[0].z), "r"(v[0].w), "r"(v[1].x), "r"(v[1].y), "r"(v[1].z), "r"(v[1].w), "r"(v[2].x), "r"(v[2].y), "r"(v[2].z), "r"(v[2].w), "r"(v[3].x), "r"(v[3].y), "r"(v[3].z), "r"(v[3].w), "r"(v[4].x), "r"(v[4].y), "r"(v[4].z), "r"(v[4].w), "r"(v[5].x), "r"(v[5].y), "r"(v[5].z), "r"(v[5].w), "r"(v[6].x), "r"(v[6].y), "r"(v[6].z), "r"(v[6].w), "r"(v[7].x), "r"(v[7].y), "r"(v[7].z), "r"(v[7].w) : "memory");
}
__device__ __forceinline__ void tm_ld32(uint32_t taddr, uint4 (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(v[0].x), "=r"(v[0].y), "=r"(v[0].z), "=r"(v[0].w), "=r"(v[1].x), "=r"(v[1].y), "=r"(v[1].z), "=r"(v[1].w), "=r"(v[2].x), "=r"(v[2].y), "=r"(v[2].z), "=r"(v[2].w), "=r"(v[3].x), "=r"(v[3].y), "=r"(v[3].z), "=r"(v[3].w), "=r"(v[4].x), "=r"(v[4].y), "=r"(v[4].z), "=r"(v[4].w), "=r"(v[5].x), "=r"(v[5].y), "=r"(v[5].z), "=r"(v[5].w), "=r"(v[6].x), "=r"(v[6].y), "=r"(v[6].z), "=r"(v[6].w), "=r"(v[7].x), "=r"(v[7].y), "=r"(v[7].z), "=r"(v[7].w) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// f(integral_constant<int, I>) for I = B .. E-1, unrolled at compile time
template <int B, int E, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// One CTA: a tile of BM rows x 1024 columns of C.  With TM (tall tiles),
// the tile has two halves of NWARP*4*R rows: one in registers, the other in
// tensor memory; the halves swap once per pass, after the first half's
// lookups, so the tables of a pass serve twice the rows (table cost /
// lookup cost = 2^k / BM halves) for one store + load of half a tile.  The
// swap goes by chunks of 8 row-groups (one 32-column tensor-memory access):
// a chunk is stored as soon as its lookups of the pass are done, and the
// other half's chunk j+1 is loaded while chunk j is looked up, so that the
// tensor-memory traffic runs behind shared-memory lookups.
template <int KB, int NT, int R, int NWARP, bool TM>
__global__ void __launch_bounds__(NWARP * 32, 1) m4rm_kernel(Params P)
{
    constexpr int NTH = NWARP * 32;
    constexpr int KG = KB * NT;          // rows of B per pass = bits of each A row per pass
    constexpr int TROWS = 1 << KB;
    constexpr int HM = NWARP * 4 * R;    // rows held in registers
    constexpr int BM = TM ? 2 * HM : HM;
    constexpr unsigned IMASK = (1u << KB) - 1u;
    static_assert(KG <= 64, "a pass reads at most 64 bits of a row of A");
    static_assert(!TM || (NWARP == 8 && R == 32), "tensor-memory halves: 8 warps x 128 columns per slot");

    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint4 *tab = reinterpret_cast<uint4 *>(smem_raw);        // NT * TROWS * 8
    uint4 *stg = tab + NT * TROWS * LPR;                       // 2 * KG * 8   (B rows of a pass)
    uint4 *sta = stg + 2 * KG * LPR;                           // 2 * BM       (A words of a pass)
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sta + 2 * BM);

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int chunk = lane & 7;
    const int64_t w0 = (int64_t)blockIdx.x * TILE_WORDS;
    const int64_t row0 = (int64_t)blockIdx.y * BM;
    const int bidx = blockIdx.z / P.ksplit;
    const int split = blockIdx.z % P.ksplit;

    const uint64_t *A = P.A + (int64_t)bidx * P.bsA;
    const uint64_t *B = P.B + (int64_t)bidx * P.bsB;
    uint64_t *C = P.C + (int64_t)bidx * P.bsC;

    const int64_t nW = words_of(P.n);
    const int64_t lW = words_of(P.l);
    const int groups = (int)((P.l + KG - 1) / KG);
    const int g_begin = split * (int)P.groups_per_split;
    const int g_end = min(groups, g_begin + (int)P.groups_per_split);

    const int64_t cw = w0 + 2 * chunk;
    const uint64_t cm0 = word_mask(cw, P.n), cm1 = word_mask(cw + 1, P.n);
    const uint4 cmask = make_uint4((uint32_t)cm0, (uint32_t)(cm0 >> 32), (uint32_t)cm1,
                                   (uint32_t)(cm1 >> 32));

    const int trow = warp * 4 * R + (lane >> 3);               // tile row of row-group r: trow + 4r

    // tensor memory: warp w owns lanes 32 (w % 4) .. +31 and the 256 columns
    // starting at 256 (w / 4), as two slots of 128 columns (R row-groups)
    uint32_t t_other = 0, t_free = 0;
    if constexpr (TM) {
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                         ::"r"((uint32_t)__cvta_generic_to_shared(tslot)) : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        const uint32_t tb = *tslot + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 256);
        t_other = tb;
        t_free = tb + 128;
    }
    int cur = 0;                 // the half in registers

    uint4 acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = make_uint4(0, 0, 0, 0);

    // the half in tensor memory starts as zeros, so every pass can fetch it
    if constexpr (TM) {
#pragma unroll
        for (int j = 0; j < R / 8; ++j) tm_st32(t_other + 32 * j, *reinterpret_cast<const uint4(*)[8]>(&acc[8 * j]));
        tm_wait_st();
    }

    // Stage pass g: its KG rows of B (tile columns) and the words of each
    // tile row of A that hold columns g*KG .. g*KG+KG-1.  When KG divides 128
    // (CHUNKED_A), A is staged one aligned 16-byte chunk per row (128
    // columns = 128/KG passes) at the first pass of the previous chunk;
    // otherwise the 1-2 words of every pass are staged with the pass.
    constexpr bool CHUNKED_A = (128 % KG) == 0;
    constexpr int PPC = CHUNKED_A ? 128 / KG : 1;          // passes per A chunk
    auto issue_stage = [&](int g, int buf, bool a_chunk) {
#pragma unroll 1
        for (int i = tid; i < KG * LPR; i += NTH) {
            const int rr = i >> 3, cc = i & 7;
            const int64_t brow = (int64_t)g * KG + rr;
            const int64_t bw = w0 + 2 * cc;
            const bool valid = (brow < P.l) && (bw < nW);
            cp_async16(&stg[buf * KG * LPR + i], valid ? (B + brow * P.ldb + bw) : B, valid);
        }
        if (CHUNKED_A) {
            if (a_chunk) {
                const int c = g / PPC;                    // A chunk holding pass g
                const int64_t wa = 2 * (int64_t)c;
                const int abuf = c & 1;
#pragma unroll 1
                for (int i = tid; i < BM; i += NTH) {
                    const int64_t row = row0 + i;
                    const bool valid = (row < P.m) && (wa < lW);
                    cp_async16(&sta[abuf * BM + i], A + (valid ? row * P.lda + wa : 0), valid);
                }
            }
        } else {
            const int64_t kb = (int64_t)g * KG;
            const int64_t wa = kb >> 6;
            const bool two = ((kb & 63) + KG > 64) && (wa + 1 < lW);
#pragma unroll 1
            for (int i = tid; i < BM; i += NTH) {
                const int64_t row = row0 + i;
                const bool valid = row < P.m;
                const uint64_t *src = A + (valid ? row * P.lda + wa : 0);
                uint4 *dst = &sta[buf * BM + i];
                cp_async8(dst, src, valid);
                if (two) cp_async8(reinterpret_cast<char *>(dst) + 8, src + 1, valid);
            }
        }
        cp_async_commit();
    };

    // ReadBits + AddRowFromTable for NT tables (Algorithms 1 and 3) on the
    // rows of half h of the tile, pass g, row-groups J*RC .. J*RC+RC-1 (with
    // tall tiles a chunk is the 8 row-groups one tensor-memory access moves)
    constexpr int RC = TM ? 8 : R;
    constexpr int NCH = R / RC;
    auto lookups = [&](int g, int buf, int h, auto J) {
        constexpr int rb = decltype(J)::value * RC;
        const int64_t kb = (int64_t)g * KG;
        const int64_t wa = kb >> 6;
        const int sh = (int)(kb & 63);
        const uint64_t mlo = word_mask(wa, P.l);
        const uint64_t mhi = (sh + KG > 64) ? word_mask(wa + 1, P.l) : 0ull;
        const uint4 *arow = sta + (CHUNKED_A ? ((g / PPC) & 1) : buf) * BM + h * HM + trow;
        const int aoff = CHUNKED_A ? (int)(wa & 1) : 0;          // word inside the staged chunk
        if constexpr (CHUNKED_A && KG <= 32 && !TM) {
            // the pass's KG bits of a row lie in one 32-bit half of the
            // staged chunk: read them for every row-group first, so that
            // the lookups below do not wait on these loads
            const uint32_t *a32 = reinterpret_cast<const uint32_t *>(arow) + 2 * aoff + (sh >> 5);
            const int s32 = sh & 31;
            const uint32_t am = (uint32_t)(mlo >> (sh & 32)) >> s32;
            uint32_t ab[RC];
#pragma unroll
            for (int q = 0; q < RC; ++q) ab[q] = (a32[16 * (rb + q)] >> s32) & am;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int r = rb + q;
                uint4 a = acc[r];
#pragma unroll
                for (int ti = 0; ti < NT; ++ti) {
                    const unsigned x = (ab[q] >> (ti * KB)) & IMASK;
                    a = x4(a, tab[(ti * TROWS + (int)x) * LPR + chunk]);
                }
                acc[r] = a;
                // keeps the compiler from hoisting the loads of later
                // row-groups: t loads in flight per warp already saturate
                // shared memory
                asm volatile("" ::: "memory");
            }
        } else {
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int r = rb + q;
                const uint2 aw = reinterpret_cast<const uint2 *>(&arow[4 * r])[aoff];
                const uint64_t lo = ((uint64_t)aw.y << 32 | aw.x) & mlo;
                uint64_t bits = lo >> sh;
                if (!CHUNKED_A && sh + KG > 64) {
                    const uint2 aw2 = reinterpret_cast<const uint2 *>(&arow[4 * r])[1];
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
    };

    // the first pass stages the A chunk holding it (a K split may start
    // inside a chunk); every later chunk is staged one pass before its first
    if (g_begin < g_end) issue_stage(g_begin, 0, true);

#pragma unroll 1
    for (int g = g_begin; g < g_end; ++g) {
        const int buf = (g - g_begin) & 1;
        cp_async_wait_all();
        __syncthreads();                       // staged rows visible; previous lookups done
        if (g + 1 < g_end) {
            const bool next_chunk = CHUNKED_A && ((g + 1) % PPC) == 0;
            issue_stage(g + 1, buf ^ 1, next_chunk);
        }
        build_tables<KB, NT, NTH, LPR>(tab, stg + buf * KG * LPR, tid, cmask);
        __syncthreads();                       // tables complete
        if constexpr (TM) {
            // half cur: each chunk goes to tensor memory as soon as its
            // lookups of this pass are done, behind the next chunk's lookups
            static_for<0, NCH>([&](auto J) {
                lookups(g, buf, cur, J);
                tm_st32(t_free + 32 * decltype(J)::value,
                        *reinterpret_cast<const uint4(*)[8]>(&acc[RC * decltype(J)::value]));
            });
            tm_wait_st();
            // the other half: chunk J+1 is fetched while chunk J is looked up
            tm_ld32(t_other, *reinterpret_cast<uint4(*)[8]>(&acc[0]));
            tm_wait_ld();
            static_for<0, NCH>([&](auto J) {
                constexpr int j = decltype(J)::value;
                if constexpr (j + 1 < NCH)
                    tm_ld32(t_other + 32 * (j + 1), *reinterpret_cast<uint4(*)[8]>(&acc[RC * (j + 1)]));
                lookups(g, buf, cur ^ 1, J);
                if constexpr (j + 1 < NCH) tm_wait_ld();
            });
            const uint32_t t = t_other;
            t_other = t_free;
            t_free = t;
            cur ^= 1;
        } else {
            static_for<0, NCH>([&](auto J) { lookups(g, buf, cur, J); });
        }
    }

    // write the C rows of half h from acc: one loop per mode so that the row
    // loop stays simple
    auto write_half = [&](int h) {
        if (cw >= nW) return;
        const int64_t first = row0 + h * HM + trow;
        const int64_t left = P.m - first;               // rows of this thread: first + 4r, r < R
        const int nrows = left <= 0 ? 0 : (left < 4 * R ? (int)left : 4 * R);
        uint64_t *cr = C + first * P.ldc + cw;
        const int64_t step = 4 * P.ldc;
        if (P.mode == 0 && cw + 1 < nW) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (4 * r < nrows)
                    *reinterpret_cast<uint4 *>(cr + r * step) = and4(acc[r], cmask);
            }
        } else {
            const bool two = (cw + 1 < nW);
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                if (4 * r >= nrows) break;
                uint4 a = make_uint4(0, 0, 0, 0);
#pragma unroll
                for (int q = 0; q < R; ++q)
                    if (q == r) a = acc[q];
                const uint64_t v0 = ((uint64_t)a.y << 32 | a.x) & cm0;
                const uint64_t v1 = ((uint64_t)a.w << 32 | a.z) & cm1;
                uint64_t *c = cr + r * step;
                if (P.mode == 0) {
                    c[0] = v0;
                } else if (P.mode == 1) {
                    c[0] ^= v0;
                    if (two) c[1] ^= v1;
                } else {
                    atomicXor(reinterpret_cast<unsigned long long *>(c), (unsigned long long)v0);
                    if (two) atomicXor(reinterpret_cast<unsigned long long *>(c + 1), (unsigned long long)v1);
                }
            }
        }
    };
    write_half(cur);
    if constexpr (TM) {
        // the other half, from tensor memory (zeros if no pass ran)
#pragma unroll
        for (int j = 0; j < R / 8; ++j) tm_ld32(t_other + 32 * j, *reinterpret_cast<uint4(*)[8]>(&acc[8 * j]));
        tm_wait_ld();
        write_half(cur ^ 1);
        tm_fence_before();
        __syncthreads();
        tm_fence_after();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(*tslot) : "memory");
    }
}

// Standalone MakeTable (Algorithm 1) into global memory, using the same
// build routine as the base case: one CTA per 1024-column tile.
template <int KB>
__global__ void __launch_bounds__(256) make_table_kernel(DMat T, DMat B, int64_t r0)
{
    constexpr int NTH = 256;
    constexpr int TROWS = 1 << KB;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint4 *tab = reinterpret_cast<uint4 *>(smem_raw);
    uint4 *stg = tab + TROWS * LPR;
    const int tid = threadIdx.x;
    const int64_t w0 = (int64_t)blockIdx.x * TILE_WORDS;
    const int64_t nW = words_of(B.cols);
    for (int i = tid; i < KB * LPR; i += NTH) {
        const int rr = i >> 3, cc = i & 7;
        const int64_t brow = r0 + rr;
        const int64_t bw = w0 + 2 * cc;
        const bool valid = (brow < B.rows) && (bw < nW);
        cp_async16(&stg[i], valid ? (B.p + brow * B.ld + bw) : B.p, valid);
    }
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    const int chunk = tid & 7;
    const int64_t cw = w0 + 2 * chunk;
    const uint64_t cm0 = word_mask(cw, B.cols), cm1 = word_mask(cw + 1, B.cols);
    const uint4 cmask = make_uint4((uint32_t)cm0, (uint32_t)(cm0 >> 32), (uint32_t)cm1,
                                   (uint32_t)(cm1 >> 32));
    build_tables<KB, 1, NTH, LPR>(tab, stg, tid, cmask);
    __syncthreads();
    for (int i = tid; i < TROWS * LPR; i += NTH) {
        const int x = i >> 3, c = i & 7;
        const int64_t w = w0 + 2 * c;
        if (w >= nW) continue;
        const uint4 v = tab[i];
        uint64_t *dst = T.p + (int64_t)x * T.ld + w;
        dst[0] = ((uint64_t)v.y << 32) | v.x;
        if (w + 1 < nW) dst[1] = ((uint64_t)v.w << 32) | v.z;
    }
}

using KernelFn = void (*)(Params);

struct Variant {
    int k, t, bm, nw;     // bits per table, tables per pass, tile rows, warps per CTA
    KernelFn fn;
    int smem;
};

// Tile rows BM = 4 * R * NW (twice that with the tensor-memory half).
// Tall tiles use 8 warps holding 32 row-groups each (128 accumulator
// registers per thread, no spills).
template <int KB, int NT, int R, int NW, bool TM = false>
Variant make_variant()
{
    constexpr int BM = 4 * R * NW * (TM ? 2 : 1);
    return Variant{KB, NT, BM, NW, &m4rm_kernel<KB, NT, R, NW, TM>,
                   (int)(NT * (1 << KB) * LPR * 16 + 2 * KB * NT * LPR * 16 + 2 * BM * 16 + (TM ? 16 : 0))};
}

const Variant kVariants[] = {
    make_variant<8, 4, 32, 8, true>(),
    make_variant<8, 4, 32, 8>(), make_variant<8, 2, 32, 8>(), make_variant<7, 8, 32, 8>(),
    make_variant<6, 8, 32, 8>(), make_variant<9, 2, 32, 8>(), make_variant<10, 1, 32, 8>(),
    make_variant<5, 8, 32, 8>(), make_variant<4, 8, 32, 8>(),
    make_variant<8, 4, 16, 16>(),
    make_variant<8, 4, 4, 16>(), make_variant<6, 8, 4, 16>(), make_variant<4, 8, 4, 16>(),
    make_variant<8, 4, 1, 16>(), make_variant<6, 8, 1, 16>(), make_variant<4, 8, 1, 16>(),
};

const Variant *find_variant(int k, int t, int bm)
{
    for (const Variant &v : kVariants)
        if (v.k == k && v.t == t && v.bm == bm) return &v;
    return nullptr;
}

}  // namespace

bool m4rm_supported(int k, int t)
{
    for (const Variant &v : kVariants)
        if (v.k == k && v.t == t) return true;
    return false;
}

static int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Row-tile height and (k, t) for a shape: tall tiles (2048 rows, half of
// them in tensor memory, then 1024) amortise the 2^k-row table over many
// lookups (table cost / lookup cost = 2^k / BM, Section 3.2's trade-off);
// small problems take shorter tiles and smaller k so that every SM has
// work, and split K when even that is not enough.
void m4rm_pick(int64_t m, int64_t l, int64_t n, int batch, int *k, int *t, int *bm, int *ksplit)
{
    const int sms = sm_count();
    const int64_t tn = (words_of(n) + TILE_WORDS - 1) / TILE_WORDS;
    // Shared-memory wavefronts per bit of K of one tile (table-row reads,
    // table build, A-index and staged-B reads), counted for the default
    // (k, t) of each height: 2048 rows k=8 t=4, 1024 rows k=8 t=4, 256 rows
    // k=6 t=8, 64 rows k=4 t=8; and the CTAs of that variant one SM holds
    // (they share its shared-memory bandwidth).  The estimate is waves x
    // resident CTAs x cost: with many tiles it is tiles x cost / SMs (a
    // ragged m, 2111 rows say, is cheaper in 256-row tiles than in two
    // 2048-row ones), and with few it charges the partly empty last wave.
    // A shorter tile has to win by 5 %: the costs are estimates.
    const int bms[4] = {2048, 1024, 256, 64};
    const double cost[4] = {316.0, 180.0, 56.8, 22.5};
    const int occ[4] = {1, 1, 2, 4};
    int b = 64;
    double best = 1e300;
    for (int i = 0; i < 4; ++i) {
        if (bms[i] == 2048 && m <= 1024) continue;  // the tensor-memory half would hold no rows
        const int64_t tm = (m + bms[i] - 1) / bms[i];
        const int64_t ctas = (int64_t)batch * tn * tm;
        const int64_t slots = (int64_t)sms * occ[i];
        const double c = (double)((ctas + slots - 1) / slots) * occ[i] * cost[i];
        if (c < 0.95 * best) { best = c; b = bms[i]; }
    }
    int kk = (b >= 1024) ? 8 : (b == 256 ? 6 : 4);
    int tt = (b >= 1024) ? 4 : 8;
    if (*k > 0 || *t > 0) {
        if (*k > 0) kk = *k;
        tt = *t;
        if (tt <= 0) {
            tt = 0;
            for (const Variant &v : kVariants)
                if (v.k == kk && v.bm == 1024) { tt = v.t; break; }
        }
        // keep the requested (k, t); fall back to the tallest tile that has it
        if (!find_variant(kk, tt, b)) b = 1024;
    }
    const int64_t ctas = (int64_t)batch * tn * ((m + b - 1) / b);
    const int64_t groups = (l + kk * tt - 1) / (kk * tt);
    // split K (partial products XORed into C) only when two or more splits
    // of every tile fit in one wave
    int ks = 1;
    if (2 * ctas <= sms && groups > 1) {
        ks = (int)((sms + ctas - 1) / ctas);
        if (ks > groups) ks = (int)groups;
        if (ks > 64) ks = 64;
    }
    *k = kk; *t = tt; *bm = b; *ksplit = ks;
}

int m4rm_launch(const M4rmLaunch &L, cudaStream_t s)
{
    if (L.batch <= 0 || L.m <= 0 || L.n <= 0) return GF2_OK;
    int k = L.k, t = L.t, bm = 1024, ks_auto = 1;
    m4rm_pick(L.m, L.l, L.n, L.batch, &k, &t, &bm, &ks_auto);
    if (L.bm > 0) bm = L.bm;
    int ks = L.ksplit > 0 ? L.ksplit : ks_auto;
    const Variant *v = find_variant(k, t, bm);
    if (!v) v = find_variant(k, t, 1024);
    if (!v) return GF2_EUNSUPPORTED;
    const int KG = v->k * v->t;
    const int64_t groups = (L.l + KG - 1) / KG;
    if (groups <= 1) ks = 1;
    if (ks > groups && groups > 0) ks = (int)groups;
    const int64_t gps = groups > 0 ? (groups + ks - 1) / ks : 0;
    if (groups > 0) ks = (int)((groups + gps - 1) / gps);

    Params P;
    P.A = L.A; P.lda = L.lda; P.bsA = L.bsA;
    P.B = L.B; P.ldb = L.ldb; P.bsB = L.bsB;
    P.C = L.C; P.ldc = L.ldc; P.bsC = L.bsC;
    P.m = L.m; P.l = L.l; P.n = L.n;
    P.ksplit = ks;
    P.groups_per_split = gps;
    if (ks > 1) {
        // partial products of the K splits are XORed into C (order-free)
        if (!L.accumulate) {
            for (int b = 0; b < L.batch; ++b)
                GF2_CUDA_TRY(cudaMemset2DAsync(L.C + b * L.bsC, L.ldc * 8, 0,
                                               (size_t)words_of(L.n) * 8, (size_t)L.m, s));
        }
        P.mode = 2;
    } else {
        P.mode = L.accumulate ? 1 : 0;
    }
    dim3 grid((unsigned)div_up(words_of(L.n), TILE_WORDS), (unsigned)div_up(L.m, v->bm),
              (unsigned)(L.batch * ks));
    if (grid.y > 65535u || grid.z > 65535u) return GF2_EUNSUPPORTED;
    // the dynamic shared-memory limit is set once per variant and device
    // (bit d of the variant's mask; devices past 63 set it on every launch)
    static std::atomic<uint64_t> attr_set[sizeof(kVariants) / sizeof(kVariants[0])];
    int dev = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    std::atomic<uint64_t> &done = attr_set[v - kVariants];
    const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
    if (!bit || !(done.load(std::memory_order_acquire) & bit)) {
        GF2_CUDA_TRY(cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v->smem));
        done.fetch_or(bit, std::memory_order_acq_rel);
    }
    ProfScope ps(PF_M4RM, s);
    v->fn<<<grid, v->nw * 32, v->smem, s>>>(P);
    note_launch();
    return check_launch();
}

int make_table_launch(DMat T, DMat B, int64_t r0, int k, cudaStream_t s)
{
    using Fn = void (*)(DMat, DMat, int64_t);
    static const Fn fns[11] = {nullptr,
                               make_table_kernel<1>, make_table_kernel<2>, make_table_kernel<3>,
                               make_table_kernel<4>, make_table_kernel<5>, make_table_kernel<6>,
                               make_table_kernel<7>, make_table_kernel<8>, make_table_kernel<9>,
                               make_table_kernel<10>};
    if (k < 1 || k > 10) return GF2_EINVAL;
    if (B.cols <= 0) return GF2_OK;
    const int smem = (1 << k) * LPR * 16 + k * LPR * 16;
    GF2_CUDA_TRY(cudaFuncSetAttribute(fns[k], cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    dim3 grid((unsigned)div_up(words_of(B.cols), TILE_WORDS));
    ProfScope ps(PF_TABLE, s);
    fns[k]<<<grid, 256, smem, s>>>(T, B, r0);
    note_launch();
    return check_launch();
}

}  // namespace gf2
