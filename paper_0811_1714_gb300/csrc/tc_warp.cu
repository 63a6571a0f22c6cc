// tc_warp.cu -- the warp-level tensor-core base cases (mma.sync, sm_103a):
// C = A B over GF(2) from 0/1 int8 products (int32 sums), or from the packed
// words themselves (1-bit AND + popcount, int32 sums).
//
// Section 2.3: a GF(2) dot product is the parity of the integer dot product
// of the 0/1 vectors; with B transposed it is the parity of popcount(a AND
// b) over the packed words of a row of A and a row of B^T.
//  * int8 form: every bit becomes the int8 value 0 or 1 and
//    mma.sync.m16n8k32.s8.s8.s32 sums the products exactly in int32;
//  * binary form: mma.sync.m16n8k256.b1.b1.s32.and.popc sums popcounts of
//    ANDed 32-bit words, 256 entries of K per instruction, also in int32.
//    A register of its fragments holds 32 consecutive entries of K, which
//    is exactly a packed half-word, so the operands need no unpacking.
// Either way a sum is at most K < 2^31, so the parity of each accumulator
// is the entry of C and no K-chunking is needed.  tcgen05 has no int8 or
// binary kind on sm_103a, so these forms use the warp-level instructions;
// they exist for the comparison with the FP8 tcgen05 form and are never
// chosen automatically (that form and the packed M4RM base case are many
// times faster on this part).
//
// One CTA (8 warps) owns a 128 x 128 tile of C; warp (wm, wn) owns rows
// 64 wm .. +63 and columns 32 wn .. +31 as 4 x 4 m16n8 accumulators.  Per
// 256-entry K block, cp.async stages the packed words of the tile's 128 rows
// of A and 128 rows of B^T (32 bytes each, rows padded to 48 bytes so that
// the fragment loads of 8 rows hit 8 different banks).  The int8 form
// expands each thread's fragment bits straight into registers (4 bits -> 4
// int8 ones by one multiply and one mask) for eight 32-entry steps; the
// binary form loads the fragment words as they are for one 256-entry step.
#include "common.cuh"

#include <mutex>

namespace gf2 {
namespace {

constexpr int TM = 128, TN = 128;       // tile rows of A / rows of B^T
constexpr int KBW = 4;                  // packed words per row per K block (256 entries)
constexpr int ROWB = 48;                // bytes per staged row (32 used)
constexpr int ROWW = ROWB / 4;          // 32-bit words per staged row
constexpr int STAGE = (TM + TN) * ROWB; // bytes per stage
constexpr int NTHR = 256;

struct WarpParams {
    const uint64_t *A; int64_t lda, bsA;
    const uint64_t *Bt; int64_t ldb, bsB;
    uint64_t *C; int64_t ldc, bsC;
    int64_t m, l, n;
    int accumulate;
};

__device__ __forceinline__ void cp16(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}

// 4 bits -> 4 bytes of value 0/1 (bit b to bit 8b): the copies of the
// nibble at shifts 0, 7, 14, 21 do not overlap, so no carries.
__device__ __forceinline__ uint32_t ones4(uint32_t x) { return ((x & 0xFu) * 0x00204081u) & 0x01010101u; }

// The bits of K entries k0 .. k0+31 that lie below l.
__device__ __forceinline__ uint32_t k_mask(int64_t l, int64_t k0)
{
    return (l - k0 >= 32) ? 0xFFFFFFFFu : (l > k0 ? (1u << (l - k0)) - 1u : 0u);
}

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 "
                 "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_b1(int (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile("mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc "
                 "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
                 : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool BIN>
__global__ void __launch_bounds__(NTHR) tc_warp_kernel(WarpParams P)
{
    __shared__ __align__(16) unsigned char sm[2 * STAGE];
    __shared__ unsigned char par[TM][TN + 4];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int g = lane >> 2, tig = lane & 3;
    const int bz = blockIdx.z;
    const uint64_t *A = P.A + (int64_t)bz * P.bsA;
    const uint64_t *Bt = P.Bt + (int64_t)bz * P.bsB;
    uint64_t *C = P.C + (int64_t)bz * P.bsC;
    const int64_t row0 = (int64_t)blockIdx.y * TM, col0 = (int64_t)blockIdx.x * TN;
    const int64_t lW = words_of(P.l);
    const int nkb = (int)((P.l + 255) / 256);

    // stage K block kb: thread tid copies 16 bytes of row tid / 2 (A rows
    // 0..127 then B^T rows 0..127), half tid % 2
    auto stage = [&](int kb, int buf) {
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
            const int idx = tid + rep * NTHR;            // 0..511
            const int r = idx >> 1, h = idx & 1;
            const int64_t w = (int64_t)kb * KBW + 2 * h;
            unsigned char *dst = sm + buf * STAGE + r * ROWB + h * 16;
            if (r < TM) {
                const int64_t gr = row0 + r;
                const bool ok = gr < P.m && w < lW;
                cp16(dst, ok ? (const void *)(A + gr * P.lda + w) : (const void *)A, ok);
            } else {
                const int64_t gr = col0 + (r - TM);
                const bool ok = gr < P.n && w < lW;
                cp16(dst, ok ? (const void *)(Bt + gr * P.ldb + w) : (const void *)Bt, ok);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    int acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0;

    // Entries beyond K: A's last word is masked; B^T's are zero there (the
    // transpose clears them, words beyond K are staged as zeros) or meet
    // A's zeros.
    if (nkb > 0) stage(0, 0);
    for (int kb = 0; kb < nkb; ++kb) {
        const int buf = kb & 1;
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        if (kb + 1 < nkb) stage(kb + 1, buf ^ 1);
        const uint32_t *sa = reinterpret_cast<const uint32_t *>(sm + buf * STAGE);
        const uint32_t *sb = reinterpret_cast<const uint32_t *>(sm + buf * STAGE + TM * ROWB);
        const int64_t kb0 = (int64_t)kb * 256;
        if constexpr (BIN) {
            // fragment words: A rows g and g+8 of each 16-row block, B^T
            // row g of each 8-row block; words tig and 4+tig of the block
            // (K entries 32 tig .. +31 and 128 + 32 tig .. +31)
            const uint32_t m0 = k_mask(P.l, kb0 + 32 * tig), m1 = k_mask(P.l, kb0 + 128 + 32 * tig);
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int r = wm * 64 + 16 * i + g;
                af[i][0] = sa[r * ROWW + tig] & m0;
                af[i][1] = sa[(r + 8) * ROWW + tig] & m0;
                af[i][2] = sa[r * ROWW + 4 + tig] & m1;
                af[i][3] = sa[(r + 8) * ROWW + 4 + tig] & m1;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = wn * 32 + 8 * j + g;
                bf[j][0] = sb[r * ROWW + tig];
                bf[j][1] = sb[r * ROWW + 4 + tig];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_b1(acc[i][j], af[i], bf[j]);
        } else {
#pragma unroll 2
            for (int kk = 0; kk < 8; ++kk) {            // 32-entry steps: 32-bit word kk of the block
                const uint32_t km = k_mask(P.l, kb0 + 32 * kk);
                uint32_t af[4][4], bf[4][2];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int r = wm * 64 + 16 * i + g;
                    const uint32_t x0 = sa[r * ROWW + kk] & km;
                    const uint32_t x1 = sa[(r + 8) * ROWW + kk] & km;
                    af[i][0] = ones4(x0 >> (4 * tig));
                    af[i][1] = ones4(x1 >> (4 * tig));
                    af[i][2] = ones4(x0 >> (16 + 4 * tig));
                    af[i][3] = ones4(x1 >> (16 + 4 * tig));
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = wn * 32 + 8 * j + g;
                    const uint32_t y = sb[r * ROWW + kk];
                    bf[j][0] = ones4(y >> (4 * tig));
                    bf[j][1] = ones4(y >> (16 + 4 * tig));
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) mma_s8(acc[i][j], af[i], bf[j]);
            }
        }
    }

    // parities: accumulator (i, j) holds rows g, g+8 and columns 2 tig, 2 tig+1
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = wm * 64 + 16 * i + g, c = wn * 32 + 8 * j + 2 * tig;
            par[r][c] = (unsigned char)(acc[i][j][0] & 1);
            par[r][c + 1] = (unsigned char)(acc[i][j][1] & 1);
            par[r + 8][c] = (unsigned char)(acc[i][j][2] & 1);
            par[r + 8][c + 1] = (unsigned char)(acc[i][j][3] & 1);
        }
    __syncthreads();
    // thread tid packs word tid % 2 of tile row tid / 2
    {
        const int r = tid >> 1, h = tid & 1;
        const int64_t gr = row0 + r;
        const int64_t wcol = col0 / 64 + h;
        if (gr < P.m && wcol < words_of(P.n)) {
            uint64_t v = 0;
#pragma unroll 8
            for (int b = 0; b < 64; ++b) v |= (uint64_t)par[r][64 * h + b] << b;
            v &= word_mask(wcol, P.n);
            uint64_t *dst = C + gr * P.ldc + wcol;
            *dst = P.accumulate ? (*dst ^ v) : v;
        }
    }
}

template <bool BIN>
int tc_warp_launch(const TcLaunch &L, cudaStream_t s)
{
    if (L.batch <= 0 || L.m <= 0 || L.n <= 0) return GF2_OK;
    if ((L.lda & 1) || (L.ldb & 1) || (reinterpret_cast<uintptr_t>(L.A) & 15) ||
        (reinterpret_cast<uintptr_t>(L.Bt) & 15) || (L.batch > 1 && ((L.bsA & 1) || (L.bsB & 1))))
        return GF2_ELAYOUT;
    WarpParams P;
    P.A = L.A; P.lda = L.lda; P.bsA = L.bsA;
    P.Bt = L.Bt; P.ldb = L.ldb; P.bsB = L.bsB;
    P.C = L.C; P.ldc = L.ldc; P.bsC = L.bsC;
    P.m = L.m; P.l = L.l; P.n = L.n;
    P.accumulate = L.accumulate;
    const int64_t gx = div_up(L.n, TN), gy = div_up(L.m, TM);
    if (gx > 0x7FFFFFFF || gy > 65535 || L.batch > 65535) return GF2_EUNSUPPORTED;
    ProfScope ps(BIN ? PF_TC_B1 : PF_TC_S8, s);
    tc_warp_kernel<BIN><<<dim3((unsigned)gx, (unsigned)gy, (unsigned)L.batch), NTHR, 0, s>>>(P);
    note_launch();
    return check_launch();
}

}  // namespace

int tc_s8_launch(const TcLaunch &L, cudaStream_t s) { return tc_warp_launch<false>(L, s); }
int tc_b1_launch(const TcLaunch &L, cudaStream_t s) { return tc_warp_launch<true>(L, s); }

}  // namespace gf2
