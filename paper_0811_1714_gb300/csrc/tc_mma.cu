// tc_mma.cu -- exact tensor-core base case on operands expanded once in HBM:
// C = A B over GF(2) from 0/1 products on the 5th-generation tensor cores
// (tcgen05, sm_103a), in two number formats:
//   KIND_F8: FP8 E4M3, a 1-bit is the byte 0x38 (1.0), kind::f8f6f4;
//   KIND_F4: FP4 E2M1, a 1-bit is the nibble 0x2 (1.0), two entries per
//            byte, kind::mxf4 with block scale factors that are all 1.0
//            (UE8M0 127), so every block product is the plain product.
//
// Why it is exact (Section 2.3): a GF(2) dot product is an AND followed by an
// XOR accumulation, i.e. the parity of the INTEGER dot product of the 0/1
// vectors.  Each product of two entries is 0 or 1.0, and a K-chunk of at most
// 4096 (FP8) or 8192 (FP4) entries sums to an integer count <= 2^12 (2^13),
// which any accumulator keeping 12 (13) or more significant bits holds
// exactly, whatever the order of the additions (FP32 keeps 24).  After each
// chunk the accumulator D is read from tensor memory; the parity of count is
// the last mantissa bit of D + 2^23 (whose ulp is 1), and the parities of
// successive chunks are XORed: the GF(2) sum over all of K.
//
// Kernels:
//  - expand_kernel<KIND>: the packed operand rows (Section 2.1 layout, a
//    batch of equal matrices) become rows of FP8 bytes or FP4 nibbles, padded
//    with zeros to a whole number of 128-byte rows of K (128 FP8 or 256 FP4
//    entries).  HBM-bound: it reads each packed word once and writes 8 (FP8)
//    or 4 (FP4) times its bytes, in coalesced 512-byte warp stores.  B is
//    transposed (packed) first, so its rows are B's columns.
//  - tc_mma_kernel<KIND, PAIR, TN>: persistent, one CTA of 10 warps per SM.
//    Warp 0 issues TMA tensor copies of 128-byte K blocks of the expanded A
//    and B^T into a ring of stages in the 128-byte swizzled K-major layout the
//    MMA reads; warp 1 owns the tensor memory and one of its threads issues
//    tcgen05.mma (K = 32 FP8 / 64 FP4 entries per instruction, A and B both
//    from shared memory) into FP32 accumulators in tensor memory; warps 2-9
//    (two per tensor-memory lane quarter, one per column half) read an
//    accumulator with tcgen05.ld, hand it back at once, and turn their FP32
//    values into parity words of C in registers.  No bit expansion competes
//    with the tensor core.  PAIR = 1: clusters of two CTAs over 256 x 256
//    tiles with one tcgen05.mma.cta_group::2 stream (M = 256), two K blocks
//    per stage; PAIR = 0: one CTA per 128 x TN tile.  Accumulators are
//    double-buffered (the MMAs of the next tile run while the epilogue reads
//    the last one) except on single-CTA FP4 256-column tiles: FP8 pairs take
//    256-column tiles (accumulators at columns 0 and 256 of tensor memory),
//    FP4 pairs 224-column tiles (accumulators at 0 and 256, the scale factors
//    in the 32 columns after each), whose ends fall on 32-bit boundaries of
//    C's words.
//  - the batched form (many products of uneven shapes): expand_batched_kernel
//    (A rows) and expand_t_batched_kernel (B^T rows straight from packed B,
//    transposed by ballots in shared-memory-staged 64 x 512-entry units), then
//    one tc_mma_kernel launch over a list of (product, tile row, tile column)
//    whose tensor maps live in device memory, each CTA taking runs of one
//    product's tiles (longest first, least loaded CTA), all as a CUDA graph.
// Hand-offs use mbarriers: full (TMA transaction bytes) / empty (one
// tcgen05.commit per stage) per stage, accumulator full (commit) / empty
// (epilogue arrivals).  Every wait is bounded: an expired wait records
// GF2_ETIMEOUT in the device status word and the CTA winds down (waits for its
// copies and MMAs in flight, frees its tensor memory) instead of hanging.
#include "common.cuh"
#include "tcgen05.cuh"
#include "expand.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

namespace gf2 {
namespace {

using namespace gf2::tc;

constexpr int BM = 128;                       // rows of a tile per CTA (MMA M per CTA)
constexpr int BN = 256;                       // tile columns (MMA N) of single products
constexpr int ROWB = 128;                     // bytes of K per operand row per stage
constexpr int A_BYTES = BM * ROWB;            // 16 KB
constexpr int TMA_WARP = 0, MMA_WARP = 1, EPI_WARP0 = 2, NUM_EPI_WARPS = 8;
constexpr int NTHREADS = (EPI_WARP0 + NUM_EPI_WARPS) * 32;    // 320
constexpr uint32_t TMEM_COLS = 512;
constexpr int PTN_F4 = 224;                   // tile columns of the FP4 pairs (two accumulators)

// Tensor-memory columns of a tile width: accumulator b at b * ACC, FP4 scale
// factors (32 columns each, every byte 1.0) at SFA and SFB.  256-column tiles
// hold one FP4 accumulator (scale factors at 256 and 320); 224-column tiles
// two (at 0 and 256, scale factors in the 32 columns after each); 128-column
// tiles two (at 0 and 128).
template <int TN> struct Cols {
    static constexpr uint32_t ACC = TN == 224 ? 256 : TN;
    static constexpr uint32_t SFA = TN == 224 ? 224 : 256;
    static constexpr uint32_t SFB = TN == 224 ? 480 : 320;
};

// Per-CTA stage and ring: KBS 128-byte K blocks per stage; per block one CTA
// holds its A tile and the whole B^T tile (48 KB), each CTA of a pair its A
// tile and one half of the pair's B^T tile (32 KB).  The ring takes what fits
// beside the barriers in 227 KB.
template <int PAIR, int KBS, int TN = BN> struct Ring {
    static constexpr int A_SUB = A_BYTES;                                  // one K block of A
    static constexpr int B_SUB = (PAIR ? TN / 2 : TN) * ROWB;              // one K block of B^T
    static constexpr int STAGE_BYTES = KBS * (A_SUB + B_SUB);
    static constexpr int STAGES = (232448 - 1024 - 256) / STAGE_BYTES > 8 ? 8 : (232448 - 1024 - 256) / STAGE_BYTES;
    static constexpr int NBARS = 2 * STAGES + 4 + 1;
    static constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + NBARS * 8 + 16;
    static_assert(STAGES >= 2 && SMEM_BYTES <= 232448, "shared memory per CTA");
};
constexpr int KBS_PAIR = 2, KBS_ONE = 1;      // K blocks per stage

template <int KIND> struct Fmt;
template <> struct Fmt<KIND_F8> {
    static constexpr int EPR = 128;           // entries per 128-byte row
    static constexpr int nacc(int) { return 2; }   // accumulators in tensor memory
    static constexpr int KCHUNK = 4096;       // entries per exact accumulation (sums <= 2^12)
    // D = F32 (bits 4-5 = 1), A = B = E4M3 (bits 7-9, 10-12 = 0), both
    // K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
    static constexpr uint32_t idesc(int M, int N) { return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24); }
};
template <> struct Fmt<KIND_F4> {
    static constexpr int EPR = 256;
    // with the scale factors beside them, 256-column tiles have room for one
    // accumulator, 224- and 128-column tiles for two
    static constexpr int nacc(int TN) { return TN == 256 ? 1 : 2; }
    // chunks of 8192 entries (sums <= 2^13, exact with 13 significant bits):
    // one accumulator hand-off per tile of a depth-2 leaf of n = 32768
    static constexpr int KCHUNK = 8192;
    // block-scaled descriptor: scale-factor ids 0 (bits 4-5, 29-30), A = B =
    // E2M1 (code 1 at bits 7-9 and 10-12), both K-major, N >> 3 at bits
    // 17-22, scale type UE8M0 (bit 23 = 1), M >> 4 at bits 24-28
    static constexpr uint32_t idesc(int M, int N)
    {
        return (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (1u << 23) | ((uint32_t)(M >> 4) << 24);
    }
};

// One product of a batch of uneven shapes: tensor maps of its expanded A and
// B^T (built on the host, kept in device memory) and its output.
struct alignas(128) TcxProd {
    CUtensorMap mapA;
    CUtensorMap mapB;
    uint64_t *C;
    int64_t ldc, m, n, nkb;
};

struct Params {
    int64_t m, n;            // rows of A (and of C), rows of B^T (columns of C) per product
    int64_t nkb;             // 128-byte K blocks per row
    int tiles_m, tiles_n;    // tile rows of 128 (one CTA) or 256 (a pair) rows, tile columns of TN
    int batch;
    uint64_t *C;
    int64_t ldc, bsC;
    int accumulate;
    unsigned int *status;
    // products of uneven shapes (null for a uniform batch; one CTA per tile):
    // tile t is tlist[t] = (product, tile row, tile column); CTA c takes tiles
    // cstart[c] .. cstart[c + 1] - 1 (runs of tiles of one product)
    const TcxProd *prods;
    const int4 *tlist;
    const int *cstart;
    int64_t ntiles;
};

// One tile: its operands' maps, coordinates, extent and output.
struct Tile {
    const CUtensorMap *ma, *mb;
    int z, tm, tn;
    int64_t m, n, nkb;
    uint64_t *C;
    int64_t ldc;
};

// One MMA step of 32 bytes of K: M = 128 (one CTA, cta_group::1) or M = 256
// over the pair (cta_group::2, issued by the pair's first CTA; A rows 0-127
// and B^T rows 0-127 from its shared memory, rows 128-255 from its peer's,
// each CTA's accumulator rows in its own tensor memory).
template <int KIND, int PAIR, int TN>
__device__ __forceinline__ void mma_issue(uint32_t d, uint64_t ad, uint64_t bd, uint32_t sfa, uint32_t sfb, uint32_t acc)
{
    constexpr uint32_t ID = Fmt<KIND>::idesc(PAIR ? 2 * BM : BM, TN);
    if (KIND == KIND_F8) {
        if (PAIR)
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(d), "l"(ad), "l"(bd), "r"(ID), "r"(acc) : "memory");
        else
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                         ::"r"(d), "l"(ad), "l"(bd), "r"(ID), "r"(acc) : "memory");
    } else {
        if (PAIR)
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
                         "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}"
                         ::"r"(d), "l"(ad), "l"(bd), "r"(ID), "r"(sfa), "r"(sfb), "r"(acc)
                         : "memory");
        else
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}"
                         ::"r"(d), "l"(ad), "l"(bd), "r"(ID), "r"(sfa), "r"(sfb), "r"(acc)
                         : "memory");
    }
}

// Arrival on `bar` once this thread's MMAs so far have completed: on this
// CTA's barrier (one CTA), or on the barrier at that offset in both CTAs of
// the pair (ctaMask 3) or in the first one only (ctaMask 1).
template <int PAIR>
__device__ __forceinline__ void commit(uint32_t bar, unsigned short mask)
{
    if (PAIR)
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                     ::"r"(bar), "h"(mask) : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The shared::cluster address of `addr` (a shared::cta address) in the
// cluster's CTA `rank`.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void arrive_cluster(uint32_t cluster_bar)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// TMA copy into this CTA's shared memory that completes on a barrier of
// either CTA of the pair (its shared::cluster address).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                                 uint32_t cluster_bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(cluster_bar)
        : "memory");
}

// Tile t of a uniform batch: leaf b, then bands of GM tile rows, each band
// walked column by column (GM tiles of one column, then the next), so that
// the tiles the CTAs run at one time share a few row blocks of A and column
// blocks of B^T in L2 (a band of 8 x ~10 tiles for 76 pairs) instead of
// streaming all of B^T once per row block when a leaf exceeds the L2.
constexpr int GM = 8;

__device__ __forceinline__ void tile_coords(const Params &P, int64_t t, int &b, int &tm, int &tn)
{
    const int64_t per = (int64_t)P.tiles_m * P.tiles_n;
    int64_t r;
    if (per * P.batch <= 0x7FFFFFFF) {
        // 32-bit divisions (the 64-bit ones are long subroutines)
        const uint32_t tt = (uint32_t)t, pp = (uint32_t)per;
        b = (int)(tt / pp);
        r = (int64_t)(tt - (uint32_t)b * pp);
    } else {
        b = (int)(t / per);
        r = t - (int64_t)b * per;
    }
    const uint32_t band_tiles = (uint32_t)GM * (uint32_t)P.tiles_n;
    const uint32_t band = (uint32_t)r / band_tiles;
    const uint32_t in = (uint32_t)r - band * band_tiles;
    const uint32_t left = (uint32_t)P.tiles_m - band * GM;
    const uint32_t rows = left < (uint32_t)GM ? left : (uint32_t)GM;      // tile rows of this band
    const uint32_t col = in / rows;
    tm = (int)(band * GM + (in - col * rows));
    tn = (int)col;
}

__device__ __forceinline__ Tile get_tile(const Params &P, const CUtensorMap *ma, const CUtensorMap *mb, int64_t t)
{
    Tile T;
    if (!P.prods) {
        int b, tm, tn;
        tile_coords(P, t, b, tm, tn);
        T.ma = ma; T.mb = mb; T.z = b; T.tm = tm; T.tn = tn;
        T.m = P.m; T.n = P.n; T.nkb = P.nkb;
        T.C = P.C + (int64_t)b * P.bsC;
        T.ldc = P.ldc;
    } else {
        const int4 e = P.tlist[t];
        const TcxProd &pr = P.prods[e.x];
        T.ma = &pr.mapA; T.mb = &pr.mapB; T.z = 0; T.tm = e.y; T.tn = e.z;
        T.m = pr.m; T.n = pr.n; T.nkb = pr.nkb;
        T.C = pr.C;
        T.ldc = pr.ldc;
    }
    return T;
}

template <int PAIR>
__device__ __forceinline__ void alloc_tmem(uint32_t slot)
{
    if (PAIR) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
        tmem_alloc(slot, TMEM_COLS);
    }
}

template <int PAIR>
__device__ __forceinline__ void free_tmem(uint32_t taddr)
{
    if (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
    else
        tmem_dealloc(taddr, TMEM_COLS);
}

// PAIR = 0: one CTA per 128 x 256 tile.  PAIR = 1: clusters of two CTAs per
// 256 x 256 tile, one tcgen05.mma.cta_group::2 stream issued by the first
// CTA; each CTA copies its 128 rows of A and its 128-row half of B^T into its
// own shared memory, the copies of both complete on the first CTA's stage
// barrier, the MMA commits release the stage in both CTAs, and both CTAs'
// epilogues arrive on the first CTA's accumulator-empty barrier.
template <int KIND, int PAIR, int TN>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_mma_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Params P)
{
    static_assert(TN == 256 || (TN == 224 && PAIR) || (TN == 128 && !PAIR),
                  "tile widths: 256, 224 on pairs, 128 on one CTA");
    constexpr int KBS = PAIR ? KBS_PAIR : KBS_ONE;
    using R = Ring<PAIR, KBS, TN>;
    constexpr int NACC = Fmt<KIND>::nacc(TN);
    constexpr int G = TN / 32;                  // 32-column groups of a tile
    constexpr int GH = (G + 1) / 2;             // groups of the first epilogue column half
    constexpr int SPC = Fmt<KIND>::KCHUNK / Fmt<KIND>::EPR / KBS;   // stages per K-chunk
    constexpr int STAGES = R::STAGES;
    constexpr int STAGE_BYTES = R::STAGE_BYTES;
    constexpr int TILE_ROWS = PAIR ? 2 * BM : BM;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // stages sit on 1024-byte boundaries (128-byte swizzle atoms)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sbase = smem_raw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sbase + STAGES * STAGE_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + R::NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = PAIR ? cluster_rank() : 0u;      // 0: the CTA that issues the MMAs
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * s; };
    auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
    const uint32_t done_bar = bar0 + 8u * (2 * STAGES + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);            // the issuing CTA's expect_tx arrival
            mbar_init(empty_bar(s), 1);           // tcgen05.commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), NUM_EPI_WARPS * (PAIR ? 2 : 1));   // every epilogue warp of the pair
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) alloc_tmem<PAIR>(smem_u32(tmem_slot));
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if (KIND == KIND_F4 && warp >= EPI_WARP0 && warp < EPI_WARP0 + 4) {
        // every scale factor 1.0 (UE8M0 127): whatever bytes of these columns
        // the MMA reads for A and for B, each block product is unscaled
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        tmem_fill32(tmem_base + lanes + Cols<TN>::SFA, 0x7F7F7F7Fu);
        tmem_fill32(tmem_base + lanes + Cols<TN>::SFB, 0x7F7F7F7Fu);
        tmem_wait_st();
    }
    fence_before();
    __syncthreads();
    // the peer's copies, commits and arrivals target this CTA's barriers and
    // tensor memory: both CTAs are set up before either issues anything
    if (PAIR) cluster_sync();
    fence_after();
    int64_t tiles, t0, tstep;
    if (P.prods) {
        t0 = P.cstart[blockIdx.x];
        tiles = P.cstart[blockIdx.x + 1];
        tstep = 1;
    } else {
        tiles = (int64_t)P.tiles_m * P.tiles_n * P.batch;
        t0 = PAIR ? blockIdx.x / 2 : blockIdx.x;
        tstep = PAIR ? gridDim.x / 2 : gridDim.x;
    }
    // stages per tile: ceil(K blocks / KBS) (a last partial stage copies K
    // blocks beyond the row, which arrive as zeros)

    // every role walks its tiles t = t0, t0 + tstep, ...
    if (warp == TMA_WARP) {
        // ------------------------------------------------------------ TMA issuer
        if (lane == 0) {
            if (!P.prods) {
                asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB) : "memory");
            }
            int64_t q = 0;
            bool ok = true;
            const CUtensorMap *last = nullptr;
            for (int64_t t = t0; t < tiles && ok; t += tstep) {
                const Tile T = get_tile(P, &mapA, &mapB, t);
                if (P.prods && T.ma != last) {
                    // maps written by the host into device memory: acquire them
                    // for the tensor-copy proxy before their first use here
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(T.ma) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(T.mb) : "memory");
                    last = T.ma;
                }
                const int b = T.z, tm = T.tm, tn = T.tn;
                const int64_t nst = (T.nkb + KBS - 1) / KBS;
                for (int64_t ks = 0; ks < nst; ++ks, ++q) {
                    const int s = (int)(q % STAGES);
                    if (!mbar_wait(empty_bar(s), (uint32_t)((q / STAGES) & 1) ^ 1u, P.status, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst = base + s * STAGE_BYTES;
                    if (PAIR) {
                        // both CTAs' copies complete on the first CTA's barrier
                        const uint32_t fb = cluster_addr(full_bar(s), 0);
                        if (rank == 0) mbar_arrive_expect_tx(full_bar(s), 2 * STAGE_BYTES);
#pragma unroll
                        for (int j = 0; j < KBS; ++j) {
                            const int x = (int)((ks * KBS + j) * ROWB);
                            tma_load_3d_pair(dst + j * R::A_SUB, T.ma, x, tm * TILE_ROWS + (int)rank * BM, b, fb);
                            tma_load_3d_pair(dst + KBS * R::A_SUB + j * R::B_SUB, T.mb, x,
                                             tn * TN + (int)rank * (TN / 2), b, fb);
                        }
                    } else {
                        mbar_arrive_expect_tx(full_bar(s), STAGE_BYTES);
#pragma unroll
                        for (int j = 0; j < KBS; ++j) {
                            const int x = (int)((ks * KBS + j) * ROWB);
                            const uint32_t db = dst + KBS * R::A_SUB + j * R::B_SUB;
                            tma_load_3d(dst + j * R::A_SUB, T.ma, x, tm * BM, b, full_bar(s));
                            tma_load_3d(db, T.mb, x, tn * TN, b, full_bar(s));     // B^T rows in boxes of 128
                            if (TN == 256) tma_load_3d(db + 128 * ROWB, T.mb, x, tn * TN + 128, b, full_bar(s));
                        }
                    }
                }
            }
            // wind down: copies issued but not consumed (only after an abort)
            // still land in shared memory; wait for them before the CTA exits
            // (the issuing CTA's barriers see both CTAs' copies)
            if (rank == 0)
                for (int64_t r = (q > STAGES ? q - STAGES : 0); r < q; ++r)
                    mbar_drain(full_bar((int)(r % STAGES)), (uint32_t)((r / STAGES) & 1), P.status);
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0 && rank == 0) {
            uint32_t u = 0;                              // accumulator uses
            int s = 0;                                   // ring stage and its phase bit
            uint32_t ph = 0;
            bool ok = true;
            const uint32_t sfa = tmem_base + Cols<TN>::SFA, sfb = tmem_base + Cols<TN>::SFB;
            const uint64_t da_first = smem_desc_sw128(base);
            uint64_t da = da_first, db = da_first + (uint64_t)((KBS * R::A_SUB) >> 4);
            for (int64_t t = t0; t < tiles && ok; t += tstep) {
                const Tile T = get_tile(P, &mapA, &mapB, t);
                const int64_t nst = (T.nkb + KBS - 1) / KBS;
                const int nchunks = (int)((nst + SPC - 1) / SPC);
                for (int c = 0; c < nchunks && ok; ++c, ++u) {
                    const int ab = (int)(u % NACC);
                    if (!mbar_wait(tempty_bar(ab), ((u / NACC) & 1u) ^ 1u, P.status, abort_flag)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t dt = tmem_base + (uint32_t)ab * Cols<TN>::ACC;
                    const int64_t ks0 = (int64_t)c * SPC;
                    const int64_t ks1 = std::min<int64_t>(nst, ks0 + SPC);
                    for (int64_t ks = ks0; ks < ks1; ++ks) {
                        // the MMA pipe idles while this thread does anything but
                        // issue MMAs: between stages, a non-blocking test first
                        if (!mbar_test_wait(full_bar(s), ph) && !mbar_wait(full_bar(s), ph, P.status, abort_flag)) {
                            ok = false;
                            break;
                        }
                        fence_after();
                        const uint32_t acc0 = ks > ks0 ? 1u : 0u;
#pragma unroll
                        for (int j = 0; j < KBS; ++j)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)  // 32 bytes of K per instruction
                                mma_issue<KIND, PAIR, TN>(dt, da + (uint64_t)((j * R::A_SUB + kk * 32) >> 4),
                                                          db + (uint64_t)((j * R::B_SUB + kk * 32) >> 4), sfa, sfb,
                                                          (j > 0 || kk > 0) ? 1u : acc0);
                        commit<PAIR>(empty_bar(s), 3);     // stage free (in both CTAs) once these MMAs read it
                        // descriptors of the next stage's first K block (the others are
                        // constant offsets: start address >> 4 in the low bits)
                        if (++s == STAGES) {
                            s = 0;
                            ph ^= 1u;
                            da = da_first;
                        } else {
                            da += (uint64_t)(STAGE_BYTES >> 4);
                        }
                        db = da + (uint64_t)((KBS * R::A_SUB) >> 4);
                    }
                    if (!ok) break;
                    commit<PAIR>(tfull_bar(ab), 3);        // accumulator ready for the epilogue(s)
                }
            }
            // wind down: wait until every issued MMA has completed
            commit<PAIR>(done_bar, 1);
            mbar_drain(done_bar, 0, P.status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;                   // TMEM lanes 32*quarter.. = tile rows
        const int half = (warp - EPI_WARP0) >> 2;       // column groups GH * half ..
        const int ng = half == 0 ? GH : G - GH;         // this warp's 32-column groups
        const int row_in_tile = (int)rank * BM + quarter * 32 + lane;
        uint32_t u = 0;
        for (int64_t t = t0; t < tiles && !warp_aborted(abort_flag); t += tstep) {
            const Tile T = get_tile(P, &mapA, &mapB, t);
            const int tm = T.tm, tn = T.tn;
            const int64_t nst = (T.nkb + KBS - 1) / KBS;
            const int nchunks = (int)((nst + SPC - 1) / SPC);
            const int64_t nW = words_of(T.n);
            uint32_t par[GH];
#pragma unroll
            for (int g = 0; g < GH; ++g) par[g] = 0u;
            bool ok = true;
            for (int c = 0; c < nchunks; ++c, ++u) {
                const int ab = (int)(u % NACC);
                if (!warp_wait(tfull_bar(ab), (u / NACC) & 1u, P.status, abort_flag)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                       (uint32_t)ab * Cols<TN>::ACC + (uint32_t)(half * GH * 32);
                uint32_t r[32 * GH];
#pragma unroll
                for (int g = 0; g < GH; ++g)
                    if (g < ng) tmem_ld32(taddr + 32 * g, r + 32 * g);
                tmem_wait_ld();
                // the accumulator is in registers: hand it back to the MMA
                fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (PAIR) arrive_cluster(cluster_addr(tempty_bar(ab), 0));
                    else mbar_arrive(tempty_bar(ab));
                }
#pragma unroll
                for (int g = 0; g < GH; ++g) {
                    if (g >= ng) break;
                    uint32_t word = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        // D = count <= 2^13, an integer: the ulp of D + 2^23 is 1
                        const uint32_t f = __float_as_uint(__uint_as_float(r[32 * g + j]) + 8388608.0f);
                        word |= (f & 1u) << j;
                    }
                    par[g] ^= word;
                }
            }
            if (!ok) break;
            const int64_t grow = (int64_t)tm * TILE_ROWS + row_in_tile;
            if (grow < T.m) {
                uint64_t *C = T.C + grow * T.ldc;
                if constexpr (TN % 64 == 0 && GH % 2 == 0) {
                    // whole 64-bit words of C per column half
#pragma unroll
                    for (int i = 0; i < GH / 2; ++i) {
                        const int64_t wcol = (int64_t)tn * (TN / 64) + half * (GH / 2) + i;
                        if (wcol < nW) {
                            const uint64_t v = (((uint64_t)par[2 * i + 1] << 32) | par[2 * i]) & word_mask(wcol, T.n);
                            C[wcol] = P.accumulate ? (C[wcol] ^ v) : v;
                        }
                    }
                } else {
                    // 224-column tiles: the column halves end on 32-bit
                    // boundaries, so 32-bit words of C (the low and high halves
                    // of its little-endian 64-bit words), each owned by one tile
                    uint32_t *C32 = reinterpret_cast<uint32_t *>(C);
#pragma unroll
                    for (int g = 0; g < GH; ++g) {
                        const int64_t w32 = (int64_t)tn * G + half * GH + g;
                        if (g < ng && w32 < 2 * nW) {
                            const uint32_t v = par[g] & (uint32_t)(word_mask(w32 >> 1, T.n) >> (32 * (w32 & 1)));
                            C32[w32] = P.accumulate ? (C32[w32] ^ v) : v;
                        }
                    }
                    // the high half of the row's last 64-bit word can lie past
                    // the last tile (no tile holds a column there): written as
                    // zero like every bit past the last column
                    const int64_t wn = (int64_t)(tn + 1) * G;
                    if (half == 1 && !P.accumulate && wn < 2 * nW && 32 * wn >= T.n) C32[wn] = 0u;
                }
            }
        }
    }

    fence_before();
    __syncthreads();
    // the peer may still copy into this CTA's shared memory, arrive on its
    // barriers or be written by the pair's MMAs until both have drained
    if (PAIR) cluster_sync();
    fence_after();
    if (warp == MMA_WARP) free_tmem<PAIR>(tmem_base);
}

// Rows of a batch of packed matrices (rows x cols, stride ld, batch stride
// bs words) -> rows of `rowbytes` expanded bytes (entries beyond cols 0),
// row f = b * rows + r at Y + f * rowbytes.  A warp takes whole rows; per
// group of 32 consecutive words of the row (one coalesced 256-byte load,
// the loads of up to four groups issued before any store) it writes their
// expansion as 16-byte chunks, chunk c of the group by lane c mod 32 (each
// store instruction writes 512 contiguous bytes); the word a chunk comes
// from is fetched from its lane by a shuffle.
template <int KIND>
__device__ __forceinline__ uint4 expand_chunk(uint64_t xs, int c)
{
    if (KIND == KIND_F8) {
        const uint32_t h = (uint32_t)(xs >> (16 * (c & 3)));
        return make_uint4(f8_of_nibble(h & 15u), f8_of_nibble((h >> 4) & 15u), f8_of_nibble((h >> 8) & 15u),
                          f8_of_nibble((h >> 12) & 15u));
    }
    const uint32_t h = (uint32_t)(xs >> (32 * (c & 1)));
    return make_uint4(f4_of_byte(h), f4_of_byte(h >> 8), f4_of_byte(h >> 16), f4_of_byte(h >> 24));
}

template <int KIND>
__global__ void __launch_bounds__(256)
expand_kernel(const uint64_t *__restrict__ X, int64_t ld, int64_t bs, int64_t rows, int64_t cols, int64_t nrows,
              uint8_t *__restrict__ Y, int64_t rowbytes)
{
    constexpr int CPW = KIND == KIND_F8 ? 4 : 2;                     // 16-byte chunks per packed word
    constexpr int U = 4;                                             // groups whose loads are in flight
    const int lane = threadIdx.x & 31;
    const int64_t W = words_of(cols);
    const int64_t kpw = rowbytes / (16 * CPW);                       // packed words per expanded row
    const int ngroups = (int)((kpw + 31) / 32);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const bool small = nrows <= 0x7FFFFFFF && rows <= 0x7FFFFFFF;
    for (int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < nrows; f += nwarps) {
        int64_t b, r;
        if (small) {
            // 32-bit division (the 64-bit one is a long subroutine)
            const uint32_t bb = (uint32_t)f / (uint32_t)rows;
            b = bb;
            r = (int64_t)((uint32_t)f - bb * (uint32_t)rows);
        } else {
            b = f / rows;
            r = f - b * rows;
        }
        const uint64_t *xr = X + b * bs + r * ld;
        uint4 *orow = reinterpret_cast<uint4 *>(Y + f * rowbytes);
        for (int g0 = 0; g0 < ngroups; g0 += U) {
            uint64_t x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t w = (int64_t)(g0 + u) * 32 + lane;
                x[u] = (g0 + u < ngroups && w < W) ? (xr[w] & word_mask(w, cols)) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int wg = g0 + u;
                if (wg >= ngroups) break;
                uint4 *o = orow + (int64_t)wg * 32 * CPW;
                const int64_t left = (kpw - (int64_t)wg * 32) * CPW;   // chunks of this row from here on
#pragma unroll
                for (int q = 0; q < CPW; ++q) {
                    const int c = 32 * q + lane;                      // chunk of the group
                    const uint64_t xs = __shfl_sync(0xffffffffu, x[u], c / CPW);
                    if (c < left) o[c] = expand_chunk<KIND>(xs, c);
                }
            }
        }
    }
}

// Expanded rows of B^T straight from a batch of packed B (rows = K entries,
// cols = N, stride ld, batch stride bs words): row f = b * N + j of Y holds
// column j of product b's B.  One warp per 64 x 64 block (K word rb, column
// block cb): a ballot over the lanes of bit j gathers column j, so lane i
// ends with K word rb of rows 64 cb + i and 64 cb + 32 + i of B^T, expands
// each and writes it as one piece of 32 (FP4) or 64 (FP8) bytes -- whole
// sectors -- of its row.  K words up to the padded row length are written
// (rows of B beyond K read as zeros).
template <int KIND>
__device__ __forceinline__ void store_expanded_word(uint8_t *dst, uint64_t x)
{
    uint4 *o = reinterpret_cast<uint4 *>(dst);
    if (KIND == KIND_F8) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t h = (uint32_t)(x >> (16 * q));
            o[q] = make_uint4(f8_of_nibble(h & 15u), f8_of_nibble((h >> 4) & 15u), f8_of_nibble((h >> 8) & 15u),
                              f8_of_nibble((h >> 12) & 15u));
        }
    } else {
        const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
        o[0] = make_uint4(f4_of_byte(lo), f4_of_byte(lo >> 8), f4_of_byte(lo >> 16), f4_of_byte(lo >> 24));
        o[1] = make_uint4(f4_of_byte(hi), f4_of_byte(hi >> 8), f4_of_byte(hi >> 16), f4_of_byte(hi >> 24));
    }
}

// One unit of the transposed expansion: 64 columns (cb) of B by 8 K words
// (g: words 8g .. 8g + 7, each 64 entries of K).  Warp w takes K word 8g + w
// of the 64 columns (a ballot over the lanes of bit j gathers column j, so
// lane i ends with that word of B^T rows 64 cb + i and 64 cb + 32 + i),
// expands it into shared memory, and the CTA then writes each of the 64 rows'
// 8 expanded words as one contiguous piece (256 bytes FP4, 512 bytes FP8).
constexpr int XT_WORDS = 8;
template <int KIND> struct XtSmem {
    static constexpr int WB = KIND == KIND_F8 ? 64 : 32;          // expanded bytes per packed word
    static constexpr int ROW = XT_WORDS * WB + 16;                // padded to spread the banks
    static constexpr int BYTES = 64 * ROW;
};

template <int KIND>
__device__ __forceinline__ void expand_t_unit(const uint64_t *__restrict__ X, int64_t ld, int64_t krows,
                                              int64_t ncols, int64_t kw, int64_t g, int64_t cb,
                                              uint8_t *__restrict__ Y, int64_t rowbytes, unsigned char *sm)
{
    using S = XtSmem<KIND>;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t rb = g * XT_WORDS + w;
    if (rb < kw) {
        const uint64_t cm = word_mask(cb, ncols);
        const int64_t r0 = rb * 64 + lane, r1 = r0 + 32;
        const uint64_t x0 = (r0 < krows) ? (X[r0 * ld + cb] & cm) : 0ull;
        const uint64_t x1 = (r1 < krows) ? (X[r1 * ld + cb] & cm) : 0ull;
        uint64_t out0 = 0, out1 = 0;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const uint32_t a = __ballot_sync(0xffffffffu, (x0 >> j) & 1);
            const uint32_t c = __ballot_sync(0xffffffffu, (x1 >> j) & 1);
            const uint32_t e = __ballot_sync(0xffffffffu, (x0 >> (j + 32)) & 1);
            const uint32_t f = __ballot_sync(0xffffffffu, (x1 >> (j + 32)) & 1);
            if (lane == j) {
                out0 = (uint64_t)a | ((uint64_t)c << 32);
                out1 = (uint64_t)e | ((uint64_t)f << 32);
            }
        }
        store_expanded_word<KIND>(sm + lane * S::ROW + w * S::WB, out0);
        store_expanded_word<KIND>(sm + (lane + 32) * S::ROW + w * S::WB, out1);
    }
    __syncthreads();
    const int64_t nw = kw - g * XT_WORDS < XT_WORDS ? kw - g * XT_WORDS : XT_WORDS;
    const int cpr = (int)(nw * S::WB / 16);                       // 16-byte chunks per row
    for (int c = threadIdx.x; c < 64 * cpr; c += blockDim.x) {
        const int r = c / cpr, k = c - r * cpr;
        const int64_t row = cb * 64 + r;
        if (row < ncols)
            *reinterpret_cast<uint4 *>(Y + row * rowbytes + g * XT_WORDS * S::WB + k * 16) =
                *reinterpret_cast<const uint4 *>(sm + r * S::ROW + k * 16);
    }
    __syncthreads();
}

// cuTensorMapEncodeTiled from the driver, looked up once.
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn()
{
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// 3-D byte map over expanded rows: x = byte in the row (rowbytes), y = row
// (rows; rows beyond arrive as zeros), z = product of the batch.  Box: one
// 128-byte K block x box_rows, 128-byte swizzle.
int make_map(CUtensorMap *map, const uint8_t *base, int64_t rowbytes, int64_t rows, int batch, int box_rows)
{
    EncodeFn fn = encode_fn();
    if (!fn) return GF2_EUNSUPPORTED;
    const cuuint64_t dims[3] = {(cuuint64_t)rowbytes, (cuuint64_t)rows, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)rowbytes, (cuuint64_t)(rows * rowbytes)};
    const cuuint32_t box[3] = {(cuuint32_t)ROWB, (cuuint32_t)box_rows, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GF2_OK : GF2_ECUDA;
}

bool pairs_disabled()
{
    const char *e = getenv("GF2_TC_PAIRS");
    return e && e[0] == '0';
}

template <int KIND, int PAIR, int TN>
int mma_launch_v(const CUtensorMap &mapA, const CUtensorMap &mapB, const Params &P, int sms, cudaStream_t s)
{
    constexpr int SMEM = Ring<PAIR, PAIR ? KBS_PAIR : KBS_ONE, TN>::SMEM_BYTES;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    static int max_clusters = 0;
    std::call_once(once, [&] {
        attr_err = cudaFuncSetAttribute(tc_mma_kernel<KIND, PAIR, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (attr_err == cudaSuccess && PAIR) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3((unsigned)(sms / 2 * 2));
            cfg.blockDim = dim3(NTHREADS);
            cfg.dynamicSmemBytes = SMEM;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            if (cudaOccupancyMaxActiveClusters(&max_clusters, tc_mma_kernel<KIND, PAIR, TN>, &cfg) != cudaSuccess) {
                cudaGetLastError();
                max_clusters = 0;
            }
        }
    });
    if (attr_err != cudaSuccess) return GF2_ECUDA;
    if (PAIR && max_clusters < 1) return GF2_EUNSUPPORTED;
    const int64_t tiles = (int64_t)P.tiles_m * P.tiles_n * P.batch;
    ProfScope ps(KIND == KIND_F8 ? PF_TC : PF_TC_F4, s);
    if (!PAIR) {
        const int64_t grid = tiles < sms ? tiles : sms;
        tc_mma_kernel<KIND, PAIR, TN><<<(unsigned)grid, NTHREADS, SMEM, s>>>(mapA, mapB, P);
    } else {
        const int64_t clusters = std::min<int64_t>(tiles, max_clusters);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(clusters * 2));
        cfg.blockDim = dim3(NTHREADS);
        cfg.dynamicSmemBytes = SMEM;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        GF2_CUDA_TRY(cudaLaunchKernelEx(&cfg, tc_mma_kernel<KIND, PAIR, TN>, mapA, mapB, P));
    }
    note_launch();
    return check_launch();
}

template <int KIND>
int mma_launch(const TcxLaunch &L, cudaStream_t s)
{
    int dev = 0, sms = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    GF2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // pairs of CTAs on 256-row tiles wherever there are at least two 128-row
    // tile rows; single CTAs otherwise (or with GF2_TC_PAIRS=0)
    const bool pair = L.m > BM && !pairs_disabled();
    // FP4 pairs take 224-column tiles, whose two accumulators and scale
    // factors fit the 512 columns of tensor memory; everything else 256
    constexpr int PTN = KIND == KIND_F4 ? PTN_F4 : BN;
    Params P;
    P.m = L.m; P.n = L.n;
    P.nkb = L.rowbytes / ROWB;
    P.tiles_m = div_up(L.m, pair ? 2 * BM : BM);
    P.tiles_n = div_up(L.n, pair ? PTN : BN);
    P.batch = L.batch;
    P.C = L.C; P.ldc = L.ldc; P.bsC = L.bsC;
    P.accumulate = L.accumulate;
    P.status = L.status;
    P.prods = nullptr;
    P.tlist = nullptr;
    P.cstart = nullptr;
    P.ntiles = 0;
    CUtensorMap mapA, mapB;
    int rc = make_map(&mapA, L.XA, L.rowbytes, L.m, L.batch, BM);
    if (rc) return rc;
    if (pair) {
        rc = make_map(&mapB, L.XB, L.rowbytes, L.n, L.batch, PTN / 2);   // each CTA's half of a B^T tile
        if (rc) return rc;
        rc = mma_launch_v<KIND, 1, PTN>(mapA, mapB, P, sms, s);
        if (rc != GF2_EUNSUPPORTED) return rc;
        P.tiles_m = div_up(L.m, BM);
        P.tiles_n = div_up(L.n, BN);
    }
    rc = make_map(&mapB, L.XB, L.rowbytes, L.n, L.batch, BN / 2);     // B^T tiles as 128-row halves
    if (rc) return rc;
    return mma_launch_v<KIND, 0, BN>(mapA, mapB, P, sms, s);
}

// ------------------------------------------------------------------ batched form
// Descriptors of the batched transposed expansion (B, rows = K x cols = N
// packed, -> N expanded rows of ldt bytes at T) and of the batched expansion
// (rows of X -> expanded rows of Y).
struct TDesc {
    const uint64_t *X;
    uint64_t *T;
    int64_t rows, cols, ldx, ldt;
};
struct XDesc {
    const uint64_t *X;
    int64_t ld, rows, cols;
    uint8_t *Y;
    int64_t rowbytes;
};

// Work of one CTA of the batched transpose / expansion: a matrix and the
// first of the TBATCH (XBATCH) units of it this CTA takes, listed on the host
// so that every CTA has work.
constexpr int TBATCH = 4;                    // units of the transposed expansion per CTA
constexpr int BTN = 256;                     // tile columns of the batched form
constexpr int XBATCH = 1024;                 // packed words per CTA (4 per thread)

// B^T of every product expanded straight from its packed B, in the units of
// expand_t_unit, each CTA TBATCH units of one product.
template <int KIND>
__global__ void __launch_bounds__(256) expand_t_batched_kernel(const TDesc *__restrict__ d,
                                                               const int2 *__restrict__ work)
{
    __shared__ __align__(16) unsigned char sm[XtSmem<KIND>::BYTES];
    const int2 wk = work[blockIdx.x];
    const TDesc D = d[wk.x];
    const int64_t kw = D.ldt / XtSmem<KIND>::WB;             // ldt holds the expanded row bytes
    const int64_t CB = (D.cols + 63) / 64;
    const int64_t units = ((kw + XT_WORDS - 1) / XT_WORDS) * CB;
    const int64_t u1 = std::min<int64_t>(units, (int64_t)wk.y + TBATCH);
    for (int64_t u = wk.y; u < u1; ++u) {
        const int64_t g = u / CB, cb = u - g * CB;
        expand_t_unit<KIND>(D.X, D.ldx, D.rows, D.cols, kw, g, cb, reinterpret_cast<uint8_t *>(D.T), D.ldt, sm);
    }
}

// The expansion of expand_kernel over many matrices of their own shapes:
// blockIdx.y = the matrix, one thread per packed word of its expanded rows
// (consecutive threads write consecutive 16-byte chunks of Y).
template <int KIND>
__global__ void __launch_bounds__(256) expand_batched_kernel(const XDesc *__restrict__ d, const int2 *__restrict__ work)
{
  constexpr int CPW = KIND == KIND_F8 ? 4 : 2;
  {
    const int2 wk = work[blockIdx.x];
    const XDesc D = d[wk.x];
    const uint32_t W = (uint32_t)words_of(D.cols);
    const uint32_t kpw = (uint32_t)(D.rowbytes / (16 * CPW));
    const uint32_t total = std::min<uint32_t>((uint32_t)D.rows * kpw, (uint32_t)wk.y + XBATCH);
    for (uint32_t i = (uint32_t)wk.y + threadIdx.x; i < total; i += blockDim.x) {
        const uint32_t r = i / kpw, w = i - r * kpw;
        const uint64_t x = (w < W) ? (D.X[(int64_t)r * D.ld + w] & word_mask(w, D.cols)) : 0ull;
        uint4 *o = reinterpret_cast<uint4 *>(D.Y + (int64_t)r * D.rowbytes) + (int64_t)w * CPW;
        if (KIND == KIND_F8) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t h = (uint32_t)(x >> (16 * q));
                o[q] = make_uint4(f8_of_nibble(h & 15u), f8_of_nibble((h >> 4) & 15u), f8_of_nibble((h >> 8) & 15u),
                                  f8_of_nibble((h >> 12) & 15u));
            }
        } else {
            const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
            o[0] = make_uint4(f4_of_byte(lo), f4_of_byte(lo >> 8), f4_of_byte(lo >> 16), f4_of_byte(lo >> 24));
            o[1] = make_uint4(f4_of_byte(hi), f4_of_byte(hi >> 8), f4_of_byte(hi >> 16), f4_of_byte(hi >> 24));
        }
    }
  }
}

struct TcGraph {
    std::vector<unsigned long long> key;
    void *dev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};
std::mutex g_tcb_mu;
std::list<TcGraph> g_tcb;   // most recently used first

void tcb_free(TcGraph &e)
{
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    if (e.dev) cudaFree(e.dev);
    e.exec = nullptr;
    e.graph = nullptr;
    e.dev = nullptr;
}

int add_kernel_node(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *deps, int ndeps, void *fn,
                    dim3 grid, dim3 block, unsigned smem, void **args)
{
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof kp);
    kp.func = fn;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = smem;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(node, g, deps, (size_t)ndeps, &kp) == cudaSuccess ? GF2_OK : GF2_ECUDA;
}

template <int KIND>
int batched_build(TcGraph &e, gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[],
                  const std::vector<int> &live, int accumulate, cudaStream_t s)
{
    // layout of the entry's device memory: expanded A and B^T, products,
    // tiles, expansion descriptors and work tables
    const size_t np = live.size();
    std::vector<size_t> xa_off(np), xb_off(np);
    std::vector<int64_t> rb(np);
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) { off = (off + align - 1) / align * align; const size_t a = off; off += bytes; return a; };
    for (size_t j = 0; j < np; ++j) {
        const int i = live[j];
        const int64_t m = A[i]->rows, l = A[i]->cols, n = B[i]->cols;
        rb[j] = tc_expanded_rowbytes(KIND, l);
        xa_off[j] = take((size_t)(m * rb[j]), 256);
        xb_off[j] = take((size_t)(n * rb[j]), 256);
    }
    const size_t prod_off = take(sizeof(TcxProd) * np, 128);
    // tiles in runs of one product, the runs spread over the CTAs longest
    // first onto the least loaded CTA (work of a tile ~ its K blocks + a fixed
    // cost), each CTA's runs contiguous in the list
    int dev0 = 0, sms0 = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev0));
    GF2_CUDA_TRY(cudaDeviceGetAttribute(&sms0, cudaDevAttrMultiProcessorCount, dev0));
    int64_t ntile_all = 0;
    double work_all = 0.0;
    for (size_t j = 0; j < np; ++j) {
        const int i = live[j];
        const int64_t t = (int64_t)div_up(A[i]->rows, BM) * div_up(B[i]->cols, BTN);
        ntile_all += t;
        work_all += (double)t * (double)(rb[j] / ROWB + 2);
    }
    const int G = (int)std::min<int64_t>(ntile_all, sms0);
    struct Run { int j; int first, count; double work; };
    std::vector<Run> runs;
    const double target = work_all / G / 4.0;            // about four runs per CTA
    for (size_t j = 0; j < np; ++j) {
        const int i = live[j];
        const int tnn = div_up(B[i]->cols, BTN);
        const int t = div_up(A[i]->rows, BM) * tnn;
        const double wt = (double)(rb[j] / ROWB + 2);
        const int per = (int)std::max<double>(1.0, std::min<double>((double)t, target / wt));
        for (int f = 0; f < t; f += per) runs.push_back(Run{(int)j, f, std::min(per, t - f), wt * std::min(per, t - f)});
    }
    std::stable_sort(runs.begin(), runs.end(), [](const Run &a, const Run &b) { return a.work > b.work; });
    std::vector<std::vector<int>> byc(G);
    std::vector<double> load(G, 0.0);
    for (size_t r = 0; r < runs.size(); ++r) {
        const int c = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        byc[c].push_back((int)r);
        load[c] += runs[r].work;
    }
    std::vector<int4> tiles;
    std::vector<int> cstart(G + 1, 0);
    for (int c = 0; c < G; ++c) {
        cstart[c] = (int)tiles.size();
        for (const int r : byc[c]) {
            const Run &R = runs[r];
            const int tnn = div_up(B[live[R.j]]->cols, BTN);
            for (int k = R.first; k < R.first + R.count; ++k) tiles.push_back(make_int4(R.j, k / tnn, k % tnn, 0));
        }
    }
    cstart[G] = (int)tiles.size();
    const size_t tile_off = take(sizeof(int4) * tiles.size(), 16);
    const size_t cs_off = take(sizeof(int) * (G + 1), 16);
    const size_t td_off = take(sizeof(TDesc) * np, 16);
    const size_t xd_off = take(sizeof(XDesc) * np, 16);
    // per-CTA work tables of the two expansions (sizes known from the shapes
    // alone): 64 x 64 blocks of B (transposed), packed words of A
    const int64_t WB = KIND == KIND_F8 ? 64 : 32;           // expanded bytes per packed word
    size_t nt_work = 0, nx_work = 0;
    for (size_t j = 0; j < np; ++j) {
        const int i = live[j];
        const int64_t m = A[i]->rows, n = B[i]->cols;
        const int64_t kw = rb[j] / WB;
        nt_work += (size_t)((((kw + XT_WORDS - 1) / XT_WORDS) * ((n + 63) / 64) + TBATCH - 1) / TBATCH);
        nx_work += (size_t)((m * kw + XBATCH - 1) / XBATCH);
    }
    const size_t tw_off = take(sizeof(int2) * nt_work, 16);
    const size_t xw_off = take(sizeof(int2) * nx_work, 16);
    if (cudaMalloc(&e.dev, off) != cudaSuccess) { cudaGetLastError(); e.dev = nullptr; return GF2_ENOMEM; }
    char *base = static_cast<char *>(e.dev);
    std::vector<TcxProd> prods(np);
    std::vector<TDesc> tds(np);
    std::vector<XDesc> xds(np);
    std::vector<int2> twork, xwork;               // (matrix, first unit) per CTA
    for (size_t j = 0; j < np; ++j) {
        const int i = live[j];
        const int64_t m = A[i]->rows, l = A[i]->cols, n = B[i]->cols;
        uint8_t *xa = reinterpret_cast<uint8_t *>(base + xa_off[j]);
        uint8_t *xb = reinterpret_cast<uint8_t *>(base + xb_off[j]);
        memset(&prods[j], 0, sizeof(TcxProd));
        int rc = make_map(&prods[j].mapA, xa, rb[j], m, 1, BM);
        if (!rc) rc = make_map(&prods[j].mapB, xb, rb[j], n, 1, 128);
        if (rc) return rc;
        prods[j].C = C[i]->data;
        prods[j].ldc = C[i]->stride_words;
        prods[j].m = m; prods[j].n = n; prods[j].nkb = rb[j] / ROWB;
        // B^T expanded straight from B (K = l rows, n columns; ldt = expanded row bytes)
        tds[j] = TDesc{B[i]->data, reinterpret_cast<uint64_t *>(xb), l, n, B[i]->stride_words, rb[j]};
        xds[j] = XDesc{A[i]->data, A[i]->stride_words, m, l, xa, rb[j]};
        const int64_t kw = rb[j] / WB;
        const int64_t tb = ((kw + XT_WORDS - 1) / XT_WORDS) * ((n + 63) / 64);
        if (m * kw > INT32_MAX - XBATCH || tb > INT32_MAX - TBATCH) return GF2_EUNSUPPORTED;
        for (int64_t u = 0; u < tb; u += TBATCH) twork.push_back(make_int2((int)j, (int)u));
        for (int64_t u = 0; u < m * kw; u += XBATCH) xwork.push_back(make_int2((int)j, (int)u));
    }
    if (cudaMemcpy(base + prod_off, prods.data(), sizeof(TcxProd) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + tile_off, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + cs_off, cstart.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + td_off, tds.data(), sizeof(TDesc) * np, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + xd_off, xds.data(), sizeof(XDesc) * np, cudaMemcpyHostToDevice) != cudaSuccess)
        return GF2_ECUDA;
    if (twork.size() != nt_work || xwork.size() != nx_work) return GF2_ECUDA;
    if (cudaMemcpy(base + tw_off, twork.data(), sizeof(int2) * nt_work, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + xw_off, xwork.data(), sizeof(int2) * nx_work, cudaMemcpyHostToDevice) != cudaSuccess)
        return GF2_ECUDA;
    Params P;
    memset(&P, 0, sizeof P);
    P.accumulate = accumulate;
    int rc = tc_status_address(&P.status);
    if (rc) return rc;
    P.prods = reinterpret_cast<const TcxProd *>(base + prod_off);
    P.tlist = reinterpret_cast<const int4 *>(base + tile_off);
    P.cstart = reinterpret_cast<const int *>(base + cs_off);
    P.ntiles = (int64_t)tiles.size();
    constexpr int SMEM = Ring<0, KBS_ONE, BTN>::SMEM_BYTES;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_mma_kernel<KIND, 0, BTN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    });
    if (attr_err != cudaSuccess) return GF2_ECUDA;
    int dev = 0, sms = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    GF2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the uniform-batch map parameters are unused in this mode
    CUtensorMap unused;
    memset(&unused, 0, sizeof unused);
    const TDesc *dtd = reinterpret_cast<const TDesc *>(base + td_off);
    const XDesc *dxd = reinterpret_cast<const XDesc *>(base + xd_off);
    const int2 *dtw = reinterpret_cast<const int2 *>(base + tw_off);
    const int2 *dxw = reinterpret_cast<const int2 *>(base + xw_off);
    if (nt_work > INT32_MAX || nx_work > INT32_MAX) return GF2_EUNSUPPORTED;
    if (cudaGraphCreate(&e.graph, 0) != cudaSuccess) return GF2_ECUDA;
    cudaGraphNode_t nt, nx, nk;
    void *targs[2] = {(void *)&dtd, (void *)&dtw};
    if ((rc = add_kernel_node(e.graph, &nt, nullptr, 0, (void *)expand_t_batched_kernel<KIND>,
                              dim3((unsigned)nt_work), dim3(256), 0, targs)))
        return rc;
    void *xargs[2] = {(void *)&dxd, (void *)&dxw};
    if ((rc = add_kernel_node(e.graph, &nx, nullptr, 0, (void *)expand_batched_kernel<KIND>, dim3((unsigned)nx_work),
                              dim3(256), 0, xargs)))
        return rc;
    const cudaGraphNode_t both[2] = {nt, nx};
    void *kargs[3] = {(void *)&unused, (void *)&unused, (void *)&P};
    if ((rc = add_kernel_node(e.graph, &nk, both, 2, (void *)tc_mma_kernel<KIND, 0, BTN>,
                              dim3((unsigned)G), dim3(NTHREADS), SMEM,
                              kargs)))
        return rc;
    if (cudaGraphInstantiate(&e.exec, e.graph, 0) != cudaSuccess) { cudaGetLastError(); return GF2_ECUDA; }
    return GF2_OK;
}

}  // namespace

int64_t tc_expanded_rowbytes(int kind, int64_t l)
{
    const int64_t epr = kind == KIND_F8 ? 128 : 256;
    const int64_t kp = (l + epr - 1) / epr * epr;
    return kind == KIND_F8 ? kp : kp / 2;
}

int tc_expand_launch(int kind, const uint64_t *X, int64_t ld, int64_t bs, int64_t rows, int64_t cols, int batch,
                     uint8_t *Y, int64_t rowbytes, cudaStream_t s)
{
    const int64_t nrows = (int64_t)batch * rows;
    if (nrows <= 0 || rowbytes <= 0) return GF2_OK;
    if ((reinterpret_cast<uintptr_t>(Y) & 15) || (rowbytes % ROWB)) return GF2_ELAYOUT;
    int dev = 0, sms = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    GF2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = (nrows + 7) / 8;                  // 8 warps per block, one row each
    const int64_t grid = std::min<int64_t>(want, (int64_t)sms * 16);
    ProfScope ps(PF_EXPAND, s);
    if (kind == KIND_F8)
        expand_kernel<KIND_F8><<<(unsigned)grid, 256, 0, s>>>(X, ld, bs, rows, cols, nrows, Y, rowbytes);
    else
        expand_kernel<KIND_F4><<<(unsigned)grid, 256, 0, s>>>(X, ld, bs, rows, cols, nrows, Y, rowbytes);
    note_launch();
    return check_launch();
}

int tc_mma_launch(const TcxLaunch &L, cudaStream_t s)
{
    if (L.batch <= 0 || L.m <= 0 || L.n <= 0) return GF2_OK;
    if ((reinterpret_cast<uintptr_t>(L.XA) & 15) || (reinterpret_cast<uintptr_t>(L.XB) & 15) ||
        (L.rowbytes % ROWB) || L.rowbytes <= 0)
        return GF2_ELAYOUT;
    if (L.m > INT32_MAX || L.n > INT32_MAX || L.rowbytes > INT32_MAX || L.batch > 65535) return GF2_EUNSUPPORTED;
    return L.kind == KIND_F8 ? mma_launch<KIND_F8>(L, s) : mma_launch<KIND_F4>(L, s);
}

bool tc_fp8_available()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return major == 10 && minor == 3 && encode_fn() != nullptr;     // built for sm_103a only
}

// C[i] = A[i] B[i] for device operands (arguments already checked) on the
// tcgen05 base case of `kind`: one batched transpose of every B, one batched
// expansion of every A and B^T, one persistent launch over a (product, tile
// row, tile column) list, kept as a CUDA graph per set of operands.
int tc_batched_mul(gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[], int count,
                   int accumulate, int kind, cudaStream_t s)
{
    if (count <= 0) return GF2_OK;
    // empty products first (every call: the cached graph covers only the rest)
    std::vector<int> live;
    for (int i = 0; i < count; ++i) {
        const int64_t m = A[i]->rows, l = A[i]->cols, n = B[i]->cols;
        if (m == 0 || n == 0) continue;
        if (l == 0) {
            if (!accumulate)
                GF2_CUDA_TRY(cudaMemset2DAsync(C[i]->data, C[i]->stride_words * 8, 0, words_of(n) * 8, m, s));
            continue;
        }
        if (m > INT32_MAX || n > INT32_MAX) return GF2_EUNSUPPORTED;
        live.push_back(i);
    }
    if (live.empty()) return GF2_OK;
    std::vector<unsigned long long> key;
    key.reserve(9 * live.size() + 3);
    for (const int i : live) {
        key.push_back((unsigned long long)(uintptr_t)A[i]->data);
        key.push_back((unsigned long long)(uintptr_t)B[i]->data);
        key.push_back((unsigned long long)(uintptr_t)C[i]->data);
        key.push_back((unsigned long long)A[i]->stride_words);
        key.push_back((unsigned long long)B[i]->stride_words);
        key.push_back((unsigned long long)C[i]->stride_words);
        key.push_back((unsigned long long)A[i]->rows);
        key.push_back((unsigned long long)A[i]->cols);
        key.push_back((unsigned long long)B[i]->cols);
    }
    key.push_back((unsigned long long)(uintptr_t)s);
    key.push_back((unsigned long long)accumulate);
    key.push_back((unsigned long long)kind);
    const int fam = kind == KIND_F8 ? PF_TC : PF_TC_F4;
    std::lock_guard<std::mutex> lk(g_tcb_mu);
    for (auto it = g_tcb.begin(); it != g_tcb.end(); ++it) {
        if (it->key == key) {
            g_tcb.splice(g_tcb.begin(), g_tcb, it);
            ProfScope ps(fam, s);
            GF2_CUDA_TRY(cudaGraphLaunch(g_tcb.front().exec, s));
            note_launch(3);
            return GF2_OK;
        }
    }
    TcGraph e;
    e.key = key;
    const int rc = kind == KIND_F8 ? batched_build<KIND_F8>(e, C, A, B, live, accumulate, s)
                                   : batched_build<KIND_F4>(e, C, A, B, live, accumulate, s);
    if (rc) {
        tcb_free(e);
        return rc;
    }
    {
        ProfScope ps(fam, s);
        if (cudaGraphLaunch(e.exec, s) != cudaSuccess) { tcb_free(e); return GF2_ECUDA; }
    }
    note_launch(3);
    g_tcb.push_front(std::move(e));
    while (g_tcb.size() > 8) {
        // an older graph may still be running on its stream: wait before freeing
        cudaDeviceSynchronize();
        tcb_free(g_tcb.back());
        g_tcb.pop_back();
    }
    return GF2_OK;
}

void tc_batched_release()
{
    std::lock_guard<std::mutex> lk(g_tcb_mu);
    if (!g_tcb.empty()) cudaDeviceSynchronize();
    for (TcGraph &e : g_tcb) tcb_free(e);
    g_tcb.clear();
}

}  // namespace gf2
