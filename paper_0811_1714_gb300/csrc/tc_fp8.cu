// tc_fp8.cu -- exact tensor-core base case: C = A B over GF(2) from 0/1
// FP8 products on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Why it is exact (Section 2.3): a GF(2) dot product is an AND followed by an
// XOR accumulation, i.e. the parity of the INTEGER dot product of the 0/1
// vectors.  Each bit becomes one FP8 E4M3 byte, 0 for a 0-bit and a power of
// two for a 1-bit that depends on the entry's K index mod 4 (i): 2^(i-9) in
// A (bytes 0x01, 0x02, 0x04, 0x08) and 2^(-6-i) in B (0x08, 0x04, 0x02,
// 0x01).  Every product of two 1-bits is therefore exactly 2^-15, and a dot
// product over a K-chunk of at most KCHUNK = 4096 entries is count * 2^-15
// <= 2^-3 with count <= 2^12: a multiple of 2^-15 that any accumulator
// keeping 13 or more significant bits holds exactly.  After each chunk the
// FP32 accumulator D is read from tensor memory and the parity of count is
// the last mantissa bit of D + 256 (whose ulp is 2^-15); parities of
// successive chunks are XORed, which is the GF(2) sum over the whole K range.
// The position-dependent values let a byte of bits expand with one byte
// permute and one mask per 4 entries.  B's values run the other way, so its
// bits are taken reversed: the transpose that produces B^T stores each
// 32-bit half of a word bit-reversed, and no reversal is left for the
// unpackers.  Only A's K tail is masked (in the last K block): an entry of A
// beyond K is 0, and every B byte is a finite FP8 value, so B's entries
// there add nothing whatever they hold.
//
// Layout of one CTA (persistent, one per SM, 26 warps):
//   warps 0-3   epilogue: tcgen05.ld of the 128 x 192 FP32 accumulator (warp
//               w reads TMEM lanes 32w..32w+31 = rows of the tile), parity,
//               packed 64-bit words of C;
//   warp 4      TMEM allocation (all 512 columns) and the MMA issuer (one
//               thread): tcgen05.mma.cta_group::1.kind::f8f6f4 with A read
//               from TENSOR MEMORY and B from shared memory, M = 128,
//               N = 192, K = 32 per instruction;
//   warp 5      TMA issuer (one thread): cp.async.bulk.tensor loads of the
//               PACKED words of A (128 rows x 32 bytes) and B^T (192 rows x
//               32 bytes) of a 256-entry K block into a ring of packed stages
//               (rows beyond the matrices and words beyond K arrive as zeros);
//   warps 6-13  A unpackers, two per TMEM lane quarter: each thread expands
//               128 bits of its row of A (half of a 256-entry K block) into
//               128 FP8 bytes in registers and stores them with tcgen05.st
//               (lane = row, 4 K entries per 32-bit column), so A never
//               occupies shared memory;
//   warps 14-25 B unpackers: expand B^T's bits into FP8 bytes and store the
//               tile in the 128-byte-swizzled K-major layout the MMA reads
//               (two 128-entry sub-tiles per K block).
// Tensor memory: accumulators at columns 0 and 256 (192 columns each), two
// A stages of 64 columns (256 K entries) at 192 and 448.
// Bits are expanded in registers (4 bits -> 4 bytes by one byte permute and
// one mask), so shared-memory bandwidth goes to the B stores and the tensor
// core's B reads only.
// Hand-offs use mbarriers: packed full (TMA transaction bytes) / packed empty,
// stage full (every A and B unpacker warp arrives) / stage empty (one
// tcgen05.commit per K block), and accumulator full / empty (MMA <->
// epilogue).  A 256-entry K block gives the MMA thread eight MMAs per wait
// and per commit: the issue of tcgen05.mma is close to synchronous, so the
// thread's serial work between MMAs is time the tensor core idles.  Every
// wait is bounded; an expired wait records GF2_ETIMEOUT in a device status
// word and the CTA winds down (waits for its issued copies and MMAs, frees
// its tensor memory) instead of hanging.
#include "common.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <list>
#include <mutex>
#include <vector>

namespace gf2 {
namespace {

constexpr int BM = 128;            // rows of A per tile (MMA M)
constexpr int BN = 192;            // rows of B^T per tile (MMA N; 3 words of C)
constexpr int BK = 256;            // K entries per stage (two 128-byte swizzle rows of FP8)
constexpr int KW = BK / 64;        // packed words per row per stage
constexpr int STAGES = 2;          // unpacked stages (A in tensor memory, B in shared memory)
constexpr int PSTAGES = 8;         // packed stages
constexpr int KCHUNK = 4096;       // exact-sum bound (entries per accumulation)
constexpr int KB_PER_CHUNK = KCHUNK / BK;
constexpr int SUB_BYTES = BN * 128;          // B^T x 128 K entries (one swizzle-row sub-tile)
constexpr int STAGE_BYTES = 2 * SUB_BYTES;   // 48 KB
constexpr int PA_BYTES = BM * KW * 8;        // packed A block: 128 rows x 4 words
constexpr int PB_BYTES = BN * KW * 8;        // packed B^T block: 192 rows x 4 words
constexpr int PSTAGE_BYTES = PA_BYTES + PB_BYTES;
constexpr int NUM_EPI_WARPS = 4;
constexpr int MMA_WARP = 4;
constexpr int TMA_WARP = 5;
constexpr int AUNP_WARP0 = 6;      // A unpackers: two per TMEM lane quarter (one per 128 K entries)
constexpr int NUM_AUNP_WARPS = 8;
constexpr int UNP_WARP0 = AUNP_WARP0 + NUM_AUNP_WARPS;         // B unpackers
constexpr int NUM_UNP_WARPS = 12;
constexpr int NTHREADS = (UNP_WARP0 + NUM_UNP_WARPS) * 32;     // 832
constexpr int NUNP = NUM_UNP_WARPS * 32;                        // 384 = 2 * BN half rows
constexpr int UNP_ARRIVALS = NUM_AUNP_WARPS + NUM_UNP_WARPS;    // arrivals that fill a stage
constexpr uint32_t TMEM_COLS = 512;
constexpr unsigned long long WAIT_LIMIT = 4000000000ull;        // clock64 cycles (~2 s)
static_assert(NUNP == 2 * BN, "one half row of each 128-entry sub-tile per B unpacker thread");
static_assert(NUM_AUNP_WARPS == 8, "A unpackers: every lane quarter x both 128-entry halves");

// tensor memory: accumulators at columns 0 and 256 (192 columns each), A
// stages of 64 columns (256 K entries) at 192 and 448
__host__ __device__ constexpr uint32_t acc_col(int b) { return (uint32_t)b * 256u; }
__host__ __device__ constexpr uint32_t a_col(int s) { return (uint32_t)s * 256u + 192u; }

// barriers: pfull[P], pempty[P], full[S], empty[S], tfull[2], tempty[2], done
constexpr int NBARS = 2 * PSTAGES + 2 * STAGES + 5;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + PSTAGES * PSTAGE_BYTES + NBARS * 8 + 16 + 1024;
static_assert(SMEM_BYTES <= 232448, "shared memory per CTA");

// One product of a batch of uneven shapes: tensor maps of its packed A and
// B^T (built on the host) and its output.
struct alignas(128) TcProd {
    CUtensorMap mapA;
    CUtensorMap mapB;
    uint64_t *C;
    int64_t ldc, m, l, n;
};

// FP8 E4M3 0x08 = 2^-6: a 1-bit.  Instruction descriptor (kind::f8f6f4):
// D format F32 (bits 4-5 = 1), A = B = E4M3 (bits 7-9, 10-12 = 0), both
// K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

struct Params {
    int64_t m, l, n;
    int tiles_m, tiles_n;
    int64_t tiles;
    uint64_t *C;
    int64_t ldc, bsC;
    int accumulate;
    unsigned int *status;
    // products of uneven shapes (null for a uniform batch): tile t is
    // tlist[t] = (product, tile row, tile column)
    const TcProd *prods;
    const int4 *tlist;
};

// One tile: where its operands and output are, and its K extent.
struct TileInfo {
    const CUtensorMap *ma, *mb;
    int z, tm, tn;
    int64_t m, l, n;
    uint64_t *C;
    int64_t ldc;
    int64_t nkb;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and the status word set) when the limit expires.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned int *status,
                                          volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if ((unsigned long long)(clock64() - t0) > WAIT_LIMIT) {
            if (status) atomicExch(status, (unsigned int)(-GF2_ETIMEOUT));
            *abort_flag = 1;
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag (used to drain copies in flight).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, unsigned int *status)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if ((unsigned long long)(clock64() - t0) > WAIT_LIMIT) {
            if (status) atomicExch(status, (unsigned int)(-GF2_ETIMEOUT));
            return;
        }
    }
}

// Warp-uniform bounded wait: lane 0 polls, the outcome is broadcast, so all
// lanes leave together (the warp-collective tcgen05 instructions that
// follow need every lane).
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, unsigned int *status,
                                          volatile int *abort_flag)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, status, abort_flag) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

// Warp-uniform read of the abort flag.
__device__ __forceinline__ bool warp_aborted(volatile int *abort_flag)
{
    int a = 0;
    if ((threadIdx.x & 31) == 0) a = *abort_flag;
    return __shfl_sync(0xffffffffu, a, 0) != 0;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    // tcgen05 shared-memory matrix descriptor: start >> 4, leading byte
    // offset 16 (unused by swizzled K-major), stride byte offset 1024 (8
    // rows x 128 bytes), fixed version 1 at bit 46, 128-byte swizzle (2).
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// D (+)= A B^T with A in tensor memory (lane = row of A, 4 FP8 entries of K
// per 32-bit column, 8 columns per K = 32) and B^T in shared memory.
__device__ __forceinline__ void mma_f8_ta(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n\t}"
        ::"r"(dtmem), "r"(atmem), "l"(bdesc), "r"(IDESC), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31]) : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// A: 32 bits x (K entries 32h .. 32h+31) -> 8 words of 4 FP8 bytes; byte i
// of word n is entry 4n+i: bit 4n+i of x moved to bit i (value 2^(i-9)).
// The byte holding the nibble is replicated by a byte permute and the mask
// keeps bit i of copy i.
__device__ __forceinline__ void expand_a(uint32_t x, uint32_t *out)
{
    const uint32_t xs = x >> 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        out[2 * k] = __byte_perm(x, 0, 0x1111u * k) & 0x08040201u;
        out[2 * k + 1] = __byte_perm(xs, 0, 0x1111u * k) & 0x08040201u;
    }
}

// B: as expand_a with bit 4n+i moved to bit 3-i (value 2^(-6-i)).  B^T's
// 32-bit halves arrive bit-reversed (r): nibble n of the natural half x is
// nibble 7-n of r with its bits reversed, so replicating its byte and
// masking bit 3-i of copy i does it.
__device__ __forceinline__ uint32_t expand_b_nibble(uint32_t r, uint32_t rs, int n)
{
    const int m = 7 - n;                       // nibble of r
    return __byte_perm((m & 1) ? rs : r, 0, 0x1111u * (uint32_t)(m >> 1)) & 0x01020408u;
}

// Tile t -> (batch, tile row, tile column).
__device__ __forceinline__ void tile_coords(const Params &P, int64_t t, int &b, int &tm, int &tn)
{
    const int64_t per = (int64_t)P.tiles_m * P.tiles_n;
    b = (int)(t / per);
    const int64_t r = t - (int64_t)b * per;
    tm = (int)(r / P.tiles_n);
    tn = (int)(r - (int64_t)tm * P.tiles_n);
}

__device__ __forceinline__ TileInfo get_tile(const Params &P, const CUtensorMap *mapA, const CUtensorMap *mapB,
                                             int64_t t)
{
    TileInfo T;
    if (!P.prods) {
        int b, tm, tn;
        tile_coords(P, t, b, tm, tn);
        T.ma = mapA; T.mb = mapB; T.z = b; T.tm = tm; T.tn = tn;
        T.m = P.m; T.l = P.l; T.n = P.n;
        T.C = P.C + (int64_t)b * P.bsC;
        T.ldc = P.ldc;
    } else {
        const int4 e = P.tlist[t];
        const TcProd &pr = P.prods[e.x];
        T.ma = &pr.mapA; T.mb = &pr.mapB; T.z = 0; T.tm = e.y; T.tn = e.z;
        T.m = pr.m; T.l = pr.l; T.n = pr.n;
        T.C = pr.C;
        T.ldc = pr.ldc;
    }
    T.nkb = (T.l + BK - 1) / BK;
    return T;
}

__global__ void __launch_bounds__(NTHREADS, 1)
tc_fp8_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Params P)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // unpacked stages must sit on 1024-byte boundaries (128-byte swizzle atoms)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sbase = smem_raw + (base - raw);
    unsigned char *pbase = sbase + STAGES * STAGE_BYTES;                     // packed ring
    uint64_t *bars = reinterpret_cast<uint64_t *>(pbase + PSTAGES * PSTAGE_BYTES);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NBARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t bar0 = smem_u32(bars);
    auto pfull_bar = [&](int s) { return bar0 + 8u * s; };
    auto pempty_bar = [&](int s) { return bar0 + 8u * (PSTAGES + s); };
    auto full_bar = [&](int s) { return bar0 + 8u * (2 * PSTAGES + s); };
    auto empty_bar = [&](int s) { return bar0 + 8u * (2 * PSTAGES + STAGES + s); };
    auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * PSTAGES + 2 * STAGES + b); };
    auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * PSTAGES + 2 * STAGES + 2 + b); };
    const uint32_t done_bar = bar0 + 8u * (2 * PSTAGES + 2 * STAGES + 4);

    if (threadIdx.x == 0) {
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(pfull_bar(s), 1);                   // the TMA thread's expect_tx arrival
            mbar_init(pempty_bar(s), UNP_ARRIVALS);
        }
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), UNP_ARRIVALS);         // one arrival per unpacker warp (A and B)
            mbar_init(empty_bar(s), 1);                   // tcgen05.commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull_bar(b), 1);
            mbar_init(tempty_bar(b), NUM_EPI_WARPS * 32);
        }
        mbar_init(done_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_slot)), "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    // every role walks the CTA's tiles t = blockIdx.x, +gridDim.x, ... and,
    // inside a tile, its K blocks; q counts K blocks in that order

    if (warp == TMA_WARP) {
        // ------------------------------------------------------------ TMA issuer
        if (lane == 0) {
            if (!P.prods) {
                asm volatile("prefetch.tensormap [%0];" ::"l"(&mapA) : "memory");
                asm volatile("prefetch.tensormap [%0];" ::"l"(&mapB) : "memory");
            }
            int64_t q = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
                const TileInfo T = get_tile(P, &mapA, &mapB, t);
                if (P.prods) {
                    // maps written by the host into reused device memory: acquire
                    // them for the tensor-copy proxy before their first use here
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(T.ma) : "memory");
                    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(T.mb) : "memory");
                }
                for (int64_t kb = 0; kb < T.nkb; ++kb, ++q) {
                    const int ps = (int)(q % PSTAGES);
                    if (!mbar_wait(pempty_bar(ps), (uint32_t)((q / PSTAGES) & 1) ^ 1u, P.status, abort_flag)) { ok = false; break; }
                    const uint32_t dst = smem_u32(pbase + ps * PSTAGE_BYTES);
                    mbar_arrive_expect_tx(pfull_bar(ps), PSTAGE_BYTES);
                    tma_load_3d(dst, T.ma, (int)(kb * KW), T.tm * BM, T.z, pfull_bar(ps));
                    tma_load_3d(dst + PA_BYTES, T.mb, (int)(kb * KW), T.tn * BN, T.z, pfull_bar(ps));
                }
            }
            // wind down: copies issued but not consumed (only after an abort)
            // still land in shared memory; wait for them before the CTA exits
            for (int64_t r = (q > PSTAGES ? q - PSTAGES : 0); r < q; ++r)
                mbar_drain(pfull_bar((int)(r % PSTAGES)), (uint32_t)((r / PSTAGES) & 1), P.status);
        }
        __syncwarp();
    } else if (warp >= AUNP_WARP0 && warp < UNP_WARP0) {
        // ------------------------------------------------------------ A unpackers
        // thread = row of the A tile = its TMEM lane (warp w owns lanes 32 (w % 4) ..);
        // warps 6-9 expand K entries 0-127 of the stage, warps 10-13 entries 128-255
        const int row = (warp & 3) * 32 + lane;
        const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;
        const int h = (warp - AUNP_WARP0) >> 2;
        int64_t q = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
          const TileInfo T = get_tile(P, &mapA, &mapB, t);
          for (int64_t kb = 0; kb < T.nkb; ++kb, ++q) {
            const int ps = (int)(q % PSTAGES);
            const int s = (int)(q % STAGES);
            if (!warp_wait(pfull_bar(ps), (uint32_t)((q / PSTAGES) & 1), P.status, abort_flag)) { ok = false; break; }
            if (!warp_wait(empty_bar(s), (uint32_t)((q / STAGES) & 1) ^ 1u, P.status, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint64_t *pk = reinterpret_cast<const uint64_t *>(pbase + ps * PSTAGE_BYTES) + KW * row;
            // A's entries beyond K (only in the last K block) are masked to 0
            uint64_t w0 = pk[2 * h], w1 = pk[2 * h + 1];
            if (kb == T.nkb - 1) {
                w0 &= word_mask(kb * KW + 2 * h, T.l);
                w1 &= word_mask(kb * KW + 2 * h + 1, T.l);
            }
            uint32_t v[32];                            // K entries 128h + 4j .. 4j+3 in v[j]
            expand_a((uint32_t)w0, v);
            expand_a((uint32_t)(w0 >> 32), v + 8);
            expand_a((uint32_t)w1, v + 16);
            expand_a((uint32_t)(w1 >> 32), v + 24);
            tmem_st32(tmem_base + tlane + a_col(s) + 32 * h, v);
            tmem_wait_st();
            // the stores are complete: order them before the arrival the MMA
            // thread acquires, then hand the packed stage back
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(full_bar(s));
                mbar_arrive(pempty_bar(ps));
            }
          }
        }
    } else if (warp >= UNP_WARP0) {
        // ------------------------------------------------------------ B unpackers
        // thread pt: half row pt of each 128-entry sub-tile (row pt / 2)
        const int pt = threadIdx.x - UNP_WARP0 * 32;      // 0..NUNP-1
        const int row = pt >> 1, half = pt & 1;
        const int sw = row & 7;
        const int rowoff = (row >> 3) * 1024 + (row & 7) * 128;
        int64_t q = 0;
        bool ok = true;
        for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
          const TileInfo T = get_tile(P, &mapA, &mapB, t);
          for (int64_t kb = 0; kb < T.nkb; ++kb, ++q) {
            const int ps = (int)(q % PSTAGES);
            const int s = (int)(q % STAGES);
            if (!warp_wait(pfull_bar(ps), (uint32_t)((q / PSTAGES) & 1), P.status, abort_flag)) { ok = false; break; }
            if (!warp_wait(empty_bar(s), (uint32_t)((q / STAGES) & 1) ^ 1u, P.status, abort_flag)) { ok = false; break; }
            const uint64_t *pk = reinterpret_cast<const uint64_t *>(pbase + ps * PSTAGE_BYTES + PA_BYTES) + KW * row;
            unsigned char *st = sbase + s * STAGE_BYTES + rowoff;
#pragma unroll
            for (int sub = 0; sub < 2; ++sub) {
                const uint64_t wv = pk[2 * sub + half];       // halves bit-reversed, tail unmasked
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const uint32_t r = (uint32_t)(wv >> (32 * hh));
                    const uint32_t rs = r >> 4;
#pragma unroll
                    for (int q2 = 0; q2 < 2; ++q2) {        // 16 entries -> one 16-byte chunk
                        const int qq = 2 * hh + q2;
                        const int chunk = (half * 4 + qq) ^ sw;   // 128-byte swizzle
                        *reinterpret_cast<uint4 *>(st + sub * SUB_BYTES + chunk * 16) =
                            make_uint4(expand_b_nibble(r, rs, 4 * q2), expand_b_nibble(r, rs, 4 * q2 + 1),
                                       expand_b_nibble(r, rs, 4 * q2 + 2), expand_b_nibble(r, rs, 4 * q2 + 3));
                    }
                }
            }
            // each lane makes its stores visible to the tensor core (async
            // proxy), then one arrival per warp on the stage, and the packed
            // stage is handed back to the TMA thread
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(full_bar(s));
                mbar_arrive(pempty_bar(ps));
            }
          }
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t it = 0, u = 0;                        // K blocks, accumulator units
            bool ok = true;
            for (int64_t t = blockIdx.x; t < P.tiles && ok; t += gridDim.x) {
                const TileInfo T = get_tile(P, &mapA, &mapB, t);
                const int64_t nkb = T.nkb;
                const int nchunks = (int)((nkb + KB_PER_CHUNK - 1) / KB_PER_CHUNK);
                for (int c = 0; c < nchunks && ok; ++c, ++u) {
                    const int ab = (int)(u & 1u);
                    if (!mbar_wait(tempty_bar(ab), ((u >> 1) & 1u) ^ 1u, P.status, abort_flag)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t dt = tmem_base + acc_col(ab);
                    const int kb0 = c * KB_PER_CHUNK;
                    const int kb1 = (int)min(nkb, (int64_t)kb0 + KB_PER_CHUNK);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = (int)(it & (STAGES - 1));
                        if (!mbar_wait(full_bar(s), (it / STAGES) & 1u, P.status, abort_flag)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t sb = base + s * STAGE_BYTES;
                        const uint32_t ta = tmem_base + a_col(s);
#pragma unroll
                        for (int kk = 0; kk < BK / 32; ++kk) {
                            // K step of 32 FP8 entries: 8 TMEM columns of A,
                            // 32 bytes inside a swizzle row of B's sub-tile
                            mma_f8_ta(dt, ta + 8 * kk, smem_desc_sw128(sb + (kk >> 2) * SUB_BYTES + (kk & 3) * 32),
                                      (kb > kb0 || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(empty_bar(s));          // stage free once these MMAs have read it
                    }
                    if (!ok) break;
                    mma_commit(tfull_bar(ab));             // accumulator ready for the epilogue
                }
            }
            // wind down: wait until every issued MMA has completed
            mma_commit(done_bar);
            mbar_drain(done_bar, 0, P.status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int row_in_tile = warp * 32 + lane;          // TMEM lane = tile row
        uint32_t u = 0;
        for (int64_t t = blockIdx.x; t < P.tiles && !warp_aborted(abort_flag); t += gridDim.x) {
            const TileInfo T = get_tile(P, &mapA, &mapB, t);
            const int nchunks = (int)((T.nkb + KB_PER_CHUNK - 1) / KB_PER_CHUNK);
            uint32_t par[BN / 32];
#pragma unroll
            for (int i = 0; i < BN / 32; ++i) par[i] = 0;
            bool ok = true;
            for (int c = 0; c < nchunks; ++c, ++u) {
                const int ab = (int)(u & 1u);
                if (!warp_wait(tfull_bar(ab), (u >> 1) & 1u, P.status, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(warp * 32) << 16) + acc_col(ab);
#pragma unroll 1
                for (int g = 0; g < BN / 32; ++g) {
                    uint32_t r[32];
                    tmem_ld32(taddr + g * 32, r);
                    tmem_wait_ld();
                    uint32_t word = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        // D = count * 2^-15 <= 2^-3: the ulp of D + 256 is 2^-15
                        const uint32_t f = __float_as_uint(__uint_as_float(r[j]) + 256.0f);
                        word |= (f & 1u) << j;
                    }
                    par[g] ^= word;
                }
                tc_fence_before();
                mbar_arrive(tempty_bar(ab));
            }
            if (!ok) break;
            const int64_t grow = (int64_t)T.tm * BM + row_in_tile;
            if (grow < T.m) {
                uint64_t *C = T.C + grow * T.ldc;
                const int64_t nW = words_of(T.n);
#pragma unroll
                for (int i = 0; i < BN / 64; ++i) {
                    const int64_t wcol = (int64_t)T.tn * (BN / 64) + i;
                    if (wcol < nW) {
                        const uint64_t v = (((uint64_t)par[2 * i + 1] << 32) | par[2 * i]) & word_mask(wcol, T.n);
                        C[wcol] = P.accumulate ? (C[wcol] ^ v) : v;
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                     : "memory");
    }
}

__device__ unsigned int g_tc_status;   // -GF2_ETIMEOUT after an expired wait

// Failure-detection self test: one wait that nothing can satisfy (an mbarrier
// nobody arrives on), bounded by `limit` clock cycles; it records
// GF2_ETIMEOUT in the status word exactly like the product kernels do.
__global__ void wait_selftest_kernel(unsigned long long limit, unsigned int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (!mbar_try_wait(smem_u32(&bar), 0)) {
            if ((unsigned long long)(clock64() - t0) > limit) {
                atomicExch(status, (unsigned int)(-GF2_ETIMEOUT));
                break;
            }
        }
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once (no link-time
// dependency on the driver library).
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

// 3-D map over packed words: x = word in the row (extent ceil(l/64): words
// beyond K are filled with zeros), y = row (extent rows), z = product of the
// batch.  Box: KW words x box_rows x 1.
int make_map(CUtensorMap *map, const uint64_t *base, int64_t words, int64_t rows, int64_t ld, int batch,
             int64_t bs, int box_rows)
{
    EncodeFn fn = encode_fn();
    if (!fn) return GF2_EUNSUPPORTED;
    const cuuint64_t dims[3] = {(cuuint64_t)words, (cuuint64_t)rows, (cuuint64_t)batch};
    const int64_t bstride = batch > 1 ? bs * 8 : rows * ld * 8;
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * 8), (cuuint64_t)(bstride > 0 ? bstride : ld * 8)};
    const cuuint32_t box[3] = {(cuuint32_t)KW, (cuuint32_t)box_rows, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<uint64_t *>(base), dims, strides, box,
                          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GF2_OK : GF2_ECUDA;
}

// ------------------------------------------------------------------ batched form
// B^T of every product of a batch in one launch: one warp per 64 x 64 block
// (a ballot over the lanes of bit j gathers column j); the block's product
// is found by binary search over the prefix sums of the block counts.  Each
// 32-bit half of an output word is stored bit-reversed, the order the
// unpackers expand.
struct TDesc {
    const uint64_t *X;
    uint64_t *T;
    int64_t rows, cols, ldx, ldt;     // X is rows x cols; T = X^T is cols x rows
};

__global__ void transpose_batched_kernel(const TDesc *__restrict__ d, const long long *__restrict__ prefix,
                                         int count, long long total)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long b = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < total; b += nwarps) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= b) lo = mid; else hi = mid - 1;
        }
        const TDesc D = d[lo];
        const long long local = b - prefix[lo];
        const int64_t CB = words_of(D.cols);
        const int64_t rb = local / CB, cb = local - rb * CB;
        const int64_t r0 = rb * 64 + lane, r1 = r0 + 32;
        const uint64_t cm = word_mask(cb, D.cols);
        const uint64_t x0 = (r0 < D.rows) ? (D.X[r0 * D.ldx + cb] & cm) : 0ull;
        const uint64_t x1 = (r1 < D.rows) ? (D.X[r1 * D.ldx + cb] & cm) : 0ull;
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
        const uint64_t tm = word_mask(rb, D.rows);
        out0 &= tm;
        out1 &= tm;
        out0 = ((uint64_t)__brev((uint32_t)(out0 >> 32)) << 32) | __brev((uint32_t)out0);
        out1 = ((uint64_t)__brev((uint32_t)(out1 >> 32)) << 32) | __brev((uint32_t)out1);
        const int64_t t0 = cb * 64 + lane, t1 = t0 + 32;
        if (t0 < D.cols) D.T[t0 * D.ldt + rb] = out0;
        if (t1 < D.cols) D.T[t1 * D.ldt + rb] = out1;
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

}  // namespace

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

int wait_selftest_launch(long long limit, cudaStream_t s)
{
    unsigned int *st = nullptr;
    GF2_CUDA_TRY(cudaGetSymbolAddress((void **)&st, g_tc_status));
    wait_selftest_kernel<<<1, 32, 0, s>>>((unsigned long long)limit, st);
    note_launch();
    return check_launch();
}

int tc_status_address(unsigned int **p)
{
    GF2_CUDA_TRY(cudaGetSymbolAddress((void **)p, g_tc_status));
    return GF2_OK;
}

int tc_status_read_and_clear(unsigned int *out, cudaStream_t s)
{
    unsigned int *p = nullptr;
    GF2_CUDA_TRY(cudaGetSymbolAddress((void **)&p, g_tc_status));
    unsigned int v = 0;
    GF2_CUDA_TRY(cudaMemcpyAsync(&v, p, sizeof v, cudaMemcpyDeviceToHost, s));
    GF2_CUDA_TRY(cudaStreamSynchronize(s));
    GF2_CUDA_TRY(cudaMemsetAsync(p, 0, sizeof v, s));
    *out = v;
    return GF2_OK;
}

int tc_fp8_launch(const TcLaunch &L, cudaStream_t s)
{
    if (L.batch <= 0 || L.m <= 0 || L.n <= 0) return GF2_OK;
    // operand rows must start on 16-byte boundaries for the tensor copies
    if ((L.lda & 1) || (L.ldb & 1) || (reinterpret_cast<uintptr_t>(L.A) & 15) ||
        (reinterpret_cast<uintptr_t>(L.Bt) & 15) || (L.batch > 1 && ((L.bsA & 1) || (L.bsB & 1))))
        return GF2_ELAYOUT;
    if (L.m > INT32_MAX || L.n > INT32_MAX || words_of(L.l) > INT32_MAX || L.batch > 65535) return GF2_EUNSUPPORTED;
    Params P;
    P.m = L.m; P.l = L.l; P.n = L.n;
    P.tiles_m = div_up(L.m, BM);
    P.tiles_n = div_up(L.n, BN);
    P.tiles = (int64_t)L.batch * P.tiles_m * P.tiles_n;
    P.C = L.C; P.ldc = L.ldc; P.bsC = L.bsC;
    P.accumulate = L.accumulate;
    P.prods = nullptr;
    P.tlist = nullptr;
    unsigned int *st = L.status;
    if (!st) GF2_CUDA_TRY(cudaGetSymbolAddress((void **)&st, g_tc_status));
    P.status = st;
    CUtensorMap mapA, mapB;
    int rc = make_map(&mapA, L.A, words_of(L.l), L.m, L.lda, L.batch, L.bsA, BM);
    if (rc) return rc;
    rc = make_map(&mapB, L.Bt, words_of(L.l), L.n, L.ldb, L.batch, L.bsB, BN);
    if (rc) return rc;
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    });
    if (attr_err != cudaSuccess) return GF2_ECUDA;
    int dev = 0, sms = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    GF2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t grid = P.tiles < sms ? P.tiles : sms;
    ProfScope ps(PF_TC_PACKED, s);
    tc_fp8_kernel<<<(unsigned)grid, NTHREADS, SMEM_BYTES, s>>>(mapA, mapB, P);
    note_launch();
    return check_launch();
}


// C[i] = A[i] B[i] for device operands (arguments already checked), one
// batched transpose and one persistent tensor-core launch, kept as a CUDA
// graph per set of operands.
int tc_batched_mul(gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[], int count,
                   int accumulate, cudaStream_t s)
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
        if ((A[i]->stride_words & 1) || (reinterpret_cast<uintptr_t>(A[i]->data) & 15)) return GF2_ELAYOUT;
        if (m > INT32_MAX || n > INT32_MAX) return GF2_EUNSUPPORTED;
        live.push_back(i);
    }
    if (live.empty()) return GF2_OK;
    std::vector<unsigned long long> key;
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
    std::lock_guard<std::mutex> lk(g_tcb_mu);
    for (auto it = g_tcb.begin(); it != g_tcb.end(); ++it) {
        if (it->key == key) {
            g_tcb.splice(g_tcb.begin(), g_tcb, it);
            ProfScope ps(PF_TC_PACKED, s);
            GF2_CUDA_TRY(cudaGraphLaunch(g_tcb.front().exec, s));
            note_launch(2);
            return GF2_OK;
        }
    }
    // layout of the entry's device memory: B^T buffers, products, tiles,
    // transpose descriptors, prefix sums
    std::vector<size_t> bt_off(count);
    size_t off = 0;
    auto take = [&](size_t bytes, size_t align) { off = (off + align - 1) / align * align; const size_t a = off; off += bytes; return a; };
    for (const int i : live)
        bt_off[i] = take((size_t)(B[i]->cols * even_up(words_of(A[i]->cols))) * 8, 256);
    const size_t prod_off = take(sizeof(TcProd) * live.size(), 128);
    std::vector<int4> tiles;
    for (size_t j = 0; j < live.size(); ++j) {
        const int i = live[j];
        const int tmn = div_up(A[i]->rows, BM), tnn = div_up(B[i]->cols, BN);
        for (int tm = 0; tm < tmn; ++tm)
            for (int tn = 0; tn < tnn; ++tn) tiles.push_back(make_int4((int)j, tm, tn, 0));
    }
    // longest K first
    std::stable_sort(tiles.begin(), tiles.end(), [&](const int4 &a, const int4 &b) {
        return A[live[a.x]]->cols > A[live[b.x]]->cols;
    });
    const size_t tile_off = take(sizeof(int4) * tiles.size(), 16);
    const size_t td_off = take(sizeof(TDesc) * live.size(), 16);
    const size_t pre_off = take(sizeof(long long) * (live.size() + 1), 16);
    TcGraph e;
    e.key = key;
    if (cudaMalloc(&e.dev, off) != cudaSuccess) { cudaGetLastError(); return GF2_ENOMEM; }
    char *base = static_cast<char *>(e.dev);
    std::vector<TcProd> prods(live.size());
    std::vector<TDesc> tds(live.size());
    std::vector<long long> prefix(live.size() + 1, 0);
    for (size_t j = 0; j < live.size(); ++j) {
        const int i = live[j];
        const int64_t m = A[i]->rows, l = A[i]->cols, n = B[i]->cols;
        uint64_t *bt = reinterpret_cast<uint64_t *>(base + bt_off[i]);
        const int64_t ldt = even_up(words_of(l));
        memset(&prods[j], 0, sizeof(TcProd));
        int rc = make_map(&prods[j].mapA, A[i]->data, words_of(l), m, A[i]->stride_words, 1, 0, BM);
        if (!rc) rc = make_map(&prods[j].mapB, bt, words_of(l), n, ldt, 1, 0, BN);
        if (rc) { tcb_free(e); return rc; }
        prods[j].C = C[i]->data;
        prods[j].ldc = C[i]->stride_words;
        prods[j].m = m; prods[j].l = l; prods[j].n = n;
        tds[j] = TDesc{B[i]->data, bt, l, n, B[i]->stride_words, ldt};
        prefix[j + 1] = prefix[j] + (long long)((l + 63) / 64) * (long long)words_of(n);
    }
    if (cudaMemcpy(base + prod_off, prods.data(), sizeof(TcProd) * prods.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + tile_off, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + td_off, tds.data(), sizeof(TDesc) * tds.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(base + pre_off, prefix.data(), sizeof(long long) * prefix.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        tcb_free(e);
        return GF2_ECUDA;
    }
    Params P;
    memset(&P, 0, sizeof P);
    P.tiles = (int64_t)tiles.size();
    P.accumulate = accumulate;
    GF2_CUDA_TRY(cudaGetSymbolAddress((void **)&P.status, g_tc_status));
    P.prods = reinterpret_cast<const TcProd *>(base + prod_off);
    P.tlist = reinterpret_cast<const int4 *>(base + tile_off);
    static std::once_flag once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(once, [] {
        attr_err = cudaFuncSetAttribute(tc_fp8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    });
    if (attr_err != cudaSuccess) { tcb_free(e); return GF2_ECUDA; }
    int dev = 0, sms = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    GF2_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the uniform-batch map parameters are unused in this mode
    CUtensorMap unused;
    memset(&unused, 0, sizeof unused);
    const TDesc *dtd = reinterpret_cast<const TDesc *>(base + td_off);
    const long long *dpre = reinterpret_cast<const long long *>(base + pre_off);
    int cnt = (int)live.size();
    long long total = prefix.back();
    long long tblocks = (total * 32 + 255) / 256;
    if (tblocks > 152 * 32) tblocks = 152 * 32;
    if (cudaGraphCreate(&e.graph, 0) != cudaSuccess) { tcb_free(e); return GF2_ECUDA; }
    cudaGraphNode_t nt, nk;
    {
        void *args[4] = {(void *)&dtd, (void *)&dpre, (void *)&cnt, (void *)&total};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = (void *)transpose_batched_kernel;
        kp.gridDim = dim3((unsigned)(tblocks > 0 ? tblocks : 1));
        kp.blockDim = dim3(256);
        kp.kernelParams = args;
        if (cudaGraphAddKernelNode(&nt, e.graph, nullptr, 0, &kp) != cudaSuccess) { tcb_free(e); return GF2_ECUDA; }
    }
    {
        void *args[3] = {(void *)&unused, (void *)&unused, (void *)&P};
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = (void *)tc_fp8_kernel;
        kp.gridDim = dim3((unsigned)std::min<int64_t>((int64_t)tiles.size(), sms));
        kp.blockDim = dim3(NTHREADS);
        kp.sharedMemBytes = SMEM_BYTES;
        kp.kernelParams = args;
        if (cudaGraphAddKernelNode(&nk, e.graph, &nt, 1, &kp) != cudaSuccess) { tcb_free(e); return GF2_ECUDA; }
    }
    if (cudaGraphInstantiate(&e.exec, e.graph, 0) != cudaSuccess) { cudaGetLastError(); tcb_free(e); return GF2_ECUDA; }
    {
        ProfScope ps(PF_TC_PACKED, s);
        if (cudaGraphLaunch(e.exec, s) != cudaSuccess) { tcb_free(e); return GF2_ECUDA; }
    }
    note_launch(2);
    g_tcb.push_front(std::move(e));
    while (g_tcb.size() > 8) {
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
