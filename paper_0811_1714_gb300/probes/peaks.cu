// peaks.cu -- throughput probes for the roofline denominators that the
// library's kernels are held against and that a copy/GEMM benchmark does not
// give: shared-memory reads in the lookup pattern of the Method of the Four
// Russians tables (Section 3), L2 reads by LDG and by TMA bulk copies, the
// warp-level mma.sync s8 and b1 rates, and the tcgen05 kind::f8f6f4 and
// kind::mxf4 (block-scaled, scale factors 1.0) MMA-only rates.  Each MMA
// probe is first checked bit for bit on a 0/1 product (exact integer sums).
// Every wait is bounded; a wait that gives up sets a status word that is
// reported.  Output: one JSON object on the last line of stdout.
//
// Build: part of the package build (an executable next to libgf2.so).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#define CK(x)                                                                                  \
    do {                                                                                       \
        cudaError_t e_ = (x);                                                                  \
        if (e_ != cudaSuccess) {                                                               \
            fprintf(stderr, "CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            exit(1);                                                                           \
        }                                                                                      \
    } while (0)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, unsigned long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if ((unsigned long long)(clock64() - t0) > limit) return false;
    return true;
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// kind::mxf4 instruction descriptor: A, B = E2M1 (code 1 at bits 7-9 / 10-12), both
// K-major, N >> 3 at 17-22, scale type UE8M0 (bit 23), M >> 4 at 24-28, scale ids 0.
__host__ __device__ constexpr uint32_t idesc_mxf4(int M, int N)
{
    return (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | (1u << 23) | ((uint32_t)(M >> 4) << 24);
}
// kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3 (0), K-major.
__host__ __device__ constexpr uint32_t idesc_f8(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_mxf4(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t sfa,
                                         uint32_t sfb, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}"
        ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_f8(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, uint32_t v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(v)
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

constexpr int TA = 128 * 128;          // A image bytes (128 rows x 128 B)
constexpr int TB = 256 * 128;          // B image bytes (256 rows x 128 B)
constexpr uint32_t SFA_COL = 384, SFB_COL = 448, D_COL = 0;

// KIND 0: mxf4 (K = 256 per 128-byte row, 4 MMAs of K = 64); KIND 1: f8f6f4 (K = 128, 4 of 32).
// reps > 0: repeat the 4 MMAs reps times into one accumulator.  D (may be null) receives
// the 128 x 256 FP32 accumulator.
template <int KIND>
__global__ void __launch_bounds__(128, 1)
mma_probe(const uint8_t *Aimg, const uint8_t *Bimg, float *D, unsigned *status, int reps, int ntile)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t raw = smem_u32(sm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sb = sm + (base - raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sb + TA + TB);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (TA + TB) / 16; i += blockDim.x) {
        const uint4 v = i < TA / 16 ? reinterpret_cast<const uint4 *>(Aimg)[i]
                                    : reinterpret_cast<const uint4 *>(Bimg)[i - TA / 16];
        reinterpret_cast<uint4 *>(sb)[i] = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = *slot;
    if (KIND == 0) {
        const uint32_t lanes = (uint32_t)(warp * 32) << 16;
        tmem_st32(tb + lanes + SFA_COL, 0x7F7F7F7Fu);     // UE8M0 127 = 1.0 in every byte
        tmem_st32(tb + lanes + SFB_COL, 0x7F7F7F7Fu);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t a0 = base, b0 = base + TA;
        for (int r = 0; r < reps; ++r) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc = (r > 0 || kk > 0) ? 1u : 0u;
                if (KIND == 0)
                    mma_mxf4(tb + D_COL, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc_mxf4(128, 256),
                             tb + SFA_COL, tb + SFB_COL, acc);
                else
                    mma_f8(tb + D_COL, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc_f8(128, 256), acc);
            }
        }
        mma_commit(smem_u32(bar));
        if (!mbar_wait_bounded(smem_u32(bar), 0, 4000000000ull)) atomicExch(status, 1u);
    }
    __syncthreads();
    tc_fence_after();
    if (D && blockIdx.x == 0) {
        const uint32_t taddr = tb + ((uint32_t)(warp * 32) << 16) + D_COL;
        for (int g = 0; g < 8; ++g) {
            uint32_t r[32];
            tmem_ld32(taddr + 32 * g, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            for (int j = 0; j < 32; ++j) D[(size_t)(warp * 32 + lane) * 256 + 32 * g + j] = __uint_as_float(r[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(512) : "memory");
}

// ---- L2 read bandwidth: every CTA reads the whole (L2-resident) buffer
__global__ void l2_ldg(const uint4 *__restrict__ buf, unsigned n16_log2, int passes, uint4 *out)
{
    const size_t n16 = (size_t)1 << n16_log2, mask = n16 - 1;
    uint4 acc = make_uint4(0, 0, 0, 0);
    const size_t start = (size_t)blockIdx.x * 65536;
    for (int p = 0; p < passes; ++p)
        for (size_t i = 0; i < n16; i += (size_t)blockDim.x * 4) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcg(buf + ((i + (size_t)u * blockDim.x + threadIdx.x + start) & mask));
#pragma unroll
            for (int u = 0; u < 4; ++u) { acc.x ^= v[u].x; acc.y ^= v[u].y; acc.z ^= v[u].z; acc.w ^= v[u].w; }
        }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x9E3779B9u) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// ---- L2 -> shared memory by TMA bulk copies (one issuing thread per CTA, ring of 4 x 32 KB)
__global__ void __launch_bounds__(32, 1) l2_tma(const uint8_t *buf, size_t nchunks, int chunks, unsigned *status)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + 4 * 32768);
    if (threadIdx.x != 0) return;
    for (int s = 0; s < 4; ++s) mbar_init(smem_u32(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    int issued = 0;
    for (int c = 0; c < chunks; ++c) {
        const int s = c & 3;
        if (c >= 4 && !mbar_wait_bounded(smem_u32(&bars[s]), (uint32_t)(((c >> 2) - 1) & 1), 4000000000ull)) {
            atomicExch(status, 2u);
            break;
        }
        const size_t chunk = ((size_t)blockIdx.x * 97 + (size_t)c) % nchunks;
        mbar_arrive_expect_tx(smem_u32(&bars[s]), 32768);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(smem_u32(sm + s * 32768)), "l"(buf + chunk * 32768), "r"(32768), "r"(smem_u32(&bars[s]))
            : "memory");
        issued = c + 1;
    }
    // drain the copies issued and not yet waited for (bounded)
    for (int c = issued - 4 < 0 ? 0 : issued - 4; c < issued; ++c)
        if (!mbar_wait_bounded(smem_u32(&bars[c & 3]), (uint32_t)((c >> 2) & 1), 4000000000ull)) atomicExch(status, 3u);
}

// ---- shared-memory lookup rate: each quarter-warp reads one 128-byte row (8 x 16 B),
// four independent rows per thread per iteration, rows drawn by an LCG shared by the quarter
__global__ void __launch_bounds__(256) smem_lookup(int iters, uint4 *out)
{
    extern __shared__ uint4 tab[];          // 1024 rows x 128 B = 128 KB
    for (int i = threadIdx.x; i < 8192; i += blockDim.x) tab[i] = make_uint4(i, i * 3u, i * 7u, i * 11u);
    __syncthreads();
    const int lane = threadIdx.x & 31, q = lane >> 3, l8 = lane & 7;
    uint32_t x = (uint32_t)((threadIdx.x >> 5) * 4 + q) * 2654435761u + blockIdx.x * 40503u + 1u;
    uint4 acc = make_uint4(0, 0, 0, 0);
    for (int it = 0; it < iters; ++it) {
        const uint32_t r0 = x & 1023, r1 = (x >> 10) & 1023, r2 = (x >> 20) & 1023, r3 = ((x >> 5) ^ (x >> 17)) & 1023;
        const uint4 v0 = tab[r0 * 8 + l8], v1 = tab[r1 * 8 + l8], v2 = tab[r2 * 8 + l8], v3 = tab[r3 * 8 + l8];
        acc.x ^= v0.x ^ v1.x ^ v2.x ^ v3.x;
        acc.y ^= v0.y ^ v1.y ^ v2.y ^ v3.y;
        acc.z ^= v0.z ^ v1.z ^ v2.z ^ v3.z;
        acc.w ^= v0.w ^ v1.w ^ v2.w ^ v3.w;
        x = x * 1664525u + 1013904223u;
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x12345u) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// ---- mma.sync rates (register operands, 8 independent accumulators per warp)
// ---- integer LOP3 rate (the XORs of the lookup-accumulate): 8 independent
// 3-input XOR chains per thread, one lop3.b32 per step, full occupancy
__global__ void __launch_bounds__(256) lop3_rate(int iters, uint32_t *out)
{
    const uint32_t b = threadIdx.x * 0x9E3779B9u + blockIdx.x, c = b ^ 0x7F4A7C15u;
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = b + (uint32_t)i * 0x01000193u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < 8; ++i) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(b), "r"(c));
    }
    uint32_t x = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) x ^= a[i];
    if (x == 0x2545F491u) out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

template <bool B1>
__global__ void __launch_bounds__(256) mma_sync_rate(int iters, int *out)
{
    uint32_t a[4], b[2];
    for (int i = 0; i < 4; ++i) a[i] = threadIdx.x * 0x01010101u + i;
    for (int i = 0; i < 2; ++i) b[i] = threadIdx.x * 0x00010001u + 7 * i;
    int d[8][4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (B1)
                asm volatile(
                    "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                    : "+r"(d[u][0]), "+r"(d[u][1]), "+r"(d[u][2]), "+r"(d[u][3])
                    : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
            else
                asm volatile(
                    "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                    : "+r"(d[u][0]), "+r"(d[u][1]), "+r"(d[u][2]), "+r"(d[u][3])
                    : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
        }
    }
    int s = 0;
    for (int u = 0; u < 8; ++u) s += d[u][0] + d[u][1] + d[u][2] + d[u][3];
    if (s == 0x7654321) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------------- host
static void swizzle_rows(const std::vector<uint8_t> &rows, int R, std::vector<uint8_t> &img)
{
    img.assign((size_t)R * 128, 0);
    for (int r = 0; r < R; ++r)
        for (int j = 0; j < 8; ++j)
            memcpy(&img[(size_t)r * 128 + ((j ^ (r & 7)) * 16)], &rows[(size_t)r * 128 + j * 16], 16);
}

static uint64_t sm64(uint64_t &s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double run_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    return ms;
}


struct MmaResult {
    long wrong = -1;
    unsigned status = 0;
    double ms = 0, tflops = 0;
};

// KIND 0: kind::mxf4 (E2M1 1.0 = nibble 0x2), 1: kind::f8f6f4 (E4M3 1.0 = 0x38).
template <int KIND>
static MmaResult mma_rate(int sms)
{
    MmaResult res;
    const int K = KIND == 0 ? 256 : 128;      // entries per 128-byte row
    std::vector<uint8_t> abit(128 * K), bbit(256 * K);
    uint64_t s = 12345 + KIND;
    for (auto &v : abit) v = sm64(s) & 1;
    for (auto &v : bbit) v = (sm64(s) % 10) < 7;
    auto enc = [&](const std::vector<uint8_t> &bits, int R, std::vector<uint8_t> &rows) {
        rows.assign((size_t)R * 128, 0);
        for (int r = 0; r < R; ++r)
            for (int k = 0; k < K; ++k) {
                if (!bits[(size_t)r * K + k]) continue;
                if (KIND == 0) rows[(size_t)r * 128 + k / 2] |= (uint8_t)(0x2u << (4 * (k & 1)));
                else rows[(size_t)r * 128 + k] = 0x38;
            }
    };
    std::vector<uint8_t> arow, brow, aimg, bimg;
    enc(abit, 128, arow);
    enc(bbit, 256, brow);
    swizzle_rows(arow, 128, aimg);
    swizzle_rows(brow, 256, bimg);
    uint8_t *dA, *dB;
    float *dD;
    unsigned *dst;
    CK(cudaMalloc(&dA, TA));
    CK(cudaMalloc(&dB, TB));
    CK(cudaMalloc(&dD, 128 * 256 * 4));
    CK(cudaMalloc(&dst, 4));
    CK(cudaMemcpy(dA, aimg.data(), TA, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dB, bimg.data(), TB, cudaMemcpyHostToDevice));
    CK(cudaMemset(dst, 0, 4));
    CK(cudaMemset(dD, 0xFF, 128 * 256 * 4));
    const int smem = 120 * 1024;        // one CTA per SM: one 512-column TMEM allocation each
    CK(cudaFuncSetAttribute(mma_probe<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    mma_probe<KIND><<<1, 128, smem>>>(dA, dB, dD, dst, 1, 0);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&res.status, dst, 4, cudaMemcpyDeviceToHost));
    std::vector<float> D(128 * 256);
    CK(cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost));
    long bad = 0;
    for (int i = 0; i < 128; ++i)
        for (int j = 0; j < 256; ++j) {
            int e = 0;
            for (int k = 0; k < K; ++k) e += abit[(size_t)i * K + k] & bbit[(size_t)j * K + k];
            if (D[(size_t)i * 256 + j] != (float)e) ++bad;
        }
    res.wrong = bad;
    if (!bad && !res.status) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        const int reps = 20000;
        for (int pass = 0; pass < 2; ++pass) {          // the second of two identical launches
            CK(cudaEventRecord(e0));
            mma_probe<KIND><<<sms, 128, smem>>>(dA, dB, nullptr, dst, reps, 0);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            res.ms = run_ms(e0, e1);
            res.tflops = 2.0 * 128 * 256 * K * (double)reps * sms / res.ms / 1e9;
        }
        CK(cudaMemcpy(&res.status, dst, 4, cudaMemcpyDeviceToHost));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(dst);
    return res;
}

// Instruction variants at M = 128: VAR 0 kind::mxf4 (UE8M0 scales), 1 kind::mxf4nvf4
// scale_vec::4X (UE4M3 scales 0x38 = 1.0), 2 kind::f8f6f4, 3 kind::mxf4 with A read
// from tensor memory (zeros; throughput only); N = NN.
template <int VAR, int NN>
__global__ void __launch_bounds__(128, 1)
mma_var(const uint8_t *Aimg, const uint8_t *Bimg, float *D, unsigned *status, int reps)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t raw = smem_u32(sm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sb = sm + (base - raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sb + TA + TB);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (TA + TB) / 16; i += blockDim.x) {
        const uint4 v = i < TA / 16 ? reinterpret_cast<const uint4 *>(Aimg)[i]
                                    : reinterpret_cast<const uint4 *>(Bimg)[i - TA / 16];
        reinterpret_cast<uint4 *>(sb)[i] = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = *slot;
    {
        const uint32_t lanes = (uint32_t)(warp * 32) << 16;
        const uint32_t sv = VAR == 1 ? 0x38383838u : 0x7F7F7F7Fu;
        tmem_st32(tb + lanes + SFA_COL, sv);
        tmem_st32(tb + lanes + SFB_COL, sv);
        tmem_st32(tb + lanes + 256, 0u);       // A in TMEM (VAR 3): zeros
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t a0 = base, b0 = base + TA;
        for (int r = 0; r < reps; ++r) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc = (r > 0 || kk > 0) ? 1u : 0u;
                const uint64_t ad = sdesc(a0 + kk * 32), bd = sdesc(b0 + kk * 32);
                if (VAR == 0)
                    mma_mxf4(tb, ad, bd, idesc_mxf4(128, NN), tb + SFA_COL, tb + SFB_COL, acc);
                else if (VAR == 1)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], [%5], p;\n\t}"
                        ::"r"(tb), "l"(ad), "l"(bd), "r"(idesc_mxf4(128, NN) & ~(1u << 23)), "r"(tb + SFA_COL),
                          "r"(tb + SFB_COL), "r"(acc)
                        : "memory");
                else if (VAR == 2)
                    mma_f8(tb, ad, bd, idesc_f8(128, NN), acc);
                else
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], [%1], %2, %3, [%4], [%5], p;\n\t}"
                        ::"r"(tb), "r"(tb + 256 + 8 * kk), "l"(bd), "r"(idesc_mxf4(128, NN)), "r"(tb + SFA_COL),
                          "r"(tb + SFB_COL), "r"(acc)
                        : "memory");
            }
        }
        mma_commit(smem_u32(bar));
        if (!mbar_wait_bounded(smem_u32(bar), 0, 4000000000ull)) atomicExch(status, 1u);
    }
    __syncthreads();
    tc_fence_after();
    if (D && blockIdx.x == 0) {
        const uint32_t taddr = tb + ((uint32_t)(warp * 32) << 16);
        for (int g = 0; g < NN / 32; ++g) {
            uint32_t r[32];
            tmem_ld32(taddr + 32 * g, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            for (int j = 0; j < 32; ++j) D[(size_t)(warp * 32 + lane) * 256 + 32 * g + j] = __uint_as_float(r[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(512) : "memory");
}


template <int VAR, int NN>
static MmaResult var_rate(int sms, bool check)
{
    MmaResult res;
    const int K = VAR == 2 ? 128 : 256;
    std::vector<uint8_t> abit(128 * K), bbit(256 * K);
    uint64_t s = 777 + VAR;
    for (auto &v : abit) v = sm64(s) & 1;
    for (auto &v : bbit) v = (sm64(s) % 10) < 7;
    std::vector<uint8_t> arow((size_t)128 * 128, 0), brow((size_t)256 * 128, 0);
    auto put = [&](std::vector<uint8_t> &rows, int r, int k) {
        if (VAR == 2) rows[(size_t)r * 128 + k] = 0x38;
        else rows[(size_t)r * 128 + k / 2] |= (uint8_t)(0x2u << (4 * (k & 1)));
    };
    for (int r = 0; r < 128; ++r)
        for (int k = 0; k < K; ++k)
            if (abit[(size_t)r * K + k]) put(arow, r, k);
    for (int r = 0; r < 256; ++r)
        for (int k = 0; k < K; ++k)
            if (bbit[(size_t)r * K + k]) put(brow, r, k);
    std::vector<uint8_t> aimg, bimg;
    swizzle_rows(arow, 128, aimg);
    swizzle_rows(brow, 256, bimg);
    uint8_t *dA, *dB;
    float *dD;
    unsigned *dst;
    CK(cudaMalloc(&dA, TA)); CK(cudaMalloc(&dB, TB)); CK(cudaMalloc(&dD, 128 * 256 * 4)); CK(cudaMalloc(&dst, 4));
    CK(cudaMemcpy(dA, aimg.data(), TA, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dB, bimg.data(), TB, cudaMemcpyHostToDevice));
    CK(cudaMemset(dst, 0, 4));
    const int smem = 120 * 1024;
    CK(cudaFuncSetAttribute(mma_var<VAR, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    res.wrong = 0;
    if (check) {
        CK(cudaMemset(dD, 0xFF, 128 * 256 * 4));
        mma_var<VAR, NN><<<1, 128, smem>>>(dA, dB, dD, dst, 1);
        CK(cudaGetLastError());
        CK(cudaDeviceSynchronize());
        std::vector<float> D(128 * 256);
        CK(cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost));
        for (int i = 0; i < 128; ++i)
            for (int j = 0; j < NN; ++j) {
                int e = 0;
                for (int k = 0; k < K; ++k) e += abit[(size_t)i * K + k] & bbit[(size_t)j * K + k];
                if (D[(size_t)i * 256 + j] != (float)e) ++res.wrong;
            }
    }
    CK(cudaMemcpy(&res.status, dst, 4, cudaMemcpyDeviceToHost));
    if (!res.wrong && !res.status) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        const int reps = 20000;
        for (int pass = 0; pass < 2; ++pass) {
            CK(cudaEventRecord(e0));
            mma_var<VAR, NN><<<sms, 128, smem>>>(dA, dB, nullptr, dst, reps);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            res.ms = run_ms(e0, e1);
            res.tflops = 2.0 * 128 * NN * K * (double)reps * sms / res.ms / 1e9;
        }
        CK(cudaMemcpy(&res.status, dst, 4, cudaMemcpyDeviceToHost));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(dst);
    return res;
}

// CTA-pair MMA (cta_group::2, M = 256 over a 2-CTA cluster, N = NN), one
// stream issued by the first CTA: each CTA holds its 128 rows of A and its
// NN / 2 rows of B in shared memory (the same offsets in both), the commit
// arrives on the barrier at that offset in both CTAs.  KIND 0: kind::mxf4
// (UE8M0 scale factors 1.0), 1: kind::f8f6f4.
__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int KIND, int NN>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128, 1)
mma_pair(const uint8_t *Aimg, const uint8_t *Bimg, float *D, unsigned *status, int reps)
{
    constexpr int TBH = NN / 2 * 128;        // this CTA's half of the B image
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t raw = smem_u32(sm);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *sb = sm + (base - raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sb + TA + TBH);
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cl_rank();
    const uint4 *ga = reinterpret_cast<const uint4 *>(Aimg + rank * TA);
    const uint4 *gb = reinterpret_cast<const uint4 *>(Bimg + rank * TBH);
    for (int i = threadIdx.x; i < (TA + TBH) / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(sb)[i] = i < TA / 16 ? ga[i] : gb[i - TA / 16];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = *slot;
    if (KIND == 0) {
        const uint32_t lanes = (uint32_t)(warp * 32) << 16;
        tmem_st32(tb + lanes + SFA_COL, 0x7F7F7F7Fu);
        tmem_st32(tb + lanes + SFB_COL, 0x7F7F7F7Fu);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cl_sync();                               // both CTAs set up before the first MMA
    tc_fence_after();
    if (rank == 0 && threadIdx.x == 0) {
        const uint32_t a0 = base, b0 = base + TA;
        const uint32_t id = KIND == 0 ? idesc_mxf4(256, NN) : idesc_f8(256, NN);
        for (int r = 0; r < reps; ++r) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t acc = (r > 0 || kk > 0) ? 1u : 0u;
                const uint64_t ad = sdesc(a0 + kk * 32), bd = sdesc(b0 + kk * 32);
                if (KIND == 0)
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
                        "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}"
                        ::"r"(tb), "l"(ad), "l"(bd), "r"(id), "r"(tb + SFA_COL), "r"(tb + SFB_COL), "r"(acc)
                        : "memory");
                else
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
                        ::"r"(tb), "l"(ad), "l"(bd), "r"(id), "r"(acc)
                        : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                     ::"r"(smem_u32(bar)), "h"((unsigned short)3) : "memory");
    }
    if (threadIdx.x == 0 && !mbar_wait_bounded(smem_u32(bar), 0, 4000000000ull)) atomicExch(status, 4u);
    __syncthreads();
    tc_fence_after();
    if (D && blockIdx.x < 2) {
        const uint32_t taddr = tb + ((uint32_t)(warp * 32) << 16);
        for (int g = 0; g < NN / 32; ++g) {
            uint32_t r[32];
            tmem_ld32(taddr + 32 * g, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            for (int j = 0; j < 32; ++j)
                D[(size_t)(rank * 128 + warp * 32 + lane) * 256 + 32 * g + j] = __uint_as_float(r[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    cl_sync();                               // the peer's MMAs and reads are done
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(512) : "memory");
}

template <int KIND, int NN>
static MmaResult pair_rate(int sms)
{
    MmaResult res;
    const int K = KIND == 0 ? 256 : 128;
    std::vector<uint8_t> abit(256 * K), bbit(256 * K);
    uint64_t s = 4242 + KIND * 10 + NN;
    for (auto &v : abit) v = sm64(s) & 1;
    for (auto &v : bbit) v = (sm64(s) % 10) < 7;
    std::vector<uint8_t> arow((size_t)256 * 128, 0), brow((size_t)256 * 128, 0);
    auto put = [&](std::vector<uint8_t> &rows, int r, int k) {
        if (KIND == 1) rows[(size_t)r * 128 + k] = 0x38;
        else rows[(size_t)r * 128 + k / 2] |= (uint8_t)(0x2u << (4 * (k & 1)));
    };
    for (int r = 0; r < 256; ++r)
        for (int k = 0; k < K; ++k) {
            if (abit[(size_t)r * K + k]) put(arow, r, k);
            if (bbit[(size_t)r * K + k]) put(brow, r, k);
        }
    std::vector<uint8_t> aimg, bimg;
    swizzle_rows(arow, 256, aimg);
    swizzle_rows(brow, 256, bimg);
    uint8_t *dA, *dB;
    float *dD;
    unsigned *dst;
    CK(cudaMalloc(&dA, 256 * 128)); CK(cudaMalloc(&dB, 256 * 128));
    CK(cudaMalloc(&dD, 256 * 256 * 4)); CK(cudaMalloc(&dst, 4));
    CK(cudaMemcpy(dA, aimg.data(), 256 * 128, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dB, bimg.data(), 256 * 128, cudaMemcpyHostToDevice));
    CK(cudaMemset(dst, 0, 4));
    CK(cudaMemset(dD, 0xFF, 256 * 256 * 4));
    const int smem = 120 * 1024;
    CK(cudaFuncSetAttribute(mma_pair<KIND, NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    mma_pair<KIND, NN><<<2, 128, smem>>>(dA, dB, dD, dst, 1);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    std::vector<float> Dh(256 * 256);
    CK(cudaMemcpy(Dh.data(), dD, Dh.size() * 4, cudaMemcpyDeviceToHost));
    res.wrong = 0;
    for (int i = 0; i < 256; ++i)
        for (int j = 0; j < NN; ++j) {
            int e = 0;
            for (int k = 0; k < K; ++k) e += abit[(size_t)i * K + k] & bbit[(size_t)j * K + k];
            if (Dh[(size_t)i * 256 + j] != (float)e) ++res.wrong;
        }
    CK(cudaMemcpy(&res.status, dst, 4, cudaMemcpyDeviceToHost));
    if (!res.wrong && !res.status) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        const int reps = 20000, grid = sms / 2 * 2;
        for (int pass = 0; pass < 2; ++pass) {
            CK(cudaEventRecord(e0));
            mma_pair<KIND, NN><<<grid, 128, smem>>>(dA, dB, nullptr, dst, reps);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            res.ms = run_ms(e0, e1);
            res.tflops = 2.0 * 256 * NN * K * (double)reps * (grid / 2) / res.ms / 1e9;
        }
        CK(cudaMemcpy(&res.status, dst, 4, cudaMemcpyDeviceToHost));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(dst);
    return res;
}

static void print_mma(const char *name, const MmaResult &r, bool last)
{
    printf("\"%s\": {\"wrong\": %ld, \"status\": %u, \"ms\": %.3f, \"tflops\": %.1f}%s", name, r.wrong, r.status,
           r.ms, r.tflops, last ? "" : ", ");
}

int main()
{
    int sms = 0, khz = 0;
    CK(cudaSetDevice(0));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double l2_ldg_tbs[3] = {0, 0, 0}, l2_tma_tbs[2] = {0, 0};
    unsigned tma_status = 0;
    {
        const unsigned lg = 22;            // 4 Mi x 16 B = 64 MiB, resident in L2
        const size_t bytes = (size_t)16 << lg;
        uint4 *buf, *out;
        CK(cudaMalloc(&buf, bytes));
        CK(cudaMalloc(&out, (size_t)sms * 8 * 512 * 16));
        CK(cudaMemset(buf, 1, bytes));
        int i = 0;
        for (int ctas : {sms, 2 * sms, 4 * sms}) {
            const int passes = 2;
            l2_ldg<<<ctas, 512>>>(buf, lg, 1, out);
            CK(cudaEventRecord(e0));
            l2_ldg<<<ctas, 512>>>(buf, lg, passes, out);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            l2_ldg_tbs[i++] = (double)ctas * bytes * passes / run_ms(e0, e1) / 1e9;
        }
        unsigned *dst;
        CK(cudaMalloc(&dst, 4));
        CK(cudaMemset(dst, 0, 4));
        CK(cudaFuncSetAttribute(l2_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 32768 + 64));
        i = 0;
        for (int ctas : {sms, 2 * sms}) {
            const int chunks = 2000;
            const size_t nchunks = bytes / 32768;
            l2_tma<<<ctas, 32, 4 * 32768 + 64>>>((const uint8_t *)buf, nchunks, 100, dst);
            CK(cudaEventRecord(e0));
            l2_tma<<<ctas, 32, 4 * 32768 + 64>>>((const uint8_t *)buf, nchunks, chunks, dst);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            l2_tma_tbs[i++] = (double)ctas * chunks * 32768.0 / run_ms(e0, e1) / 1e9;
        }
        CK(cudaMemcpy(&tma_status, dst, 4, cudaMemcpyDeviceToHost));
        cudaFree(buf); cudaFree(out); cudaFree(dst);
    }
    double smem_tbs = 0, smem_ms = 0;
    {
        uint4 *out;
        CK(cudaMalloc(&out, (size_t)sms * 4 * 256 * 16));
        CK(cudaFuncSetAttribute(smem_lookup, cudaFuncAttributeMaxDynamicSharedMemorySize, 131072));
        const int iters = 20000;
        smem_lookup<<<sms, 256, 131072>>>(100, out);
        CK(cudaEventRecord(e0));
        smem_lookup<<<sms, 256, 131072>>>(iters, out);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        CK(cudaGetLastError());
        smem_ms = run_ms(e0, e1);
        smem_tbs = (double)sms * 256 * iters * 64.0 / smem_ms / 1e9;
        cudaFree(out);
    }
    double sync_tops[2] = {0, 0};
    {
        int *out;
        CK(cudaMalloc(&out, (size_t)sms * 4 * 256 * 4));
        const int iters = 4000;
        for (int b1 = 0; b1 < 2; ++b1) {
            if (b1) mma_sync_rate<true><<<sms * 4, 256>>>(10, out);
            else mma_sync_rate<false><<<sms * 4, 256>>>(10, out);
            CK(cudaEventRecord(e0));
            if (b1) mma_sync_rate<true><<<sms * 4, 256>>>(iters, out);
            else mma_sync_rate<false><<<sms * 4, 256>>>(iters, out);
            CK(cudaEventRecord(e1));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            const double ops = (double)sms * 4 * 8 * iters * 8 * (b1 ? 2.0 * 16 * 8 * 256 : 2.0 * 16 * 8 * 32);
            sync_tops[b1] = ops / run_ms(e0, e1) / 1e9;
        }
        cudaFree(out);
    }
    double lop3_per_s = 0;
    {
        uint32_t *out;
        CK(cudaMalloc(&out, (size_t)sms * 8 * 256 * 4));
        const int iters = 20000;
        lop3_rate<<<sms * 8, 256>>>(10, out);
        CK(cudaEventRecord(e0));
        lop3_rate<<<sms * 8, 256>>>(iters, out);
        CK(cudaEventRecord(e1));
        CK(cudaEventSynchronize(e1));
        CK(cudaGetLastError());
        lop3_per_s = (double)sms * 8 * 256 * iters * 32.0 / (run_ms(e0, e1) * 1e-3);
        cudaFree(out);
    }
    const MmaResult f8 = mma_rate<1>(sms);
    const MmaResult f4 = mma_rate<0>(sms);
    const MmaResult v0 = var_rate<0, 128>(sms, true);
    const MmaResult v1 = var_rate<2, 128>(sms, true);
    const MmaResult v2 = var_rate<1, 256>(sms, true);
    const MmaResult v3 = var_rate<3, 256>(sms, false);
    const MmaResult p4_256 = pair_rate<0, 256>(sms);
    const MmaResult p4_224 = pair_rate<0, 224>(sms);
    const MmaResult p4_192 = pair_rate<0, 192>(sms);
    const MmaResult p4_128 = pair_rate<0, 128>(sms);
    const MmaResult p8_256 = pair_rate<1, 256>(sms);
    const MmaResult p8_128 = pair_rate<1, 128>(sms);
    printf("{\"sms\": %d, \"max_sm_mhz\": %d, "
           "\"smem_lookup_tbs\": %.2f, \"smem_lookup_bytes_per_clk_per_sm\": %.1f, "
           "\"l2_ldg_tbs\": [%.2f, %.2f, %.2f], \"l2_ldg_ctas\": [%d, %d, %d], "
           "\"l2_tma_bulk_tbs\": [%.2f, %.2f], \"l2_tma_ctas\": [%d, %d], \"l2_tma_status\": %u, "
           "\"mma_sync_s8_tops\": %.1f, \"mma_sync_b1_tops\": %.1f, "
           "\"lop3_per_s\": %.4g, \"lop3_per_clk_per_sm\": %.1f, ",
           sms, khz / 1000, smem_tbs, smem_tbs * 1e12 / sms / (khz * 1e3), l2_ldg_tbs[0], l2_ldg_tbs[1],
           l2_ldg_tbs[2], sms, 2 * sms, 4 * sms, l2_tma_tbs[0], l2_tma_tbs[1], sms, 2 * sms, tma_status,
           sync_tops[0], sync_tops[1], lop3_per_s, lop3_per_s / sms / (khz * 1e3));
    print_mma("tcgen05_f8f6f4_m128n256", f8, false);
    print_mma("tcgen05_mxf4_m128n256", f4, false);
    print_mma("tcgen05_mxf4_m128n128", v0, false);
    print_mma("tcgen05_f8f6f4_m128n128", v1, false);
    print_mma("tcgen05_mxf4nvf4_4x_m128n256", v2, false);
    print_mma("tcgen05_mxf4_a_in_tmem_m128n256", v3, false);
    print_mma("tcgen05_pair_mxf4_m256n256", p4_256, false);
    print_mma("tcgen05_pair_mxf4_m256n224", p4_224, false);
    print_mma("tcgen05_pair_mxf4_m256n192", p4_192, false);
    print_mma("tcgen05_pair_mxf4_m256n128", p4_128, false);
    print_mma("tcgen05_pair_f8f6f4_m256n256", p8_256, false);
    print_mma("tcgen05_pair_f8f6f4_m256n128", p8_128, true);
    printf("}\n");
    const bool bad = f8.wrong || f4.wrong || v0.wrong || v1.wrong || v2.wrong || f8.status || f4.status ||
                     v0.status || v1.status || v2.status || v3.status || tma_status;
    const MmaResult *pairs[] = {&p4_256, &p4_224, &p4_192, &p4_128, &p8_256, &p8_128};
    bool pair_bad = false;
    for (const MmaResult *p : pairs) pair_bad = pair_bad || p->wrong || p->status;
    return (bad || pair_bad) ? 1 : 0;
}
