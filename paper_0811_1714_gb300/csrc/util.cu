// util.cu -- device helpers: seeded bit generator, bit transpose, the packed
// matrix-vector product used by Freivalds' check, the cubic product of
// Section 2.3 for right factors of at most 64 columns, launch bookkeeping and
// device-time accounting.
#include "common.cuh"

#include <atomic>
#include <mutex>
#include <vector>

namespace gf2 {

static std::atomic<long long> g_launches{0};

// ---- device-time accounting (gf2_profile_*) --------------------------------
namespace {
struct ProfRec {
    int fam;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRec> g_prof_recs;
double g_prof_ms[PF_COUNT];
long long g_prof_n[PF_COUNT];

void prof_drain()   // caller holds g_prof_mu
{
    for (ProfRec &r : g_prof_recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_prof_ms[r.fam] += ms;
            g_prof_n[r.fam] += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_recs.clear();
    cudaGetLastError();
}
}  // namespace

ProfScope::ProfScope(int family, cudaStream_t stream) : fam(family), s(stream), rec(nullptr)
{
    if (!g_prof_on.load(std::memory_order_relaxed)) return;
    ProfRec *r = new ProfRec{family, nullptr, nullptr};
    if (cudaEventCreate(&r->a) != cudaSuccess || cudaEventCreate(&r->b) != cudaSuccess ||
        cudaEventRecord(r->a, stream) != cudaSuccess) {
        cudaGetLastError();
        if (r->a) cudaEventDestroy(r->a);
        if (r->b) cudaEventDestroy(r->b);
        delete r;
        return;
    }
    rec = r;
}

ProfScope::~ProfScope()
{
    if (!rec) return;
    ProfRec *r = static_cast<ProfRec *>(rec);
    if (cudaEventRecord(r->b, s) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_recs.push_back(*r);
    } else {
        cudaGetLastError();
    }
    delete r;
}

int profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    for (int i = 0; i < PF_COUNT; ++i) { g_prof_ms[i] = 0; g_prof_n[i] = 0; }
    g_prof_on.store(on != 0);
    return GF2_OK;
}

int profile_read(int fam, double *ms, long long *n)
{
    if (fam < 0 || fam >= PF_COUNT) return GF2_EINVAL;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain();
    if (ms) *ms = g_prof_ms[fam];
    if (n) *n = g_prof_n[fam];
    return GF2_OK;
}

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }

int check_launch()
{
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GF2_OK : GF2_ECUDA;
}

namespace {

// SplitMix64 (Steele, Lea, Flood 2014): output n of the stream seeded with s
// is mix(s + n * 0x9E3779B97F4A7C15).
__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void random_kernel(DMat M, uint64_t seed, uint32_t thr, int half)
{
    const int64_t W = words_of(M.cols);
    const int64_t total = M.rows * M.ld;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / M.ld, w = i - r * M.ld;
        uint64_t v = 0;
        if (w < W) {
            const uint64_t idx = (uint64_t)(r * W + w);
            if (half) {
                v = sm64(seed, idx + 1);
            } else {
                for (int j = 0; j < 32; ++j) {
                    const uint64_t o = sm64(seed, idx * 32 + j + 1);
                    v |= (uint64_t)((uint32_t)o < thr) << (2 * j);
                    v |= (uint64_t)((uint32_t)(o >> 32) < thr) << (2 * j + 1);
                }
            }
            v &= word_mask(w, M.cols);
        }
        M.p[r * M.ld + w] = v;
    }
}

__global__ void seeded_words_kernel(uint64_t *X, int64_t n, uint64_t seed)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        X[i] = sm64(seed, (uint64_t)i + 1);
}

// T = X^T, one warp per 64 x 64 block: lane i holds rows i and i+32 of the
// block; a ballot over the lanes of bit j gathers column j.
__global__ void transpose_kernel(DMat T, DMat X)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t RB = (X.rows + 63) / 64;          // row blocks of X
    const int64_t CB = words_of(X.cols);            // column blocks (words) of X
    const int64_t nblk = RB * CB;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t b = warp_global; b < nblk; b += nwarps) {
        const int64_t rb = b / CB, cb = b - rb * CB;
        const int64_t r0 = rb * 64 + lane, r1 = r0 + 32;
        const uint64_t cm = word_mask(cb, X.cols);
        const uint64_t x0 = (r0 < X.rows) ? (X.p[r0 * X.ld + cb] & cm) : 0ull;
        const uint64_t x1 = (r1 < X.rows) ? (X.p[r1 * X.ld + cb] & cm) : 0ull;
        uint64_t out0 = 0, out1 = 0;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            const uint32_t a = __ballot_sync(0xffffffffu, (x0 >> j) & 1);
            const uint32_t c = __ballot_sync(0xffffffffu, (x1 >> j) & 1);
            const uint32_t d = __ballot_sync(0xffffffffu, (x0 >> (j + 32)) & 1);
            const uint32_t e = __ballot_sync(0xffffffffu, (x1 >> (j + 32)) & 1);
            if (lane == j) {
                out0 = (uint64_t)a | ((uint64_t)c << 32);
                out1 = (uint64_t)d | ((uint64_t)e << 32);
            }
        }
        // out0: row cb*64+lane of T, word rb; out1: row cb*64+32+lane
        const uint64_t tm = word_mask(rb, T.cols);
        out0 &= tm;
        out1 &= tm;
        const int64_t t0 = cb * 64 + lane, t1 = t0 + 32;
        if (t0 < T.rows) T.p[t0 * T.ld + rb] = out0;
        if (t1 < T.rows) T.p[t1 * T.ld + rb] = out1;
    }
}

// Y[i] = M[i] X for 64 vectors: bit v of Y[i] is the parity of
// (row i of M) AND (packed vector v), with XT the 64 x cols transpose of X.
// Section 2.3's dot product (AND, XOR accumulation, parity).  One warp per row.
__global__ void matvec64_kernel(const uint64_t *M, int64_t rows, int64_t cols, int64_t ld,
                                const uint64_t *XT, int64_t ldx, uint64_t *Y)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = words_of(cols);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < rows; i += nwarps) {
        uint64_t y = 0;
        for (int vb = 0; vb < 64; vb += 16) {
            uint64_t acc[16];
#pragma unroll
            for (int v = 0; v < 16; ++v) acc[v] = 0;
            for (int64_t w = lane; w < W; w += 32) {
                const uint64_t mw = M[i * ld + w] & word_mask(w, cols);
#pragma unroll
                for (int v = 0; v < 16; ++v) acc[v] ^= mw & XT[(int64_t)(vb + v) * ldx + w];
            }
#pragma unroll
            for (int v = 0; v < 16; ++v) {
                const unsigned p = (unsigned)(__popcll(acc[v]) & 1);
                const unsigned q = __reduce_xor_sync(0xffffffffu, p);
                y |= (uint64_t)q << (vb + v);
            }
        }
        if (lane == 0) Y[i] = y;
    }
}

// The cubic product of Section 2.3 for a right factor of at most 64 columns
// (the paper's choice there instead of M4RM): row i of C is one word whose
// bit j is the parity of (row i of A) AND (row j of B^T).  One warp per row
// of A; BT holds the n columns of B as rows (64 rows, rows n..63 zero).
__global__ void cubic_narrow_kernel(const uint64_t *A, int64_t lda, int64_t m, int64_t l,
                                    const uint64_t *BT, int64_t ldbt, uint64_t *C, int64_t ldc,
                                    int64_t n, int accumulate)
{
    const int lane = threadIdx.x & 31;
    const int64_t W = words_of(l);
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int vmax = (int)((n + 15) / 16) * 16;              // columns in passes of 16
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nwarps) {
        uint64_t y = 0;
        for (int vb = 0; vb < vmax; vb += 16) {
            uint64_t acc[16];
#pragma unroll
            for (int v = 0; v < 16; ++v) acc[v] = 0;
            for (int64_t w = lane; w < W; w += 32) {
                const uint64_t aw = A[i * lda + w] & word_mask(w, l);
#pragma unroll
                for (int v = 0; v < 16; ++v) acc[v] ^= aw & BT[(int64_t)(vb + v) * ldbt + w];
            }
#pragma unroll
            for (int v = 0; v < 16; ++v) {
                const unsigned q = __reduce_xor_sync(0xffffffffu, (unsigned)(__popcll(acc[v]) & 1));
                y |= (uint64_t)q << (vb + v);
            }
        }
        if (lane == 0) {
            y &= word_mask(0, n);
            C[i * ldc] = accumulate ? (C[i * ldc] ^ y) : y;
        }
    }
}

__global__ void xor_count_kernel(const uint64_t *a, const uint64_t *b, int64_t n,
                                 unsigned long long *count)
{
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        c += (a[i] != b[i]);
    if (c) atomicAdd(count, c);
}

int blocks_for(int64_t total, int per = 256)
{
    int64_t b = (total + per - 1) / per;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int random_launch(DMat M, uint64_t seed, double p, cudaStream_t s)
{
    if (M.rows <= 0 || M.ld <= 0) return GF2_OK;
    const int half = (p == 0.5);
    double t = p * 4294967296.0;
    uint32_t thr;
    if (t <= 0) thr = 0;
    else if (t >= 4294967295.0) thr = 0xffffffffu;
    else thr = (uint32_t)t;
    ProfScope ps(PF_RANDOM, s);
    random_kernel<<<blocks_for(M.rows * M.ld), 256, 0, s>>>(M, seed, thr, half);
    note_launch();
    return check_launch();
}

int seeded_words_launch(uint64_t *X, int64_t n, uint64_t seed, cudaStream_t s)
{
    if (n <= 0) return GF2_OK;
    ProfScope ps(PF_RANDOM, s);
    seeded_words_kernel<<<blocks_for(n), 256, 0, s>>>(X, n, seed);
    note_launch();
    return check_launch();
}

int transpose_launch(DMat T, DMat X, cudaStream_t s)
{
    const int64_t nblk = ((X.rows + 63) / 64) * words_of(X.cols);
    if (nblk <= 0) return GF2_OK;
    int64_t blocks = (nblk * 32 + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    ProfScope ps(PF_TRANSPOSE, s);
    transpose_kernel<<<(unsigned)blocks, 256, 0, s>>>(T, X);
    note_launch();
    return check_launch();
}

int matvec64_launch(const uint64_t *M, int64_t rows, int64_t cols, int64_t ld,
                    const uint64_t *XT, uint64_t *Y, cudaStream_t s)
{
    // XT: 64 x cols, stride = words_of(cols) rounded to even
    if (rows <= 0) return GF2_OK;
    const int64_t ldx = even_up(words_of(cols));
    int64_t blocks = (rows * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    ProfScope ps(PF_MATVEC, s);
    matvec64_kernel<<<(unsigned)blocks, 256, 0, s>>>(M, rows, cols, ld, XT, ldx, Y);
    note_launch();
    return check_launch();
}

int cubic_narrow_launch(const uint64_t *A, int64_t lda, int64_t m, int64_t l, const uint64_t *BT,
                        int64_t ldbt, uint64_t *C, int64_t ldc, int64_t n, int accumulate, cudaStream_t s)
{
    if (m <= 0 || n <= 0) return GF2_OK;
    if (n > 64) return GF2_EINVAL;
    int64_t blocks = (m * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    ProfScope ps(PF_M4RM, s);
    cubic_narrow_kernel<<<(unsigned)blocks, 256, 0, s>>>(A, lda, m, l, BT, ldbt, C, ldc, n, accumulate);
    note_launch();
    return check_launch();
}

int xor_count_launch(const uint64_t *a, const uint64_t *b, int64_t n, unsigned long long *count,
                     cudaStream_t s)
{
    if (n <= 0) return GF2_OK;
    ProfScope ps(PF_MATVEC, s);
    xor_count_kernel<<<blocks_for(n), 256, 0, s>>>(a, b, n, count);
    note_launch();
    return check_launch();
}

}  // namespace gf2
