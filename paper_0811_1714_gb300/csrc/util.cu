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

// Transpose of a 32 x 32 bit block held by a warp, lane = row, bit j of the
// lane's word = column j: five exchange steps of the standard recursive
// block swap (blocks of 16, 8, 4, 2, 1), partner lane ^ w by a shuffle.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane)
{
    const uint32_t M[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int w = 16 >> st;
        const uint32_t m = M[st];
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, w);
        x = (lane & w) ? ((x & ~m) | ((y >> w) & m)) : ((x & m) | ((y & m) << w));
    }
    return x;
}

// T = X^T, one warp per 256 x 256 block (256 rows x 4 words of X): lane i
// holds rows i + 32 k (k < 8) of the block, 4 words each, so every row's 32
// bytes are read by one lane (whole sectors); each 64 x 64 sub-block is four
// 32 x 32 shuffle transposes with its off-diagonal quarters swapped, and
// lane i ends with 4 consecutive words of 8 rows of T.  V16: rows of X and T
// start on 16-byte boundaries, so words move in pairs (16-byte loads and
// stores), and lanes 2j, 2j + 1 trade halves so that each store instruction
// writes 16 whole 32-byte sectors instead of 32 halves.
template <bool V16>
__global__ void __launch_bounds__(256) transpose_kernel(DMat T, DMat X)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t RB = (X.rows + 255) / 256;         // 256-row blocks of X
    const int64_t XW = words_of(X.cols);
    const int64_t CB = (XW + 3) / 4;                 // 4-word column blocks of X
    const int64_t TW = words_of(T.cols);
    const int64_t nblk = RB * CB;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t blk = warp_global; blk < nblk; blk += nwarps) {
        const int64_t rb = blk / CB, cb = blk - rb * CB;
        uint64_t x[8][4];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t r = rb * 256 + 32 * k + lane;
            const uint64_t *xr = X.p + r * X.ld;
#pragma unroll
            for (int c = 0; c < 4; c += 2) {
                const int64_t w = cb * 4 + c;
                if (V16) {
                    // words w and w + 1 (w even; w + 1 is still inside the even stride)
                    ulonglong2 v = make_ulonglong2(0ull, 0ull);
                    if (r < X.rows && w < XW) v = *reinterpret_cast<const ulonglong2 *>(xr + w);
                    x[k][c] = v.x & word_mask(w, X.cols);
                    x[k][c + 1] = v.y & word_mask(w + 1, X.cols);
                } else {
                    x[k][c] = (r < X.rows && w < XW) ? (xr[w] & word_mask(w, X.cols)) : 0ull;
                    x[k][c + 1] = (r < X.rows && w + 1 < XW) ? (xr[w + 1] & word_mask(w + 1, X.cols)) : 0ull;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            // rows (cb * 4 + c) * 64 + lane (h = 0) and + 32 (h = 1) of T, words rb * 4 + q
            uint64_t o[2][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // sub-block: rows 64 q + lane (x0) and 64 q + 32 + lane (x1) of the block, word c
                const uint64_t x0 = x[2 * q][c], x1 = x[2 * q + 1][c];
                const uint32_t a = transpose32((uint32_t)x0, lane);           // rows 0-31, cols 0-31
                const uint32_t b = transpose32((uint32_t)x1, lane);           // rows 32-63, cols 0-31
                const uint32_t d = transpose32((uint32_t)(x0 >> 32), lane);   // rows 0-31, cols 32-63
                const uint32_t e = transpose32((uint32_t)(x1 >> 32), lane);   // rows 32-63, cols 32-63
                o[0][q] = (uint64_t)a | ((uint64_t)b << 32);
                o[1][q] = (uint64_t)d | ((uint64_t)e << 32);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t t = (cb * 4 + c) * 64 + 32 * h + lane;
                uint64_t v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = o[h][q] & word_mask(rb * 4 + q, T.cols);
                if (V16) {
                    // lanes 2j and 2j + 1 (rows t and t + 1 of T) trade halves so that
                    // each 16-byte store pairs with its neighbour lane's into one whole
                    // 32-byte sector: first both halves of the even lane's row, then
                    // both halves of the odd lane's
                    const int odd = lane & 1;
                    const uint64_t s0 = odd ? v[0] : v[2], s1 = odd ? v[1] : v[3];
                    const uint64_t r0 = __shfl_xor_sync(0xffffffffu, s0, 1), r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
                    const int64_t w = rb * 4 + 2 * odd;
                    const int64_t row0 = t - odd;                        // the even lane's row
                    const uint64_t a0 = odd ? r0 : v[0], a1 = odd ? r1 : v[1];   // row0, words w, w + 1
                    const uint64_t b0 = odd ? v[2] : r0, b1 = odd ? v[3] : r1;   // row0 + 1
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int64_t row = row0 + k;
                        if (row >= T.rows) continue;
                        uint64_t *tr = T.p + row * T.ld;
                        const uint64_t x0 = k ? b0 : a0, x1 = k ? b1 : a1;
                        if (w + 1 < TW) {
                            *reinterpret_cast<ulonglong2 *>(tr + w) = make_ulonglong2(x0, x1);
                        } else if (w < TW) {
                            tr[w] = x0;
                        }
                    }
                } else {
                    if (t >= T.rows) continue;
                    uint64_t *tr = T.p + t * T.ld;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (rb * 4 + q < TW) tr[rb * 4 + q] = v[q];
                }
            }
        }
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
    const int64_t nblk = ((X.rows + 255) / 256) * ((words_of(X.cols) + 3) / 4);
    if (nblk <= 0) return GF2_OK;
    int64_t blocks = (nblk * 32 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const bool v16 = (X.ld % 2 == 0) && (T.ld % 2 == 0) && !(reinterpret_cast<uintptr_t>(X.p) & 15) &&
                     !(reinterpret_cast<uintptr_t>(T.p) & 15);
    ProfScope ps(PF_TRANSPOSE, s);
    if (v16)
        transpose_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(T, X);
    else
        transpose_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(T, X);
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
