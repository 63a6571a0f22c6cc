// api.cu -- the C ABI of libgf2: argument checks, the Strassen-Winograd
// plan (Section 4, Algorithm 4) with its per-(device, stream) scratch arena,
// dispatch to the base cases, odd sizes by virtual padding or by peeling
// (Section 4), the autotuner's choice of base case x depth and of padding vs
// peeling (timed on the caller's operands, cached per shape), host staging,
// the batched entry point, and Freivalds' check.
#include "common.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

namespace gf2 {
long long launch_count();
int profile_enable(int on);
int profile_read(int fam, double *ms, long long *n);
}

using namespace gf2;

namespace {

// The tensor-core base cases read B transposed (rows of B^T = columns of B).
bool is_tc(int base)
{
    return base == GF2_BASE_TC_FP8 || base == GF2_BASE_TC_S8 || base == GF2_BASE_TC_B1 || base == GF2_BASE_TC_FP4;
}

// The tcgen05 base cases run on operands expanded once in HBM (FP8 bytes or
// FP4 nibbles); the warp-level ones read the packed words.
bool is_expanded(int base) { return base == GF2_BASE_TC_FP8 || base == GF2_BASE_TC_FP4; }
int kind_of(int base) { return base == GF2_BASE_TC_FP4 ? KIND_F4 : KIND_F8; }

const char *base_name(int base)
{
    switch (base) {
    case GF2_BASE_TC_FP8: return "tc_fp8";
    case GF2_BASE_TC_S8: return "tc_s8";
    case GF2_BASE_TC_B1: return "tc_b1";
    case GF2_BASE_TC_FP4: return "tc_fp4";
    default: return "m4rm";
    }
}

// ---------------------------------------------------------------- arenas
// One arena per (device, stream).  A caller holds the arena's mutex from
// arena_get until it has queued all work that uses the arena, so another
// host thread on the same stream can neither grow (free) it nor hand the same
// bytes out in between.
struct Arena {
    std::mutex mu;
    void *ptr = nullptr;
    size_t bytes = 0;
    ~Arena() { if (ptr) cudaFree(ptr); }
};
std::mutex g_arena_mu;   // guards the map, not the arenas
std::map<std::pair<int, uintptr_t>, std::shared_ptr<Arena>> g_arenas;

// Non-blocking side streams per device (0, 1, 2; created on first use), for
// copies and transposes that overlap work on the caller's stream; ordered by
// events.
cudaStream_t side_stream(int dev, int which = 0)
{
    static std::mutex mu;
    static cudaStream_t st[64][3] = {};
    if (dev < 0 || dev >= 64 || which < 0 || which > 2) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    cudaStream_t &x = st[dev][which];
    if (!x && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        x = nullptr;
    }
    return x;
}

// On an early return from a call that queued copies on side streams, the
// caller's stream waits for whatever they still have queued (copies into the
// arena) and is synchronised, so that the next user of the arena cannot
// overwrite buffers still being copied.  Disarmed once the call has waited
// for everything itself.
struct SideJoin {
    cudaStream_t s;
    cudaStream_t side[3];
    bool armed = true;
    ~SideJoin()
    {
        if (!armed) return;
        for (cudaStream_t x : side) {
            if (!x || x == s) continue;
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) break;
            if (cudaEventRecord(e, x) == cudaSuccess) cudaStreamWaitEvent(s, e, 0);
            cudaEventDestroy(e);
        }
        cudaStreamSynchronize(s);
        cudaGetLastError();
    }
};

struct ArenaHold {
    std::shared_ptr<Arena> arena;
    std::unique_lock<std::mutex> lock;
};

int arena_get(cudaStream_t s, size_t bytes, void **out, ArenaHold *hold)
{
    *out = nullptr;
    if (bytes == 0) return GF2_OK;
    int dev = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    std::shared_ptr<Arena> ap;
    {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        auto &slot = g_arenas[{dev, reinterpret_cast<uintptr_t>(s)}];
        if (!slot) slot = std::make_shared<Arena>();
        ap = slot;
    }
    std::unique_lock<std::mutex> lk(ap->mu);
    Arena &a = *ap;
    if (a.bytes < bytes) {
        if (a.ptr) {
            // earlier work queued on this stream may still use the old arena
            GF2_CUDA_TRY(cudaStreamSynchronize(s));
            cudaFree(a.ptr);
            a.ptr = nullptr;
            a.bytes = 0;
        }
        const size_t want = (bytes + (1u << 21) - 1) & ~(size_t)((1u << 21) - 1);
        if (cudaMalloc(&a.ptr, want) != cudaSuccess) {
            cudaGetLastError();
            a.ptr = nullptr;
            return GF2_ENOMEM;
        }
        a.bytes = want;
    }
    *out = a.ptr;
    hold->arena = std::move(ap);
    hold->lock = std::move(lk);
    return GF2_OK;
}

// ---------------------------------------------------------------- checks
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int check_mat(const gf2_mat *M)
{
    if (!M) return GF2_EINVAL;
    if (M->rows < 0 || M->cols < 0) return GF2_EINVAL;
    if (M->rows == 0 || M->cols == 0) return GF2_OK;
    if (!M->data) return GF2_EINVAL;
    if (M->stride_words < words_of(M->cols)) return GF2_ELAYOUT;
    if ((M->stride_words & 1) || !aligned16(M->data)) return GF2_ELAYOUT;
    return GF2_OK;
}

size_t mat_bytes(const gf2_mat *M)
{
    if (M->rows == 0 || M->cols == 0) return 0;
    return (size_t)((M->rows - 1) * M->stride_words + words_of(M->cols)) * 8;
}

bool overlaps(const gf2_mat *X, const gf2_mat *Y)
{
    if (X->device != Y->device) return false;
    const size_t bx = mat_bytes(X), by = mat_bytes(Y);
    if (!bx || !by) return false;
    const uintptr_t x0 = reinterpret_cast<uintptr_t>(X->data), y0 = reinterpret_cast<uintptr_t>(Y->data);
    return x0 < y0 + by && y0 < x0 + bx;
}

gf2_opts resolve(const gf2_opts *o)
{
    gf2_opts r;
    gf2_default_opts(&r);
    if (o) r = *o;
    return r;
}

int check_opts(const gf2_opts &o)
{
    if (o.base < GF2_BASE_AUTO || o.base > GF2_BASE_TC_FP4) return GF2_EINVAL;
    if (o.depth < -1 || o.depth > 8) return GF2_EINVAL;
    if (o.k < 0 || o.k > 10 || o.t < 0 || o.t > 16) return GF2_EINVAL;
    if (o.accumulate != 0 && o.accumulate != 1) return GF2_EINVAL;
    if (o.peel < -1 || o.peel > 1) return GF2_EINVAL;
    if (o.reserved[0] || o.reserved[1]) return GF2_EINVAL;
    if (o.k > 0 && o.t > 0 && !m4rm_supported(o.k, o.t)) return GF2_EUNSUPPORTED;
    return GF2_OK;
}

// ---------------------------------------------------------------- the plan
// Strassen-Winograd, breadth first (Algorithm 4 applied `depth` times to all
// sub-problems of a level at once).  Padded sizes: rows to a multiple of
// 2^depth, column counts to a multiple of 128 * 2^depth so that every
// quadrant starts on a 16-byte boundary (Section 4's "good" sizes, reached
// by virtual zero padding).  Arena: A-operand, B-operand and product slabs of
// every level, then the transposed B for the tensor-core base, then host
// staging buffers.
constexpr int kMaxDepth = 8;

struct Plan {
    int64_t m, l, n;
    int base;
    int depth;
    int64_t M, L, N;
    int k, t;
    // per level j (1..depth): offsets (bytes) and strides (words)
    size_t offA[kMaxDepth + 1], offB[kMaxDepth + 1], offP[kMaxDepth + 1];
    int64_t ldA[kMaxDepth + 1], ldB[kMaxDepth + 1], ldP[kMaxDepth + 1];
    int64_t slabA[kMaxDepth + 1], slabB[kMaxDepth + 1], slabP[kMaxDepth + 1];
    size_t offBt;        // transposed B (tensor-core base, depth 0 or top of the split;
    int64_t ldBt;        // the cubic form: 64 rows)
    size_t offXA, offXB; // expanded leaf operands (FP8 / FP4 tensor-core base cases)
    int64_t rowbytes;    // bytes per expanded row
    bool cubic;          // depth 0, at most 64 columns: the cubic product of Section 2.3
    size_t bytes;        // total device scratch (without host staging)
};

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

int auto_depth(int64_t m, int64_t l, int64_t n, int base)
{
    // Recurse while every dimension of the sub-problems stays at or above the
    // cutoff (Section 5's c_o): each level saves 1/8 of the base-case work
    // and costs O(n^2) streaming additions.
    const int64_t cutoff = (base == GF2_BASE_M4RM || base == GF2_BASE_AUTO) ? 4096 : 8192;
    int d = 0;
    int64_t mm = m, ll = l, nn = n;
    while (d < 6 && mm / 2 >= cutoff && ll / 2 >= cutoff && nn / 2 >= cutoff) {
        mm /= 2; ll /= 2; nn /= 2; ++d;
    }
    return d;
}

int make_plan(int64_t m, int64_t l, int64_t n, const gf2_opts &o, Plan *p)
{
    memset(p, 0, sizeof(*p));
    p->m = m; p->l = l; p->n = n;
    p->base = o.base;
    if (p->base == GF2_BASE_AUTO) p->base = GF2_BASE_M4RM;
    if (is_expanded(p->base) && !tc_fp8_available()) return GF2_EUNSUPPORTED;
    p->depth = (o.depth < 0) ? auto_depth(m, l, n, p->base) : o.depth;
    if (m == 0 || n == 0 || l == 0) p->depth = 0;
    const int d = p->depth;
    const int64_t rq = (int64_t)1 << d, cq = (int64_t)128 << d;
    p->M = d ? round_up(m, rq) : m;
    p->L = d ? round_up(l, cq) : l;
    p->N = d ? round_up(n, cq) : n;
    if (d && (p->M < 2 * rq / 2 || p->M / rq < 1)) return GF2_EUNSUPPORTED;
    p->k = o.k; p->t = o.t;
    const bool tc = is_tc(p->base);   // B held transposed
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += (bytes + 255) & ~(size_t)255;
        return at;
    };
    int64_t cnt = 1;
    for (int j = 1; j <= d; ++j) {
        cnt *= 7;
        const int64_t Mj = p->M >> j, Lj = p->L >> j, Nj = p->N >> j;
        p->ldA[j] = Lj / 64;
        p->slabA[j] = Mj * p->ldA[j];
        p->offA[j] = take((size_t)(cnt * p->slabA[j]) * 8);
        if (tc) {   // right factors stored transposed: Nj x Lj
            p->ldB[j] = Lj / 64;
            p->slabB[j] = Nj * p->ldB[j];
        } else {
            p->ldB[j] = Nj / 64;
            p->slabB[j] = Lj * p->ldB[j];
        }
        p->offB[j] = take((size_t)(cnt * p->slabB[j]) * 8);
        p->ldP[j] = Nj / 64;
        p->slabP[j] = Mj * p->ldP[j];
        p->offP[j] = take((size_t)(cnt * p->slabP[j]) * 8);
    }
    if (tc) {
        p->ldBt = even_up(words_of(l));
        p->offBt = take((size_t)(n * p->ldBt) * 8);
    }
    if (is_expanded(p->base) && m > 0 && l > 0 && n > 0) {
        // every leaf operand expanded once: A leaves (Md rows) and B^T leaves
        // (Nd rows), rows of rowbytes
        const int64_t Md = d ? (p->M >> d) : m, Ld = d ? (p->L >> d) : l, Nd = d ? (p->N >> d) : n;
        p->rowbytes = tc_expanded_rowbytes(kind_of(p->base), Ld);
        p->offXA = take((size_t)(cnt * Md) * (size_t)p->rowbytes);
        p->offXB = take((size_t)(cnt * Nd) * (size_t)p->rowbytes);
    }
    // a right factor of at most 64 columns (Section 2.3, the paper's choice
    // over M4RM there): one word of C per row, from B's columns as rows
    p->cubic = (p->base == GF2_BASE_M4RM && d == 0 && o.k == 0 && o.t == 0 && m > 0 && l > 0 && n > 0 &&
                n <= 64);
    if (p->cubic) {
        p->ldBt = even_up(words_of(l));
        p->offBt = take((size_t)(64 * p->ldBt) * 8);
    }
    p->bytes = off;
    return GF2_OK;
}

bool fuses_expansion(const Plan &p);

std::string plan_text(const Plan &p)
{
    char buf[512];
    snprintf(buf, sizeof buf,
             "base=%s depth=%d padded=%lldx%lldx%lld leaves=%lld leaf=%lldx%lldx%lld k=%d t=%d scratch=%zu",
             base_name(p.base), p.depth, (long long)p.M, (long long)p.L,
             (long long)p.N, (long long)[&] { long long c = 1; for (int j = 0; j < p.depth; ++j) c *= 7; return c; }(),
             (long long)(p.M >> p.depth), (long long)(p.L >> p.depth), (long long)(p.N >> p.depth), p.k, p.t,
             p.bytes);
    std::string t(buf);
    if (p.cubic) t += " cubic=1";
    if (fuses_expansion(p)) t += " fused_expand=1";
    return t;
}

// Whether the last level of Algorithm 4's additions writes the leaf operands
// expanded (expanded tensor-core base case below at least one level, leaf rows
// needing no padding to whole 128-byte K blocks).
bool fuses_expansion(const Plan &p)
{
    return is_expanded(p.base) && p.depth >= 1 &&
           p.rowbytes == (kind_of(p.base) == KIND_F8 ? (p.L >> p.depth) : (p.L >> p.depth) / 2);
}

// Base case over `batch` products with dense or user layouts.
int run_base(const Plan &p, const uint64_t *A, int64_t lda, int64_t bsA, const uint64_t *B,
             int64_t ldb, int64_t bsB, uint64_t *C, int64_t ldc, int64_t bsC, int64_t m, int64_t l,
             int64_t n, int batch, int accumulate, char *scratch, cudaStream_t s, bool a_expanded = false,
             bool b_expanded = false)
{
    if (is_expanded(p.base)) {
        // expand the packed leaves once (HBM-bound), then the MMA kernel
        // (A's leaves already expanded when a_expanded)
        const int kind = kind_of(p.base);
        uint8_t *XA = reinterpret_cast<uint8_t *>(scratch + p.offXA);
        uint8_t *XB = reinterpret_cast<uint8_t *>(scratch + p.offXB);
        int rc = a_expanded ? GF2_OK : tc_expand_launch(kind, A, lda, bsA, m, l, batch, XA, p.rowbytes, s);
        if (!rc && !b_expanded) rc = tc_expand_launch(kind, B, ldb, bsB, n, l, batch, XB, p.rowbytes, s);
        if (rc) return rc;
        TcxLaunch X;
        X.kind = kind;
        X.XA = XA; X.XB = XB; X.rowbytes = p.rowbytes;
        X.C = C; X.ldc = ldc; X.bsC = bsC;
        X.m = m; X.n = n; X.batch = batch; X.accumulate = accumulate;
        if ((rc = tc_status_address(&X.status))) return rc;
        return tc_mma_launch(X, s);
    }
    if (is_tc(p.base)) {
        TcLaunch L;
        L.A = A; L.lda = lda; L.bsA = bsA;
        L.Bt = B; L.ldb = ldb; L.bsB = bsB;
        L.C = C; L.ldc = ldc; L.bsC = bsC;
        L.m = m; L.l = l; L.n = n; L.batch = batch; L.accumulate = accumulate;
        L.status = nullptr;
        return p.base == GF2_BASE_TC_S8 ? tc_s8_launch(L, s) : tc_b1_launch(L, s);
    }
    M4rmLaunch L;
    L.A = A; L.lda = lda; L.bsA = bsA;
    L.B = B; L.ldb = ldb; L.bsB = bsB;
    L.C = C; L.ldc = ldc; L.bsC = bsC;
    L.m = m; L.l = l; L.n = n; L.batch = batch; L.accumulate = accumulate;
    L.k = p.k; L.t = p.t; L.ksplit = 0; L.bm = 0;
    return m4rm_launch(L, s);
}

// C = A B (or C ^= A B) for device matrices on the current device.
// b_leaves: the right factor's leaves (and B^T) are already in the plan's
// scratch from a call on the same B with the same plan apart from m (row
// blocks of A), so B's transposition, additions and expansion are skipped.
// b_only: only that preparation of B's leaves (A and C are not read).
int mul_device(const gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const Plan &p, int accumulate,
               char *scratch, cudaStream_t s, cudaEvent_t b_ready = nullptr, bool bt_ready = false,
               bool b_leaves = false, bool b_only = false)
{
    const int64_t m = p.m, l = p.l, n = p.n;
    if (m == 0 || n == 0) return GF2_OK;
    if (l == 0) {
        if (accumulate) return GF2_OK;
        GF2_CUDA_TRY(cudaMemset2DAsync(C->data, C->stride_words * 8, 0, words_of(n) * 8, m, s));
        return GF2_OK;
    }
    const bool tc = is_tc(p.base);
    const uint64_t *Bsrc = B->data;
    int64_t ldBsrc = B->stride_words;
    const int d = p.depth;
    // expanded tensor-core base cases: the last level of additions writes the
    // leaf operands already expanded (no packed leaves, no expansion pass)
    // when the leaves' rows need no padding to whole 128-byte K blocks
    const bool fused = fuses_expansion(p);
    // the left factor's additions need nothing of B: with B still arriving
    // (b_ready), they run first and B's work waits for the event
    auto split_A = [&](int j, int step, int64_t cnt) {
        const int jt = j + step - 1;                       // level written
        const int64_t Mp = p.M >> (j - 1), Lp = p.L >> (j - 1);
        SplitLaunch SA;
        SA.nparent = (int)cnt;
        SA.side = 0;
        SA.rows = Mp; SA.cols = Lp;
        if (j == 1) {
            SA.X = A->data; SA.ld = A->stride_words; SA.bs = 0; SA.vrows = m; SA.vcols = l;
        } else {
            SA.X = reinterpret_cast<const uint64_t *>(scratch + p.offA[j - 1]);
            SA.ld = p.ldA[j - 1]; SA.bs = p.slabA[j - 1]; SA.vrows = Mp; SA.vcols = Lp;
        }
        SA.out = reinterpret_cast<uint64_t *>(scratch + p.offA[jt]);
        SA.cld = p.ldA[jt]; SA.cbs = p.slabA[jt];
        if (fused && jt == d) {
            SA.xout = reinterpret_cast<uint8_t *>(scratch + p.offXA);
            SA.rowbytes = p.rowbytes;
            SA.xkind = kind_of(p.base) + 1;
        }
        return step == 2 ? sw_split2_launch(SA, s) : sw_split_launch(SA, s);
    };
    // the fused expansion writes the leaves from a single-level split (the
    // two-level one, holding 28 operand blocks per thread, writes 49 expanded
    // leaves at half the HBM rate)
    auto split_step = [&](int j) {
        const int st = (d - j + 1 >= 2) ? 2 : 1;
        return (fused && st == 2 && j + 1 == d) ? 1 : st;
    };
    if (d > 0 && !b_only) {
        int64_t cnt = 1;
        for (int j = 1; j <= d;) {
            const int step = split_step(j);
            int rc = split_A(j, step, cnt);
            if (rc) return rc;
            cnt *= (step == 2) ? 49 : 7;
            j += step;
        }
    }
    // the expanded tensor-core base cases: A's leaves are expanded before B
    // is needed, so that this runs while B is still arriving
    bool a_expanded = fused;
    if (!b_only && !fused && is_expanded(p.base) && !(d == 0 && p.cubic)) {
        int64_t cntA = 1;
        for (int j = 0; j < d; ++j) cntA *= 7;
        const uint64_t *XA = d == 0 ? A->data : reinterpret_cast<const uint64_t *>(scratch + p.offA[d]);
        const int64_t ldXA = d == 0 ? A->stride_words : p.ldA[d];
        const int64_t bsXA = d == 0 ? 0 : p.slabA[d];
        const int64_t Md = d == 0 ? m : p.M >> d, Ld = d == 0 ? l : p.L >> d;
        const int rc = tc_expand_launch(kind_of(p.base), XA, ldXA, bsXA, Md, Ld, (int)cntA,
                                        reinterpret_cast<uint8_t *>(scratch + p.offXA), p.rowbytes, s);
        if (rc) return rc;
        a_expanded = true;
    }
    if (b_ready) GF2_CUDA_TRY(cudaStreamWaitEvent(s, b_ready, 0));
    // the tensor-core base cases read B transposed
    if (tc) {
        uint64_t *Bt = reinterpret_cast<uint64_t *>(scratch + p.offBt);
        if (!bt_ready && !b_leaves) {
            DMat T{Bt, n, l, p.ldBt};
            DMat X{B->data, l, n, B->stride_words};
            int rc = transpose_launch(T, X, s);
            if (rc) return rc;
        }
        Bsrc = Bt;
        ldBsrc = p.ldBt;
    }
    if (d == 0 && p.cubic) {
        uint64_t *BT = reinterpret_cast<uint64_t *>(scratch + p.offBt);
        GF2_CUDA_TRY(cudaMemsetAsync(BT, 0, (size_t)(64 * p.ldBt) * 8, s));
        DMat T{BT, n, l, p.ldBt};
        DMat X{B->data, l, n, B->stride_words};
        int rc = transpose_launch(T, X, s);
        if (rc) return rc;
        return cubic_narrow_launch(A->data, A->stride_words, m, l, BT, p.ldBt, C->data, C->stride_words, n,
                                   accumulate, s);
    }
    if (d == 0 && b_only)
        return is_expanded(p.base) ? tc_expand_launch(kind_of(p.base), Bsrc, ldBsrc, 0, n, l, 1,
                                                      reinterpret_cast<uint8_t *>(scratch + p.offXB),
                                                      p.rowbytes, s)
                                   : GF2_OK;
    if (d == 0)
        return run_base(p, A->data, A->stride_words, 0, Bsrc, ldBsrc, 0, C->data, C->stride_words, 0,
                        m, l, n, 1, accumulate, scratch, s, a_expanded, b_leaves && is_expanded(p.base));

    // top-down: the additions of Algorithm 4 (the left factor's above, the
    // right factor's here) for every sub-problem of each level; two levels
    // per launch while at least two remain (the middle level's operands then
    // never leave registers)
    int64_t cnt = 1;
    for (int j = 1; j <= d;) {
        const int step = split_step(j);
        if (b_leaves) {
            cnt *= (step == 2) ? 49 : 7;
            j += step;
            continue;
        }
        const int jt = j + step - 1;                       // level written
        const int64_t Lp = p.L >> (j - 1), Np = p.N >> (j - 1);
        SplitLaunch SB;
        SB.nparent = (int)cnt;
        if (tc) {
            // right factor held transposed (Np x Lp): quadrant NE of B^T is
            // (B_SW)^T and SW is (B_NE)^T; side 2 swaps their roles
            SB.side = 2; SB.rows = Np; SB.cols = Lp;
            if (j == 1) {
                SB.X = Bsrc; SB.ld = ldBsrc; SB.bs = 0; SB.vrows = n;
                SB.vcols = l;
            } else {
                SB.X = reinterpret_cast<const uint64_t *>(scratch + p.offB[j - 1]);
                SB.ld = p.ldB[j - 1]; SB.bs = p.slabB[j - 1]; SB.vrows = Np; SB.vcols = Lp;
            }
        } else {
            SB.side = 1; SB.rows = Lp; SB.cols = Np;
            if (j == 1) {
                SB.X = B->data; SB.ld = B->stride_words; SB.bs = 0; SB.vrows = l; SB.vcols = n;
            } else {
                SB.X = reinterpret_cast<const uint64_t *>(scratch + p.offB[j - 1]);
                SB.ld = p.ldB[j - 1]; SB.bs = p.slabB[j - 1]; SB.vrows = Lp; SB.vcols = Np;
            }
        }
        SB.out = reinterpret_cast<uint64_t *>(scratch + p.offB[jt]);
        SB.cld = p.ldB[jt]; SB.cbs = p.slabB[jt];
        if (fused && jt == d) {
            SB.xout = reinterpret_cast<uint8_t *>(scratch + p.offXB);
            SB.rowbytes = p.rowbytes;
            SB.xkind = kind_of(p.base) + 1;
        }
        const int rc = step == 2 ? sw_split2_launch(SB, s) : sw_split_launch(SB, s);
        if (rc) return rc;
        cnt *= (step == 2) ? 49 : 7;
        j += step;
    }
    if (b_only) {
        // B's leaves expanded here when its last level of additions did not
        const int64_t Ld = p.L >> d, Nd = p.N >> d;
        return (is_expanded(p.base) && !fused)
                   ? tc_expand_launch(kind_of(p.base), reinterpret_cast<const uint64_t *>(scratch + p.offB[d]),
                                      p.ldB[d], p.slabB[d], Nd, Ld, (int)cnt,
                                      reinterpret_cast<uint8_t *>(scratch + p.offXB), p.rowbytes, s)
                   : GF2_OK;
    }
    // all 7^d leaf products in one launch of the base case
    {
        const int64_t Md = p.M >> d, Ld = p.L >> d, Nd = p.N >> d;
        int rc = run_base(p, reinterpret_cast<const uint64_t *>(scratch + p.offA[d]), p.ldA[d], p.slabA[d],
                          reinterpret_cast<const uint64_t *>(scratch + p.offB[d]), p.ldB[d], p.slabB[d],
                          reinterpret_cast<uint64_t *>(scratch + p.offP[d]), p.ldP[d], p.slabP[d], Md, Ld,
                          Nd, (int)cnt, 0, scratch, s, a_expanded, fused || (b_leaves && is_expanded(p.base)));
        if (rc) return rc;
    }
    // bottom-up: the 7 final additions of Algorithm 4, Augment and Stack,
    // two levels per launch while at least two remain
    for (int j = d; j >= 1;) {
        const int step = (j >= 2) ? 2 : 1;
        const int jp = j - step;                           // level written (0 = C itself)
        cnt /= (step == 2) ? 49 : 7;
        const int64_t Mp = p.M >> jp, Np = p.N >> jp;
        CombineLaunch CL;
        CL.P = reinterpret_cast<const uint64_t *>(scratch + p.offP[j]);
        CL.pld = p.ldP[j]; CL.pbs = p.slabP[j];
        CL.rows = Mp; CL.cols = Np; CL.nparent = (int)cnt;
        if (jp == 0) {
            CL.X = C->data; CL.ld = C->stride_words; CL.bs = 0; CL.vrows = m; CL.vcols = n;
            CL.accumulate = accumulate;
        } else {
            CL.X = reinterpret_cast<uint64_t *>(scratch + p.offP[jp]);
            CL.ld = p.ldP[jp]; CL.bs = p.slabP[jp]; CL.vrows = Mp; CL.vcols = Np;
            CL.accumulate = 0;
        }
        int rc = step == 2 ? sw_combine2_launch(CL, s) : sw_combine_launch(CL, s);
        if (rc) return rc;
        j -= step;
    }
    return GF2_OK;
}

// ---------------------------------------------------------------- peeling
// Section 4's alternative to padding for sizes that do not halve evenly:
// Strassen-Winograd on the largest core whose rows are a multiple of 2^d and
// whose column counts are multiples of 128 * 2^d (the quadrants of every
// level then start on 16-byte boundaries), and the leftovers by base-case
// products on views of the same matrices:
//   C[0:M', 0:N']  = A[0:M', 0:L'] B[0:L', 0:N']   (recursion)
//                  ^ A[0:M', L':l] B[L':l, 0:N']   (leftover K entries)
//   C[0:M', N':n]  = A[0:M', :] B[:, N':n]          (leftover columns)
//   C[M':m, :]     = A[M':m, :] B                   (leftover rows)
// The paper peels one row or column per level; peeling the whole remainder
// once, at the top, gives the same product with fewer and larger launches.
struct PeelCore {
    int base, depth;
    int64_t M1, L1, N1;       // the core; all zero when nothing is peeled
};

PeelCore peel_core(int64_t m, int64_t l, int64_t n, const gf2_opts &o)
{
    PeelCore c;
    c.base = o.base == GF2_BASE_AUTO ? GF2_BASE_M4RM : o.base;
    c.depth = o.depth < 0 ? auto_depth(m, l, n, c.base) : o.depth;
    const int64_t rq = (int64_t)1 << c.depth, cq = (int64_t)128 << c.depth;
    c.M1 = m / rq * rq; c.L1 = l / cq * cq; c.N1 = n / cq * cq;
    if (c.depth == 0 || c.M1 == 0 || c.L1 == 0 || c.N1 == 0 || (c.M1 == m && c.L1 == l && c.N1 == n))
        c.M1 = c.L1 = c.N1 = 0;
    return c;
}

int mul_peeled(gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const gf2_opts &o, void *stream)
{
    const int64_t m = A->rows, l = A->cols, n = B->cols;
    const PeelCore pc = peel_core(m, l, n, o);
    const int base = pc.base, d = pc.depth;
    const int64_t M1 = pc.M1, L1 = pc.L1, N1 = pc.N1;
    gf2_opts plain = o;
    plain.peel = 0;
    plain.base = base;
    if (M1 == 0) {
        plain.depth = d;
        return gf2_mul(C, A, B, &plain, stream);      // nothing to peel, or no core
    }
    auto view = [](const gf2_mat *X, int64_t r0, int64_t c0, int64_t rows, int64_t cols) {
        gf2_mat v = *X;
        v.data = X->data + r0 * X->stride_words + c0 / 64;   // c0 is a multiple of 128
        v.rows = rows;
        v.cols = cols;
        return v;
    };
    int rc;
    // core
    {
        gf2_mat a = view(A, 0, 0, M1, L1), b = view(B, 0, 0, L1, N1), c = view(C, 0, 0, M1, N1);
        gf2_opts oc = plain;
        oc.depth = d;
        if ((rc = gf2_mul(&c, &a, &b, &oc, stream))) return rc;
    }
    gf2_opts ob = plain;
    ob.depth = 0;
    if (L1 < l) {
        gf2_mat a = view(A, 0, L1, M1, l - L1), b = view(B, L1, 0, l - L1, N1), c = view(C, 0, 0, M1, N1);
        gf2_opts oa = ob;
        oa.accumulate = 1;
        if ((rc = gf2_mul(&c, &a, &b, &oa, stream))) return rc;
    }
    if (N1 < n) {
        gf2_mat a = view(A, 0, 0, M1, l), b = view(B, 0, N1, l, n - N1), c = view(C, 0, N1, M1, n - N1);
        if ((rc = gf2_mul(&c, &a, &b, &ob, stream))) return rc;
    }
    if (M1 < m) {
        gf2_mat a = view(A, M1, 0, m - M1, l), c = view(C, M1, 0, m - M1, n);
        if ((rc = gf2_mul(&c, &a, B, &ob, stream))) return rc;
    }
    return GF2_OK;
}

// ---------------------------------------------------------------- autotuning
// gf2_mul with an automatic base case and/or depth on a large product
// (m*l*n >= 2^36) asks the autotuner: a cached choice for this shape, or,
// on the first call, every candidate (base in {M4RM, TC}, depth d0-1..d0+1
// around the cutoff rule's d0) is timed once on the caller's operands and
// the fastest is cached.  GF2_AUTOTUNE=0 turns this off.
bool autotune_enabled()
{
    const char *e = getenv("GF2_AUTOTUNE");
    return !(e && e[0] == '0');
}

std::string tune_key(int64_t m, int64_t l, int64_t n, const gf2_opts &o)
{
    char b[160];
    snprintf(b, sizeof b, "mul-%s-%lldx%lldx%lld-b%d-d%d-k%d-t%d", arch_tag().c_str(), (long long)m,
             (long long)l, (long long)n, o.base, o.depth, o.k, o.t);
    return b;
}

constexpr size_t kTuneScratchCap = (size_t)48 << 30;   // bytes of scratch a timed candidate may need

// The plan(s) to run: one resolved option set, or the candidates to time.
bool wants_tuning(int64_t m, int64_t l, int64_t n, const gf2_opts &o, std::vector<gf2_opts> *cands,
                  std::string *key)
{
    cands->clear();
    const double vol = (double)m * (double)l * (double)n;
    const bool automatic = (o.base == GF2_BASE_AUTO || o.depth < 0);
    if (!automatic || o.accumulate || vol < 68719476736.0 || !autotune_enabled()) {
        cands->push_back(o);
        return false;
    }
    *key = tune_key(m, l, n, o);
    std::string v;
    int b = 0, d = 0;
    if (tune_get(*key, &v) && sscanf(v.c_str(), "b%dd%d", &b, &d) == 2) {
        gf2_opts r = o;
        r.base = b;
        r.depth = d;
        cands->push_back(r);
        return false;
    }
    std::vector<int> bases;
    if (o.base != GF2_BASE_AUTO) bases.push_back(o.base);
    else {
        bases.push_back(GF2_BASE_M4RM);
        if (tc_fp8_available()) {
            bases.push_back(GF2_BASE_TC_FP4);
            bases.push_back(GF2_BASE_TC_FP8);
        }
    }
    for (int base : bases) {
        std::vector<int> depths;
        if (o.depth >= 0) depths.push_back(o.depth);
        else {
            const int d0 = auto_depth(m, l, n, base);
            for (int d = d0 - 1; d <= d0 + 1; ++d) {
                const int64_t mn = std::min(m, std::min(l, n));
                if (d < 0 || d > 6 || (mn >> d) < 1024) continue;
                depths.push_back(d);
            }
        }
        for (int d : depths) {
            gf2_opts r = o;
            r.base = base;
            r.depth = d;
            // skip plans whose scratch alone would take a large share of the
            // device (expanded tensor-core operands deep in the recursion)
            Plan pl;
            if (make_plan(m, l, n, r, &pl) != GF2_OK || pl.bytes > kTuneScratchCap) continue;
            cands->push_back(r);
        }
    }
    if (cands->empty()) cands->push_back(o);
    if (cands->size() <= 1) return false;
    return true;
}

size_t staged_bytes(const gf2_mat *M)
{
    return (size_t)(M->rows * even_up(words_of(M->cols))) * 8;
}

// Padding or peeling for this shape (opts.peel == -1): 0 = pad, 1 = peel,
// 2 = C already holds A B (computed while timing), or a negative status.
// Where the autotuner does not run (small products, accumulate, tuning
// off, or nothing to peel) the answer is padding; otherwise the first call
// for a shape times both on the caller's operands and caches the faster.
int choose_peel(gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const gf2_opts &o, void *stream)
{
    const int64_t m = A->rows, l = A->cols, n = B->cols;
    const double vol = (double)m * (double)l * (double)n;
    if (o.accumulate || vol < 68719476736.0 || !autotune_enabled()) return 0;
    if (!peel_core(m, l, n, o).M1) return 0;
    const std::string key = "peel|" + tune_key(m, l, n, o);
    std::string v;
    if (tune_get(key, &v)) return v == "peel" ? 1 : 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gf2_opts op = o, oq = o;
    op.peel = 0;
    oq.peel = 1;
    int rc = gf2_mul(C, A, B, &op, stream);              // warms (and tunes) the padded plan
    if (rc) return rc;
    ScopedEvents<3> ev;
    if ((rc = ev.create())) return rc;
    cudaEvent_t *e = ev.e;
    float t_pad = 0.f, t_peel = 0.f;
    cudaEventRecord(e[0], s);
    rc = gf2_mul(C, A, B, &op, stream);
    cudaEventRecord(e[1], s);
    if (!rc) rc = mul_peeled(C, A, B, oq, stream);
    cudaEventRecord(e[2], s);
    if (!rc && cudaEventSynchronize(e[2]) == cudaSuccess) {
        cudaEventElapsedTime(&t_pad, e[0], e[1]);
        cudaEventElapsedTime(&t_peel, e[1], e[2]);
    }
    if (rc) return rc;
    tune_put(key, t_peel < t_pad ? "peel" : "pad");
    return 2;
}

}  // namespace

namespace gf2 {

// gf2_mul for device operands with caller-owned scratch (no allocation):
// the checks of gf2_mul, then the cutoff rule's plan (no autotuning, odd
// sizes padded; peeling is refused) and the device path on `scratch`.
int mul_with_scratch(gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const gf2_opts *opts,
                     void *scratch, size_t scratch_bytes, void *stream)
{
    int rc;
    if ((rc = check_mat(A)) || (rc = check_mat(B)) || (rc = check_mat(C))) return rc;
    if (A->cols != B->rows || C->rows != A->rows || C->cols != B->cols) return GF2_EINVAL;
    const gf2_opts o = resolve(opts);
    if ((rc = check_opts(o))) return rc;
    if (o.peel == 1) return GF2_EUNSUPPORTED;
    if (overlaps(C, A) || overlaps(C, B)) return GF2_EALIAS;
    int dev = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    const gf2_mat *mats[3] = {A, B, C};
    for (const gf2_mat *M : mats)
        if (M->rows && M->cols && M->device != dev) return GF2_EINVAL;
    Plan p;
    if ((rc = make_plan(A->rows, A->cols, B->cols, o, &p))) return rc;
    if (p.bytes > scratch_bytes) return GF2_ESCRATCH;
    return mul_device(C, A, B, p, o.accumulate, static_cast<char *>(scratch),
                      static_cast<cudaStream_t>(stream));
}

}  // namespace gf2

namespace {

// Row blocks of the host-buffer product: rows per block at least kHostBlockRows,
// at most kHostBlocks blocks.  Measured at n = 32768 (FP4, depth 2) per call:
// 1 block 8.80 ms, 2 blocks 8.52, 4 blocks 8.63 (the leaf products of thinner
// blocks lose more on the MMA launches than the extra overlap hides).
constexpr int64_t kHostBlockRows = 8192;
constexpr int kHostBlocks = 2;

int host_row_blocks(int64_t m, const Plan &p)
{
    if (p.cubic) return 1;
    return (int)std::max<int64_t>(1, std::min<int64_t>(kHostBlocks, m / kHostBlockRows));
}

// C = A B with A, B and C in host memory, A and C in nblk row blocks: every
// row of C depends only on the same row of A, so block i of C is the product
// A_i B, and the right factor's transposition, additions and expansion (the
// same for every block) are done once, first.  The copies run on side
// streams: B (in row blocks, each transposed on a second side stream for the
// tensor-core base cases while the next crosses the link), then A_0, A_1,
// ...; B's additions run while A_0 crosses the link, the product of block i
// waits for A_i, and C_i's copy back to the host (the other direction of the
// link) runs while block i + 1 is computed.
int mul_host_blocks(gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const gf2_opts &oc, int nblk,
                    cudaStream_t s, int dev)
{
    const int64_t m = A->rows, l = A->cols, n = B->cols;
    const int64_t mb = round_up((m + nblk - 1) / nblk, 64);
    Plan p;
    int rc = make_plan(mb, l, n, oc, &p);
    if (rc) return rc;
    size_t total = (p.bytes + 255) & ~(size_t)255;
    const size_t offA = total;
    total += (staged_bytes(A) + 255) & ~(size_t)255;
    const size_t offB = total;
    total += (staged_bytes(B) + 255) & ~(size_t)255;
    const size_t offC = total;
    total += (staged_bytes(C) + 255) & ~(size_t)255;
    void *scratch = nullptr;
    ArenaHold hold;
    if ((rc = arena_get(s, total, &scratch, &hold))) return rc;
    char *base = static_cast<char *>(scratch);
    cudaStream_t sIn = side_stream(dev, 0), sT = side_stream(dev, 1), sOut = side_stream(dev, 2);
    if (!sIn || !sT || !sOut) return GF2_ECUDA;
    struct Events {
        std::vector<cudaEvent_t> e;
        ~Events() { for (cudaEvent_t x : e) cudaEventDestroy(x); }
        cudaEvent_t make()
        {
            cudaEvent_t x = nullptr;
            if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) return nullptr;
            e.push_back(x);
            return x;
        }
    } ev;
    SideJoin join{s, {sIn, sT, sOut}};
    gf2_mat dA = *A, dB = *B, dC = *C;
    dA.data = reinterpret_cast<uint64_t *>(base + offA);
    dA.stride_words = even_up(words_of(l));
    dA.device = dev;
    dB.data = reinterpret_cast<uint64_t *>(base + offB);
    dB.stride_words = even_up(words_of(n));
    dB.device = dev;
    dC.data = reinterpret_cast<uint64_t *>(base + offC);
    dC.stride_words = even_up(words_of(n));
    dC.device = dev;
    auto rows_of = [&](int i, int64_t *r0) {
        *r0 = (int64_t)i * mb;
        return std::max<int64_t>(0, std::min<int64_t>(m, *r0 + mb) - *r0);
    };
    // the input copies, in the order the products need them
    cudaEvent_t start = ev.make();
    if (!start) return GF2_ECUDA;
    GF2_CUDA_TRY(cudaEventRecord(start, s));                // after the caller's earlier work
    GF2_CUDA_TRY(cudaStreamWaitEvent(sIn, start, 0));
    std::vector<cudaEvent_t> a_ready(nblk);
    auto copy_A = [&](int i) {
        int64_t r0 = 0;
        const int64_t rows = rows_of(i, &r0);
        if (rows)
            GF2_CUDA_TRY(cudaMemcpy2DAsync(dA.data + r0 * dA.stride_words, dA.stride_words * 8,
                                           A->data + r0 * A->stride_words, A->stride_words * 8,
                                           words_of(l) * 8, rows, cudaMemcpyHostToDevice, sIn));
        if (!(a_ready[i] = ev.make())) return GF2_ECUDA;
        GF2_CUDA_TRY(cudaEventRecord(a_ready[i], sIn));
        return GF2_OK;
    };
    cudaEvent_t b_ready = ev.make();
    if (!b_ready) return GF2_ECUDA;
    const bool tr = is_tc(p.base);
    if (tr) {
        // row block [r0, r1) of B is columns [r0, r1) of B^T, words r0 / 64
        // onwards of its rows
        uint64_t *Bt = reinterpret_cast<uint64_t *>(base + p.offBt);
        const int64_t ch = std::max<int64_t>(256, (l / 8 + 255) / 256 * 256);
        for (int64_t r0 = 0; r0 < l; r0 += ch) {
            const int64_t r1 = std::min(l, r0 + ch);
            uint64_t *dst = dB.data + r0 * dB.stride_words;
            GF2_CUDA_TRY(cudaMemcpy2DAsync(dst, dB.stride_words * 8, B->data + r0 * B->stride_words,
                                           B->stride_words * 8, words_of(n) * 8, r1 - r0,
                                           cudaMemcpyHostToDevice, sIn));
            cudaEvent_t landed = ev.make();
            if (!landed) return GF2_ECUDA;
            GF2_CUDA_TRY(cudaEventRecord(landed, sIn));
            GF2_CUDA_TRY(cudaStreamWaitEvent(sT, landed, 0));
            DMat T{Bt + r0 / 64, n, r1 - r0, p.ldBt};
            DMat X{dst, r1 - r0, n, dB.stride_words};
            if ((rc = transpose_launch(T, X, sT))) return rc;
        }
        GF2_CUDA_TRY(cudaEventRecord(b_ready, sT));
    } else {
        GF2_CUDA_TRY(cudaMemcpy2DAsync(dB.data, dB.stride_words * 8, B->data, B->stride_words * 8,
                                       words_of(n) * 8, l, cudaMemcpyHostToDevice, sIn));
        GF2_CUDA_TRY(cudaEventRecord(b_ready, sIn));
    }
    for (int i = 0; i < nblk; ++i)
        if ((rc = copy_A(i))) return rc;
    // B's leaves, then the products, each block's C copied back as soon as
    // it is complete
    if ((rc = mul_device(&dC, &dA, &dB, p, 0, base, s, b_ready, tr, false, true))) return rc;
    for (int i = 0; i < nblk; ++i) {
        int64_t r0 = 0;
        const int64_t rows = rows_of(i, &r0);
        if (!rows) break;
        Plan pi = p;
        pi.m = rows;
        gf2_mat Ai = dA, Ci = dC;
        Ai.data = dA.data + r0 * dA.stride_words;
        Ai.rows = rows;
        Ci.data = dC.data + r0 * dC.stride_words;
        Ci.rows = rows;
        GF2_CUDA_TRY(cudaStreamWaitEvent(s, a_ready[i], 0));
        rc = mul_device(&Ci, &Ai, &dB, pi, 0, base, s, nullptr, false, true);
        if (rc) return rc;
        cudaEvent_t c_done = ev.make();
        if (!c_done) return GF2_ECUDA;
        GF2_CUDA_TRY(cudaEventRecord(c_done, s));
        GF2_CUDA_TRY(cudaStreamWaitEvent(sOut, c_done, 0));
        GF2_CUDA_TRY(cudaMemcpy2DAsync(C->data + r0 * C->stride_words, C->stride_words * 8, Ci.data,
                                       Ci.stride_words * 8, words_of(n) * 8, rows, cudaMemcpyDeviceToHost,
                                       sOut));
    }
    cudaEvent_t out_done = ev.make();
    if (!out_done) return GF2_ECUDA;
    GF2_CUDA_TRY(cudaEventRecord(out_done, sOut));
    GF2_CUDA_TRY(cudaStreamWaitEvent(s, out_done, 0));
    GF2_CUDA_TRY(cudaStreamSynchronize(s));
    join.armed = false;                  // everything queued has been waited for
    return GF2_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

void gf2_default_opts(gf2_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->base = GF2_BASE_AUTO;
    o->depth = -1;
    o->peel = -1;
}

const char *gf2_strerror(int status)
{
    switch (status) {
    case GF2_OK: return "ok";
    case GF2_EINVAL: return "invalid argument (null pointer, negative or mismatched dimensions, bad option)";
    case GF2_EALIAS: return "output overlaps an input";
    case GF2_ELAYOUT: return "bad layout (stride below ceil(cols/64), odd stride, or data not 16-byte aligned)";
    case GF2_ENOMEM: return "out of memory";
    case GF2_ECUDA: return "CUDA error";
    case GF2_ETIMEOUT: return "device-side wait timed out";
    case GF2_EUNSUPPORTED: return "unsupported option for this shape or device";
    case GF2_EMISMATCH: return "verification failed";
    case GF2_ESCRATCH: return "the plan needs more scratch than the fixed no-allocation buffer holds";
    default: return "unknown status";
    }
}

int gf2_alloc(gf2_mat *M, int64_t rows, int64_t cols)
{
    if (!M || rows < 0 || cols < 0) return GF2_EINVAL;
    memset(M, 0, sizeof(*M));
    M->rows = rows;
    M->cols = cols;
    M->stride_words = even_up(words_of(cols));
    int dev = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    M->device = dev;
    if (rows == 0 || cols == 0) return GF2_OK;
    void *p = nullptr;
    const size_t bytes = (size_t)(rows * M->stride_words) * 8;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        M->data = nullptr;
        return GF2_ENOMEM;
    }
    if (cudaMemset(p, 0, bytes) != cudaSuccess) {
        cudaFree(p);
        return GF2_ECUDA;
    }
    M->data = static_cast<uint64_t *>(p);
    return GF2_OK;
}

int gf2_free(gf2_mat *M)
{
    if (!M) return GF2_EINVAL;
    if (M->data) {
        if (M->device == GF2_HOST) return GF2_EINVAL;
        GF2_CUDA_TRY(cudaFree(M->data));
    }
    M->data = nullptr;
    return GF2_OK;
}

int64_t gf2_scratch_bytes(int64_t m, int64_t l, int64_t n, const gf2_opts *opts)
{
    const gf2_opts o = resolve(opts);
    if (m < 0 || l < 0 || n < 0 || check_opts(o)) return GF2_EINVAL;
    Plan p;
    const int rc = make_plan(m, l, n, o, &p);
    if (rc) return rc;
    return (int64_t)p.bytes;
}

int gf2_describe_plan(int64_t m, int64_t l, int64_t n, const gf2_opts *opts, char *buf, int32_t cap)
{
    if (!buf || cap <= 0) return GF2_EINVAL;
    const gf2_opts o = resolve(opts);
    if (m < 0 || l < 0 || n < 0) return GF2_EINVAL;
    int rc = check_opts(o);
    if (rc) return rc;
    std::vector<gf2_opts> cands;
    std::string key;
    gf2_opts eff = o;
    std::string peeled;
    int policy = o.peel;
    if (policy == -1) {      // the autotuner's cached choice for this shape, else padding
        std::string v;
        policy = (tune_get("peel|" + tune_key(m, l, n, o), &v) && v == "peel") ? 1 : 0;
    }
    if (policy == 1) {
        const PeelCore pc = peel_core(m, l, n, o);
        eff.peel = 0;
        eff.base = pc.base;
        eff.depth = pc.depth;
        if (pc.M1) {
            char pb[160];
            snprintf(pb, sizeof pb, " peel core=%lldx%lldx%lld leftover rows=%lld cols=%lld k=%lld",
                     (long long)pc.M1, (long long)pc.L1, (long long)pc.N1, (long long)(m - pc.M1),
                     (long long)(n - pc.N1), (long long)(l - pc.L1));
            peeled = pb;
            m = pc.M1; l = pc.L1; n = pc.N1;              // the recursion's plan is the core's
        }
    }
    if (!wants_tuning(m, l, n, eff, &cands, &key)) eff = cands[0];
    Plan p;
    rc = make_plan(m, l, n, eff, &p);
    if (rc) return rc;
    std::string t = plan_text(p) + peeled;
    if (p.base == GF2_BASE_M4RM && !p.cubic && m > 0 && n > 0) {
        int k = o.k, tt = o.t, bm = 0, ks = 0;
        const int d = p.depth;
        int batch = 1;
        for (int j = 0; j < d; ++j) batch *= 7;
        m4rm_pick(p.M >> d, p.L >> d, p.N >> d, batch, &k, &tt, &bm, &ks);
        char extra[128];
        snprintf(extra, sizeof extra, " m4rm_k=%d m4rm_t=%d tile_rows=%d ksplit=%d", k, tt, bm, ks);
        t += extra;
    }
    snprintf(buf, (size_t)cap, "%s", t.c_str());
    return GF2_OK;
}

int gf2_reserve_scratch(int64_t bytes, void *stream)
{
    if (bytes < 0) return GF2_EINVAL;
    void *p = nullptr;
    ArenaHold hold;
    return arena_get(static_cast<cudaStream_t>(stream), (size_t)bytes, &p, &hold);
}

int gf2_release_scratch(void)
{
    int dev = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    gf2::batched_release();
    gf2::tc_batched_release();
    std::vector<std::shared_ptr<Arena>> gone;
    {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        for (auto it = g_arenas.begin(); it != g_arenas.end();) {
            if (it->first.first == dev) {
                gone.push_back(it->second);
                it = g_arenas.erase(it);
            } else {
                ++it;
            }
        }
    }
    // wait for callers still queueing work into these arenas, then for the
    // device; an arena still held elsewhere is freed when its holder drops it
    for (auto &a : gone) std::lock_guard<std::mutex> wait(a->mu);
    GF2_CUDA_TRY(cudaDeviceSynchronize());
    gone.clear();
    return GF2_OK;
}

int64_t gf2_launch_count(void) { return (int64_t)gf2::launch_count(); }

int gf2_profile_enable(int32_t on) { return gf2::profile_enable(on); }

int gf2_selftest_wait(int64_t limit_cycles, void *stream)
{
    if (limit_cycles < 1 || limit_cycles > 4000000000ll) return GF2_EINVAL;
    return gf2::wait_selftest_launch(limit_cycles, static_cast<cudaStream_t>(stream));
}

int gf2_device_status(void *stream)
{
    unsigned int v = 0;
    const int rc = gf2::tc_status_read_and_clear(&v, static_cast<cudaStream_t>(stream));
    if (rc) return rc;
    return v ? -(int)v : GF2_OK;
}

int gf2_profile_read(int32_t family, double *ms, int64_t *launches)
{
    long long n = 0;
    const int rc = gf2::profile_read(family, ms, &n);
    if (launches) *launches = (int64_t)n;
    return rc;
}

const char *gf2_profile_name(int32_t family)
{
    static const char *names[PF_COUNT] = {"m4rm", "tc_fp8", "sw_split", "sw_combine", "transpose",
                                          "random", "freivalds", "make_table", "batched", "tc_s8", "tc_b1",
                                          "tc_fp4", "expand"};
    if (family < 0 || family >= PF_COUNT) return nullptr;
    return names[family];
}

int gf2_mul(gf2_mat *C, const gf2_mat *A, const gf2_mat *B, const gf2_opts *opts, void *stream)
{
    int rc;
    if ((rc = check_mat(A)) || (rc = check_mat(B)) || (rc = check_mat(C))) return rc;
    if (A->cols != B->rows || C->rows != A->rows || C->cols != B->cols) return GF2_EINVAL;
    const gf2_opts o = resolve(opts);
    if ((rc = check_opts(o))) return rc;
    if (overlaps(C, A) || overlaps(C, B)) return GF2_EALIAS;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    const gf2_mat *mats[3] = {A, B, C};
    for (const gf2_mat *M : mats)
        if (M->device != GF2_HOST && M->device != dev && M->rows && M->cols) return GF2_EINVAL;

    const int64_t m = A->rows, l = A->cols, n = B->cols;
    if (o.peel && A->device != GF2_HOST && B->device != GF2_HOST && C->device != GF2_HOST) {
        if (o.peel == 1) return mul_peeled(C, A, B, o, stream);
        const int choice = choose_peel(C, A, B, o, stream);
        if (choice < 0) return choice;                   // an error
        if (choice == 2) return GF2_OK;                  // C computed while choosing
        if (choice == 1) return mul_peeled(C, A, B, o, stream);
    }
    // candidate plans: one, or several when the autotuner picks base / depth
    std::vector<gf2_opts> cands;
    std::string tkey;
    const bool tuning = wants_tuning(m, l, n, o, &cands, &tkey);
    std::vector<Plan> plans(cands.size());
    size_t most = 0;
    for (size_t i = 0; i < cands.size(); ++i) {
        if ((rc = make_plan(m, l, n, cands[i], &plans[i]))) return rc;
        most = std::max(most, plans[i].bytes);
    }

    const bool hA = A->device == GF2_HOST, hB = B->device == GF2_HOST, hC = C->device == GF2_HOST;
    if (hA && hB && hC && !tuning && !o.accumulate && m && l && n) {
        const int nblk = host_row_blocks(m, plans[0]);
        if (nblk > 1) return mul_host_blocks(C, A, B, cands[0], nblk, s, dev);
    }
    size_t total = (most + 255) & ~(size_t)255;
    size_t offA = total, offB = 0, offC = 0;
    if (hA) { offA = total; total += (staged_bytes(A) + 255) & ~(size_t)255; }
    if (hB) { offB = total; total += (staged_bytes(B) + 255) & ~(size_t)255; }
    if (hC) { offC = total; total += (staged_bytes(C) + 255) & ~(size_t)255; }
    void *scratch = nullptr;
    ArenaHold hold;
    if ((rc = arena_get(s, total, &scratch, &hold))) return rc;
    char *base = static_cast<char *>(scratch);

    gf2_mat dA = *A, dB = *B, dC = *C;
    bool bt_ready = false;                   // B^T already in the plan's scratch
    // with both factors on the host, B is copied on a side stream while the
    // left factor's Strassen-Winograd additions run (they need only A)
    cudaEvent_t b_ready = nullptr, s_ready = nullptr;
    cudaStream_t sB = s;
    if (hA && hB && m && l && n) {
        sB = side_stream(dev);
        if (!(sB && cudaEventCreateWithFlags(&b_ready, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&s_ready, cudaEventDisableTiming) == cudaSuccess)) {
            cudaGetLastError();
            if (b_ready) cudaEventDestroy(b_ready);
            if (s_ready) cudaEventDestroy(s_ready);
            b_ready = s_ready = nullptr;
            sB = s;
        }
    }
    struct EventGuard {
        cudaEvent_t a, b;
        ~EventGuard() { if (a) cudaEventDestroy(a); if (b) cudaEventDestroy(b); }
    } guard{b_ready, s_ready};
    SideJoin join{s, {sB, side_stream(dev, 1), nullptr}};
    join.armed = hA || hB || hC;
    if (hA && m && l) {
        dA.data = reinterpret_cast<uint64_t *>(base + offA);
        dA.stride_words = even_up(words_of(l));
        dA.device = dev;
        GF2_CUDA_TRY(cudaMemcpy2DAsync(dA.data, dA.stride_words * 8, A->data, A->stride_words * 8,
                                       words_of(l) * 8, m, cudaMemcpyHostToDevice, s));
    }
    if (s_ready) {
        // B's copy follows A's (they would share the link) and everything
        // queued on s before it; it then overlaps A's additions
        GF2_CUDA_TRY(cudaEventRecord(s_ready, s));
        GF2_CUDA_TRY(cudaStreamWaitEvent(sB, s_ready, 0));
    }
    if (hB && l && n) {
        dB.data = reinterpret_cast<uint64_t *>(base + offB);
        dB.stride_words = even_up(words_of(n));
        dB.device = dev;
        cudaStream_t sT = (b_ready && !tuning && is_tc(plans[0].base) && !plans[0].cubic) ? side_stream(dev, 1)
                                                                                           : nullptr;
        if (sT) {
            // the tensor-core base cases read B transposed: B is copied in row
            // blocks on one side stream, and each block is transposed on a
            // second one while the next crosses the link (row block [r0, r1)
            // of B is columns [r0, r1) of B^T, words r0 / 64 onwards of its
            // rows)
            uint64_t *Bt = reinterpret_cast<uint64_t *>(base + plans[0].offBt);
            const int64_t ch = std::max<int64_t>(256, (l / 8 + 255) / 256 * 256);
            for (int64_t r0 = 0; r0 < l; r0 += ch) {
                const int64_t r1 = std::min(l, r0 + ch);
                uint64_t *dst = dB.data + r0 * dB.stride_words;
                GF2_CUDA_TRY(cudaMemcpy2DAsync(dst, dB.stride_words * 8, B->data + r0 * B->stride_words,
                                               B->stride_words * 8, words_of(n) * 8, r1 - r0,
                                               cudaMemcpyHostToDevice, sB));
                cudaEvent_t landed = nullptr;
                GF2_CUDA_TRY(cudaEventCreateWithFlags(&landed, cudaEventDisableTiming));
                const cudaError_t e1 = cudaEventRecord(landed, sB);
                const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(sT, landed, 0) : e1;
                cudaEventDestroy(landed);                 // released once the wait has passed
                if (e2 != cudaSuccess) return GF2_ECUDA;
                DMat T{Bt + r0 / 64, n, r1 - r0, plans[0].ldBt};
                DMat X{dst, r1 - r0, n, dB.stride_words};
                if ((rc = transpose_launch(T, X, sT))) return rc;
            }
            bt_ready = true;
            GF2_CUDA_TRY(cudaEventRecord(b_ready, sT));
        } else {
            GF2_CUDA_TRY(cudaMemcpy2DAsync(dB.data, dB.stride_words * 8, B->data, B->stride_words * 8,
                                           words_of(n) * 8, l, cudaMemcpyHostToDevice, sB));
            if (b_ready) GF2_CUDA_TRY(cudaEventRecord(b_ready, sB));
        }
    }
    if (hC && m && n) {
        dC.data = reinterpret_cast<uint64_t *>(base + offC);
        dC.stride_words = even_up(words_of(n));
        dC.device = dev;
        if (o.accumulate)
            GF2_CUDA_TRY(cudaMemcpy2DAsync(dC.data, dC.stride_words * 8, C->data, C->stride_words * 8,
                                           words_of(n) * 8, m, cudaMemcpyHostToDevice, s));
    }
    if (!tuning) {
        rc = mul_device(&dC, &dA, &dB, plans[0], o.accumulate, base, s, b_ready, bt_ready);
        if (rc) return rc;
    } else {
        // time every candidate on these operands (each computes the same C)
        ScopedEvents<2> ev;
        if ((rc = ev.create())) return rc;
        cudaEvent_t e0 = ev.e[0], e1 = ev.e[1];
        size_t best = 0;
        float best_ms = 1e30f;
        if (b_ready) GF2_CUDA_TRY(cudaStreamWaitEvent(s, b_ready, 0));
        for (size_t i = 0; i < plans.size(); ++i) {
            cudaEventRecord(e0, s);
            rc = mul_device(&dC, &dA, &dB, plans[i], 0, base, s);
            cudaEventRecord(e1, s);
            float ms = 1e30f;
            if (rc == GF2_OK && cudaEventSynchronize(e1) == cudaSuccess)
                cudaEventElapsedTime(&ms, e0, e1);
            if (rc == GF2_OK && ms < best_ms) { best_ms = ms; best = i; }
            if (rc) break;
        }
        if (rc) return rc;
        if (best + 1 != plans.size()) {     // leave the chosen plan's result, as a plain call would
            rc = mul_device(&dC, &dA, &dB, plans[best], 0, base, s);
            if (rc) return rc;
        }
        char v[32];
        snprintf(v, sizeof v, "b%dd%d", plans[best].base, plans[best].depth);
        tune_put(tkey, v);
    }
    if (hC && m && n) {
        GF2_CUDA_TRY(cudaMemcpy2DAsync(C->data, C->stride_words * 8, dC.data, dC.stride_words * 8,
                                       words_of(n) * 8, m, cudaMemcpyDeviceToHost, s));
    }
    if (hA || hB || hC) GF2_CUDA_TRY(cudaStreamSynchronize(s));
    join.armed = false;
    return GF2_OK;
}

int gf2_mul_batched_ex(gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[],
                       int32_t count, const gf2_opts *opts, int32_t variant, int32_t *chosen, void *stream)
{
    if (count < 0 || (count > 0 && (!C || !A || !B))) return GF2_EINVAL;
    const gf2_opts o = resolve(opts);
    int rc = check_opts(o);
    if (rc) return rc;
    if (variant < -1 || variant >= gf2::batched_variant_count()) return GF2_EINVAL;
    int dev = 0;
    for (int i = 0; i < count; ++i) {
        if (!C[i] || !A[i] || !B[i]) return GF2_EINVAL;
        if ((rc = check_mat(A[i])) || (rc = check_mat(B[i])) || (rc = check_mat(C[i]))) return rc;
        if (A[i]->cols != B[i]->rows || C[i]->rows != A[i]->rows || C[i]->cols != B[i]->cols)
            return GF2_EINVAL;
        if (A[i]->device == GF2_HOST || B[i]->device == GF2_HOST || C[i]->device == GF2_HOST)
            return GF2_EINVAL;
        if (overlaps(C[i], A[i]) || overlaps(C[i], B[i])) return GF2_EALIAS;
    }
    if (chosen) *chosen = -1;
    if (count == 0) return GF2_OK;
    GF2_CUDA_TRY(cudaGetDevice(&dev));
    for (int i = 0; i < count; ++i) {
        const gf2_mat *ms[3] = {A[i], B[i], C[i]};
        for (const gf2_mat *M : ms)
            if (M->rows && M->cols && M->device != dev) return GF2_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // products for the single persistent launch, and the rest (recursing or
    // tensor-core plans) run one by one
    std::vector<gf2_mat *> bc, tcc;
    std::vector<const gf2_mat *> ba, bb, tca, tcb;
    for (int i = 0; i < count; ++i) {
        const int64_t m = A[i]->rows, l = A[i]->cols, n = B[i]->cols;
        const int base = o.base == GF2_BASE_AUTO ? GF2_BASE_M4RM : o.base;
        const int depth = o.depth < 0 ? auto_depth(m, l, n, base) : o.depth;
        if (base == GF2_BASE_M4RM && depth == 0) {
            bc.push_back(C[i]);
            ba.push_back(A[i]);
            bb.push_back(B[i]);
        } else if (is_expanded(base) && depth == 0 && tc_fp8_available()) {
            tcc.push_back(C[i]);
            tca.push_back(A[i]);
            tcb.push_back(B[i]);
        } else {
            rc = gf2_mul(C[i], A[i], B[i], &o, stream);
            if (rc) return rc;
        }
    }
    if (!tcc.empty()) {
        rc = gf2::tc_batched_mul(tcc.data(), tca.data(), tcb.data(), (int)tcc.size(), o.accumulate,
                                 kind_of(o.base), s);
        if (rc) return rc;
    }
    if (bc.empty()) return GF2_OK;
    int ch = -1;
    rc = gf2::batched_mul(bc.data(), ba.data(), bb.data(), (int)bc.size(), o.accumulate, variant, s, &ch);
    if (chosen) *chosen = ch;
    return rc;
}

int gf2_mul_batched(gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[],
                    int32_t count, const gf2_opts *opts, void *stream)
{
    return gf2_mul_batched_ex(C, A, B, count, opts, -1, nullptr, stream);
}

int32_t gf2_batched_variant_count(void) { return gf2::batched_variant_count(); }

const char *gf2_batched_variant_name(int32_t variant) { return gf2::batched_variant_name(variant); }

int gf2_sw_split(uint64_t *out, int64_t slab_words, const gf2_mat *X, int32_t side, void *stream)
{
    int rc = check_mat(X);
    if (rc) return rc;
    if (!out || side < 0 || side > 2) return GF2_EINVAL;
    if ((X->rows & 1) || (X->cols % 128)) return GF2_EINVAL;
    const int64_t cld = even_up(X->cols / 128);
    if (slab_words < (X->rows / 2) * cld || !aligned16(out) || (slab_words & 1)) return GF2_ELAYOUT;
    if (X->rows == 0 || X->cols == 0) return GF2_OK;
    if ((X->cols / 128) & 1) return GF2_EUNSUPPORTED;   // quadrants must be whole 16-byte chunks
    SplitLaunch L;
    L.X = X->data; L.ld = X->stride_words; L.bs = 0;
    L.rows = X->rows; L.cols = X->cols; L.vrows = X->rows; L.vcols = X->cols;
    L.out = out; L.cld = cld; L.cbs = slab_words; L.nparent = 1; L.side = side;
    return sw_split_launch(L, static_cast<cudaStream_t>(stream));
}

int gf2_sw_combine(gf2_mat *C, const uint64_t *P, int64_t slab_words, void *stream)
{
    int rc = check_mat(C);
    if (rc) return rc;
    if (!P || (C->rows & 1) || (C->cols % 128)) return GF2_EINVAL;
    const int64_t pld = even_up(C->cols / 128);
    if (slab_words < (C->rows / 2) * pld || !aligned16(P) || (slab_words & 1)) return GF2_ELAYOUT;
    if (C->rows == 0 || C->cols == 0) return GF2_OK;
    if ((C->cols / 128) & 1) return GF2_EUNSUPPORTED;
    CombineLaunch L;
    L.P = P; L.pld = pld; L.pbs = slab_words;
    L.X = C->data; L.ld = C->stride_words; L.bs = 0;
    L.rows = C->rows; L.cols = C->cols; L.vrows = C->rows; L.vcols = C->cols;
    L.nparent = 1; L.accumulate = 0;
    return sw_combine_launch(L, static_cast<cudaStream_t>(stream));
}

int gf2_make_table(gf2_mat *T, const gf2_mat *B, int64_t r0, int32_t k, void *stream)
{
    int rc;
    if ((rc = check_mat(T)) || (rc = check_mat(B))) return rc;
    if (k < 1 || k > 10 || r0 < 0) return GF2_EINVAL;
    if (T->rows != ((int64_t)1 << k) || T->cols != B->cols) return GF2_EINVAL;
    if (overlaps(T, B)) return GF2_EALIAS;
    DMat Td{T->data, T->rows, T->cols, T->stride_words};
    DMat Bd{B->data, B->rows, B->cols, B->stride_words};
    return make_table_launch(Td, Bd, r0, k, static_cast<cudaStream_t>(stream));
}

int gf2_random(gf2_mat *M, uint64_t seed, double p, void *stream)
{
    int rc = check_mat(M);
    if (rc) return rc;
    if (!(p >= 0.0 && p <= 1.0)) return GF2_EINVAL;
    if (M->device == GF2_HOST) return GF2_EINVAL;
    DMat D{M->data, M->rows, M->cols, M->stride_words};
    return random_launch(D, seed, p, static_cast<cudaStream_t>(stream));
}

int gf2_transpose(gf2_mat *T, const gf2_mat *X, void *stream)
{
    int rc;
    if ((rc = check_mat(T)) || (rc = check_mat(X))) return rc;
    if (T->rows != X->cols || T->cols != X->rows) return GF2_EINVAL;
    if (overlaps(T, X)) return GF2_EALIAS;
    DMat Td{T->data, T->rows, T->cols, T->stride_words};
    DMat Xd{X->data, X->rows, X->cols, X->stride_words};
    return transpose_launch(Td, Xd, static_cast<cudaStream_t>(stream));
}

int gf2_freivalds(const gf2_mat *C, const gf2_mat *A, const gf2_mat *B, uint64_t seed,
                  int64_t *mismatched_rows, void *stream)
{
    int rc;
    if (!mismatched_rows) return GF2_EINVAL;
    if ((rc = check_mat(A)) || (rc = check_mat(B)) || (rc = check_mat(C))) return rc;
    if (A->cols != B->rows || C->rows != A->rows || C->cols != B->cols) return GF2_EINVAL;
    if (A->device == GF2_HOST || B->device == GF2_HOST || C->device == GF2_HOST) return GF2_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t m = A->rows, l = A->cols, n = B->cols;
    *mismatched_rows = 0;
    if (m == 0) return GF2_OK;
    const int64_t ldxn = even_up(words_of(n)), ldxl = even_up(words_of(l));
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t a = off; off += (bytes + 255) & ~(size_t)255; return a; };
    const size_t oX = take((size_t)std::max<int64_t>(n, 1) * 8);
    const size_t oXT = take((size_t)(64 * ldxn) * 8);
    const size_t oY1 = take((size_t)std::max<int64_t>(l, 1) * 8);
    const size_t oY1T = take((size_t)(64 * ldxl) * 8);
    const size_t oY2 = take((size_t)m * 8);
    const size_t oY3 = take((size_t)m * 8);
    const size_t oCnt = take(8);
    void *scr = nullptr;
    ArenaHold hold;
    if ((rc = arena_get(s, off, &scr, &hold))) return rc;
    char *b = static_cast<char *>(scr);
    uint64_t *X = reinterpret_cast<uint64_t *>(b + oX), *XT = reinterpret_cast<uint64_t *>(b + oXT);
    uint64_t *Y1 = reinterpret_cast<uint64_t *>(b + oY1), *Y1T = reinterpret_cast<uint64_t *>(b + oY1T);
    uint64_t *Y2 = reinterpret_cast<uint64_t *>(b + oY2), *Y3 = reinterpret_cast<uint64_t *>(b + oY3);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(b + oCnt);
    GF2_CUDA_TRY(cudaMemsetAsync(cnt, 0, 8, s));
    GF2_CUDA_TRY(cudaMemsetAsync(Y1T, 0, (size_t)(64 * ldxl) * 8, s));
    GF2_CUDA_TRY(cudaMemsetAsync(XT, 0, (size_t)(64 * ldxn) * 8, s));
    if ((rc = seeded_words_launch(X, n, seed, s))) return rc;
    // XT = X^T (64 x n), X seen as an n x 64 matrix with one word per row
    if (n > 0 && (rc = transpose_launch(DMat{XT, 64, n, ldxn}, DMat{X, n, 64, 1}, s))) return rc;
    if (l > 0) {
        // Y1 = B X (l words), Y1T = Y1^T
        if ((rc = matvec64_launch(B->data, l, n, B->stride_words, XT, Y1, s))) return rc;
        if ((rc = transpose_launch(DMat{Y1T, 64, l, ldxl}, DMat{Y1, l, 64, 1}, s))) return rc;
    }
    // Y2 = A (B X), Y3 = C X
    if ((rc = matvec64_launch(A->data, m, l, A->stride_words, Y1T, Y2, s))) return rc;
    if ((rc = matvec64_launch(C->data, m, n, C->stride_words, XT, Y3, s))) return rc;
    if ((rc = xor_count_launch(Y2, Y3, m, cnt, s))) return rc;
    unsigned long long h = 0;
    GF2_CUDA_TRY(cudaMemcpyAsync(&h, cnt, 8, cudaMemcpyDeviceToHost, s));
    GF2_CUDA_TRY(cudaStreamSynchronize(s));
    *mismatched_rows = (int64_t)h;
    return GF2_OK;
}

}  // extern "C"
