// common.cuh -- shared definitions of the CUDA side of libgf2 (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "gf2.h"

namespace gf2 {

// Dense view of a packed matrix on the device (Section 2.1 layout).
struct DMat {
    uint64_t *p;       // word (0, 0)
    int64_t rows;
    int64_t cols;
    int64_t ld;        // stride in words
};

__host__ __device__ inline int64_t words_of(int64_t cols) { return (cols + 63) >> 6; }
__host__ __device__ inline int64_t even_up(int64_t w) { return w + (w & 1); }
__host__ __device__ inline uint64_t tail_mask(int64_t cols)
{
    const int r = (int)(cols & 63);
    return r ? ((1ull << r) - 1ull) : ~0ull;
}

// Mask for word w of a row with `cols` entries (0 beyond the row).
__host__ __device__ inline uint64_t word_mask(int64_t w, int64_t cols)
{
    const int64_t W = words_of(cols);
    if (w < W - 1) return ~0ull;
    if (w == W - 1) return tail_mask(cols);
    return 0ull;
}

// Counts launches for gf2_launch_count (host side).
void note_launch(int n = 1);

// Kernel families for the device-time accounting of gf2_profile_*.
enum ProfFamily { PF_M4RM = 0, PF_TC, PF_SPLIT, PF_COMBINE, PF_TRANSPOSE, PF_RANDOM, PF_MATVEC,
                  PF_TABLE, PF_BATCHED, PF_TC_S8, PF_TC_B1, PF_TC_F4, PF_EXPAND, PF_COUNT };

// Brackets the launches made during its lifetime with CUDA events on `s`
// when accounting is on.
struct ProfScope {
    int fam;
    cudaStream_t s;
    void *rec;
    ProfScope(int family, cudaStream_t stream);
    ~ProfScope();
};

// Checks the last launch; returns GF2_OK or GF2_ECUDA.
int check_launch();

inline int div_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// ---- kernel entry points implemented in the .cu files --------------------

// M4RM base case (Section 3): C = A B (batch of `batch` products with
// element strides bsA/bsB/bsC between them).  k bits per table, t tables.
struct M4rmLaunch {
    const uint64_t *A; int64_t lda, bsA;
    const uint64_t *B; int64_t ldb, bsB;
    uint64_t *C; int64_t ldc, bsC;
    int64_t m, l, n;
    int batch;
    int accumulate;   // C ^= A B instead of C = A B
    int k, t;         // 0 = automatic
    int ksplit;       // 0 = automatic
    int bm;           // tile rows, 0 = automatic
};
int m4rm_launch(const M4rmLaunch &L, cudaStream_t s);
bool m4rm_supported(int k, int t);
void m4rm_pick(int64_t m, int64_t l, int64_t n, int batch, int *k, int *t, int *bm, int *ksplit);

// Table of Algorithm 1 for one stripe, into global memory.
int make_table_launch(DMat T, DMat B, int64_t r0, int k, cudaStream_t s);

// Strassen-Winograd additions (Algorithm 4).
// Level split of `nparent` parents (each rows x cols, stride ld, batch stride
// bs) into 7*nparent children (rows/2 x cols/2, stride cld, batch stride cbs,
// child 7*i+j of parent i).  side 0: A operands, 1: B operands.  For the top
// level the parent is the user's matrix: `vrows`/`vcols` are its real extent
// (reads beyond are virtual zeros); rows/cols are the padded extent.
struct SplitLaunch {
    const uint64_t *X; int64_t ld, bs; int64_t rows, cols, vrows, vcols;
    uint64_t *out; int64_t cld, cbs;
    int nparent; int side;
    // xkind != 0: the children are written expanded for the tensor-core base
    // case instead (KIND_F8 + 1 or KIND_F4 + 1): row r of child c at
    // xout + (c * child rows + r) * rowbytes, rowbytes = the child's entries
    // (FP8) or half of them (FP4), no padding
    uint8_t *xout = nullptr; int64_t rowbytes = 0; int xkind = 0;
};
int sw_split_launch(const SplitLaunch &L, cudaStream_t s);

// Combine of `nparent` groups of 7 products (each rows/2 x cols/2 at stride
// pld, product j of group i at P + (7*i+j)*pbs) into parents (rows x cols,
// stride ld, batch stride bs).  Writes only rows < vrows, cols < vcols of
// the parent (tail bits cleared); with accumulate the parent is XORed into.
struct CombineLaunch {
    const uint64_t *P; int64_t pld, pbs;
    uint64_t *X; int64_t ld, bs; int64_t rows, cols, vrows, vcols;
    int nparent; int accumulate;
};
int sw_combine_launch(const CombineLaunch &L, cudaStream_t s);

// Two levels at once (rows divisible by 4, cols by 512): split writes the 49
// grandchild operands (out, cld, cbs describe the grandchild slabs); combine
// reads the 49 grandchild products (P, pld, pbs) and writes the parent.
int sw_split2_launch(const SplitLaunch &L, cudaStream_t s);
int sw_combine2_launch(const CombineLaunch &L, cudaStream_t s);

// Utilities.
int random_launch(DMat M, uint64_t seed, double p, cudaStream_t s);
// T = X^T
int transpose_launch(DMat T, DMat X, cudaStream_t s);
int zero_launch(DMat M, cudaStream_t s);   // clears rows x stride words
// Y (rows words) = M X with X one word per column of M (64 vectors).
int matvec64_launch(const uint64_t *M, int64_t rows, int64_t cols, int64_t ld,
                    const uint64_t *X, uint64_t *Y, cudaStream_t s);
int xor_count_launch(const uint64_t *a, const uint64_t *b, int64_t n,
                     unsigned long long *count, cudaStream_t s);
int seeded_words_launch(uint64_t *X, int64_t n, uint64_t seed, cudaStream_t s);

// Warp-level tensor-core base cases (mma.sync on 0/1 int8 or packed 1-bit
// operands, int32 sums, parity).
struct TcLaunch {
    const uint64_t *A; int64_t lda, bsA;     // m x l
    const uint64_t *Bt; int64_t ldb, bsB;    // n x l (B transposed)
    uint64_t *C; int64_t ldc, bsC;           // m x n
    int64_t m, l, n;
    int batch;
    int accumulate;
    unsigned int *status;                    // device word for timeouts (may be null)
};
// Device status word of the tensor-core kernels' bounded waits.
int tc_status_address(unsigned int **p);

// Tensor-core base case on operands expanded once in HBM (tc_mma.cu):
// KIND_F8 = FP8 E4M3 0/1 bytes (kind::f8f6f4), KIND_F4 = FP4 E2M1 0/1
// nibbles (kind::mxf4, scale factors 1.0).  Each operand row of l entries
// becomes tc_expanded_rowbytes(kind, l) bytes (l rounded up to 128 FP8 or
// 256 FP4 entries, zeros beyond l).
enum TcKind { KIND_F8 = 0, KIND_F4 = 1 };
int64_t tc_expanded_rowbytes(int kind, int64_t l);
// Y (batch x rows rows of rowbytes bytes) = expansion of the packed X
// (batch x rows x cols, stride ld words, batch stride bs words).
int tc_expand_launch(int kind, const uint64_t *X, int64_t ld, int64_t bs, int64_t rows, int64_t cols, int batch,
                     uint8_t *Y, int64_t rowbytes, cudaStream_t s);
struct TcxLaunch {
    int kind;
    const uint8_t *XA;       // batch x m expanded rows of A
    const uint8_t *XB;       // batch x n expanded rows of B^T
    int64_t rowbytes;        // bytes per expanded row (a multiple of 128)
    uint64_t *C; int64_t ldc, bsC;   // m x n packed
    int64_t m, n;
    int batch;
    int accumulate;
    unsigned int *status;
};
int tc_mma_launch(const TcxLaunch &L, cudaStream_t s);
int tc_s8_launch(const TcLaunch &L, cudaStream_t s);
// Binary tensor-core base case (mma.sync .b1 .and.popc on the packed words).
int tc_b1_launch(const TcLaunch &L, cudaStream_t s);
// Cubic product (Section 2.3) for at most 64 columns of C: BT = the n
// columns of B as rows, 64 rows (rows n..63 zero), stride ldbt words.
int cubic_narrow_launch(const uint64_t *A, int64_t lda, int64_t m, int64_t l, const uint64_t *BT,
                        int64_t ldbt, uint64_t *C, int64_t ldc, int64_t n, int accumulate, cudaStream_t s);

// Autotuner cache (tune.cu): text signature -> text choice.
bool tune_get(const std::string &key, std::string *value);
void tune_put(const std::string &key, const std::string &value);
std::string arch_tag();

// Batched persistent M4RM (one launch, graph-replayed, autotuned).
int batched_mul(gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[], int count,
                int accumulate, int force_variant, cudaStream_t s, int *chosen);
int batched_variant_count();
const char *batched_variant_name(int i);
void batched_release();
int tc_status_read_and_clear(unsigned int *out, cudaStream_t s);
int wait_selftest_launch(long long limit, cudaStream_t s);
// Batched products of uneven shapes on a tcgen05 base case of `kind` (one
// batched transpose, one batched expansion and one persistent launch,
// graph-replayed).
int tc_batched_mul(gf2_mat *const C[], const gf2_mat *const A[], const gf2_mat *const B[], int count,
                   int accumulate, int kind, cudaStream_t s);
void tc_batched_release();
bool tc_fp8_available();

}  // namespace gf2

#define GF2_CUDA_TRY(expr)                                     \
    do {                                                       \
        cudaError_t e_ = (expr);                               \
        if (e_ != cudaSuccess) return GF2_ECUDA;               \
    } while (0)

namespace gf2 {

// Timing events owned for the length of a scope: every one that was created
// is destroyed on every return path.
template <int N>
struct ScopedEvents {
    cudaEvent_t e[N] = {};
    ScopedEvents() = default;
    ScopedEvents(const ScopedEvents &) = delete;
    ScopedEvents &operator=(const ScopedEvents &) = delete;
    ~ScopedEvents()
    {
        for (cudaEvent_t ev : e)
            if (ev) cudaEventDestroy(ev);
    }
    int create()
    {
        for (cudaEvent_t &ev : e)
            if (cudaEventCreate(&ev) != cudaSuccess) {
                ev = nullptr;
                return GF2_ECUDA;
            }
        return GF2_OK;
    }
};

}  // namespace gf2
