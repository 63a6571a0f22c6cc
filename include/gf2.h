/*
 * gf2.h -- C ABI of libgf2: dense matrix multiplication over GF(2) on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Albrecht, Bard and Hart, "Efficient Multiplication of Dense
 * Matrices over GF(2)".  C = A B where addition is XOR and multiplication is
 * AND (Abstract).  The product runs Strassen-Winograd recursion (Section 4,
 * Algorithm 4) down to a base case, which is either the Method of the Four
 * Russians (Section 3, Algorithms 1-3) on bit-packed words, or an exact
 * tensor-core form that multiplies 0/1 values and keeps the parity of each
 * integer dot product (Section 2.3: a GF(2) dot product is an AND followed by
 * an XOR accumulation, i.e. the integer dot product mod 2).
 *
 * Matrix layout (Section 2.1, "flat row-major representation"): 64
 * consecutive entries of a row are packed into one 64-bit word.  Entry
 * (r, c) is bit (c % 64) of word data[r * stride_words + c / 64].
 * stride_words >= ceil(cols / 64); the library requires it to be even and
 * `data` to be 16-byte aligned (rows are read with 128-bit loads).
 * Bits of columns >= cols are IGNORED on input and written as 0 on output.
 *
 * Conventions for every call:
 *  - return GF2_OK (0) on success, a negative GF2_E* status otherwise;
 *    nothing is launched when a call fails its argument checks;
 *  - device work is asynchronous on `cuda_stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  Results are valid once the stream has
 *    reached the point after the call;
 *  - the caller owns every gf2_mat; the library owns only its scratch arenas
 *    (one per device and stream, grown on demand, released by
 *    gf2_release_scratch) and its autotuning cache;
 *  - calls may come from several host threads, on the same stream or on
 *    different ones: a call holds its stream's arena until it has queued
 *    all work that uses it (gf2_mul_noalloc's fixed buffer excepted, see
 *    there);
 *  - a matrix with device >= 0 lives in that device's global memory; with
 *    device == GF2_HOST it lives in host memory (pinned memory gives full
 *    copy speed).  gf2_mul accepts host operands and then copies them
 *    through its device scratch inside the call.
 */
#ifndef GF2_H
#define GF2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define GF2_OK            0
#define GF2_EINVAL       (-1)  /* NULL pointer, negative size, A.cols != B.rows, C not m x n, bad option */
#define GF2_EALIAS       (-2)  /* C overlaps A or B                                           */
#define GF2_ELAYOUT      (-3)  /* stride < ceil(cols/64), odd stride, or data not 16-byte aligned */
#define GF2_ENOMEM       (-4)  /* device or host allocation failed                            */
#define GF2_ECUDA        (-5)  /* CUDA runtime / launch error                                 */
#define GF2_ETIMEOUT     (-6)  /* a bounded device-side wait expired                          */
#define GF2_EUNSUPPORTED (-7)  /* option not available for this shape or device               */
#define GF2_EMISMATCH    (-8)  /* verification found C != A B                                 */
#define GF2_ESCRATCH     (-9)  /* gf2_mul_noalloc: the plan needs more than its fixed scratch  */

#define GF2_HOST (-1)          /* gf2_mat.device value for host memory */

/* ---- base cases -------------------------------------------------------- */
#define GF2_BASE_AUTO   0      /* autotuner's choice                                         */
#define GF2_BASE_M4RM   1      /* Method of the Four Russians on packed words (Sections 3.x) */
#define GF2_BASE_TC_FP8 2      /* 0/1 FP8 e4m3 tensor-core product, parity of exact sums
                                  (Section 2.3); operands expanded once to FP8 bytes        */
#define GF2_BASE_TC_S8  3      /* 0/1 int8 warp-level tensor product (mma.sync), int32 sums;
                                  never chosen automatically (slow on this part)             */
#define GF2_BASE_TC_B1  4      /* binary warp-level tensor product on the packed words
                                  (mma.sync .b1 .and.popc, Section 2.3's popcount of
                                  AND-ed rows of A and B^T), int32 sums; never chosen
                                  automatically (slow on this part)                          */
#define GF2_BASE_TC_FP4 5      /* 0/1 FP4 e2m1 block-scaled tensor-core product (scale
                                  factors 1.0), parity of exact sums (Section 2.3);
                                  operands expanded once to FP4 nibbles                     */

typedef struct gf2_mat {
    uint64_t *data;        /* first word of row 0                                  */
    int64_t rows;          /* number of rows                                       */
    int64_t cols;          /* number of entries per row                            */
    int64_t stride_words;  /* words between the starts of consecutive rows         */
    int32_t device;        /* CUDA device ordinal, or GF2_HOST                     */
    int32_t reserved;
} gf2_mat;

typedef struct gf2_opts {
    int32_t base;          /* GF2_BASE_*                                                 */
    int32_t depth;         /* Strassen-Winograd levels: -1 = auto, 0 = base case only    */
    int32_t k;             /* M4RM bits per table (Section 3.1 "k"): 0 = auto, else 4..10 */
    int32_t t;             /* M4RM tables per pass (Section 3.3 "t"): 0 = auto            */
    int32_t accumulate;    /* 0: C = A B;  1: C ^= A B                                    */
    int32_t peel;          /* sizes that do not halve evenly (Section 4): 0 = virtual
                              zero padding; 1 = peeling: Strassen-Winograd on the largest
                              evenly halving core, the leftover rows, columns and K
                              entries by base-case products (device operands); -1 = the
                              autotuner times both on the first call for a shape
                              (gf2_default_opts; padding where it does not tune)       */
    int32_t reserved[2];   /* must be 0                                                   */
} gf2_opts;

/* Fill *opts with the defaults: everything automatic, C = A B.  Algorithm 1
 * starts from C = GenerateZeroMatrix(m, n), so overwriting C is the default
 * and accumulate = 0; the depth (Section 4's cutoff, Section 5's c_s) and the
 * table shape (Section 3.1's k, Section 3.3's t) are chosen by the library. */
void gf2_default_opts(gf2_opts *opts);

/* Message for a status code (static string, never NULL).  The statuses are
 * the boundary's own error convention (the paper's algorithms have no error
 * paths); they cover the preconditions the paper states for the product:
 * A.cols == B.rows and C of m x n (Section 3 problem statement), and the
 * Section 2.1 layout (stride, alignment). */
const char *gf2_strerror(int status);

/* ---- memory -------------------------------------------------------------
 * gf2_alloc: Algorithm 1's "C <- GenerateZeroMatrix(m, n)" as a call: a
 * rows x cols device matrix on the CURRENT CUDA device in the Section 2.1
 * flat row-major layout, zero-filled, stride ceil(cols/64) rounded up to
 * even.  rows or cols may be 0 (data is then NULL).  On failure *M is left
 * with data == NULL.  Synchronises with the device (cudaMalloc semantics).
 */
int gf2_alloc(gf2_mat *M, int64_t rows, int64_t cols);

/* gf2_free: releases a matrix of gf2_alloc (Algorithm 1's GenerateZeroMatrix,
 * Section 2.1 layout); idempotent (data set to NULL); GF2_EINVAL for a host
 * matrix.  Synchronises with the device (cudaFree semantics). */
int gf2_free(gf2_mat *M);

/* ---- the product ---------------------------------------------------------
 * C = A B  (or C ^= A B with opts->accumulate), A m x l, B l x n, C m x n.
 * Section 4 (Algorithm 4) recursion to opts->depth levels -- operands are
 * zero-padded virtually to even, word-aligned sizes (Section 4, "padding"),
 * or with opts->peel the largest evenly halving core recurses and the
 * leftover rows, columns and K entries are base-case products ("peeling")
 * -- then the base case of opts->base on all 7^depth leaf products at once.
 * Temporaries live in the scratch arena of (device, stream).  opts may be
 * NULL (defaults).  C must not overlap A or B (GF2_EALIAS).  Zero-sized
 * operands are valid: C is cleared (or left alone when accumulating).
 * Device operands must all be on the current device; host operands
 * (device == GF2_HOST) are copied in and C is copied back inside the call,
 * which then returns only after the stream has finished it.  With A, B and
 * C all on the host, m >= 16384 and accumulate 0, A and C go in two row
 * blocks (C_i = A_i B, B's Strassen-Winograd additions done once), so that
 * copies in either direction overlap the products; the result is the same.
 * Autotuning: when opts->base is GF2_BASE_AUTO and/or opts->depth is -1,
 * accumulate is 0 and m*l*n >= 2^36, the plan comes from the autotuner: a
 * cached choice for this (architecture, shape, options), or, on the first
 * call, every candidate (base case x depth around the cutoff rule) is run
 * once on these operands, timed, and the fastest is cached (in memory, and
 * in the JSON file named by GF2_TUNE_CACHE when set).  That first call
 * synchronises the stream.  GF2_AUTOTUNE=0 disables it (cutoff rule only).
 */
int gf2_mul(gf2_mat *C, const gf2_mat *A, const gf2_mat *B,
            const gf2_opts *opts, void *cuda_stream);

/* ---- batched products ----------------------------------------------------
 * C[i] = A[i] B[i] for i < count, independent shapes.  Each product is the
 * one gf2_mul computes: Section 4's Algorithm 4 where it recurses, else the
 * base case of Section 3 (Algorithms 1 and 3, t tables) or the tensor-core
 * form of Section 2.3's integer dot products mod 2.  The products that do
 * not recurse run in ONE launch of a persistent kernel that pulls tiles of
 * all of them from one work queue (device operands only).  Same
 * per-product rules as gf2_mul; details under gf2_mul_batched_ex.
 */
int gf2_mul_batched(gf2_mat *const C[], const gf2_mat *const A[],
                    const gf2_mat *const B[], int32_t count,
                    const gf2_opts *opts, void *cuda_stream);

/* gf2_mul_batched_ex: gf2_mul_batched (Section 3's Algorithms 1 and 3 per
 * product, one persistent launch) with the batched base case's tile
 * variant pinned (variant >= 0, see gf2_batched_variant_name) or chosen by
 * the autotuner (variant = -1).  *chosen (may be NULL) receives the variant
 * used.  Details of the batched form:
 *  - products whose automatic plan recurses (every dimension >= 8192) or that
 *    request depth > 0 or the tensor-core base are run one by one as gf2_mul;
 *    all others go into ONE CUDA graph of persistent launches of the packed
 *    M4RM kernel whose CTAs pull tiles of all products from one work queue,
 *    longest K first: one launch, or two for the split variants (the tall
 *    k = 8 slot kernel over the row blocks of at least r rows, then the slot
 *    kernel over the rest);
 *  - the first call for a set of operands (pointers, shapes, strides,
 *    stream, options) times every variant on that batch (the autotuner),
 *    keeps the fastest, and builds a CUDA graph {reset the queue, launch};
 *    later calls with the same operands replay the graph.  The tuned choice
 *    is cached per shape signature and, when the environment variable
 *    GF2_TUNE_CACHE names a file, persisted there as JSON;
 *  - the first call synchronises the stream (autotuning, table upload).
 */
int gf2_mul_batched_ex(gf2_mat *const C[], const gf2_mat *const A[],
                       const gf2_mat *const B[], int32_t count,
                       const gf2_opts *opts, int32_t variant, int32_t *chosen,
                       void *cuda_stream);

/* Number of tile variants of the batched base case: shapes of Section 3's
 * tables (k bits, Section 3.1; t tables, Section 3.3) x tile width x rows. */
int32_t gf2_batched_variant_count(void);

/* Name of one batched tile variant (NULL beyond the last), with k and t as
 * in Sections 3.1 and 3.3: "k<k>t<t>-w<columns>-bm<rows>" (one product per
 * tile), "slots-k<k>t<t>-bm<rows>" (8 products' 128-column slices per tile),
 * "tall-k8t4-bm512" (slot tiles of 512 rows), and
 * "tall-k8t4-bm512-from<r>+slots-..." (row blocks of at least r rows on the
 * tall kernel, the rest on the slot kernel). */
const char *gf2_batched_variant_name(int32_t variant);

/* ---- steps of the path, callable alone ------------------------------------
 * gf2_sw_split: the 8 additions of Algorithm 4 for one level.  From X
 * (rows x cols, both even, cols a multiple of 128) writes the 7 operands of
 * the products P0..P6 into out[0..6] (each rows/2 x cols/2, dense stride
 * cols/128 words rounded up to even, out[i] = base + i * slab_words).
 * side = 0 treats X as the left factor A: out = A_NW, A_NE, S3, A_SE, S0, S1,
 * S2 with S0 = A_SW+A_SE, S1 = S0+A_NW, S2 = A_NW+A_SW, S3 = A_NE+S1.
 * side = 1 treats X as the right factor B: out = B_NW, B_SW, B_SE, T3, T0, T1,
 * T2 with T0 = B_NE+B_NW, T1 = B_SE+T0, T2 = B_SE+B_NE, T3 = T1+B_SW.
 * (Over GF(2) every "-" of Algorithm 4 is "+" = XOR.)
 */
int gf2_sw_split(uint64_t *out, int64_t slab_words, const gf2_mat *X,
                 int32_t side, void *cuda_stream);

/* gf2_sw_combine: the 7 final additions of Algorithm 4 plus Augment/Stack.
 * P holds the 7 products P0..P6 (each rows/2 x cols/2, dense layout as
 * written by gf2_sw_split, P[i] = base + i * slab_words); writes
 * C = [[U0, U4], [U5, U6]] into the rows x cols matrix C.
 */
int gf2_sw_combine(gf2_mat *C, const uint64_t *P, int64_t slab_words,
                   void *cuda_stream);

/* gf2_make_table: the table of Algorithm 1's MakeTable for one stripe:
 * T[x] = sum of rows r0+j of B (all columns) over the bits j set in x, for
 * x < 2^k (bit j of x selects row r0+j; rows >= B.rows count as zero).
 * T is a 2^k x B.cols device matrix.  1 <= k <= 10.
 */
int gf2_make_table(gf2_mat *T, const gf2_mat *B, int64_t r0, int32_t k,
                   void *cuda_stream);

/* ---- helpers ---------------------------------------------------------------
 * gf2_random: the random dense matrices the paper times (Section 6, Tables
 * 5-7) as seeded synthetic input: fill a device matrix with the seeded SplitMix64 bits (p = 0.5
 * takes whole outputs; otherwise one 32-bit uniform per bit), tail bits and
 * padding words 0.  Word (r, w) uses output r*ceil(cols/64)+w+1 of the stream
 * seeded with `seed` (p = 0.5), or outputs (r*W+w)*32+j+1, j < 32 (p != 0.5).
 */
int gf2_random(gf2_mat *M, uint64_t seed, double p, void *cuda_stream);

/* gf2_transpose: T = X^T (T is X.cols x X.rows), Section 2.1 layout on both
 * sides.  Section 2.3's cubic product reads B transposed (rows of B^T are the
 * columns of B); the tensor-core base cases do too. */
int gf2_transpose(gf2_mat *T, const gf2_mat *X, void *cuda_stream);

/* gf2_freivalds: checks C == A B with 64 random vectors at once (Freivalds'
 * test; the paper has no verification step, the dot products are Section
 * 2.3's AND + parity on packed words): X = seeded n x 64 bits, compares A (B X) with C X.  A wrong C
 * passes with probability <= 2^-64.  *mismatched_rows receives the number of
 * rows of A(BX) + CX that are non-zero (0 means the check passed).  Blocks
 * the calling thread until the stream has finished the check.
 */
int gf2_freivalds(const gf2_mat *C, const gf2_mat *A, const gf2_mat *B,
                  uint64_t seed, int64_t *mismatched_rows, void *cuda_stream);

/* ---- scratch ---------------------------------------------------------------
 * gf2_scratch_bytes: device scratch that gf2_mul needs for these shapes and
 * options (0 when it needs none): the temporaries of Section 4's Algorithm 4
 * (operand and product slabs of every level, breadth first; Section 4
 * discusses the paper's own two-temporary schedule) plus the transposed B of
 * the tensor-core base cases.
 */
int64_t gf2_scratch_bytes(int64_t m, int64_t l, int64_t n, const gf2_opts *opts);

/* gf2_reserve_scratch: grow the arena of (current device, stream), which
 * holds Algorithm 4's temporaries (Section 4), to at least `bytes` now, so
 * that later calls do not allocate. */
int gf2_reserve_scratch(int64_t bytes, void *cuda_stream);

/* gf2_release_scratch: free every arena of Algorithm 4's temporaries
 * (Section 4) on the current device (synchronises the device first). */
int gf2_release_scratch(void);

/* Number of kernels this library has launched in this process (all devices).
 * Bookkeeping of the boundary; the paper has no counterpart (it times whole
 * products, Section 6). */
int64_t gf2_launch_count(void);

/* gf2_device_status: failure detection of the boundary (the paper has no
 * counterpart; it guards the tensor-core form of Section 2.3's dot
 * products): waits for `cuda_stream`, then reads and clears the
 * device status word of the tensor-core base case.  Returns GF2_OK, or
 * GF2_ETIMEOUT when one of its bounded waits expired since the last read
 * (its kernels then stop early and the product is not valid).
 */
int gf2_device_status(void *cuda_stream);

/* gf2_selftest_wait: tests the failure detection without a GPU fault (the
 * paper has no counterpart; the wait is the one the Section 2.3 tensor-core
 * form's pipeline uses).
 * Launches one CTA whose single wait can never be satisfied (an mbarrier no
 * one arrives on); after `limit_cycles` SM clock cycles (1 .. 4e9) the wait
 * gives up and records GF2_ETIMEOUT in the same status word the tensor-core
 * kernels use, so the next gf2_device_status returns GF2_ETIMEOUT and the
 * context stays usable.
 */
int gf2_selftest_wait(int64_t limit_cycles, void *cuda_stream);

/* ---- device-time accounting ----------------------------------------------
 * gf2_profile_enable(1) clears the counters and starts bracketing every
 * kernel launch of the library with CUDA events on its stream; (0) stops.
 * The per-step breakdown of Section 6's timings (Tables 5-7 time whole
 * products; this splits them by kernel family).
 */
int gf2_profile_enable(int32_t on);

/* gf2_profile_read waits for the recorded events and returns the summed
 * device time (ms) and launch count of one kernel family (Section 6's
 * timings split by step):
 *   0 m4rm base case (Section 3), 1 FP8 tensor-core base case (Section 2.3),
 *   2 Strassen split, 3 Strassen combine (Section 4, Algorithm 4),
 *   4 transpose, 5 generator, 6 Freivalds products, 7 MakeTable
 *   (Algorithm 1), 8 batched base case, 9 int8 tensor-core base case,
 *   10 binary tensor-core base case, 11 FP4 tensor-core base case,
 *   12 expansion of packed operands to FP8 / FP4 entries (Section 2.3).
 */
int gf2_profile_read(int32_t family, double *ms, int64_t *launches);

/* gf2_profile_name gives the name of a gf2_profile_read family (Section 6's
 * timings split by step; NULL beyond the last one). */
const char *gf2_profile_name(int32_t family);

/* ---- product without allocation --------------------------------------------
 * The paper has no counterpart: this entry point exists for callers of this
 * library that cannot allocate device memory.  Two kinds of caller need it:
 * code that runs inside a framework which has already reserved nearly all
 * of the GPU's memory for its own allocator (a cudaMalloc of the scratch
 * would fail there), and code on a latency-critical path that must not
 * absorb the device-wide synchronisation that cudaMalloc and cudaFree
 * imply.
 *
 * gf2_mul_noalloc computes the same product as gf2_mul (the result is
 * unique, so the words of C are identical) for device operands, with the
 * same kernels, but takes the Strassen-Winograd temporaries (and the
 * transposed B of the tensor-core base case) from one fixed buffer of
 * GF2_NOALLOC_SCRATCH_BYTES that lives in the library's device image: every
 * GPU that loads the library holds that buffer until the process exits.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.  The caller
 * still provides A, B and C.
 *
 *  - Its plan is the cutoff rule's, not the autotuner's: base GF2_BASE_AUTO
 *    means the packed base case, depth -1 the cutoff rule's depth, and odd
 *    sizes are padded (peel 0 or -1).  gf2_mul may pick another base case
 *    or depth for large shapes after timing them; peel = 1 is refused with
 *    GF2_EUNSUPPORTED.
 *  - The first call on a device, in each CUDA context, looks up the
 *    buffer's device address (cudaGetSymbolAddress, with that device
 *    current) and keeps it for that context; make that first call before
 *    any stream capture (also after a cudaDeviceReset, which starts a new
 *    context).
 *  - If the plan for these shapes and options needs more scratch than the
 *    buffer holds, the call launches nothing and returns GF2_ESCRATCH
 *    (gf2_scratch_bytes gives the need; lower opts->depth to reduce it).
 *    With 32 MiB, square products fit up to n = 6912 at depth 1 and
 *    n = 4096 at depth 2; depth 0 needs none with the packed base case.
 *  - All calls share the one buffer, which keeps the last call's contents
 *    (every part a call reads is written by that call first).  Calls whose
 *    work overlaps on the GPU (several streams, or several host threads)
 *    race on the buffer: serialise them, e.g. on one stream.
 *  - Host operands (GF2_HOST) are rejected with GF2_EINVAL.
 */
#define GF2_NOALLOC_SCRATCH_BYTES ((int64_t)32 << 20)
int gf2_mul_noalloc(gf2_mat *C, const gf2_mat *A, const gf2_mat *B,
                    const gf2_opts *opts, void *cuda_stream);

/* Plan that gf2_mul would use for these shapes and options, as text (for
 * logs and tests): Section 4's recursion depth and padding or peeling, and
 * the base case's table shape (Sections 3.1 and 3.3, tuned as in Section 5).
 * Writes at most `cap` bytes including the terminating NUL.
 */
int gf2_describe_plan(int64_t m, int64_t l, int64_t n, const gf2_opts *opts,
                      char *buf, int32_t cap);

#ifdef __cplusplus
}
#endif
#endif /* GF2_H */
