/*
 * gf2_oracle.c -- CPU oracle for matrix multiplication over GF(2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA library.
 *
 * What it computes is the plain definition of the product the paper's
 * algorithms reach exactly:
 *
 *     C[i][j] = XOR over t < l of (A[i][t] AND B[t][j])
 *
 * (Abstract: addition in GF(2) is XOR and multiplication is AND; Section 3,
 * problem statement C = AB for A m x l and B l x n; Section 2.3: a dot
 * product is an AND followed by an XOR accumulation.)  The work is done on
 * UNPACKED bytes, one entry per byte, by a naive triple loop; the packed
 * layout (Section 2.1: 64 consecutive entries of a row in one word) is only
 * converted at the edges by this file's own pack / unpack.
 *
 * Packed layout read and written here: row r, column c lives in 64-bit word
 * r*stride + c/64 at bit position c%64.  Bits at columns >= cols are ignored
 * on input and written as 0 on output.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int gf2o_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void gf2o_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* packed -> one byte per entry (Section 2.1 layout, LSB-first in a word) */
void gf2o_unpack(const uint64_t *P, int64_t rows, int64_t cols, int64_t stride,
                 uint8_t *bits)
{
    for (int64_t r = 0; r < rows; ++r)
        for (int64_t c = 0; c < cols; ++c)
            bits[r * cols + c] = (uint8_t)((P[r * stride + c / 64] >> (c % 64)) & 1u);
}

/* one byte per entry -> packed; words beyond the entries are cleared */
void gf2o_pack(const uint8_t *bits, int64_t rows, int64_t cols, int64_t stride,
               uint64_t *P)
{
    for (int64_t r = 0; r < rows; ++r) {
        memset(P + r * stride, 0, (size_t)stride * sizeof(uint64_t));
        for (int64_t c = 0; c < cols; ++c)
            if (bits[r * cols + c] & 1u)
                P[r * stride + c / 64] |= (uint64_t)1 << (c % 64);
    }
}

/*
 * Naive cubic product on unpacked entries: C = A B over GF(2).
 * A is m x l, B is l x n, C is m x n, all one byte per entry, row-major.
 * The loops follow the definition; the (i, t, j) order only lets the
 * innermost loop run over contiguous memory.
 */
void gf2o_mul_unpacked(const uint8_t *A, const uint8_t *B, uint8_t *C,
                       int64_t m, int64_t l, int64_t n)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        uint8_t *c = C + i * n;
        for (int64_t j = 0; j < n; ++j) c[j] = 0;
        for (int64_t t = 0; t < l; ++t) {
            const uint8_t a = A[i * l + t] & 1u;
            const uint8_t *b = B + t * n;
            for (int64_t j = 0; j < n; ++j)
                c[j] ^= (uint8_t)(a & b[j]);
        }
    }
}

/*
 * C = A B on packed operands: unpack, naive cubic, pack.
 * Strides are in 64-bit words.  Returns 0, or -1 when memory runs out.
 */
int gf2o_mul_packed(const uint64_t *A, int64_t sa, const uint64_t *B, int64_t sb,
                    uint64_t *C, int64_t sc, int64_t m, int64_t l, int64_t n)
{
    uint8_t *a = (uint8_t *)malloc((size_t)(m * l) + 1);
    uint8_t *b = (uint8_t *)malloc((size_t)(l * n) + 1);
    uint8_t *c = (uint8_t *)malloc((size_t)(m * n) + 1);
    if (!a || !b || !c) { free(a); free(b); free(c); return -1; }
    gf2o_unpack(A, m, l, sa, a);
    gf2o_unpack(B, l, n, sb, b);
    gf2o_mul_unpacked(a, b, c, m, l, n);
    gf2o_pack(c, m, n, sc, C);
    free(a); free(b); free(c);
    return 0;
}

/*
 * Matrix-vector products in the packed form of Section 2.3: with the vector
 * stored as a row, a dot product is a word-wise AND, an XOR accumulation of
 * the words, and the parity of the accumulated word.
 *
 * Y = M X for an r x c matrix M (packed rows, stride sm words) and a block
 * X of 64 column vectors stored as one 64-bit word per row of X (X has c
 * rows; bit v of X[t] is entry t of vector v).  Output Y has r words.
 * Computed one vector v at a time: vector v is gathered into a packed row,
 * then each row of M is dotted with it.
 */
void gf2o_matvec64(const uint64_t *M, int64_t r, int64_t c, int64_t sm,
                   const uint64_t *X, uint64_t *Y)
{
    const int64_t W = (c + 63) / 64;
    uint64_t *xv = (uint64_t *)calloc((size_t)(64 * W) + 1, sizeof(uint64_t));
    if (!xv) return;
    for (int v = 0; v < 64; ++v)
        for (int64_t t = 0; t < c; ++t)
            if ((X[t] >> v) & 1u) xv[v * W + t / 64] |= (uint64_t)1 << (t % 64);
    const uint64_t tail = (c % 64) ? (((uint64_t)1 << (c % 64)) - 1) : ~(uint64_t)0;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < r; ++i) {
        uint64_t y = 0;
        for (int v = 0; v < 64; ++v) {
            uint64_t acc = 0;
            for (int64_t w = 0; w < W; ++w) {
                uint64_t mw = M[i * sm + w];
                if (w == W - 1) mw &= tail;
                acc ^= mw & xv[v * W + w];
            }
            /* parity of acc */
            acc ^= acc >> 32; acc ^= acc >> 16; acc ^= acc >> 8;
            acc ^= acc >> 4;  acc ^= acc >> 2;  acc ^= acc >> 1;
            y |= (acc & 1u) << v;
        }
        Y[i] = y;
    }
    free(xv);
}
