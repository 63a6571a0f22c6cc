// strassen.cu -- the additions of Strassen-Winograd (Section 4, Algorithm 4).
//
// Over GF(2) every addition and subtraction of Algorithm 4 is a word-wise XOR,
// so these kernels are pure HBM streams: read the four quadrants of each
// parent once, write the seven product operands (split), or read the seven
// products and write the four quadrants of the parent (combine).  They run
// breadth first, one launch per recursion level for all 7^j sub-problems of
// that level, so the GPU stays full at every level.  Operands below the top
// level live in dense slabs of the scratch arena (the "copy out" of
// Section 4 happens for all three matrices, which keeps every leaf product
// contiguous).
//
// Top level: the parent is the caller's matrix; entries beyond its real
// extent (vrows x vcols) read as zeros -- the virtual padding of Section 4 --
// and the combine writes back only the real extent, tail bits cleared.
#include "common.cuh"

namespace gf2 {
namespace {

__device__ __forceinline__ uint4 xr(uint4 a, uint4 b)
{
    return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
}
__device__ __forceinline__ uint4 ld4(const uint64_t *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}
__device__ __forceinline__ void st4(uint64_t *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

// Two words of a (possibly virtual) top-level matrix: zero beyond the real
// rows / columns, tail bits masked.
__device__ __forceinline__ uint4 ld_virtual(const uint64_t *X, int64_t ld, int64_t r, int64_t w,
                                            int64_t vrows, int64_t vcols)
{
    if (r >= vrows) return make_uint4(0, 0, 0, 0);
    const int64_t vW = words_of(vcols);
    uint64_t a = 0, b = 0;
    const uint64_t *row = X + r * ld;
    if (w < vW) a = row[w] & word_mask(w, vcols);
    if (w + 1 < vW) b = row[w + 1] & word_mask(w + 1, vcols);
    return make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
}

template <bool TOP>
__global__ void __launch_bounds__(256) sw_split_kernel(SplitLaunch L)
{
    const int64_t hr = L.rows / 2;            // child rows
    const int64_t hw = L.cols / 128;          // child words per row (even)
    const int64_t hq = hw / 2;                // child 16-byte chunks per row
    const int64_t per_parent = hr * hq;
    const int64_t total = per_parent * L.nparent;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t par = i / per_parent;
        const int64_t rem = i - par * per_parent;
        const int64_t r = rem / hq;
        const int64_t w = (rem - r * hq) * 2;
        const uint64_t *X = L.X + par * L.bs;
        uint4 nw, ne, sw, se;
        if (TOP) {
            nw = ld_virtual(X, L.ld, r, w, L.vrows, L.vcols);
            ne = ld_virtual(X, L.ld, r, w + hw, L.vrows, L.vcols);
            sw = ld_virtual(X, L.ld, r + hr, w, L.vrows, L.vcols);
            se = ld_virtual(X, L.ld, r + hr, w + hw, L.vrows, L.vcols);
        } else {
            nw = ld4(X + r * L.ld + w);
            ne = ld4(X + r * L.ld + w + hw);
            sw = ld4(X + (r + hr) * L.ld + w);
            se = ld4(X + (r + hr) * L.ld + w + hw);
        }
        uint4 o[7];
        if (L.side == 0) {
            // A side: S0 = A_SW + A_SE, S1 = S0 + A_NW, S2 = A_NW + A_SW, S3 = A_NE + S1
            const uint4 s0 = xr(sw, se);
            const uint4 s1 = xr(s0, nw);
            const uint4 s2 = xr(nw, sw);
            const uint4 s3 = xr(ne, s1);
            // left factors of P0..P6: A_NW, A_NE, S3, A_SE, S0, S1, S2
            o[0] = nw; o[1] = ne; o[2] = s3; o[3] = se; o[4] = s0; o[5] = s1; o[6] = s2;
        } else {
            // side 2: X is B^T, whose NE quadrant is (B_SW)^T and SW is (B_NE)^T
            if (L.side == 2) { const uint4 tmp = ne; ne = sw; sw = tmp; }
            // B side: T0 = B_NE + B_NW, T1 = B_SE + T0, T2 = B_SE + B_NE, T3 = T1 + B_SW
            const uint4 t0 = xr(ne, nw);
            const uint4 t1 = xr(se, t0);
            const uint4 t2 = xr(se, ne);
            const uint4 t3 = xr(t1, sw);
            // right factors of P0..P6: B_NW, B_SW, B_SE, T3, T0, T1, T2 (transposed
            // for side 2, where B_SW^T is the NE quadrant swapped in above)
            o[0] = nw; o[1] = sw; o[2] = se; o[3] = t3; o[4] = t0; o[5] = t1; o[6] = t2;
        }
        uint64_t *dst = L.out + (par * 7) * L.cbs + r * L.cld + w;
#pragma unroll
        for (int j = 0; j < 7; ++j) st4(dst + j * L.cbs, o[j]);
    }
}

template <bool TOP>
__global__ void __launch_bounds__(256) sw_combine_kernel(CombineLaunch L)
{
    const int64_t hr = L.rows / 2;
    const int64_t hw = L.cols / 128;
    const int64_t hq = hw / 2;
    const int64_t per_parent = hr * hq;
    const int64_t total = per_parent * L.nparent;
    const int64_t vW = words_of(L.vcols);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t par = i / per_parent;
        const int64_t rem = i - par * per_parent;
        const int64_t r = rem / hq;
        const int64_t w = (rem - r * hq) * 2;
        const uint64_t *Pp = L.P + (par * 7) * L.pbs + r * L.pld + w;
        const uint4 p0 = ld4(Pp), p1 = ld4(Pp + L.pbs), p2 = ld4(Pp + 2 * L.pbs),
                    p3 = ld4(Pp + 3 * L.pbs), p4 = ld4(Pp + 4 * L.pbs), p5 = ld4(Pp + 5 * L.pbs),
                    p6 = ld4(Pp + 6 * L.pbs);
        // the 7 final additions of Algorithm 4
        const uint4 u0 = xr(p0, p1);
        const uint4 u1 = xr(p0, p5);
        const uint4 u2 = xr(u1, p6);
        const uint4 u3 = xr(u1, p4);
        const uint4 u4 = xr(u3, p2);
        const uint4 u5 = xr(u2, p3);
        const uint4 u6 = xr(u2, p4);
        // C = Stack(Augment(U0, U4), Augment(U5, U6))
        uint64_t *X = L.X + par * L.bs;
        const uint4 q[4] = {u0, u4, u5, u6};
        const int64_t qr[4] = {r, r, r + hr, r + hr};
        const int64_t qw[4] = {w, w + hw, w, w + hw};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint64_t *d = X + qr[j] * L.ld + qw[j];
            if (TOP) {
                if (qr[j] >= L.vrows) continue;
                const uint64_t a = ((uint64_t)q[j].y << 32) | q[j].x;
                const uint64_t b = ((uint64_t)q[j].w << 32) | q[j].z;
                if (qw[j] < vW) {
                    const uint64_t v = a & word_mask(qw[j], L.vcols);
                    d[0] = L.accumulate ? (d[0] ^ v) : v;
                }
                if (qw[j] + 1 < vW) {
                    const uint64_t v = b & word_mask(qw[j] + 1, L.vcols);
                    d[1] = L.accumulate ? (d[1] ^ v) : v;
                }
            } else {
                st4(d, L.accumulate ? xr(*reinterpret_cast<const uint4 *>(d), q[j]) : q[j]);
            }
        }
    }
}

int grid_for(int64_t total)
{
    int64_t b = (total + 255) / 256;
    const int64_t cap = 152 * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

int sw_split_launch(const SplitLaunch &L, cudaStream_t s)
{
    const int64_t total = (L.rows / 2) * (L.cols / 256) * L.nparent;
    if (total <= 0) return GF2_OK;
    const bool top = (L.vrows != L.rows) || (L.vcols != L.cols) || (L.ld & 1) ||
                     (reinterpret_cast<uintptr_t>(L.X) & 15);
    ProfScope ps(PF_SPLIT, s);
    if (top)
        sw_split_kernel<true><<<grid_for(total), 256, 0, s>>>(L);
    else
        sw_split_kernel<false><<<grid_for(total), 256, 0, s>>>(L);
    note_launch();
    return check_launch();
}

int sw_combine_launch(const CombineLaunch &L, cudaStream_t s)
{
    const int64_t total = (L.rows / 2) * (L.cols / 256) * L.nparent;
    if (total <= 0) return GF2_OK;
    const bool top = (L.vrows != L.rows) || (L.vcols != L.cols) || (L.ld & 1) ||
                     (reinterpret_cast<uintptr_t>(L.X) & 15);
    ProfScope ps(PF_COMBINE, s);
    if (top)
        sw_combine_kernel<true><<<grid_for(total), 256, 0, s>>>(L);
    else
        sw_combine_kernel<false><<<grid_for(total), 256, 0, s>>>(L);
    note_launch();
    return check_launch();
}

}  // namespace gf2
