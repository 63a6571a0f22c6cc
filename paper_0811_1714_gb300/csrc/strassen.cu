// strassen.cu -- the additions of Strassen-Winograd (Section 4, Algorithm 4).
//
// Over GF(2) every addition and subtraction of Algorithm 4 is a word-wise XOR,
// so these kernels are pure HBM streams: read the four quadrants of each
// parent once, write the seven product operands (split), or read the seven
// products and write the four quadrants of the parent (combine).  They run
// breadth first, one launch for all 7^j sub-problems of a level, so the GPU
// stays full at every level; two levels are fused per launch while two
// remain (sw_split2 / sw_combine2: 16 sub-blocks in, 49 operands out, and
// back, the middle level never leaving registers).  Operands below the top
// level live in dense slabs of the scratch arena (the "copy out" of
// Section 4 happens for all three matrices, which keeps every leaf product
// contiguous).
//
// Top level: the parent is the caller's matrix; entries beyond its real
// extent (vrows x vcols) read as zeros -- the virtual padding of Section 4 --
// and the combine writes back only the real extent, tail bits cleared.
#include "common.cuh"
#include "expand.cuh"

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

// One operand position (two words, row r of child c): packed (EX = 0) at
// L.out, or expanded for the tensor-core base case (EX = KIND_F8 + 1 / KIND_F4
// + 1): 128 or 64 bytes at L.xout, row (c * child rows + r), byte 64 w or 32 w.
// COOP: the 32 lanes of the warp hold 64 consecutive words of one row (lane
// i words w0 + 2i, w0 + 2i + 1), and the warp writes their expansion in
// 512-byte rounds, 16 bytes per lane, fetching each chunk's source words by
// shuffles (whole sectors per store instead of 16 bytes of every 64).
template <int EX, bool COOP>
__device__ __forceinline__ void st_child(const SplitLaunch &L, int64_t c, int64_t crows, int64_t r, int64_t w,
                                         uint4 v)
{
    if (EX == 0) {
        st4(L.out + c * L.cbs + r * L.cld + w, v);
    } else if (!COOP) {
        constexpr bool FP8 = EX == KIND_F8 + 1;
        uint4 o[FP8 ? 8 : 4];
        expand_words<FP8>(((uint64_t)v.y << 32) | v.x, ((uint64_t)v.w << 32) | v.z, o);
        uint4 *d = reinterpret_cast<uint4 *>(L.xout + (c * crows + r) * L.rowbytes + w * (FP8 ? 64 : 32));
#pragma unroll
        for (int q = 0; q < (FP8 ? 8 : 4); ++q) d[q] = o[q];
    } else {
        constexpr bool FP8 = EX == KIND_F8 + 1;
        constexpr int CPL = FP8 ? 8 : 4;                  // 16-byte chunks per lane's two words
        const int lane = threadIdx.x & 31;
        uint4 *d = reinterpret_cast<uint4 *>(L.xout + (c * crows + r) * L.rowbytes + (w - 2 * lane) * (FP8 ? 64 : 32));
        // the 32-bit component a lane's chunks come from: FP4 component lane % 4
        // (32 entries), FP8 component (lane % 8) / 2, 16-bit half lane % 2
        const int comp = FP8 ? (lane & 7) >> 1 : lane & 3;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const int src = (32 * q + lane) / CPL;
            const uint32_t a = __shfl_sync(0xffffffffu, v.x, src), b = __shfl_sync(0xffffffffu, v.y, src),
                           e = __shfl_sync(0xffffffffu, v.z, src), f = __shfl_sync(0xffffffffu, v.w, src);
            const uint32_t h = comp == 0 ? a : comp == 1 ? b : comp == 2 ? e : f;
            uint4 o;
            if (FP8) {
                const uint32_t x = (lane & 1) ? (h >> 16) : h;
                o = make_uint4(f8_of_nibble(x & 15u), f8_of_nibble((x >> 4) & 15u), f8_of_nibble((x >> 8) & 15u),
                               f8_of_nibble((x >> 12) & 15u));
            } else {
                o = make_uint4(f4_of_byte(h), f4_of_byte(h >> 8), f4_of_byte(h >> 16), f4_of_byte(h >> 24));
            }
            d[32 * q + lane] = o;
        }
    }
}

// The 8 additions of Algorithm 4 for one position of the four quadrants:
// the operands of P0..P6.  side 0: left factor A (S0..S3); side 1: right
// factor B (T0..T3); side 2: B^T, whose NE quadrant is (B_SW)^T and SW is
// (B_NE)^T (so the roles of NE and SW swap).
__device__ __forceinline__ void split_one(int side, uint4 nw, uint4 ne, uint4 sw, uint4 se, uint4 (&o)[7])
{
    if (side == 0) {
        // S0 = A_SW + A_SE, S1 = S0 + A_NW, S2 = A_NW + A_SW, S3 = A_NE + S1
        const uint4 s0 = xr(sw, se);
        const uint4 s1 = xr(s0, nw);
        const uint4 s2 = xr(nw, sw);
        const uint4 s3 = xr(ne, s1);
        // left factors of P0..P6: A_NW, A_NE, S3, A_SE, S0, S1, S2
        o[0] = nw; o[1] = ne; o[2] = s3; o[3] = se; o[4] = s0; o[5] = s1; o[6] = s2;
    } else {
        if (side == 2) { const uint4 tmp = ne; ne = sw; sw = tmp; }
        // T0 = B_NE + B_NW, T1 = B_SE + T0, T2 = B_SE + B_NE, T3 = T1 + B_SW
        const uint4 t0 = xr(ne, nw);
        const uint4 t1 = xr(se, t0);
        const uint4 t2 = xr(se, ne);
        const uint4 t3 = xr(t1, sw);
        // right factors of P0..P6: B_NW, B_SW, B_SE, T3, T0, T1, T2 (transposed
        // for side 2, where B_SW^T is the NE quadrant swapped in above)
        o[0] = nw; o[1] = sw; o[2] = se; o[3] = t3; o[4] = t0; o[5] = t1; o[6] = t2;
    }
}

// The 7 final additions of Algorithm 4 for one position: q = the values of
// the quadrants NW, NE, SW, SE of Stack(Augment(U0, U4), Augment(U5, U6)).
__device__ __forceinline__ void combine_one(const uint4 (&p)[7], uint4 (&q)[4])
{
    const uint4 u0 = xr(p[0], p[1]);
    const uint4 u1 = xr(p[0], p[5]);
    const uint4 u2 = xr(u1, p[6]);
    const uint4 u3 = xr(u1, p[4]);
    const uint4 u4 = xr(u3, p[2]);
    const uint4 u5 = xr(u2, p[3]);
    const uint4 u6 = xr(u2, p[4]);
    q[0] = u0; q[1] = u4; q[2] = u5; q[3] = u6;
}

template <bool TOP, int EX, bool COOP>
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
        split_one(L.side, nw, ne, sw, se, o);
#pragma unroll
        for (int j = 0; j < 7; ++j) st_child<EX, COOP>(L, par * 7 + j, hr, r, w, o[j]);
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
        const uint4 pp[7] = {p0, p1, p2, p3, p4, p5, p6};
        uint4 qv[4];
        combine_one(pp, qv);
        const uint4 u0 = qv[0], u4 = qv[1], u5 = qv[2], u6 = qv[3];
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

// Two levels of Algorithm 4 in one pass (the recursion applied to all 7
// operands of a level without writing them out): each thread reads the 16
// sub-blocks (q1 = quadrant, q2 = its quadrant) of one position of a parent
// and writes the 49 operands of the grandchild products, product
// 7 * (7 * parent + j1) + j2, the same order two single levels give.
template <bool TOP, int EX, bool COOP>
__global__ void __launch_bounds__(256) sw_split2_kernel(SplitLaunch L)
{
    const int64_t qr = L.rows / 4;            // grandchild rows
    const int64_t qw = L.cols / 256;          // grandchild words per row (even)
    const int64_t qq = qw / 2;
    const int64_t hrw = L.rows / 2, hw = L.cols / 128;
    const int64_t per_parent = qr * qq;
    const int64_t total = per_parent * L.nparent;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t par = i / per_parent;
        const int64_t rem = i - par * per_parent;
        const int64_t r = rem / qq;
        const int64_t w = (rem - r * qq) * 2;
        const uint64_t *X = L.X + par * L.bs;
        uint4 child[7][4];                    // level-1 operands at the 4 sub-positions
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
            uint4 v[4];
#pragma unroll
            for (int q1 = 0; q1 < 4; ++q1) {
                const int64_t row = (q1 >> 1) * hrw + (q2 >> 1) * qr + r;
                const int64_t wd = (q1 & 1) * hw + (q2 & 1) * qw + w;
                v[q1] = TOP ? ld_virtual(X, L.ld, row, wd, L.vrows, L.vcols) : ld4(X + row * L.ld + wd);
            }
            uint4 o[7];
            split_one(L.side, v[0], v[1], v[2], v[3], o);
#pragma unroll
            for (int j = 0; j < 7; ++j) child[j][q2] = o[j];
        }
#pragma unroll
        for (int j1 = 0; j1 < 7; ++j1) {
            uint4 g[7];
            split_one(L.side, child[j1][0], child[j1][1], child[j1][2], child[j1][3], g);
#pragma unroll
            for (int j2 = 0; j2 < 7; ++j2) st_child<EX, COOP>(L, par * 49 + j1 * 7 + j2, qr, r, w, g[j2]);
        }
    }
}

// Two levels of the final additions in one pass: reads the 49 grandchild
// products of one position and writes the 16 sub-blocks of the parent.
template <bool TOP>
__global__ void __launch_bounds__(256) sw_combine2_kernel(CombineLaunch L)
{
    const int64_t qr = L.rows / 4;
    const int64_t qw = L.cols / 256;
    const int64_t qq = qw / 2;
    const int64_t hrw = L.rows / 2, hw = L.cols / 128;
    const int64_t per_parent = qr * qq;
    const int64_t total = per_parent * L.nparent;
    const int64_t vW = words_of(L.vcols);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t par = i / per_parent;
        const int64_t rem = i - par * per_parent;
        const int64_t r = rem / qq;
        const int64_t w = (rem - r * qq) * 2;
        const uint64_t *Pp = L.P + (par * 49) * L.pbs + r * L.pld + w;
        uint4 cq[7][4];                       // quadrant values of the 7 level-1 products
#pragma unroll
        for (int j1 = 0; j1 < 7; ++j1) {
            uint4 p[7];
#pragma unroll
            for (int j2 = 0; j2 < 7; ++j2) p[j2] = ld4(Pp + (j1 * 7 + j2) * L.pbs);
            uint4 q[4];
            combine_one(p, q);
#pragma unroll
            for (int q2 = 0; q2 < 4; ++q2) cq[j1][q2] = q[q2];
        }
        uint64_t *X = L.X + par * L.bs;
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
            const uint4 p[7] = {cq[0][q2], cq[1][q2], cq[2][q2], cq[3][q2], cq[4][q2], cq[5][q2], cq[6][q2]};
            uint4 out[4];
            combine_one(p, out);
#pragma unroll
            for (int q1 = 0; q1 < 4; ++q1) {
                const int64_t row = (q1 >> 1) * hrw + (q2 >> 1) * qr + r;
                const int64_t wd = (q1 & 1) * hw + (q2 & 1) * qw + w;
                uint64_t *d = X + row * L.ld + wd;
                if (TOP) {
                    if (row >= L.vrows) continue;
                    const uint64_t a = ((uint64_t)out[q1].y << 32) | out[q1].x;
                    const uint64_t b = ((uint64_t)out[q1].w << 32) | out[q1].z;
                    if (wd < vW) {
                        const uint64_t v = a & word_mask(wd, L.vcols);
                        d[0] = L.accumulate ? (d[0] ^ v) : v;
                    }
                    if (wd + 1 < vW) {
                        const uint64_t v = b & word_mask(wd + 1, L.vcols);
                        d[1] = L.accumulate ? (d[1] ^ v) : v;
                    }
                } else {
                    st4(d, L.accumulate ? xr(*reinterpret_cast<const uint4 *>(d), out[q1]) : out[q1]);
                }
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
    if (L.xkind && (!L.xout || (reinterpret_cast<uintptr_t>(L.xout) & 15) || (L.rowbytes & 15))) return GF2_ELAYOUT;
    ProfScope ps(PF_SPLIT, s);
    const unsigned g = (unsigned)grid_for(total);
    // whole warps on one row's 64 words when a child row has a multiple of 32 word pairs
    const bool coop = (L.cols / 256) % 32 == 0;
    if (L.xkind == KIND_F8 + 1) {
        if (coop) { if (top) sw_split_kernel<true, KIND_F8 + 1, true><<<g, 256, 0, s>>>(L); else sw_split_kernel<false, KIND_F8 + 1, true><<<g, 256, 0, s>>>(L); }
        else { if (top) sw_split_kernel<true, KIND_F8 + 1, false><<<g, 256, 0, s>>>(L); else sw_split_kernel<false, KIND_F8 + 1, false><<<g, 256, 0, s>>>(L); }
    } else if (L.xkind == KIND_F4 + 1) {
        if (coop) { if (top) sw_split_kernel<true, KIND_F4 + 1, true><<<g, 256, 0, s>>>(L); else sw_split_kernel<false, KIND_F4 + 1, true><<<g, 256, 0, s>>>(L); }
        else { if (top) sw_split_kernel<true, KIND_F4 + 1, false><<<g, 256, 0, s>>>(L); else sw_split_kernel<false, KIND_F4 + 1, false><<<g, 256, 0, s>>>(L); }
    } else {
        if (top) sw_split_kernel<true, 0, false><<<g, 256, 0, s>>>(L);
        else sw_split_kernel<false, 0, false><<<g, 256, 0, s>>>(L);
    }
    note_launch();
    return check_launch();
}

int sw_split2_launch(const SplitLaunch &L, cudaStream_t s)
{
    const int64_t total = (L.rows / 4) * (L.cols / 512) * L.nparent;
    if (total <= 0) return GF2_OK;
    const bool top = (L.vrows != L.rows) || (L.vcols != L.cols) || (L.ld & 1) ||
                     (reinterpret_cast<uintptr_t>(L.X) & 15);
    if (L.xkind && (!L.xout || (reinterpret_cast<uintptr_t>(L.xout) & 15) || (L.rowbytes & 15))) return GF2_ELAYOUT;
    ProfScope ps(PF_SPLIT, s);
    const unsigned g = (unsigned)grid_for(total);
    // whole warps on one row's 64 words when a child row has a multiple of 32 word pairs
    const bool coop = (L.cols / 512) % 32 == 0;
    if (L.xkind == KIND_F8 + 1) {
        if (coop) { if (top) sw_split2_kernel<true, KIND_F8 + 1, true><<<g, 256, 0, s>>>(L); else sw_split2_kernel<false, KIND_F8 + 1, true><<<g, 256, 0, s>>>(L); }
        else { if (top) sw_split2_kernel<true, KIND_F8 + 1, false><<<g, 256, 0, s>>>(L); else sw_split2_kernel<false, KIND_F8 + 1, false><<<g, 256, 0, s>>>(L); }
    } else if (L.xkind == KIND_F4 + 1) {
        if (coop) { if (top) sw_split2_kernel<true, KIND_F4 + 1, true><<<g, 256, 0, s>>>(L); else sw_split2_kernel<false, KIND_F4 + 1, true><<<g, 256, 0, s>>>(L); }
        else { if (top) sw_split2_kernel<true, KIND_F4 + 1, false><<<g, 256, 0, s>>>(L); else sw_split2_kernel<false, KIND_F4 + 1, false><<<g, 256, 0, s>>>(L); }
    } else {
        if (top) sw_split2_kernel<true, 0, false><<<g, 256, 0, s>>>(L);
        else sw_split2_kernel<false, 0, false><<<g, 256, 0, s>>>(L);
    }
    note_launch();
    return check_launch();
}

int sw_combine2_launch(const CombineLaunch &L, cudaStream_t s)
{
    const int64_t total = (L.rows / 4) * (L.cols / 512) * L.nparent;
    if (total <= 0) return GF2_OK;
    const bool top = (L.vrows != L.rows) || (L.vcols != L.cols) || (L.ld & 1) ||
                     (reinterpret_cast<uintptr_t>(L.X) & 15);
    ProfScope ps(PF_COMBINE, s);
    if (top)
        sw_combine2_kernel<true><<<grid_for(total), 256, 0, s>>>(L);
    else
        sw_combine2_kernel<false><<<grid_for(total), 256, 0, s>>>(L);
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
