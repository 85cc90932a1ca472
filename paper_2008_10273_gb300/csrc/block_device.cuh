// Device building blocks of the block residual (Sec. 2.2, Eqs. 2-3) used by
// the block kernels (k_block.cu).
//
// G of every block shape w x h (w, h <= 16) is stored whole: row i of the
// N x N matrix (N = w h, pixel index y w + x) at tab.G + tab.goff[shape] +
// i * rowlen(N), rows padded to a multiple of 8 floats with zeros.  Since G
// is symmetric, row p_j is the Green's function of point p_j (Eq. 2), so
//   r = a + sum_j c_j G[p_j, :]                       (Eq. 3)
// is a sum of coalesced row loads, and G_PP is a gather of single entries.
#pragma once

#include "hivc_internal.cuh"

namespace hivc {

__host__ __device__ __forceinline__ int g_rowlen(int n) { return (n + 7) & ~7; }
__host__ __device__ __forceinline__ int shape_index(int w, int h) { return (w - 1) * 16 + (h - 1); }

__device__ __forceinline__ const float *green_rows(const BlockTables &t, int w, int h)
{
    return t.G + __ldg(t.goff + shape_index(w, h));
}

// The 16 x 16 block is symmetric under the 8 symmetries of the square
// (reflections x -> 15 - x, y -> 15 - y, the transpose), and so is its
// operator with mirrored boundaries: G[p, q] = G[s(p), s(q)] for each such
// s.  Every point p maps to one of the 36 points (bx, by), bx <= by <= 7,
// by s = (reflect x if rx) then (reflect y if ry) then (transpose if tr);
// bi = by (by + 1) / 2 + bx numbers them.  The tables are built so that
// this holds bit for bit (the rows of the 36 points define the others).
struct Sym16 {
    int bi, rx, ry, tr;
};
__host__ __device__ __forceinline__ Sym16 sym16(int p)
{
    const int px = p & 15, py = p >> 4;
    Sym16 s;
    s.rx = px > 7;
    s.ry = py > 7;
    const int fx = s.rx ? 15 - px : px, fy = s.ry ? 15 - py : py;
    s.tr = fx > fy;
    const int bx = s.tr ? fy : fx, by = s.tr ? fx : fy;
    s.bi = by * (by + 1) / 2 + bx;
    return s;
}
// s(q) for the symmetry of sym16(p)
__host__ __device__ __forceinline__ int sym16_apply(const Sym16 &s, int q)
{
    int x = q & 15, y = q >> 4;
    x = s.rx ? 15 - x : x;
    y = s.ry ? 15 - y : y;
    return s.tr ? x * 16 + y : y * 16 + x;
}
// Rows of the 36 points in 4 orientations o = rx + 2 tr, so that a point's
// row is read as contiguous runs: G[p, (x, y)] = G16o[o][bi][ry ? 15 - y :
// y][x] (256 floats per row, y * 16 + x).
constexpr int kSym16Rows = 36;
constexpr size_t kSym16Floats = (size_t)4 * kSym16Rows * 256;

// the job holding global block gb: the last k with p[k].block_base <= gb
// (block bases increase with k; binary search over at most kMaxJobs)
__device__ __forceinline__ int find_job(const BlockJobs &J, int gb)
{
    int lo = 0, hi = J.n - 1;
#pragma unroll 1
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (gb >= J.p[mid].block_base) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct BlockGeom {
    int lb, w, h, x0, y0;
    uint32_t s;
    int K;
    uint32_t bad;  // error bits for block_ptr / K
};

__device__ __forceinline__ BlockGeom block_geom(const BlockPlane &P, int lb)
{
    BlockGeom g;
    g.lb = lb;
    const int bx = lb % P.nbx, by = lb / P.nbx;
    g.x0 = bx * P.block;
    g.y0 = by * P.block;
    g.w = min(P.block, P.width - g.x0);
    g.h = min(P.block, P.height - g.y0);
    const uint32_t s = __ldg(P.block_ptr + lb), e = __ldg(P.block_ptr + lb + 1);
    g.bad = 0;
    if (e < s || e > (uint32_t)P.n_points || (lb == 0 && s != 0)) g.bad = kFlagBlockPtr;
    g.s = s;
    g.K = g.bad ? 0 : (int)(e - s);
    if (!g.bad && g.K > g.w * g.h - 1) {
        g.bad = kFlagK;
        g.K = 0;
    }
    return g;
}

// Position j of the block (index y w + x): inside and strictly increasing.
__device__ __forceinline__ bool load_pos(const BlockPlane &P, const BlockGeom &g, int j, int &p)
{
    p = __ldg(P.pos + g.s + j);
    const int prev = j > 0 ? (int)__ldg(P.pos + g.s + j - 1) : -1;
    return p < g.w * g.h && p > prev;
}

// Sum over the lanes of a SEG-lane segment.
template <int SEG>
__device__ __forceinline__ float seg_sum(float v)
{
#pragma unroll
    for (int o = SEG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, SEG);
    return v;
}

// Coefficients of one block per SEG-lane segment (SEG = 8, 16 or 32) with
// K <= KM <= SEG points (KM a compile-time bound, so every loop unrolls
// without exits).  Lane i < K of the segment holds point p (its index in
// the block) and the values v0 (v1: a second plane with the same points);
// on return c0 (c1) and the segment-uniform a0 (a1).
//   G_PP = L L^T (row i of G_PP and of L in lane i's registers)
//   L y_v = v, L y_1 = 1;  a = (y_1 . y_v) / (y_1 . y_1) = 1^T G^-1 v / 1^T G^-1 1
//   L^T c = y_v - a y_1   (so sum c = 0 and G_PP c + a 1 = v)
// Rows i >= K are zero rows and stay zero, so no step needs a K test: a
// zero pivot only scales zeros.  Lt is SEG x (SEG+1) shared scratch per
// segment for the transpose of L.  Returns false if a pivot of a real row
// was not positive.
template <int SEG, int KM, bool TWO>
__device__ __forceinline__ bool seg_block_coef(const float *__restrict__ G, int rl, int K, int i, int p, float v0,
                                               float v1, float (*Lt)[SEG + 1], float &c0, float &c1, float &a0,
                                               float &a1)
{
    float a[KM];
    const float *row = G + p * rl;
    const bool live = i < K;
#pragma unroll
    for (int j = 0; j < KM; ++j) {
        const int pj = __shfl_sync(0xffffffffu, p, j, SEG);
        a[j] = (live && j <= i && j < K) ? __ldg(row + pj) : 0.f;
    }
    bool spd = true;
    float ri = 0.f;  // 1 / L_ii
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const float d = __shfl_sync(0xffffffffu, a[k], k, SEG);
        spd = spd && (k >= K || d > 0.f);
        const float isd = rsqrtf(fmaxf(d, 1e-30f));
        const bool isk = i == k, below = i > k;
        a[k] = isk ? d * isd : (below ? a[k] * isd : a[k]);
        ri = isk ? isd : ri;
        const float lik = below ? a[k] : 0.f;
#pragma unroll
        for (int j = 1; j < KM; ++j) {  // constant trip count: unrolls fully
            if (j > k) {
                const float ljk = __shfl_sync(0xffffffffu, a[k], j, SEG);
                a[j] = j <= i ? fmaf(-lik, ljk, a[j]) : a[j];
            }
        }
    }
    // forward: L y = b for b = v0, v1, 1
    float y0 = live ? v0 : 0.f, y1 = live ? v1 : 0.f, y2 = live ? 1.f : 0.f;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const float inv = __shfl_sync(0xffffffffu, ri, k, SEG);
        const float z0 = __shfl_sync(0xffffffffu, y0, k, SEG) * inv;
        const float z1 = TWO ? __shfl_sync(0xffffffffu, y1, k, SEG) * inv : 0.f;
        const float z2 = __shfl_sync(0xffffffffu, y2, k, SEG) * inv;
        const bool isk = i == k, below = i > k;
        y0 = isk ? z0 : (below ? fmaf(-a[k], z0, y0) : y0);
        if (TWO) y1 = isk ? z1 : (below ? fmaf(-a[k], z1, y1) : y1);
        y2 = isk ? z2 : (below ? fmaf(-a[k], z2, y2) : y2);
    }
    const float r22 = __frcp_rn(seg_sum<SEG>(y2 * y2));
    a0 = seg_sum<SEG>(y2 * y0) * r22;
    a1 = TWO ? seg_sum<SEG>(y2 * y1) * r22 : 0.f;
    float b0 = fmaf(-a0, y2, y0), b1 = TWO ? fmaf(-a1, y2, y1) : 0.f;
    // backward: L^T c = b, with column i of L read back from Lt
#pragma unroll
    for (int j = 0; j < KM; ++j) Lt[i][j] = a[j];
    __syncwarp();
#pragma unroll
    for (int k = KM - 1; k >= 0; --k) {
        const float inv = __shfl_sync(0xffffffffu, ri, k, SEG);
        const float z0 = __shfl_sync(0xffffffffu, b0, k, SEG) * inv;
        const float z1 = TWO ? __shfl_sync(0xffffffffu, b1, k, SEG) * inv : 0.f;
        const bool isk = i == k, above = i < k;
        const float l = above ? Lt[k][i] : 0.f;  // L[k][i]
        b0 = isk ? z0 : fmaf(-l, z0, b0);
        if (TWO) b1 = isk ? z1 : fmaf(-l, z1, b1);
    }
    __syncwarp();
    c0 = b0;
    c1 = b1;
    return spd;
}


// Coefficients of one block with 16 < K <= 32 by one warp, G_PP factored
// in shared memory (M is 32 x 33); same outputs as seg_block_coef with
// SEG = 32.  Lane i < K holds point p and the values.
__device__ __forceinline__ bool warp_block_coef_smem(const float *__restrict__ G, int rl, int K, int i, int p,
                                                     float v0, float v1, float (*M)[33], float &c0, float &c1,
                                                     float &a0, float &a1)
{
    const bool live = i < K;
    const float *row = G + p * rl;
    for (int j = 0; j < K; ++j) {
        const int pj = __shfl_sync(0xffffffffu, p, j);
        if (live && j <= i) M[i][j] = __ldg(row + pj);
    }
    __syncwarp();
    bool spd = true;
    for (int k = 0; k < K; ++k) {
        const float d = M[k][k];
        spd = spd && d > 0.f;
        const float isd = rsqrtf(fmaxf(d, 1e-30f));
        __syncwarp();
        if (i == k) M[k][k] = d * isd;
        else if (i > k && live) M[i][k] *= isd;
        __syncwarp();
        if (i > k && live) {
            const float lik = M[i][k];
            for (int j = k + 1; j <= i; ++j) M[i][j] = fmaf(-lik, M[j][k], M[i][j]);
        }
        __syncwarp();
    }
    float y0 = live ? v0 : 0.f, y1 = live ? v1 : 0.f, y2 = live ? 1.f : 0.f;
    for (int k = 0; k < K; ++k) {
        const float inv = 1.0f / M[k][k];
        const float z0 = __shfl_sync(0xffffffffu, y0, k) * inv;
        const float z1 = __shfl_sync(0xffffffffu, y1, k) * inv;
        const float z2 = __shfl_sync(0xffffffffu, y2, k) * inv;
        if (i == k) {
            y0 = z0; y1 = z1; y2 = z2;
        } else if (i > k && live) {
            const float l = M[i][k];
            y0 = fmaf(-l, z0, y0); y1 = fmaf(-l, z1, y1); y2 = fmaf(-l, z2, y2);
        }
    }
    const float r22 = __frcp_rn(seg_sum<32>(y2 * y2));
    a0 = seg_sum<32>(y2 * y0) * r22;
    a1 = seg_sum<32>(y2 * y1) * r22;
    float b0 = fmaf(-a0, y2, y0), b1 = fmaf(-a1, y2, y1);
    for (int k = K - 1; k >= 0; --k) {
        const float inv = 1.0f / M[k][k];
        const float z0 = __shfl_sync(0xffffffffu, b0, k) * inv;
        const float z1 = __shfl_sync(0xffffffffu, b1, k) * inv;
        if (i == k) {
            b0 = z0; b1 = z1;
        } else if (i < k) {
            const float l = M[k][i];
            b0 = fmaf(-l, z0, b0); b1 = fmaf(-l, z1, b1);
        }
    }
    __syncwarp();
    c0 = b0;
    c1 = b1;
    return spd;
}

}  // namespace hivc
