// Block-based pseudodifferential inpainting of the residual (Sec. 2.2,
// Eqs. 2-4; Sec. 2.3), harmonic operator A = -L with mirrored boundaries on
// each w x h block (w, h <= 16).
//
// Per block with K points p_j and values v_j:
//   1. coefficients: the (K+1) x (K+1) saddle system
//        [G_PP 1; 1^T 0] [c; a] = [v; 0]
//      solved as a = 1^T G_PP^-1 v / 1^T G_PP^-1 1, c = G_PP^-1 (v - a 1),
//      with G_PP = L L^T (Cholesky; G_PP is SPD for 1 <= K < w*h because G
//      is the pseudo-inverse of A and E_P x is never constant).
//      G(x, x') is read from a per-shape table T on a 2w x 2h grid:
//        G = T(|dx|,|dy|) + T(|dx|,sy) + T(sx,|dy|) + T(sx,sy),
//        sx = x + x' + 1, sy = y + y' + 1,
//        T(al, be) = 1/4 sum_{(p,q)!=0} c_p^2 c_q^2 cos(pi p al/w) cos(pi q be/h) / mu_pq,
//      the Toeplitz-plus-Hankel structure of G stated in Sec. 2.2.
//   2. evaluation by Eq. (4): spectrum D = lambda o C(M c) of the sparse
//      coefficient image (lambda = 1/mu, 0 for the constant mode), inverse
//      2-D DCT-II as two 16-point matrix passes, + a; r(p_j) = v_j.
//
// Tables are computed on the host in double precision and stored as float.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "hivc_internal.cuh"

namespace hivc {
namespace {

// ---- table layout --------------------------------------------------------
// DCT-II basis for n = 1..16:  phi_n[p*n + x] at offset sum_{m<n} m^2.
constexpr int kPhiSize = 1496;  // sum_{n=1}^{16} n^2
// Per shape (w, h) in 1..16: w*h spectral weights, 4*w*h Green's table.
constexpr int kShapeSize = 18496;  // (sum_{n=1}^{16} n)^2
constexpr int kTSize = 4 * kShapeSize;

__host__ __device__ __forceinline__ int phi_off(int n) { return (n - 1) * n * (2 * n - 1) / 6; }
__host__ __device__ __forceinline__ int tri(int n) { return n * (n + 1) / 2; }
// offset of shape (w, h) among all shapes, w-major
__host__ __device__ __forceinline__ int shape_off(int w, int h) { return tri(w - 1) * 136 + w * tri(h - 1); }

static __device__ float d_phi[kPhiSize];
static __device__ float d_lam[kShapeSize];
static __device__ float d_T[kTSize];

std::mutex g_tab_mu;
uint64_t g_tab_devices = 0;  // bit d: tables uploaded to device d

void build_tables(std::vector<float> &phi, std::vector<float> &lam, std::vector<float> &T)
{
    const double pi = 3.14159265358979323846;
    phi.assign(kPhiSize, 0.f);
    lam.assign(kShapeSize, 0.f);
    T.assign(kTSize, 0.f);
    std::vector<double> c2(17 * 17), mu1(17 * 17);
    for (int n = 1; n <= 16; ++n)
        for (int p = 0; p < n; ++p) {
            double c = p == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
            c2[n * 17 + p] = c * c;
            double s = std::sin(pi * p / (2.0 * n));
            mu1[n * 17 + p] = 4.0 * s * s;
            for (int x = 0; x < n; ++x)
                phi[phi_off(n) + p * n + x] = (float)(c * std::cos(pi * p * (2.0 * x + 1.0) / (2.0 * n)));
        }
    std::vector<double> cw(32 * 16), ch(32 * 16);
    for (int w = 1; w <= 16; ++w)
        for (int h = 1; h <= 16; ++h) {
            const int so = shape_off(w, h);
            for (int q = 0; q < h; ++q)
                for (int p = 0; p < w; ++p) {
                    double mu = mu1[w * 17 + p] + mu1[h * 17 + q];
                    lam[so + q * w + p] = (p == 0 && q == 0) ? 0.f : (float)(1.0 / mu);
                }
            for (int a = 0; a < 2 * w; ++a)
                for (int p = 0; p < w; ++p) cw[a * 16 + p] = std::cos(pi * p * a / w);
            for (int b = 0; b < 2 * h; ++b)
                for (int q = 0; q < h; ++q) ch[b * 16 + q] = std::cos(pi * q * b / h);
            float *Tw = T.data() + 4 * so;
            for (int b = 0; b < 2 * h; ++b)
                for (int a = 0; a < 2 * w; ++a) {
                    double s = 0.0;
                    for (int q = 0; q < h; ++q)
                        for (int p = 0; p < w; ++p) {
                            if (p == 0 && q == 0) continue;
                            double mu = mu1[w * 17 + p] + mu1[h * 17 + q];
                            s += c2[w * 17 + p] * c2[h * 17 + q] * cw[a * 16 + p] * ch[b * 16 + q] / mu;
                        }
                    Tw[b * (2 * w) + a] = (float)(0.25 * s);
                }
        }
}

// ---- device helpers ------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float green(const float *__restrict__ T, int w2, int xi, int yi, int xj, int yj)
{
    const int a1 = abs(xi - xj), a2 = xi + xj + 1, b1 = abs(yi - yj), b2 = yi + yj + 1;
    return (__ldg(T + b1 * w2 + a1) + __ldg(T + b2 * w2 + a1)) + (__ldg(T + b1 * w2 + a2) + __ldg(T + b2 * w2 + a2));
}

__device__ __forceinline__ int find_job(const BlockJobs &J, int gb)
{
    int j = 0;
#pragma unroll 1
    for (int k = 1; k < J.n; ++k)
        if (gb >= J.p[k].block_base) j = k;
    return j;
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

// Positions of one 32-point chunk: validity (inside, increasing).
__device__ __forceinline__ bool load_point(const BlockPlane &P, const BlockGeom &g, int j, int &px, int &py)
{
    const int p = __ldg(P.pos + g.s + j);
    const int prev = j > 0 ? (int)__ldg(P.pos + g.s + j - 1) : -1;
    px = p % g.w;
    py = p / g.w;
    return p < g.w * g.h && p > prev;
}

// ---- coefficient stage: one warp per block, K <= 32 ----------------------
__global__ void __launch_bounds__(128) block_coef_kernel(const __grid_constant__ BlockJobs J, BlockScratch S)
{
    __shared__ float smat[4][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * 4 + warp;
    if (gb >= J.total_blocks) return;
    const BlockPlane &P = J.p[find_job(J, gb)];
    const BlockGeom g = block_geom(P, gb - P.block_base);
    if (g.bad) {
        if (lane == 0) atomicOr(S.flags, g.bad);
        return;
    }
    const int K = g.K;
    if (K == 0) return;
    if (K > kWarpK) {
        if (lane == 0) {
            const uint32_t i = atomicAdd(S.large_count, 1u);
            if (i < (uint32_t)S.large_cap) S.large_list[i] = (uint32_t)gb;
        }
        return;
    }
    const bool two = P.val[1] != nullptr;
    int px = 0, py = 0;
    float v0 = 0.f, v1 = 0.f;
    bool ok = true;
    if (lane < K) {
        ok = load_point(P, g, lane, px, py);
        v0 = (float)__ldg(P.val[0] + g.s + lane);
        if (two) v1 = (float)__ldg(P.val[1] + g.s + lane);
    }
    if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0) atomicOr(S.flags, kFlagPos);
        return;
    }
    const float *T = d_T + 4 * shape_off(g.w, g.h);
    const int w2 = 2 * g.w;
    float(*M)[33] = smat[warp];
    // assemble the lower triangle of G_PP, lane i owns row i
    for (int j = 0; j < K; ++j) {
        const int xj = __shfl_sync(0xffffffffu, px, j), yj = __shfl_sync(0xffffffffu, py, j);
        if (lane < K && j <= lane) M[lane][j] = green(T, w2, px, py, xj, yj);
    }
    __syncwarp();
    // Cholesky G_PP = L L^T in place (right-looking)
    bool spd = true;
    for (int k = 0; k < K; ++k) {
        float d = M[k][k];
        spd = spd && (d > 0.f);
        d = fmaxf(d, 1e-30f);
        const float sd = sqrtf(d), isd = 1.0f / sd;
        __syncwarp();
        if (lane == k) M[k][k] = sd;
        else if (lane > k && lane < K) M[lane][k] *= isd;
        __syncwarp();
        if (lane > k && lane < K) {
            const float lik = M[lane][k];
            for (int j = k + 1; j <= lane; ++j) M[lane][j] = fmaf(-lik, M[j][k], M[lane][j]);
        }
        __syncwarp();
    }
    // L y = [v0 v1 1], then L^T z = y; lane i holds entry i
    float b0 = v0, b1 = v1, b2 = lane < K ? 1.f : 0.f;
    for (int k = 0; k < K; ++k) {
        const float inv = 1.0f / M[k][k];
        const float y0 = __shfl_sync(0xffffffffu, b0, k) * inv;
        const float y1 = __shfl_sync(0xffffffffu, b1, k) * inv;
        const float y2 = __shfl_sync(0xffffffffu, b2, k) * inv;
        if (lane == k) {
            b0 = y0; b1 = y1; b2 = y2;
        } else if (lane > k && lane < K) {
            const float l = M[lane][k];
            b0 = fmaf(-l, y0, b0); b1 = fmaf(-l, y1, b1); b2 = fmaf(-l, y2, b2);
        }
    }
    for (int k = K - 1; k >= 0; --k) {
        const float inv = 1.0f / M[k][k];
        const float z0 = __shfl_sync(0xffffffffu, b0, k) * inv;
        const float z1 = __shfl_sync(0xffffffffu, b1, k) * inv;
        const float z2 = __shfl_sync(0xffffffffu, b2, k) * inv;
        if (lane == k) {
            b0 = z0; b1 = z1; b2 = z2;
        } else if (lane < k) {
            const float l = M[k][lane];
            b0 = fmaf(-l, z0, b0); b1 = fmaf(-l, z1, b1); b2 = fmaf(-l, z2, b2);
        }
    }
    // a = 1^T G^-1 v / 1^T G^-1 1 ;  c = G^-1 v - a G^-1 1  (sum c = 0)
    const float s2 = warp_sum(lane < K ? b2 : 0.f);
    const float a0 = warp_sum(lane < K ? b0 : 0.f) / s2;
    const float a1 = two ? warp_sum(lane < K ? b1 : 0.f) / s2 : 0.f;
    if (lane < K) {
        P.coef[0][g.s + lane] = fmaf(-a0, b2, b0);
        if (two) P.coef[1][g.s + lane] = fmaf(-a1, b2, b1);
    }
    if (lane == 0) {
        P.acoef[0][g.lb] = a0;
        if (two) P.acoef[1][g.lb] = a1;
        if (!spd) atomicOr(S.flags, kFlagNotSPD);
    }
}

// ---- coefficient stage for K > 32: one CTA per block, packed Cholesky ----
constexpr int kLargeThreads = 256;
constexpr int kLargeMaxK = 255;
constexpr size_t kLargeSmem =
    sizeof(float) * ((size_t)kLargeMaxK * (kLargeMaxK + 1) / 2 + 3 * kLargeMaxK) + sizeof(int) * 2 * kLargeMaxK;

__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

__global__ void __launch_bounds__(kLargeThreads) block_coef_large_kernel(const __grid_constant__ BlockJobs J,
                                                                         BlockScratch S)
{
    extern __shared__ float sm[];
    __shared__ float red[3][kLargeThreads / 32];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    const uint32_t count = min(*S.large_count, (uint32_t)S.large_cap);
    for (uint32_t it = blockIdx.x; it < count; it += gridDim.x) {
        const int gb = (int)S.large_list[it];
        const BlockPlane &P = J.p[find_job(J, gb)];
        const BlockGeom g = block_geom(P, gb - P.block_base);
        const int K = g.K;  // > 32 and valid by construction of the list
        const bool two = P.val[1] != nullptr;
        float *L = sm;
        float *b = sm + (size_t)K * (K + 1) / 2;  // b[r*K + i]
        int *px = reinterpret_cast<int *>(b + 3 * K);
        int *py = px + K;
        if (tid == 0) s_bad = 0;
        __syncthreads();
        for (int j = tid; j < K; j += kLargeThreads) {
            int x, y;
            if (!load_point(P, g, j, x, y)) s_bad = 1;
            px[j] = x;
            py[j] = y;
            b[j] = (float)__ldg(P.val[0] + g.s + j);
            b[K + j] = two ? (float)__ldg(P.val[1] + g.s + j) : 0.f;
            b[2 * K + j] = 1.f;
        }
        __syncthreads();
        if (s_bad) {
            if (tid == 0) atomicOr(S.flags, kFlagPos);
            __syncthreads();
            continue;
        }
        const float *T = d_T + 4 * shape_off(g.w, g.h);
        const int w2 = 2 * g.w;
        for (int i = tid; i < K; i += kLargeThreads)
            for (int j = 0; j <= i; ++j) L[pk(i, j)] = green(T, w2, px[i], py[i], px[j], py[j]);
        __syncthreads();
        bool spd = true;
        for (int k = 0; k < K; ++k) {
            const float d = L[pk(k, k)];
            spd = spd && d > 0.f;
            const float sd = sqrtf(fmaxf(d, 1e-30f)), isd = 1.0f / sd;
            __syncthreads();
            if (tid == 0) L[pk(k, k)] = sd;
            for (int i = k + 1 + tid; i < K; i += kLargeThreads) L[pk(i, k)] *= isd;
            __syncthreads();
            for (int i = k + 1 + tid; i < K; i += kLargeThreads) {
                const float lik = L[pk(i, k)];
                for (int j = k + 1; j <= i; ++j) L[pk(i, j)] = fmaf(-lik, L[pk(j, k)], L[pk(i, j)]);
            }
            __syncthreads();
        }
        for (int k = 0; k < K; ++k) {
            if (tid < 3) b[tid * K + k] /= L[pk(k, k)];
            __syncthreads();
            for (int i = k + 1 + tid; i < K; i += kLargeThreads) {
                const float l = L[pk(i, k)];
                b[i] = fmaf(-l, b[k], b[i]);
                b[K + i] = fmaf(-l, b[K + k], b[K + i]);
                b[2 * K + i] = fmaf(-l, b[2 * K + k], b[2 * K + i]);
            }
            __syncthreads();
        }
        for (int k = K - 1; k >= 0; --k) {
            if (tid < 3) b[tid * K + k] /= L[pk(k, k)];
            __syncthreads();
            for (int i = tid; i < k; i += kLargeThreads) {
                const float l = L[pk(k, i)];
                b[i] = fmaf(-l, b[k], b[i]);
                b[K + i] = fmaf(-l, b[K + k], b[K + i]);
                b[2 * K + i] = fmaf(-l, b[2 * K + k], b[2 * K + i]);
            }
            __syncthreads();
        }
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int i = tid; i < K; i += kLargeThreads) {
            s0 += b[i];
            s1 += b[K + i];
            s2 += b[2 * K + i];
        }
        s0 = warp_sum(s0);
        s1 = warp_sum(s1);
        s2 = warp_sum(s2);
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = s0;
            red[1][tid >> 5] = s1;
            red[2][tid >> 5] = s2;
        }
        __syncthreads();
        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
        for (int k = 0; k < kLargeThreads / 32; ++k) {
            t0 += red[0][k];
            t1 += red[1][k];
            t2 += red[2][k];
        }
        const float a0 = t0 / t2, a1 = t1 / t2;
        for (int i = tid; i < K; i += kLargeThreads) {
            P.coef[0][g.s + i] = fmaf(-a0, b[2 * K + i], b[i]);
            if (two) P.coef[1][g.s + i] = fmaf(-a1, b[2 * K + i], b[K + i]);
        }
        if (tid == 0) {
            P.acoef[0][g.lb] = a0;
            if (two) P.acoef[1][g.lb] = a1;
            if (!spd) atomicOr(S.flags, kFlagNotSPD);
        }
        __syncthreads();
    }
}

// ---- evaluation stage: r = C^-1 diag(lambda) C (M c) + a, one warp/block --
__global__ void __launch_bounds__(128) block_eval_kernel(const __grid_constant__ BlockJobs J, uint32_t *flags)
{
    __shared__ float sD[4][16][17];  // D[q][p]
    __shared__ float sE[4][16][17];  // E[q][x]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * 4 + warp;
    if (gb >= J.total_blocks) return;
    const BlockPlane &P = J.p[find_job(J, gb)];
    const BlockGeom g = block_geom(P, gb - P.block_base);
    const int K = g.K, w = g.w, h = g.h;
    bool valid = true;
    for (int j0 = 0; j0 < K; j0 += 32) {
        int x, y;
        const bool ok = (j0 + lane < K) ? load_point(P, g, j0 + lane, x, y) : true;
        valid = valid && !__any_sync(0xffffffffu, !ok);
    }
    if (!valid && lane == 0) atomicOr(flags, kFlagPos);
    const int nch = P.val[1] != nullptr ? 2 : 1;
    const float *phw = d_phi + phi_off(w);
    const float *phh = d_phi + phi_off(h);
    const float *lam = d_lam + shape_off(w, h);
    const int p = lane & 15, xq = lane & 15, q0 = (lane >> 4) * 8;
    for (int ch = 0; ch < nch; ++ch) {
        float *R = P.r[ch];
        if (R == nullptr) continue;
        float *Rb = R + (size_t)g.y0 * P.r_pitch + g.x0;
        if (K == 0 || !valid) {
            for (int i = lane; i < w * h; i += 32) Rb[(i / w) * P.r_pitch + (i % w)] = 0.f;
            continue;
        }
        // sparse forward transform of the coefficient image
        float acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.f;
        for (int j0 = 0; j0 < K; j0 += 32) {
            int cx = 0, cy = 0;
            float cc = 0.f;
            if (j0 + lane < K) {
                const int pp = __ldg(P.pos + g.s + j0 + lane);
                cx = pp % w;
                cy = pp / w;
                cc = __ldg(P.coef[ch] + g.s + j0 + lane);
            }
            const int n = min(32, K - j0);
            for (int t = 0; t < n; ++t) {
                const int xj = __shfl_sync(0xffffffffu, cx, t);
                const int yj = __shfl_sync(0xffffffffu, cy, t);
                const float cj = __shfl_sync(0xffffffffu, cc, t);
                const float tp = p < w ? cj * __ldg(phw + p * w + xj) : 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int q = q0 + k;
                    if (q < h) acc[k] = fmaf(tp, __ldg(phh + q * h + yj), acc[k]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int q = q0 + k;
            sD[warp][q][p] = (p < w && q < h) ? acc[k] * __ldg(lam + q * w + p) : 0.f;
        }
        __syncwarp();
        // inverse transform, pass 1 (x): E(q, x) = sum_p phi_w(p, x) D(p, q)
        float e8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) e8[k] = 0.f;
        for (int pp = 0; pp < w; ++pp) {
            const float f = xq < w ? __ldg(phw + pp * w + xq) : 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) e8[k] = fmaf(f, sD[warp][q0 + k][pp], e8[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) sE[warp][q0 + k][xq] = e8[k];
        __syncwarp();
        // pass 2 (y): r(x, y) = sum_q phi_h(q, y) E(q, x) + a
        const float a = __ldg(P.acoef[ch] + g.lb);
        float r8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) r8[k] = a;
        const int y0 = q0;
        for (int q = 0; q < h; ++q) {
            const float ev = sE[warp][q][xq];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (y0 + k < h) r8[k] = fmaf(__ldg(phh + q * h + y0 + k), ev, r8[k]);
        }
        if (xq < w) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (y0 + k < h) Rb[(size_t)(y0 + k) * P.r_pitch + xq] = r8[k];
        }
        __syncwarp();
        // the data at the points, exactly
        for (int j = lane; j < K; j += 32) {
            const int pp = __ldg(P.pos + g.s + j);
            Rb[(size_t)(pp / w) * P.r_pitch + (pp % w)] = (float)__ldg(P.val[ch] + g.s + j);
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t ensure_block_tables()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (dev < 64 && (g_tab_devices >> dev) & 1ull) return cudaSuccess;
    static std::vector<float> phi, lam, T;
    if (phi.empty()) build_tables(phi, lam, T);
    if ((e = cudaMemcpyToSymbol(d_phi, phi.data(), phi.size() * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(d_lam, lam.data(), lam.size() * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(d_T, T.data(), T.size() * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(block_coef_large_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kLargeSmem)) != cudaSuccess)
        return e;
    if (dev < 64) g_tab_devices |= 1ull << dev;
    return cudaSuccess;
}

cudaError_t launch_block_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st, int *launches)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(s.large_count, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    block_coef_kernel<<<(jobs.total_blocks + 3) / 4, 128, 0, st>>>(jobs, s);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(sms, jobs.total_blocks));
    block_coef_large_kernel<<<grid, kLargeThreads, kLargeSmem, st>>>(jobs, s);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_block_eval(const BlockJobs &jobs, uint32_t *flags, cudaStream_t st)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    block_eval_kernel<<<(jobs.total_blocks + 3) / 4, 128, 0, st>>>(jobs, flags);
    return cudaGetLastError();
}

}  // namespace hivc
