// Block-based pseudodifferential inpainting of the residual (Sec. 2.2,
// Eqs. 2-4; Sec. 2.3), harmonic operator A = -L (or the biharmonic L^2)
// with mirrored boundaries on each w x h block (w, h <= 16).
//
// Per block with K points p_j and values v_j:
//   1. coefficients: the (K+1) x (K+1) saddle system
//        [G_PP 1; 1^T 0] [c; a] = [v; 0]
//      solved through the Cholesky factor of G_PP (SPD for 1 <= K < w h:
//      G is the pseudo-inverse of A and E_P x is never constant);
//   2. evaluation of Eq. (3): r = G M c + a, r(p_j) = v_j.
//
// G of every shape is built once on the host in double precision from the
// DCT-II diagonalisation of A (Eq. 4): with c_p(n)^2 = 1/n (p = 0), 2/n,
// and mu_pq = 4 sin^2(pi p / 2w) + 4 sin^2(pi q / 2h),
//   G(x,y; x',y') = T(|x-x'|,|y-y'|) + T(|x-x'|,y+y'+1) + T(x+x'+1,|y-y'|) + T(x+x'+1,y+y'+1),
//   T(al, be) = 1/4 sum_{(p,q) != 0} c_p^2 c_q^2 cos(pi p al / w) cos(pi q be / h) / mu_pq
// (/ mu_pq^2 for the biharmonic operator)
// (the Toeplitz-plus-Hankel structure of G, Sec. 2.2), stored as float
// and, for the FP64 re-solve of blocks above the condition threshold, as
// double.
//
// Kernels: the coefficient stage (one thread per block for K <= 12; warps
// for K <= 32, two blocks at once in 16-lane halves when both have
// K <= 16; blocks with K > 32, and FP64 re-solves, by the CTA of the
// block's range, packed Cholesky in the range's scratch slot) and the
// evaluation into residual planes (one warp per block; also the
// coefficient mode, which dequantises instead of solving).
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "block_device.cuh"

namespace hivc {
namespace {

constexpr int kGSize = 2283904;  // sum over shapes of N * rowlen(N)

// one table per operator (0 harmonic, 1 biharmonic)
static __device__ __align__(256) float d_G[kNumOps * kGSize];
static __device__ __align__(256) double d_G64[kNumOps * kGSize];
static __device__ int d_goff[256];

std::mutex g_tab_mu;
BlockTables g_tabs[64][kNumOps];
uint64_t g_tab_devices = 0;  // bit d: tables uploaded to device d

// Tables of operator op: the Green's eigenvalues are 1/mu (harmonic) or
// 1/mu^2 (biharmonic, A = L^2); the eigenvectors, and with them the
// Toeplitz-plus-Hankel structure, are the same.
void build_tables(int op, std::vector<float> &G, std::vector<double> &G64, std::vector<int> &goff)
{
    const double pi = 3.14159265358979323846;
    G.assign(kGSize, 0.f);
    G64.assign(kGSize, 0.0);
    goff.assign(256, 0);
    int off = 0;
    std::vector<double> T, cw, chq;
    for (int w = 1; w <= 16; ++w)
        for (int h = 1; h <= 16; ++h) {
            const int N = w * h, rl = g_rowlen(N);
            goff[shape_index(w, h)] = off;
            T.assign(4 * N, 0.0);
            cw.assign(2 * w * w, 0.0);
            chq.assign(2 * h * h, 0.0);
            for (int a = 0; a < 2 * w; ++a)
                for (int p = 0; p < w; ++p) cw[a * w + p] = std::cos(pi * p * a / w) * (p == 0 ? 1.0 : 2.0) / w;
            for (int b = 0; b < 2 * h; ++b)
                for (int q = 0; q < h; ++q) chq[b * h + q] = std::cos(pi * q * b / h) * (q == 0 ? 1.0 : 2.0) / h;
            for (int b = 0; b < 2 * h; ++b)
                for (int a = 0; a < 2 * w; ++a) {
                    double s = 0.0;
                    for (int q = 0; q < h; ++q)
                        for (int p = 0; p < w; ++p) {
                            if (p == 0 && q == 0) continue;
                            const double sp = std::sin(pi * p / (2.0 * w)), sq = std::sin(pi * q / (2.0 * h));
                            const double mu = 4.0 * sp * sp + 4.0 * sq * sq;
                            s += cw[a * w + p] * chq[b * h + q] / (op == 1 ? mu * mu : mu);
                        }
                    T[b * 2 * w + a] = 0.25 * s;
                }
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    const int xi = i % w, yi = i / w, xj = j % w, yj = j / w;
                    const int a1 = std::abs(xi - xj), a2 = xi + xj + 1, b1 = std::abs(yi - yj), b2 = yi + yj + 1;
                    const double g = T[b1 * 2 * w + a1] + T[b2 * 2 * w + a1] + T[b1 * 2 * w + a2] + T[b2 * 2 * w + a2];
                    G[off + i * rl + j] = (float)g;
                    G64[off + i * rl + j] = g;
                }
            off += N * rl;
        }
}

// ---- coefficient stage ---------------------------------------------------
struct SegBlock {
    const BlockPlane *P;
    BlockGeom g;
};

// geometry of global block gb (no side effects); K = 0 for missing or bad
// blocks and for K > 32 (those go to the large-block kernel)
__device__ __forceinline__ SegBlock seg_block(const BlockJobs &J, int gb)
{
    SegBlock b;
    b.P = nullptr;
    b.g.K = 0;
    b.g.bad = 0;
    b.g.s = 0;
    b.g.w = b.g.h = 1;
    b.g.lb = 0;
    if (gb >= J.total_blocks) return b;
    b.P = &J.p[find_job(J, gb)];
    b.g = block_geom(*b.P, gb - b.P->block_base);
    return b;
}

__device__ __forceinline__ int seg_k(const SegBlock &b) { return (b.g.bad || b.g.K > kWarpK) ? 0 : b.g.K; }

// A block whose positions are bad gets a = NaN: the evaluation then takes
// its residual as zero.
__device__ __forceinline__ void mark_bad(const BlockPlane &P, int lb)
{
    P.acoef[0][lb] = __int_as_float(0x7fc00000);
    if (P.val[1] != nullptr) P.acoef[1][lb] = __int_as_float(0x7fc00000);
}

constexpr int kCoefThreads = 128;
constexpr int kF64Bit = 1 << 30;  // list entry: block re-solved in FP64

// The largest condition bound seen (non-negative floats order like their bits).
__device__ __forceinline__ void note_kappa(const BlockScratch &S, float kappa)
{
    if (S.cstat && kappa > 0.f) atomicMax(S.cstat, __float_as_uint(kappa));
}

// kappa = amax tr(G_PP) / (1 - K/N) >= cond_2(G_PP), amax >= the largest
// eigenvalue of the operator (8 harmonic, 64 biharmonic)
__device__ __forceinline__ float cond_bound(float amax, float tr, int K, int N)
{
    return amax * tr / (1.f - (float)K / (float)N);
}

// validity of the positions of a segment's block (inside, increasing):
// returns K, or 0 (and a flag) when any is bad
template <int SEG>
__device__ __forceinline__ int seg_validate(const SegBlock &b, int i, int seg, const BlockScratch &S)
{
    const int K = b.g.K;
    bool ok = true;
    if (i < K) {
        int p;
        ok = load_pos(*b.P, b.g, i, p);
    }
    const unsigned bad = __ballot_sync(0xffffffffu, !ok);
    const unsigned mine = SEG == 32 ? bad : (bad >> (seg * SEG)) & ((1u << SEG) - 1u);
    if (mine) {
        if (i == 0) {
            atomicOr(S.flags, kFlagPos);
            mark_bad(*b.P, b.g.lb);
        }
        return 0;
    }
    return K;
}

// One block with K <= KM <= SEG per segment of SEG lanes (lane i of the
// segment is point i), by the register routine, or (KM = 0, SEG = 32) by
// the shared-memory routine.  Lt: SEG x (SEG+1) floats of shared scratch.
// Writes c (per point) and a (per block).
// A block above the condition threshold goes to the CTA's list (entry
// gb | kF64Bit) for an FP64 re-solve after the warp phase.
template <int SEG, int KM>
__device__ __forceinline__ void seg_run(const SegBlock &b, int K, int i, float *Lt, const BlockTables &tab,
                                        const BlockScratch &S, int gb, int *s_list, int *s_n)
{
    const BlockPlane *P = b.P;
    const bool two = K > 0 && P->val[1] != nullptr;
    int p = 0;
    float v0 = 0.f, v1 = 0.f;
    if (i < K) {
        p = __ldg(P->pos + b.g.s + i);
        v0 = (float)__ldg(P->val[0] + b.g.s + i);
        if (two) v1 = (float)__ldg(P->val[1] + b.g.s + i);
    }
    const float *G = K > 0 ? green_rows(tab, b.g.w, b.g.h) : tab.G;
    const int rl = K > 0 ? g_rowlen(b.g.w * b.g.h) : 8;
    float c0, c1, a0, a1;
    bool spd;
    if constexpr (KM == 0)
        spd = warp_block_coef_smem(G, rl, K, i, p, v0, v1, reinterpret_cast<float(*)[33]>(Lt), c0, c1, a0, a1);
    else
        spd = seg_block_coef<SEG, KM, true>(G, rl, K, i, p, v0, v1, reinterpret_cast<float(*)[SEG + 1]>(Lt), c0, c1,
                                            a0, a1);
    const float tr = seg_sum<SEG>(i < K ? __ldg(G + p * rl + p) : 0.f);
    if (K > 0) {
        if (i < K) {
            P->coef[0][b.g.s + i] = c0;
            if (two) P->coef[1][b.g.s + i] = c1;
        }
        if (i == 0) {
            P->acoef[0][b.g.lb] = a0;
            if (two) P->acoef[1][b.g.lb] = a1;
            if (!spd) atomicOr(S.flags, kFlagNotSPD);
            const float kappa = cond_bound(tab.amax, tr, K, b.g.w * b.g.h);
            note_kappa(S, kappa);
            if (kappa > S.tau) s_list[atomicAdd(s_n, 1)] = gb | kF64Bit;
        }
    }
}

// ---- one thread per block (K <= kTK) -------------------------------------
constexpr int kTK = 12;
__host__ __device__ constexpr int tri(int i) { return i * (i + 1) / 2; }

// Coefficients of one block by one thread, K <= kTK: G_PP padded to
// kTK x kTK with the identity (the padding rows of L are unit rows and the
// padding entries of every solution are zero), Cholesky-Crout in
// registers, fully unrolled, so that no control flow depends on K.
//   L y_v = v, L y_1 = 1 (on the K points);  a = (y_1 . y_v) / (y_1 . y_1)
//   L^T c = y_v - a y_1
// Returns false if a pivot of a real row was not positive; tr = tr(G_PP).
template <bool TWO>
__device__ __forceinline__ bool thread_block_coef(const float *__restrict__ G, int rl, int K, const int (&p)[kTK],
                                                  const float (&v0)[kTK], const float (&v1)[kTK], float (&c0)[kTK],
                                                  float (&c1)[kTK], float &a0, float &a1, float &tr)
{
    float L[tri(kTK)], inv[kTK];
#pragma unroll
    for (int i = 0; i < kTK; ++i) {
        const float *row = G + p[i] * rl;
#pragma unroll
        for (int j = 0; j <= i; ++j) L[tri(i) + j] = (i < K && j < K) ? __ldg(row + p[j]) : (i == j ? 1.f : 0.f);
    }
    tr = 0.f;
#pragma unroll
    for (int i = 0; i < kTK; ++i)
        if (i < K) tr += L[tri(i) + i];
    bool spd = true;
#pragma unroll
    for (int k = 0; k < kTK; ++k) {
        float d = L[tri(k) + k];
#pragma unroll
        for (int m = 0; m < k; ++m) d = fmaf(-L[tri(k) + m], L[tri(k) + m], d);
        spd = spd && (k >= K || d > 0.f);
        const float isd = rsqrtf(fmaxf(d, 1e-30f));
        L[tri(k) + k] = d * isd;
        inv[k] = isd;
#pragma unroll
        for (int i = k + 1; i < kTK; ++i) {
            float s = L[tri(i) + k];
#pragma unroll
            for (int m = 0; m < k; ++m) s = fmaf(-L[tri(i) + m], L[tri(k) + m], s);
            L[tri(i) + k] = s * isd;
        }
    }
    float y0[kTK], y1[kTK], y2[kTK];
#pragma unroll
    for (int i = 0; i < kTK; ++i) {
        float s0 = v0[i], s1 = TWO ? v1[i] : 0.f, s2 = i < K ? 1.f : 0.f;
#pragma unroll
        for (int m = 0; m < i; ++m) {
            s0 = fmaf(-L[tri(i) + m], y0[m], s0);
            if (TWO) s1 = fmaf(-L[tri(i) + m], y1[m], s1);
            s2 = fmaf(-L[tri(i) + m], y2[m], s2);
        }
        y0[i] = s0 * inv[i];
        y1[i] = TWO ? s1 * inv[i] : 0.f;
        y2[i] = s2 * inv[i];
    }
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
#pragma unroll
    for (int i = 0; i < kTK; ++i) {
        d0 = fmaf(y2[i], y0[i], d0);
        if (TWO) d1 = fmaf(y2[i], y1[i], d1);
        d2 = fmaf(y2[i], y2[i], d2);
    }
    const float r22 = __frcp_rn(d2);
    a0 = d0 * r22;
    a1 = TWO ? d1 * r22 : 0.f;
#pragma unroll
    for (int i = kTK - 1; i >= 0; --i) {
        float s0 = fmaf(-a0, y2[i], y0[i]), s1 = TWO ? fmaf(-a1, y2[i], y1[i]) : 0.f;
#pragma unroll
        for (int m = i + 1; m < kTK; ++m) {
            s0 = fmaf(-L[tri(m) + i], c0[m], s0);
            if (TWO) s1 = fmaf(-L[tri(m) + i], c1[m], s1);
        }
        c0[i] = s0 * inv[i];
        c1[i] = TWO ? s1 * inv[i] : 0.f;
    }
    return spd;
}

// one block with 1 <= K <= kTK by the calling thread: positions checked,
// then c (per point) and a (per block) written.  Returns the block's
// condition bound (0 for bad positions).
template <bool TWO>
__device__ __forceinline__ float thread_run(const BlockPlane &P, const BlockGeom &g, const BlockTables &tab,
                                            const BlockScratch &S)
{
    const int K = g.K, N = g.w * g.h;
    int p[kTK];
    float v0[kTK], v1[kTK];
    bool ok = true;
    int prev = -1;
#pragma unroll
    for (int i = 0; i < kTK; ++i) {
        p[i] = 0;
        v0[i] = v1[i] = 0.f;
        if (i < K) {
            p[i] = __ldg(P.pos + g.s + i);
            v0[i] = (float)__ldg(P.val[0] + g.s + i);
            if (TWO) v1[i] = (float)__ldg(P.val[1] + g.s + i);
            ok = ok && p[i] < N && p[i] > prev;
            prev = p[i];
        }
    }
    if (!ok) {
        atomicOr(S.flags, kFlagPos);
        mark_bad(P, g.lb);
        return 0.f;
    }
    float c0[kTK], c1[kTK], a0, a1, tr;
    const bool spd =
        thread_block_coef<TWO>(green_rows(tab, g.w, g.h), g_rowlen(N), K, p, v0, v1, c0, c1, a0, a1, tr);
#pragma unroll
    for (int i = 0; i < kTK; ++i)
        if (i < K) {
            P.coef[0][g.s + i] = c0[i];
            if (TWO) P.coef[1][g.s + i] = c1[i];
        }
    P.acoef[0][g.lb] = a0;
    if (TWO) P.acoef[1][g.lb] = a1;
    if (!spd) atomicOr(S.flags, kFlagNotSPD);
    return cond_bound(tab.amax, tr, K, N);
}

// ---- CTA solves: K > 32, and FP64 re-solves of blocks above the condition
// threshold; packed Cholesky in global scratch (or shared memory) ----------
__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

template <typename T>
__device__ __forceinline__ T cta_sum(T v, T *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = 0;
    for (int k = 0; k < kCoefThreads / 32; ++k) t += red[k];
    return t;
}

__device__ __forceinline__ float rsqrt_pos(float d) { return rsqrtf(fmaxf(d, 1e-30f)); }
__device__ __forceinline__ double rsqrt_pos(double d) { return rsqrt(fmax(d, 1e-300)); }

// Coefficients of one block with valid positions s_p by the whole CTA in
// precision T: G_PP packed in L (then the three right-hand sides v0, v1, 1).
// Same steps as seg_block_coef: L y_v = v, L y_1 = 1, a = (y_1.y_v)/(y_1.y_1),
// L^T c = y_v - a y_1.  Returns false for a non-positive pivot.
template <typename T>
__device__ bool cta_solve(const BlockPlane &P, const BlockGeom &g, const unsigned char *s_p, const T *G, int rl, T *L,
                          T *red)
{
    const int tid = threadIdx.x, K = g.K;
    const bool two = P.val[1] != nullptr;
    T *b = L + pk(K, 0);  // b[r*K + i]
    for (int j = tid; j < K; j += kCoefThreads) {
        b[j] = (T)__ldg(P.val[0] + g.s + j);
        b[K + j] = two ? (T)__ldg(P.val[1] + g.s + j) : (T)0;
        b[2 * K + j] = 1;
    }
    for (int i = tid; i < K; i += kCoefThreads)
        for (int j = 0; j <= i; ++j) L[pk(i, j)] = __ldg(G + s_p[i] * rl + s_p[j]);
    __syncthreads();
    bool spd = true;
    for (int k = 0; k < K; ++k) {
        const T d = L[pk(k, k)];
        spd = spd && d > (T)0;
        const T isd = rsqrt_pos(d);
        __syncthreads();
        if (tid == 0) L[pk(k, k)] = d * isd;
        for (int i = k + 1 + tid; i < K; i += kCoefThreads) L[pk(i, k)] *= isd;
        __syncthreads();
        for (int i = k + 1 + tid; i < K; i += kCoefThreads) {
            const T lik = L[pk(i, k)];
            for (int j = k + 1; j <= i; ++j) L[pk(i, j)] = fma(-lik, L[pk(j, k)], L[pk(i, j)]);
        }
        __syncthreads();
    }
    for (int k = 0; k < K; ++k) {  // forward L y = b (three right-hand sides)
        if (tid < 3) b[tid * K + k] /= L[pk(k, k)];
        __syncthreads();
        for (int i = k + 1 + tid; i < K; i += kCoefThreads) {
            const T l = L[pk(i, k)];
            b[i] = fma(-l, b[k], b[i]);
            b[K + i] = fma(-l, b[K + k], b[K + i]);
            b[2 * K + i] = fma(-l, b[2 * K + k], b[2 * K + i]);
        }
        __syncthreads();
    }
    T s0 = 0, s1 = 0, s2 = 0;  // a = (y_1 . y_v) / (y_1 . y_1)
    for (int i = tid; i < K; i += kCoefThreads) {
        const T y2 = b[2 * K + i];
        s0 += y2 * b[i];
        s1 += y2 * b[K + i];
        s2 += y2 * y2;
    }
    s2 = cta_sum(s2, red);
    const T a0 = cta_sum(s0, red) / s2, a1 = cta_sum(s1, red) / s2;
    __syncthreads();
    for (int i = tid; i < K; i += kCoefThreads) {
        b[i] = fma(-a0, b[2 * K + i], b[i]);
        b[K + i] = fma(-a1, b[2 * K + i], b[K + i]);
    }
    __syncthreads();
    for (int k = K - 1; k >= 0; --k) {  // backward L^T c = y_v - a y_1
        if (tid < 2) b[tid * K + k] /= L[pk(k, k)];
        __syncthreads();
        for (int i = tid; i < k; i += kCoefThreads) {
            const T l = L[pk(k, i)];
            b[i] = fma(-l, b[k], b[i]);
            b[K + i] = fma(-l, b[K + k], b[K + i]);
        }
        __syncthreads();
    }
    for (int i = tid; i < K; i += kCoefThreads) {
        P.coef[0][g.s + i] = (float)b[i];
        if (two) P.coef[1][g.s + i] = (float)b[K + i];
    }
    if (tid == 0) {
        P.acoef[0][g.lb] = (float)a0;
        if (two) P.acoef[1][g.lb] = (float)a1;
    }
    return spd;
}

// One list entry by the whole CTA: a block with K > 32 (FP32 in the range's
// slot unless its condition bound exceeds the threshold) or a block already
// found above the threshold (kF64Bit), re-solved in FP64 in the slot, or in
// w64 (shared, K <= kTK) when the CTA has no slot.
__device__ __noinline__ void cta_block(const BlockJobs &J, const BlockTables &tab, const BlockScratch &S, int entry,
                                       float *slot, double *w64, unsigned char *s_p, float *redf, double *redd,
                                       int *s_bad)
{
    const int tid = threadIdx.x;
    const int gb = entry & ~kF64Bit;
    const BlockPlane &P = J.p[find_job(J, gb)];
    const BlockGeom g = block_geom(P, gb - P.block_base);
    const int K = g.K, N = g.w * g.h;
    if (tid == 0) *s_bad = 0;
    __syncthreads();
    for (int j = tid; j < K; j += kCoefThreads) {
        int p;
        if (!load_pos(P, g, j, p)) *s_bad = 1;
        s_p[j] = (unsigned char)p;
    }
    __syncthreads();
    if (*s_bad) {
        if (tid == 0) {
            atomicOr(S.flags, kFlagPos);
            mark_bad(P, g.lb);
        }
        __syncthreads();
        return;
    }
    const int off = __ldg(tab.goff + shape_index(g.w, g.h)), rl = g_rowlen(N);
    bool f64 = (entry & kF64Bit) != 0;
    if (!f64) {
        float d = 0.f;
        for (int i = tid; i < K; i += kCoefThreads) d += __ldg(tab.G + off + s_p[i] * rl + s_p[i]);
        const float kappa = cond_bound(tab.amax, cta_sum(d, redf), K, N);
        if (tid == 0) note_kappa(S, kappa);
        f64 = kappa > S.tau;
    }
    if (f64 && K > (slot ? kF64MaxK : kTK)) {
        if (tid == 0) atomicOr(S.flags, kFlagCond);
        f64 = false;
    }
    const bool spd = f64 ? cta_solve<double>(P, g, s_p, tab.G64 + off, rl, slot ? reinterpret_cast<double *>(slot) : w64,
                                             redd)
                         : cta_solve<float>(P, g, s_p, tab.G + off, rl, slot, redf);
    if (tid == 0) {
        if (!spd) atomicOr(S.flags, kFlagNotSPD);
        if (S.cstat && f64) atomicAdd(S.cstat + 1, 1u);
        if (S.cstat && K > kWarpK) atomicAdd(S.cstat + 2, 1u);
    }
    __syncthreads();
}

// Warp path: warp w of a warp-path CTA scans the 32 blocks gb0 .. gb0+31
// and solves those with kTK < K <= 32: K <= 16 two at a time in 16-lane
// halves, K <= 24 with all lanes (both in registers, fully unrolled: in a
// launch over many frames many warps of an SM share the code), larger K
// with the shared-memory routine.  Blocks with K > 32 go to the CTA's list.
__device__ __forceinline__ void warp_path(const BlockJobs &J, const BlockTables &tab, const BlockScratch &S, int gb0,
                                          int lane, float *sm, int *s_large, int *s_nlarge)
{
    const SegBlock own = seg_block(J, gb0 + lane);
    if (own.P != nullptr && !own.g.bad && own.g.K > kWarpK) s_large[atomicAdd(s_nlarge, 1)] = gb0 + lane;
    const int k = seg_k(own);
    unsigned m16 = __ballot_sync(0xffffffffu, k > kTK && k <= 16);
    unsigned m32 = __ballot_sync(0xffffffffu, k > 16);
    const int half = lane >> 4, i = lane & 15;
    while (m16) {
        const int ba = __ffs(m16) - 1;
        m16 &= m16 - 1;
        int bb = -1;
        if (m16) {
            bb = __ffs(m16) - 1;
            m16 &= m16 - 1;
        }
        const int mine = half ? bb : ba;
        const int gb = mine >= 0 ? gb0 + mine : J.total_blocks;
        SegBlock b = seg_block(J, gb);
        b.g.K = seg_k(b);
        const int K = seg_validate<16>(b, i, half, S);
        seg_run<16, 16>(b, K, i, sm + half * 16 * 17, tab, S, gb, s_large, s_nlarge);
        __syncwarp();
    }
    while (m32) {
        const int ba = __ffs(m32) - 1;
        m32 &= m32 - 1;
        SegBlock b = seg_block(J, gb0 + ba);
        b.g.K = seg_k(b);
        const int K = seg_validate<32>(b, lane, 0, S);
        if (K > 24) seg_run<32, 0>(b, K, lane, sm, tab, S, gb0 + ba, s_large, s_nlarge);
        else if (K > 0) seg_run<32, 24>(b, K, lane, sm, tab, S, gb0 + ba, s_large, s_nlarge);
        __syncwarp();
    }
}

// Coefficient stage.  The grid has two halves over the same ranges of
// kRange blocks.  Thread-path CTA nrange + c: thread t takes block
// kRange c + t and solves it when K <= 12.  Warp-path CTA c: its warps
// solve the range's blocks with 12 < K <= 32, then the whole CTA those with
// K > 32, one after the other in the range's scratch slot.  Blocks whose
// condition bound exceeds the threshold are re-solved in FP64 by their CTA
// after its first phase (thread path: in shared memory; warp path: in the
// slot).  No counters: the kernel's completion publishes every result.
__device__ __forceinline__ void coef_body(const BlockJobs &J, const BlockTables &tab, const BlockScratch &S)
{
    static_assert(kCoefThreads == kRange, "one thread per block of a range");
    __shared__ float lts[kCoefThreads / 32][32 * 33];
    __shared__ unsigned char s_p[kBigMaxK];
    __shared__ float red[kCoefThreads / 32];
    __shared__ double redd[kCoefThreads / 32];
    __shared__ double w64[tri(kTK) + 3 * kTK];
    __shared__ int s_large[kRange], s_nlarge, s_bad;
    const int nrange = block_ranges(J.total_blocks);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_nlarge = 0;
    __syncthreads();
    // the heavier warp-path CTAs come first in the grid, so that the light
    // thread-path CTAs fill the tail
    if ((int)blockIdx.x >= nrange) {
        const int gb = (blockIdx.x - nrange) * kRange + threadIdx.x;
        float kappa = 0.f;
        if (gb < J.total_blocks) {
            const BlockPlane &P = J.p[find_job(J, gb)];
            const BlockGeom g = block_geom(P, gb - P.block_base);
            if (g.bad) {
                atomicOr(S.flags, g.bad);
            } else if (g.K > 0 && g.K <= kTK) {
                kappa = P.val[1] != nullptr ? thread_run<true>(P, g, tab, S) : thread_run<false>(P, g, tab, S);
            }
        }
        if (kappa > S.tau) s_large[atomicAdd(&s_nlarge, 1)] = gb | kF64Bit;
        if (S.cstat) {
            const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(kappa));
            if (lane == 0 && m) atomicMax(S.cstat, m);
        }
        __syncthreads();
        const int n = s_nlarge;
        for (int i = 0; i < n; ++i) cta_block(J, tab, S, s_large[i], nullptr, w64, s_p, red, redd, &s_bad);
        return;
    }
    const int range = blockIdx.x;
    const int gb0 = range * kRange + warp * 32;
    if (gb0 < J.total_blocks) warp_path(J, tab, S, gb0, lane, lts[warp], s_large, &s_nlarge);
    __syncthreads();
    const int n = s_nlarge;
    if (n == 0) return;
    if (range >= S.big_ranges) {  // no scratch slot: the caller sized it wrongly
        if (threadIdx.x == 0) atomicOr(S.flags, kFlagK);
        return;
    }
    float *slot = S.big + (size_t)range * kBigFloats;
    for (int i = 0; i < n; ++i) cta_block(J, tab, S, s_large[i], slot, w64, s_p, red, redd, &s_bad);
}

// The coefficient stage reads only the caller's block data, never what the
// preceding kernel wrote, so as a programmatic dependent it runs alongside
// that kernel: the kernel after it may be scheduled at once, and the wait
// for the preceding grid comes last, so that this grid completes after it
// (every later kernel that waits for this grid sees the earlier ones done).
__global__ void __launch_bounds__(kCoefThreads, 3) block_coef_kernel(const __grid_constant__ BlockJobs J,
                                                                     BlockTables tab, BlockScratch S)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    coef_body(J, tab, S);
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- evaluation stage into residual fields, one warp per block -----------
// Lane l covers the block pixels 4l .. 4l+3 and 128 + 4l .. 128 + 4l + 3
// (index y w + x).  The points sit in the lanes, 32 at a time; c_j and p_j
// reach every lane by shuffles, and the Green's rows of several points are
// in flight (16-byte loads, each warp instruction 512 contiguous bytes)
// before their products are summed.  The constant a is loaded beside the
// block pointers.  A 16-wide block goes out as 16-byte stores (a lane's
// four pixels of rows l / 4 and 8 + l / 4);
// then the data at the points, exactly.  Bad positions give a zero block.
// QC (coefficient mode): c_j from the dead-zone indices, a transmitted, no
// overwrite at the points; K = 0 gives r = a.  An index -128 gives a zero
// block and the flag kFlagQ.
template <bool TWO, bool QC>
__device__ __forceinline__ void eval_block(const BlockPlane &P, const BlockGeom &g, const float *__restrict__ G,
                                           float a0, float a1, float *R0, float *R1, int pitch, int lane,
                                           uint32_t *flags)
{
    const int K = g.K, w = g.w, N = g.w * g.h, rl = g_rowlen(N);
    // lane l covers pixels 4l .. 4l+3 and 128 + 4l .. 128 + 4l + 3: each
    // 16-byte load instruction of the warp reads 512 contiguous bytes of a
    // Green's row (four 128-byte lines)
    const int q0 = 4 * lane, q1 = 128 + 4 * lane;
    const bool act = q0 < N, act1 = q1 < N;
    float r0[8], r1[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        r0[t] = a0;
        r1[t] = a1;
    }
    bool valid = QC || K > 0, badq = false;
    int prev = -1;
    for (int j0 = 0; j0 < K; j0 += 32) {
        const int j = j0 + lane;
        int p = 0;
        float c0 = 0.f, c1 = 0.f;
        bool qb = false;
        if (j < K) {
            p = __ldg(P.pos + g.s + j);
            if (QC) {
                const int qi = __ldg(P.q + g.s + j);
                qb = qi == -128;
                const float qf = (float)qi;
                c0 = qi == 0 ? 0.f : copysignf((fabsf(qf) + P.qoff) * P.qstep, qf);
            } else {
                c0 = __ldg(P.coef[0] + g.s + j);
                if (TWO) c1 = __ldg(P.coef[1] + g.s + j);
            }
        }
        // inside the block and increasing (the previous chunk's last point
        // for lane 0)
        const int up = __shfl_up_sync(0xffffffffu, p, 1);  // every lane takes part
        const int before = lane == 0 ? prev : up;
        if (__any_sync(0xffffffffu, j < K && (p >= N || p <= before))) valid = false;
        if (QC && __any_sync(0xffffffffu, qb)) {
            valid = false;
            badq = true;
        }
        prev = __shfl_sync(0xffffffffu, p, 31);
        if (!valid) break;
        const int n = min(32, K - j0);
        const float *Gq = G + q0;  // + 128 for the second half
#pragma unroll 4
        for (int u = 0; u < n; ++u) {
            const float cu0 = __shfl_sync(0xffffffffu, c0, u);
            const float cu1 = TWO ? __shfl_sync(0xffffffffu, c1, u) : 0.f;
            const int pu = __shfl_sync(0xffffffffu, p, u);
            if (act) {
                const float *row = Gq + pu * rl;
                const float4 lo = __ldg(reinterpret_cast<const float4 *>(row));
                const float4 hi = act1 ? __ldg(reinterpret_cast<const float4 *>(row + 128)) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float gv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    r0[t] = fmaf(cu0, gv[t], r0[t]);
                    if (TWO) r1[t] = fmaf(cu1, gv[t], r1[t]);
                }
            }
        }
    }
    if (!valid) {
        if (K > 0 && lane == 0 && flags) atomicOr(flags, badq ? kFlagQ : kFlagPos);
#pragma unroll
        for (int t = 0; t < 8; ++t) r0[t] = r1[t] = 0.f;
    }
    // 16-byte stores need 16-byte aligned rows (callers may pass any pitch)
    const bool vec = w == 16 && ((reinterpret_cast<uintptr_t>(R0) | reinterpret_cast<uintptr_t>(R1) |
                                  (uintptr_t)pitch * 4) & 15) == 0;
    if (act) {
        if (vec) {
            // pixels 4l .. 4l+3 are columns 4 (l % 4) .. +3 of row l / 4,
            // the second half the same columns of row 8 + l / 4
            const size_t o = (size_t)(lane >> 2) * pitch + 4 * (lane & 3), o1 = o + (size_t)8 * pitch;
            reinterpret_cast<float4 *>(R0 + o)[0] = make_float4(r0[0], r0[1], r0[2], r0[3]);
            if (act1) reinterpret_cast<float4 *>(R0 + o1)[0] = make_float4(r0[4], r0[5], r0[6], r0[7]);
            if (TWO && R1) {
                reinterpret_cast<float4 *>(R1 + o)[0] = make_float4(r1[0], r1[1], r1[2], r1[3]);
                if (act1) reinterpret_cast<float4 *>(R1 + o1)[0] = make_float4(r1[4], r1[5], r1[6], r1[7]);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int q = (t < 4 ? q0 : q1 - 4) + t;
                if (q < N) {
                    const int y = q / w, x = q - y * w;
                    R0[(size_t)y * pitch + x] = r0[t];
                    if (TWO && R1) R1[(size_t)y * pitch + x] = r1[t];
                }
            }
        }
    }
    if (QC || !valid) return;
    __syncwarp();
    // the data at the points, exactly
    const float rw = __frcp_rn((float)w);
    for (int j = lane; j < K; j += 32) {
        const int p = __ldg(P.pos + g.s + j);
        const int y = __float2int_rz(((float)p + 0.5f) * rw), x = p - y * w;  // p / w, exact for p < 256
        R0[(size_t)y * pitch + x] = (float)__ldg(P.val[0] + g.s + j);
        if (TWO && R1) R1[(size_t)y * pitch + x] = (float)__ldg(P.val[1] + g.s + j);
    }
}

template <bool QC>
__global__ void __launch_bounds__(128, 8) block_eval_kernel(const __grid_constant__ BlockJobs J, BlockTables tab,
                                                            uint32_t *flags)
{
    // the coefficients come from the preceding grid
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * 4 + warp;
    if (gb >= J.total_blocks) return;
    const BlockPlane &P = J.p[find_job(J, gb)];
    const int lb = gb - P.block_base;
    const bool two = P.val[1] != nullptr;
    // a depends on the block index only: its load goes out with the pointers
    const float a0 = __ldg(P.acoef[0] + lb), a1 = two ? __ldg(P.acoef[1] + lb) : 0.f;
    const BlockGeom g = block_geom(P, lb);
    const int pitch = P.r_pitch;
    float *R0 = P.r[0] + (size_t)g.y0 * pitch + g.x0;
    float *R1 = two && P.r[1] ? P.r[1] + (size_t)g.y0 * pitch + g.x0 : nullptr;
    const float *G = green_rows(tab, g.w, g.h);
    if (QC) {
        // no coefficient stage ran: block pointer errors are reported here
        // (the block reconstructs as zero)
        if (g.bad && lane == 0 && flags) atomicOr(flags, g.bad);
        eval_block<false, true>(P, g, G, g.bad ? 0.f : a0, 0.f, R0, nullptr, pitch, lane, flags);
    } else if (two) eval_block<true, false>(P, g, G, a0, a1, R0, R1, pitch, lane, flags);
    else eval_block<false, false>(P, g, G, a0, a1, R0, R1, pitch, lane, flags);
}

}  // namespace

cudaError_t ensure_block_tables()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if ((g_tab_devices >> dev) & 1ull) return cudaSuccess;
    static std::vector<float> G[kNumOps];
    static std::vector<double> G64[kNumOps];
    static std::vector<int> goff;
    float *dG = nullptr;
    double *dG64 = nullptr;
    const int *dgoff = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&dG, d_G)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&dG64, d_G64)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&dgoff, d_goff)) != cudaSuccess) return e;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    for (int op = 0; op < kNumOps; ++op) {
        if (G[op].empty()) build_tables(op, G[op], G64[op], goff);
        if ((e = cudaMemcpy(dG + (size_t)op * kGSize, G[op].data(), G[op].size() * sizeof(float),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(dG64 + (size_t)op * kGSize, G64[op].data(), G64[op].size() * sizeof(double),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        BlockTables &t = g_tabs[dev][op];
        t.G = dG + (size_t)op * kGSize;
        t.G64 = dG64 + (size_t)op * kGSize;
        t.goff = dgoff;
        t.sms = sms;
        t.amax = op == 1 ? 64.f : 8.f;
    }
    if ((e = cudaMemcpyToSymbol(d_goff, goff.data(), goff.size() * sizeof(int))) != cudaSuccess) return e;
    if ((e = intra_init()) != cudaSuccess) return e;
    g_tab_devices |= 1ull << dev;
    return cudaSuccess;
}

const BlockTables &block_tables(int op)
{
    int dev = 0;
    cudaGetDevice(&dev);
    return g_tabs[dev < 64 ? dev : 0][op == 1 ? 1 : 0];
}

namespace {

struct PdlConfig {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    PdlConfig(dim3 grid, dim3 block, cudaStream_t st, bool pdl)
    {
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = pdl ? 1 : 0;
    }
};

}  // namespace

cudaError_t launch_block_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st, int *launches, bool pdl)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    PdlConfig c(dim3(2 * block_ranges(jobs.total_blocks)), dim3(kCoefThreads), st, pdl);
    const cudaError_t e = cudaLaunchKernelEx(&c.cfg, block_coef_kernel, jobs, block_tables(jobs.op), s);
    if (launches) *launches += 1;
    return e;
}

cudaError_t launch_block_eval(const BlockJobs &jobs, uint32_t *flags, cudaStream_t st, bool pdl)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    PdlConfig c(dim3((jobs.total_blocks + 3) / 4), dim3(128), st, pdl);
    if (jobs.p[0].q) return cudaLaunchKernelEx(&c.cfg, block_eval_kernel<true>, jobs, block_tables(jobs.op), flags);
    return cudaLaunchKernelEx(&c.cfg, block_eval_kernel<false>, jobs, block_tables(jobs.op), flags);
}

}  // namespace hivc
