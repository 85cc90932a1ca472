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
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>

#include "block_device.cuh"

namespace hivc {
namespace {

constexpr int kGSize = 2283904;  // sum over shapes of N * rowlen(N)

// one table per operator (0 harmonic, 1 biharmonic)
static __device__ __align__(256) float d_G[kNumOps * kGSize];
static __device__ __align__(256) double d_G64[kNumOps * kGSize];
static __device__ int d_goff[256];
static __device__ __align__(256) float d_G16o[kNumOps * kSym16Floats];

std::mutex g_tab_mu;
BlockTables g_tabs[64][kNumOps];
uint64_t g_tab_devices = 0;  // bit d: tables uploaded to device d

void symmetrise16(std::vector<float> &G, std::vector<double> &G64, int off);

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
    symmetrise16(G, G64, goff[shape_index(16, 16)]);
}

// The 16 x 16 rows agree with the symmetries of the square only up to
// rounding (the sums above run in different orders for a pair and its
// images).  Each entry takes the value of one fixed member of its orbit
// under those symmetries and under (p, q) -> (q, p), so that the table is
// exactly symmetric and exactly invariant, and the 36 rows of the compact
// table give back every row bit for bit.
void symmetrise16(std::vector<float> &G, std::vector<double> &G64, int off)
{
    const std::vector<double> g0(G64.begin() + off, G64.begin() + off + 256 * 256);
    for (int p = 0; p < 256; ++p)
        for (int q = 0; q < 256; ++q) {
            int best = 1 << 30;
            for (int k = 0; k < 8; ++k) {
                const Sym16 s{0, k & 1, (k >> 1) & 1, k >> 2};
                const int a = sym16_apply(s, p), b = sym16_apply(s, q);
                best = std::min(best, std::min(a * 256 + b, b * 256 + a));
            }
            G64[off + p * 256 + q] = g0[best];
            G[off + p * 256 + q] = (float)g0[best];
        }
}

// The compact 16 x 16 table: for each of the 36 points b = (bx, by),
// bx <= by <= 7, and each orientation o = rx + 2 tr, the row of b read in
// the order that a point mapped to b by (rx, ry = 0, tr) needs.
void build_sym16(const std::vector<float> &G, int off, std::vector<float> &S)
{
    S.assign(kSym16Floats, 0.f);
    for (int by = 0; by < 8; ++by)
        for (int bx = 0; bx <= by; ++bx) {
            const int bi = by * (by + 1) / 2 + bx, b = by * 16 + bx;
            for (int o = 0; o < 4; ++o)
                for (int y = 0; y < 16; ++y)
                    for (int x = 0; x < 16; ++x) {
                        const Sym16 s{bi, o & 1, 0, o >> 1};
                        S[((size_t)(o * kSym16Rows + bi) * 16 + y) * 16 + x] = G[off + b * 256 + sym16_apply(s, y * 16 + x)];
                    }
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

// Coefficients of one block by one thread, K <= KM (KM = 8 or kTK = 12):
// G_PP padded to KM x KM with the identity (the padding rows of L are unit rows and the
// padding entries of every solution are zero), Cholesky-Crout in
// registers, fully unrolled, so that no control flow depends on K.
//   L y_v = v, L y_1 = 1 (on the K points);  a = (y_1 . y_v) / (y_1 . y_1)
//   L^T c = y_v - a y_1
// Returns false if a pivot of a real row was not positive; tr = tr(G_PP).
// The padding leaves every real entry's arithmetic as it is (padding
// entries of L, y and c are exact zeros that enter sums as +0), so KM = 8
// and KM = 12 give the same bits for K <= 8.
template <int KM, bool TWO>
__device__ __forceinline__ bool thread_block_coef(const float *__restrict__ G, int rl, int K, const int (&p)[KM],
                                                  const float (&v0)[KM], const float (&v1)[KM], float (&c0)[KM],
                                                  float (&c1)[KM], float &a0, float &a1, float &tr)
{
    float L[tri(KM)], inv[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        const float *row = G + p[i] * rl;
#pragma unroll
        for (int j = 0; j <= i; ++j) L[tri(i) + j] = (i < K && j < K) ? __ldg(row + p[j]) : (i == j ? 1.f : 0.f);
    }
    tr = 0.f;
#pragma unroll
    for (int i = 0; i < KM; ++i)
        if (i < K) tr += L[tri(i) + i];
    bool spd = true;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        float d = L[tri(k) + k];
#pragma unroll
        for (int m = 0; m < k; ++m) d = fmaf(-L[tri(k) + m], L[tri(k) + m], d);
        spd = spd && (k >= K || d > 0.f);
        const float isd = rsqrtf(fmaxf(d, 1e-30f));
        L[tri(k) + k] = d * isd;
        inv[k] = isd;
#pragma unroll
        for (int i = k + 1; i < KM; ++i) {
            float s = L[tri(i) + k];
#pragma unroll
            for (int m = 0; m < k; ++m) s = fmaf(-L[tri(i) + m], L[tri(k) + m], s);
            L[tri(i) + k] = s * isd;
        }
    }
    float y0[KM], y1[KM], y2[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i) {
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
    for (int i = 0; i < KM; ++i) {
        d0 = fmaf(y2[i], y0[i], d0);
        if (TWO) d1 = fmaf(y2[i], y1[i], d1);
        d2 = fmaf(y2[i], y2[i], d2);
    }
    const float r22 = __frcp_rn(d2);
    a0 = d0 * r22;
    a1 = TWO ? d1 * r22 : 0.f;
#pragma unroll
    for (int i = KM - 1; i >= 0; --i) {
        float s0 = fmaf(-a0, y2[i], y0[i]), s1 = TWO ? fmaf(-a1, y2[i], y1[i]) : 0.f;
#pragma unroll
        for (int m = i + 1; m < KM; ++m) {
            s0 = fmaf(-L[tri(m) + i], c0[m], s0);
            if (TWO) s1 = fmaf(-L[tri(m) + i], c1[m], s1);
        }
        c0[i] = s0 * inv[i];
        c1[i] = TWO ? s1 * inv[i] : 0.f;
    }
    return spd;
}

// one block with 1 <= K <= KM by the calling thread: positions checked,
// then c (per point) and a (per block) written.  Returns the block's
// condition bound (0 for bad positions).
template <int KM, bool TWO>
__device__ __forceinline__ float thread_run(const BlockPlane &P, const BlockGeom &g, const BlockTables &tab,
                                            const BlockScratch &S)
{
    const int K = g.K, N = g.w * g.h;
    int p[KM];
    float v0[KM], v1[KM];
    bool ok = true;
    int prev = -1;
#pragma unroll
    for (int i = 0; i < KM; ++i) {
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
    float c0[KM], c1[KM], a0, a1, tr;
    const bool spd =
        thread_block_coef<KM, TWO>(green_rows(tab, g.w, g.h), g_rowlen(N), K, p, v0, v1, c0, c1, a0, a1, tr);
#pragma unroll
    for (int i = 0; i < KM; ++i)
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

// ---- plan of a coefficient launch ------------------------------------------
// class of a block with K >= 1 points, in queue order (heavy first):
// K > 32, 25..32, 17..24, 13..16, 9..12, 1..8
__device__ __forceinline__ int k_class(int K)
{
    return K > 32 ? 0 : (K > 24 ? 1 : (K > 16 ? 2 : (K > 12 ? 3 : (K > 8 ? 4 : 5))));
}
// blocks per work item of each class: a CTA, a warp each, two per warp,
// a thread each
__host__ __device__ __forceinline__ int class_item(int c)
{
    return c == 0 ? 1 : (c <= 2 ? kCoefThreads / 32 : (c == 3 ? 2 * kCoefThreads / 32 : kCoefThreads));
}

// FNV-1a over 32-bit words: the fingerprint of a layout
__device__ __forceinline__ unsigned long long fnv(unsigned long long h, uint32_t v)
{
    return (h ^ v) * 0x100000001b3ull;
}

// Layout table (layout groups on): a block with 1 <= K <= kGroupMaxK and
// valid positions enters its layout (job, w, h, K, positions) into the
// table and counts it; the block that makes a layout's count kGroupMin
// claims a group for it, unless the layout's condition bound is above the
// threshold (those blocks stay on the FP64-aware path).  Returns the slot,
// or -1 (not a candidate, or the table crowded).
__device__ __forceinline__ int enter_layout(const BlockPlan &L, const BlockTables &tab, float tau, int k,
                                            const BlockPlane &P, const BlockGeom &g, int gb)
{
    if (g.bad || g.K < 1 || g.K > kGroupMaxK) return -1;
    const int K = g.K, N = g.w * g.h;
    unsigned long long h = 0xcbf29ce484222325ull;
    h = fnv(h, (uint32_t)k);
    h = fnv(h, (uint32_t)(g.w | (g.h << 8) | (K << 16)));
    int prev = -1;
    for (int j = 0; j < K; ++j) {
        const int p = __ldg(P.pos + g.s + j);
        if (p >= N || p <= prev) return -1;  // the coefficient stage reports it
        prev = p;
        h = fnv(h, (uint32_t)p);
    }
    if (h == 0) h = 1;
    uint32_t slot = (uint32_t)(h ^ (h >> 32)) & L.hmask;
    int probe = 0;
    for (; probe < kHashProbes; ++probe) {
        const unsigned long long old = atomicCAS(L.hkey + slot, 0ull, h);
        if (old == 0ull || old == h) break;
        slot = (slot + 1) & L.hmask;
    }
    if (probe == kHashProbes) return -1;
    const uint32_t c = atomicAdd(L.hcnt + slot, 1u) + 1u;
    if (c == (uint32_t)kGroupMin) {
        const float *G = green_rows(tab, g.w, g.h);
        const int rl = g_rowlen(N);
        float tr = 0.f;
        for (int j = 0; j < K; ++j) {
            const int p = __ldg(P.pos + g.s + j);
            tr += __ldg(G + p * rl + p);
        }
        if (cond_bound(tab.amax, tr, K, N) <= tau) {
            const uint32_t gid = atomicAdd(&L.st->ngroups, 1u);
            if (gid < (uint32_t)kMaxGroups) {
                L.st->gslot[gid] = (int)slot;
                L.st->grep[gid] = gb;
                L.hgid[slot] = gid + 1;
            }
        }
    }
    return (int)slot;
}

// Exclusive prefix of f(0), ..., f(n-1) into s_out[0..n] (s_out[n] = the
// total): a block-wide scan, a chunk of blockDim entries at a time (any
// block size that is a multiple of 32).  Every CTA computes the same.
template <class F>
__device__ __forceinline__ void block_prefix(int n, F f, int *s_out)
{
    __shared__ int s_warp[32], s_carry;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + t;
        const int own = i < n ? f(i) : 0;
        int v = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += x;
        }
        if (lane == 31) s_warp[w] = v;
        __syncthreads();
        int before = s_carry;
        for (int k = 0; k < w; ++k) before += s_warp[k];
        if (i < n) s_out[i] = before + v - own;
        __syncthreads();
        if (t == blockDim.x - 1) s_carry = before + v;
        __syncthreads();
    }
    if (t == 0) s_out[n] = s_carry;
    __syncthreads();
}

// member-entry offset of each group into s_off (entries are reserved at two
// per block of the group's slot count: the plane pair of a shared chroma
// layout takes two); returns the number of groups
__device__ __forceinline__ int group_offsets(const BlockPlan &L, int *s_off)
{
    const int ng = min((int)*(volatile uint32_t *)&L.st->ngroups, kMaxGroups);
    block_prefix(ng, [&](int g) { return 2 * (int)__ldg(L.hcnt + L.st->gslot[g]); }, s_off);
    return ng;
}

// Whether block gb (job k, geometry g) belongs to its layout's group: the
// same job, shape, K and positions as the group's block, and values that
// the product takes exactly.  Members are listed (one entry per value
// plane) and marked; their coefficients are never formed.
__device__ __forceinline__ bool group_member(const BlockJobs &J, const BlockPlan &L, int k, const BlockGeom &g,
                                             int gb, const int *s_off)
{
    const int slot = L.slot_of[gb];
    if (slot < 0) return false;
    const int gid = (int)L.hgid[slot] - 1;
    if (gid < 0) return false;
    const int rep = L.st->grep[gid];
    if (find_job(J, rep) != k) return false;
    const BlockPlane &P = J.p[k];
    const BlockGeom gr = block_geom(P, rep - P.block_base);
    if (gr.w != g.w || gr.h != g.h || gr.K != g.K) return false;
    const bool two = P.val[1] != nullptr;
    for (int j = 0; j < g.K; ++j) {
        if (__ldg(P.pos + g.s + j) != __ldg(P.pos + gr.s + j)) return false;
        // the product takes the values as bf16: integers up to 256 are exact
        if (abs((int)__ldg(P.val[0] + g.s + j)) > 256) return false;
        if (two && abs((int)__ldg(P.val[1] + g.s + j)) > 256) return false;
    }
    const uint32_t idx = atomicAdd(L.st->gfill + gid, two ? 2u : 1u);
    int32_t *e = L.gmem + s_off[gid] + idx;
    e[0] = 2 * gb;
    if (two) e[1] = 2 * gb + 1;
    L.member[gb] = 1;
    return true;
}

// The plan: every block's class, appended to the class lists by
// warp-aggregated atomics, and (layout groups on) its layout entered into
// the table.  Bad block pointers are reported here.
__global__ void __launch_bounds__(256) block_plan_kernel(const __grid_constant__ BlockJobs J, BlockPlan L,
                                                         BlockTables tab, float tau, uint32_t *flags)
{
    // the lists may still be read by the previous coefficient launch
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int gb = blockIdx.x * 256 + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int cls = -1;
    if (gb < J.total_blocks) {
        const int k = find_job(J, gb);
        const BlockPlane &P = J.p[k];
        const BlockGeom g = block_geom(P, gb - P.block_base);
        if (g.bad) atomicOr(flags, g.bad);
        else if (g.K > 0) cls = k_class(g.K);
        if (L.hkey) {
            L.slot_of[gb] = enter_layout(L, tab, tau, k, P, g, gb);
            L.member[gb] = 0;  // the coefficient kernel decides
        }
    }
#pragma unroll
    for (int c = 0; c < kClasses; ++c) {
        const unsigned m = __ballot_sync(0xffffffffu, cls == c);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(L.st->count + c, (uint32_t)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (cls == c) L.list[(size_t)c * L.cap + base + __popc(m & ((1u << lane) - 1u))] = gb;
    }
}

// ---- factorisation of a layout group -------------------------------------
// For a fixed layout P the residual is linear in the values v (Eqs. 2-3):
// with z = G_PP^-1 1, s = 1^T z and W = G_PP^-1 - z z^T / s (symmetric),
//   a = z^T v / s,  c = W v,  r(x) = G[x, P] c + a = E[x, :] v,
//   E[x, :] = G[x, P] W + z^T / s.
// G_PP^-1 comes from Gauss-Jordan elimination on [G_PP | I] (G_PP is SPD,
// so no pivoting), K steps with the whole CTA; then every pixel's row of E
// is an independent K x K product (no dependent chains).  The rows of E at
// the points are the unit rows, which makes r exact there, as the
// per-block path's overwrite does.  E is stored as three bf16 parts (hi,
// mid, lo: 24 significant bits together) for the tensor-core product, in
// row-major pairs of columns, kGroupMaxK columns per row (zero beyond K)
// and kGroupRows rows (zero beyond the block's pixels).  A group takes two
// work items: rows 0..127 and 128..255.
constexpr int kFactorItems = 2;
static_assert(kFactorItems * kCoefThreads == kGroupRows, "a row of E per thread");

template <int KP>
__device__ __forceinline__ void group_row(const float *__restrict__ G, int rl, int K, int x, const unsigned char *s_p,
                                          const float (*A)[2 * kGroupMaxK + 1], const float *zs, float (&e)[kGroupMaxK])
{
    float acc[KP];
#pragma unroll
    for (int k = 0; k < KP; ++k) acc[k] = k < K ? zs[k] : 0.f;
    const float *row = G + x * rl;
    for (int j = 0; j < K; ++j) {
        const float g = __ldg(row + s_p[j]);
#pragma unroll
        for (int k = 0; k < KP; ++k) acc[k] = fmaf(g, A[j][kGroupMaxK + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < kGroupMaxK; ++k) e[k] = (k < KP && k < K) ? acc[k < KP ? k : 0] : 0.f;
}

__device__ __noinline__ void group_factor(const BlockJobs &J, const BlockPlan &L, const BlockTables &tab, int gid,
                                          int part, float (*A)[2 * kGroupMaxK + 1], float *wv, unsigned char *s_p)
{
    const int tid = threadIdx.x;
    const int rep = L.st->grep[gid];
    const BlockPlane &P = J.p[find_job(J, rep)];
    const BlockGeom g = block_geom(P, rep - P.block_base);
    const int K = g.K, N = g.w * g.h, rl = g_rowlen(N);
    const float *G = green_rows(tab, g.w, g.h);
    for (int j = tid; j < K; j += kCoefThreads) s_p[j] = __ldg(P.pos + g.s + j);
    __syncthreads();
    // [G_PP | I]: columns 0..K-1 and kGroupMaxK .. kGroupMaxK + K - 1
    for (int q = tid; q < K * K; q += kCoefThreads) {
        const int i = q / K, j = q - i * K;
        A[i][j] = __ldg(G + s_p[i] * rl + s_p[j]);
        A[i][kGroupMaxK + j] = i == j ? 1.f : 0.f;
    }
    __syncthreads();
    float *f = wv + 64;  // column k before its elimination
    for (int k = 0; k < K; ++k) {
        const float rp = 1.f / A[k][k];
        for (int i = tid; i < K; i += kCoefThreads) f[i] = A[i][k];
        __syncthreads();
        for (int j = tid; j < 2 * kGroupMaxK; j += kCoefThreads) A[k][j] *= rp;
        __syncthreads();
        for (int q = tid; q < K * 2 * kGroupMaxK; q += kCoefThreads) {
            const int i = q / (2 * kGroupMaxK), j = q - i * (2 * kGroupMaxK);
            if (i != k) A[i][j] = fmaf(-f[i], A[k][j], A[i][j]);
        }
        __syncthreads();
    }
    // z = G_PP^-1 1, zs = z / s, W = G_PP^-1 - z z^T / s (in place)
    if (tid < K) {
        float z = 0.f;
        for (int j = 0; j < K; ++j) z += A[tid][kGroupMaxK + j];
        wv[tid] = z;
    }
    __syncthreads();
    if (tid == 0) {
        float sum = 0.f;
        for (int j = 0; j < K; ++j) sum += wv[j];
        wv[96] = 1.f / sum;
    }
    __syncthreads();
    const float rs = wv[96];
    for (int q = tid; q < K * K; q += kCoefThreads) {
        const int i = q / K, j = q - i * K;
        A[i][kGroupMaxK + j] = fmaf(-wv[i] * rs, wv[j], A[i][kGroupMaxK + j]);
    }
    if (tid < K) wv[32 + tid] = wv[tid] * rs;
    __syncthreads();
    uint32_t *E = reinterpret_cast<uint32_t *>(L.E + (size_t)gid * 3 * kGroupRows * kGroupMaxK);
    constexpr int kPairs = kGroupMaxK / 2;
    const int x = part * kCoefThreads + tid;  // one row of E per thread
    float e[kGroupMaxK];
#pragma unroll
    for (int k = 0; k < kGroupMaxK; ++k) e[k] = 0.f;
    int jp = -1;
    for (int j = 0; j < K; ++j)
        if (s_p[j] == x) jp = j;
    if (x < N && jp >= 0) {
#pragma unroll
        for (int k = 0; k < kGroupMaxK; ++k) e[k] = k == jp ? 1.f : 0.f;
    } else if (x < N) {
        if (K <= 16) group_row<16>(G, rl, K, x, s_p, A, wv + 32, e);
        else group_row<32>(G, rl, K, x, s_p, A, wv + 32, e);
    }
#pragma unroll
    for (int q = 0; q < kPairs; ++q) {
        uint32_t w[3];
        float v0 = e[2 * q], v1 = e[2 * q + 1];
#pragma unroll
        for (int pt = 0; pt < 3; ++pt) {
            const __nv_bfloat16 b0 = __float2bfloat16_rn(v0), b1 = __float2bfloat16_rn(v1);
            w[pt] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
            v0 -= __bfloat162float(b0);  // exact: the next part carries the remainder
            v1 -= __bfloat162float(b1);
        }
#pragma unroll
        for (int pt = 0; pt < 3; ++pt) E[((size_t)pt * kGroupRows + x) * kPairs + q] = w[pt];
    }
    __syncthreads();
}

// ---- the persistent coefficient kernel ------------------------------------
// Work items, taken from one queue (an atomic counter) by every CTA: first
// the layout groups' factorisations (a CTA each), then the class lists in
// queue order: K > 32 a block per CTA, K in 17..32 a block per warp, K in
// 13..16 two per warp (16-lane halves), K <= 12 a block per thread (the
// system padded to 12 x 12, or 8 x 8 for K <= 8).  Blocks with K > 32 need
// a scratch slot: they sit on a queue of their own that only the first
// S.big_ranges CTAs (the ones with a slot) take, before the main queue.
// Blocks above the condition threshold are re-solved in FP64 by their CTA
// after the item (K <= 12 in shared memory, larger in the slot); a CTA
// without a slot defers a larger one to a list that the last CTA to finish
// drains with slot 0 (the kernel's completion count; no CTA waits).
// a member of a layout group (groups on): listed for the group's product,
// counted, and left without coefficients
__device__ __forceinline__ bool take_member(const BlockJobs &J, const BlockScratch &S, int k, const BlockGeom &g,
                                            int gb, const int *s_off)
{
    if (!S.plan.hkey || !group_member(J, S.plan, k, g, gb, s_off)) return false;
    if (S.cstat) atomicAdd(S.cstat + 3, J.p[k].val[1] != nullptr ? 2u : 1u);
    return true;
}

__device__ __forceinline__ void thread_item(const BlockJobs &J, const BlockTables &tab, const BlockScratch &S,
                                            int c, const int32_t *lst, int n, int *s_large, int *s_nlarge,
                                            const int *s_off)
{
    const int t = threadIdx.x;
    float kappa = 0.f;
    int gb = -1;
    if (t < n) {
        gb = lst[t];
        const int k = find_job(J, gb);
        const BlockPlane &P = J.p[k];
        const BlockGeom g = block_geom(P, gb - P.block_base);
        const bool two = P.val[1] != nullptr;
        if (take_member(J, S, k, g, gb, s_off)) {
        } else if (c == 4) {
            kappa = two ? thread_run<kTK, true>(P, g, tab, S) : thread_run<kTK, false>(P, g, tab, S);
        } else {
            kappa = two ? thread_run<8, true>(P, g, tab, S) : thread_run<8, false>(P, g, tab, S);
        }
    }
    if (kappa > S.tau) s_large[atomicAdd(s_nlarge, 1)] = gb | kF64Bit;
    if (S.cstat) {
        const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(kappa));
        if ((t & 31) == 0 && m) atomicMax(S.cstat, m);
    }
}

__device__ __forceinline__ void warp_item(const BlockJobs &J, const BlockTables &tab, const BlockScratch &S, int c,
                                          const int32_t *lst, int n, float *sm, int *s_large, int *s_nlarge,
                                          const int *s_off)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // a member of a layout group: the segment's first lane lists it, the
    // segment solves nothing
    auto member = [&](int gb, int seg_lane0) {
        int mem = 0;
        if (lane == seg_lane0 && gb < J.total_blocks) {
            const int k = find_job(J, gb);
            mem = take_member(J, S, k, block_geom(J.p[k], gb - J.p[k].block_base), gb, s_off) ? 1 : 0;
        }
        return __shfl_sync(0xffffffffu, mem, seg_lane0) != 0;
    };
    if (c == 3) {  // 13..16: two blocks per warp in 16-lane halves
        const int half = lane >> 4, i = lane & 15, idx = 2 * warp + half;
        const int gb = idx < n ? lst[idx] : J.total_blocks;
        const bool m0 = S.plan.hkey ? member(gb, 0) : false;  // every lane takes part in both
        const bool m1 = S.plan.hkey ? member(gb, 16) : false;
        SegBlock b = seg_block(J, gb);
        b.g.K = (half ? m1 : m0) ? 0 : seg_k(b);
        const int K = seg_validate<16>(b, i, half, S);
        seg_run<16, 16>(b, K, i, sm + half * 16 * 17, tab, S, gb, s_large, s_nlarge);
        __syncwarp();
        return;
    }
    if (warp >= n) return;  // the whole warp
    const int gb = lst[warp];
    if (S.plan.hkey && member(gb, 0)) return;
    SegBlock b = seg_block(J, gb);
    b.g.K = seg_k(b);
    const int K = seg_validate<32>(b, lane, 0, S);
    if (K > 24) seg_run<32, 0>(b, K, lane, sm, tab, S, gb, s_large, s_nlarge);
    else if (K > 0) seg_run<32, 24>(b, K, lane, sm, tab, S, gb, s_large, s_nlarge);
    __syncwarp();
}

__global__ void __launch_bounds__(kCoefThreads, 3) block_coef_kernel(const __grid_constant__ BlockJobs J,
                                                                     BlockTables tab, BlockScratch S)
{
    // the plan's lists come from the preceding grid
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    static_assert(kCoefThreads == kRange, "one thread per block of a thread item");
    __shared__ float lts[kCoefThreads / 32][32 * 33];
    __shared__ unsigned char s_p[kBigMaxK];
    __shared__ float red[kCoefThreads / 32];
    __shared__ double redd[kCoefThreads / 32];
    __shared__ double w64[tri(kTK) + 3 * kTK];
    __shared__ int s_large[kRange], s_nlarge, s_bad, s_item, s_last;
    __shared__ int s_ofs[kClasses + 1], s_cnt[kClasses];
    __shared__ int s_off[kMaxGroups + 1];  // member-entry offsets of the layout groups
    const BlockPlan &L = S.plan;
    const int tid = threadIdx.x;
    if (L.hkey) {
        const int ng = group_offsets(L, s_off);
        if (S.cstat && blockIdx.x == 0 && tid == 0) atomicAdd(S.cstat + 4, (uint32_t)ng);
    }
    const bool has_slot = (int)blockIdx.x < S.big_ranges;
    float *slot = has_slot ? S.big + (size_t)blockIdx.x * kBigFloats : nullptr;
    if (tid == 0) {
        s_nlarge = 0;
        // items of the main queue: groups, then classes 1..5
        s_ofs[0] = L.hkey ? kFactorItems * min((int)L.st->ngroups, kMaxGroups) : 0;
        for (int c = 0; c < kClasses; ++c) s_cnt[c] = (int)L.st->count[c];
        for (int c = 1; c < kClasses; ++c) s_ofs[c] = s_ofs[c - 1] + (s_cnt[c] + class_item(c) - 1) / class_item(c);
        s_ofs[kClasses] = s_ofs[kClasses - 1];
    }
    __syncthreads();
    // K > 32: CTAs with a slot only
    if (has_slot) {
        for (;;) {
            if (tid == 0) s_item = (int)atomicAdd(&L.st->next0, 1u);
            __syncthreads();
            const int item = s_item;
            __syncthreads();
            if (item >= s_cnt[0]) break;
            cta_block(J, tab, S, L.list[item], slot, w64, s_p, red, redd, &s_bad);
        }
    }
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(&L.st->next, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= s_ofs[kClasses - 1]) break;
        if (item < s_ofs[0]) {
            group_factor(J, L, tab, item / kFactorItems, item % kFactorItems,
                         reinterpret_cast<float(*)[2 * kGroupMaxK + 1]>(lts[0]), lts[2], s_p);
            continue;
        }
        int c = 1;
        while (item >= s_ofs[c]) ++c;
        const int first = (item - s_ofs[c - 1]) * class_item(c);
        const int n = min(class_item(c), s_cnt[c] - first);
        const int32_t *lst = L.list + (size_t)c * L.cap + first;
        if (c >= 4) thread_item(J, tab, S, c, lst, n, s_large, &s_nlarge, s_off);
        else warp_item(J, tab, S, c, lst, n, lts[tid >> 5], s_large, &s_nlarge, s_off);
        __syncthreads();
        const int nl = s_nlarge;
        for (int i = 0; i < nl; ++i) {
            const int entry = s_large[i];
            const int gbl = entry & ~kF64Bit;
            const BlockPlane &P = J.p[find_job(J, gbl)];
            const int K = block_geom(P, gbl - P.block_base).K;
            if (slot || K <= kTK) {
                cta_block(J, tab, S, entry, slot, w64, s_p, red, redd, &s_bad);
            } else if (tid == 0) {
                L.deferred[atomicAdd(&L.st->ndef, 1u)] = entry;
            }
        }
        __syncthreads();
        if (tid == 0) s_nlarge = 0;
        __syncthreads();
    }
    // the last CTA to finish re-solves the deferred blocks in slot 0
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&L.st->finished, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int nd = (int)*(volatile uint32_t *)&L.st->ndef;
    for (int i = 0; i < nd; ++i)
        cta_block(J, tab, S, *(volatile int32_t *)(L.deferred + i), S.big, w64, s_p, red, redd, &s_bad);
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
// A 16 x 16 block reads its rows from the compact table S (36 points in 4
// orientations, 147 KB, which stays in L1): the lane owning point p sends
// the offset of p's row in S and whether the row's y order is reversed
// (bit 16) in place of p; rows 0..7 of a point's row are then rows 15..8 of
// the stored one, in the same 512-byte span.  Other shapes send p * rl.
template <bool TWO, bool QC>
__device__ __forceinline__ void eval_block(const BlockPlane &P, const BlockGeom &g, const float *__restrict__ G,
                                           const float *__restrict__ S, float a0, float a1, float *R0, float *R1,
                                           int pitch, int lane, uint32_t *flags)
{
    const int K = g.K, w = g.w, N = g.w * g.h, rl = g_rowlen(N);
    // lane l covers pixels 4l .. 4l+3 and 128 + 4l .. 128 + 4l + 3: each
    // 16-byte load instruction of the warp reads 512 contiguous bytes of a
    // Green's row (four 128-byte lines)
    const int q0 = 4 * lane, q1 = 128 + 4 * lane;
    const bool act = q0 < N, act1 = q1 < N;
    const bool sym = S != nullptr && N == 256;
    const float *__restrict__ Gb = sym ? S : G;
    // row offsets of the lane's pixels, as stored and y-reversed
    const int lo_n = q0, lo_r = (15 - (lane >> 2)) * 16 + 4 * (lane & 3);
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
        int key = p * rl;
        if (sym) {
            const Sym16 t = sym16(p);
            key = ((t.rx + 2 * t.tr) * kSym16Rows + t.bi) * 256 + (t.ry << 16);
        }
#pragma unroll 4
        for (int u = 0; u < n; ++u) {
            const float cu0 = __shfl_sync(0xffffffffu, c0, u);
            const float cu1 = TWO ? __shfl_sync(0xffffffffu, c1, u) : 0.f;
            const int ku = __shfl_sync(0xffffffffu, key, u);
            if (act) {
                const bool rev = ku >> 16;
                const float *row = Gb + (ku & 0xffff) + (rev ? lo_r : lo_n);
                const float4 lo = __ldg(reinterpret_cast<const float4 *>(row));
                const float4 hi = act1 ? __ldg(reinterpret_cast<const float4 *>(row + (rev ? -128 : 128)))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
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

// ---- the layout groups' residual planes on the tensor cores ---------------
// Per group, R (members x pixels) = V (members x K) E^T (K x pixels):
// mma.sync m16n8k16 with bf16 operands and FP32 accumulation.  The values
// are integers of at most 9 bits (|v| <= 256, checked by the plan), exact
// in bf16; E enters as three bf16 parts, so every product is exact and the
// sum carries FP32 rounding only.  A CTA of 8 warps takes an m-tile of 16
// members; warp w covers pixels 32 w .. 32 w + 31 (four n-tiles of 8), its
// E fragments loaded once per tile.  Accumulator element (m, n) is member
// m's pixel n: two neighbouring pixels of one row per register pair.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// one member row of an m-tile: its residual plane base and values
struct GroupRow {
    float *R;
    const int16_t *v;
    int pitch;
};

__device__ __forceinline__ GroupRow group_row_of(const BlockJobs &J, int entry)
{
    GroupRow r{nullptr, nullptr, 0};
    if (entry < 0) return r;
    const int gb = entry >> 1, sel = entry & 1;
    const BlockPlane &P = J.p[find_job(J, gb)];
    const BlockGeom g = block_geom(P, gb - P.block_base);
    r.pitch = P.r_pitch;
    r.R = P.r[sel] + (size_t)g.y0 * P.r_pitch + g.x0;
    r.v = P.val[sel] + g.s;
    return r;
}

// The layout groups' products, by the first ncta CTAs of the evaluation
// launch (4 warps each): work item = an m-tile of 16 member rows of one
// group; warp w covers the pixels 64 w .. 64 w + 63 (eight n-tiles), E's
// fragments loaded per n-tile.
__device__ __forceinline__ void group_tiles(const BlockJobs &J, const BlockPlan &L, int cta, int ncta)
{
    __shared__ int s_off[kMaxGroups + 1], s_it[kMaxGroups + 1];
    const int ng = group_offsets(L, s_off);
    block_prefix(ng, [&](int g) { return ((int)L.st->gfill[g] + 15) / 16; }, s_it);
    const int total = s_it[ng];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
    constexpr int kPairs = kGroupMaxK / 2;
    for (int item = cta; item < total; item += ncta) {
        int g = 0;
        while (g + 1 < ng && s_it[g + 1] <= item) ++g;
        const int mt = item - s_it[g];
        const int rep = L.st->grep[g];
        const BlockPlane &Pr = J.p[find_job(J, rep)];
        const BlockGeom gr = block_geom(Pr, rep - Pr.block_base);
        const int K = gr.K, w = gr.w, N = gr.w * gr.h;
        const int fill = min((int)L.st->gfill[g], s_off[g + 1] - s_off[g]);
        const int m0 = 16 * mt + gq, m1 = m0 + 8;
        const GroupRow r0 = group_row_of(J, m0 < fill ? L.gmem[s_off[g] + m0] : -1);
        const GroupRow r1 = group_row_of(J, m1 < fill ? L.gmem[s_off[g] + m1] : -1);
        const int nks = (K + 15) / 16;  // 1 or 2 k-steps
        auto val = [&](const GroupRow &r, int k) { return (r.v && k < K) ? (float)__ldg(r.v + k) : 0.f; };
        uint32_t a[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k = 16 * ks + 2 * tq;
            a[ks][0] = pack_bf16(val(r0, k), val(r0, k + 1));
            a[ks][1] = pack_bf16(val(r1, k), val(r1, k + 1));
            a[ks][2] = pack_bf16(val(r0, k + 8), val(r0, k + 9));
            a[ks][3] = pack_bf16(val(r1, k + 8), val(r1, k + 9));
        }
        const uint32_t *E = reinterpret_cast<const uint32_t *>(L.E + (size_t)g * 3 * kGroupRows * kGroupMaxK);
        for (int nt = 0; nt < 8; ++nt) {
            const int n0 = 64 * warp + 8 * nt;
            if (n0 >= N) break;  // the whole warp
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                if (ks >= nks) break;
#pragma unroll
                for (int part = 2; part >= 0; --part) {
                    const uint32_t *row = E + ((size_t)part * kGroupRows + n0 + gq) * kPairs + 8 * ks + tq;
                    mma_bf16(d, a[ks], __ldg(row), __ldg(row + 4));
                }
            }
            const int px = n0 + 2 * tq;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const GroupRow &r = h ? r1 : r0;
                if (!r.R) continue;
                const float v0 = d[2 * h], v1 = d[2 * h + 1];
                const int y = px / w, x = px - y * w;
                float *o = r.R + (size_t)y * r.pitch + x;
                if (px + 1 < N && x + 1 < w && (reinterpret_cast<uintptr_t>(o) & 7) == 0) {
                    *reinterpret_cast<float2 *>(o) = make_float2(v0, v1);
                } else {
                    if (px < N) *o = v0;
                    if (px + 1 < N) {
                        const int y1 = (px + 1) / w, x1 = px + 1 - y1 * w;
                        r.R[(size_t)y1 * r.pitch + x1] = v1;
                    }
                }
            }
        }
    }
}
// member: per block 1 when its layout group's product evaluates it (or
// nullptr: no groups)
// The evaluation launch.  Its first ngemm CTAs compute the layout groups'
// products (the plan has them, groups on); the others take a block per
// warp, skipping the groups' members.
template <bool QC>
__global__ void __launch_bounds__(128, 8) block_eval_kernel(const __grid_constant__ BlockJobs J, BlockTables tab,
                                                            uint32_t *flags, const __grid_constant__ BlockPlan L,
                                                            int ngemm)
{
    // the coefficients (and the groups' E) come from the preceding grid
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if ((int)blockIdx.x < ngemm) {
        group_tiles(J, L, blockIdx.x, ngemm);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = (blockIdx.x - ngemm) * 4 + warp;
    if (gb >= J.total_blocks) return;
    if (L.hkey && L.member[gb]) return;
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
    const float *S = tab.G16o;
    if (QC) {
        // no coefficient stage ran: block pointer errors are reported here
        // (the block reconstructs as zero)
        if (g.bad && lane == 0 && flags) atomicOr(flags, g.bad);
        eval_block<false, true>(P, g, G, S, g.bad ? 0.f : a0, 0.f, R0, nullptr, pitch, lane, flags);
    } else if (two) eval_block<true, false>(P, g, G, S, a0, a1, R0, R1, pitch, lane, flags);
    else eval_block<false, false>(P, g, G, S, a0, a1, R0, R1, pitch, lane, flags);
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
    static std::vector<float> S[kNumOps];
    float *dG = nullptr, *dS = nullptr;
    double *dG64 = nullptr;
    const int *dgoff = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&dG, d_G)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&dG64, d_G64)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&dgoff, d_goff)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&dS, d_G16o)) != cudaSuccess) return e;
    int sms = 0;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    for (int op = 0; op < kNumOps; ++op) {
        if (G[op].empty()) {
            build_tables(op, G[op], G64[op], goff);
            build_sym16(G[op], goff[shape_index(16, 16)], S[op]);
        }
        if ((e = cudaMemcpy(dS + (size_t)op * kSym16Floats, S[op].data(), S[op].size() * sizeof(float),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(dG + (size_t)op * kGSize, G[op].data(), G[op].size() * sizeof(float),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(dG64 + (size_t)op * kGSize, G64[op].data(), G64[op].size() * sizeof(double),
                            cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        BlockTables &t = g_tabs[dev][op];
        t.G = dG + (size_t)op * kGSize;
        t.G64 = dG64 + (size_t)op * kGSize;
        t.G16o = dS + (size_t)op * kSym16Floats;
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

int block_coef_ctas()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    return 3 * sms;  // the kernel's launch bounds: 3 CTAs per SM
}

namespace {

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

uint32_t table_slots(int total_blocks)
{
    uint32_t n = 1024;
    while (n < 2u * (uint32_t)total_blocks && n < (1u << 20)) n <<= 1;
    return n;
}

}  // namespace

size_t block_plan_bytes(int total_blocks, bool groups)
{
    const size_t cap = (size_t)std::max(total_blocks, 1);
    size_t b = a256(sizeof(BlockPlanState)) + a256(4 * cap * kClasses) + a256(4 * cap);  // + deferred
    if (groups) {
        const size_t slots = table_slots(total_blocks);
        b += a256(8 * slots) + 2 * a256(4 * slots) + a256(4 * cap) + a256(cap) + a256(8 * cap) +
             a256((size_t)kMaxGroups * 3 * kGroupRows * kGroupMaxK * 2);
    }
    return b;
}

BlockPlan carve_block_plan(void *mem, int total_blocks, bool groups)
{
    const size_t cap = (size_t)std::max(total_blocks, 1);
    char *m = static_cast<char *>(mem);
    auto take = [&](size_t bytes) {
        char *q = m;
        m += a256(bytes);
        return q;
    };
    BlockPlan L{};
    L.st = reinterpret_cast<BlockPlanState *>(take(sizeof(BlockPlanState)));
    L.list = reinterpret_cast<int32_t *>(take(4 * cap * kClasses));
    L.deferred = reinterpret_cast<int32_t *>(take(4 * cap));
    L.cap = (int32_t)cap;
    if (groups) {
        const uint32_t slots = table_slots(total_blocks);
        L.hmask = slots - 1;
        L.hkey = reinterpret_cast<unsigned long long *>(take(8 * (size_t)slots));
        L.hcnt = reinterpret_cast<uint32_t *>(take(4 * (size_t)slots));
        L.hgid = reinterpret_cast<uint32_t *>(take(4 * (size_t)slots));
        L.slot_of = reinterpret_cast<int32_t *>(take(4 * cap));
        L.member = reinterpret_cast<uint8_t *>(take(cap));
        L.gmem = reinterpret_cast<int32_t *>(take(8 * cap));
        L.E = reinterpret_cast<uint16_t *>(take((size_t)kMaxGroups * 3 * kGroupRows * kGroupMaxK * 2));
    }
    return L;
}

namespace {

// "<gpu>|coef|<blocks rounded up to a power of two>" in the tuner's table
std::string coef_key(int total_blocks)
{
    int b = 1024;
    while (b < total_blocks && b < (1 << 30)) b <<= 1;
    return gpu_name() + "|coef|" + std::to_string(b);
}

// CTAs per SM of the persistent coefficient kernel, timed on this launch's
// own work: 1, 2 and 3 per SM, twice each, round robin, with the plan's
// queues reset before every run (each run computes the same coefficients;
// the timing runs leave the statistics alone).  The choice goes to the
// tuner's table; a later launch computes the coefficients once more.
int tune_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st, int sms)
{
    BlockScratch quiet = s;
    quiet.cstat = nullptr;
    quiet.plan.hkey = nullptr;  // the timing runs solve every block and list no group members
    cudaEvent_t ev[7];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < 7 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
    char *queues = reinterpret_cast<char *>(s.plan.st) + offsetof(BlockPlanState, next);
    const size_t qbytes = offsetof(BlockPlanState, ngroups) - offsetof(BlockPlanState, next);
    for (int t = 0; t < 6 && e == cudaSuccess; ++t) {
        e = cudaMemsetAsync(queues, 0, qbytes, st);
        if (e != cudaSuccess) break;
        PdlConfig c(dim3((t % 3 + 1) * sms), dim3(kCoefThreads), st, false);
        e = cudaLaunchKernelEx(&c.cfg, block_coef_kernel, jobs, block_tables(jobs.op), quiet);
        if (e == cudaSuccess) e = cudaEventRecord(ev[t + 1], st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[6]);
    float best[3] = {1e30f, 1e30f, 1e30f};
    for (int t = 0; t < 6 && e == cudaSuccess; ++t) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ev[t], ev[t + 1]) == cudaSuccess) best[t % 3] = std::min(best[t % 3], ms);
    }
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    // the queues again for the launch that follows
    cudaMemsetAsync(queues, 0, qbytes, st);
    if (e != cudaSuccess) return 3;
    int pick = 3;  // the most CTAs unless fewer are at least 2 % faster
    for (int m = 1; m <= 2; ++m)
        if (best[m - 1] < 0.98f * best[pick - 1]) pick = m;
    tune_store(coef_key(jobs.total_blocks), pick);
    return pick;
}

}  // namespace

cudaError_t launch_block_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st, int *launches, bool pdl)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    const BlockPlan &L = s.plan;
    if (!L.st || L.cap < jobs.total_blocks || s.big_ranges < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(L.st, 0, sizeof(BlockPlanState), st);
    if (e != cudaSuccess) return e;
    const int nb = (jobs.total_blocks + 255) / 256;
    int n = 0;
    if (L.hkey) {
        // clear the layout table (keys, counts and group ids lie back to
        // back, carve_block_plan's order)
        const size_t slots = (size_t)L.hmask + 1;
        if ((e = cudaMemsetAsync(L.hkey, 0, 16 * slots, st)) != cudaSuccess) return e;
    }
    block_plan_kernel<<<nb, 256, 0, st>>>(jobs, L, block_tables(jobs.op), s.tau, s.flags);
    ++n;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    (void)pdl;
    const int sms = block_coef_ctas() / 3;
    const std::string key = coef_key(jobs.total_blocks);
    int per_sm = tune_lookup(key);
    if (per_sm < 1 || per_sm > 3) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
            per_sm = tune_coef(jobs, s, st, sms);
            n += 6;
        } else {
            per_sm = 3;
        }
    }
    PdlConfig c(dim3(per_sm * sms), dim3(kCoefThreads), st, true);
    e = cudaLaunchKernelEx(&c.cfg, block_coef_kernel, jobs, block_tables(jobs.op), s);
    if (launches) *launches += n + 1;
    return e;
}

cudaError_t launch_block_eval(const BlockJobs &jobs, uint32_t *flags, cudaStream_t st, bool pdl, const BlockPlan *plan)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    BlockPlan L{};
    if (plan && plan->hkey) L = *plan;
    // the groups' products: two CTAs per SM at most, before the per-block CTAs
    const int ngemm = L.hkey ? std::max(1, block_coef_ctas() / 3 * 2) : 0;
    PdlConfig c(dim3(ngemm + (jobs.total_blocks + 3) / 4), dim3(128), st, pdl);
    if (jobs.p[0].q)
        return cudaLaunchKernelEx(&c.cfg, block_eval_kernel<true>, jobs, block_tables(jobs.op), flags, L, 0);
    return cudaLaunchKernelEx(&c.cfg, block_eval_kernel<false>, jobs, block_tables(jobs.op), flags, L, ngemm);
}


}  // namespace hivc
