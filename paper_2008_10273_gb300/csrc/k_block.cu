// Block-based pseudodifferential inpainting of the residual (Sec. 2.2,
// Eqs. 2-4; Sec. 2.3), harmonic operator A = -L with mirrored boundaries on
// each w x h block (w, h <= 16).
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
// (the Toeplitz-plus-Hankel structure of G, Sec. 2.2), stored as float.
//
// Kernels: the coefficient stage (16-lane segments, two blocks per warp,
// when both have K <= 16; one block per warp for K <= 32), the large-block
// stage (one CTA per block with K > 32, packed Cholesky in shared memory)
// and the evaluation into a residual field.  The fused inter-frame kernel
// (k_pframe.cu) evaluates with the same routine.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "block_device.cuh"

namespace hivc {
namespace {

constexpr int kGSize = 2283904;  // sum over shapes of N * rowlen(N)

static __device__ __align__(256) float d_G[kGSize];
static __device__ int d_goff[256];

std::mutex g_tab_mu;
BlockTables g_tabs[64];
uint64_t g_tab_devices = 0;  // bit d: tables uploaded to device d

void build_tables(std::vector<float> &G, std::vector<int> &goff)
{
    const double pi = 3.14159265358979323846;
    G.assign(kGSize, 0.f);
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
                            s += cw[a * w + p] * chq[b * h + q] / (4.0 * sp * sp + 4.0 * sq * sq);
                        }
                    T[b * 2 * w + a] = 0.25 * s;
                }
            for (int i = 0; i < N; ++i)
                for (int j = 0; j < N; ++j) {
                    const int xi = i % w, yi = i / w, xj = j % w, yj = j / w;
                    const int a1 = std::abs(xi - xj), a2 = xi + xj + 1, b1 = std::abs(yi - yj), b2 = yi + yj + 1;
                    const double g = T[b1 * 2 * w + a1] + T[b2 * 2 * w + a1] + T[b1 * 2 * w + a2] + T[b2 * 2 * w + a2];
                    G[off + i * rl + j] = (float)g;
                }
            off += N * rl;
        }
}

// ---- coefficient stage ---------------------------------------------------
// A warp takes four consecutive blocks.  When all have K <= 8 it solves them
// at once in 8-lane segments; otherwise pairs in 16-lane segments (K <= 16)
// or single blocks with all 32 lanes (K <= 32).  K > 32 goes to the large-
// block kernel.
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
        if (i == 0) atomicOr(S.flags, kFlagPos);
        return 0;
    }
    return K;
}

// KM = 0: the shared-memory warp routine (16 < K <= 32)
template <int SEG, int KM>
__device__ __forceinline__ void seg_run(const SegBlock &b, int K, int i, float (*Lt)[SEG + 1], const BlockTables &tab,
                                        const BlockScratch &S)
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
        spd = warp_block_coef_smem(G, rl, K, i, p, v0, v1, reinterpret_cast<float(*)[33]>(&Lt[0][0]), c0, c1, a0, a1);
    else
        spd = seg_block_coef<SEG, KM, true>(G, rl, K, i, p, v0, v1, Lt, c0, c1, a0, a1);
    if (K > 0) {
        if (i < K) {
            P->coef[0][b.g.s + i] = c0;
            if (two) P->coef[1][b.g.s + i] = c1;
        }
        if (i == 0) {
            P->acoef[0][b.g.lb] = a0;
            if (two) P->acoef[1][b.g.lb] = a1;
            if (!spd) atomicOr(S.flags, kFlagNotSPD);
        }
    }
}

__device__ __forceinline__ void coef_quad(const BlockJobs &J, const BlockTables &tab, const BlockScratch &S, int gb0,
                                          int lane, float *lts)
{
    // lane q < 4 owns block gb0 + q: error flags and the large-block list
    int kq;
    {
        const SegBlock bq = seg_block(J, gb0 + (lane & 3));
        kq = seg_k(bq);
        if (lane < 4 && bq.P != nullptr) {
            if (bq.g.bad) {
                atomicOr(S.flags, bq.g.bad);
            } else if (bq.g.K > kWarpK) {
                const uint32_t i = atomicAdd(S.ctr + kCtrLargeCount, 1u);
                if (i < (uint32_t)S.large_cap) S.large_list[i] = (uint32_t)(gb0 + lane);
            }
        }
    }
    const int k0 = __shfl_sync(0xffffffffu, kq, 0), k1 = __shfl_sync(0xffffffffu, kq, 1);
    const int k2 = __shfl_sync(0xffffffffu, kq, 2), k3 = __shfl_sync(0xffffffffu, kq, 3);
    const int k01 = max(k0, k1), k23 = max(k2, k3);
    if (max(k01, k23) == 0) return;
    if (max(k01, k23) <= 8) {
        const int seg = lane >> 3, i = lane & 7;
        SegBlock bb = seg_block(J, gb0 + seg);
        bb.g.K = seg_k(bb);
        const int K = seg_validate<8>(bb, i, seg, S);
        seg_run<8, 8>(bb, K, i, reinterpret_cast<float(*)[9]>(lts + seg * 8 * 9), tab, S);
        __syncwarp();
        return;
    }
#pragma unroll 1
    for (int pr = 0; pr < 2; ++pr) {
        const int kp = pr ? k23 : k01;
        if (kp == 0) continue;
        if (kp <= 16) {
            const int seg = lane >> 4, i = lane & 15;
            SegBlock bb = seg_block(J, gb0 + 2 * pr + seg);
            bb.g.K = seg_k(bb);
            const int K = seg_validate<16>(bb, i, seg, S);
            auto Lt = reinterpret_cast<float(*)[17]>(lts + seg * 16 * 17);
            seg_run<16, 16>(bb, K, i, Lt, tab, S);
        } else {
            auto Lt = reinterpret_cast<float(*)[33]>(lts);
#pragma unroll 1
            for (int k = 0; k < 2; ++k) {
                SegBlock bb = seg_block(J, gb0 + 2 * pr + k);
                bb.g.K = seg_k(bb);
                const int K = seg_validate<32>(bb, lane, 0, S);
                if (K == 0) continue;
                if (K <= 24) seg_run<32, 24>(bb, K, lane, Lt, tab, S);
                else seg_run<32, 0>(bb, K, lane, Lt, tab, S);
            }
        }
        __syncwarp();
    }
}

// ---- large blocks (K > 32): one CTA, packed Cholesky in global scratch ----
constexpr int kCoefThreads = 128;

__device__ __forceinline__ int pk(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

__device__ __forceinline__ float cta_sum(float v, float *red)
{
    v = seg_sum<32>(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    for (int k = 0; k < kCoefThreads / 32; ++k) t += red[k];
    return t;
}

// One block with K > 32 by the whole CTA: G_PP packed in S.big (global),
// right-hand sides in S.big after it.  Same arithmetic as seg_block_coef.
__device__ __noinline__ void cta_large_solve(const BlockJobs &J, const BlockTables &tab, const BlockScratch &S, int gb,
                                unsigned char *s_p, float *red, int *s_bad)
{
    const int tid = threadIdx.x;
    const BlockPlane &P = J.p[find_job(J, gb)];
    const BlockGeom g = block_geom(P, gb - P.block_base);
    const int K = g.K;
    const bool two = P.val[1] != nullptr;
    float *L = S.big;
    float *b = S.big + (size_t)kBigMaxK * (kBigMaxK + 1) / 2;  // b[r*K + i]
    if (tid == 0) *s_bad = 0;
    __syncthreads();
    for (int j = tid; j < K; j += kCoefThreads) {
        int p;
        if (!load_pos(P, g, j, p)) *s_bad = 1;
        s_p[j] = (unsigned char)p;
        b[j] = (float)__ldg(P.val[0] + g.s + j);
        b[K + j] = two ? (float)__ldg(P.val[1] + g.s + j) : 0.f;
        b[2 * K + j] = 1.f;
    }
    __syncthreads();
    if (*s_bad) {
        if (tid == 0) atomicOr(S.flags, kFlagPos);
        __syncthreads();
        return;
    }
    const float *G = green_rows(tab, g.w, g.h);
    const int rl = g_rowlen(g.w * g.h);
    for (int i = tid; i < K; i += kCoefThreads)
        for (int j = 0; j <= i; ++j) L[pk(i, j)] = __ldg(G + s_p[i] * rl + s_p[j]);
    __syncthreads();
    bool spd = true;
    for (int k = 0; k < K; ++k) {
        const float d = L[pk(k, k)];
        spd = spd && d > 0.f;
        const float isd = rsqrtf(fmaxf(d, 1e-30f));
        __syncthreads();
        if (tid == 0) L[pk(k, k)] = d * isd;
        for (int i = k + 1 + tid; i < K; i += kCoefThreads) L[pk(i, k)] *= isd;
        __syncthreads();
        for (int i = k + 1 + tid; i < K; i += kCoefThreads) {
            const float lik = L[pk(i, k)];
            for (int j = k + 1; j <= i; ++j) L[pk(i, j)] = fmaf(-lik, L[pk(j, k)], L[pk(i, j)]);
        }
        __syncthreads();
    }
    for (int k = 0; k < K; ++k) {  // forward L y = b (three right-hand sides)
        if (tid < 3) b[tid * K + k] /= L[pk(k, k)];
        __syncthreads();
        for (int i = k + 1 + tid; i < K; i += kCoefThreads) {
            const float l = L[pk(i, k)];
            b[i] = fmaf(-l, b[k], b[i]);
            b[K + i] = fmaf(-l, b[K + k], b[K + i]);
            b[2 * K + i] = fmaf(-l, b[2 * K + k], b[2 * K + i]);
        }
        __syncthreads();
    }
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;  // a = (y_1 . y_v) / (y_1 . y_1)
    for (int i = tid; i < K; i += kCoefThreads) {
        const float y2 = b[2 * K + i];
        s0 += y2 * b[i];
        s1 += y2 * b[K + i];
        s2 += y2 * y2;
    }
    s2 = cta_sum(s2, red);
    const float a0 = cta_sum(s0, red) / s2, a1 = cta_sum(s1, red) / s2;
    __syncthreads();
    for (int i = tid; i < K; i += kCoefThreads) {
        b[i] = fmaf(-a0, b[2 * K + i], b[i]);
        b[K + i] = fmaf(-a1, b[2 * K + i], b[K + i]);
    }
    __syncthreads();
    for (int k = K - 1; k >= 0; --k) {  // backward L^T c = y_v - a y_1
        if (tid < 2) b[tid * K + k] /= L[pk(k, k)];
        __syncthreads();
        for (int i = tid; i < k; i += kCoefThreads) {
            const float l = L[pk(k, i)];
            b[i] = fmaf(-l, b[k], b[i]);
            b[K + i] = fmaf(-l, b[K + k], b[K + i]);
        }
        __syncthreads();
    }
    for (int i = tid; i < K; i += kCoefThreads) {
        P.coef[0][g.s + i] = b[i];
        if (two) P.coef[1][g.s + i] = b[K + i];
    }
    if (tid == 0) {
        P.acoef[0][g.lb] = a0;
        if (two) P.acoef[1][g.lb] = a1;
        if (!spd) atomicOr(S.flags, kFlagNotSPD);
    }
    __syncthreads();
}

// Coefficient stage: warp w of CTA c solves quad 4c + w (blocks 16c + 4w ..
// +3).  Blocks with K > 32 are listed; the last CTA to finish solves them
// and clears the list (a done counter, no waiting).
__global__ void __launch_bounds__(kCoefThreads, 7) block_coef_kernel(const __grid_constant__ BlockJobs J,
                                                                     BlockTables tab, BlockScratch S)
{
    __shared__ float lts[4][32 * 33];
    __shared__ unsigned char s_p[kBigMaxK];
    __shared__ float red[kCoefThreads / 32];
    __shared__ int s_last, s_bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the fused kernel that follows may start its prologue (tensor-memory
    // copies of flow and references) now; it waits for this grid's results
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int gb0 = (blockIdx.x * 4 + warp) * 4;
    if (gb0 < J.total_blocks) coef_quad(J, tab, S, gb0, lane, lts[warp]);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(S.ctr + kCtrCoefDone, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const uint32_t n = min(*(volatile uint32_t *)(S.ctr + kCtrLargeCount), (uint32_t)S.large_cap);
    for (uint32_t it = 0; it < n; ++it) cta_large_solve(J, tab, S, (int)S.large_list[it], s_p, red, &s_bad);
    if (threadIdx.x == 0) {
        S.ctr[kCtrLargeCount] = 0;
        S.ctr[kCtrCoefDone] = 0;
        __threadfence();
    }
}

// ---- evaluation stage into residual fields, one warp per block -----------
__global__ void __launch_bounds__(128) block_eval_kernel(const __grid_constant__ BlockJobs J, BlockTables tab,
                                                         uint32_t *flags)
{
    __shared__ float cs[4][2][256];
    __shared__ unsigned char ps[4][256];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x * 4 + warp;
    if (gb >= J.total_blocks) return;
    const BlockPlane &P = J.p[find_job(J, gb)];
    const BlockGeom g = block_geom(P, gb - P.block_base);
    const int K = g.K, w = g.w, N = g.w * g.h;
    const bool two = P.val[1] != nullptr;
    bool valid = true;
    for (int j0 = 0; j0 < K; j0 += 32) {
        int p = 0;
        const bool ok = (j0 + lane < K) ? load_pos(P, g, j0 + lane, p) : true;
        valid = valid && !__any_sync(0xffffffffu, !ok);
        if (j0 + lane < K) {
            ps[warp][j0 + lane] = (unsigned char)p;
            cs[warp][0][j0 + lane] = __ldg(P.coef[0] + g.s + j0 + lane);
            if (two) cs[warp][1][j0 + lane] = __ldg(P.coef[1] + g.s + j0 + lane);
        }
    }
    if (!valid && lane == 0) atomicOr(flags, kFlagPos);
    __syncwarp();
    const int pitch = P.r_pitch;
    float *R0 = P.r[0] + (size_t)g.y0 * pitch + g.x0;
    float *R1 = two && P.r[1] ? P.r[1] + (size_t)g.y0 * pitch + g.x0 : nullptr;
    if (K == 0 || !valid) {
        for (int i = lane; i < N; i += 32) {
            R0[(i / w) * pitch + i % w] = 0.f;
            if (R1) R1[(i / w) * pitch + i % w] = 0.f;
        }
        return;
    }
    const float a0 = __ldg(P.acoef[0] + g.lb), a1 = two ? __ldg(P.acoef[1] + g.lb) : 0.f;
    const float *G = green_rows(tab, g.w, g.h);
    auto out = [&](int x, int y, float v0, float v1) {
        const int o = y * pitch + x;
        R0[o] = v0;
        if (R1) R1[o] = v1;
    };
    if (two) warp_block_eval<true>(G, w, N, K, ps[warp], cs[warp][0], cs[warp][1], a0, a1, lane, out);
    else warp_block_eval<false>(G, w, N, K, ps[warp], cs[warp][0], cs[warp][1], a0, a1, lane, out);
    __syncwarp();
    // the data at the points, exactly
    for (int j = lane; j < K; j += 32) {
        const size_t o = (size_t)(ps[warp][j] / w) * pitch + ps[warp][j] % w;
        R0[o] = (float)__ldg(P.val[0] + g.s + j);
        if (R1) R1[o] = (float)__ldg(P.val[1] + g.s + j);
    }
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
    static std::vector<float> G;
    static std::vector<int> goff;
    if (G.empty()) build_tables(G, goff);
    if ((e = cudaMemcpyToSymbol(d_G, G.data(), G.size() * sizeof(float))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(d_goff, goff.data(), goff.size() * sizeof(int))) != cudaSuccess) return e;
    BlockTables t{};
    if ((e = cudaGetSymbolAddress((void **)&t.G, d_G)) != cudaSuccess) return e;
    if ((e = cudaGetSymbolAddress((void **)&t.goff, d_goff)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&t.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = fused_init()) != cudaSuccess) return e;
    g_tabs[dev] = t;
    g_tab_devices |= 1ull << dev;
    return cudaSuccess;
}

const BlockTables &block_tables()
{
    int dev = 0;
    cudaGetDevice(&dev);
    return g_tabs[dev < 64 ? dev : 0];
}

cudaError_t launch_block_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st, int *launches)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    block_coef_kernel<<<(jobs.total_blocks + 15) / 16, kCoefThreads, 0, st>>>(jobs, block_tables(), s);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_block_eval(const BlockJobs &jobs, uint32_t *flags, cudaStream_t st)
{
    if (jobs.total_blocks == 0) return cudaSuccess;
    block_eval_kernel<<<(jobs.total_blocks + 3) / 4, 128, 0, st>>>(jobs, block_tables(), flags);
    return cudaGetLastError();
}

}  // namespace hivc
