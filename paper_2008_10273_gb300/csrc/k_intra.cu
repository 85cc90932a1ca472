// Intra prediction: homogeneous diffusion inpainting (Sec. 2.1, Eq. 1) with
// A = -L, the 5-point Laplacian with reflecting boundaries, h = 1.
//
//   u_i = f_i on the mask,   (L u)_i = sum_{in-image nbrs j} (u_j - u_i) = 0 elsewhere.
//
// Correction loop (the host drives the cycles):
//   the iterate u is a float-float pair (hi + lo, ~48-bit significand);
//   r = (L u)_U is evaluated exactly enough for residuals down to ~1e-11 by
//   TwoSum on the neighbour differences, and stored as FP32; the correction
//   equation (-L_UU) e = r is relaxed in FP32 by red-black SOR sweeps
//   (e = 0 on the mask); then u += e in float-float.  Each cycle shrinks the
//   residual by the inner solve's reduction, so the iterate reaches
//   residuals far below the FP32 rounding floor.  (GB300 runs FP64 at a
//   small fraction of its FP32 rate, so the extended precision is built
//   from FP32 operations.)  With precision = 1 the lo part stays zero and
//   the residual is plain FP32.
//
// The SOR kernel is temporally blocked: a tile with a halo of 2S pixels is
// staged in shared memory, split into its red and black cells, and S full
// red-black sweeps run there before the interior is written back (each half
// sweep invalidates one more halo ring).
#include <cfloat>

#include "hivc_internal.cuh"

namespace hivc {
namespace {

// ---- SOR tile geometry ---------------------------------------------------
constexpr int kS = 4;                   // full sweeps per launch
constexpr int kHL = 2 * kS;             // halo
constexpr int kRW = 128, kRH = 64;      // staged region
constexpr int kTX = kRW - 2 * kHL;      // 112 output columns
constexpr int kTY = kRH - 2 * kHL;      // 48 output rows
constexpr int kHW = kRW / 2;            // cells per colour and row
constexpr int kTY_THREADS = 8;          // thread rows; each thread owns kRH/8 rows
constexpr int kRows = kRH / kTY_THREADS;

constexpr int kResThreads = 256;

__device__ __forceinline__ int find_plane(const IntraJobs &J, int t)
{
    int j = 0;
    for (int k = 1; k < J.n; ++k)
        if (t >= J.p[k].tile_base) j = k;
    return j;
}

// error-free transformations (Knuth TwoSum, Dekker FastTwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// u + e as a normalised float-float
__device__ __forceinline__ void ff_add(float h, float l, float e, float &oh, float &ol)
{
    float s, t;
    two_sum(h, e, s, t);
    fast_two_sum(s, __fadd_rn(t, l), oh, ol);
}

// sum of mask values (exact, integer) + index validation; plane = blockIdx.y
__global__ void intra_sum_kernel(const __grid_constant__ IntraJobs J, uint32_t *flags)
{
    const IntraPlane &P = J.p[blockIdx.y];
    const uint32_t N = (uint32_t)P.width * (uint32_t)P.height;
    unsigned long long s = 0;
    bool bad = false;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.n; k += gridDim.x * blockDim.x) {
        const uint32_t i = __ldg(P.idx + k);
        bad |= (i >= N) || (k > 0 && __ldg(P.idx + k - 1) >= i);
        s += __ldg(P.val + k);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(P.vsum, s);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagMaskIdx);
}

// u = mean mask value (hi), lo = 0, mask = 0
__global__ void intra_fill_kernel(const __grid_constant__ IntraJobs J)
{
    const IntraPlane &P = J.p[blockIdx.y];
    const float mean = P.n > 0 ? (float)((double)*P.vsum / (double)P.n) : 0.f;
    const size_t total = (size_t)P.height * P.pitch;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        P.uh[0][i] = mean;
        P.ul[0][i] = 0.f;
        P.mask[i] = 0;
    }
}

// u = f, mask = 1 at the mask pixels (indices out of range are skipped)
__global__ void intra_scatter_kernel(const __grid_constant__ IntraJobs J)
{
    const IntraPlane &P = J.p[blockIdx.y];
    const uint32_t N = (uint32_t)P.width * (uint32_t)P.height;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.n; k += gridDim.x * blockDim.x) {
        const uint32_t i = __ldg(P.idx + k);
        if (i >= N) continue;
        const size_t o = (size_t)(i / P.width) * P.pitch + (i % P.width);
        P.uh[0][o] = (float)__ldg(P.val + k);
        P.mask[o] = 1;
    }
}

// u_out = u_in + e (unknown pixels; float-float), res = (L u_out)_i, and the
// max |res| per plane.  Persistent grid: each CTA walks rows of all planes.
__global__ void __launch_bounds__(kResThreads) intra_residual_kernel(const __grid_constant__ IntraJobs J, int e_in,
                                                                     int add_e)
{
    __shared__ float red[kResThreads / 32];
    for (int pl = 0; pl < J.n; ++pl) {
        const IntraPlane &P = J.p[pl];
        const int W = P.width, H = P.height, pitch = P.pitch;
        const float *uh = P.uh[0], *ul = P.ul[0];
        const float *e = P.e[e_in];
        const bool ff = P.ff != 0;
        float rmax = 0.f;
        const long total = (long)H * W;
        for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long)gridDim.x * blockDim.x) {
            const int y = (int)(k / W), x = (int)(k - (long)y * W);
            const size_t i = (size_t)y * pitch + x;
            auto get = [&](size_t j, float &h, float &l) {
                h = uh[j];
                l = ff ? ul[j] : 0.f;
                if (add_e) {
                    const float d = e[j];
                    if (ff) ff_add(h, l, d, h, l);
                    else h = __fadd_rn(h, d);
                }
            };
            float ch, cl;
            get(i, ch, cl);
            if (add_e) {
                P.uh[1][i] = ch;
                if (ff) P.ul[1][i] = cl;
            }
            float r = 0.f;
            if (!P.mask[i]) {
                // sum_j (h_j - h_i) exactly as float-float, plus the lo parts
                float S = 0.f, E = 0.f, tail = 0.f;
                auto acc = [&](size_t j) {
                    float h, l, d, de, s2, e2;
                    get(j, h, l);
                    two_sum(h, -ch, d, de);
                    two_sum(S, d, s2, e2);
                    S = s2;
                    E = __fadd_rn(E, __fadd_rn(e2, de));
                    tail = __fadd_rn(tail, __fsub_rn(l, cl));
                };
                if (x > 0) acc(i - 1);
                if (x < W - 1) acc(i + 1);
                if (y > 0) acc(i - pitch);
                if (y < H - 1) acc(i + pitch);
                r = __fadd_rn(S, __fadd_rn(E, tail));
            }
            P.res[i] = r;
            rmax = fmaxf(rmax, fabsf(r));
        }
        for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int w = 0; w < kResThreads / 32; ++w) m = fmaxf(m, red[w]);
            if (m > 0.f) atomicMax(P.rnorm, __float_as_uint(m));  // non-negative floats order like their bits
        }
        __syncthreads();
    }
}

// S red-black SOR sweeps on (-L_UU) e = res in a shared-memory tile.
// Thread (tx, ty) owns the cell pair hx = tx (columns 2tx, 2tx+1) in rows
// ty + 8k; within a half sweep all its cells of one colour sit at the same
// column offset b, so per-cell coefficients stay in registers.
__global__ void __launch_bounds__(kHW *kTY_THREADS, 2) intra_sor_kernel(const __grid_constant__ IntraJobs J, int e_in,
                                                                        int from_zero)
{
    __shared__ float E[2][kRH][kHW];
    const IntraPlane &P = J.p[find_plane(J, blockIdx.x)];
    const int lt = blockIdx.x - P.tile_base;
    const int tx0 = (lt % P.tiles_x) * kTX, ty0 = (lt / P.tiles_x) * kTY;
    const int gx0 = tx0 - kHL, gy0 = ty0 - kHL;
    const int W = P.width, H = P.height, pitch = P.pitch;
    const int x = threadIdx.x, ty = threadIdx.y;
    const int par = (tx0 + ty0) & 1;
    const float *ein = P.e[e_in];
    float *eout = P.e[e_in ^ 1];
    float inv[2][kRows], rinv[2][kRows];  // [colour][k]
    const int col0 = (ty + par) & 1;  // colour of the pair's left cell (ly has the parity of ty)
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int ly = ty + kTY_THREADS * k, gy = gy0 + ly;
        float ev[2], iv[2], rv[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int gx = gx0 + 2 * x + b;
            ev[b] = 0.f;
            iv[b] = 0.f;
            rv[b] = 0.f;
            if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
                const size_t i = (size_t)gy * pitch + gx;
                if (!P.mask[i]) {
                    const int n = (gx > 0) + (gx < W - 1) + (gy > 0) + (gy < H - 1);
                    iv[b] = n == 4 ? 0.25f : (n == 3 ? (1.0f / 3.0f) : (n == 2 ? 0.5f : 1.0f));
                    rv[b] = P.res[i] * iv[b];
                    if (!from_zero) ev[b] = ein[i];
                }
            }
        }
        // cell b of the pair has colour col0 ^ b
        E[col0][ly][x] = ev[0];
        E[col0 ^ 1][ly][x] = ev[1];
        inv[0][k] = col0 ? iv[1] : iv[0];
        inv[1][k] = col0 ? iv[0] : iv[1];
        rinv[0][k] = col0 ? rv[1] : rv[0];
        rinv[1][k] = col0 ? rv[0] : rv[1];
    }
    __syncthreads();
    const float omega = P.omega;
#pragma unroll
    for (int m = 1; m <= 2 * kS; ++m) {
        const int c = (m - 1) & 1, o = c ^ 1;
        const int b = (c + ty + par) & 1;
        const int lx = 2 * x + b;
        if (lx >= m && lx < kRW - m) {
#pragma unroll
            for (int k = 0; k < kRows; ++k) {
                const int ly = ty + kTY_THREADS * k;
                if (ly >= m && ly < kRH - m) {
                    const float s = (E[o][ly][x + b - 1] + E[o][ly][x + b]) + (E[o][ly - 1][x] + E[o][ly + 1][x]);
                    const float e = E[c][ly][x];
                    // fixed cells have inv = rinv = 0 and e = 0: they stay 0
                    E[c][ly][x] = fmaf(omega, fmaf(s, inv[c][k], rinv[c][k] - e), e);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int ly = ty + kTY_THREADS * k, gy = gy0 + ly;
        if (ly < kHL || ly >= kHL + kTY || gy >= H) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int lx = 2 * x + b, gx = gx0 + lx;
            if (lx < kHL || lx >= kHL + kTX || gx >= W) continue;
            eout[(size_t)gy * pitch + gx] = E[(b + ty + par) & 1][ly][x];
        }
    }
}

}  // namespace

cudaError_t launch_intra_init(IntraJobs &J, uint32_t *flags, cudaStream_t st, int *launches)
{
    for (int k = 0; k < J.n; ++k) {
        cudaError_t e = cudaMemsetAsync(J.p[k].vsum, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    intra_sum_kernel<<<dim3(32, J.n), 256, 0, st>>>(J, flags);
    intra_fill_kernel<<<dim3(304, J.n), 256, 0, st>>>(J);
    intra_scatter_kernel<<<dim3(64, J.n), 256, 0, st>>>(J);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_intra_residual(IntraJobs &J, int e_in, bool add_e, cudaStream_t st)
{
    long px = 0;
    for (int k = 0; k < J.n; ++k) {
        cudaError_t e = cudaMemsetAsync(J.p[k].rnorm, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
        px += (long)J.p[k].width * J.p[k].height;
    }
    if (px == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long want = (px / 3 + kResThreads - 1) / kResThreads;
    const int grid = (int)std::max(1L, std::min((long)sms * 8, want));
    intra_residual_kernel<<<grid, kResThreads, 0, st>>>(J, e_in, add_e ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_intra_sor(IntraJobs &J, int e_in, bool from_zero, int sweeps, cudaStream_t st, int *e_out,
                             int *launches)
{
    int base = 0;
    for (int k = 0; k < J.n; ++k) {
        IntraPlane &P = J.p[k];
        P.tiles_x = (P.width + kTX - 1) / kTX;
        P.tile_base = base;
        base += P.tiles_x * ((P.height + kTY - 1) / kTY);
    }
    int cur = e_in;
    const int n = (sweeps + kS - 1) / kS;
    for (int l = 0; l < n; ++l) {
        intra_sor_kernel<<<base, dim3(kHW, kTY_THREADS), 0, st>>>(J, cur, (from_zero && l == 0) ? 1 : 0);
        cur ^= 1;
    }
    if (launches) *launches += n;
    *e_out = cur;
    return cudaGetLastError();
}

int intra_sweeps_per_launch() { return kS; }

}  // namespace hivc
