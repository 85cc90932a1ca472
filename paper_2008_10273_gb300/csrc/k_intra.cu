// Intra prediction: homogeneous diffusion inpainting (Sec. 2.1, Eq. 1) with
// A = -L, the 5-point Laplacian with reflecting boundaries, h = 1.
//
//   u_i = f_i on the mask,   (L u)_i = sum_{in-image nbrs j} (u_j - u_i) = 0 elsewhere.
//
// Mixed-precision correction loop (the host drives the cycles):
//   u (FP64) holds the iterate; r = (L u)_U is evaluated in FP64 and stored
//   as FP32; the correction equation (-L_UU) e = r is relaxed in FP32 by
//   red-black SOR sweeps (e = 0 on the mask); then u += e in FP64.  Each
//   cycle shrinks the residual by the inner solve's reduction, so the FP64
//   iterate reaches residuals far below the FP32 rounding floor.
//
// The SOR kernel is temporally blocked: a tile with a halo of 2S pixels is
// staged in shared memory and S full red-black sweeps run there before the
// interior is written back (each half sweep invalidates one more halo ring).
#include <cfloat>

#include "hivc_internal.cuh"

namespace hivc {
namespace {

constexpr int kTX = 64, kTY = 32;  // SOR output tile
constexpr int kSweeps = 4;         // full sweeps per SOR launch
constexpr int kHalo = 2 * kSweeps;
constexpr int kRW = kTX + 2 * kHalo, kRH = kTY + 2 * kHalo;
constexpr int kRT = 32, kRT_Y = 8;  // residual kernel tile (32 x 8 threads)

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }

__device__ __forceinline__ int find_plane(const IntraJobs &J, int t)
{
    int j = 0;
    for (int k = 1; k < J.n; ++k)
        if (t >= J.p[k].tile_base) j = k;
    return j;
}

// sum of mask values + index validation (grid-stride per plane = blockIdx.y)
__global__ void intra_sum_kernel(const __grid_constant__ IntraJobs J, uint32_t *flags)
{
    const IntraPlane &P = J.p[blockIdx.y];
    const uint32_t N = (uint32_t)P.width * (uint32_t)P.height;
    double s = 0.0;
    bool bad = false;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.n; k += gridDim.x * blockDim.x) {
        const uint32_t i = __ldg(P.idx + k);
        bad |= (i >= N) || (k > 0 && __ldg(P.idx + k - 1) >= i);
        s += (double)__ldg(P.val + k);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagMaskIdx);
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(P.sum, t);
    }
}

// u = mean mask value, mask = 0 everywhere (pitched plane)
__global__ void intra_fill_kernel(const __grid_constant__ IntraJobs J)
{
    const IntraPlane &P = J.p[blockIdx.y];
    const double mean = P.n > 0 ? *P.sum / P.n : 0.0;
    const size_t total = (size_t)P.height * P.pitch;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        P.u[0][i] = mean;
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
        P.u[0][o] = (double)__ldg(P.val + k);
        P.mask[o] = 1;
    }
}

// FP64: u_out = u_in + e (unknown pixels), res = float((L u_out)_i), max |.|
__global__ void __launch_bounds__(kRT * kRT_Y) intra_residual_kernel(const __grid_constant__ IntraJobs J, int in,
                                                                      int e_in, int add_e)
{
    const int t = blockIdx.x;
    const IntraPlane &P = J.p[find_plane(J, t)];
    const int lt = t - P.tile_base;
    const int x = (lt % P.tiles_x) * kRT + (threadIdx.x & 31);
    const int y = (lt / P.tiles_x) * kRT_Y + (threadIdx.x >> 5);
    double rabs = 0.0;
    if (x < P.width && y < P.height) {
        const double *u = P.u[in];
        const float *e = P.e[e_in];
        const size_t i = (size_t)y * P.pitch + x;
        auto val = [&](size_t k) -> double { return add_e ? u[k] + (double)e[k] : u[k]; };
        const double c = val(i);
        if (add_e) P.u[in ^ 1][i] = c;
        if (!P.mask[i]) {
            double s = 0.0;
            if (x > 0) s += val(i - 1) - c;
            if (x < P.width - 1) s += val(i + 1) - c;
            if (y > 0) s += val(i - P.pitch) - c;
            if (y < P.height - 1) s += val(i + P.pitch) - c;
            P.res[i] = (float)s;
            rabs = fabs(s);
        } else {
            P.res[i] = 0.f;
        }
    }
    for (int o = 16; o > 0; o >>= 1) rabs = fmax(rabs, __shfl_xor_sync(0xffffffffu, rabs, o));
    __shared__ double red[kRT_Y];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rabs;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int k = 0; k < kRT_Y; ++k) m = fmax(m, red[k]);
        atomicMax(P.rnorm, dbits(m));  // non-negative doubles order like their bits
    }
}

// S red-black SOR sweeps on (-L_UU) e = res in a shared-memory tile
__global__ void __launch_bounds__(256) intra_sor_kernel(const __grid_constant__ IntraJobs J, int e_in, int from_zero)
{
    __shared__ float se[kRH * kRW];
    __shared__ float sr[kRH * kRW];
    __shared__ unsigned char sn[kRH * kRW];  // 0: fixed (mask / outside), else neighbour count
    const int t = blockIdx.x;
    const IntraPlane &P = J.p[find_plane(J, t)];
    const int lt = t - P.tile_base;
    const int tx0 = (lt % P.tiles_x) * kTX, ty0 = (lt / P.tiles_x) * kTY;
    const int gx0 = tx0 - kHalo, gy0 = ty0 - kHalo;
    const int W = P.width, H = P.height;
    const float *ein = P.e[e_in];
    float *eout = P.e[e_in ^ 1];
    for (int k = threadIdx.x; k < kRH * kRW; k += blockDim.x) {
        const int lx = k % kRW, ly = k / kRW;
        const int gx = gx0 + lx, gy = gy0 + ly;
        float ev = 0.f, rv = 0.f;
        unsigned char n = 0;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const size_t i = (size_t)gy * P.pitch + gx;
            if (!P.mask[i]) {
                n = (unsigned char)((gx > 0) + (gx < W - 1) + (gy > 0) + (gy < H - 1));
                rv = P.res[i];
                if (!from_zero) ev = ein[i];
            }
        }
        se[k] = ev;
        sr[k] = rv;
        sn[k] = n;
    }
    __syncthreads();
    const float omega = P.omega;
    const int par = (tx0 + ty0) & 1;  // parity offset of local -> global coordinates
    for (int m = 1; m <= 2 * kSweeps; ++m) {
        const int colour = (m - 1) & 1;  // red (even x+y) first
        for (int k = threadIdx.x; k < (kRW / 2) * kRH; k += blockDim.x) {
            const int ly = k / (kRW / 2);
            const int lx = 2 * (k % (kRW / 2)) + ((colour + ly + par) & 1);
            if (ly < m || ly >= kRH - m || lx < m || lx >= kRW - m) continue;
            const int i = ly * kRW + lx;
            const int n = sn[i];
            if (n == 0) continue;
            const float s = (se[i - 1] + se[i + 1]) + (se[i - kRW] + se[i + kRW]) + sr[i];
            const float inv = n == 4 ? 0.25f : (n == 3 ? (1.0f / 3.0f) : (n == 2 ? 0.5f : 1.0f));
            se[i] = fmaf(omega, fmaf(s, inv, -se[i]), se[i]);
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < kTX * kTY; k += blockDim.x) {
        const int lx = kHalo + k % kTX, ly = kHalo + k / kTX;
        const int gx = gx0 + lx, gy = gy0 + ly;
        if (gx < W && gy < H) eout[(size_t)gy * P.pitch + gx] = se[ly * kRW + lx];
    }
}

}  // namespace

cudaError_t launch_intra_init(IntraJobs &J, uint32_t *flags, cudaStream_t st, int *launches)
{
    for (int k = 0; k < J.n; ++k) {
        cudaError_t e = cudaMemsetAsync(J.p[k].sum, 0, sizeof(double), st);
        if (e != cudaSuccess) return e;
    }
    dim3 g(64, J.n);
    intra_sum_kernel<<<g, 256, 0, st>>>(J, flags);
    intra_fill_kernel<<<dim3(256, J.n), 256, 0, st>>>(J);
    intra_scatter_kernel<<<g, 256, 0, st>>>(J);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_intra_residual(IntraJobs &J, int in, int e_in, bool add_e, cudaStream_t st)
{
    int base = 0;
    for (int k = 0; k < J.n; ++k) {
        IntraPlane &P = J.p[k];
        P.tiles_x = (P.width + kRT - 1) / kRT;
        P.tile_base = base;
        base += P.tiles_x * ((P.height + kRT_Y - 1) / kRT_Y);
        cudaError_t e = cudaMemsetAsync(P.rnorm, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    if (base == 0) return cudaSuccess;
    intra_residual_kernel<<<base, kRT * kRT_Y, 0, st>>>(J, in, e_in, add_e ? 1 : 0);
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
    const int launches_needed = (sweeps + kSweeps - 1) / kSweeps;
    for (int l = 0; l < launches_needed; ++l) {
        intra_sor_kernel<<<base, 256, 0, st>>>(J, cur, (from_zero && l == 0) ? 1 : 0);
        cur ^= 1;
    }
    if (launches) *launches += launches_needed;
    *e_out = cur;
    return cudaGetLastError();
}

}  // namespace hivc
