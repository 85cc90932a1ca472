// Inter prediction by backward warping (Sec. 2, Sec. 2.3) and the final
// correction step (prediction + residual, clamped to [0, 255]), plus the
// uint8 pack.  One launch covers all planes of a frame.  The 4:4:4 colour
// path (RCT planes) has its own kernel that also applies the inverse RCT.
//
// pred(x) = ref(x + v(x)), bilinear; the sample position is clamped to the
// plane.  The integer part and the fraction of v are split in FP32
// (v - floor(v) is exact), so the interpolation weights do not lose bits to
// the pixel coordinate.  4:2:0 chroma planes use v_c = half the mean of the
// in-plane luma vectors among the co-sited 2 x 2.
#include "hivc_internal.cuh"

namespace hivc {
namespace {

constexpr int kTW = 32, kTH = 8;

__device__ __forceinline__ int find_warp_job(const WarpJobs &J, int t)
{
    int j = 0;
    for (int k = 1; k < J.n; ++k)
        if (t >= J.p[k].tile_base) j = k;
    return j;
}

__device__ __forceinline__ void split_axis(float d, int x, int n, int &i0, float &a)
{
    float f = floorf(d);
    a = d - f;
    f = fminf(fmaxf(f, -2.0f * n - 4.0f), 2.0f * n + 4.0f);  // also maps NaN into range
    i0 = x + (int)f;
    if (i0 < 0) {
        i0 = 0;
        a = 0.f;
    } else if (i0 >= n - 1) {
        i0 = n > 1 ? n - 2 : 0;
        a = n > 1 ? 1.f : 0.f;
    }
}

__device__ __forceinline__ float sample(const float *__restrict__ R, int pitch, int W, int H, int x, int y, float dx,
                                        float dy)
{
    int x0, y0;
    float ax, ay;
    split_axis(dx, x, W, x0, ax);
    split_axis(dy, y, H, y0, ay);
    const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
    const float *r0 = R + (size_t)y0 * pitch, *r1 = R + (size_t)y1 * pitch;
    const float bx = 1.f - ax, by = 1.f - ay;
    return bx * by * __ldg(r0 + x0) + ax * by * __ldg(r0 + x1) + bx * ay * __ldg(r1 + x0) + ax * ay * __ldg(r1 + x1);
}

__global__ void __launch_bounds__(kTW *kTH) warp_add_kernel(const __grid_constant__ WarpJobs J)
{
    const int t = blockIdx.x;
    const WarpPlane &P = J.p[find_warp_job(J, t)];
    const int lt = t - P.tile_base;
    const int x = (lt % P.tiles_x) * kTW + (threadIdx.x & 31);
    const int y = (lt / P.tiles_x) * kTH + (threadIdx.x >> 5);
    if (x >= P.width || y >= P.height) return;
    float pred;
    if (P.ref != nullptr) {
        float dx, dy;
        const float2 *fl = reinterpret_cast<const float2 *>(P.flow);
        if (!P.chroma_flow) {
            const float2 f = __ldg(fl + (size_t)y * P.flow_w + x);
            dx = f.x;
            dy = f.y;
        } else {
            float sx = 0.f, sy = 0.f;
            int n = 0;
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int lx = 2 * x + a, ly = 2 * y + b;
                    if (lx < P.flow_w && ly < P.flow_h) {
                        const float2 f = __ldg(fl + (size_t)ly * P.flow_w + lx);
                        sx += f.x;
                        sy += f.y;
                        ++n;
                    }
                }
            const float s = n == 4 ? 0.125f : (n == 2 ? 0.25f : 0.5f);
            dx = sx * s;
            dy = sy * s;
        }
        pred = sample(P.ref, P.ref_pitch, P.width, P.height, x, y, dx, dy);
    } else {
        const size_t i = (size_t)y * P.src_pitch + x;
        const bool s1 = P.src_sel && *P.src_sel;  // which buffer of the ping-pong holds the solution
        const float *hi = s1 ? P.src_hi1 : P.src_hi, *lo = s1 ? P.src_lo1 : P.src_lo;
        pred = lo ? __fadd_rn(hi[i], lo[i]) : hi[i];
    }
    if (P.pred_out) P.pred_out[(size_t)y * P.pred_pitch + x] = pred;
    float v = pred;
    if (P.r) v += P.r[(size_t)y * P.r_pitch + x];
    v = fminf(fmaxf(v, 0.f), 255.f);
    if (P.ref_out) P.ref_out[(size_t)y * P.ref_out_pitch + x] = v;
    if (P.out) P.out[(size_t)y * P.out_pitch + x] = (uint8_t)__float2int_rd(v + 0.5f);
}

// 4:4:4 colour path (Sec. 2.3): the three RCT planes of a pixel together.
// The flow is read once and its interpolation weights serve all planes.
__global__ void __launch_bounds__(kTW *kTH) rct_kernel(const __grid_constant__ RctFrame F)
{
    const int x = blockIdx.x * kTW + (threadIdx.x & 31), y = blockIdx.y * kTH + (threadIdx.x >> 5);
    if (x >= F.width || y >= F.height) return;
    const size_t i = (size_t)y * F.pitch + x;
    float pred[3];
    if (F.flow) {
        const float2 f = __ldg(reinterpret_cast<const float2 *>(F.flow) + (size_t)y * F.width + x);
        int x0, y0;
        float ax, ay;
        split_axis(f.x, x, F.width, x0, ax);
        split_axis(f.y, y, F.height, y0, ay);
        const int x1 = min(x0 + 1, F.width - 1), y1 = min(y0 + 1, F.height - 1);
        const float bx = 1.f - ax, by = 1.f - ay;
        const size_t o00 = (size_t)y0 * F.pitch + x0, o01 = (size_t)y0 * F.pitch + x1;
        const size_t o10 = (size_t)y1 * F.pitch + x0, o11 = (size_t)y1 * F.pitch + x1;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const float *R = F.ref[p];
            pred[p] = bx * by * __ldg(R + o00) + ax * by * __ldg(R + o01) + bx * ay * __ldg(R + o10) +
                      ax * ay * __ldg(R + o11);
        }
    } else {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const bool s1 = F.src_sel && F.src_sel[p];  // which buffer of the ping-pong holds the solution
            const float *hi = s1 ? F.src_hi1[p] : F.src_hi[p], *lo = s1 ? F.src_lo1[p] : F.src_lo[p];
            pred[p] = lo ? __fadd_rn(hi[i], lo[i]) : hi[i];
        }
    }
    int q[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        float v = pred[p];
        if (F.r[p]) v += F.r[p][i];
        v = fminf(fmaxf(v, p == 0 ? 0.f : -255.f), 255.f);
        F.ref_out[p][i] = v;
        q[p] = __float2int_rd(v + 0.5f);
    }
    // inverse RCT: G = Y - floor((U + V) / 4), R = V + G, B = U + G
    const int G = q[0] - ((q[1] + q[2]) >> 2);  // arithmetic shift: floor for negative sums
    const int c[3] = {q[2] + G, G, q[1] + G};
#pragma unroll
    for (int p = 0; p < 3; ++p) F.out[p][(size_t)y * F.out_pitch[p] + x] = (uint8_t)min(max(c[p], 0), 255);
}

}  // namespace

cudaError_t launch_rct(const RctFrame &f, cudaStream_t st)
{
    const dim3 grid((f.width + kTW - 1) / kTW, (f.height + kTH - 1) / kTH);
    rct_kernel<<<grid, kTW * kTH, 0, st>>>(f);
    return cudaGetLastError();
}

cudaError_t launch_warp_add(WarpJobs &J, cudaStream_t st)
{
    int base = 0;
    for (int k = 0; k < J.n; ++k) {
        WarpPlane &P = J.p[k];
        P.tiles_x = (P.width + kTW - 1) / kTW;
        P.tile_base = base;
        base += P.tiles_x * ((P.height + kTH - 1) / kTH);
    }
    J.total_tiles = base;
    if (base == 0) return cudaSuccess;
    warp_add_kernel<<<base, kTW * kTH, 0, st>>>(J);
    return cudaGetLastError();
}

}  // namespace hivc
