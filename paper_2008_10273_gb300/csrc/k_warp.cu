// Inter prediction by backward warping (Sec. 2, Sec. 2.3) and the final
// correction step (prediction + residual, clamped to [0, 255]), plus the
// uint8 pack.  One launch covers all planes of a frame.
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
        pred = P.src_lo ? __fadd_rn(P.src_hi[i], P.src_lo[i]) : P.src_hi[i];
    }
    if (P.pred_out) P.pred_out[(size_t)y * P.pred_pitch + x] = pred;
    float v = pred;
    if (P.r) v += P.r[(size_t)y * P.r_pitch + x];
    v = fminf(fmaxf(v, 0.f), 255.f);
    if (P.ref_out) P.ref_out[(size_t)y * P.ref_out_pitch + x] = v;
    if (P.out) P.out[(size_t)y * P.out_pitch + x] = (uint8_t)__float2int_rd(v + 0.5f);
}

}  // namespace

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
