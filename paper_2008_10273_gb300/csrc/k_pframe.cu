// Inter-frame pixel kernel (Sec. 2, Sec. 2.3): the backward bilinear warp
// of the previous reconstruction along the transmitted flow (4:2:0 chroma
// flow = half the mean of the co-sited 2 x 2 luma vectors), + the residual
// planes that the block kernels evaluated (Eq. 3), clamped to [0, 255]: the
// new FP32 reference and the uint8 output.
//
// Thread (qx, qy) takes the luma quad at columns 2 qx, 2 qx + 1 and rows
// 2 qy, 2 qy + 1 and, with chroma, the co-sited pixel (qx, qy) of Cb and
// Cr.  Every access is a coalesced global load or store: the reference
// samples of neighbouring threads share cache lines, so each reference line
// comes from HBM about once.  (Variants that staged macroblock tiles of the
// flow and the references in shared memory with the tensor memory
// accelerator measured slower on this gather pattern.)
#include "hivc_internal.cuh"

namespace hivc {
namespace {

// Integer part and fraction of one sample coordinate x + d, clamped to the
// plane [0, n-1]: returns i0 in [0, max(n-2, 0)] and the weight a of i0+1.
// floor(d) and d - floor(d) are exact, so the weight does not lose bits to
// the pixel coordinate; NaN flow samples the plane edge.
__device__ __forceinline__ int split_axis(float d, int x, int n, float &a)
{
    const float f = floorf(d);
    a = d - f;
    int i0 = x + __float2int_rn(fminf(fmaxf(f, -32768.f), 32768.f));
    a = i0 < 0 ? 0.f : (i0 >= n - 1 ? 1.f : a);
    return max(min(i0, n - 2), 0);
}

// bilinear sample of R at (x + dx, y + dy), sample position clamped
__device__ __forceinline__ float sample(const float *__restrict__ R, int pitch, int W, int H, int x, int y, float dx,
                                        float dy)
{
    float ax, ay;
    const int x0 = split_axis(dx, x, W, ax), y0 = split_axis(dy, y, H, ay);
    const int ox = min(x0 + 1, W - 1) - x0, oyn = min(y0 + 1, H - 1) - y0;
    const float *g = R + (size_t)y0 * pitch + x0;
    const float r00 = __ldg(g), r01 = __ldg(g + ox), r10 = __ldg(g + (size_t)oyn * pitch),
                r11 = __ldg(g + (size_t)oyn * pitch + ox);
    const float top = fmaf(ax, r01 - r00, r00);
    const float bot = fmaf(ax, r11 - r10, r10);
    return fmaf(ay, bot - top, top);
}

// residual + prediction, clamped to [0, 255]: the new FP32 reference and
// the uint8 output (round half up)
__device__ __forceinline__ void put_pixel(float pred, float r, float *ref_out, uint8_t *out)
{
    const float v = fminf(fmaxf(pred + r, 0.f), 255.f);
    *ref_out = v;
    *out = (uint8_t)__float2int_rd(v + 0.5f);
}

constexpr int kQX = 32, kQY = 4;  // quads per CTA: 32 x 4 (128 threads)

template <bool CHROMA>
__global__ void __launch_bounds__(kQX *kQY) pframe_kernel(const __grid_constant__ InterFrame F)
{
    // the preceding launch wrote the residual planes or the references
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int qx = blockIdx.x * kQX + threadIdx.x, qy = blockIdx.y * kQY + threadIdx.y;
    const int W = F.width, H = F.height;
    const int x0 = 2 * qx, y0 = 2 * qy;
    if (x0 >= W || y0 >= H) return;
    const bool in1 = x0 + 1 < W, inr = y0 + 1 < H;
    const float2 *fl = reinterpret_cast<const float2 *>(F.flow);
    float2 f[4];  // (row, column): 00, 01, 10, 11; zero outside the plane
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const bool rin = rr == 0 || inr;
        const float2 *row = fl + (size_t)(y0 + rr) * W + x0;
        f[2 * rr] = rin ? __ldg(row) : make_float2(0.f, 0.f);
        f[2 * rr + 1] = (rin && in1) ? __ldg(row + 1) : make_float2(0.f, 0.f);
    }
    const int yp = F.ref_pitch[0], op = F.out_pitch[0], rp = F.r_pitch[0];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = x0 + (q & 1), y = y0 + (q >> 1);
        if (!((q & 1) == 0 || in1) || !((q >> 1) == 0 || inr)) continue;
        const float pred = sample(F.ref[0], yp, W, H, x, y, f[q].x, f[q].y);
        put_pixel(pred, __ldg(F.r[0] + (size_t)y * rp + x), F.ref_out[0] + (size_t)y * yp + x,
                  F.out[0] + (size_t)y * op + x);
    }
    if (CHROMA) {
        // half the mean of the in-plane vectors of the quad
        const int cw = (W + 1) / 2, ch = (H + 1) / 2;
        const int n = (1 + (int)in1) * (1 + (int)inr);
        const float sc = n == 4 ? 0.125f : (n == 2 ? 0.25f : 0.5f);
        const float dx = ((f[0].x + f[1].x) + (f[2].x + f[3].x)) * sc;
        const float dy = ((f[0].y + f[1].y) + (f[2].y + f[3].y)) * sc;
#pragma unroll
        for (int pl = 1; pl < 3; ++pl) {
            const float pred = sample(F.ref[pl], F.ref_pitch[pl], cw, ch, qx, qy, dx, dy);
            put_pixel(pred, __ldg(F.r[pl] + (size_t)qy * F.r_pitch[pl] + qx),
                      F.ref_out[pl] + (size_t)qy * F.ref_pitch[pl] + qx, F.out[pl] + (size_t)qy * F.out_pitch[pl] + qx);
        }
    }
}

}  // namespace

cudaError_t launch_pframe(const InterFrame &F, cudaStream_t st, bool pdl)
{
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    const int qw = (F.width + 1) / 2, qh = (F.height + 1) / 2;
    cfg.gridDim = dim3((qw + kQX - 1) / kQX, (qh + kQY - 1) / kQY);
    cfg.blockDim = dim3(kQX, kQY);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (F.chroma) return cudaLaunchKernelEx(&cfg, pframe_kernel<true>, F);
    return cudaLaunchKernelEx(&cfg, pframe_kernel<false>, F);
}

}  // namespace hivc
