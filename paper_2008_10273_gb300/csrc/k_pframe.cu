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
// comes from HBM about once.  Whole quads of even-width planes take 16-byte
// flow loads and issue all 24 bilinear samples before any store (about 12 %
// faster than a pixel at a time, same values); edge quads and odd widths go
// a pixel at a time.  (Variants that staged macroblock tiles of the flow and
// the references in shared memory with the tensor memory accelerator, and
// one that shared a 3 x 3 patch between the quad's samples, were not
// faster on this gather pattern.)
#include "block_device.cuh"
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

// bilinear interpolation of the corners r00, r01 (next column), r10 (next
// row), r11 with weights ax (columns) and ay (rows)
__device__ __forceinline__ float lerp2(float ax, float ay, float r00, float r01, float r10, float r11)
{
    const float top = fmaf(ax, r01 - r00, r00);
    const float bot = fmaf(ax, r11 - r10, r10);
    return fmaf(ay, bot - top, top);
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
    return lerp2(ax, ay, r00, r01, r10, r11);
}

// residual + prediction, clamped to [0, 255]: the new FP32 reference
__device__ __forceinline__ float recon(float pred, float r) { return fminf(fmaxf(pred + r, 0.f), 255.f); }
// the uint8 output (round half up)
__device__ __forceinline__ uint8_t to_u8(float v) { return (uint8_t)__float2int_rd(v + 0.5f); }

__device__ __forceinline__ void put_pixel(float pred, float r, float *ref_out, uint8_t *out)
{
    const float v = recon(pred, r);
    *ref_out = v;
    *out = to_u8(v);
}

constexpr int kQX = 32, kQY = 4;  // quads per CTA: 32 x 4 (128 threads)

// A whole quad of an even-width plane with 8-byte aligned rows (the host
// checks pointers and pitches): the quad's flow as two 16-byte loads, its
// luma residual as two 8-byte loads, and every bilinear sample of the quad
// (16 luma, 8 chroma) issued before any store, so that they are in flight
// together; the new reference and the output go out as row pairs.  The
// arithmetic is the scalar path's, value for value.
// The residual of the quad comes from res(r, rc), called after the flow
// loads: r the four luma pixels row by row, rc the Cb and Cr pixels.
template <bool CHROMA, class Res>
__device__ __forceinline__ void whole_quad_r(const InterFrame &F, int qx, int qy, const Res &res)
{
    const int W = F.width, H = F.height;
    const int x0 = 2 * qx, y0 = 2 * qy;
    const int yp = F.ref_pitch[0], op = F.out_pitch[0];
    const float4 *fl = reinterpret_cast<const float4 *>(F.flow + 2 * (y0 * W + x0));
    const float4 fa = __ldcs(fl), fb = __ldcs(fl + W / 2);  // read once: evict first
    const float2 f[4] = {make_float2(fa.x, fa.y), make_float2(fa.z, fa.w), make_float2(fb.x, fb.y),
                         make_float2(fb.z, fb.w)};
    float r[4], rc[2] = {0.f, 0.f};
    res(r, rc);
    const float *__restrict__ RY = F.ref[0];
    float ax[4], ay[4], g[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int sx = split_axis(f[k].x, x0 + (k & 1), W, ax[k]);
        const int sy = split_axis(f[k].y, y0 + (k >> 1), H, ay[k]);
        const int ox = min(sx + 1, W - 1) - sx, oy = (min(sy + 1, H - 1) - sy) * yp;
        const int o = sy * yp + sx;
        g[k][0] = __ldg(RY + o);
        g[k][1] = __ldg(RY + o + ox);
        g[k][2] = __ldg(RY + o + oy);
        g[k][3] = __ldg(RY + o + oy + ox);
    }
    float cax = 0.f, cay = 0.f, c[2][4];
    int cp = 0;
    if (CHROMA) {
        const int cw = (W + 1) / 2, ch = (H + 1) / 2;
        const float dx = ((f[0].x + f[1].x) + (f[2].x + f[3].x)) * 0.125f;
        const float dy = ((f[0].y + f[1].y) + (f[2].y + f[3].y)) * 0.125f;
        const int cx0 = split_axis(dx, qx, cw, cax), cy0 = split_axis(dy, qy, ch, cay);
        cp = F.ref_pitch[1];
        const int cox = min(cx0 + 1, cw - 1) - cx0, coy = (min(cy0 + 1, ch - 1) - cy0) * cp;
        const int co = cy0 * cp + cx0;
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
            const float *__restrict__ R = F.ref[pl + 1];
            c[pl][0] = __ldg(R + co);
            c[pl][1] = __ldg(R + co + cox);
            c[pl][2] = __ldg(R + co + coy);
            c[pl][3] = __ldg(R + co + coy + cox);
        }
    }
    float v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = recon(lerp2(ax[k], ay[k], g[k][0], g[k][1], g[k][2], g[k][3]), r[k]);
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        *reinterpret_cast<float2 *>(F.ref_out[0] + (y0 + rr) * yp + x0) = make_float2(v[2 * rr], v[2 * rr + 1]);
        __stcs(reinterpret_cast<uchar2 *>(F.out[0] + (y0 + rr) * op + x0),
               make_uchar2(to_u8(v[2 * rr]), to_u8(v[2 * rr + 1])));
    }
    if (CHROMA) {
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
            const float cv = recon(lerp2(cax, cay, c[pl][0], c[pl][1], c[pl][2], c[pl][3]), rc[pl]);
            F.ref_out[pl + 1][qy * cp + qx] = cv;
            __stcs(reinterpret_cast<char *>(F.out[pl + 1] + qy * F.out_pitch[pl + 1] + qx), (char)to_u8(cv));
        }
    }
}

// (the residual from the residual planes; early: the preceding grid is
// waited for only here, after the flow and residual loads are issued)
template <bool CHROMA>
__device__ __forceinline__ void whole_quad(const InterFrame &F, int qx, int qy, bool early)
{
    whole_quad_r<CHROMA>(F, qx, qy, [&](float (&r)[4], float (&rc)[2]) {
        const int x0 = 2 * qx, y0 = 2 * qy, rp = F.r_pitch[0];
        const float2 *rr0 = reinterpret_cast<const float2 *>(F.r[0] + y0 * rp + x0);
        const float2 rl0 = __ldcs(rr0), rl1 = __ldcs(rr0 + rp / 2);
        r[0] = rl0.x;
        r[1] = rl0.y;
        r[2] = rl1.x;
        r[3] = rl1.y;
        if (CHROMA) {
            rc[0] = __ldcs(F.r[1] + qy * F.r_pitch[1] + qx);
            rc[1] = __ldcs(F.r[2] + qy * F.r_pitch[2] + qx);
        }
        if (early) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        }
    });
}

// Any quad (cut by the right or bottom edge, odd widths, unaligned rows):
// one pixel at a time.
template <bool CHROMA>
__device__ __forceinline__ void any_quad(const InterFrame &F, int qx, int qy)
{
    const int W = F.width, H = F.height;
    const int x0 = 2 * qx, y0 = 2 * qy;
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
                      F.ref_out[pl] + (size_t)qy * F.ref_pitch[pl] + qx,
                      F.out[pl] + (size_t)qy * F.out_pitch[pl] + qx);
        }
    }
}

// early: the preceding grid is the previous frame's pixel kernel, which
// itself waited for the residual planes; the flow and the residual planes
// are then loaded before waiting for it (they do not depend on it), so
// that the first CTAs of this frame fill the SMs that the previous frame's
// last wave leaves idle.  Otherwise the preceding launch wrote the
// residual planes, and every read waits for it.
template <bool CHROMA>
__global__ void __launch_bounds__(kQX *kQY, 12) pframe_kernel(const __grid_constant__ InterFrame F, int vec,
                                                               int early)
{
    if (!early) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    const int qx = blockIdx.x * kQX + threadIdx.x, qy = blockIdx.y * kQY + threadIdx.y;
    if (2 * qx >= F.width || 2 * qy >= F.height) return;
    if (vec && 2 * qy + 1 < F.height) {
        whole_quad<CHROMA>(F, qx, qy, early != 0);
    } else {
        if (early) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        }
        any_quad<CHROMA>(F, qx, qy);
    }
}


// ---- the fused kernel: residual evaluation and pixels of a frame ----------
// A CTA takes a 32 x 32 luma macroblock.  Warp w takes the 16 x 16 luma
// block (2 mbx + (w & 1), 2 mby + (w >> 1)) and the quarter of the chroma
// block (mbx, mby) co-sited with it.  Phase 1 evaluates Eq. 3 for the
// warp's pixels into shared memory with the evaluation kernel's arithmetic
// (r = a, then r = fma(c_j, G[p_j, q], r) in the order of the points, the
// Green's rows as 16-byte loads, then the data at the points exactly; bad
// positions give a zero block and a flag).  Phase 2 is the pixel kernel's
// whole-quad path with the residual read from shared memory: lane l takes
// the two quads of luma rows 2 (l / 4) + {0, 1}, columns 4 (l % 4) .. + 3.
// The values equal those of the evaluation kernel followed by
// pframe_kernel, bit for bit; the residual planes never reach memory.
// Opt-in: on a GB300 it takes about 36 us per FullHD 4:2:0 frame against
// 15 us for pframe_kernel plus 8 us of batched evaluation.  A warp runs
// its latency-bound evaluation and then its gathers, and with two quads a
// lane and 32 warps an SM it keeps fewer samples in flight than
// pframe_kernel's one quad a thread and 48 warps.
constexpr int kFusedWarps = 4;

constexpr int kFusedRow = 20;  // luma row stride: the quads' reads spread over the banks
struct __align__(16) FusedRes {
    float y[16][kFusedRow];  // the luma block
    float c[2][8][8];        // the Cb and Cr quarter
};

// Eq. 3 for the luma block lb of job P into R.
__device__ __forceinline__ void fused_luma(const BlockPlane &P, const BlockTables &tab, int lb,
                                           float (*R)[kFusedRow], int lane, uint32_t *flags)
{
    const BlockGeom g = block_geom(P, lb);
    const float a0 = __ldcg(P.acoef[0] + lb);
    const int K = g.K, w = g.w, N = g.w * g.h, rl = g_rowlen(N);
    const float *__restrict__ G = green_rows(tab, g.w, g.h);
    const int q0 = 4 * lane, q1 = 128 + 4 * lane;
    const bool act = q0 < N, act1 = q1 < N;
    float r0[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) r0[t] = a0;
    bool valid = K > 0;
    int prev = -1;
    for (int j0 = 0; j0 < K; j0 += 32) {
        const int j = j0 + lane;
        int p = 0;
        float c0 = 0.f;
        if (j < K) {
            p = __ldg(P.pos + g.s + j);
            c0 = __ldcg(P.coef[0] + g.s + j);
        }
        const int up = __shfl_up_sync(0xffffffffu, p, 1);
        const int before = lane == 0 ? prev : up;
        if (__any_sync(0xffffffffu, j < K && (p >= N || p <= before))) valid = false;
        prev = __shfl_sync(0xffffffffu, p, 31);
        if (!valid) break;
        const int n = min(32, K - j0);
        const float *Gq = G + q0;
#pragma unroll 4
        for (int u = 0; u < n; ++u) {
            const float cu = __shfl_sync(0xffffffffu, c0, u);
            const int pu = __shfl_sync(0xffffffffu, p, u);
            if (act) {
                const float *row = Gq + pu * rl;
                const float4 lo = __ldg(reinterpret_cast<const float4 *>(row));
                const float4 hi = act1 ? __ldg(reinterpret_cast<const float4 *>(row + 128)) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float gv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
                for (int t = 0; t < 8; ++t) r0[t] = fmaf(cu, gv[t], r0[t]);
            }
        }
    }
    if (!valid) {
        if (K > 0 && lane == 0 && flags) atomicOr(flags, kFlagPos);
#pragma unroll
        for (int t = 0; t < 8; ++t) r0[t] = 0.f;
    }
    if (w == 16) {
        // pixels 4l .. 4l+3 are columns 4 (l % 4) .. +3 of row l / 4, the
        // second half the same columns of row 8 + l / 4
        if (act) *reinterpret_cast<float4 *>(&R[lane >> 2][4 * (lane & 3)]) = make_float4(r0[0], r0[1], r0[2], r0[3]);
        if (act1)
            *reinterpret_cast<float4 *>(&R[8 + (lane >> 2)][4 * (lane & 3)]) = make_float4(r0[4], r0[5], r0[6], r0[7]);
    } else {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int q = (t < 4 ? q0 : q1 - 4) + t;
            if (q < N) {
                const int y = q / w;
                R[y][q - y * w] = r0[t];
            }
        }
    }
    if (!valid) return;
    __syncwarp();
    // the data at the points, exactly
    for (int j = lane; j < K; j += 32) {
        const int p = __ldg(P.pos + g.s + j), y = p / w;
        R[y][p - y * w] = (float)__ldg(P.val[0] + g.s + j);
    }
}

// Eq. 3 for the quarter (qx0, qy0) + [0, 8)^2 of chroma block cb of job P
// into R[0] (values and coefficients [0]) and, TWO, R[1] ([1]).  Lane l
// takes the quarter's pixels (2 (l % 4) + {0, 1}, l / 4).
template <bool TWO>
__device__ __forceinline__ void fused_chroma(const BlockPlane &P, const BlockTables &tab, int cb, int qx0, int qy0,
                                             float (*R0)[8], float (*R1)[8], int lane, uint32_t *flags)
{
    const BlockGeom g = block_geom(P, cb);
    const float a0 = __ldcg(P.acoef[0] + cb), a1 = TWO ? __ldcg(P.acoef[1] + cb) : 0.f;
    const int K = g.K, w = g.w, N = g.w * g.h, rl = g_rowlen(N);
    const float *__restrict__ G = green_rows(tab, g.w, g.h);
    const int ly = lane >> 2, lx = 2 * (lane & 3);
    const int cy = qy0 + ly, cx = qx0 + lx;
    const bool in0 = cy < g.h && cx < w, in1 = cy < g.h && cx + 1 < w;
    const int qa = cy * w + cx;
    float r0[2] = {a0, a0}, r1[2] = {a1, a1};
    bool valid = K > 0;
    int prev = -1;
    for (int j0 = 0; j0 < K; j0 += 32) {
        const int j = j0 + lane;
        int p = 0;
        float c0 = 0.f, c1 = 0.f;
        if (j < K) {
            p = __ldg(P.pos + g.s + j);
            c0 = __ldcg(P.coef[0] + g.s + j);
            if (TWO) c1 = __ldcg(P.coef[1] + g.s + j);
        }
        const int up = __shfl_up_sync(0xffffffffu, p, 1);
        const int before = lane == 0 ? prev : up;
        if (__any_sync(0xffffffffu, j < K && (p >= N || p <= before))) valid = false;
        prev = __shfl_sync(0xffffffffu, p, 31);
        if (!valid) break;
        const int n = min(32, K - j0);
#pragma unroll 4
        for (int u = 0; u < n; ++u) {
            const float cu0 = __shfl_sync(0xffffffffu, c0, u);
            const float cu1 = TWO ? __shfl_sync(0xffffffffu, c1, u) : 0.f;
            const int pu = __shfl_sync(0xffffffffu, p, u);
            const float *row = G + pu * rl + qa;
            const float g0 = in0 ? __ldg(row) : 0.f, g1 = in1 ? __ldg(row + 1) : 0.f;
            r0[0] = fmaf(cu0, g0, r0[0]);
            r0[1] = fmaf(cu0, g1, r0[1]);
            if (TWO) {
                r1[0] = fmaf(cu1, g0, r1[0]);
                r1[1] = fmaf(cu1, g1, r1[1]);
            }
        }
    }
    if (!valid) {
        if (K > 0 && lane == 0 && flags) atomicOr(flags, kFlagPos);
        r0[0] = r0[1] = r1[0] = r1[1] = 0.f;
    }
    R0[ly][lx] = r0[0];
    R0[ly][lx + 1] = r0[1];
    if (TWO) {
        R1[ly][lx] = r1[0];
        R1[ly][lx + 1] = r1[1];
    }
    if (!valid) return;
    __syncwarp();
    for (int j = lane; j < K; j += 32) {
        const int p = __ldg(P.pos + g.s + j), y = p / w, x = p - y * w;
        if (y < qy0 || y >= qy0 + 8 || x < qx0 || x >= qx0 + 8) continue;
        R0[y - qy0][x - qx0] = (float)__ldg(P.val[0] + g.s + j);
        if (TWO) R1[y - qy0][x - qx0] = (float)__ldg(P.val[1] + g.s + j);
    }
}

// NC: chroma jobs (0 grey, 1 paired Cb + Cr, 2 separate)
template <int NC>
__global__ void __launch_bounds__(32 * kFusedWarps, 8)
    pframe_fused_kernel(const __grid_constant__ FusedFrame F, const __grid_constant__ BlockTables tab)
{
    constexpr bool CHROMA = NC > 0;
    __shared__ FusedRes sres[kFusedWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = 2 * blockIdx.x + (warp & 1), by = 2 * blockIdx.y + (warp >> 1);
    const int W = F.px.width, H = F.px.height;
    const bool inside = 16 * bx < W && 16 * by < H;
    // with early, the preceding grid waited for its own predecessor before
    // it let this one start, so the block stage's coefficients are complete
    if (!F.early) asm volatile("griddepcontrol.wait;" ::: "memory");
    FusedRes &R = sres[warp];
    if (inside) {
        fused_luma(F.y, tab, by * F.y.nbx + bx, R.y, lane, F.flags);
        if (CHROMA) {
            const int cb = (by >> 1) * F.c[0].nbx + (bx >> 1), qx0 = 8 * (bx & 1), qy0 = 8 * (by & 1);
            if (NC == 1) {
                fused_chroma<true>(F.c[0], tab, cb, qx0, qy0, R.c[0], R.c[1], lane, F.flags);
            } else {
                fused_chroma<false>(F.c[0], tab, cb, qx0, qy0, R.c[0], nullptr, lane, F.flags);
                fused_chroma<false>(F.c[1], tab, cb, qx0, qy0, R.c[1], nullptr, lane, F.flags);
            }
        }
    }
    // the preceding frame's references are read from here on
    if (F.early) asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (!inside) return;
    __syncwarp();
    const int i = lane >> 2, j = lane & 3;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int qx = 8 * bx + 2 * j + k, qy = 8 * by + i;
        if (2 * qx >= W || 2 * qy >= H) continue;
        whole_quad_r<CHROMA>(F.px, qx, qy, [&](float (&r)[4], float (&rc)[2]) {
            const int cx = 4 * j + 2 * k;
            r[0] = R.y[2 * i][cx];
            r[1] = R.y[2 * i][cx + 1];
            r[2] = R.y[2 * i + 1][cx];
            r[3] = R.y[2 * i + 1][cx + 1];
            if (CHROMA) {
                rc[0] = R.c[0][i][2 * j + k];
                rc[1] = R.c[1][i][2 * j + k];
            }
        });
    }
}

}  // namespace

cudaError_t launch_pframe(const InterFrame &F, cudaStream_t st, bool pdl, bool early)
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
    // the whole-quad path: an even width (16-byte flow pairs), even pitches
    // and 8-byte (flow: 16-byte) aligned planes
    auto al = [](const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; };
    bool vec = F.width % 2 == 0 && al(F.flow, 16) && F.ref_pitch[0] % 2 == 0 && F.r_pitch[0] % 2 == 0 &&
               F.out_pitch[0] % 2 == 0 && al(F.ref[0], 8) && al(F.ref_out[0], 8) && al(F.r[0], 8) &&
               al(F.out[0], 2);
    const int vi = vec ? 1 : 0, ei = early ? 1 : 0;
    if (F.chroma) return cudaLaunchKernelEx(&cfg, pframe_kernel<true>, F, vi, ei);
    return cudaLaunchKernelEx(&cfg, pframe_kernel<false>, F, vi, ei);
}

namespace {
bool whole_quads_ok(const InterFrame &F)
{
    auto al = [](const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; };
    return F.width % 2 == 0 && al(F.flow, 16) && F.ref_pitch[0] % 2 == 0 && F.r_pitch[0] % 2 == 0 &&
           F.out_pitch[0] % 2 == 0 && al(F.ref[0], 8) && al(F.ref_out[0], 8) && al(F.r[0], 8) && al(F.out[0], 2);
}
}  // namespace

bool pframe_fused_ok(const InterFrame &F, int block)
{
    InterFrame G = F;
    G.r_pitch[0] = 2;  // no residual planes
    G.r[0] = F.ref[0];
    return (F.chroma == 0 || F.chroma == 1) && block == 16 && F.width % 2 == 0 && F.height % 2 == 0 &&
           whole_quads_ok(G);
}

cudaError_t launch_pframe_fused(const FusedFrame &f, cudaStream_t st, bool pdl)
{
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    const int nbx = (f.px.width + 15) / 16, nby = (f.px.height + 15) / 16;
    cfg.gridDim = dim3((nbx + 1) / 2, (nby + 1) / 2);
    cfg.blockDim = dim3(32 * kFusedWarps);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const BlockTables tab = block_tables(f.op);
    if (f.px.chroma == 0) return cudaLaunchKernelEx(&cfg, pframe_fused_kernel<0>, f, tab);
    if (f.nc == 1) return cudaLaunchKernelEx(&cfg, pframe_fused_kernel<1>, f, tab);
    return cudaLaunchKernelEx(&cfg, pframe_fused_kernel<2>, f, tab);
}

}  // namespace hivc
