// Fused inter-frame kernel (Sec. 2, Sec. 2.2, Sec. 2.3): one CTA decodes a
// 32 x 32 luma macroblock and its 16 x 16 Cb and Cr tiles:
//   1. per residual block of the macroblock (one warp each): the evaluation
//      r = a + sum_j c_j G[p_j, :] (Eq. 3) into a shared-memory residual
//      tile, with r = v at the points; c and a come from the coefficient
//      stage (k_block.cu), launched before;
//   2. the backward bilinear warp of the previous reconstruction along the
//      transmitted flow (chroma flow = half the mean of the co-sited 2 x 2
//      luma vectors), + residual, clamp to [0, 255], the new FP32
//      reference and the uint8 output.
// The residual field never goes through global memory.
#include "block_device.cuh"

namespace hivc {
namespace {

constexpr int kMB = 32;  // luma macroblock edge
constexpr int kThreads = 128;

struct WarpScratch {
    float cs[2][256];
    unsigned char ps[256];
};

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

// bilinear sample of R (pitch floats) at (x + dx, y + dy), clamped
__device__ __forceinline__ float sample(const float *__restrict__ R, int pitch, int W, int H, int x, int y, float dx,
                                        float dy)
{
    float ax, ay;
    const int x0 = split_axis(dx, x, W, ax), y0 = split_axis(dy, y, H, ay);
    const int o0 = y0 * pitch + x0;
    const int ox = min(x0 + 1, W - 1) - x0, oy = min(y0 + 1, H - 1) > y0 ? pitch : 0;
    const float bx = 1.f - ax, by = 1.f - ay;
    return bx * by * __ldg(R + o0) + ax * by * __ldg(R + o0 + ox) + bx * ay * __ldg(R + o0 + oy) +
           ax * ay * __ldg(R + o0 + oy + ox);
}

// One residual block of the macroblock into its shared tile(s).
__device__ void mb_block(const BlockPlane &P, int lb, const BlockTables &tab, WarpScratch &S, float *tile0,
                         float *tile1, int tpitch, int ox, int oy, int lane, uint32_t *flags)
{
    const BlockGeom g = block_geom(P, lb);
    const int K = g.K, w = g.w, N = g.w * g.h;
    const bool two = P.val[1] != nullptr;
    bool valid = g.bad == 0;  // block_ptr / K errors are flagged by the coefficient stage
    for (int j0 = 0; j0 < K; j0 += 32) {
        int p = 0;
        const bool ok = (j0 + lane < K) ? load_pos(P, g, j0 + lane, p) : true;
        valid = valid && !__any_sync(0xffffffffu, !ok);
        if (j0 + lane < K) {
            S.ps[j0 + lane] = (unsigned char)p;
            S.cs[0][j0 + lane] = __ldg(P.coef[0] + g.s + j0 + lane);
            if (two) S.cs[1][j0 + lane] = __ldg(P.coef[1] + g.s + j0 + lane);
        }
    }
    __syncwarp();
    if (!valid || K == 0) {
        for (int i = lane; i < N; i += 32) {
            tile0[(oy + i / w) * tpitch + ox + i % w] = 0.f;
            if (two) tile1[(oy + i / w) * tpitch + ox + i % w] = 0.f;
        }
        __syncwarp();
        return;
    }
    const float a0 = __ldg(P.acoef[0] + g.lb), a1 = two ? __ldg(P.acoef[1] + g.lb) : 0.f;
    const float *G = green_rows(tab, g.w, g.h);
    auto out = [&](int x, int y, float v0, float v1) {
        const int o = (oy + y) * tpitch + ox + x;
        tile0[o] = v0;
        if (two) tile1[o] = v1;
    };
    if (two) warp_block_eval<true>(G, w, N, K, S.ps, S.cs[0], S.cs[1], a0, a1, lane, out);
    else warp_block_eval<false>(G, w, N, K, S.ps, S.cs[0], S.cs[1], a0, a1, lane, out);
    __syncwarp();
    for (int j = lane; j < K; j += 32) {
        const int o = (oy + S.ps[j] / w) * tpitch + ox + S.ps[j] % w;
        tile0[o] = (float)__ldg(P.val[0] + g.s + j);
        if (two) tile1[o] = (float)__ldg(P.val[1] + g.s + j);
    }
    __syncwarp();
}

template <bool CHROMA>
__global__ void __launch_bounds__(kThreads, 8) pframe_fused_kernel(const __grid_constant__ FusedFrame F, BlockTables tab,
                                                                uint32_t *flags)
{
    __shared__ float ry[kMB][kMB + 1];
    __shared__ float rc[2][kMB / 2][kMB / 2 + 1];
    __shared__ WarpScratch scr[kThreads / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int B = F.block;
    const int nl = kMB / B, nc = (kMB / 2) / B;  // blocks per macroblock side
    const int nlum = nl * nl, nchr = nc * nc;
    const int ntask = nlum + (CHROMA ? nchr * (F.nblk - 1) : 0);
    const int W = F.width, H = F.height, cw = (W + 1) / 2, chh = (H + 1) / 2;
    __shared__ int s_mb;
    for (;;) {
        // dynamic macroblock scheduling: the CTA grabs the next macroblock
        if (threadIdx.x == 0) s_mb = (int)atomicAdd(F.ctr + kCtrFusedWork, 1u);
        __syncthreads();
        const int mb = s_mb;
        if (mb >= F.nmb) break;
        const int mx = mb % F.nmbx, my = mb / F.nmbx;
        // ---- residual tiles ------------------------------------------------
        for (int t = warp; t < ntask; t += kThreads / 32) {
            if (t < nlum) {
                const BlockPlane &P = F.bp[0];
                const int bx = mx * nl + t % nl, by = my * nl + t / nl;
                if (bx * B >= W || by * B >= H) continue;
                mb_block(P, by * P.nbx + bx, tab, scr[warp], &ry[0][0], nullptr, kMB + 1, (t % nl) * B,
                         (t / nl) * B, lane, flags);
            } else {
                const int u = t - nlum, job = 1 + u / nchr, k = u % nchr;
                const BlockPlane &P = F.bp[job];
                const int bx = mx * nc + k % nc, by = my * nc + k / nc;
                if (bx * B >= cw || by * B >= chh) continue;
                float *t0 = &rc[job - 1][0][0];  // job 1: Cb (+ Cr when paired), job 2: Cr
                float *t1 = &rc[1][0][0];
                mb_block(P, by * P.nbx + bx, tab, scr[warp], t0, t1, kMB / 2 + 1, (k % nc) * B, (k / nc) * B, lane,
                         flags);
            }
        }
        __syncthreads();
        // ---- warp + residual + clamp + pack ----------------------------------
        const int x = threadIdx.x & 31, ty = threadIdx.x >> 5;
        const int gx = mx * kMB + x;
        const float2 *fl = reinterpret_cast<const float2 *>(F.flow);
        float2 f[4][2];
        bool in[4][2];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int gy = my * kMB + 2 * (ty + 4 * jj) + rr;
                in[jj][rr] = gx < W && gy < H;
                f[jj][rr] = in[jj][rr] ? __ldg(fl + gy * W + gx) : make_float2(0.f, 0.f);
            }
        float py[4][2];
        const float *ry0 = F.ref[0];
        const int yp = F.ref_pitch[0];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int gy = my * kMB + 2 * (ty + 4 * jj) + rr;
                py[jj][rr] = in[jj][rr] ? sample(ry0, yp, W, H, gx, gy, f[jj][rr].x, f[jj][rr].y) : 0.f;
            }
        // chroma: even lanes Cb, odd lanes Cr, one chroma column per lane pair
        const int cp = x & 1;
        const int cxg = mx * (kMB / 2) + (x >> 1);
        const float *rcp = cp ? F.ref[2] : F.ref[1];
        const int cpitch = cp ? F.ref_pitch[2] : F.ref_pitch[1];
        float pc[4];
        bool cin[4];
        if (CHROMA) {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                float sx = f[jj][0].x + f[jj][1].x, sy = f[jj][0].y + f[jj][1].y;
                int n = (int)in[jj][0] + (int)in[jj][1];
                sx += __shfl_xor_sync(0xffffffffu, sx, 1);
                sy += __shfl_xor_sync(0xffffffffu, sy, 1);
                n += __shfl_xor_sync(0xffffffffu, n, 1);
                const float sc = n == 4 ? 0.125f : (n == 2 ? 0.25f : 0.5f);
                const int cyg = my * (kMB / 2) + ty + 4 * jj;
                cin[jj] = cxg < cw && cyg < chh;
                pc[jj] = cin[jj] ? sample(rcp, cpitch, cw, chh, cxg, cyg, sx * sc, sy * sc) : 0.f;
            }
        }
        float *oy0 = F.ref_out[0];
        uint8_t *uy0 = F.out[0];
        const int op = F.out_pitch[0];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                if (!in[jj][rr]) continue;
                const int ly = 2 * (ty + 4 * jj) + rr, gy = my * kMB + ly;
                const float v = fminf(fmaxf(py[jj][rr] + ry[ly][x], 0.f), 255.f);
                oy0[gy * yp + gx] = v;
                uy0[gy * op + gx] = (uint8_t)__float2int_rd(v + 0.5f);
            }
        if (CHROMA) {
            float *ocp = cp ? F.ref_out[2] : F.ref_out[1];
            uint8_t *ucp = cp ? F.out[2] : F.out[1];
            const int uop = cp ? F.out_pitch[2] : F.out_pitch[1];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                if (!cin[jj]) continue;
                const int j = ty + 4 * jj, cyg = my * (kMB / 2) + j;
                const float v = fminf(fmaxf(pc[jj] + rc[cp][j][x >> 1], 0.f), 255.f);
                ocp[cyg * cpitch + cxg] = v;
                ucp[cyg * uop + cxg] = (uint8_t)__float2int_rd(v + 0.5f);
            }
        }
        __syncthreads();
    }
    // all threads left the loop after the same __syncthreads; the last CTA
    // clears the counters for the next frame
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(F.ctr + kCtrFusedDone, 1u) == gridDim.x - 1) {
            F.ctr[kCtrFusedWork] = 0;
            F.ctr[kCtrFusedDone] = 0;
            __threadfence();
        }
    }
}

template <bool CHROMA>
int fused_grid(const FusedFrame &F, int sms)
{
    static int per_sm[2] = {0, 0};
    int &o = per_sm[CHROMA ? 1 : 0];
    if (o == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, pframe_fused_kernel<CHROMA>, kThreads, 0) !=
                cudaSuccess ||
            o < 1)
            o = 1;
    }
    return std::max(1, std::min(F.nmb, sms * o));
}

}  // namespace

bool fused_supported(int block) { return block == 16 || block == 8; }

cudaError_t launch_pframe_fused(FusedFrame &F, uint32_t *flags, cudaStream_t st)
{
    F.nmbx = (F.width + kMB - 1) / kMB;
    F.nmb = F.nmbx * ((F.height + kMB - 1) / kMB);
    const BlockTables &t = block_tables();
    if (F.chroma)
        pframe_fused_kernel<true><<<fused_grid<true>(F, t.sms), kThreads, 0, st>>>(F, t, flags);
    else
        pframe_fused_kernel<false><<<fused_grid<false>(F, t.sms), kThreads, 0, st>>>(F, t, flags);
    return cudaGetLastError();
}

}  // namespace hivc
