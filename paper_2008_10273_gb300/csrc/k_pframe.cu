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
//
// TMA variant: a persistent CTA takes macroblocks from a work counter and,
// while it evaluates the residual of one macroblock, the tensor memory
// accelerator copies the next macroblock's flow tile and its reference
// tiles (with an 8-pixel luma / 4-pixel chroma halo) into a second shared
// stage.  Samples that leave the halo read global memory.  The kernel is
// launched with programmatic dependent launch: the first copies overlap the
// coefficient kernel, and griddepcontrol.wait orders the coefficient reads.
#include <cuda.h>

#include "block_device.cuh"

namespace hivc {
namespace {

constexpr int kMB = 32;  // luma macroblock edge
constexpr int kThreads = 128;
constexpr int kHalo = 8, kTL = kMB + 2 * kHalo;        // luma reference tile 48 x 48
constexpr int kCHalo = 4, kTC = kMB / 2 + 2 * kCHalo;  // chroma reference tile 24 x 24
constexpr long kMbarSpins = 1L << 22;                  // bounded waits

struct WarpScratch {
    float cs[2][256];
    unsigned char ps[256];
};

struct __align__(128) Stage {
    float flow[kMB][2 * kMB];  // 32 rows of 32 (dx, dy)
    float ry[kTL][kTL];
    float rc[2][kTC][kTC];
};

struct Tiles {
    float ry[kMB][kMB + 1];
    float rc[2][kMB / 2][kMB / 2 + 1];
    WarpScratch scr[kThreads / 32];
};

constexpr size_t kTmaSmem = sizeof(Stage) + sizeof(Tiles) + 64;

// ---- PTX helpers (TMA, mbarrier, programmatic dependent launch) ----------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false when the copies did not land within the limit
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (long i = 0; i < kMbarSpins; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- sampling ------------------------------------------------------------
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

// bilinear sample at (x + dx, y + dy), clamped; from the staged tile (origin
// tx0, ty0, edge T) when the 2 x 2 footprint lies in it, else from R
template <int T>
__device__ __forceinline__ float sample(const float *__restrict__ R, int pitch, int W, int H, int x, int y, float dx,
                                        float dy, const float *tile, int tx0, int ty0)
{
    float ax, ay;
    const int x0 = split_axis(dx, x, W, ax), y0 = split_axis(dy, y, H, ay);
    const int ox = min(x0 + 1, W - 1) - x0, oyn = min(y0 + 1, H - 1) - y0;
    const float bx = 1.f - ax, by = 1.f - ay;
    float r00, r01, r10, r11;
    const int lx = x0 - tx0, ly = y0 - ty0;
    if (T > 0 && (unsigned)lx < (unsigned)(T - 1) && (unsigned)ly < (unsigned)(T - 1)) {
        const float *t = tile + ly * T + lx;
        r00 = t[0];
        r01 = t[ox];
        r10 = t[oyn * T];
        r11 = t[oyn * T + ox];
    } else {
        const float *g = R + y0 * pitch + x0;
        r00 = __ldg(g);
        r01 = __ldg(g + ox);
        r10 = __ldg(g + oyn * pitch);
        r11 = __ldg(g + oyn * pitch + ox);
    }
    return bx * by * r00 + ax * by * r01 + bx * ay * r10 + ax * ay * r11;
}

// ---- residual tiles ------------------------------------------------------
// One residual block of the macroblock into its shared tile(s).
__device__ void mb_block(const BlockPlane &P, int lb, const BlockTables &tab, WarpScratch &S, float *tile0,
                         float *tile1, int tpitch, int ox, int oy, int lane)
{
    const BlockGeom g = block_geom(P, lb);
    const int K = g.K, w = g.w, N = g.w * g.h;
    const bool two = P.val[1] != nullptr;
    bool valid = g.bad == 0;  // errors are flagged by the coefficient stage
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
            const int y = i / w, x = i - y * w;
            tile0[(oy + y) * tpitch + ox + x] = 0.f;
            if (two) tile1[(oy + y) * tpitch + ox + x] = 0.f;
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
__device__ __forceinline__ void mb_residual(const FusedFrame &F, const BlockTables &tab, Tiles &tl, int mx, int my,
                                            int warp, int lane)
{
    const int B = F.block;
    const int nl = kMB / B, nc = (kMB / 2) / B;  // blocks per macroblock side
    const int nlum = nl * nl, nchr = nc * nc;
    const int ntask = nlum + (CHROMA ? nchr * (F.nblk - 1) : 0);
    const int W = F.width, H = F.height, cw = (W + 1) / 2, chh = (H + 1) / 2;
    for (int t = warp; t < ntask; t += kThreads / 32) {
        if (t < nlum) {
            const BlockPlane &P = F.bp[0];
            const int bx = mx * nl + t % nl, by = my * nl + t / nl;
            if (bx * B >= W || by * B >= H) continue;
            mb_block(P, by * P.nbx + bx, tab, tl.scr[warp], &tl.ry[0][0], nullptr, kMB + 1, (t % nl) * B,
                     (t / nl) * B, lane);
        } else {
            const int u = t - nlum, job = 1 + u / nchr, k = u % nchr;
            const BlockPlane &P = F.bp[job];
            const int bx = mx * nc + k % nc, by = my * nc + k / nc;
            if (bx * B >= cw || by * B >= chh) continue;
            // job 1: Cb (+ Cr when paired), job 2: Cr
            mb_block(P, by * P.nbx + bx, tab, tl.scr[warp], &tl.rc[job - 1][0][0], &tl.rc[1][0][0], kMB / 2 + 1,
                     (k % nc) * B, (k / nc) * B, lane);
        }
    }
}

// bilinear sample from a staged tile at tile coordinates (lx + fx, ly + fy),
// fraction (ax, ay); the caller checked that the 2 x 2 footprint is inside
template <int T>
__device__ __forceinline__ float tile_lerp(const float *tile, int lx, int ly, float ax, float ay)
{
    const float *t = tile + ly * T + lx;
    const float top = fmaf(ax, t[1] - t[0], t[0]);
    const float bot = fmaf(ax, t[T + 1] - t[T], t[T]);
    return fmaf(ay, bot - top, top);
}

struct PixelCtx {
    int W, H, cw, chh, yp, op;
    const float *ry0;
    float *oy0;
    uint8_t *uy0;
    const float *rcp;
    float *ocp;
    uint8_t *ucp;
    int cpitch, uop;
};

// warp + residual + clamp + pack of one macroblock; st = staged tiles or null
template <bool CHROMA>
__device__ __forceinline__ void mb_pixels(const PixelCtx &c, const Tiles &tl, const Stage *st, int mx, int my,
                                          const float2 *__restrict__ fl)
{
    const int W = c.W, H = c.H;
    const int x = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int gx = mx * kMB + x;
    const int tx0 = mx * kMB - kHalo, ty0 = my * kMB - kHalo;
    // tile-coordinate window in which a sample needs neither the plane
    // clamp nor global memory: the tile interior, intersected with the plane
    const int lx_lo = max(0, -tx0), lx_hi = min(kTL - 2, W - 2 - tx0);
    const int ly_lo = max(0, -ty0), ly_hi = min(kTL - 2, H - 2 - ty0);
    const int cp = x & 1;
    const int cxg = mx * (kMB / 2) + (x >> 1);
    const int cx0 = mx * (kMB / 2) - kCHalo, cy0 = my * (kMB / 2) - kCHalo;
    const int cx_lo = max(0, -cx0), cx_hi = min(kTC - 2, c.cw - 2 - cx0);
    const int cy_lo = max(0, -cy0), cy_hi = min(kTC - 2, c.chh - 2 - cy0);
#pragma unroll 2
    for (int jj = 0; jj < 4; ++jj) {
        float2 f[2];
        bool in[2];
        float py[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int ly = 2 * (ty + 4 * jj) + rr, gy = my * kMB + ly;
            in[rr] = gx < W && gy < H;
            if (st) f[rr] = make_float2(st->flow[ly][2 * x], st->flow[ly][2 * x + 1]);
            else f[rr] = in[rr] ? __ldg(fl + gy * W + gx) : make_float2(0.f, 0.f);
            // fast path: the footprint lies in the staged tile and the plane
            const float fx = floorf(f[rr].x), fy = floorf(f[rr].y);
            const float ax = f[rr].x - fx, ay = f[rr].y - fy;
            const int lx = x + kHalo + __float2int_rn(fx), lyy = ly + kHalo + __float2int_rn(fy);
            const bool fast = st != nullptr && lx >= lx_lo && lx <= lx_hi && lyy >= ly_lo && lyy <= ly_hi &&
                              ax == ax && ay == ay;
            if (__all_sync(0xffffffffu, fast || !in[rr])) {
                py[rr] = fast ? tile_lerp<kTL>(&st->ry[0][0], lx, lyy, ax, ay) : 0.f;
            } else {
                py[rr] = in[rr] ? (st ? sample<kTL>(c.ry0, c.yp, W, H, gx, gy, f[rr].x, f[rr].y, &st->ry[0][0],
                                                    tx0, ty0)
                                      : sample<0>(c.ry0, c.yp, W, H, gx, gy, f[rr].x, f[rr].y, nullptr, 0, 0))
                                : 0.f;
            }
        }
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            if (!in[rr]) continue;
            const int ly = 2 * (ty + 4 * jj) + rr, gy = my * kMB + ly;
            const float v = fminf(fmaxf(py[rr] + tl.ry[ly][x], 0.f), 255.f);
            c.oy0[gy * c.yp + gx] = v;
            c.uy0[gy * c.op + gx] = (uint8_t)__float2int_rd(v + 0.5f);
        }
        if (CHROMA) {
            // chroma: even lanes Cb, odd lanes Cr, one chroma column per lane pair
            float sx = f[0].x + f[1].x, sy = f[0].y + f[1].y;
            int n = (int)in[0] + (int)in[1];
            sx += __shfl_xor_sync(0xffffffffu, sx, 1);
            sy += __shfl_xor_sync(0xffffffffu, sy, 1);
            n += __shfl_xor_sync(0xffffffffu, n, 1);
            const float sc = n == 4 ? 0.125f : (n == 2 ? 0.25f : 0.5f);
            const float dx = sx * sc, dy = sy * sc;
            const int j = ty + 4 * jj, cyg = my * (kMB / 2) + j;
            const bool cin = cxg < c.cw && cyg < c.chh;
            const float fx = floorf(dx), fy = floorf(dy);
            const float ax = dx - fx, ay = dy - fy;
            const int lx = (x >> 1) + kCHalo + __float2int_rn(fx), lyy = j + kCHalo + __float2int_rn(fy);
            const bool fast = st != nullptr && lx >= cx_lo && lx <= cx_hi && lyy >= cy_lo && lyy <= cy_hi &&
                              ax == ax && ay == ay;
            float pc;
            if (__all_sync(0xffffffffu, fast || !cin)) {
                pc = fast ? tile_lerp<kTC>(&st->rc[cp][0][0], lx, lyy, ax, ay) : 0.f;
            } else {
                pc = cin ? (st ? sample<kTC>(c.rcp, c.cpitch, c.cw, c.chh, cxg, cyg, dx, dy, &st->rc[cp][0][0], cx0,
                                             cy0)
                               : sample<0>(c.rcp, c.cpitch, c.cw, c.chh, cxg, cyg, dx, dy, nullptr, 0, 0))
                         : 0.f;
            }
            if (cin) {
                const float v = fminf(fmaxf(pc + tl.rc[cp][j][x >> 1], 0.f), 255.f);
                c.ocp[cyg * c.cpitch + cxg] = v;
                c.ucp[cyg * c.uop + cxg] = (uint8_t)__float2int_rd(v + 0.5f);
            }
        }
    }
}

template <bool CHROMA>
__device__ __forceinline__ PixelCtx pixel_ctx(const FusedFrame &F)
{
    PixelCtx c;
    c.W = F.width;
    c.H = F.height;
    c.cw = (F.width + 1) / 2;
    c.chh = (F.height + 1) / 2;
    c.yp = F.ref_pitch[0];
    c.op = F.out_pitch[0];
    c.ry0 = F.ref[0];
    c.oy0 = F.ref_out[0];
    c.uy0 = F.out[0];
    const int cp = threadIdx.x & 1;
    if (CHROMA) {
        c.rcp = cp ? F.ref[2] : F.ref[1];
        c.ocp = cp ? F.ref_out[2] : F.ref_out[1];
        c.ucp = cp ? F.out[2] : F.out[1];
        c.cpitch = cp ? F.ref_pitch[2] : F.ref_pitch[1];
        c.uop = cp ? F.out_pitch[2] : F.out_pitch[1];
    } else {
        c.rcp = nullptr;
        c.ocp = nullptr;
        c.ucp = nullptr;
        c.cpitch = c.uop = 0;
    }
    return c;
}

// the last CTA to leave clears the macroblock counters for the next frame
__device__ __forceinline__ void release_mb_counters(const FusedFrame &F)
{
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(F.ctr + kCtrFusedDone, 1u) == gridDim.x - 1) {
            F.ctr[kCtrFusedWork] = 0;
            F.ctr[kCtrFusedDone] = 0;
            __threadfence();
        }
    }
}

// ---- plain variant: global loads only ------------------------------------
template <bool CHROMA>
__global__ void __launch_bounds__(kThreads, 8) pframe_fused_kernel(const __grid_constant__ FusedFrame F, BlockTables tab,
                                                                uint32_t *flags)
{
    __shared__ Tiles tl;
    __shared__ int s_mb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PixelCtx pc = pixel_ctx<CHROMA>(F);
    const float2 *fl = reinterpret_cast<const float2 *>(F.flow);
    grid_dependency_wait();
    for (;;) {
        if (threadIdx.x == 0) s_mb = (int)atomicAdd(F.ctr + kCtrFusedWork, 1u);
        __syncthreads();
        const int mb = s_mb;
        if (mb >= F.nmb) break;
        const int mx = mb % F.nmbx, my = mb / F.nmbx;
        mb_residual<CHROMA>(F, tab, tl, mx, my, warp, lane);
        __syncthreads();
        mb_pixels<CHROMA>(pc, tl, nullptr, mx, my, fl);
        __syncthreads();
    }
    release_mb_counters(F);
}

// ---- TMA variant ---------------------------------------------------------
template <bool CHROMA>
__device__ __forceinline__ void issue_stage(const FusedFrame &F, Stage &st, uint64_t *bar, int mb,
                                            const CUtensorMap *mf, const CUtensorMap *mry, const CUtensorMap *mcb,
                                            const CUtensorMap *mcr)
{
    const int mx = mb % F.nmbx, my = mb / F.nmbx;
    const uint32_t bytes = sizeof(st.flow) + sizeof(st.ry) + (CHROMA ? sizeof(st.rc) : 0);
    mbar_expect_tx(bar, bytes);
    tma_load_2d(&st.flow[0][0], mf, mx * 2 * kMB, my * kMB, bar);
    tma_load_2d(&st.ry[0][0], mry, mx * kMB - kHalo, my * kMB - kHalo, bar);
    if (CHROMA) {
        tma_load_2d(&st.rc[0][0][0], mcb, mx * (kMB / 2) - kCHalo, my * (kMB / 2) - kCHalo, bar);
        tma_load_2d(&st.rc[1][0][0], mcr, mx * (kMB / 2) - kCHalo, my * (kMB / 2) - kCHalo, bar);
    }
}

template <bool CHROMA>
__global__ void __launch_bounds__(kThreads, 6) pframe_tma_kernel(const __grid_constant__ FusedFrame F,
                                                                 const __grid_constant__ CUtensorMap mflow,
                                                                 const __grid_constant__ CUtensorMap mrefy,
                                                                 const __grid_constant__ CUtensorMap mrefcb,
                                                                 const __grid_constant__ CUtensorMap mrefcr,
                                                                 BlockTables tab, uint32_t *flags)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Stage &st = *reinterpret_cast<Stage *>(smem);
    Tiles &tl = *reinterpret_cast<Tiles *>(smem + sizeof(Stage));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + sizeof(Stage) + sizeof(Tiles));
    __shared__ int s_mb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PixelCtx pc = pixel_ctx<CHROMA>(F);
    const float2 *fl = reinterpret_cast<const float2 *>(F.flow);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_proxy_async();
    }
    uint32_t parity = 0u;
    bool ok = true, first = true;
    for (;;) {
        // the CTA takes the next macroblock and starts the tensor-memory
        // copies of its flow and reference tiles; the residual evaluation
        // runs while they are in flight
        if (threadIdx.x == 0) {
            s_mb = (int)atomicAdd(F.ctr + kCtrFusedWork, 1u);
            if (s_mb < F.nmb && ok) {
                fence_proxy_async();  // the stage was last read by the generic proxy
                issue_stage<CHROMA>(F, st, bar, s_mb, &mflow, &mrefy, &mrefcb, &mrefcr);
            }
        }
        __syncthreads();
        const int mb = s_mb;
        if (mb >= F.nmb) break;
        const bool issued = ok;
        if (first) {
            // the reference planes and the flow were complete before the
            // coefficient kernel started; its coefficients are not yet
            grid_dependency_wait();
            first = false;
        }
        const int mx = mb % F.nmbx, my = mb / F.nmbx;
        mb_residual<CHROMA>(F, tab, tl, mx, my, warp, lane);
        __syncthreads();
        bool landed = false;
        if (issued) {
            landed = mbar_wait(bar, parity);
            if (landed) parity ^= 1u;
            else if (threadIdx.x == 0) atomicOr(flags, kFlagTimeout);
        }
        // a timed-out copy may still land later: stop issuing and finish on
        // global loads (the staged tile is not read)
        ok = ok && landed;
        mb_pixels<CHROMA>(pc, tl, landed ? &st : nullptr, mx, my, fl);
        __syncthreads();
    }
    if (first) grid_dependency_wait();
    if (!ok) mbar_wait(bar, parity);  // bounded: let a late copy land first
    release_mb_counters(F);
}

template <class Kern>
int occupancy(Kern k, size_t smem)
{
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, kThreads, smem) != cudaSuccess || o < 1) o = 1;
    return o;
}

}  // namespace

bool fused_supported(int block) { return block == 16 || block == 8; }

cudaError_t fused_init()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(pframe_tma_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kTmaSmem)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(pframe_tma_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem);
}

cudaError_t launch_pframe_fused(FusedFrame &F, const FusedMaps *maps, uint32_t *flags, cudaStream_t st, bool pdl)
{
    F.nmbx = (F.width + kMB - 1) / kMB;
    F.nmb = F.nmbx * ((F.height + kMB - 1) / kMB);
    const BlockTables &t = block_tables();
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (maps) {
        static int occ[2] = {0, 0};
        int &o = occ[F.chroma ? 1 : 0];
        if (o == 0)
            o = F.chroma ? occupancy(pframe_tma_kernel<true>, kTmaSmem) : occupancy(pframe_tma_kernel<false>, kTmaSmem);
        cfg.gridDim = dim3(std::max(1, std::min(F.nmb, t.sms * o)));
        cfg.dynamicSmemBytes = kTmaSmem;
        if (F.chroma)
            return cudaLaunchKernelEx(&cfg, pframe_tma_kernel<true>, F, maps->flow, maps->ref[0], maps->ref[1],
                                      maps->ref[2], t, flags);
        return cudaLaunchKernelEx(&cfg, pframe_tma_kernel<false>, F, maps->flow, maps->ref[0], maps->ref[1],
                                  maps->ref[2], t, flags);
    }
    static int occ[2] = {0, 0};
    int &o = occ[F.chroma ? 1 : 0];
    if (o == 0) o = F.chroma ? occupancy(pframe_fused_kernel<true>, 0) : occupancy(pframe_fused_kernel<false>, 0);
    cfg.gridDim = dim3(std::max(1, std::min(F.nmb, t.sms * o)));
    cfg.dynamicSmemBytes = 0;
    if (F.chroma) return cudaLaunchKernelEx(&cfg, pframe_fused_kernel<true>, F, t, flags);
    return cudaLaunchKernelEx(&cfg, pframe_fused_kernel<false>, F, t, flags);
}

}  // namespace hivc
