// Fused inter-frame kernel (Sec. 2, Sec. 2.2, Sec. 2.3): one CTA decodes a
// 32 x 32 luma macroblock and its 16 x 16 Cb and Cr tiles in two phases:
//   B. the evaluation r = a + sum_j c_j G[p_j, :] (Eq. 3) of the
//      macroblock's residual blocks into a shared residual tile, with r = v
//      at the points; c and a come from the coefficient kernel (k_block.cu),
//      launched before this one;
//   C. the backward bilinear warp of the previous reconstruction along the
//      transmitted flow (chroma flow = half the mean of the co-sited 2 x 2
//      luma vectors), + residual, clamp to [0, 255]: the new FP32 reference
//      and the uint8 output.
// The residual field never goes through global memory.
//
// CTA c of a grid of G decodes the macroblocks c, c + G, c + 2G, ...  In
// the TMA variant the tensor memory accelerator copies a macroblock's flow
// tile and its reference tiles (8-pixel luma / 4-pixel chroma halo) into
// one of two shared stages two macroblocks ahead, so that the copies of the
// next macroblock are in flight while one is decoded; samples that leave
// the halo read global memory.  The kernel is launched as a programmatic
// dependent of the preceding launch.  After this frame's coefficient kernel
// its first copies overlap that grid (griddepcontrol.wait orders the
// coefficient reads); after the previous frame's fused kernel (a batch of
// frames, coefficients already complete) it waits for that grid, which
// wrote its references, before the first copy.
#include <atomic>
#include <cuda.h>

#include "block_device.cuh"

namespace hivc {
namespace {

constexpr int kMB = 32;  // luma macroblock edge
constexpr int kThreads = 128;
constexpr int kHalo = 8, kTL = kMB + 2 * kHalo;        // luma reference tile 48 x 48
constexpr int kCHalo = 4, kTC = kMB / 2 + 2 * kCHalo;  // chroma reference tile 24 x 24
constexpr long kMbarSpins = 1L << 22;                  // bounded waits
constexpr int kRYP = kMB + 4;                          // luma residual tile pitch (16-byte rows)
constexpr int kRCP = kMB / 2 + 4;                      // chroma residual tile pitch
constexpr int kRCS = (kMB / 2) * kRCP + 16;            // chroma plane stride (other banks)
constexpr float kFastFlow = 7.f;                       // |flow| below this never leaves the halo

struct __align__(128) Stage {
    float flow[kMB][2 * kMB];  // 32 rows of 32 (dx, dy)
    float ry[kTL][kTL];
    float rc[2][kTC][kTC];
};

// residual tiles of one macroblock
struct __align__(16) Tiles {
    float ry[kMB * kRYP];
    float rc[2 * kRCS];
};

// shared memory: two stages (TMA variant), the residual tiles, two barriers
template <bool TMA>
__host__ __device__ constexpr size_t kernel_smem()
{
    return (TMA ? 2 * sizeof(Stage) : 0) + sizeof(Tiles) + 16;
}

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

// bilinear sample of R at (x + dx, y + dy), clamped, from global memory: the
// path of the samples whose footprint leaves the staged tile (rare, so it
// is kept out of line)
__device__ __noinline__ float sample_global(const float *__restrict__ R, int pitch, int W, int H, int x, int y,
                                            float dx, float dy)
{
    float ax, ay;
    const int x0 = split_axis(dx, x, W, ax), y0 = split_axis(dy, y, H, ay);
    const int ox = min(x0 + 1, W - 1) - x0, oyn = min(y0 + 1, H - 1) - y0;
    const float *g = R + (size_t)y0 * pitch + x0;
    const float r00 = __ldg(g), r01 = __ldg(g + ox), r10 = __ldg(g + (size_t)oyn * pitch),
                r11 = __ldg(g + (size_t)oyn * pitch + ox);
    // the same interpolation steps as tile_lerp, so that a sample gives the
    // same value whichever path it takes
    const float top = fmaf(ax, r01 - r00, r00);
    const float bot = fmaf(ax, r11 - r10, r10);
    return fmaf(ay, bot - top, top);
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

// residual + prediction, clamped to [0, 255]: the new FP32 reference and
// the uint8 output (round half up)
__device__ __forceinline__ void put_pixel(float pred, float r, float *ref_out, uint8_t *out)
{
    const float v = fminf(fmaxf(pred + r, 0.f), 255.f);
    *ref_out = v;
    *out = (uint8_t)__float2int_rd(v + 0.5f);
}

// y = p / w and x = p - y w for p < 256, w <= 16: (p + 1/2) / w lies at
// least 1 / (2w) from an integer, far beyond the rounding of the product
__device__ __forceinline__ void split_pos(int p, int w, float rw, int &y, int &x)
{
    y = __float2int_rz(((float)p + 0.5f) * rw);
    x = p - y * w;
}

// ---- phase B: residual tiles (Eq. 3) ---------------------------------------
// One residual block as the evaluation reads it: K = 0 for an empty block,
// one outside the plane, and one with bad data (block pointers or K, which
// the coefficient kernel flags, or positions, for which it sets a = NaN).
struct BlkView {
    const float *G;      // Green's rows of the block's shape
    const float *cs;     // its coefficients c_j,
    const uint8_t *ps;   // positions p_j
    const int16_t *vs;   // and values v_j
    int rl, w, h, K;
    int ox, oy;          // offset in the macroblock (plane pixels)
    float a;
};

// block (bx, by) of plane data P (value set vi), at (ox, oy) in the
// macroblock; reads the coefficient kernel's a
__device__ __forceinline__ BlkView block_view(const BlockPlane &P, int vi, int bx, int by, int ox, int oy,
                                              bool present, const BlockTables &tab)
{
    BlkView V;
    V.G = tab.G;
    V.cs = nullptr;
    V.ps = nullptr;
    V.vs = nullptr;
    V.rl = 8;
    V.w = V.h = 1;
    V.K = 0;
    V.ox = ox;
    V.oy = oy;
    V.a = 0.f;
    if (!present) return V;
    const BlockGeom g = block_geom(P, by * P.nbx + bx);
    V.w = g.w;
    V.h = g.h;
    V.rl = g_rowlen(g.w * g.h);
    V.G = green_rows(tab, g.w, g.h);
    if (g.bad || g.K == 0) return V;
    const float a = __ldg(P.acoef[vi] + g.lb);
    if (!(a == a)) return V;
    V.K = g.K;
    V.a = a;
    V.cs = P.coef[vi] + g.s;
    V.ps = P.pos + g.s;
    V.vs = P.val[vi] + g.s;
    return V;
}

// Whole-block rows: the N pixels q0 .. q0 + N - 1 (N = 8 or 2, q0 a
// multiple of N) of one block, for one or two planes with the same points:
//   r[t] = a + sum_j c_j G[p_j, q0 + t]
// The GRP lanes of an aligned lane group share one block (GRP = 32 or 8):
// lane u of the group holds point j0 + u of a chunk, so that the loop body
// gets c_j and p_j by shuffles and its Green's-row loads are independent.
// Kmax is the warp's largest K; c = 0 past a block's own K.
template <int N, bool TWO, int GRP>
__device__ __forceinline__ void eval_row(const float *G, int rl, const float *cs0, const float *cs1,
                                         const uint8_t *ps, int K, int Kmax, int q0, float a0, float a1,
                                         float (&r0)[N], float (&r1)[N])
{
    const int lane = threadIdx.x & 31, base = lane & ~(GRP - 1), sub = lane & (GRP - 1);
#pragma unroll
    for (int t = 0; t < N; ++t) {
        r0[t] = a0;
        r1[t] = a1;
    }
    const float *Gq = G + q0;
    for (int j0 = 0; j0 < Kmax; j0 += GRP) {
        const int jj = j0 + sub;
        const bool live = jj < K;
        const float h0 = live ? __ldg(cs0 + jj) : 0.f, h1 = (TWO && live) ? __ldg(cs1 + jj) : 0.f;
        const int hp = live ? __ldg(ps + jj) : 0;
        const int n = min(GRP, Kmax - j0);
#pragma unroll 4
        for (int u = 0; u < n; ++u) {
            const float c0 = __shfl_sync(0xffffffffu, h0, base + u);
            const float c1 = TWO ? __shfl_sync(0xffffffffu, h1, base + u) : 0.f;
            const float *g = Gq + __shfl_sync(0xffffffffu, hp, base + u) * rl;
            float gv[N];
            if (N == 8) {
                const float4 lo = __ldg(reinterpret_cast<const float4 *>(g));
                const float4 hi = __ldg(reinterpret_cast<const float4 *>(g) + 1);
                gv[0] = lo.x;
                gv[1] = lo.y;
                gv[2 % N] = lo.z;
                gv[3 % N] = lo.w;
                gv[4 % N] = hi.x;
                gv[5 % N] = hi.y;
                gv[6 % N] = hi.z;
                gv[7 % N] = hi.w;
            } else {
                const float2 v = __ldg(reinterpret_cast<const float2 *>(g));
                gv[0] = v.x;
                gv[1 % N] = v.y;
            }
#pragma unroll
            for (int t = 0; t < N; ++t) {
                r0[t] = fmaf(c0, gv[t], r0[t]);
                if (TWO) r1[t] = fmaf(c1, gv[t], r1[t]);
            }
        }
    }
}

// Any block (cut by the plane edge): N pixels of block row y from block
// column x0, scalar loads; pixels outside the block get a.
template <int N>
__device__ __forceinline__ void eval_any(const BlkView &V, int y, int x0, float (&r)[N])
{
    int q[N];
#pragma unroll
    for (int t = 0; t < N; ++t) {
        q[t] = (y < V.h && x0 + t < V.w) ? y * V.w + x0 + t : 0;
        r[t] = V.a;
    }
    for (int j = 0; j < V.K; ++j) {
        const float c = __ldg(V.cs + j);
        const float *g = V.G + __ldg(V.ps + j) * V.rl;
#pragma unroll
        for (int t = 0; t < N; ++t) r[t] = fmaf(c, __ldg(g + q[t]), r[t]);
    }
}

// r = v at the points of a block (the exact data), into a tile of pitch
// tp; points in block rows [ylo, yhi) only
__device__ __forceinline__ void put_points(const BlkView &V, float *tile, int tp, int ylo, int yhi, int lane)
{
    const float rw = __frcp_rn((float)V.w);
    for (int j = lane; j < V.K; j += 32) {
        int y, x;
        split_pos(__ldg(V.ps + j), V.w, rw, y, x);
        if (y >= ylo && y < yhi) tile[(V.oy + y) * tp + V.ox + x] = (float)__ldg(V.vs + j);
    }
}

// Luma: B = 16, warp w evaluates block w of the macroblock (lane l: row
// l / 2, columns 8 (l % 2) .. +7); B = 8, warp w the blocks of block row w
// (lane l: block l / 8, row l % 8).  Eight pixels per lane, written as two
// 16-byte rows.
template <int B>
__device__ __forceinline__ void phase_b_luma(const FusedFrame &F, const BlockTables &tab, Tiles &T, int mx, int my,
                                             int warp, int lane)
{
    constexpr int NBL = kMB / B, LPB = B * B / 8;  // blocks per macroblock row, lanes per block
    const int bi = B == 16 ? warp : warp * 4 + lane / LPB;
    const int ox = (bi % NBL) * B, oy = (bi / NBL) * B;
    const int l = lane % LPB, y = (8 * l) / B, x0 = (8 * l) % B;
    const bool present = mx * kMB + ox < F.width && my * kMB + oy < F.height;
    const BlkView V = block_view(F.bp[0], 0, mx * NBL + ox / B, my * NBL + oy / B, ox, oy, present, tab);
    int Kmax = V.K;
    if (B == 8) {
#pragma unroll
        for (int o = 8; o < 32; o <<= 1) Kmax = max(Kmax, __shfl_xor_sync(0xffffffffu, Kmax, o));
    }
    float r[8], rd[8];
    if (__all_sync(0xffffffffu, V.w == B && V.h == B))
        eval_row<8, false, LPB>(V.G, V.rl, V.cs, V.cs, V.ps, V.K, Kmax, 8 * l, V.a, 0.f, r, rd);
    else
        eval_any<8>(V, y, x0, r);
    float *row = T.ry + (oy + y) * kRYP + ox + x0;
    reinterpret_cast<float4 *>(row)[0] = make_float4(r[0], r[1], r[2], r[3]);
    reinterpret_cast<float4 *>(row)[1] = make_float4(r[4], r[5], r[6], r[7]);
    __syncwarp();
    if (B == 16) {
        put_points(V, T.ry, kRYP, 0, B, lane);
    } else {
        // the warp's four blocks one after the other, all lanes each
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            const BlkView U = block_view(F.bp[0], 0, mx * NBL + b, my * NBL + warp, b * B, warp * B,
                                         mx * kMB + b * B < F.width && my * kMB + warp * B < F.height, tab);
            put_points(U, T.ry, kRYP, 0, B, lane);
        }
    }
}

// Chroma: B = 16, warp w evaluates rows 4w .. 4w+3 of the block (lane l:
// row 4w + l / 8, columns 2 (l % 8), +1); B = 8, warp w block w (lane l:
// row l / 4, columns 2 (l % 4), +1).  Both planes; one loop when Cb and Cr
// share their points.
template <int B>
__device__ __forceinline__ void phase_b_chroma(const FusedFrame &F, const BlockTables &tab, Tiles &T, int mx, int my,
                                               int warp, int lane)
{
    constexpr int NBC = kMB / 2 / B;
    const int blk = B == 16 ? 0 : warp;
    const int ox = (blk % NBC) * B, oy = (blk / NBC) * B;
    const int y = B == 16 ? 4 * warp + lane / 8 : lane / 4, x0 = B == 16 ? 2 * (lane % 8) : 2 * (lane % 4);
    const int ylo = B == 16 ? 4 * warp : 0, yhi = B == 16 ? 4 * warp + 4 : B;
    const int bx = mx * NBC + ox / B, by = my * NBC + oy / B;
    const bool present = mx * (kMB / 2) + ox < (F.width + 1) / 2 && my * (kMB / 2) + oy < (F.height + 1) / 2;
    const bool paired = F.nblk == 2;
    const BlkView V0 = block_view(F.bp[1], 0, bx, by, ox, oy, present, tab);
    const BlkView V1 = paired ? block_view(F.bp[1], 1, bx, by, ox, oy, present && F.bp[1].val[1] != nullptr, tab)
                              : block_view(F.bp[2], 0, bx, by, ox, oy, present, tab);
    const bool whole0 = V0.w == B && V0.h == B, whole1 = V1.w == B && V1.h == B;
    float r0[2], r1[2];
    const int q0 = y * B + x0;
    if (paired && __all_sync(0xffffffffu, whole0 && whole1 && V0.K == V1.K)) {
        eval_row<2, true, 32>(V0.G, V0.rl, V0.cs, V1.cs, V0.ps, V0.K, V0.K, q0, V0.a, V1.a, r0, r1);
    } else {
        float d[2];
        if (__all_sync(0xffffffffu, whole0))
            eval_row<2, false, 32>(V0.G, V0.rl, V0.cs, V0.cs, V0.ps, V0.K, V0.K, q0, V0.a, 0.f, r0, d);
        else eval_any<2>(V0, y, x0, r0);
        if (__all_sync(0xffffffffu, whole1))
            eval_row<2, false, 32>(V1.G, V1.rl, V1.cs, V1.cs, V1.ps, V1.K, V1.K, q0, V1.a, 0.f, r1, d);
        else eval_any<2>(V1, y, x0, r1);
    }
    *reinterpret_cast<float2 *>(T.rc + (oy + y) * kRCP + ox + x0) = make_float2(r0[0], r0[1]);
    *reinterpret_cast<float2 *>(T.rc + kRCS + (oy + y) * kRCP + ox + x0) = make_float2(r1[0], r1[1]);
    __syncwarp();
    put_points(V0, T.rc, kRCP, ylo, yhi, lane);
    put_points(V1, T.rc + kRCS, kRCP, ylo, yhi, lane);
}

// ---- phase C: warp + residual + clamp + pack -------------------------------
struct PixelCtx {
    int W, H, cw, chh, yp, op;
    const float *ry0;
    float *oy0;
    uint8_t *uy0;
    const float *rcp;  // this lane's chroma plane (x & 1: Cb, Cr)
    float *ocp;
    uint8_t *ucp;
    int cpitch, uop;
    float *oc[2];      // both chroma planes (Cb, Cr)
    uint8_t *uc[2];
    int ocp2[2], uop2[2];
    bool vec2;         // luma output rows take 8-byte (ref) and 2-byte (uint8) pairs
};

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
    for (int k = 0; k < 2; ++k) {
        c.oc[k] = F.ref_out[1 + k];
        c.uc[k] = F.out[1 + k];
        c.ocp2[k] = F.ref_pitch[1 + k];
        c.uop2[k] = F.out_pitch[1 + k];
    }
    c.vec2 = (((uintptr_t)F.ref_out[0] | (uintptr_t)F.ref_pitch[0] * 4) & 7) == 0 &&
             (((uintptr_t)F.out[0] | (uintptr_t)F.out_pitch[0]) & 1) == 0;
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

// The residual of a macroblock as phase C reads it: luma rows yp floats
// apart, the two chroma planes' rows cp floats apart (shared tiles, or the
// global residual fields at the macroblock's origin).
struct ResView {
    const float *y;
    const float *c[2];
    int yp, cp;
};

// Thread (x, ty) takes luma rows 2 ty + 8 jj + {0, 1} of column x and
// chroma row ty + 4 jj of column x / 2 in plane x & 1, whose flow is half
// the mean of the four co-sited luma vectors: the thread's two rows and the
// neighbouring lane's.  FAST (macroblock inside the plane with its halo,
// every |flow| < 7, so every footprint lies in the staged tiles): no range
// checks.  Otherwise each sample is checked and the ones that leave the
// staged tile (or all, st = null) read global memory.
template <bool CHROMA, bool FAST>
__device__ __forceinline__ void phase_c(const PixelCtx &c, const ResView &R, const Stage *st, int mx, int my,
                                        const float2 *__restrict__ fl)
{
    const int W = c.W, H = c.H;
    const float *rcp = (threadIdx.x & 1) ? R.c[1] : R.c[0];
    const int x = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int gx = mx * kMB + x;
    const int tx0 = mx * kMB - kHalo, ty0 = my * kMB - kHalo;
    const int lx_lo = max(0, -tx0), lx_hi = min(kTL - 2, W - 2 - tx0);
    const int ly_lo = max(0, -ty0), ly_hi = min(kTL - 2, H - 2 - ty0);
    const int cp = x & 1, cx = x >> 1;
    const int cxg = mx * (kMB / 2) + cx;
    const int cx0 = mx * (kMB / 2) - kCHalo, cy0 = my * (kMB / 2) - kCHalo;
    const int cx_lo = max(0, -cx0), cx_hi = min(kTC - 2, c.cw - 2 - cx0);
    const int cy_lo = max(0, -cy0), cy_hi = min(kTC - 2, c.chh - 2 - cy0);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
        float2 f[2];
        bool in[2];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
            const int ly = 2 * ty + 8 * jj + rr, gy = my * kMB + ly;
            in[rr] = FAST || (gx < W && gy < H);
            if (st) f[rr] = *reinterpret_cast<const float2 *>(&st->flow[ly][2 * x]);
            else f[rr] = in[rr] ? __ldg(fl + (size_t)gy * W + gx) : make_float2(0.f, 0.f);
            if (!in[rr]) continue;
            const float fx = floorf(f[rr].x), fy = floorf(f[rr].y);
            const float ax = f[rr].x - fx, ay = f[rr].y - fy;
            const int lx = x + kHalo + __float2int_rn(fx), lyy = ly + kHalo + __float2int_rn(fy);
            float pred;
            if (FAST) {
                pred = tile_lerp<kTL>(&st->ry[0][0], lx, lyy, ax, ay);
            } else {
                const bool fast = st != nullptr && lx >= lx_lo && lx <= lx_hi && lyy >= ly_lo && lyy <= ly_hi &&
                                  ax == ax && ay == ay;
                pred = fast ? tile_lerp<kTL>(&st->ry[0][0], lx, lyy, ax, ay)
                            : sample_global(c.ry0, c.yp, W, H, gx, gy, f[rr].x, f[rr].y);
            }
            put_pixel(pred, R.y[ly * R.yp + x], c.oy0 + (size_t)gy * c.yp + gx, c.uy0 + (size_t)gy * c.op + gx);
        }
        if (CHROMA) {
            // row sums first, as in the quad paths: ((f00 + f01) + (f10 + f11)),
            // vectors outside the plane are zero
            const float r0x = f[0].x + __shfl_xor_sync(0xffffffffu, f[0].x, 1);
            const float r0y = f[0].y + __shfl_xor_sync(0xffffffffu, f[0].y, 1);
            const float r1x = f[1].x + __shfl_xor_sync(0xffffffffu, f[1].x, 1);
            const float r1y = f[1].y + __shfl_xor_sync(0xffffffffu, f[1].y, 1);
            const float sx = r0x + r1x, sy = r0y + r1y;
            int n = 4;
            if (!FAST) {
                n = (int)in[0] + (int)in[1];
                n += __shfl_xor_sync(0xffffffffu, n, 1);
            }
            const int j = ty + 4 * jj, cyg = my * (kMB / 2) + j;
            if (FAST || (cxg < c.cw && cyg < c.chh)) {
                const float sc = n == 4 ? 0.125f : (n == 2 ? 0.25f : 0.5f);
                const float dx = sx * sc, dy = sy * sc;
                const float fx = floorf(dx), fy = floorf(dy);
                const float ax = dx - fx, ay = dy - fy;
                const int lx = cx + kCHalo + __float2int_rn(fx), lyy = j + kCHalo + __float2int_rn(fy);
                float pred;
                if (FAST) {
                    pred = tile_lerp<kTC>(&st->rc[cp][0][0], lx, lyy, ax, ay);
                } else {
                    const bool fast = st != nullptr && lx >= cx_lo && lx <= cx_hi && lyy >= cy_lo && lyy <= cy_hi &&
                                      ax == ax && ay == ay;
                    pred = fast ? tile_lerp<kTC>(&st->rc[cp][0][0], lx, lyy, ax, ay)
                                : sample_global(c.rcp, c.cpitch, c.cw, c.chh, cxg, cyg, dx, dy);
                }
                put_pixel(pred, rcp[j * R.cp + cx], c.ocp + (size_t)cyg * c.cpitch + cxg,
                          c.ucp + (size_t)cyg * c.uop + cxg);
            }
        }
    }
}

// The fast case (macroblock inside the plane with its halo, every
// |flow| < 7): item (l, j) of 16 x 16 is the luma quad at columns 2l, 2l+1
// and rows 2j, 2j+1 with the co-sited chroma pixel (l, j) of Cb and Cr,
// whose flow is half the mean of the quad's four vectors; thread t takes
// the items t and t + 128.  Every footprint lies in the staged tiles.  The
// residual comes from shared tiles (luma rows RYP floats apart, chroma rows
// RCP apart, the Cr tile RCS after Cb).  Luma results leave as pairs where
// the output rows allow (vec2: 8-byte ref_out rows, 2-byte uint8 rows).
template <bool CHROMA, int RYP, int RCP, int RCS>
__device__ __forceinline__ void phase_c_quads(const PixelCtx &c, const float *ryt, const float *rct, const Stage &st,
                                              int mx, int my)
{
    const bool vec2 = c.vec2;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int item = threadIdx.x + it * kThreads, l = item & 15, j = item >> 4;
        const int ly = 2 * j, lx = 2 * l;
        const float4 fa = *reinterpret_cast<const float4 *>(&st.flow[ly][2 * lx]);
        const float4 fb = *reinterpret_cast<const float4 *>(&st.flow[ly + 1][2 * lx]);
        const float2 fv[4] = {{fa.x, fa.y}, {fa.z, fa.w}, {fb.x, fb.y}, {fb.z, fb.w}};
        float pv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float fx = floorf(fv[q].x), fy = floorf(fv[q].y);
            pv[q] = tile_lerp<kTL>(&st.ry[0][0], lx + (q & 1) + kHalo + __float2int_rn(fx),
                                   ly + (q >> 1) + kHalo + __float2int_rn(fy), fv[q].x - fx, fv[q].y - fy);
        }
        const float2 r0 = *reinterpret_cast<const float2 *>(ryt + ly * RYP + lx);
        const float2 r1 = *reinterpret_cast<const float2 *>(ryt + (ly + 1) * RYP + lx);
        const float rr[4] = {r0.x, r0.y, r1.x, r1.y};
        float v[4];
        uint8_t u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            v[q] = fminf(fmaxf(pv[q] + rr[q], 0.f), 255.f);
            u[q] = (uint8_t)__float2int_rd(v[q] + 0.5f);
        }
        const size_t gx = (size_t)mx * kMB + lx, gy = (size_t)my * kMB + ly;
        float *o0 = c.oy0 + gy * c.yp + gx;
        uint8_t *b0 = c.uy0 + gy * c.op + gx;
        if (vec2) {
            *reinterpret_cast<float2 *>(o0) = make_float2(v[0], v[1]);
            *reinterpret_cast<float2 *>(o0 + c.yp) = make_float2(v[2], v[3]);
            *reinterpret_cast<uint16_t *>(b0) = (uint16_t)(u[0] | (u[1] << 8));
            *reinterpret_cast<uint16_t *>(b0 + c.op) = (uint16_t)(u[2] | (u[3] << 8));
        } else {
            o0[0] = v[0];
            o0[1] = v[1];
            o0[c.yp] = v[2];
            o0[c.yp + 1] = v[3];
            b0[0] = u[0];
            b0[1] = u[1];
            b0[c.op] = u[2];
            b0[c.op + 1] = u[3];
        }
        if (CHROMA) {
            const float dx = ((fv[0].x + fv[1].x) + (fv[2].x + fv[3].x)) * 0.125f;
            const float dy = ((fv[0].y + fv[1].y) + (fv[2].y + fv[3].y)) * 0.125f;
            const float fx = floorf(dx), fy = floorf(dy);
            const int tx = l + kCHalo + __float2int_rn(fx), tyy = j + kCHalo + __float2int_rn(fy);
            const size_t cx = (size_t)mx * (kMB / 2) + l, cy = (size_t)my * (kMB / 2) + j;
#pragma unroll
            for (int pl = 0; pl < 2; ++pl) {
                const float pred = tile_lerp<kTC>(&st.rc[pl][0][0], tx, tyy, dx - fx, dy - fy);
                const float vv = fminf(fmaxf(pred + rct[pl * RCS + j * RCP + l], 0.f), 255.f);
                c.oc[pl][cy * c.ocp2[pl] + cx] = vv;
                c.uc[pl][cy * c.uop2[pl] + cx] = (uint8_t)__float2int_rd(vv + 0.5f);
            }
        }
    }
}

// every luma flow vector of the thread's pixels below kFastFlow in size
// (false for NaN)
__device__ __forceinline__ bool small_flow(const Stage &st)
{
    const int x = threadIdx.x & 31, ty = threadIdx.x >> 5;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float2 f = *reinterpret_cast<const float2 *>(&st.flow[2 * ty + 8 * (k >> 1) + (k & 1)][2 * x]);
        ok = ok && fabsf(f.x) < kFastFlow && fabsf(f.y) < kFastFlow;
    }
    return ok;
}

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

// The fused inter-frame kernel.  TMA = false reads the flow and the
// references from global memory only (a flow whose rows a tensor map
// cannot describe).
template <bool CHROMA, int B, bool TMA>
__global__ void __launch_bounds__(kThreads, TMA ? 4 : 6) pframe_kernel(const __grid_constant__ FusedFrame F,
                                                                       const __grid_constant__ CUtensorMap mflow,
                                                                       const __grid_constant__ CUtensorMap mrefy,
                                                                       const __grid_constant__ CUtensorMap mrefcb,
                                                                       const __grid_constant__ CUtensorMap mrefcr,
                                                                       BlockTables tab, uint32_t *flags)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Stage *stages = reinterpret_cast<Stage *>(smem);
    Tiles &T = *reinterpret_cast<Tiles *>(smem + (TMA ? 2 * sizeof(Stage) : 0));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (TMA ? 2 * sizeof(Stage) : 0) + sizeof(Tiles));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const PixelCtx pc = pixel_ctx<CHROMA>(F);
    const float2 *fl = reinterpret_cast<const float2 *>(F.flow);
    // pend[s]: the iteration whose tiles stage s is receiving (-1: none);
    // ph[s]: the phase of stage s's barrier at its next completion
    // (scalars, not arrays indexed by s, which would live in local memory)
    int pend0 = TMA && (int)blockIdx.x < F.nmb ? 0 : -1, pend1 = TMA && (int)blockIdx.x + G < F.nmb ? 1 : -1;
    uint32_t ph0 = 0u, ph1 = 0u;
    bool ok = true;  // false after a copy timed out: the stages are not refilled
    // early: the flow and the references were complete before the preceding
    // launch (this frame's coefficient kernel) started, so the first copies
    // may overlap it; otherwise the preceding launch wrote the references
    if (!F.early) grid_dependency_wait();
    if (TMA && threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
        // the first two macroblocks' tiles
        if (pend0 >= 0) issue_stage<CHROMA>(F, stages[0], &bar[0], blockIdx.x, &mflow, &mrefy, &mrefcb, &mrefcr);
        if (pend1 >= 0) issue_stage<CHROMA>(F, stages[1], &bar[1], blockIdx.x + G, &mflow, &mrefy, &mrefcb, &mrefcr);
    }
    __syncthreads();
    // the coefficients are read from here on
    grid_dependency_wait();
    // the next launch in the stream may start now: it waits for this grid's
    // completion before it reads what this grid writes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    int it = 0;
    for (int mb = blockIdx.x; mb < F.nmb; mb += G, ++it) {
        const int s = it & 1;
        const int mx = mb % F.nmbx, my = mb / F.nmbx;
        phase_b_luma<B>(F, tab, T, mx, my, warp, lane);
        if (CHROMA) phase_b_chroma<B>(F, tab, T, mx, my, warp, lane);
        const bool issued = TMA && (s ? pend1 : pend0) == it;
        bool landed = false;
        if (issued) {
            landed = mbar_wait(&bar[s], s ? ph1 : ph0);
            if (landed) {
                if (s) {
                    ph1 ^= 1u;
                    pend1 = -1;
                } else {
                    ph0 ^= 1u;
                    pend0 = -1;
                }
            } else if (threadIdx.x == 0) {
                atomicOr(flags, kFlagTimeout);
            }
        }
        const Stage *st = landed ? &stages[s] : nullptr;
        const bool interior = mx * kMB - kHalo >= 0 && my * kMB - kHalo >= 0 &&
                              mx * kMB - kHalo + kTL <= F.width && my * kMB - kHalo + kTL <= F.height;
        const ResView R{T.ry, {T.rc, T.rc + kRCS}, kRYP, kRCP};
        if (__syncthreads_and(landed && interior && small_flow(stages[s])))
            phase_c_quads<CHROMA, kRYP, kRCP, kRCS>(pc, T.ry, T.rc, stages[s], mx, my);
        else
            phase_c<CHROMA, false>(pc, R, st, mx, my, fl);
        // a copy that timed out may still land later: from then on no stage
        // is refilled (the barrier also frees stage s and the tiles)
        if (__syncthreads_or(issued && !landed)) ok = false;
        if (TMA && ok && mb + 2 * G < F.nmb) {
            if (s) pend1 = it + 2;
            else pend0 = it + 2;
            if (threadIdx.x == 0) {
                fence_proxy_async();  // the stage was last read by the generic proxy
                issue_stage<CHROMA>(F, stages[s], &bar[s], mb + 2 * G, &mflow, &mrefy, &mrefcb, &mrefcr);
            }
        }
    }
    // bounded: let a copy that timed out land before the CTA exits
    if (TMA && pend0 >= 0) mbar_wait(&bar[0], ph0);
    if (TMA && pend1 >= 0) mbar_wait(&bar[1], ph1);
}

// ---- residual-field variant ----------------------------------------------
// The stage plus the macroblock's residual tiles (the residual planes were
// evaluated by the block kernels).
struct __align__(128) StageR {
    Stage s;
    float ry[kMB][kMB];
    float rc[2][kMB / 2][kMB / 2];
};

template <bool CHROMA>
__device__ __forceinline__ void issue_stage_rf(const FusedFrame &F, StageR &st, uint64_t *bar, int mb,
                                               const CUtensorMap *mf, const CUtensorMap *mry, const CUtensorMap *mcb,
                                               const CUtensorMap *mcr, const CUtensorMap *mrfy,
                                               const CUtensorMap *mrfb, const CUtensorMap *mrfr)
{
    const int mx = mb % F.nmbx, my = mb / F.nmbx;
    const uint32_t bytes = sizeof(st.s.flow) + sizeof(st.s.ry) + sizeof(st.ry) +
                           (CHROMA ? sizeof(st.s.rc) + sizeof(st.rc) : 0);
    mbar_expect_tx(bar, bytes);
    tma_load_2d(&st.s.flow[0][0], mf, mx * 2 * kMB, my * kMB, bar);
    tma_load_2d(&st.s.ry[0][0], mry, mx * kMB - kHalo, my * kMB - kHalo, bar);
    tma_load_2d(&st.ry[0][0], mrfy, mx * kMB, my * kMB, bar);
    if (CHROMA) {
        tma_load_2d(&st.s.rc[0][0][0], mcb, mx * (kMB / 2) - kCHalo, my * (kMB / 2) - kCHalo, bar);
        tma_load_2d(&st.s.rc[1][0][0], mcr, mx * (kMB / 2) - kCHalo, my * (kMB / 2) - kCHalo, bar);
        tma_load_2d(&st.rc[0][0][0], mrfb, mx * (kMB / 2), my * (kMB / 2), bar);
        tma_load_2d(&st.rc[1][0][0], mrfr, mx * (kMB / 2), my * (kMB / 2), bar);
    }
}

constexpr size_t kRfSmem = 2 * sizeof(StageR) + 16;

// Warp + residual + clamp + pack with the residual tiles staged beside the
// flow and reference tiles; the same macroblock order, stages and waits as
// the fused kernel.  A macroblock whose copies timed out reads the
// residual planes from global memory.
template <bool CHROMA>
__global__ void __launch_bounds__(kThreads, 4) pframe_rf_kernel(const __grid_constant__ FusedFrame F,
                                                                const __grid_constant__ FusedMaps M, uint32_t *flags)
{
    extern __shared__ __align__(128) unsigned char smem[];
    StageR *stages = reinterpret_cast<StageR *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * sizeof(StageR));
    const int G = gridDim.x;
    const PixelCtx pc = pixel_ctx<CHROMA>(F);
    const float2 *fl = reinterpret_cast<const float2 *>(F.flow);
    int pend0 = (int)blockIdx.x < F.nmb ? 0 : -1, pend1 = (int)blockIdx.x + G < F.nmb ? 1 : -1;
    uint32_t ph0 = 0u, ph1 = 0u;
    bool ok = true;
    // the preceding launch may have written the references or the residual
    // planes (its own frame's evaluation, or the previous frame)
    grid_dependency_wait();
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_proxy_async();
        if (pend0 >= 0)
            issue_stage_rf<CHROMA>(F, stages[0], &bar[0], blockIdx.x, &M.flow, &M.ref[0], &M.ref[1], &M.ref[2],
                                   &M.rf[0], &M.rf[1], &M.rf[2]);
        if (pend1 >= 0)
            issue_stage_rf<CHROMA>(F, stages[1], &bar[1], blockIdx.x + G, &M.flow, &M.ref[0], &M.ref[1], &M.ref[2],
                                   &M.rf[0], &M.rf[1], &M.rf[2]);
    }
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    int it = 0;
    for (int mb = blockIdx.x; mb < F.nmb; mb += G, ++it) {
        const int s = it & 1;
        const int mx = mb % F.nmbx, my = mb / F.nmbx;
        const bool issued = (s ? pend1 : pend0) == it;
        bool landed = false;
        if (issued) {
            landed = mbar_wait(&bar[s], s ? ph1 : ph0);
            if (landed) {
                if (s) {
                    ph1 ^= 1u;
                    pend1 = -1;
                } else {
                    ph0 ^= 1u;
                    pend0 = -1;
                }
            } else if (threadIdx.x == 0) {
                atomicOr(flags, kFlagTimeout);
            }
        }
        ResView R;
        if (landed) {
            R = ResView{&stages[s].ry[0][0], {&stages[s].rc[0][0][0], &stages[s].rc[1][0][0]}, kMB, kMB / 2};
        } else {
            const size_t cy = (size_t)my * (kMB / 2), cx = (size_t)mx * (kMB / 2);
            R = ResView{F.rfield[0] + (size_t)my * kMB * F.rfield_pitch[0] + (size_t)mx * kMB,
                        {CHROMA ? F.rfield[1] + cy * F.rfield_pitch[1] + cx : nullptr,
                         CHROMA ? F.rfield[2] + cy * F.rfield_pitch[2] + cx : nullptr},
                        F.rfield_pitch[0], CHROMA ? F.rfield_pitch[1] : 0};
        }
        const bool interior = mx * kMB - kHalo >= 0 && my * kMB - kHalo >= 0 &&
                              mx * kMB - kHalo + kTL <= F.width && my * kMB - kHalo + kTL <= F.height;
        const Stage *st = landed ? &stages[s].s : nullptr;
        if (__syncthreads_and(landed && interior && small_flow(stages[s].s)))
            phase_c_quads<CHROMA, kMB, kMB / 2, (kMB / 2) * (kMB / 2)>(pc, &stages[s].ry[0][0], &stages[s].rc[0][0][0],
                                                                       stages[s].s, mx, my);
        else
            phase_c<CHROMA, false>(pc, R, st, mx, my, fl);
        if (__syncthreads_or(issued && !landed)) ok = false;
        if (ok && mb + 2 * G < F.nmb) {
            if (s) pend1 = it + 2;
            else pend0 = it + 2;
            if (threadIdx.x == 0) {
                fence_proxy_async();
                issue_stage_rf<CHROMA>(F, stages[s], &bar[s], mb + 2 * G, &M.flow, &M.ref[0], &M.ref[1], &M.ref[2],
                                       &M.rf[0], &M.rf[1], &M.rf[2]);
            }
        }
    }
    if (pend0 >= 0) mbar_wait(&bar[0], ph0);
    if (pend1 >= 0) mbar_wait(&bar[1], ph1);
}

// ---- residual-plane variant without staging ------------------------------
// Thread (qx, qy) takes the luma quad at columns 2 qx, 2 qx + 1 and rows
// 2 qy, 2 qy + 1 and, with chroma, the co-sited pixel (qx, qy) of Cb and
// Cr, all from global memory (the reference samples of neighbouring
// threads share cache lines).  The arithmetic is the staged kernels':
// split_axis, the lerp steps of tile_lerp, the chroma flow
// ((f00 + f01) + (f10 + f11)) / 8 over the in-plane vectors, put_pixel.
__device__ __forceinline__ float lerp_global(const float *__restrict__ R, int pitch, int W, int H, int x, int y,
                                             float dx, float dy)
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

constexpr int kQX = 32, kQY = 4;  // quads per CTA: 32 x 4 (128 threads)

template <bool CHROMA>
__global__ void __launch_bounds__(kQX *kQY) pframe_rq_kernel(const __grid_constant__ FusedFrame F)
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
    const int yp = F.ref_pitch[0], op = F.out_pitch[0], rp = F.rfield_pitch[0];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = x0 + (q & 1), y = y0 + (q >> 1);
        if (!((q & 1) == 0 || in1) || !((q >> 1) == 0 || inr)) continue;
        const float pred = lerp_global(F.ref[0], yp, W, H, x, y, f[q].x, f[q].y);
        put_pixel(pred, __ldg(F.rfield[0] + (size_t)y * rp + x), F.ref_out[0] + (size_t)y * yp + x,
                  F.out[0] + (size_t)y * op + x);
    }
    if (CHROMA) {
        const int cw = (W + 1) / 2, ch = (H + 1) / 2;
        if (qx >= cw || qy >= ch) return;
        const int n = (1 + (int)in1) * (1 + (int)inr);
        const float sc = n == 4 ? 0.125f : (n == 2 ? 0.25f : 0.5f);
        const float dx = ((f[0].x + f[1].x) + (f[2].x + f[3].x)) * sc;
        const float dy = ((f[0].y + f[1].y) + (f[2].y + f[3].y)) * sc;
#pragma unroll
        for (int pl = 1; pl < 3; ++pl) {
            const float pred = lerp_global(F.ref[pl], F.ref_pitch[pl], cw, ch, qx, qy, dx, dy);
            put_pixel(pred, __ldg(F.rfield[pl] + (size_t)qy * F.rfield_pitch[pl] + qx),
                      F.ref_out[pl] + (size_t)qy * F.ref_pitch[pl] + qx, F.out[pl] + (size_t)qy * F.out_pitch[pl] + qx);
        }
    }
}

template <class Kern>
int occupancy(Kern k, size_t smem)
{
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, kThreads, smem) != cudaSuccess || o < 1) o = 1;
    return o;
}

template <bool C, int B, bool TMA>
cudaError_t launch_variant(FusedFrame &F, const FusedMaps *maps, uint32_t *flags, cudaLaunchConfig_t &cfg,
                           const BlockTables &t)
{
    static std::atomic<int> occ{0};
    int o = occ.load(std::memory_order_relaxed);
    if (o == 0) occ.store(o = occupancy(pframe_kernel<C, B, TMA>, kernel_smem<TMA>()), std::memory_order_relaxed);
    cfg.gridDim = dim3(std::max(1, std::min(F.nmb, t.sms * o)));
    cfg.dynamicSmemBytes = kernel_smem<TMA>();
    static const FusedMaps none{};
    const FusedMaps &m = maps ? *maps : none;
    return cudaLaunchKernelEx(&cfg, pframe_kernel<C, B, TMA>, F, m.flow, m.ref[0], m.ref[1], m.ref[2], t, flags);
}

template <bool C, int B, bool TMA>
cudaError_t allow_smem()
{
    return cudaFuncSetAttribute(pframe_kernel<C, B, TMA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kernel_smem<TMA>());
}

}  // namespace

bool fused_supported(int block) { return block == 16 || block == 8; }

cudaError_t fused_init()
{
    cudaError_t e;
    if ((e = allow_smem<true, 16, true>()) != cudaSuccess) return e;
    if ((e = allow_smem<false, 16, true>()) != cudaSuccess) return e;
    if ((e = allow_smem<true, 8, true>()) != cudaSuccess) return e;
    if ((e = allow_smem<false, 8, true>()) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(pframe_rf_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kRfSmem)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(pframe_rf_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRfSmem);
}

cudaError_t launch_pframe_rq(const FusedFrame &F, cudaStream_t st, bool pdl)
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
    if (F.chroma) return cudaLaunchKernelEx(&cfg, pframe_rq_kernel<true>, F);
    return cudaLaunchKernelEx(&cfg, pframe_rq_kernel<false>, F);
}

cudaError_t launch_pframe_rf(FusedFrame &F, const FusedMaps &maps, uint32_t *flags, cudaStream_t st, bool pdl)
{
    F.nmbx = (F.width + kMB - 1) / kMB;
    F.nmb = F.nmbx * ((F.height + kMB - 1) / kMB);
    const BlockTables &t = block_tables(F.op);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cfg.dynamicSmemBytes = kRfSmem;
    static std::atomic<int> occ[2] = {{0}, {0}};
    const int c = F.chroma ? 1 : 0;
    int o = occ[c].load(std::memory_order_relaxed);
    if (o == 0) {
        o = c ? occupancy(pframe_rf_kernel<true>, kRfSmem) : occupancy(pframe_rf_kernel<false>, kRfSmem);
        occ[c].store(o, std::memory_order_relaxed);
    }
    cfg.gridDim = dim3(std::max(1, std::min(F.nmb, t.sms * o)));
    if (c) return cudaLaunchKernelEx(&cfg, pframe_rf_kernel<true>, F, maps, flags);
    return cudaLaunchKernelEx(&cfg, pframe_rf_kernel<false>, F, maps, flags);
}

cudaError_t launch_pframe_fused(FusedFrame &F, const FusedMaps *maps, uint32_t *flags, cudaStream_t st, bool pdl)
{
    if (!fused_supported(F.block)) return cudaErrorInvalidValue;
    F.nmbx = (F.width + kMB - 1) / kMB;
    F.nmb = F.nmbx * ((F.height + kMB - 1) / kMB);
    const BlockTables &t = block_tables(F.op);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const bool c = F.chroma != 0;
    if (maps) {
        if (F.block == 16)
            return c ? launch_variant<true, 16, true>(F, maps, flags, cfg, t)
                     : launch_variant<false, 16, true>(F, maps, flags, cfg, t);
        return c ? launch_variant<true, 8, true>(F, maps, flags, cfg, t)
                 : launch_variant<false, 8, true>(F, maps, flags, cfg, t);
    }
    if (F.block == 16)
        return c ? launch_variant<true, 16, false>(F, maps, flags, cfg, t)
                 : launch_variant<false, 16, false>(F, maps, flags, cfg, t);
    return c ? launch_variant<true, 8, false>(F, maps, flags, cfg, t)
             : launch_variant<false, 8, false>(F, maps, flags, cfg, t);
}

}  // namespace hivc
