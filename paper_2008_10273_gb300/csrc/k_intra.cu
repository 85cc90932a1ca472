// Intra prediction: homogeneous diffusion inpainting (Sec. 2.1, Eq. 1) with
// A = -L, the 5-point Laplacian with reflecting boundaries, h = 1.
//
//   u_i = f_i on the mask,   (L u)_i = sum_{in-image nbrs j} (u_j - u_i) = 0 elsewhere.
//
// Correction loop (driven by the device; the host only launches it):
//   the iterate u is a float-float pair (hi + lo, ~48-bit significand);
//   r = (L u)_U is evaluated exactly enough for residuals down to ~1e-11
//   (u as 64-bit fixed point, the neighbour sum in integers), and stored
//   as FP32; the correction
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
//
// Control: an IntraCtl word block in device memory holds each plane's
// residual norm, observed contraction rate, relaxation factor and planned
// sweep launches.  The last CTA of every residual launch plans the next
// cycle (plan_cycle) and the first CTA of every sweep launch hands the pair
// count on (pair_step); both set the handles of a CUDA graph with two nested
// conditional WHILE nodes (cycles; sweep launches in pairs of fixed
// parity), so a whole solve is one graph launch with no host round trip,
// and convergence is read at the decoder's sync.  Sweep launches read the
// plan beside their first data loads and return at once when their plane
// has no sweep left in this cycle.  No CTA ever waits for another.
#include <algorithm>
#include <atomic>
#include <vector>
#include <mutex>
#include <map>
#include <cfloat>

#include "hivc_internal.cuh"

namespace hivc {
namespace {

// ---- SOR tile geometry ---------------------------------------------------
constexpr int kS = 4;                   // full sweeps per launch
constexpr int kHL = 2 * kS;             // halo
// staged region RW x kRH (RW = 128 or 112 columns: the launcher picks the
// faster one per plane geometry), output (RW - 2 kHL) x (kRH - 2 kHL)
constexpr int kRH = 128;
constexpr int kTY = kRH - 2 * kHL;      // 112 output rows
constexpr int kTY_THREADS = 16;         // thread rows; each thread owns kRH/16 consecutive rows
constexpr int kRows = kRH / kTY_THREADS;
// the chroma phase's regions: 128 x 88 staged, 112 x 72 output, 11 thread
// rows (the two 960 x 540 planes of FullHD 4:2:0 in 144 regions, one wave)
constexpr int kRHc = 88;
__host__ __device__ constexpr int sor_tx(int rw) { return rw - 2 * kHL; }
__host__ __device__ constexpr size_t sor_smem_bytes(int rw, int rh = kRH)
{
    return 2 * (rh + 2) * (rw / 2 + 2) * sizeof(float);  // bordered colour arrays
}
// pairs of sweep launches a cycle may plan, and cycles a solve may run: a
// loop condition never stays set beyond these, whatever the control state
// or the configuration holds
constexpr int kMaxPairs = 1 << 14;
constexpr int kMaxCycles = 1000;

// residual tile: 64 x 20 (FullHD 4:2:0 planes split into whole tiles
// vertically, 2,430 of them: 4 waves of 4 CTAs per SM on 152 SMs)
constexpr int kRTW = 64, kRTH = 20;
constexpr int kResThreads = kRTW / 4 * kRTH;

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

// sum of mask values (exact, integer; signed for RCT chroma) + index
// validation; plane = blockIdx.y
__global__ void intra_sum_kernel(const __grid_constant__ IntraJobs J, uint32_t *flags)
{
    const IntraPlane &P = J.p[blockIdx.y];
    const uint32_t N = (uint32_t)P.width * (uint32_t)P.height;
    unsigned long long s = 0;
    bool bad = false;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.n; k += gridDim.x * blockDim.x) {
        const uint32_t i = __ldg(P.idx + k);
        bad |= (i >= N) || (k > 0 && __ldg(P.idx + k - 1) >= i);
        // two's complement: signed values add correctly modulo 2^64
        s += P.val16 ? (unsigned long long)(long long)__ldg(P.val16 + k) : (unsigned long long)__ldg(P.val + k);
    }
    // one atomic per CTA (the launch has a point per thread)
    __shared__ unsigned long long s_part[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flags, kFlagMaskIdx);
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        if (t) atomicAdd(P.vsum, t);
    }
}

// the mean mask value of plane P, formed once per CTA (one thread's
// double-precision division) and shared
__device__ __forceinline__ float plane_mean(const IntraPlane &P)
{
    __shared__ float s_mean;
    if (threadIdx.x == 0 && threadIdx.y == 0) s_mean = P.n > 0 ? (float)((double)(long long)*P.vsum / (double)P.n) : 0.f;
    __syncthreads();
    return s_mean;
}

// u = mean mask value (hi), lo = 0, mask = 0
__global__ void intra_fill_kernel(const __grid_constant__ IntraJobs J)
{
    const IntraPlane &P = J.p[blockIdx.y];
    const float mean = plane_mean(P);
    // 4 pixels a thread (rows are multiples of 32 pixels)
    const size_t total = (size_t)P.height * P.pitch / 4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        reinterpret_cast<float4 *>(P.uh[0])[i] = make_float4(mean, mean, mean, mean);
        reinterpret_cast<float4 *>(P.ul[0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        reinterpret_cast<uint32_t *>(P.mask)[i] = 0u;
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
        P.uh[0][o] = P.val16 ? (float)__ldg(P.val16 + k) : (float)__ldg(P.val + k);
        P.mask[o] = 1;
    }
}

// ---- the coarse start ------------------------------------------------------
// A two-level cascade for the starting iterate: coarse pixel (X, Y) of a
// plane covers the fine pixels 2X .. 2X + 1 x 2Y .. 2Y + 1.  It is known
// when one of them is, with the mean of their values; otherwise it starts
// at the plane's mean mask value.  (Fine planes after the scatter, whose
// row padding holds mask 0; plane = blockIdx.z.)  Thread (x, y) of the
// 32 x 8 CTAs takes the coarse pixels 4 t .. 4 t + 3 of row Y (t the
// thread's column), reading the eight fine mask bytes of each fine row at
// once.
__global__ void intra_restrict_kernel(const __grid_constant__ IntraJobs F, const __grid_constant__ IntraJobs C)
{
    const IntraPlane &Pf = F.p[blockIdx.z];
    const IntraPlane &Pc = C.p[blockIdx.z];
    const float mean = plane_mean(Pf);
    const int X4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x), Y = blockIdx.y * blockDim.y + threadIdx.y;
    if (X4 >= Pc.width || Y >= Pc.height) return;
    uint2 m[2];
    for (int dy = 0; dy < 2; ++dy) {
        const int y = 2 * Y + dy;
        m[dy] = y < Pf.height ? __ldg(reinterpret_cast<const uint2 *>(Pf.mask + (size_t)y * Pf.pitch + 2 * X4))
                              : make_uint2(0u, 0u);
    }
    float v[4];
    uint32_t known = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float s = 0.f;
        int k = 0;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int b = 2 * j + dx;  // byte of the row's eight
                const uint32_t w = b < 4 ? m[dy].x : m[dy].y;
                if ((w >> (8 * (b & 3))) & 0xffu) {
                    s += __ldg(Pf.uh[0] + (size_t)(2 * Y + dy) * Pf.pitch + 2 * X4 + b);
                    ++k;
                }
            }
        v[j] = k ? s / (float)k : mean;
        known |= (k ? 1u : 0u) << (8 * j);
    }
    const size_t oc = (size_t)Y * Pc.pitch + X4;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (X4 + j < Pc.width) {
            Pc.uh[0][oc + j] = v[j];
            Pc.mask[oc + j] = (known >> (8 * j)) & 1u;
        }
}

// The unknown fine pixels from the coarse solution (the iterate buffer the
// coarse control state names): bilinear between coarse cell centres (fine
// x at coarse (x - 1/2) / 2), the edge cells replicated.  lo stays 0 (the
// fill kernel's); the mask pixels keep their values.  Thread (x, y) of the
// 32 x 8 CTAs takes fine pixels 4 t .. 4 t + 3 of row y (t the thread's
// column): one 4-byte mask load, then all their samples.
__global__ void intra_prolong_kernel(const __grid_constant__ IntraJobs F, const __grid_constant__ IntraJobs C)
{
    const IntraPlane &Pf = F.p[blockIdx.z];
    const IntraPlane &Pc = C.p[blockIdx.z];
    const int x4 = 4 * (blockIdx.x * blockDim.x + threadIdx.x), y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x4 >= Pf.width || y >= Pf.height) return;
    const float *__restrict__ uc = Pc.uh[C.ctl->upar[blockIdx.z] & 1];
    const int Wc = Pc.width, Hc = Pc.height;
    const size_t o = (size_t)y * Pf.pitch + x4;
    const uint32_t m = __ldg(reinterpret_cast<const uint32_t *>(Pf.mask + o));
    const float ys = 0.5f * (float)y - 0.25f, fy = floorf(ys), ay = ys - fy;
    const int y0 = (int)fy;
    const int ya = min(max(y0, 0), Hc - 1), yb = min(max(y0 + 1, 0), Hc - 1);
    const float *ra = uc + (size_t)ya * Pc.pitch, *rb = uc + (size_t)yb * Pc.pitch;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int x = x4 + j;
        if (x >= Pf.width || ((m >> (8 * j)) & 0xffu)) continue;
        const float xs = 0.5f * (float)x - 0.25f, fx = floorf(xs), ax = xs - fx;
        const int x0 = (int)fx;
        const int xa = min(max(x0, 0), Wc - 1), xb = min(max(x0 + 1, 0), Wc - 1);
        const float a0 = __ldg(ra + xa), a1 = __ldg(ra + xb), b0 = __ldg(rb + xa), b1 = __ldg(rb + xb);
        const float top = fmaf(ax, a1 - a0, a0), bot = fmaf(ax, b1 - b0, b0);
        Pf.uh[0][o + j] = fmaf(ay, bot - top, top);
    }
}

// ---- control of the correction loop, on the device ------------------------
// The region of CTA b among the regions of the planes that work in this
// launch (a sweep launch: launch index it < the plane's launch count; a
// residual launch: every plane at the start, else the planes that swept),
// in plane order: the working CTAs come first in the grid and the rest,
// past them, exit at once.  Returns the plane (and lt, the region within
// it), or -1.
__device__ __forceinline__ int active_region(const IntraJobs &J, const IntraCtl *c, int it, bool residual, int b,
                                             int &lt)
{
    int base = 0;
    for (int p = 0; p < J.n; ++p) {
        const bool on = residual ? (it != 0 || c->nl[p] > 0) : it < c->nl[p];
        if (!on) continue;
        if (b < base + J.p[p].tiles) {
            lt = b - base;
            return p;
        }
        base += J.p[p].tiles;
    }
    lt = 0;
    return -1;
}

// Whether the calling CTA is the last of its launch to finish (every CTA
// calls this once, after its work; no CTA waits).  The last one resets the
// count for the next launch.
__device__ __forceinline__ bool last_cta(IntraCtl *c, int *s_flag)
{
    __syncthreads();
    // no fence: the last CTA reads no other CTA's plain stores (the residual
    // norms are atomics, the next launch sees every store)
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned total = gridDim.x * gridDim.y;
        const bool last = atomicAdd(&c->done_ctas, 1u) == total - 1;
        if (last) c->done_ctas = 0;
        *s_flag = last;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Planning after a residual launch (one thread): take each swept plane's
// residual norm; at the end of a cycle adapt the plane's relaxation factor
// (slower than optimal SOR at this omega predicts means omega is below the
// optimum; Young's relation (rho + omega - 1)^2 = rho omega^2 mu^2 gives the
// Jacobi radius mu and the optimal omega); then plan the next cycle: each
// plane above the tolerance sweeps towards the FP32 floor of the inner
// solve (about 1e-5) or the remaining gap to the tolerance, whichever is
// smaller, at the rate of optimally relaxed SOR, omega - 1.
// c is the launch's last CTA's shared-memory copy of the control block
// (plan_cycle_cta), rb each plane's max |residual| of the launch.
__device__ void plan_cycle(const IntraJobs &J, IntraCtl &c, const float *rb, bool first)
{
    // (single precision throughout: the plan needs a few digits, and one
    // thread's chain of double-precision divisions, pow and log would sit on
    // every cycle's tail; rn holds FP32 values)
    for (int p = 0; p < J.n; ++p) {
        if (!first && c.nl[p] == 0) continue;
        const float v = rb[p];
        c.res_pixels += (long long)J.p[p].width * J.p[p].height;
        if (first) {
            c.rn[p] = v;
            c.rate[p] = c.omega[p] - 1.f;
            continue;
        }
        const float q = v / fmaxf((float)c.rn[p], 1e-30f);
        c.rn[p] = v;
        const int S = c.nl[p] * c.spl;
        c.sweeps[p] += S;
        c.sweeps_max = max(c.sweeps_max, c.sweeps[p]);
        c.upar[p] ^= 1;  // the launch wrote u + e to the other buffer
        if (q > 1e-4f && q < 1.f) {
            const float ro = powf(q, 1.f / (float)S);
            const float om = c.omega[p];
            if (ro > (float)c.rate[p] + 0.01f) {
                const float mu = (ro + om - 1.f) / (om * sqrtf(ro));
                if (mu < 1.f) {
                    const float on = 2.f / (1.f + sqrtf(1.f - mu * mu));
                    c.omega[p] = fminf(1.98f, fmaxf(om, on));
                }
                c.rate[p] = fmaxf(c.omega[p] - 1.f, fminf(ro, 0.995f));
                if (c.omega[p] > om) c.rate[p] = c.omega[p] - 1.f;
            }
        }
    }
    c.res_launches += 1;
    if (!first) c.cycles += 1;
    int maxl = 0;
    bool conv = true;
    for (int p = 0; p < J.n; ++p) {
        c.nl[p] = 0;
        // (the test against the tolerance itself in double precision)
        conv = conv && c.rn[p] <= c.tol;
        if (!(c.rn[p] > c.tol)) continue;
        const float target = fmaxf(1e-5f, 0.3f * (float)c.tol / (float)c.rn[p]);
        const float rt = fminf(fmaxf((float)c.rate[p], 0.05f), 0.995f);
        int sw = (int)ceilf(logf(target) / logf(rt));
        sw = min(max(sw, c.spl), c.max_sweeps);
        c.nl[p] = (sw + c.spl - 1) / c.spl;
        maxl = max(maxl, c.nl[p]);
    }
    c.maxl = maxl;
    c.iter[0] = c.iter[1] = 0;
    // the launch pairs: with the chroma phase, the all-plane launches while
    // luma sweeps (at least one pair: each loop runs at least once), then
    // the chroma planes alone with regions of their own
    int pa = (maxl + 1) / 2, pb = 0;
    if (J.chroma_phase && J.n == 3) {
        const int nc = max(c.nl[1], c.nl[2]);
        pa = max(1, (c.nl[0] + 1) / 2);
        pb = nc > 2 * pa ? (nc - 2 * pa + 1) / 2 : 0;
    }
    c.pairs[0] = min(pa, kMaxPairs);
    c.pairs[1] = min(pb, kMaxPairs);
    c.converged = conv ? 1 : 0;
    const int go = (maxl > 0 && c.cycles < c.max_cycles && c.cycles < kMaxCycles) ? 1 : 0;
    c.go_outer = go;
    if (!go && !conv) c.unconverged += 1;
    if (go) {  // the next cycle's sweep launches (in pairs) and the pixels they sweep
        c.sor_launches += 2 * (c.pairs[0] + (J.chroma_phase && J.n == 3 ? max(c.pairs[1], 1) : 0));
        for (int p = 0; p < J.n; ++p) c.sor_pixels += (long long)c.nl[p] * J.p[p].width * J.p[p].height;
    }
    if (J.h_outer) cudaGraphSetConditional(J.h_outer, go);
    // the sweep loops of the next cycle start open (the last sweep launch of
    // each closed it): each loop runs at least one pair per cycle
    if (J.h_inner) cudaGraphSetConditional(J.h_inner, go);
    if (J.h_inner_c) cudaGraphSetConditional(J.h_inner_c, go);
}

// The plan, by the launch's last CTA: the control block is copied to
// shared memory a word per thread (one round of loads instead of a chain
// of round trips to L2 on the launch's tail), each plane's max |residual|
// read (and cleared for the next launch) by an atomic at L2, past any
// stale L1 line, then one thread plans, and the block goes back a word per
// thread.  During the plan no other CTA of the launch touches the block
// (they made their atomics before counting themselves done).
constexpr int kCtlWords = sizeof(IntraCtl) / 4;
static_assert(sizeof(IntraCtl) % 8 == 0, "the control block is copied in 4-byte words");
__device__ __forceinline__ void plan_cycle_cta(const IntraJobs &J, bool first)
{
    __shared__ __align__(8) uint32_t s_words[kCtlWords];
    __shared__ float s_rb[3];
    uint32_t *g = reinterpret_cast<uint32_t *>(J.ctl);
    const int t = threadIdx.x + threadIdx.y * blockDim.x, nt = blockDim.x * blockDim.y;
    for (int k = t; k < kCtlWords; k += nt) s_words[k] = g[k];
    if (t < 3) s_rb[t] = t < J.n ? __uint_as_float(atomicExch(J.ctl->rbits + t, 0u)) : 0.f;
    __syncthreads();
    IntraCtl &c = *reinterpret_cast<IntraCtl *>(s_words);
    if (t == 0) {
        c.rbits[0] = c.rbits[1] = c.rbits[2] = 0u;
        c.done_ctas = 0;  // as the last CTA left it
        plan_cycle(J, c, s_rb, first);
    }
    __syncthreads();
    for (int k = t; k < kCtlWords; k += nt) g[k] = s_words[k];
}

// The control state of a new solve (one thread).
__global__ void intra_ctl_init_kernel(IntraCtl *c, float om0, float om1, float om2, double tol, int max_cycles,
                                      int spl, int max_sweeps)
{
    IntraCtl z{};
    z.sor_launches = c->sor_launches;  // the statistics run on until the sync
    z.sor_pixels = c->sor_pixels;
    z.res_launches = c->res_launches;
    z.res_pixels = c->res_pixels;
    z.unconverged = c->unconverged;
    z.tol = tol;
    z.max_cycles = max_cycles;
    z.spl = spl;
    z.max_sweeps = max_sweeps;
    z.omega[0] = om0;
    z.omega[1] = om1;
    z.omega[2] = om2;
    *c = z;
}

// The iterate hi + lo as a 64-bit fixed-point number of 2^-40 grey levels
// (|u| < 2^23: the sum of four neighbours cannot overflow).  hi * 2^40 is
// exact and an integer for |hi| >= 2^-16; the rounding of lo * 2^40 (and
// of hi * 2^40 below 2^-16) is at most 2^-41 grey levels, far below the
// residuals the solve aims at, and the sums of these integers are exact.
constexpr float kFix = 1099511627776.f;     // 2^40
constexpr float kUnfix = 1.f / kFix;        // 2^-40, exact
__device__ __forceinline__ long long to_fix(float h, float l)
{
    return __float2ll_rn(h * kFix) + __float2ll_rn(l * kFix);
}

// u_out = u_in + e (unknown pixels; float-float), res = (L u_out)_i, and the
// max |res| per plane; first: res = (L u)_i of the starting iterate.  A 64 x
// 20 tile with a one-pixel halo is updated once per cell into shared
// memory, as fixed-point integers (to_fix); the residual of a pixel is the
// exact integer sum of its neighbours' differences, rounded once to FP32.
// Thread t takes the columns t % 16 + 16 j (j = 0..3) of tile row t / 16
// (a warp reads 64 contiguous bytes per row and load, and its shared-memory
// accesses hit consecutive words); threads 0..31 also take the same
// columns of the halo rows above and below the tile, threads 32..71 a cell
// of the halo columns left and right of it.  Every load of a thread is
// issued before any of its arithmetic.  Cells outside the plane count as
// 0 and are never written.  Planes that the plan leaves out this cycle
// (converged) are skipped.  The launch's last CTA plans the next cycle.
constexpr int kRQ = kRTW / 4;  // threads per tile row (4 columns each)
static_assert(kRQ * kRTH == kResThreads && 2 * kRQ + 2 * kRTH <= kResThreads, "4 cells per thread");

__global__ void __launch_bounds__(kResThreads, 4) intra_residual_kernel(const __grid_constant__ IntraJobs J, int first)
{
    __shared__ long long su[kRTH + 2][kRTW + 2];
    __shared__ float red[kResThreads / 32];
    __shared__ int s_last;
    IntraCtl *c = J.ctl;
    int lt;
    const int pl = active_region(J, c, first, true, blockIdx.x, lt);
    const bool add_e = !first;
    if (pl >= 0) {
        const IntraPlane &P = J.p[pl];
        const int x0 = (lt % P.tiles_x) * kRTW, y0 = (lt / P.tiles_x) * kRTH;
        const int W = P.width, H = P.height, pitch = P.pitch;
        const int up = c->upar[pl];
        const float *uh = P.uh[up], *ul = P.ul[up];
        float *uh_out = P.uh[up ^ 1], *ul_out = P.ul[up ^ 1];
        const float *e = P.e[c->nl[pl] & 1];  // after the cycle's nl launches; zero on the mask
        const bool ff = P.ff != 0;
        const int t = threadIdx.x, ty = t / kRQ, tx = t % kRQ;
        const int gy = y0 + ty, gx = x0 + tx;
        const bool rin = gy < H;
        const size_t i = (size_t)gy * pitch + gx;  // column j at i + kRQ j
        // the halo: row hr (0 above, kRTH + 1 below) at the thread's
        // columns, or the cell of column hc (0 left, kRTW + 1 right) in tile
        // row ck
        const bool hrow = t < 2 * kRQ, hcol = !hrow && t < 2 * kRQ + 2 * kRTH;
        const int hr = t < kRQ ? 0 : kRTH + 1, hy = y0 - 1 + hr;
        const int ck = (t - 2 * kRQ) % kRTH, hc = t - 2 * kRQ < kRTH ? 0 : kRTW + 1;
        const int cy = y0 + ck, cx = x0 - 1 + hc;
        const bool hin = hrow && hy >= 0 && hy < H;
        const bool cin = hcol && cy < H && cx >= 0 && cx < W;
        const size_t ih = (size_t)hy * pitch + gx, ic = (size_t)cy * pitch + cx;
        float h[4], l[4], d[4], hh[4], hl[4], hd[4];
        uint8_t m[4];
        float ch = 0.f, cl = 0.f, cd = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool in = rin && gx + kRQ * j < W, inh = hin && gx + kRQ * j < W;
            h[j] = in ? __ldg(uh + i + kRQ * j) : 0.f;
            l[j] = in && ff ? __ldg(ul + i + kRQ * j) : 0.f;
            d[j] = in && add_e ? __ldg(e + i + kRQ * j) : 0.f;
            m[j] = in ? __ldg(P.mask + i + kRQ * j) : 1;
            hh[j] = inh ? __ldg(uh + ih + kRQ * j) : 0.f;
            hl[j] = inh && ff ? __ldg(ul + ih + kRQ * j) : 0.f;
            hd[j] = inh && add_e ? __ldg(e + ih + kRQ * j) : 0.f;
        }
        if (cin) {
            ch = __ldg(uh + ic);
            if (ff) cl = __ldg(ul + ic);
            if (add_e) cd = __ldg(e + ic);
        }
        // u + e of one cell (cells outside the plane hold 0 and stay 0; e
        // is 0 there), into h, l; returns it as fixed point
        auto update = [ff, add_e](float &h, float &l, float d) {
            if (add_e) {
                if (ff) ff_add(h, l, d, h, l);
                else h = __fadd_rn(h, d);
            }
            return to_fix(h, l);
        };
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            su[ty + 1][tx + kRQ * j + 1] = update(h[j], l[j], d[j]);
            if (hrow) su[hr][tx + kRQ * j + 1] = update(hh[j], hl[j], hd[j]);
        }
        if (hcol) su[ck + 1][hc] = update(ch, cl, cd);
        if (add_e) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (rin && gx + kRQ * j < W) {
                    uh_out[i + kRQ * j] = h[j];
                    if (ff) ul_out[i + kRQ * j] = l[j];
                }
        }
        __syncthreads();
        float rmax = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = gx + kRQ * j, lx = tx + kRQ * j + 1;
            if (!rin || x >= W) continue;
            float r = 0.f;
            if (!m[j]) {
                // sum_j (u_j - u_i), exact in fixed point, rounded once
                const long long uc = su[ty + 1][lx];
                long long acc = 0;
                if (x > 0) acc += su[ty + 1][lx - 1] - uc;
                if (x < W - 1) acc += su[ty + 1][lx + 1] - uc;
                if (gy > 0) acc += su[ty][lx] - uc;
                if (gy < H - 1) acc += su[ty + 2][lx] - uc;
                r = __ll2float_rn(acc) * kUnfix;
            }
            P.res[i + kRQ * j] = r;
            rmax = fmaxf(rmax, fabsf(r));
        }
        for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = rmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.f;
            for (int w = 0; w < kResThreads / 32; ++w) m = fmaxf(m, red[w]);
            if (m > 0.f) atomicMax(c->rbits + pl, __float_as_uint(m));  // non-negative floats order like their bits
        }
    }
    if (!last_cta(c, &s_last)) return;
    plan_cycle_cta(J, first != 0);
}

// S red-black SOR sweeps on (-L_UU) e = res in a shared-memory tile.
// Thread (hx, ty) owns the cell pair hx (columns 2hx, 2hx+1) in the eight
// consecutive rows 8 ty .. 8 ty + 7.  Its cells' values stay in registers,
// indexed by colour: of the four neighbours of a cell, the vertical ones
// and one horizontal one are the thread's own cells (except at its first
// and last row), so a cell update reads one or two values from shared
// memory, where every cell's latest value is kept by colour for the
// neighbouring threads.  The colour arrays have a one-cell border, so the
// staged region's outer ring is updated like any cell (from border
// values): its values are not exact after the first half sweep, but
// exactness shrinks by one ring per half sweep anyway, and the 2S half
// sweeps leave the interior, kHL = 2S rings in, exact.  Tile corners are
// even (kTX, kTY, kHL even), so a cell's colour is known at compile time.
// Launch it = 2 i + PAR of the cycle: sweeps from e[PAR] (from zero at
// it = 0) into e[PAR ^ 1].  The control words (i, the plane's launch
// count, omega) are read beside the region's data loads, which do not
// depend on them; a plane without this launch returns false before it
// writes anything.
template <int RW, int RH, int PAR>
__device__ __forceinline__ bool sor_body(const IntraPlane &P, int pl, int lt, const IntraCtl *c)
{
    constexpr int HW = RW / 2, TX = sor_tx(RW);  // cells per colour and row; output columns
    constexpr int TY = RH - 2 * kHL, TROWS = RH / kRows;  // output rows; thread rows
    static_assert(TX % 2 == 0 && TY % 2 == 0 && kHL % 2 == 0 && RH % kRows == 0, "tiles start on even cells");
    extern __shared__ float sor_smem[];
    auto E = reinterpret_cast<float(*)[RH + 2][HW + 2]>(sor_smem);
    const int it = 2 * c->iter[PAR] + PAR, nlp = c->nl[pl];
    const float omega = c->omega[pl];
    const int tx0 = (lt % P.tiles_x) * TX, ty0 = (lt / P.tiles_x) * TY;
    const int gx0 = tx0 - kHL, gy0 = ty0 - kHL;
    const int W = P.width, H = P.height, pitch = P.pitch;
    const int hx = threadIdx.x, ty = threadIdx.y, ly0 = ty * kRows;
    const float *ein = P.e[PAR];
    float *eout = P.e[PAR ^ 1];
    // The pair starts at an even column (tx0 and the halo are even), so its
    // two cells are read as one 2-element vector.
    const int gxp = gx0 + 2 * hx;
    const bool in0 = gxp >= 0 && gxp < W, in1 = gxp >= 0 && gxp + 1 < W;
    // ec[k][c]: value of the thread's colour-c cell in row ly0 + k, which
    // sits at column 2 hx + ((c + k) & 1); wi = omega / n and wr = omega r / n
    // for unknown cells, 0 for fixed ones (whose value is 0 and stays 0)
    float ec[kRows][2], wi[kRows][2], wr[kRows][2];
    // A region with every cell inside the image and off its border (all
    // cells have four neighbours): plain loads, n = 4.
    const bool interior = gx0 >= 1 && gy0 >= 1 && gx0 + RW <= W - 1 && gy0 + RH <= H - 1;
    bool fz = false;
    float omc = 0.f;
    if (interior) {
        const size_t i0 = (size_t)(gy0 + ly0) * pitch + gxp;
        uint32_t m2[kRows];
        float2 r2[kRows], e2[kRows];
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const size_t i = i0 + (size_t)k * pitch;
            m2[k] = __ldg(reinterpret_cast<const unsigned short *>(P.mask + i));
            r2[k] = __ldg(reinterpret_cast<const float2 *>(P.res + i));
            e2[k] = __ldg(reinterpret_cast<const float2 *>(ein + i));
        }
        if (it >= nlp) return false;
        fz = it == 0;
        omc = 1.f - omega;
        const float w4 = 0.25f * omega;
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            float ev[2], iv[2], rv[2];
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const bool unk = ((m2[k] >> (8 * b)) & 0xffu) == 0;
                iv[b] = unk ? w4 : 0.f;
                rv[b] = (b ? r2[k].y : r2[k].x) * iv[b];
                ev[b] = (fz || !unk) ? 0.f : (b ? e2[k].y : e2[k].x);
            }
            const int sw = k & 1;  // 1: the pair's left cell has colour 1 (ly0 is even)
            ec[k][0] = ev[sw];
            ec[k][1] = ev[sw ^ 1];
            wi[k][0] = iv[sw];
            wi[k][1] = iv[sw ^ 1];
            wr[k][0] = rv[sw];
            wr[k][1] = rv[sw ^ 1];
        }
    } else {
        // Every load is issued unconditionally from a clamped address (rows
        // into [0, H), the pair into the pitch) and cells outside the image
        // are zeroed afterwards, so that all of them are in flight together.
        const int gxc = min(max(gxp, 0), pitch - 2);
        uint32_t m2[kRows];
        float2 r2[kRows], e2[kRows];
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const int gy = min(max(gy0 + ly0 + k, 0), H - 1);
            const size_t i = (size_t)gy * pitch + gxc;
            m2[k] = __ldg(reinterpret_cast<const unsigned short *>(P.mask + i));
            r2[k] = __ldg(reinterpret_cast<const float2 *>(P.res + i));
            e2[k] = __ldg(reinterpret_cast<const float2 *>(ein + i));
        }
        if (it >= nlp) return false;
        fz = it == 0;
        omc = 1.f - omega;
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const int gy = gy0 + ly0 + k;
            const bool yin = gy >= 0 && gy < H;
            const int ny = (gy > 0) + (gy < H - 1);
            float ev[2], iv[2], rv[2];
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const int gx = gxp + b;
                const bool unk = yin && (b ? in1 : in0) && ((m2[k] >> (8 * b)) & 0xffu) == 0;
                const int n = ny + (gx > 0) + (gx < W - 1);
                const float inv = n == 4 ? 0.25f : (n == 3 ? (1.0f / 3.0f) : (n == 2 ? 0.5f : 1.0f));
                iv[b] = unk ? omega * inv : 0.f;
                rv[b] = unk ? (b ? r2[k].y : r2[k].x) * iv[b] : 0.f;
                ev[b] = (fz || !unk) ? 0.f : (b ? e2[k].y : e2[k].x);
            }
            const int sw = k & 1;
            ec[k][0] = ev[sw];
            ec[k][1] = ev[sw ^ 1];
            wi[k][0] = iv[sw];
            wi[k][1] = iv[sw ^ 1];
            wr[k][0] = rv[sw];
            wr[k][1] = rv[sw ^ 1];
        }
    }
    // the border of the colour arrays: finite values
    for (int k = hx + ty * HW; k < 2 * (RH + 2); k += HW * TROWS) {
        E[k & 1][k >> 1][0] = 0.f;
        E[k & 1][k >> 1][HW + 1] = 0.f;
    }
    for (int k = hx + ty * HW; k < 2 * (HW + 2); k += HW * TROWS) {
        E[k & 1][0][k >> 1] = 0.f;
        E[k & 1][RH + 1][k >> 1] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        E[0][ly0 + k + 1][hx + 1] = ec[k][0];
        E[1][ly0 + k + 1][hx + 1] = ec[k][1];
    }
    __syncthreads();
#pragma unroll
    for (int m = 1; m <= 2 * kS; ++m) {
        const int c = (m - 1) & 1, o = c ^ 1;  // red (even x + y) first
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const int ly = ly0 + k + 1;      // row in the bordered arrays
            const int b = (c + k) & 1;       // column of the colour-c cell in the pair
            const float up = k > 0 ? ec[k - 1][o] : E[o][ly - 1][hx + 1];
            const float dn = k < kRows - 1 ? ec[k + 1][o] : E[o][ly + 1][hx + 1];
            const float s = (ec[k][o] + E[o][ly][hx + 2 * b]) + (up + dn);
            // e <- (1 - omega) e + omega (s + r) / n
            ec[k][c] = fmaf(s, wi[k][c], fmaf(omc, ec[k][c], wr[k][c]));
            E[c][ly][hx + 1] = ec[k][c];
        }
        __syncthreads();
    }
    // interior pairs are whole pairs (even halo and width); a pair that
    // straddles an odd right edge writes its left cell only
    const int lx = 2 * hx;
    if (lx < kHL || lx >= kHL + TX || gxp >= W) return true;
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int ly = ly0 + k, gy = gy0 + ly;
        if (ly < kHL || ly >= kHL + TY || gy >= H) continue;
        const int sw = k & 1;
        const float v0 = sw ? ec[k][1] : ec[k][0], v1 = sw ? ec[k][0] : ec[k][1];
        float *o = eout + (size_t)gy * pitch + gxp;
        if (in1) *reinterpret_cast<float2 *>(o) = make_float2(v0, v1);
        else o[0] = v0;
    }
    return true;
}

// The same sweeps with four columns per thread: a warp spans the region's
// 128 columns (lane t holds columns 4t .. 4t+3) in 8 rows, 16 warps.  Of a
// cell's horizontal neighbours one may sit in the next lane (a shuffle; the
// region border is 0 beyond lanes 0 and 31), the vertical ones of the
// warp's first and last row in the next warp (shared rows, written after
// each half sweep, then a barrier).  The neighbour sum is formed as
// (left + right) + (up + down) and the update as in intra_sor_kernel, so
// the results are the same bit for bit.
constexpr int kQWarps = kRH / kRows;  // 16 row groups of 8 rows
constexpr int kQCols = 128;           // region columns, 4 per lane

// (launch parity, control words and the early return as in sor_body)
template <int PAR>
__device__ __forceinline__ bool sor4_body(const IntraPlane &P, int pl, int lt, const IntraCtl *c)
{
    constexpr int TX = sor_tx(kQCols);
    __shared__ float rows[kQWarps][2][kQCols];  // each warp's first and last row
    const int it = 2 * c->iter[PAR] + PAR, nlp = c->nl[pl];
    const float omega = c->omega[pl];
    const int tx0 = (lt % P.tiles_x) * TX, ty0 = (lt / P.tiles_x) * kTY;
    const int gx0 = tx0 - kHL, gy0 = ty0 - kHL;
    const int W = P.width, H = P.height, pitch = P.pitch;
    const int lane = threadIdx.x, wq = threadIdx.y, ly0 = wq * kRows;
    const float *ein = P.e[PAR];
    float *eout = P.e[PAR ^ 1];
    const int gxq = gx0 + 4 * lane;  // a multiple of 4: the quad is one 16-byte vector
    // e[k][j], wi[k][j], wr[k][j]: the cell in row ly0 + k, column 4 lane + j
    float e[kRows][4], wi[kRows][4], wr[kRows][4];
    const bool interior = gx0 >= 1 && gy0 >= 1 && gx0 + kQCols <= W - 1 && gy0 + kRH <= H - 1;
    const int gxc = min(max(gxq, 0), pitch - 4);
    uint32_t m4[kRows];
    float4 r4[kRows], e4[kRows];
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int gy = interior ? gy0 + ly0 + k : min(max(gy0 + ly0 + k, 0), H - 1);
        const size_t i = (size_t)gy * pitch + (interior ? gxq : gxc);
        m4[k] = __ldg(reinterpret_cast<const unsigned int *>(P.mask + i));
        r4[k] = __ldg(reinterpret_cast<const float4 *>(P.res + i));
        e4[k] = __ldg(reinterpret_cast<const float4 *>(ein + i));
    }
    if (it >= nlp) return false;
    const bool fz = it == 0;
    const float omc = 1.f - omega;
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int gy = gy0 + ly0 + k;
        const bool yin = gy >= 0 && gy < H;
        const int ny = (gy > 0) + (gy < H - 1);
        const float rr[4] = {r4[k].x, r4[k].y, r4[k].z, r4[k].w};
        float ee[4] = {0.f, 0.f, 0.f, 0.f};
        if (!fz) {
            ee[0] = e4[k].x;
            ee[1] = e4[k].y;
            ee[2] = e4[k].z;
            ee[3] = e4[k].w;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gx = gxq + j;
            bool unk;
            float iv;
            if (interior) {
                unk = ((m4[k] >> (8 * j)) & 0xffu) == 0;
                iv = unk ? 0.25f * omega : 0.f;
            } else {
                unk = yin && gx >= 0 && gx < W && ((m4[k] >> (8 * j)) & 0xffu) == 0;
                const int n = ny + (gx > 0) + (gx < W - 1);
                const float inv = n == 4 ? 0.25f : (n == 3 ? (1.0f / 3.0f) : (n == 2 ? 0.5f : 1.0f));
                iv = unk ? omega * inv : 0.f;
            }
            wi[k][j] = iv;
            wr[k][j] = unk ? rr[j] * iv : 0.f;
            e[k][j] = (fz || !unk) ? 0.f : ee[j];
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        rows[wq][0][4 * lane + j] = e[0][j];
        rows[wq][1][4 * lane + j] = e[kRows - 1][j];
    }
    __syncthreads();
#pragma unroll
    for (int m = 1; m <= 2 * kS; ++m) {
        const int c = (m - 1) & 1;  // red (even x + y) first
#pragma unroll
        for (int k = 0; k < kRows; ++k) {
            const int b = (c + k) & 1;  // the colour-c cells of the row: columns b and b + 2
            // the neighbour beyond the quad on the needed side (every lane shuffles)
            float beyond;
            if (b == 0) {
                beyond = __shfl_up_sync(0xffffffffu, e[k][3], 1);
                if (lane == 0) beyond = 0.f;
            } else {
                beyond = __shfl_down_sync(0xffffffffu, e[k][0], 1);
                if (lane == 31) beyond = 0.f;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = b + 2 * h;
                const float L = j == 0 ? beyond : e[k][j - 1];
                const float R = j == 3 ? beyond : e[k][j + 1];
                const float U = k > 0 ? e[k - 1][j] : (wq > 0 ? rows[wq - 1][1][4 * lane + j] : 0.f);
                const float D = k < kRows - 1 ? e[k + 1][j] : (wq < kQWarps - 1 ? rows[wq + 1][0][4 * lane + j] : 0.f);
                const float sum = (L + R) + (U + D);
                e[k][j] = fmaf(sum, wi[k][j], fmaf(omc, e[k][j], wr[k][j]));
            }
        }
        // the first and last rows' new values for the neighbouring warps
        const int b0 = c & 1, b7 = (c + kRows - 1) & 1;
        rows[wq][0][4 * lane + b0] = e[0][b0];
        rows[wq][0][4 * lane + b0 + 2] = e[0][b0 + 2];
        rows[wq][1][4 * lane + b7] = e[kRows - 1][b7];
        rows[wq][1][4 * lane + b7 + 2] = e[kRows - 1][b7 + 2];
        __syncthreads();
    }
    // interior quads: columns kHL .. kHL + TX - 1 of the region
    const int lx = 4 * lane;
    if (lx < kHL || lx >= kHL + TX || gxq >= W) return true;
#pragma unroll
    for (int k = 0; k < kRows; ++k) {
        const int ly = ly0 + k, gy = gy0 + ly;
        if (ly < kHL || ly >= kHL + kTY || gy >= H) continue;
        float *o = eout + (size_t)gy * pitch + gxq;
        if (gxq + 3 < W) {
            *reinterpret_cast<float4 *>(o) = make_float4(e[k][0], e[k][1], e[k][2], e[k][3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (gxq + j < W) o[j] = e[k][j];
        }
    }
    return true;
}

// The plane and region of CTA b of a sweep launch: a static mapping (the
// launcher orders the chroma planes first, since they sweep longest), so a
// CTA addresses its data before the control words arrive.
__device__ __forceinline__ int sweep_plane(const IntraJobs &J, int b, int &lt)
{
    for (int p = 0; p < J.n; ++p)
        if (b >= J.p[p].tile_base && b < J.p[p].tile_base + J.p[p].tiles) {
            lt = b - J.p[p].tile_base;
            return p;
        }
    lt = 0;
    return 0;
}

// The pair count i handed on by the first CTA of a sweep launch (one
// thread, after its sweeps): parity 0 to the pair's second launch, parity
// 1 as i + 1 to the next pair's first launch, with whether its loop goes
// on: the planned pairs of the all-plane phase (pa), or of the chroma
// phase after it (CHROMA: pairs pa .. pa + pb - 1); never beyond
// kMaxPairs.  Each word is written while no launch that reads it runs.
template <int PAR, bool CHROMA>
__device__ __forceinline__ void pair_step(const IntraJobs &J)
{
    if (blockIdx.x != 0 || threadIdx.x != 0 || threadIdx.y != 0) return;
    IntraCtl *c = J.ctl;
    const int i = c->iter[PAR];
    if (PAR == 0) {
        c->iter[1] = i;
        return;
    }
    c->iter[0] = i + 1;
    const int end = CHROMA ? c->pairs[0] + c->pairs[1] : c->pairs[0];
    const int go = (i + 1 < end && i + 1 < kMaxPairs) ? 1 : 0;
    const unsigned long long h = CHROMA ? J.h_inner_c : J.h_inner;
    if (h) cudaGraphSetConditional(h, go);
}

// S red-black sweeps of launch it = 2 i + PAR of the cycle, over the
// planes whose launch count exceeds it (from e = 0 at it = 0, else from
// the plane's current correction in e[PAR]).  RH = kRHc: the chroma
// phase's launches (its own regions of the chroma planes).
template <int RW, int RH, int PAR>
__global__ void __launch_bounds__(RW / 2 * (RH / kRows), 1) intra_sor_kernel(const __grid_constant__ IntraJobs J)
{
    int lt;
    const int pl = sweep_plane(J, blockIdx.x, lt);
    sor_body<RW, RH, PAR>(J.p[pl], pl, lt, J.ctl);
    pair_step<PAR, RH == kRHc>(J);
}

template <int PAR>
__global__ void __launch_bounds__(32 * kQWarps, 1) intra_sor4_kernel(const __grid_constant__ IntraJobs J)
{
    int lt;
    const int pl = sweep_plane(J, blockIdx.x, lt);
    sor4_body<PAR>(J.p[pl], pl, lt, J.ctl);
    pair_step<PAR, false>(J);
}

}  // namespace

cudaError_t launch_intra_init(IntraJobs &J, uint32_t *flags, cudaStream_t st, int *launches)
{
    for (int k = 0; k < J.n; ++k) {
        cudaError_t e = cudaMemsetAsync(J.p[k].vsum, 0, sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
    }
    // a point, four pixels, a point per thread: every load of a launch in
    // flight at once (the loops inside stay correct for any grid)
    int n = 1;
    size_t px = 1;
    for (int k = 0; k < J.n; ++k) {
        n = std::max(n, J.p[k].n);
        px = std::max(px, (size_t)J.p[k].height * J.p[k].pitch / 4);
    }
    const unsigned gp = (unsigned)std::min((n + 255) / 256, 8192), gf = (unsigned)std::min<size_t>((px + 255) / 256, 16384);
    intra_sum_kernel<<<dim3(gp, J.n), 256, 0, st>>>(J, flags);
    intra_fill_kernel<<<dim3(gf, J.n), 256, 0, st>>>(J);
    intra_scatter_kernel<<<dim3(gp, J.n), 256, 0, st>>>(J);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_intra_restrict(const IntraJobs &F, const IntraJobs &C, cudaStream_t st)
{
    int w = 1, h = 1;  // the largest coarse plane: 4 pixels a thread in x
    for (int k = 0; k < C.n; ++k) {
        w = std::max(w, C.p[k].width);
        h = std::max(h, C.p[k].height);
    }
    intra_restrict_kernel<<<dim3(((w + 3) / 4 + 31) / 32, (h + 7) / 8, F.n), dim3(32, 8), 0, st>>>(F, C);
    return cudaGetLastError();
}

cudaError_t launch_intra_prolong(const IntraJobs &F, const IntraJobs &C, cudaStream_t st)
{
    int w = 1, h = 1;  // the largest fine plane: 4 pixels a thread in x
    for (int k = 0; k < F.n; ++k) {
        w = std::max(w, F.p[k].width);
        h = std::max(h, F.p[k].height);
    }
    intra_prolong_kernel<<<dim3(((w + 3) / 4 + 31) / 32, (h + 7) / 8, F.n), dim3(32, 8), 0, st>>>(F, C);
    return cudaGetLastError();
}

cudaError_t launch_intra_ctl_init(const IntraJobs &J, const float *omega0, double tol, int max_cycles,
                                  cudaStream_t st, int max_sweeps)
{
    intra_ctl_init_kernel<<<1, 1, 0, st>>>(J.ctl, omega0[0], J.n > 1 ? omega0[1] : 1.f, J.n > 2 ? omega0[2] : 1.f,
                                            tol, max_cycles, kS, std::min(std::max(max_sweeps, kS), 600));
    return cudaGetLastError();
}

namespace {

// residual tiles of kRTW x kRTH per plane
int residual_tiles(IntraJobs &J)
{
    int base = 0;
    for (int k = 0; k < J.n; ++k) {
        IntraPlane &P = J.p[k];
        P.tiles_x = (P.width + kRTW - 1) / kRTW;
        P.tile_base = base;
        P.tiles = P.tiles_x * ((P.height + kRTH - 1) / kRTH);
        base += P.tiles;
    }
    return base;
}

// sweep regions of the variant per plane; returns the CTAs, sets the block
// and the dynamic shared memory
// (kChromaPhase: the chroma phase's launches: regions of 128 x 88 of the
// chroma planes only)
constexpr int kChromaPhase = 3;
int sor_tiles(IntraJobs &J, int variant, dim3 &block, size_t &smem)
{
    const int tx = variant == 1 ? sor_tx(112) : sor_tx(128);
    const int ty = variant == kChromaPhase ? kRHc - 2 * kHL : kTY;
    int base = 0;
    // chroma planes first: they sweep longest, so the launches that sweep
    // them alone find their CTAs at the front of the grid
    for (int q = 0; q < J.n; ++q) {
        IntraPlane &P = J.p[J.n == 3 ? (q + 1) % 3 : q];
        const bool skip = variant == kChromaPhase && q == J.n - 1;  // luma: not in the chroma phase
        P.tiles_x = (P.width + tx - 1) / tx;
        P.tile_base = base;
        P.tiles = skip ? 0 : P.tiles_x * ((P.height + ty - 1) / ty);
        base += P.tiles;
    }
    block = variant == 2 ? dim3(32, kQWarps)
                         : dim3((variant == 1 ? 112 : 128) / 2, (variant == kChromaPhase ? kRHc : kRH) / kRows);
    smem = variant == 2 ? 0 : sor_smem_bytes(variant == 1 ? 112 : 128, variant == kChromaPhase ? kRHc : kRH);
    return base;
}

const void *sor_kernel(int variant, int par)
{
    if (variant == 1)
        return par ? reinterpret_cast<const void *>(intra_sor_kernel<112, kRH, 1>)
                   : reinterpret_cast<const void *>(intra_sor_kernel<112, kRH, 0>);
    if (variant == 2)
        return par ? reinterpret_cast<const void *>(intra_sor4_kernel<1>)
                   : reinterpret_cast<const void *>(intra_sor4_kernel<0>);
    if (variant == kChromaPhase)
        return par ? reinterpret_cast<const void *>(intra_sor_kernel<128, kRHc, 1>)
                   : reinterpret_cast<const void *>(intra_sor_kernel<128, kRHc, 0>);
    return par ? reinterpret_cast<const void *>(intra_sor_kernel<128, kRH, 1>)
               : reinterpret_cast<const void *>(intra_sor_kernel<128, kRH, 0>);
}

}  // namespace

cudaError_t launch_intra_residual(IntraJobs &J, bool first, cudaStream_t st)
{
    const int n = residual_tiles(J);
    if (n == 0) return cudaSuccess;
    intra_residual_kernel<<<n, kResThreads, 0, st>>>(J, first ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_intra_sor_chroma_pair(IntraJobs &J, cudaStream_t st)
{
    return launch_intra_sor_pair(J, kChromaPhase, st);
}

cudaError_t launch_intra_sor_pair(IntraJobs &J, int variant, cudaStream_t st)
{
    dim3 block;
    size_t smem;
    const int n = sor_tiles(J, variant, block, smem);
    if (n == 0) return cudaSuccess;
    void *args[] = {&J};
    cudaError_t e = cudaLaunchKernel(sor_kernel(variant, 0), dim3(n), block, args, smem, st);
    if (e == cudaSuccess) e = cudaLaunchKernel(sor_kernel(variant, 1), dim3(n), block, args, smem, st);
    return e;
}

namespace {

// Tiling autotuner.  The variants perform exactly the same global
// red-black sweeps (a cell's neighbour sum is formed in the same order), so
// the choice changes speed only.  The first solve of a set of plane sizes
// on a device times each variant, twice over groups of three launches
// (round robin), on a control state of its own (every plane active, from
// the current correction: the sweeps work on the decoder's buffers before
// the solve starts, which overwrites them), and keeps another variant than
// the first only if it is at least 2 % faster.  The choice goes to the
// tuner's table under the GPU's name and the plane sizes, so later
// processes on the same kind of GPU start with it.
constexpr int kSorVariants = 3;
std::mutex g_tune_mu;
std::map<std::vector<int>, int> g_tuned;

std::vector<int> tune_key(const IntraJobs &J)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<int> k{dev};
    for (int i = 0; i < J.n; ++i) {
        k.push_back(J.p[i].width);
        k.push_back(J.p[i].height);
    }
    return k;
}

// "<gpu>|sor|WxH,WxH,..." in the tuner's table
std::string table_key(const IntraJobs &J)
{
    std::string k = gpu_name() + "|sor|";
    for (int i = 0; i < J.n; ++i) k += (i ? "," : "") + std::to_string(J.p[i].width) + "x" + std::to_string(J.p[i].height);
    return k;
}

// a tuning control state: every plane active for as many launches as the
// timing needs, from the current correction (launches from it = 2 on)
__global__ void intra_tune_ctl_kernel(IntraCtl *c)
{
    IntraCtl z{};
    for (int p = 0; p < 3; ++p) {
        z.nl[p] = 1 << 20;
        z.omega[p] = 1.5f;
    }
    z.maxl = 1 << 20;
    z.iter[0] = z.iter[1] = 1;
    *c = z;
}

}  // namespace

std::atomic<int> g_forced{-1};  // a variant pinned by the caller, or -1

int intra_sor_variant(IntraJobs &J, IntraCtl *tune_ctl, cudaStream_t st)
{
    const int f = g_forced.load(std::memory_order_relaxed);
    if (f >= 0) return f;
    const std::vector<int> key = tune_key(J);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
        const int v = tune_lookup(table_key(J));
        if (v >= 0 && v < kSorVariants) {
            g_tuned[key] = v;
            return v;
        }
    }
    IntraJobs T = J;
    T.ctl = tune_ctl;
    T.h_outer = T.h_inner = 0;
    constexpr int kTuneGroup = 3, kTuneRounds = 2, kEv = kTuneRounds * kSorVariants + 1;
    cudaEvent_t ev[kEv];
    int made = 0;
    cudaError_t e = cudaSuccess;
    for (; made < kEv && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
    if (e == cudaSuccess) {
        intra_tune_ctl_kernel<<<1, 1, 0, st>>>(tune_ctl);
        e = cudaEventRecord(ev[0], st);
    }
    for (int t = 0; t < kEv - 1 && e == cudaSuccess; ++t) {
        for (int g = 0; g < kTuneGroup && e == cudaSuccess; ++g) e = launch_intra_sor_pair(T, t % kSorVariants, st);
        if (e == cudaSuccess) e = cudaEventRecord(ev[t + 1], st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[kEv - 1]);
    float best[kSorVariants] = {1e30f, 1e30f, 1e30f};
    for (int t = 0; t < kEv - 1 && e == cudaSuccess; ++t) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ev[t], ev[t + 1]);
        best[t % kSorVariants] = std::min(best[t % kSorVariants], ms);
    }
    for (int i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return 0;
    int rw = 0;
    for (int v = 1; v < kSorVariants; ++v)
        if (best[v] < 0.98f * best[rw]) rw = v;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = rw;
    }
    tune_store(table_key(J), rw);
    return rw;
}

cudaError_t build_intra_graph(const IntraJobs &J0, int variant, cudaGraphExec_t *exec)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    IntraJobs J = J0;
    auto fail = [&](cudaError_t err) {
        cudaGraphDestroy(g);
        return err;
    };
    // the outer loop's condition starts at 0; the first residual launch
    // (its last CTA) sets it
    if ((e = cudaGraphConditionalHandleCreate(&J.h_outer, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail(e);
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = J.h_outer;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t n_res0, n_outer, n_inner, n_sor, n_res;
    // first residual
    IntraJobs R = J;
    int one = 1, zero = 0;
    const int nres = residual_tiles(R);
    cudaKernelNodeParams kp{};
    kp.func = reinterpret_cast<void *>(intra_residual_kernel);
    kp.gridDim = dim3(nres);
    kp.blockDim = dim3(kResThreads);
    void *a0[] = {&R, &one};
    kp.kernelParams = a0;
    if ((e = cudaGraphAddKernelNode(&n_res0, g, nullptr, 0, &kp)) != cudaSuccess) return fail(e);
    if ((e = cudaGraphAddNode(&n_outer, g, &n_res0, nullptr, 1, &wp)) != cudaSuccess) return fail(e);
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    // the inner loop's condition is 1 at every pass of the outer body (a
    // cycle has at least one launch); each sweep launch sets it
    if ((e = cudaGraphConditionalHandleCreate(&J.h_inner, body, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return fail(e);
    cudaGraphNodeParams ip{};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = J.h_inner;
    ip.conditional.type = cudaGraphCondTypeWhile;
    ip.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_inner, body, nullptr, nullptr, 0, &ip)) != cudaSuccess) return fail(e);
    cudaGraph_t inner = ip.conditional.phGraph_out[0];
    // the loop's body: a pair of sweep launches (parity 0, then 1)
    IntraJobs S = J;
    dim3 block;
    size_t smem;
    const int nsor = sor_tiles(S, variant, block, smem);
    cudaKernelNodeParams sp{};
    sp.gridDim = dim3(nsor);
    sp.blockDim = block;
    sp.sharedMemBytes = (unsigned)smem;
    void *a1[] = {&S};
    sp.kernelParams = a1;
    cudaGraphNode_t n_sor0;
    sp.func = const_cast<void *>(sor_kernel(variant, 0));
    if ((e = cudaGraphAddKernelNode(&n_sor0, inner, nullptr, 0, &sp)) != cudaSuccess) return fail(e);
    sp.func = const_cast<void *>(sor_kernel(variant, 1));
    if ((e = cudaGraphAddKernelNode(&n_sor, inner, &n_sor0, 1, &sp)) != cudaSuccess) return fail(e);
    // the chroma phase: a second loop of launch pairs over the chroma planes
    // alone, with regions of their own (condition 1 at every pass of the
    // outer body; each of its second launches sets it)
    cudaGraphNode_t last = n_inner;
    IntraJobs C = J;
    if (J.chroma_phase && J.n == 3) {
        if ((e = cudaGraphConditionalHandleCreate(&J.h_inner_c, body, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
            return fail(e);
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = J.h_inner_c;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t n_inner_c, n_c0, n_c1;
        if ((e = cudaGraphAddNode(&n_inner_c, body, &n_inner, nullptr, 1, &cp)) != cudaSuccess) return fail(e);
        cudaGraph_t cbody = cp.conditional.phGraph_out[0];
        C = J;
        dim3 cblock;
        size_t csmem;
        const int nc = sor_tiles(C, kChromaPhase, cblock, csmem);
        cudaKernelNodeParams cq{};
        cq.gridDim = dim3(nc);
        cq.blockDim = cblock;
        cq.sharedMemBytes = (unsigned)csmem;
        void *a3[] = {&C};
        cq.kernelParams = a3;
        cq.func = const_cast<void *>(sor_kernel(kChromaPhase, 0));
        if ((e = cudaGraphAddKernelNode(&n_c0, cbody, nullptr, 0, &cq)) != cudaSuccess) return fail(e);
        cq.func = const_cast<void *>(sor_kernel(kChromaPhase, 1));
        if ((e = cudaGraphAddKernelNode(&n_c1, cbody, &n_c0, 1, &cq)) != cudaSuccess) return fail(e);
        last = n_inner_c;
    }
    // the cycle's residual launch, after the sweeps
    IntraJobs R2 = J;
    residual_tiles(R2);
    void *a2[] = {&R2, &zero};
    kp.kernelParams = a2;
    if ((e = cudaGraphAddKernelNode(&n_res, body, &last, 1, &kp)) != cudaSuccess) return fail(e);
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

int intra_sweeps_per_launch() { return kS; }

int set_sor_variant(int v)
{
    if (v < -1 || v >= kSorVariants) return -1;
    g_forced.store(v, std::memory_order_relaxed);
    return 0;
}

// One staged region per CTA, one CTA per SM: the colour arrays take dynamic
// shared memory beyond the static limit.  Called once per device.
cudaError_t intra_init()
{
    const void *k[6] = {reinterpret_cast<const void *>(intra_sor_kernel<128, kRH, 0>),
                        reinterpret_cast<const void *>(intra_sor_kernel<128, kRH, 1>),
                        reinterpret_cast<const void *>(intra_sor_kernel<112, kRH, 0>),
                        reinterpret_cast<const void *>(intra_sor_kernel<112, kRH, 1>),
                        reinterpret_cast<const void *>(intra_sor_kernel<128, kRHc, 0>),
                        reinterpret_cast<const void *>(intra_sor_kernel<128, kRHc, 1>)};
    const size_t bytes[6] = {sor_smem_bytes(128), sor_smem_bytes(128), sor_smem_bytes(112), sor_smem_bytes(112),
                             sor_smem_bytes(128, kRHc), sor_smem_bytes(128, kRHc)};
    for (int i = 0; i < 6; ++i) {
        const cudaError_t e = cudaFuncSetAttribute(k[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace hivc
