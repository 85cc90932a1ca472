// C ABI of libhivc: decoder objects, argument checks, the intra correction
// loop and the inter-frame pipeline.  Every step of the decode runs in the
// kernels of k_intra.cu, k_block.cu, k_pframe.cu and k_warp.cu; this file
// only allocates, validates and launches.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <mutex>

#include "hivc_internal.cuh"

using namespace hivc;

namespace {

constexpr int kPitchAlign = 32;  // elements
// sweeps of the coarse start's one cycle, at most (a start needs the smooth
// error only, which the half-size problem loses fast)
constexpr int kCoarseSweeps = 24;
// the layout the Python binding mirrors
static_assert(sizeof(hivc_stats) == 192 && offsetof(hivc_stats, kernel_pixels) == 120, "hivc_stats layout");

int round_up(int v, int a) { return (v + a - 1) / a * a; }

// scratch slots (one K > 32 system each) for a launch over nblocks blocks:
// one per range of kRange blocks, at most one per CTA of the persistent
// coefficient kernel
int coef_slots(int nblocks) { return std::max(1, std::min(block_ranges(nblocks), block_coef_ctas())); }

struct Alloc {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    bool ok = true;
    template <class T>
    T *get(size_t n)
    {
        if (!ok) return nullptr;
        void *p = nullptr;
        size_t b = std::max<size_t>(n * sizeof(T), 256);
        if (cudaMalloc(&p, b) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        bytes += b;
        return static_cast<T *>(p);
    }
    void release()
    {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
};

struct PlaneGeom {
    int w, h, pitch, nblocks, nbx;
};

// device status words of a decoder: error flags, then the statistics of
// the coefficient stage (max condition bound bits, FP64 re-solves, K > 32
// blocks, blocks evaluated by layout groups, layout groups)
constexpr int kStatusWords = 6;

bool config_ok(const hivc_config *c)
{
    return c && c->width >= 1 && c->height >= 1 && c->width <= 16384 && c->height <= 16384 &&
           (c->chroma >= 0 && c->chroma <= 2) && c->block >= 1 && c->block <= kMaxB && (c->op == 0 || c->op == 1) &&
           (c->precision == 0 || c->precision == 1) && c->iframe_tol >= 0.0 && c->max_cycles >= 1 && c->max_cycles <= 1000 &&
           c->cond_threshold >= 0.0 && (c->layout_groups == 0 || c->layout_groups == 1) && c->batch_frames >= 0 &&
           (c->fused_residual == 0 || c->fused_residual == 1) && (c->flat_start == 0 || c->flat_start == 1) &&
           c->batch_frames <= 4096;
}

int plane_count(const hivc_config *c) { return c->chroma ? 3 : 1; }

PlaneGeom plane_geom(const hivc_config *c, int p)
{
    PlaneGeom g;
    const bool half = p > 0 && c->chroma == 1;  // 4:2:0; 4:4:4 chroma planes are full size
    g.w = half ? (c->width + 1) / 2 : c->width;
    g.h = half ? (c->height + 1) / 2 : c->height;
    g.pitch = round_up(g.w, kPitchAlign);
    g.nbx = (g.w + c->block - 1) / c->block;
    g.nblocks = g.nbx * ((g.h + c->block - 1) / c->block);
    return g;
}

// Starting relaxation factor for red-black SOR from the mask density, for
// randomly scattered masks (the solve adapts it): the widest mask-free disc
// has radius about
// sqrt(ln(unknowns) / (pi * density)); its lowest Dirichlet mode sets the
// Jacobi spectral radius rho_J ~ 1 - (2.405 / R)^2 / 4, and
// omega = 2 / (1 + sqrt(1 - rho_J^2)) (Young's optimum).
float sor_omega(int w, int h, int n)
{
    const double N = (double)w * h;
    const double unknown = std::max(1.0, N - n);
    const double d = std::max(n, 1) / N;
    // the slowest modes live in irregular mask-free regions somewhat larger
    // than the widest empty disc (factor 1.4, measured on random masks)
    double R = 1.4 * std::sqrt(std::log(std::max(unknown, 2.0)) / (3.14159265358979 * d));
    R = std::min(R, 0.5 * std::max(w, h));
    const double lam = std::pow(2.405 / std::max(R, 1.0), 2.0);
    const double rho = std::max(0.0, 1.0 - lam / 4.0);
    double om = 2.0 / (1.0 + std::sqrt(std::max(0.0, 1.0 - rho * rho)));
    return (float)std::min(std::max(om, 1.0), 1.95);
}

// Batch-pool bytes for nframes inter frames at their largest (every pixel
// a residual point; Cb and Cr sharing their layout, the largest launch):
// per frame and plane the coefficients, block constants and residual
// plane, then one launch's scratch slots and plan (hivc_decode_batch's
// layout).
// Whether the decoder's inter frames go through the fused kernel (residual
// evaluated per block in shared memory, no residual planes; opt-in), as far
// as its configuration decides; the frame's pointers and pitches decide the
// rest (pframe_fused_ok).
bool fused_cfg(const hivc_config *c)
{
    return c->fused_residual == 1 && c->layout_groups == 0 && c->block == 16 && (c->chroma == 0 || c->chroma == 1) &&
           c->width % 2 == 0 && c->height % 2 == 0;
}

size_t pool_bytes_for(const hivc_config *c, int nframes)
{
    auto a256 = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t b = 0;
    int fblocks = 0;
    const bool planes = !fused_cfg(c);  // residual planes in the pool
    for (int k = 0; k < nframes; ++k)
        for (int p = 0; p < plane_count(c); ++p) {
            const PlaneGeom g = plane_geom(c, p);
            b += a256(4 * (size_t)g.w * g.h) + a256(4 * (size_t)g.nblocks) +
                 (planes ? a256(4 * (size_t)g.h * g.pitch) : 0);
        }
    for (int p = 0; p < plane_count(c); ++p) fblocks += plane_geom(c, p).nblocks;
    const int launch_blocks = (kMaxJobs / std::min(2, plane_count(c))) * fblocks;
    b += (size_t)coef_slots(launch_blocks) * kBigFloats * sizeof(float);
    b += block_plan_bytes(launch_blocks, c->layout_groups != 0);
    return b;
}

}  // namespace

struct hivc_decoder {
    hivc_config cfg{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int np = 1;
    PlaneGeom pg[3]{};
    Alloc mem;
    // reference planes (ping-pong) and their validity
    float *ref[2][3]{};
    int cur = 0;
    bool has_ref = false;
    // intra scratch
    float *uh[2][3]{}, *ul[2][3]{};
    float *res[3]{}, *e[2][3]{};
    uint8_t *mask[3]{};
    unsigned long long *vsum = nullptr;
    // the intra solve's control state (device), the SOR tuner's, a pinned
    // host copy, the loop's graph and the sweep variant it was built for
    IntraCtl *ctl = nullptr, *tune_ctl = nullptr, *h_ctl = nullptr;
    cudaGraphExec_t igraph = nullptr;
    int igraph_variant = -1;
    // the coarse start: half-size planes (iterate ping-pong, residual,
    // correction ping-pong, mask), their control state (and its pinned host
    // copy) and correction-loop graph
    int cw[3]{}, chh[3]{}, cpitch[3]{};
    float *cu[2][3]{}, *cres[3]{}, *ce[2][3]{};
    uint8_t *cmask[3]{};
    IntraCtl *ctl_c = nullptr, *h_ctl_c = nullptr;
    cudaGraphExec_t igraph_c = nullptr;
    bool intra_pending = false;  // an intra frame since the last sync
    bool has_intra = false;      // an intra frame was decoded
    // block scratch
    float *rfield[3]{}, *coef[3]{}, *acoef[3]{};
    size_t coef_cap = 0;
    float *big = nullptr;  // one K > 32 system per slot of the coefficient kernel
    int big_ranges = 0;
    BlockPlan plan{};      // work lists (and layout groups) of a frame's block stage
    uint32_t *flags = nullptr;
    // coefficients of the inter frames of one batch (grown on demand)
    void *pool = nullptr;
    size_t pool_bytes = 0;
    // host mirrors
    uint32_t *h_flags = nullptr;
    // statistics
    hivc_stats st{};
    bool timing = false;
    // side stream: the block stage of the inter frames after an intra frame
    // runs there while the intra frame decodes (fork and join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the end of an intra frame, and of each deferred evaluation launch
    cudaEvent_t ev_intra = nullptr;
    std::vector<cudaEvent_t> ev_batch;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

hivc_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HIVC_OK : HIVC_E_CUDA; }

cudaEvent_t take_event(hivc_decoder *d)
{
    if (!d->event_pool.empty()) {
        cudaEvent_t e = d->event_pool.back();
        d->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records CUDA events around a group of launches of one kernel family.
struct Timed {
    hivc_decoder *d;
    int fam;
    cudaEvent_t a = nullptr;
    Timed(hivc_decoder *dd, int f) : d(dd), fam(f)
    {
        if (d->timing) {
            a = take_event(d);
            cudaEventRecord(a, d->stream);
        }
    }
    void done(int launches)
    {
        d->st.kernel_launches[fam] += launches;
        d->st.launches += launches;
        if (a) {
            cudaEvent_t b = take_event(d);
            cudaEventRecord(b, d->stream);
            d->pending.push_back({fam, {a, b}});
            a = nullptr;
        }
    }
};

bool residual_ok(const hivc_residual &r)
{
    if (r.block_ptr == nullptr || r.n_points < 0) return false;
    if (r.n_points > 0 && (r.pos == nullptr || r.val == nullptr)) return false;
    return true;
}

bool out_ok(const hivc_decoder *d, const hivc_out *o)
{
    if (!o) return false;
    for (int p = 0; p < d->np; ++p)
        if (o->plane[p] == nullptr || o->pitch[p] < d->pg[p].w) return false;
    return true;
}

// Block jobs of one frame: Y, then Cb and Cr (one paired job when they share
// block_ptr/pos: one factorisation, two right-hand sides).  coef/acoef: the
// per-plane coefficient arrays (the decoder's own when null).
hivc_status make_block_jobs(hivc_decoder *d, const hivc_residual *res, BlockJobs &J, float *const *coef = nullptr,
                            float *const *acoef = nullptr, float *const *rfield = nullptr)
{
    if (!coef) coef = d->coef;
    if (!acoef) acoef = d->acoef;
    if (!rfield) rfield = d->rfield;
    J = BlockJobs{};
    J.op = d->cfg.op;
    for (int p = 0; p < d->np; ++p)
        if ((int64_t)res[p].n_points > (int64_t)d->pg[p].w * d->pg[p].h) return HIVC_E_INVALID;
    int base = 0;
    auto add = [&](int p, int p2) {
        BlockPlane &B = J.p[J.n++];
        const PlaneGeom &g = d->pg[p];
        B.block_ptr = res[p].block_ptr;
        B.pos = res[p].pos;
        B.val[0] = res[p].val;
        B.val[1] = p2 >= 0 ? res[p2].val : nullptr;
        B.coef[0] = coef[p];
        B.coef[1] = p2 >= 0 ? coef[p2] : nullptr;
        B.acoef[0] = acoef[p];
        B.acoef[1] = p2 >= 0 ? acoef[p2] : nullptr;
        B.r[0] = rfield[p];
        B.r[1] = p2 >= 0 ? rfield[p2] : nullptr;
        B.r_pitch = g.pitch;
        B.n_points = res[p].n_points;
        B.width = g.w;
        B.height = g.h;
        B.block = d->cfg.block;
        B.nbx = g.nbx;
        B.nblocks = g.nblocks;
        B.block_base = base;
        base += g.nblocks;
    };
    add(0, -1);
    if (d->np == 3) {
        const bool shared = res[1].block_ptr == res[2].block_ptr && res[1].pos == res[2].pos &&
                            res[1].n_points == res[2].n_points;
        if (shared) {
            add(1, 2);
        } else {
            add(1, -1);
            add(2, -1);
        }
    }
    J.total_blocks = base;
    return HIVC_OK;
}

BlockScratch scratch(hivc_decoder *d)
{
    BlockScratch S{d->flags, d->big, d->big_ranges, d->flags + 1, (float)d->cfg.cond_threshold};
    S.plan = d->plan;
    return S;
}

// Block stage of one frame: coefficients (+ large blocks), then residual
// fields (eval; else the fused pixel kernel evaluates them, from the jobs
// returned in jobs).
hivc_status run_block_residual(hivc_decoder *d, const hivc_residual *res, bool eval = true,
                               BlockJobs *jobs = nullptr)
{
    BlockJobs J;
    hivc_status s = make_block_jobs(d, res, J);
    if (s != HIVC_OK) return s;
    if (jobs) *jobs = J;
    cudaError_t e;
    {
        Timed t(d, 3);
        int l = 0;
        e = launch_block_coef(J, scratch(d), d->stream, &l, !d->timing);
        t.done(1);
    }
    if (e != cudaSuccess || !eval) return cuda_status(e);
    {
        Timed t(d, 5);
        e = launch_block_eval(J, d->flags, d->stream, !d->timing, &d->plan);
        t.done(1);
    }
    return cuda_status(e);
}

}  // namespace

extern "C" {

void hivc_config_default(hivc_config *c)
{
    if (!c) return;
    std::memset(c, 0, sizeof(*c));
    c->chroma = 1;
    c->block = 16;
    c->op = 0;
    c->precision = 0;
    c->iframe_tol = 1e-8;
    c->max_cycles = 40;
    c->cond_threshold = 1e6;
    c->stream = nullptr;
    c->layout_groups = 0;
}

const char *hivc_status_str(hivc_status s)
{
    switch (s) {
    case HIVC_OK: return "ok";
    case HIVC_E_INVALID: return "invalid argument or input data";
    case HIVC_E_NOMEM: return "device allocation failed";
    case HIVC_E_CUDA: return "CUDA error";
    case HIVC_E_NOT_CONVERGED: return "intra solve did not reach the tolerance";
    case HIVC_E_NO_REFERENCE: return "inter frame before any intra frame";
    case HIVC_E_BUDGET: return "over the device-memory budget";
    case HIVC_E_TIMEOUT: return "reserved status (bounded device wait)";
    }
    return "unknown status";
}

size_t hivc_decoder_bytes(const hivc_config *c)
{
    if (!config_ok(c)) return 0;
    size_t b = 0;
    auto add = [&](size_t n) { b += std::max<size_t>(n, 256); };
    int nblocks = 0;
    size_t maxpts = 0;
    for (int p = 0; p < plane_count(c); ++p) {
        PlaneGeom g = plane_geom(c, p);
        size_t n = (size_t)g.h * g.pitch;
        add(n * 4);
        add(n * 4);      // ref ping-pong
        add(n * 4);
        add(n * 4);
        add(n * 4);
        add(n * 4);      // u = hi + lo, ping-pong
        add(n * 4);      // res
        add(n * 4);
        add(n * 4);      // e ping-pong
        add(n);          // mask
        add(n * 4);      // residual field
        add((size_t)g.w * g.h * 4);  // coefficients
        add((size_t)g.nblocks * 4);  // constants
        nblocks += g.nblocks;
        maxpts = std::max(maxpts, (size_t)g.w * g.h);
    }
    for (int p = 0; p < plane_count(c); ++p) {  // the coarse start's half-size planes
        const PlaneGeom g = plane_geom(c, p);
        const size_t n = (size_t)((g.h + 1) / 2) * round_up((g.w + 1) / 2, kPitchAlign);
        for (int k = 0; k < 5; ++k) add(n * 4);
        add(n);
    }
    add(sizeof(IntraCtl));  // its control state
    add(3 * sizeof(unsigned long long));
    add(3 * sizeof(unsigned int));
    add((size_t)coef_slots(nblocks) * kBigFloats * sizeof(float));  // K > 32 systems
    add(block_plan_bytes(nblocks, c->layout_groups != 0));          // plan of a frame's block stage
    if (c->batch_frames > 0) add(pool_bytes_for(c, c->batch_frames));  // the batch pool made at creation
    add(4);                            // error word
    return b;
}

hivc_status hivc_decoder_create(const hivc_config *cfg, hivc_decoder **out)
{
    if (!out) return HIVC_E_INVALID;
    *out = nullptr;
    if (!config_ok(cfg)) return HIVC_E_INVALID;
    hivc_decoder *d = new (std::nothrow) hivc_decoder();
    if (!d) return HIVC_E_NOMEM;
    d->cfg = *cfg;
    if (cudaGetDevice(&d->device) != cudaSuccess) {
        delete d;
        return HIVC_E_CUDA;
    }
    if (ensure_block_tables() != cudaSuccess) {
        delete d;
        return HIVC_E_CUDA;
    }
    d->np = plane_count(cfg);
    int nblocks = 0;
    size_t maxpts = 0;
    Alloc &m = d->mem;
    for (int p = 0; p < d->np; ++p) {
        d->pg[p] = plane_geom(cfg, p);
        const PlaneGeom &g = d->pg[p];
        const size_t n = (size_t)g.h * g.pitch;
        d->ref[0][p] = m.get<float>(n);
        d->ref[1][p] = m.get<float>(n);
        d->uh[0][p] = m.get<float>(n);
        d->uh[1][p] = m.get<float>(n);
        d->ul[0][p] = m.get<float>(n);
        d->ul[1][p] = m.get<float>(n);
        d->res[p] = m.get<float>(n);
        d->e[0][p] = m.get<float>(n);
        d->e[1][p] = m.get<float>(n);
        d->mask[p] = m.get<uint8_t>(n);
        d->rfield[p] = m.get<float>(n);
        d->coef[p] = m.get<float>((size_t)g.w * g.h);
        d->acoef[p] = m.get<float>((size_t)g.nblocks);
        nblocks += g.nblocks;
        maxpts = std::max(maxpts, (size_t)g.w * g.h);
    }
    d->coef_cap = maxpts;
    d->big_ranges = coef_slots(nblocks);
    d->big = m.get<float>((size_t)d->big_ranges * kBigFloats);
    void *plan_mem = m.get<char>(block_plan_bytes(nblocks, cfg->layout_groups != 0));
    for (int p = 0; p < d->np; ++p) {
        d->cw[p] = (d->pg[p].w + 1) / 2;
        d->chh[p] = (d->pg[p].h + 1) / 2;
        d->cpitch[p] = round_up(d->cw[p], kPitchAlign);
        const size_t n = (size_t)d->chh[p] * d->cpitch[p];
        d->cu[0][p] = m.get<float>(n);
        d->cu[1][p] = m.get<float>(n);
        d->cres[p] = m.get<float>(n);
        d->ce[0][p] = m.get<float>(n);
        d->ce[1][p] = m.get<float>(n);
        d->cmask[p] = m.get<uint8_t>(n);
    }
    d->ctl_c = m.get<IntraCtl>(1);
    d->vsum = m.get<unsigned long long>(3);
    d->ctl = m.get<IntraCtl>(1);
    d->tune_ctl = m.get<IntraCtl>(1);
    d->flags = m.get<uint32_t>(kStatusWords);
    if (m.ok) d->plan = carve_block_plan(plan_mem, nblocks, cfg->layout_groups != 0);
    if (!m.ok) {
        m.release();
        delete d;
        return HIVC_E_NOMEM;
    }
    if (cudaMallocHost(&d->h_flags, 64) != cudaSuccess || cudaMallocHost(&d->h_ctl, sizeof(IntraCtl)) != cudaSuccess ||
        cudaMallocHost(&d->h_ctl_c, sizeof(IntraCtl)) != cudaSuccess) {
        if (d->h_flags) cudaFreeHost(d->h_flags);
        if (d->h_ctl) cudaFreeHost(d->h_ctl);
        if (d->h_ctl_c) cudaFreeHost(d->h_ctl_c);
        m.release();
        delete d;
        return HIVC_E_NOMEM;
    }
    std::memset(d->h_ctl, 0, sizeof(IntraCtl));
    std::memset(d->h_ctl_c, 0, sizeof(IntraCtl));
    if (cfg->stream) {
        d->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        if (cudaStreamCreateWithFlags(&d->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaFreeHost(d->h_flags);
            m.release();
            delete d;
            return HIVC_E_CUDA;
        }
        d->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d->ev_intra, cudaEventDisableTiming) != cudaSuccess ||
        cudaMemsetAsync(d->flags, 0, 4 * kStatusWords, d->stream) != cudaSuccess ||
        cudaMemsetAsync(d->ctl, 0, sizeof(IntraCtl), d->stream) != cudaSuccess ||
        cudaMemsetAsync(d->ctl_c, 0, sizeof(IntraCtl), d->stream) != cudaSuccess ||
        (cfg->batch_frames > 0 &&
         cudaMallocAsync(&d->pool, pool_bytes_for(cfg, cfg->batch_frames), d->stream) != cudaSuccess) ||
        cudaStreamSynchronize(d->stream) != cudaSuccess) {
        hivc_decoder_destroy(d);
        return HIVC_E_CUDA;
    }
    if (d->pool) d->pool_bytes = pool_bytes_for(cfg, cfg->batch_frames);
    *out = d;
    return HIVC_OK;
}

void hivc_decoder_destroy(hivc_decoder *d)
{
    if (!d) return;
    cudaSetDevice(d->device);
    if (d->side) cudaStreamSynchronize(d->side);
    if (d->pool && d->stream) cudaFreeAsync(d->pool, d->stream);  // a stream-ordered allocation
    d->pool = nullptr;
    if (d->stream) cudaStreamSynchronize(d->stream);
    if (d->side) cudaStreamDestroy(d->side);
    if (d->ev_fork) cudaEventDestroy(d->ev_fork);
    if (d->ev_join) cudaEventDestroy(d->ev_join);
    if (d->ev_intra) cudaEventDestroy(d->ev_intra);
    for (cudaEvent_t e : d->ev_batch) cudaEventDestroy(e);
    for (auto &pe : d->pending) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    for (cudaEvent_t e : d->event_pool) cudaEventDestroy(e);
    if (d->own_stream) cudaStreamDestroy(d->stream);
    if (d->h_flags) cudaFreeHost(d->h_flags);
    if (d->h_ctl) cudaFreeHost(d->h_ctl);
    if (d->h_ctl_c) cudaFreeHost(d->h_ctl_c);
    if (d->igraph) cudaGraphExecDestroy(d->igraph);
    if (d->igraph_c) cudaGraphExecDestroy(d->igraph_c);
    d->mem.release();
    delete d;
}

hivc_status hivc_decoder_reset(hivc_decoder *d)
{
    if (!d) return HIVC_E_INVALID;
    d->has_ref = false;
    return HIVC_OK;
}

hivc_status hivc_decoder_intra_solution(const hivc_decoder *d, int32_t plane, const float **hi, const float **lo,
                                        int32_t *w, int32_t *h, int32_t *pitch)
{
    if (!d || plane < 0 || plane >= d->np || !hi || !lo) return HIVC_E_INVALID;
    if (!d->has_intra) return HIVC_E_NO_REFERENCE;
    // the buffer the control state named at the last sync
    const int u = d->h_ctl->upar[plane] & 1;
    *hi = d->uh[u][plane];
    *lo = d->cfg.precision == 0 ? d->ul[u][plane] : nullptr;
    if (w) *w = d->pg[plane].w;
    if (h) *h = d->pg[plane].h;
    if (pitch) *pitch = d->pg[plane].pitch;
    return HIVC_OK;
}

void *hivc_decoder_stream(const hivc_decoder *d) { return d ? static_cast<void *>(d->stream) : nullptr; }

hivc_status hivc_decoder_set_timing(hivc_decoder *d, int32_t on)
{
    if (!d) return HIVC_E_INVALID;
    d->timing = on != 0;
    return HIVC_OK;
}

hivc_status hivc_decoder_reference(const hivc_decoder *d, int32_t plane, const float **ptr, int32_t *w, int32_t *h,
                                   int32_t *pitch)
{
    if (!d || plane < 0 || plane >= d->np || !ptr) return HIVC_E_INVALID;
    if (!d->has_ref) return HIVC_E_NO_REFERENCE;
    *ptr = d->ref[d->cur][plane];
    if (w) *w = d->pg[plane].w;
    if (h) *h = d->pg[plane].h;
    if (pitch) *pitch = d->pg[plane].pitch;
    return HIVC_OK;
}

namespace {

// The 4:4:4 colour path's pixel kernel for the frame being decoded: inter
// (flow != nullptr: warp of the current references) or intra (hi/lo: the
// inpainted planes); r: residual planes or nullptr.
// hi1, lo1, sel: the other buffers of the intra iterate's ping-pong and the
// device words (per plane) that say which buffer holds the solution
cudaError_t launch_rct_frame(hivc_decoder *d, const float *flow, float *const *hi, float *const *lo, bool residual,
                             const hivc_out *out, float *const *hi1 = nullptr, float *const *lo1 = nullptr,
                             const int32_t *sel = nullptr)
{
    RctFrame F{};
    F.flow = flow;
    F.src_sel = sel;
    const int nxt = d->cur ^ 1;
    for (int p = 0; p < 3; ++p) {
        F.ref[p] = d->ref[d->cur][p];
        F.src_hi[p] = hi ? hi[p] : nullptr;
        F.src_lo[p] = lo ? lo[p] : nullptr;
        F.src_hi1[p] = hi1 ? hi1[p] : nullptr;
        F.src_lo1[p] = lo1 ? lo1[p] : nullptr;
        F.r[p] = residual ? d->rfield[p] : nullptr;
        F.ref_out[p] = d->ref[nxt][p];
        F.out[p] = out->plane[p];
        F.out_pitch[p] = out->pitch[p];
    }
    F.pitch = d->pg[0].pitch;
    F.width = d->cfg.width;
    F.height = d->cfg.height;
    Timed t(d, 6);
    const cudaError_t e = launch_rct(F, d->stream);
    t.done(1);
    return e;
}

}  // namespace

namespace {

// One correction loop of J with the sweep tiling `variant`, decided on the
// device: one launch of the graph *graph (built once; again when
// *graph_variant, if given, names another tiling), or with per-kernel
// timing one launch at a time, with the plan read back into h between
// cycles.
cudaError_t run_intra_loop(hivc_decoder *d, IntraJobs &J, int variant, cudaGraphExec_t *graph, int *graph_variant,
                           IntraCtl *h, int fam_sweeps)
{
    cudaStream_t st = d->stream;
    cudaError_t e = cudaSuccess;
    if (d->timing) {
        {
            Timed t(d, 2);
            e = launch_intra_residual(J, true, st);
            t.done(0);
        }
        while (e == cudaSuccess) {
            e = cudaMemcpyAsync(h, J.ctl, sizeof(IntraCtl), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess || !h->go_outer) break;
            // the planned pairs: over all planes, then (the chroma phase)
            // over the chroma planes alone, at least one pair as in the graph
            const int pa = h->pairs[0], pb = J.chroma_phase ? std::max(1, h->pairs[1]) : 0;
            for (int l = 0; l < pa && e == cudaSuccess; ++l) {
                Timed t(d, fam_sweeps);
                e = launch_intra_sor_pair(J, variant, st);
                t.done(0);
            }
            for (int l = 0; l < pb && e == cudaSuccess; ++l) {
                Timed t(d, fam_sweeps);
                e = launch_intra_sor_chroma_pair(J, st);
                t.done(0);
            }
            if (e == cudaSuccess) {
                Timed t(d, 2);
                e = launch_intra_residual(J, false, st);
                t.done(0);
            }
        }
        return e;
    }
    if (!*graph || (graph_variant && *graph_variant != variant)) {
        if (*graph) cudaGraphExecDestroy(*graph);
        *graph = nullptr;
        if ((e = build_intra_graph(J, variant, graph)) != cudaSuccess) return e;
        if (graph_variant) *graph_variant = variant;
    }
    return cudaGraphLaunch(*graph, st);
}

}  // namespace

hivc_status hivc_decode_iframe(hivc_decoder *d, const hivc_iframe *f, const hivc_out *out)
{
    if (!d || !f || !out_ok(d, out)) return HIVC_E_INVALID;
    if (f->y.n < 1 || !f->y.idx || !f->y.val) return HIVC_E_INVALID;
    if ((int64_t)f->y.n > (int64_t)d->pg[0].w * d->pg[0].h) return HIVC_E_INVALID;
    const bool rct = d->cfg.chroma == 2;
    if (d->np == 3) {
        if (f->c_n < 1 || !f->c_idx || (rct ? (!f->cu_val || !f->cv_val) : (!f->cb_val || !f->cr_val)))
            return HIVC_E_INVALID;
        if ((int64_t)f->c_n > (int64_t)d->pg[1].w * d->pg[1].h) return HIVC_E_INVALID;
    }
    if (f->res)
        for (int p = 0; p < d->np; ++p)
            if (!residual_ok(f->res[p])) return HIVC_E_INVALID;
    if (cudaSetDevice(d->device) != cudaSuccess) return HIVC_E_CUDA;
    cudaStream_t st = d->stream;
    IntraJobs J{};
    J.n = d->np;
    J.ctl = d->ctl;
    // 4:2:0: the launches that sweep only the half-size chroma planes use
    // regions of their own (144 for FullHD instead of 90 of 152 SMs)
    J.chroma_phase = d->cfg.chroma == 1 && d->np == 3 ? 1 : 0;
    float om0[3] = {1.f, 1.f, 1.f};
    for (int p = 0; p < d->np; ++p) {
        IntraPlane &P = J.p[p];
        const PlaneGeom &g = d->pg[p];
        P.width = g.w;
        P.height = g.h;
        P.pitch = g.pitch;
        P.idx = p == 0 ? f->y.idx : f->c_idx;
        P.val = p == 0 ? f->y.val : (p == 1 ? f->cb_val : f->cr_val);
        P.val16 = (rct && p > 0) ? (p == 1 ? f->cu_val : f->cv_val) : nullptr;
        if (P.val16) P.val = nullptr;
        P.n = p == 0 ? f->y.n : f->c_n;
        P.mask = d->mask[p];
        P.uh[0] = d->uh[0][p];
        P.uh[1] = d->uh[1][p];
        P.ul[0] = d->ul[0][p];
        P.ul[1] = d->ul[1][p];
        P.res = d->res[p];
        P.e[0] = d->e[0][p];
        P.e[1] = d->e[1][p];
        P.vsum = d->vsum + p;
        P.ff = d->cfg.precision == 0 ? 1 : 0;
        om0[p] = sor_omega(g.w, g.h, P.n);
    }
    cudaError_t e;
    {
        Timed t(d, 0);
        int l = 0;
        e = launch_intra_init(J, d->flags, st, &l);
        t.done(l);
    }
    if (e != cudaSuccess) return HIVC_E_CUDA;
    // the sweep kernel's tiling (the first solve of a geometry times the
    // variants on launches of its own)
    const int variant = intra_sor_variant(J, d->tune_ctl, st);
    // the coarse start: the mask restricted to the half-size planes, one
    // FP32 correction cycle there (to its floor, or the tolerance), and the
    // unknown pixels prolonged from it
    bool coarse = d->cfg.flat_start == 0;
    for (int p = 0; p < d->np; ++p) coarse = coarse && d->pg[p].w >= 32 && d->pg[p].h >= 32;
    if (coarse) {
        IntraJobs C{};
        C.n = d->np;
        C.ctl = d->ctl_c;
        float omc[3] = {1.f, 1.f, 1.f};
        for (int p = 0; p < d->np; ++p) {
            IntraPlane &P = C.p[p];
            P.width = d->cw[p];
            P.height = d->chh[p];
            P.pitch = d->cpitch[p];
            P.mask = d->cmask[p];
            P.uh[0] = d->cu[0][p];
            P.uh[1] = d->cu[1][p];
            P.res = d->cres[p];
            P.e[0] = d->ce[0][p];
            P.e[1] = d->ce[1][p];
            P.vsum = d->vsum + p;
            P.ff = 0;
            // a coarse cell is known when one of its four fine pixels is
            const double N = (double)d->pg[p].w * d->pg[p].h, dens = std::min(1.0, J.p[p].n / N);
            const double nc = (double)P.width * P.height * (1.0 - std::pow(1.0 - dens, 4.0));
            P.n = (int32_t)std::max(1.0, nc);
            omc[p] = sor_omega(P.width, P.height, P.n);
        }
        {
            Timed t(d, 0);
            e = launch_intra_restrict(J, C, st);
            t.done(1);
        }
        if (e == cudaSuccess) e = launch_intra_ctl_init(C, omc, d->cfg.iframe_tol, 1, st, kCoarseSweeps);
        if (e == cudaSuccess) e = run_intra_loop(d, C, 0, &d->igraph_c, nullptr, d->h_ctl_c, 7);
        if (e == cudaSuccess) {
            Timed t(d, 0);
            e = launch_intra_prolong(J, C, st);
            t.done(1);
        }
        if (e != cudaSuccess) return HIVC_E_CUDA;
    }
    // the correction loop, decided on the device
    if (launch_intra_ctl_init(J, om0, d->cfg.iframe_tol, d->cfg.max_cycles, st) != cudaSuccess) return HIVC_E_CUDA;
    e = run_intra_loop(d, J, variant, &d->igraph, &d->igraph_variant, d->h_ctl, 1);
    if (e != cudaSuccess) return HIVC_E_CUDA;
    d->intra_pending = true;
    d->has_intra = true;
    // optional residual correction of the intra frame (Fig. 1e/f)
    if (f->res) {
        hivc_status s = run_block_residual(d, f->res);
        if (s != HIVC_OK) return s;
    }
    // the output: the solution sits in the iterate buffer the control state
    // names (upar) per plane
    const int nxt = d->cur ^ 1;
    if (rct) {
        float *hi[3], *lo[3], *hi1[3], *lo1[3];
        for (int p = 0; p < 3; ++p) {
            hi[p] = J.p[p].uh[0];
            lo[p] = J.p[p].ff ? J.p[p].ul[0] : nullptr;
            hi1[p] = J.p[p].uh[1];
            lo1[p] = J.p[p].ff ? J.p[p].ul[1] : nullptr;
        }
        if (launch_rct_frame(d, nullptr, hi, lo, f->res != nullptr, out, hi1, lo1, d->ctl->upar) != cudaSuccess)
            return HIVC_E_CUDA;
        d->cur = nxt;
        d->has_ref = true;
        d->st.frames += 1;
        return HIVC_OK;
    }
    WarpJobs W{};
    W.n = d->np;
    for (int p = 0; p < d->np; ++p) {
        WarpPlane &P = W.p[p];
        const PlaneGeom &g = d->pg[p];
        P.src_hi = J.p[p].uh[0];
        P.src_lo = J.p[p].ff ? J.p[p].ul[0] : nullptr;
        P.src_hi1 = J.p[p].uh[1];
        P.src_lo1 = J.p[p].ff ? J.p[p].ul[1] : nullptr;
        P.src_sel = d->ctl->upar + p;
        P.src_pitch = g.pitch;
        P.r = f->res ? d->rfield[p] : nullptr;
        P.r_pitch = g.pitch;
        P.ref_out = d->ref[nxt][p];
        P.ref_out_pitch = g.pitch;
        P.out = out->plane[p];
        P.out_pitch = out->pitch[p];
        P.width = g.w;
        P.height = g.h;
    }
    {
        Timed t(d, 6);
        e = launch_warp_add(W, st);
        t.done(1);
    }
    if (e != cudaSuccess) return HIVC_E_CUDA;
    d->cur = nxt;
    d->has_ref = true;
    d->st.frames += 1;
    return HIVC_OK;
}

namespace {

// The pixel kernel's view of an inter frame (r: residual planes of plane
// pitch, or null for the fused kernel) into the next reference buffer.
InterFrame pixel_frame(const hivc_decoder *d, const float *flow, const hivc_out *out, float *const *r)
{
    const int nxt = d->cur ^ 1;
    InterFrame F{};
    F.flow = flow;
    for (int p = 0; p < d->np; ++p) {
        F.ref[p] = d->ref[d->cur][p];
        F.ref_out[p] = d->ref[nxt][p];
        F.ref_pitch[p] = d->pg[p].pitch;
        F.out[p] = out->plane[p];
        F.out_pitch[p] = out->pitch[p];
        F.r[p] = r ? r[p] : nullptr;
        F.r_pitch[p] = d->pg[p].pitch;
    }
    F.width = d->cfg.width;
    F.height = d->cfg.height;
    F.chroma = d->cfg.chroma;
    return F;
}

// Whether an inter frame of d goes through the fused kernel.
bool fused_frame_ok(const hivc_decoder *d, const float *flow, const hivc_out *out)
{
    return fused_cfg(&d->cfg) && pframe_fused_ok(pixel_frame(d, flow, out, nullptr), d->cfg.block);
}

// The pixel kernel of a frame whose residual planes (plane pitches) were
// evaluated before, into the next reference buffer.
cudaError_t launch_pixels(hivc_decoder *d, const float *flow, const hivc_out *out, float *const *r,
                          bool pdl = true, bool early = false)
{
    const InterFrame F = pixel_frame(d, flow, out, r);
    Timed t(d, 4);
    const cudaError_t e = launch_pframe(F, d->stream, pdl && !d->timing, early && pdl && !d->timing);
    t.done(1);
    return e;
}

// The fused kernel of a frame whose coefficients the block stage of jobs J
// (one frame: Y, then the paired chroma job or Cb and Cr) computed.
// early: the kernel before it on the stream is the fused kernel of the
// previous frame, which waited for the block stage.
cudaError_t launch_fused(hivc_decoder *d, const float *flow, const hivc_out *out, const BlockJobs &J, bool pdl,
                         bool early)
{
    FusedFrame F{};
    F.px = pixel_frame(d, flow, out, nullptr);
    F.y = J.p[0];
    F.nc = J.n - 1;
    for (int k = 1; k < J.n && k < 3; ++k) F.c[k - 1] = J.p[k];
    F.op = d->cfg.op;
    F.flags = d->flags;
    F.early = early ? 1 : 0;
    Timed t(d, 4);
    const cudaError_t e = launch_pframe_fused(F, d->stream, pdl && !d->timing);
    t.done(1);
    return e;
}

}  // namespace

hivc_status hivc_decode_pframe(hivc_decoder *d, const hivc_pframe *f, const hivc_out *out)
{
    if (!d || !f || !out_ok(d, out) || !f->flow) return HIVC_E_INVALID;
    for (int p = 0; p < d->np; ++p)
        if (!residual_ok(f->res[p])) return HIVC_E_INVALID;
    if (!d->has_ref) return HIVC_E_NO_REFERENCE;
    if (cudaSetDevice(d->device) != cudaSuccess) return HIVC_E_CUDA;
    const int nxt = d->cur ^ 1;
    // coefficients (Eq. 2), then the fused kernel (Eq. 3 per block in
    // shared memory, warp + add + pack); or three launches: coefficients,
    // residual planes (Eq. 3), then warp + add + pack (the 4:4:4 colour
    // path: its RCT kernel)
    const bool fused = fused_frame_ok(d, f->flow, out);
    BlockJobs J;
    hivc_status s = run_block_residual(d, f->res, !fused, &J);
    if (s != HIVC_OK) return s;
    const cudaError_t e = fused                ? launch_fused(d, f->flow, out, J, true, false)
                          : d->cfg.chroma == 2 ? launch_rct_frame(d, f->flow, nullptr, nullptr, true, out)
                                               : launch_pixels(d, f->flow, out, d->rfield);
    if (e != cudaSuccess) return HIVC_E_CUDA;
    d->cur = nxt;
    d->st.frames += 1;
    return HIVC_OK;
}

namespace {

bool coef_residual_ok(const hivc_coef_residual &r, int w, int h)
{
    return r.block_ptr && r.n_points >= 0 && r.a && (r.n_points == 0 || (r.pos && r.q)) &&
           (int64_t)r.n_points <= (int64_t)w * h && std::isfinite(r.step) && r.step > 0.f &&
           std::isfinite(r.offset) && r.offset >= 0.f && r.offset < 1.f;
}

// A coefficient-mode plane as a block job (evaluation only).
void coef_job(BlockPlane &B, const hivc_coef_residual &r, int w, int h, int block, float *rf, int pitch, int base)
{
    B = BlockPlane{};
    B.block_ptr = r.block_ptr;
    B.pos = r.pos;
    B.q = r.q;
    B.qstep = r.step;
    B.qoff = r.offset;
    B.acoef[0] = const_cast<float *>(r.a);
    B.r[0] = rf;
    B.r_pitch = pitch;
    B.n_points = r.n_points;
    B.width = w;
    B.height = h;
    B.block = block;
    B.nbx = (w + block - 1) / block;
    B.nblocks = B.nbx * ((h + block - 1) / block);
    B.block_base = base;
}

}  // namespace

hivc_status hivc_decode_pframe_coef(hivc_decoder *d, const hivc_pframe_coef *f, const hivc_out *out)
{
    if (!d || !f || !out_ok(d, out) || !f->flow) return HIVC_E_INVALID;
    for (int p = 0; p < d->np; ++p)
        if (!coef_residual_ok(f->res[p], d->pg[p].w, d->pg[p].h)) return HIVC_E_INVALID;
    if (!d->has_ref) return HIVC_E_NO_REFERENCE;
    if (cudaSetDevice(d->device) != cudaSuccess) return HIVC_E_CUDA;
    BlockJobs J{};
    J.op = d->cfg.op;
    for (int p = 0; p < d->np; ++p) {
        const PlaneGeom &g = d->pg[p];
        coef_job(J.p[J.n++], f->res[p], g.w, g.h, d->cfg.block, d->rfield[p], g.pitch, J.total_blocks);
        J.total_blocks += g.nblocks;
    }
    cudaError_t e;
    {
        Timed t(d, 5);
        e = launch_block_eval(J, d->flags, d->stream, !d->timing);
        t.done(1);
    }
    if (e != cudaSuccess) return HIVC_E_CUDA;
    // warp + residual + pack
    const int nxt = d->cur ^ 1;
    e = d->cfg.chroma == 2 ? launch_rct_frame(d, f->flow, nullptr, nullptr, true, out)
                           : launch_pixels(d, f->flow, out, d->rfield);
    if (e != cudaSuccess) return HIVC_E_CUDA;
    d->cur = nxt;
    d->st.frames += 1;
    return HIVC_OK;
}

hivc_status hivc_block_residual_coef(int32_t width, int32_t height, int32_t block, int32_t op,
                                     const hivc_coef_residual *res, float *r, int32_t r_pitch, uint32_t *flags,
                                     void *stream)
{
    if (!res || !r || width < 1 || height < 1 || block < 1 || block > kMaxB || r_pitch < width ||
        (op != 0 && op != 1) || !coef_residual_ok(*res, width, height))
        return HIVC_E_INVALID;
    if (ensure_block_tables() != cudaSuccess) return HIVC_E_CUDA;
    BlockJobs J{};
    J.n = 1;
    J.op = op;
    coef_job(J.p[0], *res, width, height, block, r, r_pitch, 0);
    J.total_blocks = J.p[0].nblocks;
    const cudaError_t e = launch_block_eval(J, flags, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HIVC_OK : HIVC_E_CUDA;
}

namespace {

size_t a256(size_t b) { return (b + 255) / 256 * 256; }

bool pframe_ok(const hivc_decoder *d, const hivc_pframe *f, const hivc_out *out)
{
    if (!d || !f || !out_ok(d, out) || !f->flow) return false;
    for (int p = 0; p < d->np; ++p)
        if (!residual_ok(f->res[p]) || (int64_t)f->res[p].n_points > (int64_t)d->pg[p].w * d->pg[p].h) return false;
    return true;
}

// The decoder's batch pool holds at least bytes.  Growth is stream-ordered
// on st (the stream that will use the pool, ordered after all earlier work
// of the decoder's streams): the old pool is freed and the new one made
// there, so no host thread waits.
hivc_status ensure_pool(hivc_decoder *d, size_t bytes, cudaStream_t st)
{
    if (d->pool_bytes >= bytes) return HIVC_OK;
    if (d->pool && cudaFreeAsync(d->pool, st) != cudaSuccess) return HIVC_E_CUDA;
    d->pool = nullptr;
    d->pool_bytes = 0;
    const size_t want = bytes + bytes / 4;
    if (cudaMallocAsync(&d->pool, want, st) != cudaSuccess) {
        cudaGetLastError();
        d->pool = nullptr;
        return HIVC_E_NOMEM;
    }
    d->pool_bytes = want;
    return HIVC_OK;
}

// The block stage's results of an inter run: per frame its residual
// planes (split path) and its block jobs (coefficient arrays in the pool).
// After an intra frame the evaluation launches but the first wait for the
// intra frame and then overlap the pixel kernels of the batch before them
// (on the split path without layout groups).
constexpr bool kDeferEval = true;

struct RunBlocks {
    bool fused = false;  // the fused kernel evaluates the residual
    bool defer = false;  // evaluation launches of batches after the first deferred
    std::vector<std::array<float *, 3>> planes;
    std::vector<BlockJobs> jobs;
    std::vector<size_t> batch_first;  // index into ks of each launch's first frame
    std::vector<BlockJobs> deferred;  // the deferred launches' jobs (batches 1, 2, ...)
};

// Whether every frame of the run goes through the fused kernel.
bool fused_run(const hivc_decoder *d, const hivc_frame *frames, const hivc_out *outs, const std::vector<int> &ks)
{
    for (int k : ks)
        if (!fused_frame_ok(d, frames[k].p->flow, &outs[k])) return false;
    return !ks.empty();
}

// Block stage of the inter frames frames[k] (k in ks, in order) of decoder
// d on stream st: per up to kMaxJobs block jobs (8 FullHD 4:2:0 frames) one
// coefficient launch and (rb.fused false) one evaluation launch into each
// frame's residual planes, all in the batch pool; the frames' jobs and
// planes are returned in rb.  pdl: the first launch may overlap the kernel
// before it on st.  Every frame has been checked.
hivc_status inter_blocks(hivc_decoder *d, const hivc_frame *frames, const std::vector<int> &ks, cudaStream_t st,
                         bool pdl, RunBlocks &rb)
{
    if (cudaSetDevice(d->device) != cudaSuccess) return HIVC_E_CUDA;
    const size_t nf = ks.size();
    // pool layout: per frame and plane a256(4 n_points) + a256(4 nblocks)
    // (+ the residual plane, h x pitch floats, on the split path), then the
    // K > 32 scratch of the largest coefficient launch
    std::vector<size_t> off(nf * 3 * 3);
    size_t bytes = 0;
    for (size_t k = 0; k < nf; ++k)
        for (int p = 0; p < d->np; ++p) {
            const PlaneGeom &g = d->pg[p];
            off[(k * 3 + p) * 3] = bytes;
            bytes += a256(4 * (size_t)frames[ks[k]].p->res[p].n_points);
            off[(k * 3 + p) * 3 + 1] = bytes;
            bytes += a256(4 * (size_t)g.nblocks);
            off[(k * 3 + p) * 3 + 2] = bytes;
            if (!rb.fused) bytes += a256(4 * (size_t)g.h * g.pitch);
        }
    int fblocks = 0;
    for (int p = 0; p < d->np; ++p) fblocks += d->pg[p].nblocks;
    // frames per coefficient launch: a frame has one job per plane, or one
    // less when Cb and Cr share their layout (the job count make_block_jobs
    // gives); the fewest jobs per frame make the largest launch
    int min_jobs = d->np;
    for (size_t k = 0; k < nf; ++k) {
        const hivc_residual *r = frames[ks[k]].p->res;
        if (d->np == 3 && r[1].block_ptr == r[2].block_ptr && r[1].pos == r[2].pos && r[1].n_points == r[2].n_points)
            min_jobs = 2;
    }
    const int launch_blocks = (kMaxJobs / min_jobs) * fblocks;
    const int ranges = coef_slots(launch_blocks);
    const size_t big_off = bytes;
    bytes += (size_t)ranges * kBigFloats * sizeof(float);
    const bool groups = d->cfg.layout_groups != 0;
    const size_t plan_off = bytes;
    bytes += block_plan_bytes(launch_blocks, groups);
    hivc_status s = ensure_pool(d, bytes, st);
    if (s != HIVC_OK) return s;
    char *pool = static_cast<char *>(d->pool);
    auto at = [&](size_t k, int p, int w) {
        return p < d->np && !(w == 2 && rb.fused) ? reinterpret_cast<float *>(pool + off[(k * 3 + p) * 3 + w])
                                                  : nullptr;
    };
    std::vector<BlockJobs> jobs(nf);
    for (size_t k = 0; k < nf; ++k) {
        float *coef[3], *acoef[3], *rfield[3];
        for (int p = 0; p < 3; ++p) {
            coef[p] = at(k, p, 0);
            acoef[p] = at(k, p, 1);
            rfield[p] = at(k, p, 2);
        }
        if ((s = make_block_jobs(d, frames[ks[k]].p->res, jobs[k], coef, acoef, rfield)) != HIVC_OK) return s;
    }
    BlockScratch S{d->flags, reinterpret_cast<float *>(pool + big_off), ranges, d->flags + 1,
                   (float)d->cfg.cond_threshold};
    S.plan = carve_block_plan(pool + plan_off, launch_blocks, groups);
    BlockJobs J{};
    J.op = d->cfg.op;
    auto flush = [&]() -> cudaError_t {
        if (J.n == 0) return cudaSuccess;
        cudaError_t e;
        {
            Timed t(d, 3);
            int l = 0;
            e = launch_block_coef(J, S, st, &l, pdl && !d->timing);
            t.done(l);
        }
        pdl = true;
        if (e == cudaSuccess && !rb.fused) {
            if (rb.defer && rb.batch_first.size() > 1) {
                rb.deferred.push_back(J);
            } else {
                Timed t(d, 5);
                e = launch_block_eval(J, d->flags, st, !d->timing, &S.plan);
                t.done(1);
            }
        }
        J = BlockJobs{};
        J.op = d->cfg.op;
        return e;
    };
    rb.batch_first.clear();
    rb.deferred.clear();
    for (size_t k = 0; k < nf; ++k) {
        if (J.n + jobs[k].n > kMaxJobs && flush() != cudaSuccess) return HIVC_E_CUDA;
        if (J.n == 0) rb.batch_first.push_back(k);
        for (int q = 0; q < jobs[k].n; ++q) {
            BlockPlane B = jobs[k].p[q];
            B.block_base = J.total_blocks;
            J.total_blocks += B.nblocks;
            J.p[J.n++] = B;
        }
    }
    if (flush() != cudaSuccess) return HIVC_E_CUDA;
    rb.planes.resize(nf);
    for (size_t k = 0; k < nf; ++k) rb.planes[k] = {at(k, 0, 2), at(k, 1, 2), at(k, 2, 2)};
    rb.jobs = std::move(jobs);
    return HIVC_OK;
}

// Per inter frame the pixel kernel on the decoder's stream: the fused
// kernel (from the coefficients of inter_blocks), or the warp + residual +
// pack kernel (its residual planes).  pdl: the first launch may overlap the
// kernel before it.
hivc_status inter_pixels(hivc_decoder *d, const hivc_frame *frames, const hivc_out *outs, const std::vector<int> &ks,
                         const RunBlocks &rb, bool pdl)
{
    size_t b = 1;  // the next deferred batch
    for (size_t k = 0; k < ks.size(); ++k) {
        const hivc_pframe *f = frames[ks[k]].p;
        if (rb.defer && b < rb.batch_first.size() && k == rb.batch_first[b]) {
            // the batch's evaluation ran on the side stream
            if (cudaStreamWaitEvent(d->stream, d->ev_batch[b - 1], 0) != cudaSuccess) return HIVC_E_CUDA;
            ++b;
            const cudaError_t e = launch_pixels(d, f->flow, &outs[ks[k]], rb.planes[k].data(), false, false);
            if (e != cudaSuccess) return HIVC_E_CUDA;
            d->cur ^= 1;
            d->st.frames += 1;
            continue;
        }
        // the first fused kernel waits for the block stage before it reads
        // the coefficients; each later one may read them at once
        const cudaError_t e = rb.fused ? launch_fused(d, f->flow, &outs[ks[k]], rb.jobs[k], pdl || k > 0, k > 0)
                                       : launch_pixels(d, f->flow, &outs[ks[k]], rb.planes[k].data(), pdl || k > 0,
                                                       k > 0);
        if (e != cudaSuccess) return HIVC_E_CUDA;
        d->cur ^= 1;
        d->st.frames += 1;
    }
    return HIVC_OK;
}

hivc_status decode_inter_run(hivc_decoder *d, const hivc_frame *frames, const hivc_out *outs,
                             const std::vector<int> &ks)
{
    RunBlocks rb;
    rb.fused = fused_run(d, frames, outs, ks);
    const hivc_status s = inter_blocks(d, frames, ks, d->stream, true, rb);
    return s != HIVC_OK ? s : inter_pixels(d, frames, outs, ks, rb, true);
}

// An intra frame followed by the inter run ks: the run's block stage does
// not depend on the intra frame, so it goes to the side stream (after all
// earlier work of the decoder's stream, which may still read the pool) and
// overlaps the intra frame's sweeps and the host's waits between its
// correction cycles; the decoder's stream joins it before the first warp.
hivc_status decode_intra_then_run(hivc_decoder *d, const hivc_frame *frames, const hivc_out *outs, int ki,
                                  const std::vector<int> &ks, hivc_status &intra)
{
    if (cudaSetDevice(d->device) != cudaSuccess || cudaEventRecord(d->ev_fork, d->stream) != cudaSuccess ||
        cudaStreamWaitEvent(d->side, d->ev_fork, 0) != cudaSuccess)
        return HIVC_E_CUDA;
    RunBlocks rb;
    rb.fused = fused_run(d, frames, outs, ks);
    rb.defer = kDeferEval && !rb.fused && d->cfg.layout_groups == 0;
    const hivc_status sb = inter_blocks(d, frames, ks, d->side, false, rb);
    const bool joined = cudaEventRecord(d->ev_join, d->side) == cudaSuccess;
    intra = hivc_decode_iframe(d, frames[ki].i, &outs[ki]);
    if (!joined || cudaStreamWaitEvent(d->stream, d->ev_join, 0) != cudaSuccess) return HIVC_E_CUDA;
    if (intra != HIVC_OK && intra != HIVC_E_NOT_CONVERGED) return intra;
    if (sb != HIVC_OK) return sb;
    if (!rb.deferred.empty()) {
        // the deferred evaluations: after the intra frame, on the side
        // stream, an event after each
        while (d->ev_batch.size() < rb.deferred.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HIVC_E_CUDA;
            d->ev_batch.push_back(e);
        }
        if (cudaEventRecord(d->ev_intra, d->stream) != cudaSuccess ||
            cudaStreamWaitEvent(d->side, d->ev_intra, 0) != cudaSuccess)
            return HIVC_E_CUDA;
        for (size_t b = 0; b < rb.deferred.size(); ++b) {
            Timed t(d, 5);  // (counts only: the timing pass takes another path)
            const cudaError_t e = launch_block_eval(rb.deferred[b], d->flags, d->side, b > 0, nullptr);
            t.done(1);
            if (e != cudaSuccess || cudaEventRecord(d->ev_batch[b], d->side) != cudaSuccess) return HIVC_E_CUDA;
        }
    }
    return inter_pixels(d, frames, outs, ks, rb, false);
}

}  // namespace

namespace {

// One decoder's frames of a batch, in array order: intra frames one by one,
// each run of consecutive inter frames with shared block launches (through
// decode_intra_then_run when an intra frame precedes the run, so that the
// run's block stage overlaps it; else decode_inter_run).  Stops at the
// first error other than NOT_CONVERGED.
hivc_status decode_own_frames(hivc_decoder *d, const hivc_frame *frames, const hivc_out *outs,
                              const std::vector<int> &ks)
{
    hivc_status worst = HIVC_OK;
    for (size_t i = 0; i < ks.size();) {
        if (frames[ks[i]].type == 0 && i + 1 < ks.size() && frames[ks[i + 1]].type == 1 && d->cfg.chroma != 2 &&
            !d->timing) {
            std::vector<int> run;
            size_t j = i + 1;
            while (j < ks.size() && frames[ks[j]].type == 1) run.push_back(ks[j++]);
            hivc_status intra = HIVC_OK;
            const hivc_status s = decode_intra_then_run(d, frames, outs, ks[i], run, intra);
            if (intra != HIVC_OK && intra != HIVC_E_NOT_CONVERGED) return intra;
            if (intra != HIVC_OK) worst = intra;
            if (s != HIVC_OK) return s;
            i = j;
            continue;
        }
        if (frames[ks[i]].type == 0) {
            const hivc_status s = hivc_decode_iframe(d, frames[ks[i]].i, &outs[ks[i]]);
            if (s != HIVC_OK && s != HIVC_E_NOT_CONVERGED) return s;
            if (s != HIVC_OK) worst = s;
            ++i;
            continue;
        }
        std::vector<int> run;
        while (i < ks.size() && frames[ks[i]].type == 1) run.push_back(ks[i++]);
        hivc_status s = HIVC_OK;
        if (d->cfg.chroma != 2) {
            s = decode_inter_run(d, frames, outs, run);
        } else {
            for (int k : run)
                if ((s = hivc_decode_pframe(d, frames[k].p, &outs[k])) != HIVC_OK) break;
        }
        if (s != HIVC_OK) return s;
    }
    return worst;
}

}  // namespace

hivc_status hivc_decode_batch(hivc_decoder *const *decs, const hivc_frame *frames, int32_t n, const hivc_out *outs)
{
    if (n < 0 || (n > 0 && (!decs || !frames || !outs))) return HIVC_E_INVALID;
    // every inter frame is checked before anything is launched
    std::vector<hivc_decoder *> ds;
    std::vector<std::vector<int>> ks;
    bool any_intra = false;
    for (int k = 0; k < n; ++k) {
        hivc_decoder *d = decs[k];
        if (!d || (frames[k].type != 0 && frames[k].type != 1)) return HIVC_E_INVALID;
        if (frames[k].type == 1 && !pframe_ok(d, frames[k].p, &outs[k])) return HIVC_E_INVALID;
        any_intra |= frames[k].type == 0;
        const size_t j = std::find(ds.begin(), ds.end(), d) - ds.begin();
        if (j == ds.size()) {
            ds.push_back(d);
            ks.emplace_back();
        }
        ks[j].push_back(k);
    }
    for (size_t j = 0; j < ds.size(); ++j) {
        bool ref = ds[j]->has_ref;
        for (int k : ks[j]) {
            if (frames[k].type == 0) ref = true;
            else if (!ref) return HIVC_E_NO_REFERENCE;
        }
    }
    // Decoders are independent and each has its own stream; every call
    // below only enqueues work (the intra solves decide their cycles on the
    // device), so one host thread issues them all and the decoders' work
    // overlaps on the GPU.  Every decoder stops at its own first error.
    std::vector<hivc_status> st(ds.size(), HIVC_OK);
    for (size_t j = 0; j < ds.size(); ++j) st[j] = decode_own_frames(ds[j], frames, outs, ks[j]);
    hivc_status worst = HIVC_OK;
    for (hivc_status s : st) {
        if (s != HIVC_OK && s != HIVC_E_NOT_CONVERGED) return s;
        if (s != HIVC_OK) worst = s;
    }
    return worst;
}

hivc_status hivc_decoder_sync(hivc_decoder *d, hivc_stats *last)
{
    if (!d) return HIVC_E_INVALID;
    if (cudaSetDevice(d->device) != cudaSuccess) return HIVC_E_CUDA;
    cudaError_t e = cudaMemcpyAsync(d->h_flags, d->flags, 4 * kStatusWords, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->flags, 0, 4 * kStatusWords, d->stream);
    // the intra solves' control state and statistics (cleared for the next
    // sync), the one read-back of the correction loop
    const size_t stat_off = offsetof(IntraCtl, sor_launches);
    const bool intra = d->intra_pending;
    if (e == cudaSuccess && intra)
        e = cudaMemcpyAsync(d->h_ctl, d->ctl, sizeof(IntraCtl), cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess && intra)
        e = cudaMemsetAsync(reinterpret_cast<char *>(d->ctl) + stat_off, 0, sizeof(IntraCtl) - stat_off, d->stream);
    // (the coarse start's statistics: launches and pixels only)
    if (e == cudaSuccess && intra)
        e = cudaMemcpyAsync(d->h_ctl_c, d->ctl_c, sizeof(IntraCtl), cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess && intra)
        e = cudaMemsetAsync(reinterpret_cast<char *>(d->ctl_c) + stat_off, 0, sizeof(IntraCtl) - stat_off, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) return HIVC_E_CUDA;
    bool not_converged = false;
    if (intra) {
        const IntraCtl &c = *d->h_ctl;
        for (int p = 0; p < 3; ++p) d->st.resid[p] = p < d->np ? c.rn[p] : 0.0;
        d->st.cycles = c.cycles;
        d->st.sweeps = c.sweeps_max;
        d->st.kernel_launches[1] += (int32_t)c.sor_launches;
        d->st.kernel_launches[2] += (int32_t)c.res_launches;
        d->st.kernel_pixels[1] += c.sor_pixels;
        d->st.kernel_pixels[2] += c.res_pixels;
        d->st.launches += (int32_t)(c.sor_launches + c.res_launches);
        const IntraCtl &cc = *d->h_ctl_c;  // the coarse start's sweeps: a family of their own
        d->st.kernel_launches[7] += (int32_t)cc.sor_launches;
        d->st.kernel_launches[2] += (int32_t)cc.res_launches;
        d->st.kernel_pixels[7] += cc.sor_pixels;
        d->st.kernel_pixels[2] += cc.res_pixels;
        d->st.launches += (int32_t)(cc.sor_launches + cc.res_launches);
        not_converged = c.unconverged > 0;
        d->intra_pending = false;
    }
    d->st.device_flags = d->h_flags[0];
    std::memcpy(&d->st.max_cond, d->h_flags + 1, sizeof(float));
    d->st.fp64_blocks = (int32_t)d->h_flags[2];
    d->st.large_blocks = (int32_t)d->h_flags[3];
    d->st.group_blocks = (int32_t)d->h_flags[4];
    d->st.layout_groups = (int32_t)d->h_flags[5];
    for (auto &pe : d->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess)
            d->st.kernel_ms[pe.first] += ms;
        d->event_pool.push_back(pe.second.first);
        d->event_pool.push_back(pe.second.second);
    }
    d->pending.clear();
    if (last) *last = d->st;
    const uint32_t fl = d->st.device_flags;
    hivc_stats fresh{};
    std::memcpy(fresh.resid, d->st.resid, sizeof(fresh.resid));
    fresh.cycles = d->st.cycles;
    fresh.sweeps = d->st.sweeps;
    d->st = fresh;
    if (fl & ~kFlagCond) return HIVC_E_INVALID;
    return not_converged ? HIVC_E_NOT_CONVERGED : HIVC_OK;
}

// ---------------------------------------------------------------------------
// step entry points
// ---------------------------------------------------------------------------

size_t hivc_block_residual_workspace_bytes(int32_t width, int32_t height, int32_t block, int32_t n_points)
{
    if (width < 1 || height < 1 || block < 1 || block > kMaxB || n_points < 0) return 0;
    const size_t nb = (size_t)((width + block - 1) / block) * ((height + block - 1) / block);
    return a256(4 * (size_t)n_points) + a256(4 * nb) + 256 + a256(4 * kBigFloats * (size_t)block_ranges((int)nb)) +
           block_plan_bytes((int)nb, false);
}

hivc_status hivc_block_residual(int32_t width, int32_t height, int32_t block, const hivc_residual *res, float *r,
                                int32_t r_pitch, void *workspace, size_t ws_bytes, uint32_t *flags, void *stream)
{
    if (!res || !r || !residual_ok(*res) || r_pitch < width) return HIVC_E_INVALID;
    const size_t need = hivc_block_residual_workspace_bytes(width, height, block, res->n_points);
    if (need == 0 || !workspace || ws_bytes < need) return HIVC_E_INVALID;
    if (ensure_block_tables() != cudaSuccess) return HIVC_E_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *w = static_cast<char *>(workspace);
    const int nbx = (width + block - 1) / block;
    const int nb = nbx * ((height + block - 1) / block);
    float *coef = reinterpret_cast<float *>(w);
    w += a256(4 * (size_t)res->n_points);
    float *acoef = reinterpret_cast<float *>(w);
    w += a256(4 * (size_t)nb);
    uint32_t *own_flags = reinterpret_cast<uint32_t *>(w);
    w += 256;
    float *big = reinterpret_cast<float *>(w);
    w += a256(4 * kBigFloats * (size_t)block_ranges(nb));
    BlockScratch S{flags, big, block_ranges(nb)};
    S.plan = carve_block_plan(w, nb, false);
    if (!flags) {
        flags = own_flags;
        if (cudaMemsetAsync(flags, 0, 4, st) != cudaSuccess) return HIVC_E_CUDA;
    }
    BlockJobs J{};
    J.n = 1;
    BlockPlane &B = J.p[0];
    B.block_ptr = res->block_ptr;
    B.pos = res->pos;
    B.val[0] = res->val;
    B.coef[0] = coef;
    B.acoef[0] = acoef;
    B.r[0] = r;
    B.r_pitch = r_pitch;
    B.n_points = res->n_points;
    B.width = width;
    B.height = height;
    B.block = block;
    B.nbx = nbx;
    B.nblocks = nb;
    J.total_blocks = nb;
    S.flags = flags;
    cudaError_t e = launch_block_coef(J, S, st, nullptr);
    if (e == cudaSuccess) e = launch_block_eval(J, flags, st);
    return cuda_status(e);
}

hivc_status hivc_warp(int32_t width, int32_t height, const float *ref, int32_t ref_pitch, const float *flow,
                      int32_t flow_width, int32_t flow_height, int32_t chroma_flow, float *pred, int32_t pred_pitch,
                      void *stream)
{
    if (width < 1 || height < 1 || !ref || !flow || !pred || ref_pitch < width || pred_pitch < width)
        return HIVC_E_INVALID;
    if (chroma_flow) {
        if ((flow_width + 1) / 2 != width || (flow_height + 1) / 2 != height) return HIVC_E_INVALID;
    } else if (flow_width != width || flow_height != height) {
        return HIVC_E_INVALID;
    }
    WarpJobs W{};
    W.n = 1;
    WarpPlane &P = W.p[0];
    P.ref = ref;
    P.ref_pitch = ref_pitch;
    P.flow = flow;
    P.flow_w = flow_width;
    P.flow_h = flow_height;
    P.chroma_flow = chroma_flow ? 1 : 0;
    P.pred_out = pred;
    P.pred_pitch = pred_pitch;
    P.width = width;
    P.height = height;
    return cuda_status(launch_warp_add(W, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// side information by rectangular subdivision (Sec. 2.3)
// ---------------------------------------------------------------------------
size_t hivc_flow_from_tree_workspace_bytes(int64_t nbits)
{
    return nbits < 1 ? 0 : tree_workspace_bytes(nbits);
}

hivc_status hivc_flow_from_tree(int32_t width, int32_t height, const uint32_t *bits, int64_t nbits,
                                const float *values, int32_t n_values, float *flow, void *workspace, size_t ws_bytes,
                                uint32_t *flags, void *stream)
{
    if (width < 1 || height < 1 || width > 16384 || height > 16384 || !bits || nbits < 1 ||
        nbits > 2 * (int64_t)width * height || !values || n_values < 1 || !flow || !workspace ||
        ws_bytes < tree_workspace_bytes(nbits) || ((uintptr_t)workspace & 15) || ((uintptr_t)flow & 7) ||
        ((uintptr_t)values & 7))
        return HIVC_E_INVALID;
    if (ensure_block_tables() != cudaSuccess) return HIVC_E_CUDA;
    const cudaError_t e = launch_flow_from_tree(width, height, bits, nbits, values, n_values, flow, workspace, flags,
                                                block_tables().sms, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HIVC_OK : HIVC_E_CUDA;
}

hivc_status hivc_masks_from_trees(int32_t width, int32_t height, int32_t block, const uint32_t *bits,
                                  const uint32_t *tree_ptr, uint32_t *block_ptr, uint8_t *pos, int64_t max_points,
                                  uint32_t *flags, void *stream)
{
    if (width < 1 || height < 1 || width > 16384 || height > 16384 || block < 1 || block > kMaxB || !bits ||
        !tree_ptr || !block_ptr || (max_points > 0 && !pos) || max_points < 0)
        return HIVC_E_INVALID;
    if (ensure_block_tables() != cudaSuccess) return HIVC_E_CUDA;
    const cudaError_t e = launch_masks_from_trees(width, height, block, bits, tree_ptr, block_ptr, pos, max_points,
                                                  flags, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HIVC_OK : HIVC_E_CUDA;
}

size_t hivc_intra_mask_from_tree_workspace_bytes(int32_t width, int32_t height, int64_t nbits)
{
    if (width < 1 || height < 1 || nbits < 1) return 0;
    return intra_tree_workspace_bytes(nbits, width, height);
}

hivc_status hivc_intra_mask_from_tree(int32_t width, int32_t height, const uint32_t *bits, int64_t nbits,
                                      uint32_t *idx, int64_t max_points, int32_t *n_points, void *workspace,
                                      size_t ws_bytes, uint32_t *flags, void *stream)
{
    if (width < 1 || height < 1 || width > 16384 || height > 16384 || !bits || nbits < 1 ||
        nbits > 2 * (int64_t)width * height || max_points < 0 || (max_points > 0 && !idx) || !n_points ||
        !workspace || ws_bytes < intra_tree_workspace_bytes(nbits, width, height) || ((uintptr_t)workspace & 15))
        return HIVC_E_INVALID;
    if (ensure_block_tables() != cudaSuccess) return HIVC_E_CUDA;
    const cudaError_t e = launch_intra_mask_from_tree(width, height, bits, nbits, idx, max_points, n_points, workspace,
                                                      flags, block_tables().sms, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HIVC_OK : HIVC_E_CUDA;
}

hivc_status hivc_set_sor_variant(int32_t variant)
{
    return set_sor_variant(variant) == 0 ? HIVC_OK : HIVC_E_INVALID;
}
