// hivc_block_residual_static: the block residual of hivc_block_residual
// without any device allocation by the library or the caller.
//
// Some callers cannot allocate device memory at the point where they need a
// residual plane: a host that hands the library a fixed memory budget in
// which every allocation was made at start-up, or a latency-bound loop in
// which a cudaMalloc or cudaFree (which may synchronise the whole device)
// would stall the work of other streams.  For them the scratch that the
// coefficient stage needs (per-point coefficients, per-block constants and
// room for one system with more than 32 points per range of 128 blocks, and
// the work lists of the launch)
// lives in a fixed-size array in the library's device image instead of a
// caller workspace.
//
// The array (about 17 MB) exists once per device on which this entry point
// has run and stays allocated until the process exits.  Every call on a
// device uses the same array, so calls whose work overlaps on the GPU (for
// example on two streams) race and must be serialised by the caller.  The
// kernels keep no counters from one call to the next; a call without a
// caller error word clears the library's own before its kernels run.
#include <mutex>

#include "hivc_internal.cuh"

using namespace hivc;

namespace {

constexpr int kStaticMaxPoints = 1 << 17;  // residual points per call
constexpr int kStaticMaxBlocks = 1 << 14;  // residual blocks per call
// 4-byte words: coefficients | block constants | own error word (+ padding)
// | one K > 32 system per range of kRange blocks | the launch's plan (work
// lists by point count, no layout groups)
constexpr size_t kOffAcoef = kStaticMaxPoints;
constexpr size_t kOffFlags = kOffAcoef + kStaticMaxBlocks;
constexpr size_t kOffBig = kOffFlags + 64;  // keeps the systems 256-byte aligned
constexpr int kStaticRanges = kStaticMaxBlocks / kRange;
constexpr size_t kOffPlan = kOffBig + (size_t)kStaticRanges * kBigFloats;
// at least block_plan_bytes(kStaticMaxBlocks, false): the state (under
// 8 KB), the class lists and the deferred list (checked at run time)
constexpr size_t kPlanWords = (8192 + 4 * (size_t)kStaticMaxBlocks * (kClasses + 1)) / 4;
static_assert(sizeof(BlockPlanState) + 256 <= 8192, "plan state fits its share");
constexpr size_t kWords = kOffPlan + kPlanWords;

static __device__ __align__(256) uint32_t g_scratch[kWords];

std::mutex g_mu;
uint32_t *g_addr[64];  // device address of g_scratch, per device

}  // namespace

extern "C" hivc_status hivc_block_residual_static(int32_t width, int32_t height, int32_t block,
                                                  const hivc_residual *res, float *r, int32_t r_pitch,
                                                  uint32_t *flags, void *stream)
{
    if (!res || !r || width < 1 || height < 1 || block < 1 || block > kMaxB || r_pitch < width) return HIVC_E_INVALID;
    if (!res->block_ptr || res->n_points < 0 || (res->n_points > 0 && (!res->pos || !res->val)))
        return HIVC_E_INVALID;
    const int nbx = (width + block - 1) / block;
    const long nb = (long)nbx * ((height + block - 1) / block);
    if (res->n_points > kStaticMaxPoints || nb > kStaticMaxBlocks) return HIVC_E_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HIVC_E_CUDA;
    // first call on this device: Green's tables and the scratch address (with
    // this device current; make this call before any stream capture)
    if (ensure_block_tables() != cudaSuccess) return HIVC_E_CUDA;
    uint32_t *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return HIVC_E_CUDA;
            g_addr[dev] = static_cast<uint32_t *>(p);
        }
        base = g_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the own error word starts at zero when none is given
    if (!flags) {
        flags = base + kOffFlags;
        if (cudaMemsetAsync(flags, 0, sizeof(uint32_t), st) != cudaSuccess) return HIVC_E_CUDA;
    }
    BlockJobs J{};
    J.n = 1;
    BlockPlane &B = J.p[0];
    B.block_ptr = res->block_ptr;
    B.pos = res->pos;
    B.val[0] = res->val;
    B.coef[0] = reinterpret_cast<float *>(base);
    B.acoef[0] = reinterpret_cast<float *>(base + kOffAcoef);
    B.r[0] = r;
    B.r_pitch = r_pitch;
    B.n_points = res->n_points;
    B.width = width;
    B.height = height;
    B.block = block;
    B.nbx = nbx;
    B.nblocks = (int)nb;
    J.total_blocks = (int)nb;
    if (block_plan_bytes((int)nb, false) > 4 * kPlanWords) return HIVC_E_INVALID;
    BlockScratch S{flags, reinterpret_cast<float *>(base + kOffBig), kStaticRanges};
    S.plan = carve_block_plan(base + kOffPlan, (int)nb, false);
    cudaError_t e = launch_block_coef(J, S, st, nullptr);
    if (e == cudaSuccess) e = launch_block_eval(J, flags, st);
    return e == cudaSuccess ? HIVC_OK : HIVC_E_CUDA;
}
