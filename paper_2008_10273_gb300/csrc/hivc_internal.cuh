// Internal declarations shared by the CUDA translation units of libhivc.
// Host launchers are plain C++ functions (no relocatable device code).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

#include "hivc.h"

namespace hivc {

constexpr int kMaxB = 16;   // largest residual block edge
constexpr int kWarpK = 32;  // blocks with K <= kWarpK are solved by one warp
constexpr int kMaxJobs = 16;
constexpr int kNumOps = 2;  // residual operators: 0 harmonic (A = -L), 1 biharmonic (A = L^2)

// Error bits the kernels OR into a device status word (never trap).
enum : uint32_t {
    kFlagBlockPtr = 1u << 0,  // block_ptr decreasing, [0] != 0 or beyond n_points
    kFlagK = 1u << 1,         // K_b > w*h - 1
    kFlagPos = 1u << 2,       // position outside the block or not increasing
    kFlagNotSPD = 1u << 3,    // non-positive Cholesky pivot
    kFlagMaskIdx = 1u << 4,   // intra mask index out of range or not increasing
    // bit 5 is unused (no kernel of the library waits on another)
    kFlagCond = 1u << 6,      // information, not an error: a block above the
                              // condition threshold kept its FP32 solution
                              // (K > kF64MaxK: no room for the FP64 system)
    kFlagQ = 1u << 7,         // coefficient index -128 (outside [-127, 127])
    kFlagTree = 1u << 8,      // a subdivision tree's bits are invalid (side information)
};

// ---------------------------------------------------------------------------
// block residual (Sec. 2.2)
// ---------------------------------------------------------------------------
// One plane of block data.  val[1] != nullptr marks a second plane that
// shares block_ptr/pos (Cb/Cr with one chroma mask): one factorisation,
// two right-hand sides.
struct BlockPlane {
    const uint32_t *block_ptr;
    const uint8_t *pos;
    const int16_t *val[2];
    float *coef[2];   // per point: Green's coefficient c_j
    float *acoef[2];  // per block: the constant a
    float *r[2];      // residual field (eval stage), may be nullptr
    int32_t r_pitch;  // floats
    int32_t n_points, width, height, block, nbx, nblocks, block_base;
    // coefficient mode (evaluation only): per point the dead-zone index of c
    // (val unused), acoef[0] the transmitted constants; c = sign(q)(|q| +
    // qoff) qstep, 0 for q = 0
    const int8_t *q;
    float qstep, qoff;
};

struct BlockJobs {
    BlockPlane p[kMaxJobs];
    int32_t n;
    int32_t total_blocks;
    int32_t op;  // residual operator of every job
};

// Device addresses of the Green's matrices of all block shapes (uploaded
// once per device) and the SM count of the device.
struct BlockTables {
    const float *G;     // rows of G per shape, padded to multiples of 8 floats
    const float *G16o;  // the 16 x 16 shape's rows of 36 points in 4 orientations (block_device.cuh)
    const double *G64;  // the same in double precision (FP64 re-solves)
    const int *goff;    // offset of shape (w, h) at (w-1)*16 + (h-1)
    int sms;
    float amax;         // bound on the operator's eigenvalues (8, or 64 for L^2)
};

constexpr int kBigMaxK = 255;  // largest K of a 16 x 16 block
// one packed FP32 system (L, three right-hand sides), rounded up to 256 bytes
constexpr size_t kBigFloats = ((size_t)kBigMaxK * (kBigMaxK + 1) / 2 + 3 * kBigMaxK + 63) / 64 * 64;
// largest K whose FP64 system fits in a slot
constexpr int kF64MaxK = 179;
static_assert((size_t)kF64MaxK * (kF64MaxK + 1) / 2 + 3 * kF64MaxK <= kBigFloats / 2, "FP64 system fits a slot");
constexpr int kRange = 128;    // blocks per range of the coefficient kernel

// ranges of kRange blocks for total_blocks blocks
__host__ __device__ inline int block_ranges(int total_blocks) { return (total_blocks + kRange - 1) / kRange; }

// ---- planning of the block stage ------------------------------------------
// Every launch of the coefficient stage is planned first: the blocks go to
// work lists by their point count K (classes in queue order, heavy first:
// K > 32, 25..32, 17..24, 13..16, 9..12, 1..8), which a persistent kernel
// takes off one queue.  Optionally the blocks of each plane that share one
// mask layout (the same K and positions, at least kGroupMin of them, K <=
// kGroupMaxK) form a layout group: one factorisation for the group, and the
// residual of all its blocks as one tensor-core product (Eq. 3 for a fixed
// layout is linear in the values: r = E v).
constexpr int kClasses = 6;
constexpr int kGroupMaxK = 32;   // layouts with more points are not grouped
constexpr int kGroupMin = 16;    // blocks of one layout before it is grouped
constexpr int kMaxGroups = 256;  // groups per launch (more layouts stay per block)
constexpr int kGroupRows = 256;  // pixels of the largest block (16 x 16)
constexpr int kHashProbes = 32;  // linear probes of the layout table

// device state of one planned launch, zeroed before the plan
struct BlockPlanState {
    uint32_t count[kClasses];    // entries per class list
    uint32_t next;               // the coefficient kernel's main work queue
    uint32_t next0;              // its queue of K > 32 blocks (CTAs with a slot)
    uint32_t finished;           // CTAs of the coefficient kernel done
    uint32_t ndef;               // FP64 re-solves deferred to the last CTA
    uint32_t ngroups;            // layout groups claimed
    uint32_t gfill[kMaxGroups];  // member entries listed per group
    int32_t gslot[kMaxGroups];   // layout-table slot of group g
    int32_t grep[kMaxGroups];    // a block of group g (its layout is the group's)
};

struct BlockPlan {
    BlockPlanState *st;  // device
    int32_t *list;       // kClasses x cap global block indices
    int32_t *deferred;   // cap entries: FP64 re-solves for the last CTA
    int32_t cap;         // >= the launch's blocks
    // layout groups (hkey == nullptr: off)
    unsigned long long *hkey;  // layout table: fingerprint per slot (0 = empty)
    uint32_t *hcnt;            // blocks per slot
    uint32_t *hgid;            // group id + 1 of the slot (0 = none)
    uint32_t hmask;            // slots - 1 (a power of two)
    int32_t *slot_of;          // per block: its slot, or -1
    uint8_t *member;           // per block: 1 = evaluated by its group's product
    int32_t *gmem;             // member entries (block * 2 + value plane), 2 x cap
    uint16_t *E;               // per group: 3 bf16 splits of E, kGroupRows x kGroupMaxK each
};

// Device bytes of a plan for total_blocks blocks (with layout groups or
// not), and the plan carved from such memory (256-byte aligned).
size_t block_plan_bytes(int total_blocks, bool groups);
BlockPlan carve_block_plan(void *mem, int total_blocks, bool groups);

// Scratch of the coefficient stage: room for one K > 32 system per CTA of
// the persistent coefficient kernel (a CTA solves its large blocks one after
// the other in its slot; an FP64 re-solve uses the slot as doubles), and
// the plan of the launch.
//
// Condition control: every block's bound kappa = 8 tr(G_PP) / (1 - K/N) on
// cond_2(G_PP) (lambda_max <= tr, lambda_min >= (1 - K/N) / 8 since the
// eigenvalues of A = -L are at most 8) is compared with tau; a block above
// it is re-solved in FP64 from the FP64 Green's table.
struct BlockScratch {
    uint32_t *flags;  // device error word
    float *big;       // big_ranges * kBigFloats floats
    int32_t big_ranges;
    uint32_t *cstat = nullptr;  // nullptr, or [0] max kappa (float bits), [1] FP64 blocks, [2] K > 32 blocks,
                                // [3] blocks of layout groups (per value plane), [4] layout groups
    float tau = 1e6f;           // condition threshold
    BlockPlan plan{};           // lists and layout groups of the launch
};

// ---- autotuner table (tune.cu): choices keyed by GPU name and shape, kept
// for the process and in a JSON file; -1 when there is none ---------------
std::string gpu_name();  // of the current device
int tune_lookup(const std::string &key);
void tune_store(const std::string &key, int value);

cudaError_t ensure_block_tables();
const BlockTables &block_tables(int op = 0);  // of the current device, for operator op

// c, a for every block (a = NaN: bad positions): the plan (work lists;
// layout groups when s.plan.hkey is set, after a clear of the layout table
// and one pass that enters every block's layout), then one persistent launch:
// one thread per block for K <= 12, warps for K <= 32, a whole CTA for
// K > 32, and one CTA per layout group for its factorisation.  The
// kernels' completion publishes every result.  pdl: the first launch may
// start while the previous kernel in the stream finishes.
cudaError_t launch_block_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st, int *launches,
                              bool pdl = false);
// r-field from c, a (Eq. 3 by Green's rows), r = v at the points; or, for
// jobs in coefficient mode (p[k].q set, all jobs alike), from the
// dequantised indices and the transmitted constants, with no overwrite.
// plan: the launch's plan when its layout groups are on, else nullptr; the
// launch's first CTAs then form the groups' residual planes, per group
// R = V E^T on the tensor cores (bf16 values, E in three bf16 parts, FP32
// accumulation), beside the per-block evaluation of the other blocks.
cudaError_t launch_block_eval(const BlockJobs &jobs, uint32_t *flags, cudaStream_t st, bool pdl = false,
                              const BlockPlan *plan = nullptr);
// CTAs of the persistent coefficient kernel on this device (slots needed)
int block_coef_ctas();

// One inter frame for the pixel kernel: flow, references, the residual
// planes the block kernels evaluated, outputs.
struct InterFrame {
    const float *flow;
    const float *ref[3];
    float *ref_out[3];
    uint8_t *out[3];
    const float *r[3];
    int32_t ref_pitch[3], out_pitch[3], r_pitch[3];  // ref_out shares ref_pitch
    int32_t width, height, chroma;                   // chroma: 0 grey, 1 4:2:0
};

// Warp + residual + clamp + pack, one thread per luma quad and its co-sited
// chroma pixels.  pdl: launch as a programmatic dependent of the previous
// kernel in the stream.  early: that kernel is the previous frame's pixel
// kernel (which waited for the residual planes), so the flow and residual
// loads may go out before waiting for it.
cudaError_t launch_pframe(const InterFrame &f, cudaStream_t st, bool pdl, bool early = false);

// One inter frame through the fused pixel kernel: the residual of Eq. 3
// evaluated per block from the coefficients of the block stage into shared
// memory, then the warp, add, clamp and pack of the block's pixels (no
// residual planes in memory).  Same values as the evaluation kernel
// followed by pframe_kernel, bit for bit.
struct FusedFrame {
    InterFrame px;        // flow, references, outputs (px.r unused)
    BlockPlane y;         // the luma job (coefficients in coef[0], acoef[0])
    BlockPlane c[2];      // chroma: one paired job (Cb in [0], Cr in [1] of val/coef/acoef), or the Cb and Cr jobs
    int32_t nc;           // chroma jobs: 0 (grey), 1 (paired) or 2
    int32_t op;           // residual operator (its Green's table)
    uint32_t *flags;      // data errors (bad positions)
    int32_t early;        // 1: evaluate before waiting for the preceding grid (which itself waited)
};
// Whether the fused kernel takes this frame: 4:2:0 or grey, 16 x 16 blocks,
// even plane sizes and the pixel kernel's whole-quad alignment.
bool pframe_fused_ok(const InterFrame &f, int block);
cudaError_t launch_pframe_fused(const FusedFrame &f, cudaStream_t st, bool pdl);

// ---------------------------------------------------------------------------
// warp + add + pack (Sec. 2, 2.3)
// ---------------------------------------------------------------------------
struct WarpPlane {
    const float *ref;    // FP32 reference plane (inter), or nullptr
    const float *src_hi; // intra prediction hi (+ lo) when ref == nullptr
    const float *src_lo; // may be nullptr
    const float *src_hi1, *src_lo1;  // the other buffer of the iterate's ping-pong
    const int32_t *src_sel;          // device: 1 = take src_hi1/src_lo1 (or nullptr)
    const float *r;      // residual field or nullptr
    float *ref_out;      // new FP32 reference (clamped), or nullptr
    uint8_t *out;        // uint8 output, or nullptr
    float *pred_out;     // raw prediction (step entry point), or nullptr
    const float *flow;   // luma flow (H x W x 2) for inter planes
    int32_t ref_pitch, src_pitch, r_pitch, ref_out_pitch, out_pitch, pred_pitch;
    int32_t width, height;
    int32_t flow_w, flow_h;  // luma flow size
    int32_t chroma_flow;     // 1: v = half mean of the 2x2 luma vectors
    int32_t tiles_x, tile_base;
};

struct WarpJobs {
    WarpPlane p[kMaxJobs];
    int32_t n;
    int32_t total_tiles;
};

cudaError_t launch_warp_add(WarpJobs &jobs, cudaStream_t st);

// One 4:4:4 frame of the colour path of Sec. 2.3 (RCT planes Y, U, V of one
// size and pitch): prediction (backward warp of the three reference planes
// along the luma flow, or the intra solution), + residual, clamp (Y to
// [0, 255], U and V to [-255, 255]), new FP32 references, and the inverse
// RCT of the rounded planes packed as R, G, B.
struct RctFrame {
    const float *flow;                   // inter: luma flow (H x W x 2); nullptr: intra
    const float *ref[3];                 // inter: previous reference planes
    const float *src_hi[3], *src_lo[3];  // intra: the inpainted planes (lo may be nullptr)
    const float *src_hi1[3], *src_lo1[3];  // the other buffers of the iterate's ping-pong
    const int32_t *src_sel;              // device, per plane: 1 = take src_hi1/src_lo1 (or nullptr)
    const float *r[3];                   // residual planes, or nullptr
    float *ref_out[3];
    uint8_t *out[3];                     // R, G, B
    int32_t pitch;                       // floats, every FP32 plane
    int32_t out_pitch[3];
    int32_t width, height;
};

cudaError_t launch_rct(const RctFrame &f, cudaStream_t st);

// ---------------------------------------------------------------------------
// side information by rectangular subdivision (Sec. 2.3)
// ---------------------------------------------------------------------------
size_t tree_workspace_bytes(long long nbits);
// dense flow from the plane's tree and one vector per leaf
cudaError_t launch_flow_from_tree(int W, int H, const uint32_t *bits, long long nbits, const float *values,
                                  int n_values, float *flow, void *ws, uint32_t *flags, int sms, cudaStream_t st);
// intra mask indices (sorted) and their count from the plane's tree
size_t intra_tree_workspace_bytes(long long nbits, int W, int H);
cudaError_t launch_intra_mask_from_tree(int W, int H, const uint32_t *bits, long long nbits, uint32_t *idx,
                                        long long max_points, int32_t *n_out, void *ws, uint32_t *flags, int sms,
                                        cudaStream_t st);
// residual mask points (block_ptr, pos) from one tree per block
cudaError_t launch_masks_from_trees(int W, int H, int B, const uint32_t *bits, const uint32_t *tree_ptr,
                                    uint32_t *block_ptr, uint8_t *pos, long long max_points, uint32_t *flags,
                                    cudaStream_t st);

// ---------------------------------------------------------------------------
// intra solve (Sec. 2.1)
// ---------------------------------------------------------------------------
struct IntraPlane {
    int32_t width, height, pitch;  // pitch in elements
    const uint32_t *idx;           // mask indices
    const uint8_t *val;            // mask values
    const int16_t *val16;          // signed mask values (RCT chroma) instead, or nullptr
    int32_t n;                     // mask size
    uint8_t *mask;                 // 1 = known pixel
    float *uh[2], *ul[2];          // iterate u = hi + lo, ping-pong (IntraCtl.upar)
    float *res;                    // FP32 Eq. 1 residual
    float *e[2];                   // FP32 correction, ping-pong (launch it reads e[it & 1])
    unsigned long long *vsum;      // scratch: sum of mask values
    int32_t ff;                    // 1: float-float iterate, 0: FP32 only
    int32_t tiles_x, tile_base;    // filled by the launchers
    int32_t tiles;                 // regions of the plane (filled by the launchers)
};

// Control state of one intra solve, in device memory: the correction loop
// decides on the device (no host read between cycles).  The last CTA of
// each residual launch plans the next cycle (sweeps per plane from the
// residual reached and the observed contraction, Young's relation for the
// relaxation factor).  Sweep launches come in pairs of fixed parity (launch
// it = 2 i + parity of pair i reads correction buffer e[it & 1] and writes
// the other, so a plane's correction after its nl launches sits in
// e[nl & 1]).  A launch of parity q reads i from iter[q], and its first
// CTA hands i on: parity 0 to iter[1], parity 1 as i + 1 to iter[0], with
// whether the sweep loop goes on (no launch reads the word that another
// running launch writes).  Both publish whether the loops go on, to
// conditional graph nodes (h_outer, h_inner) and to go_outer / go_inner.
struct IntraCtl {
    double tol;                // max |(L u)_i| to reach
    double rn[3];              // residual reached per plane
    double rate[3];            // contraction per sweep per plane
    float omega[3];            // relaxation factor per plane
    int32_t max_cycles, spl;   // cycle cap, sweeps per launch
    int32_t max_sweeps, pad0;  // cap on a plane's sweeps in one cycle
    int32_t nl[3];             // sweep launches of the current cycle per plane
    int32_t maxl, cycles;      // launches of the cycle, cycles done
    int32_t iter[2];           // pairs done, as the launches of parity 0 and 1 read it
    int32_t pairs[2];          // launch pairs of the cycle: over all planes, then over the chroma planes alone
    int32_t sweeps[3], sweeps_max;
    int32_t upar[3];           // the u buffer holding a plane's current iterate
    uint32_t rbits[3];         // max |residual| of the last residual launch (float bits)
    uint32_t done_ctas;        // CTAs of the current launch that finished
    int32_t go_outer, go_inner, converged;
    // statistics since the decoder's last sync (kept across solves): sweep
    // and residual launches and the pixels they covered, solves that ended
    // above the tolerance
    int64_t sor_launches, sor_pixels, res_launches, res_pixels, unconverged;
};

struct IntraJobs {
    IntraPlane p[3];
    int32_t n;
    IntraCtl *ctl;                      // control state
    unsigned long long h_outer, h_inner;  // conditional handles (0: launched from the host)
    unsigned long long h_inner_c;       // the chroma phase's loop (0: launched from the host)
    int32_t chroma_phase;               // 1: the launches that sweep only the chroma planes use regions of their own
};

cudaError_t launch_intra_init(IntraJobs &jobs, uint32_t *flags, cudaStream_t st, int *launches);
// The coarse start: the fine planes' mask restricted to the half-size
// planes of C (after launch_intra_init), and, after C's solve, the
// unknown fine pixels set from C's solution.
cudaError_t launch_intra_restrict(const IntraJobs &fine, const IntraJobs &coarse, cudaStream_t st);
cudaError_t launch_intra_prolong(const IntraJobs &fine, const IntraJobs &coarse, cudaStream_t st);
// The control state for a new solve: omega0 per plane, tolerance, cycle
// cap, and the cap on a plane's sweeps in one cycle (kS .. 600).
cudaError_t launch_intra_ctl_init(const IntraJobs &jobs, const float *omega0, double tol, int max_cycles,
                                  cudaStream_t st, int max_sweeps = 600);
// One residual launch: first = the start of the solve (res = L u, the
// norms, the first cycle's plan), else the end of a cycle (u += e for the
// planes that swept, res, norms, the next cycle's plan).
cudaError_t launch_intra_residual(IntraJobs &jobs, bool first, cudaStream_t st);
// One pair of launches of kS red-black sweeps each over the planes the
// control state keeps active (variant: the region tiling, see
// set_sor_variant).
cudaError_t launch_intra_sor_pair(IntraJobs &jobs, int variant, cudaStream_t st);
// One pair of the chroma phase's launches (jobs.chroma_phase): the chroma
// planes alone, with regions of 128 x 88.
cudaError_t launch_intra_sor_chroma_pair(IntraJobs &jobs, cudaStream_t st);
// The SOR tiling for these planes: tuned (timing launches on tune_ctl, a
// control state of its own), looked up, or pinned.
int intra_sor_variant(IntraJobs &jobs, IntraCtl *tune_ctl, cudaStream_t st);
// The whole correction loop as a graph: the first residual launch, then
// while the plan says so: (sweep launches while the plan says so, then a
// residual launch).  Conditional WHILE nodes; jobs.ctl is the state.
cudaError_t build_intra_graph(const IntraJobs &jobs, int variant, cudaGraphExec_t *exec);
int intra_sweeps_per_launch();
cudaError_t intra_init();  // once per device
int set_sor_variant(int v);  // -1: autotune; 0..2 pin a variant (0 on success)

}  // namespace hivc
