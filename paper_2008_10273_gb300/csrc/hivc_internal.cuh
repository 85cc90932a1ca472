// Internal declarations shared by the CUDA translation units of libhivc.
// Host launchers are plain C++ functions (no relocatable device code).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

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

// Scratch of the coefficient stage: room for one K > 32 system per range
// of kRange blocks (the range's CTA solves its large blocks one after the
// other in its slot; an FP64 re-solve uses the slot as doubles).
//
// Condition control: every block's bound kappa = 8 tr(G_PP) / (1 - K/N) on
// cond_2(G_PP) (lambda_max <= tr, lambda_min >= (1 - K/N) / 8 since the
// eigenvalues of A = -L are at most 8) is compared with tau; a block above
// it is re-solved in FP64 from the FP64 Green's table.
struct BlockScratch {
    uint32_t *flags;  // device error word
    float *big;       // big_ranges * kBigFloats floats
    int32_t big_ranges;
    uint32_t *cstat = nullptr;  // nullptr, or [0] max kappa (float bits), [1] FP64 blocks, [2] K > 32 blocks
    float tau = 1e6f;           // condition threshold
};

cudaError_t ensure_block_tables();
const BlockTables &block_tables(int op = 0);  // of the current device, for operator op

// c, a for every block (a = NaN: bad positions): one thread per block for
// K <= 12, warps for K <= 32, a whole CTA for K > 32.  One launch, no
// counters: the kernel's completion publishes every result.
// pdl: launch as a programmatic dependent of the previous kernel in the
// stream (the coefficient stage overlaps it and completes after it).
cudaError_t launch_block_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st, int *launches,
                              bool pdl = false);
// r-field from c, a (Eq. 3 by Green's rows), r = v at the points; or, for
// jobs in coefficient mode (p[k].q set, all jobs alike), from the
// dequantised indices and the transmitted constants, with no overwrite.
cudaError_t launch_block_eval(const BlockJobs &jobs, uint32_t *flags, cudaStream_t st, bool pdl = false);

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
// kernel in the stream.
cudaError_t launch_pframe(const InterFrame &f, cudaStream_t st, bool pdl);

// ---------------------------------------------------------------------------
// warp + add + pack (Sec. 2, 2.3)
// ---------------------------------------------------------------------------
struct WarpPlane {
    const float *ref;    // FP32 reference plane (inter), or nullptr
    const float *src_hi; // intra prediction hi (+ lo) when ref == nullptr
    const float *src_lo; // may be nullptr
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
    float *uh[2], *ul[2];          // iterate u = hi + lo ([0] current, [1] next)
    float *res;                    // FP32 Eq. 1 residual
    float *e[2];                   // FP32 correction, ping-pong
    unsigned long long *vsum;      // scratch: sum of mask values
    unsigned int *rnorm;           // scratch: max |residual| (float bits)
    float omega;                   // SOR relaxation factor
    int32_t ff;                    // 1: float-float iterate, 0: FP32 only
    int32_t tiles_x, tile_base;    // filled by the launchers
};

struct IntraJobs {
    IntraPlane p[3];
    int32_t n;
};

cudaError_t launch_intra_init(IntraJobs &jobs, uint32_t *flags, cudaStream_t st, int *launches);
// u_next = u + e (unless first), res = (L u_next) at unknowns, rnorm = max |res|.
cudaError_t launch_intra_residual(IntraJobs &jobs, int e_in, bool add_e, cudaStream_t st);
// Red-black SOR sweeps of (-L_UU) e = res, from e = 0 (first) or e[e_in].
// Returns the index of the e buffer holding the result.
cudaError_t launch_intra_sor(IntraJobs &jobs, int e_in, bool from_zero, int sweeps, cudaStream_t st, int *e_out,
                             int *launches);
int intra_sweeps_per_launch();
cudaError_t intra_init();  // once per device
int set_sor_variant(int v);  // -1: autotune; 0..2 pin a variant (0 on success)

}  // namespace hivc
