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

// Error bits the kernels OR into a device status word (never trap).
enum : uint32_t {
    kFlagBlockPtr = 1u << 0,  // block_ptr decreasing, [0] != 0 or beyond n_points
    kFlagK = 1u << 1,         // K_b > w*h - 1
    kFlagPos = 1u << 2,       // position outside the block or not increasing
    kFlagNotSPD = 1u << 3,    // non-positive Cholesky pivot
    kFlagMaskIdx = 1u << 4,   // intra mask index out of range or not increasing
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
};

struct BlockJobs {
    BlockPlane p[kMaxJobs];
    int32_t n;
    int32_t total_blocks;
};

// Scratch for the coefficient stage of one launch.
struct BlockScratch {
    uint32_t *large_list;   // global block ids with K > kWarpK
    uint32_t *large_count;  // number of entries (zeroed before the launch)
    int32_t large_cap;
    uint32_t *flags;        // device error word
};

// Uploads the DCT-II / Green's tables once per device.
cudaError_t ensure_block_tables();

// c, a for every block (warp per block; K > 32 deferred to the CTA kernel).
cudaError_t launch_block_coef(const BlockJobs &jobs, const BlockScratch &s, cudaStream_t st,
                              int *launches);
// r-field from c, a via the DCT route (warp per block), r = v at the points.
cudaError_t launch_block_eval(const BlockJobs &jobs, uint32_t *flags, cudaStream_t st);

// ---------------------------------------------------------------------------
// warp + add + pack (Sec. 2, 2.3)
// ---------------------------------------------------------------------------
struct WarpPlane {
    const float *ref;    // FP32 reference plane (inter), or nullptr
    const double *src64; // FP64 prediction (intra), used when ref == nullptr
    const float *r;      // residual field or nullptr
    float *ref_out;      // new FP32 reference (clamped), or nullptr
    uint8_t *out;        // uint8 output, or nullptr
    float *pred_out;     // raw prediction (step entry point), or nullptr
    const float *flow;   // luma flow (H x W x 2) for inter planes
    int32_t ref_pitch, src64_pitch, r_pitch, ref_out_pitch, out_pitch, pred_pitch;
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

// ---------------------------------------------------------------------------
// intra solve (Sec. 2.1)
// ---------------------------------------------------------------------------
struct IntraPlane {
    int32_t width, height, pitch;  // pitch in elements
    const uint32_t *idx;           // mask indices
    const uint8_t *val;            // mask values
    int32_t n;                     // mask size
    uint8_t *mask;                 // 1 = known pixel
    double *u[2];                  // FP64 solution, ping-pong
    float *res;                    // FP32 copy of the Eq. 1 residual
    float *e[2];                   // FP32 correction, ping-pong
    double *sum;                   // scratch: sum of mask values
    unsigned long long *rnorm;     // scratch: max |residual| as ordered bits
    float omega;                   // SOR relaxation factor
    int32_t tiles_x, tile_base;    // filled by the launchers
};

struct IntraJobs {
    IntraPlane p[3];
    int32_t n;
};

cudaError_t launch_intra_init(IntraJobs &jobs, uint32_t *flags, cudaStream_t st, int *launches);
// FP64: u_out = u_in + e (unless first), res = float(L u_out) at unknowns,
// rnorm = max |L u_out|.
cudaError_t launch_intra_residual(IntraJobs &jobs, int in, int e_in, bool add_e, cudaStream_t st);
// S red-black SOR sweeps of (-L_UU) e = res, from e = 0 (first) or e[e_in].
// Returns the index of the e buffer holding the result.
cudaError_t launch_intra_sor(IntraJobs &jobs, int e_in, bool from_zero, int sweeps, cudaStream_t st,
                             int *e_out, int *launches);

}  // namespace hivc
