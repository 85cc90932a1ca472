/*
 * hivc.h -- C ABI of the GB300 decoder for the inpainting-based video codec
 * of Andris, Peter, Kaja Mohideen, Weickert and Hoffmann, "Inpainting-based
 * Video Compression in FullHD".
 *
 * The decoder rebuilds each frame as prediction + correction (Sec. 2):
 *   - intra frames: homogeneous diffusion inpainting of the frame from its
 *     mask pixels (Sec. 2.1, Eq. 1, A = -L, reflecting boundaries);
 *   - inter frames: backward warping of the previous reconstruction along a
 *     dense backward optic flow field (Sec. 2, Sec. 2.3);
 *   - both: a residual rebuilt per block by pseudodifferential inpainting
 *     with the harmonic operator (Sec. 2.2, Eqs. 2-4), added and clamped.
 *
 * Conventions (all entry points):
 *   - Planes are row-major; luma is width x height, 4:2:0 chroma planes are
 *     ceil(width/2) x ceil(height/2), 4:4:4 planes width x height.  Grey
 *     values are in [0, 255] (RCT chroma in [-255, 255]).
 *   - Every array pointer in the input/output structs is DEVICE memory owned
 *     by the caller.  It must stay valid and unmodified until the work is
 *     complete (hivc_decoder_sync, or the caller's stream for the step
 *     entry points).  Struct arguments themselves are read on the host
 *     during the call and may be reused right after it returns.
 *   - Calls are asynchronous on the decoder's (or the given) stream.  Host
 *     checks (sizes, null pointers, decoder state) return an error at once;
 *     data checks that need the device arrays (index order, block point
 *     counts, positions) run inside the kernels, never trap, and surface as
 *     HIVC_E_INVALID from hivc_decoder_sync.  Offending blocks or mask
 *     points are ignored by the kernels and never accessed out of bounds.
 *   - A decoder is not thread-safe; distinct decoders are independent.
 */
#ifndef HIVC_H
#define HIVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HIVC_OK = 0,
    HIVC_E_INVALID = -1,       /* bad argument or bad input data */
    HIVC_E_NOMEM = -2,         /* device allocation failed */
    HIVC_E_CUDA = -3,          /* a CUDA runtime call failed */
    HIVC_E_NOT_CONVERGED = -4, /* intra solve hit max_cycles above iframe_tol */
    HIVC_E_NO_REFERENCE = -5,  /* inter frame before any intra frame */
    HIVC_E_BUDGET = -6,        /* footprint above the caller's budget */
    HIVC_E_TIMEOUT = -7        /* reserved: no entry point returns it (no
                                  kernel of the library waits on another) */
} hivc_status;

/* Decoder configuration.  hivc_config_default() fills the defaults. */
typedef struct {
    int32_t width, height;  /* luma plane size, >= 1 */
    int32_t chroma;         /* 0 = grey (Y only), 1 = YCbCr 4:2:0,
                               2 = the paper's colour path (Sec. 2.3): 4:4:4
                               planes Y, U = B - G, V = R - G of the
                               reversible colour transform of JPEG2000 (U, V
                               in [-255, 255], moved by the luma flow); the
                               output planes are R, G, B =
                               the inverse RCT of the rounded planes */
    int32_t block;          /* residual block edge B, 1..16.  The paper uses
                               8 x 8 blocks (Sec. 2.2, 2.3); default 16 */
    int32_t op;             /* residual operator (Sec. 2.2: defined by the
                               eigenvalues of its Green's functions):
                               0 = harmonic, A = -L (Sec. 2.3; default),
                               1 = biharmonic, A = L^2 (eigenvalues mu^2) */
    int32_t precision;      /* intra solve: 0 = FP32 sweeps with a residual
                               correction of an extended-precision iterate
                               (float-float, ~48-bit; default), 1 = FP32 only */
    double iframe_tol;      /* stop when max |(L u)_i| over unknown pixels
                               <= tol, grey levels (Eq. 1 residual); default
                               1e-8; FP32-only mode floors near 1e-3 */
    int32_t max_cycles;     /* cap on outer correction cycles, 1..1000
                               (default 40); beyond it sync returns
                               HIVC_E_NOT_CONVERGED */
    double cond_threshold;  /* >= 0 (default 1e6).  Every residual block's
                               condition bound kappa = 8 tr(G_PP) / (1 - K/N)
                               >= cond_2(G_PP) (Sec. 2.2: the eigenvalues of
                               A = -L are at most 8) is compared with it; a
                               block above it is re-solved in FP64 from an
                               FP64 Green's table (K <= 179; larger K keep
                               FP32 and set device flag bit 6).  No block
                               shape reaches 4e5, so the default never
                               triggers; 0 re-solves every block */
    void *stream;           /* cudaStream_t to run on; NULL = the decoder
                               creates its own non-blocking stream */
    int32_t layout_groups;  /* 1: residual blocks of a plane that share one
                               mask layout (the same points, at least 16
                               blocks, K <= 32, values within [-256, 256])
                               are grouped: one factorisation per layout,
                               and their residual planes (Eq. 3 for a fixed
                               layout is linear in the values) as one
                               tensor-core product; 0 (default) = every
                               block on its own (the grouping pass costs
                               more than it saves unless many blocks share
                               few layouts) */
    int32_t batch_frames;   /* 0..4096 (default 0): the batch pool (the
                               coefficients and residual planes of the inter
                               frames of one hivc_decode_batch call) is made
                               at creation for this many frames at their
                               largest, so batches that fit never grow it; a
                               larger batch grows it stream-ordered (no host
                               wait).  Counted by hivc_decoder_bytes */
    int32_t fused_residual; /* 1: an inter frame with 16 x 16 blocks, 4:2:0
                               or grey planes of even size and no layout
                               groups is decoded by one fused kernel that
                               evaluates Eq. 3 block by block in shared
                               memory, then warps, adds and packs the
                               block's pixels: no residual planes in memory
                               (a smaller batch pool), but slower than the
                               default on a GB300, where the evaluation of
                               many frames in one launch overlaps the intra
                               frame; 0 (default): residual planes
                               (evaluation kernel, then the pixel kernel).
                               Both give the same bits */
    int32_t flat_start;     /* 0 (default): the intra solve starts from a
                               coarse solution (planes of at least 32 x 32):
                               the mask restricted to 2 x 2 cells, one
                               correction cycle on that half-size problem,
                               then bilinear prolongation to the unknown
                               pixels; 1: from the mean of the mask values.
                               Only the start differs: both stop at the same
                               tolerance of Eq. 1 */
} hivc_config;

/* Intra mask of one plane: n >= 1 sorted, unique linear indices y*w + x. */
typedef struct {
    int32_t n;
    const uint32_t *idx; /* device, n entries, strictly increasing, < w*h */
    const uint8_t *val;  /* device, n entries: the grey value at idx */
} hivc_points;

/*
 * Block residual data of one plane (Sec. 2.2, 2.3).  Blocks of edge B tile
 * the plane in raster order (bx fastest); edge blocks are cropped to the
 * plane and are independent images of their own size w x h.  Block b owns
 * entries block_ptr[b] .. block_ptr[b+1]-1 of pos/val:
 *   pos = ly*w + lx inside the block (strictly increasing, < w*h), and
 *   K_b = block_ptr[b+1] - block_ptr[b] <= w*h - 1;
 *   val = the residual value at that point.
 * K_b = 0 reconstructs as zero.  block_ptr has ceil(W/B)*ceil(H/B) + 1
 * entries with block_ptr[0] = 0 and block_ptr[last] <= n_points.
 */
typedef struct {
    const uint32_t *block_ptr; /* device */
    const uint8_t *pos;        /* device */
    const int16_t *val;        /* device */
    int32_t n_points;          /* entries in pos/val */
} hivc_residual;

/*
 * Block residual of one plane in coefficient mode (Sec. 2.2, 2.3): the
 * decoder receives, per point, the Green's coefficient c_j dead-zone
 * quantised to an index q in [-127, 127], and per block the constant a, and
 * only evaluates r = a + sum_j c_j G(., p_j) (Eq. 3; no solve, no overwrite
 * at the points).  Dequantisation (the paper leaves the mapping's scale
 * open): c = 0 for q = 0, c = sign(q) (|q| + offset) step otherwise.
 * block_ptr/pos as in hivc_residual (K_b <= w*h - 1); K_b = 0 gives r = a.
 * An index -128 makes its block zero and is reported as HIVC_E_INVALID.
 */
typedef struct {
    const uint32_t *block_ptr; /* device */
    const uint8_t *pos;        /* device */
    const int8_t *q;           /* device, per point */
    const float *a;            /* device, per block */
    int32_t n_points;
    float step;                /* quantiser step, > 0 */
    float offset;              /* reconstruction offset, in [0, 1) */
} hivc_coef_residual;

/* Intra frame.  The two chroma planes share one mask (Sec. 2.3). */
typedef struct {
    hivc_points y;
    int32_t c_n;              /* chroma mask size (4:2:0 only) */
    const uint32_t *c_idx;    /* device, shared by Cb and Cr */
    const uint8_t *cb_val;    /* device */
    const uint8_t *cr_val;    /* device */
    const hivc_residual *res; /* NULL, or a HOST array of 1 (grey) / 3
                                 residuals added to the inpainted planes */
    const int16_t *cu_val;    /* device, chroma 2: the U values (cb_val unused) */
    const int16_t *cv_val;    /* device, chroma 2: the V values (cr_val unused) */
} hivc_iframe;

/* Inter frame: pred(x) = ref(x + flow(x)), bilinear, sample clamped.
   Chroma uses half the mean of the 2 x 2 co-sited luma vectors. */
typedef struct {
    const float *flow;    /* device, height x width x 2 floats (dx, dy) */
    hivc_residual res[3]; /* Y, Cb, Cr (only res[0] when grey).  Cb and Cr
                             may share block_ptr/pos: one factorisation
                             then serves both */
} hivc_pframe;

/* Inter frame with its residual in coefficient mode. */
typedef struct {
    const float *flow;           /* device, height x width x 2 floats */
    hivc_coef_residual res[3];   /* Y, Cb, Cr (only res[0] when grey) */
} hivc_pframe_coef;

/* uint8 output planes (device), rows pitch bytes apart. */
typedef struct {
    uint8_t *plane[3];
    int32_t pitch[3];
} hivc_out;

typedef struct {
    int32_t type; /* 0 = intra (i), 1 = inter (p) */
    const hivc_iframe *i;
    const hivc_pframe *p;
} hivc_frame;

#define HIVC_STAT_KERNELS 8
/* Statistics of the frames completed by the last hivc_decoder_sync. */
typedef struct {
    double resid[3];        /* final Eq. 1 residual per plane (last intra) */
    int32_t cycles;         /* outer correction cycles of the last intra */
    int32_t sweeps;         /* red-black sweeps of the last intra */
    int32_t fp64_blocks;    /* residual blocks re-solved in FP64 */
    int32_t large_blocks;   /* residual blocks with K > 32 (solved by a CTA) */
    float max_cond;         /* largest residual-block condition bound kappa */
    uint32_t device_flags;  /* data errors seen by the kernels (bit set;
                               bit 6 is information, not an error) */
    int32_t frames;         /* frames since the previous sync */
    int32_t launches;       /* kernel launches since the previous sync */
    /* per kernel family: accumulated device time (ms, CUDA events, only
       when timing is on) and launch counts since the previous sync:
       0 intra setup, 1 intra sweeps, 2 intra residual, 3 block coefficients,
       4 inter pixels (warp + residual + pack), 5 block evaluate,
       6 intra output and the 4:4:4 colour path's pixels, 7 the sweeps of
       the intra solve's coarse start (its residual launches count in 2) */
    float kernel_ms[HIVC_STAT_KERNELS];
    int32_t kernel_launches[HIVC_STAT_KERNELS];
    /* per kernel family: pixels processed since the previous sync, the sum
       over launches of the pixels of the planes each launch covers.  Set
       for families 1, 2 and 7, whose launches may cover only the planes
       that still need sweeps; 0 for the others. */
    int64_t kernel_pixels[HIVC_STAT_KERNELS];
    int32_t group_blocks;   /* residual blocks evaluated by their layout
                               group's tensor-core product (Cb/Cr pairs
                               count twice) */
    int32_t layout_groups;  /* layout groups formed */
} hivc_stats;

typedef struct hivc_decoder hivc_decoder;

/* Fill *cfg with the defaults (width/height 0: the caller sets them). */
void hivc_config_default(hivc_config *cfg);

/* Create a decoder: allocates its reference planes and scratch on the
   current CUDA device.  HIVC_E_INVALID for a bad config, HIVC_E_NOMEM. */
hivc_status hivc_decoder_create(const hivc_config *cfg, hivc_decoder **out);

/* Device bytes a decoder with this config allocates (for HBM-budget
   admission); 0 for an invalid config. */
size_t hivc_decoder_bytes(const hivc_config *cfg);

/* Decode an intra frame (Sec. 2.1 + optional residual, Sec. 2.2) into out
   and make it the reference.  Asynchronous: the correction loop decides
   its cycles on the device (a graph with conditional loops; the residual
   launches plan the sweeps), so the host does not wait.  Whether the solve
   reached iframe_tol within max_cycles is reported by hivc_decoder_sync
   (HIVC_E_NOT_CONVERGED; the residual reached in hivc_stats.resid).  The
   first solve of a plane geometry in a process may time the sweep kernel's
   tilings first (see hivc_tune_lookup), which waits on the stream once. */
hivc_status hivc_decode_iframe(hivc_decoder *dec, const hivc_iframe *f, const hivc_out *out);

/* Decode an inter frame (Sec. 2, 2.3: warp + residual) into out and make it
   the reference.  Asynchronous.  HIVC_E_NO_REFERENCE before any intra. */
hivc_status hivc_decode_pframe(hivc_decoder *dec, const hivc_pframe *f, const hivc_out *out);

/* Decode an inter frame whose residual comes in coefficient mode: one
   evaluation launch for the three planes, then warp + residual + pack.
   Asynchronous.  HIVC_E_NO_REFERENCE before any intra frame. */
hivc_status hivc_decode_pframe_coef(hivc_decoder *dec, const hivc_pframe_coef *f, const hivc_out *out);

/* Decode n frames, frame k on decoder decs[k] into outs[k].  Frames of one
   decoder are decoded in array order; each run of consecutive inter frames
   of a decoder shares its block launches (Eq. 2 coefficients, Eq. 3
   residual planes).  Every inter frame is checked before anything is
   launched (HIVC_E_INVALID; HIVC_E_NO_REFERENCE for an inter frame of a
   decoder with no reference and no earlier intra frame in the batch).
   Every call only enqueues work, so the decoders' frames overlap on the
   GPU; a decoder stops at its first error, the others finish, and the call
   returns the first error in order
   of the decoders' first frames.  Intra solves that stop above the
   tolerance are reported by hivc_decoder_sync.
   The block launches of an inter run that follows an intra frame run on a
   stream the decoder owns, beside the intra frame; the decoder's stream
   waits for them (an event) before the run's first warp, so work queued on
   the decoder's stream after the call is ordered after all of it. */
hivc_status hivc_decode_batch(hivc_decoder *const *decs, const hivc_frame *frames, int32_t n,
                              const hivc_out *outs);

/* Wait for the decoder's stream; report device-side data errors
   (HIVC_E_INVALID), else HIVC_E_NOT_CONVERGED if an intra solve since the
   last sync stopped above iframe_tol, and the statistics of the frames
   since the last sync. */
hivc_status hivc_decoder_sync(hivc_decoder *dec, hivc_stats *last);

/* Forget the reference frame (the decoder is reused for a new stream: its
   next frame must be an intra frame).  Work already queued is unaffected. */
hivc_status hivc_decoder_reset(hivc_decoder *dec);

/* The intra solve's red-black sweep kernel comes in variants that perform
   the same sweeps bit for bit (0: 128-column regions, a cell pair per
   thread; 1: 112-column regions; 2: 128-column regions, four cells per
   thread).  By default (-1) the first solve of each plane geometry times
   them on its own sweeps and keeps the fastest; 0..2 pin one for every
   decoder of the process.  HIVC_E_INVALID for other values. */
hivc_status hivc_set_sor_variant(int32_t variant);

/* The autotuner's table.  The library times schedule choices that never
   change a result (the sweep kernel's region tiling; CTAs per SM of the
   persistent coefficient kernel) on the first call that needs one, and
   keeps each choice under a key of the GPU's name and the shape, e.g.
   "NVIDIA GB300|sor|1920x1080,960x540,960x540" or
   "NVIDIA GB300|coef|16384" (block count rounded up to a power of two),
   for the process and in a JSON file: HIVC_TUNE_CACHE, else
   $XDG_CACHE_HOME/hivc/tune.json, else $HOME/.cache/hivc/tune.json.
   hivc_tune_lookup returns the value under key, or -1; hivc_tune_record
   sets one (value >= 0) and rewrites the file, so that a caller can
   pre-seed or pin choices.  Neither needs a GPU. */
int32_t hivc_tune_lookup(const char *key);
hivc_status hivc_tune_record(const char *key, int32_t value);

/* Enable (1) or disable (0) per-kernel CUDA-event timing in hivc_stats. */
hivc_status hivc_decoder_set_timing(hivc_decoder *dec, int32_t on);

/* Device pointer to the current FP32 reference plane (the unrounded,
   clamped reconstruction of the last frame) with its size and pitch in
   floats.  Valid until the next decode call. */
hivc_status hivc_decoder_reference(const hivc_decoder *dec, int32_t plane, const float **ptr,
                                   int32_t *width, int32_t *height, int32_t *pitch);

/* Device pointers to the iterate of the last intra frame's diffusion solve
   (Sec. 2.1, Eq. 1) of one plane: the float-float pair u = hi + lo (lo is
   NULL with precision = 1), FP32 planes of the given size and pitch in
   floats, before the optional residual and the clamp to [0, 255].  The
   solve's reported residual (hivc_stats.resid) is max |(L u)_i| over the
   unknown pixels of this u, which a caller can recompute in FP64 from
   hi + lo.  Call after hivc_decoder_sync (which learns which buffer of the
   solve's ping-pong holds the result); valid until the next intra frame;
   HIVC_E_NO_REFERENCE before any intra frame. */
hivc_status hivc_decoder_intra_solution(const hivc_decoder *dec, int32_t plane, const float **hi,
                                        const float **lo, int32_t *width, int32_t *height, int32_t *pitch);

/* The stream the decoder runs on. */
void *hivc_decoder_stream(const hivc_decoder *dec);

void hivc_decoder_destroy(hivc_decoder *dec);

const char *hivc_status_str(hivc_status s);

/* ------------------------------------------------------------------------
 * Step entry points (stateless; device pointers; asynchronous on stream).
 * ---------------------------------------------------------------------- */

/* Scratch bytes hivc_block_residual needs for a plane with n_points
   residual points. */
size_t hivc_block_residual_workspace_bytes(int32_t width, int32_t height, int32_t block,
                                           int32_t n_points);

/* Residual plane r (width x height floats, row pitch r_pitch floats) from
   block data (Sec. 2.2, Eqs. 2-4): per block, the (K+1) x (K+1) system in
   the Green's function at the block's points is solved (coefficients c
   summing to zero and the constant a), then r = sum_j c_j g_j + a (Eq. 3)
   is summed over the block from the rows of its precomputed Green's
   matrix (built once per block shape from the DCT-II diagonalisation of
   Eq. 4); r equals the data at the points.  workspace: device scratch of at least
   hivc_block_residual_workspace_bytes() bytes.  flags: optional device
   uint32 that receives error bits for bad blocks (those blocks are zero).
   HIVC_E_INVALID for bad sizes or a short workspace. */
hivc_status hivc_block_residual(int32_t width, int32_t height, int32_t block,
                                const hivc_residual *res, float *r, int32_t r_pitch,
                                void *workspace, size_t workspace_bytes, uint32_t *flags,
                                void *stream);

/* Residual plane of a coefficient-mode plane (see hivc_coef_residual) with
   operator op (0 harmonic, 1 biharmonic) into r (device, r_pitch floats per
   row), on stream (NULL = default).  Needs no workspace.  Data errors are
   ORed into *flags (device word; NULL: not reported).  Asynchronous. */
hivc_status hivc_block_residual_coef(int32_t width, int32_t height, int32_t block, int32_t op,
                                     const hivc_coef_residual *res, float *r, int32_t r_pitch, uint32_t *flags,
                                     void *stream);

/* hivc_block_residual without allocation: the same residual plane, with
   the coefficient scratch taken from a fixed array inside the library
   instead of a caller workspace.  The paper has no counterpart; this is
   for callers that cannot allocate device memory when they need the
   residual: a host under a fixed memory budget whose every allocation is
   made at start-up, or a latency-bound loop where a cudaMalloc or cudaFree
   (which may synchronise the whole device) would stall other streams.
   Limits: at most 131072 residual points and 16384 blocks per call, else
   HIVC_E_INVALID.  The array (about 17 MB: room for one block with more
   than 32 points per range of 128 blocks) exists once per device on which
   this function has run and stays until the process exits.  All calls on a
   device share it and each call overwrites it: calls whose work overlaps
   on the GPU (e.g. on two streams) race, so serialise them.  The first call
   on a device uploads the Green's tables and looks up the array's device
   address with that device current; make that first call before any
   stream capture.  flags: optional device uint32 for error bits, as in
   hivc_block_residual.  No cudaMalloc or cudaFree is called. */
hivc_status hivc_block_residual_static(int32_t width, int32_t height, int32_t block,
                                       const hivc_residual *res, float *r, int32_t r_pitch,
                                       uint32_t *flags, void *stream);

/* Backward bilinear warp of one plane (Sec. 2, 2.3): pred(x) = ref(x + v(x)),
   sample clamped to the plane.  flow is the LUMA flow (flow_width x
   flow_height x 2 floats); when chroma_flow is 1 the plane is a 4:2:0
   chroma plane of that luma size and v is half the mean of the co-sited
   2 x 2 luma vectors, else the plane has the flow's size and v = flow. */
hivc_status hivc_warp(int32_t width, int32_t height, const float *ref, int32_t ref_pitch,
                      const float *flow, int32_t flow_width, int32_t flow_height,
                      int32_t chroma_flow, float *pred, int32_t pred_pitch, void *stream);

/*
 * Side information by rectangular subdivision (Sec. 2.3: the backward flow
 * is coded as the regions of a rectangular subdivision, each with its
 * average value; the mask points of every residual block come from a
 * subdivision as well).  The paper gives no bit format; this one is:
 *   - a node is a rectangle; a split halves its longer side (w >= h: the x
 *     side), the first part ceil(len/2) long, the second floor(len/2);
 *   - one bit per node in breadth-first order, 1 = split; a one-pixel node
 *     must carry 0; bits are packed LSB-first in 32-bit words;
 *   - leaves are numbered in breadth-first order;
 *   - a mask point is the centre pixel (x0 + (w-1)/2, y0 + (h-1)/2) of its
 *     leaf.
 * All arrays are device memory; calls are asynchronous on stream (NULL =
 * default).  Bad trees are reported by ORing bit 8 into *flags (device
 * word; NULL: not reported) and leave their output unwritten.
 */

/* Device scratch hivc_flow_from_tree needs for a tree of nbits bits. */
size_t hivc_flow_from_tree_workspace_bytes(int64_t nbits);

/* Dense backward flow (height x width x 2 floats, the inter frames' flow
   layout) from the plane's tree (nbits bits, all of them used) and one
   (dx, dy) per leaf (n_values = the number of leaves). */
hivc_status hivc_flow_from_tree(int32_t width, int32_t height, const uint32_t *bits, int64_t nbits,
                                const float *values, int32_t n_values, float *flow, void *workspace,
                                size_t ws_bytes, uint32_t *flags, void *stream);

/* Device scratch hivc_intra_mask_from_tree needs. */
size_t hivc_intra_mask_from_tree_workspace_bytes(int32_t width, int32_t height, int64_t nbits);

/* Intra mask positions (Sec. 2.3: the intra mask comes from a rectangular
   subdivision of the plane): the leaf centres of the plane's tree as
   sorted linear indices y*width + x in idx (at most max_points; the mask
   values arrive in this order), their count in *n_points (device int32;
   0 for a bad tree or too many points, with bit 8 raised). */
hivc_status hivc_intra_mask_from_tree(int32_t width, int32_t height, const uint32_t *bits, int64_t nbits,
                                      uint32_t *idx, int64_t max_points, int32_t *n_points,
                                      void *workspace, size_t ws_bytes, uint32_t *flags, void *stream);

/* Residual mask points of a width x height plane's block x block blocks
   (raster order, edge blocks cropped) from one tree per block: block b's
   tree is bits [tree_ptr[b], tree_ptr[b+1]) (nblocks + 1 entries).
   Writes block_ptr (nblocks + 1) and pos (ly w + lx, increasing within a
   block) as hivc_residual takes them; at most max_points points (more:
   pos is not written and bit 8 is raised). */
hivc_status hivc_masks_from_trees(int32_t width, int32_t height, int32_t block, const uint32_t *bits,
                                  const uint32_t *tree_ptr, uint32_t *block_ptr, uint8_t *pos,
                                  int64_t max_points, uint32_t *flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HIVC_H */
