// Side information by rectangular subdivision (Sec. 2.3): the backward flow
// as regions of a subdivision, each with its value, and the mask points of
// the residual blocks as the centres of the leaves of one subdivision per
// block.  Bit format (the paper's reference gives none): a node is a
// rectangle; a split halves its longer side (w >= h: the x side), the first
// part ceil(len/2) long; one bit per node in breadth-first order, 1 =
// split, a one-pixel node carries 0; bits LSB-first in 32-bit words;
// leaves are numbered in breadth-first order; a mask point is the leaf's
// centre pixel (x0 + (w-1)/2, y0 + (h-1)/2).
#include <climits>

#include "hivc_internal.cuh"

namespace hivc {
namespace {

constexpr int kTreeThreads = 1024;
constexpr int kFillChunk = 1024;  // pixels per unit of the fill's work list

__device__ __forceinline__ int tree_bit(const uint32_t *bits, long long i)
{
    return (int)((__ldg(bits + (i >> 5)) >> (i & 31)) & 1u);
}

__device__ __forceinline__ void split_rect(int4 r, int4 &a, int4 &b)
{
    if (r.z >= r.w) {
        const int w1 = r.z - r.z / 2;
        a = make_int4(r.x, r.y, w1, r.w);
        b = make_int4(r.x + w1, r.y, r.z / 2, r.w);
    } else {
        const int h1 = r.w - r.w / 2;
        a = make_int4(r.x, r.y, r.z, h1);
        b = make_int4(r.x, r.y + h1, r.z, r.w / 2);
    }
}

// exclusive block-wide scan of v (kTreeThreads threads); returns the prefix,
// *total the sum
__device__ int block_scan(int v, int *sh, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < kTreeThreads / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[32 + lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const int before = (warp > 0 ? sh[32 + warp - 1] : 0) + x - v;
    *total = sh[32 + kTreeThreads / 32 - 1];
    __syncthreads();
    return before;
}

// Breadth-first decode of the plane's tree by one CTA, level by level: the
// split flags of a level, scanned, place the children in the next level;
// leaves get their breadth-first numbers.  ws: two level arrays and the
// leaf array (cap entries each), then [used bits, leaves, error].
__global__ void __launch_bounds__(kTreeThreads) tree_decode_kernel(int W, int H, const uint32_t *bits,
                                                                    long long nbits, int cap, int4 *lev0, int4 *lev1,
                                                                    int4 *leaves, int *chunk_base, int *counters)
{
    __shared__ int sh[64];
    int4 *cur = lev0, *nxt = lev1;
    if (threadIdx.x == 0) cur[0] = make_int4(0, 0, W, H);
    __syncthreads();
    int n = 1, nleaf = 0, bad = 0;
    long long off = 0;
    while (n > 0 && !bad) {
        if (off + n > nbits) {
            bad = 1;
            break;
        }
        int nnext = 0;
        for (int base = 0; base < n; base += kTreeThreads) {
            const int i = base + threadIdx.x;
            int split = 0, leaf = 0, err = 0;
            int4 r = make_int4(0, 0, 0, 0);
            if (i < n) {
                r = cur[i];
                split = tree_bit(bits, off + i);
                if (split && r.z * r.w < 2) err = 1;
                leaf = !split;
            }
            int ts, tl;
            const int ps = block_scan(split, sh, &ts);
            const int pl = block_scan(leaf, sh, &tl);
            if (__syncthreads_or(err) || nnext + 2 * ts > cap || nleaf + tl > cap) {
                bad = 1;
                break;
            }
            if (i < n) {
                if (split) {
                    int4 a, b;
                    split_rect(r, a, b);
                    nxt[nnext + 2 * ps] = a;
                    nxt[nnext + 2 * ps + 1] = b;
                } else {
                    leaves[nleaf + pl] = r;
                }
            }
            nnext += 2 * ts;
            nleaf += tl;
        }
        __syncthreads();
        off += n;
        n = nnext;
        int4 *t = cur;
        cur = nxt;
        nxt = t;
    }
    // the fill's work list: leaf l covers chunks [chunk_base[l], chunk_base[l + 1])
    // of kFillChunk pixels each
    int carry = 0;
    for (int base = 0; !bad && base < nleaf; base += kTreeThreads) {
        const int l = base + threadIdx.x;
        int c = 0;
        if (l < nleaf) {
            const int4 r = leaves[l];
            c = (r.z * r.w + kFillChunk - 1) / kFillChunk;
        }
        int total;
        const int before = block_scan(c, sh, &total);
        if (l < nleaf) chunk_base[l] = carry + before;
        carry += total;
    }
    if (threadIdx.x == 0) {
        counters[0] = (int)min(off, (long long)INT_MAX);
        counters[1] = nleaf;
        counters[2] = bad;
        counters[3] = carry;
        if (!bad) chunk_base[nleaf] = carry;
    }
}

// Leaves to the dense flow: the work list of kFillChunk-pixel chunks of the
// leaves (so that large regions spread over many CTAs); CTA c takes chunks
// c, c + G, ..., finds its leaf by binary search over chunk_base.  A tree
// that did not use exactly its bits, or whose leaf count differs from the
// values', fills nothing and raises kFlagTree.
__global__ void __launch_bounds__(256) tree_fill_kernel(int W, const int4 *leaves, const int *chunk_base,
                                                        const int *counters, long long nbits, int n_values,
                                                        const float2 *values, float2 *flow, uint32_t *flags)
{
    const int nleaf = counters[1];
    const bool ok = counters[2] == 0 && (long long)counters[0] == nbits && nleaf == n_values;
    if (!ok) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && flags) atomicOr(flags, kFlagTree);
        return;
    }
    const int nchunks = counters[3];
    for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
        int lo = 0, hi = nleaf - 1;  // the last leaf with chunk_base <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (chunk_base[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const int4 r = leaves[lo];
        const float2 v = __ldg(values + lo);
        const int area = r.z * r.w;
        const int k0 = (c - chunk_base[lo]) * kFillChunk, k1 = min(area, k0 + kFillChunk);
        for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
            const int y = r.y + k / r.z, x = r.x + k % r.z;
            flow[(size_t)y * W + x] = v;
        }
    }
}

// ---- residual mask points -------------------------------------------------
// One thread per block decodes the block's tree (breadth-first, a queue of
// packed rectangles in local memory: at most 2 w h - 1 <= 511 nodes).
// Pass 0 counts the leaves into block_ptr[b + 1]; pass 1 writes the sorted
// leaf centres at block_ptr[b].
constexpr int kMaxTreeNodes = 511;

__device__ __forceinline__ uint32_t pack_rect(int x, int y, int w, int h)
{
    return (uint32_t)x | ((uint32_t)y << 5) | ((uint32_t)(w - 1) << 10) | ((uint32_t)(h - 1) << 15);
}

template <int PASS>
__global__ void __launch_bounds__(32) masks_kernel(int W, int H, int B, int nbx, int nblocks, const uint32_t *bits,
                                                    const uint32_t *tree_ptr, uint32_t *block_ptr, uint8_t *pos,
                                                    long long max_points, uint32_t *flags)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblocks) return;
    const int bx = b % nbx, by = b / nbx;
    const int w = min(B, W - bx * B), h = min(B, H - by * B);
    const long long b0 = __ldg(tree_ptr + b), b1 = __ldg(tree_ptr + b + 1);
    uint32_t q[kMaxTreeNodes];
    int head = 0, tail = 1, nl = 0;
    // a valid tree has at most kMaxTreeNodes bits: its words are read up
    // front (independent loads), then the decode runs from registers
    bool bad = b1 < b0 || b1 - b0 > kMaxTreeNodes;
    constexpr int kWords = (kMaxTreeNodes + 31) / 32 + 1;
    uint32_t wd[kWords];
    const long long w0 = b0 >> 5;
#pragma unroll
    for (int k = 0; k < kWords; ++k) wd[k] = (!bad && w0 + k <= ((b1 - 1) >> 5)) ? __ldg(bits + w0 + k) : 0u;
    long long i = b0;
    uint32_t start = 0, cnt = 0;
    if (PASS == 1) {
        // blocks that failed the count (count 0; a valid tree has a leaf)
        // and every block when the points do not fit write nothing
        start = block_ptr[b];
        cnt = block_ptr[b + 1] - start;
        if (cnt == 0 || (long long)block_ptr[nblocks] > max_points) return;
    }
    q[0] = pack_rect(0, 0, w, h);
    uint8_t *out = pos + start;
    while (!bad && head < tail) {
        const uint32_t pr = q[head++];
        const int x0 = pr & 31, y0 = (pr >> 5) & 31, rw = ((pr >> 10) & 31) + 1, rh = ((pr >> 15) & 31) + 1;
        if (i >= b1) {
            bad = true;
            break;
        }
        const long long li = i++ - (w0 << 5);
        if ((wd[li >> 5] >> (li & 31)) & 1u) {
            if (rw * rh < 2 || tail + 2 > kMaxTreeNodes) {
                bad = true;
                break;
            }
            int4 a, c;
            split_rect(make_int4(x0, y0, rw, rh), a, c);
            q[tail++] = pack_rect(a.x, a.y, a.z, a.w);
            q[tail++] = pack_rect(c.x, c.y, c.z, c.w);
        } else {
            if (PASS == 1 && (uint32_t)nl < cnt) {
                // insertion into the sorted run of this block's points
                const uint8_t p = (uint8_t)((y0 + (rh - 1) / 2) * w + x0 + (rw - 1) / 2);
                int k = nl;
                while (k > 0 && out[k - 1] > p) {
                    out[k] = out[k - 1];
                    --k;
                }
                out[k] = p;
            }
            ++nl;
        }
    }
    bad = bad || i != b1;
    if (PASS == 0) {
        block_ptr[b + 1] = bad ? 0u : (uint32_t)nl;
        if (bad && flags) atomicOr(flags, kFlagTree);
    }
}

// block_ptr[1..n] holds counts: in-place inclusive scan by one CTA
__global__ void __launch_bounds__(kTreeThreads) scan_counts_kernel(uint32_t *block_ptr, int n)
{
    __shared__ int sh[64];
    uint32_t carry = 0;
    if (threadIdx.x == 0) block_ptr[0] = 0;
    for (int base = 0; base < n; base += kTreeThreads) {
        const int i = base + threadIdx.x;
        const int v = i < n ? (int)block_ptr[i + 1] : 0;
        int total;
        const int before = block_scan(v, sh, &total);
        if (i < n) block_ptr[i + 1] = carry + (uint32_t)(before + v);
        carry += (uint32_t)total;
        __syncthreads();
    }
}

// ---- intra mask points --------------------------------------------------
// The leaf centres of the plane's tree marked in a byte map, then written
// in raster order: the map in chunks of kMarkChunk pixels, counted per
// chunk, the counts scanned, each chunk's points placed by a block scan.
constexpr int kMarkChunk = 4 * kTreeThreads;

__global__ void __launch_bounds__(256) mark_centres_kernel(int W, const int4 *leaves, const int *counters,
                                                           long long nbits, uint8_t *map)
{
    const int nleaf = counters[1];
    if (counters[2] != 0 || (long long)counters[0] != nbits) return;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nleaf; l += gridDim.x * blockDim.x) {
        const int4 r = leaves[l];
        map[(size_t)(r.y + (r.w - 1) / 2) * W + r.x + (r.z - 1) / 2] = 1;
    }
}

// PASS 0: points per chunk into cnt[c + 1]; PASS 1: the chunk's points at
// offset cnt[c] (after the scan), in raster order
template <int PASS>
__global__ void __launch_bounds__(kTreeThreads) compact_kernel(const uint8_t *map, long long npix, uint32_t *cnt,
                                                               uint32_t *idx, long long max_points)
{
    __shared__ int sh[64];
    const long long c0 = (long long)blockIdx.x * kMarkChunk;
    int v = 0;
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long i = c0 + 4LL * threadIdx.x + k;
        const int b = i < npix ? map[i] : 0;
        m |= (uint32_t)b << k;
        v += b;
    }
    int total;
    const int before = block_scan(v, sh, &total);
    if (PASS == 0) {
        if (threadIdx.x == 0) cnt[blockIdx.x + 1] = (uint32_t)total;
        return;
    }
    if ((long long)cnt[gridDim.x] > max_points) return;
    uint32_t o = cnt[blockIdx.x] + (uint32_t)before;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if ((m >> k) & 1u) idx[o++] = (uint32_t)(c0 + 4LL * threadIdx.x + k);
}

// the count (or 0 and kFlagTree for a bad tree or too many points)
__global__ void intra_count_kernel(const int *counters, long long nbits, const uint32_t *cnt, int nchunks,
                                   long long max_points, int32_t *n_out, uint32_t *flags)
{
    const bool ok = counters[2] == 0 && (long long)counters[0] == nbits && (long long)cnt[nchunks] <= max_points;
    *n_out = ok ? (int32_t)cnt[nchunks] : 0;
    if (!ok && flags) atomicOr(flags, kFlagTree);
}

}  // namespace

size_t intra_tree_workspace_bytes(long long nbits, int W, int H)
{
    const size_t npix = (size_t)W * H;
    const size_t nchunks = (npix + kMarkChunk - 1) / kMarkChunk;
    return tree_workspace_bytes(nbits) + ((npix + 255) / 256) * 256 + (nchunks + 1) * sizeof(uint32_t) + 256;
}

cudaError_t launch_intra_mask_from_tree(int W, int H, const uint32_t *bits, long long nbits, uint32_t *idx,
                                        long long max_points, int32_t *n_out, void *ws, uint32_t *flags, int sms,
                                        cudaStream_t st)
{
    const int cap = (int)(nbits < 1 ? 1 : nbits);
    int4 *lev0 = static_cast<int4 *>(ws), *lev1 = lev0 + cap, *leaves = lev1 + cap;
    int *counters = reinterpret_cast<int *>(leaves + cap);
    int *chunk_base = counters + 16;
    uint8_t *map = static_cast<uint8_t *>(ws) + tree_workspace_bytes(nbits);
    const size_t npix = (size_t)W * H;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(map + ((npix + 255) / 256) * 256);
    const int nchunks = (int)((npix + kMarkChunk - 1) / kMarkChunk);
    cudaError_t e = cudaMemsetAsync(map, 0, npix, st);
    if (e != cudaSuccess) return e;
    tree_decode_kernel<<<1, kTreeThreads, 0, st>>>(W, H, bits, nbits, cap, lev0, lev1, leaves, chunk_base, counters);
    mark_centres_kernel<<<2 * sms, 256, 0, st>>>(W, leaves, counters, nbits, map);
    compact_kernel<0><<<nchunks, kTreeThreads, 0, st>>>(map, (long long)npix, cnt, idx, max_points);
    scan_counts_kernel<<<1, kTreeThreads, 0, st>>>(cnt, nchunks);
    compact_kernel<1><<<nchunks, kTreeThreads, 0, st>>>(map, (long long)npix, cnt, idx, max_points);
    intra_count_kernel<<<1, 1, 0, st>>>(counters, nbits, cnt, nchunks, max_points, n_out, flags);
    return cudaGetLastError();
}

size_t tree_workspace_bytes(long long nbits)
{
    const size_t cap = (size_t)(nbits < 1 ? 1 : nbits);
    return 3 * cap * sizeof(int4) + (cap + 1) * sizeof(int) + 64;
}

cudaError_t launch_flow_from_tree(int W, int H, const uint32_t *bits, long long nbits, const float *values,
                                  int n_values, float *flow, void *ws, uint32_t *flags, int sms, cudaStream_t st)
{
    const int cap = (int)(nbits < 1 ? 1 : nbits);
    int4 *lev0 = static_cast<int4 *>(ws), *lev1 = lev0 + cap, *leaves = lev1 + cap;
    int *counters = reinterpret_cast<int *>(leaves + cap);  // 16 ints
    int *chunk_base = counters + 16;                         // cap + 1 ints
    tree_decode_kernel<<<1, kTreeThreads, 0, st>>>(W, H, bits, nbits, cap, lev0, lev1, leaves, chunk_base, counters);
    tree_fill_kernel<<<8 * sms, 256, 0, st>>>(W, leaves, chunk_base, counters, nbits, n_values,
                                             reinterpret_cast<const float2 *>(values), reinterpret_cast<float2 *>(flow),
                                             flags);
    return cudaGetLastError();
}

cudaError_t launch_masks_from_trees(int W, int H, int B, const uint32_t *bits, const uint32_t *tree_ptr,
                                    uint32_t *block_ptr, uint8_t *pos, long long max_points, uint32_t *flags,
                                    cudaStream_t st)
{
    const int nbx = (W + B - 1) / B, nb = nbx * ((H + B - 1) / B);
    const int grid = (nb + 31) / 32;
    masks_kernel<0><<<grid, 32, 0, st>>>(W, H, B, nbx, nb, bits, tree_ptr, block_ptr, pos, max_points, flags);
    scan_counts_kernel<<<1, kTreeThreads, 0, st>>>(block_ptr, nb);
    masks_kernel<1><<<grid, 32, 0, st>>>(W, H, B, nbx, nb, bits, tree_ptr, block_ptr, pos, max_points, flags);
    return cudaGetLastError();
}

}  // namespace hivc
