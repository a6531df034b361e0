// gc_raster.cu - binning (emit), tile ranges and the forward blend for sm_103a.
//
// Binning works in depth-rank space: Gaussians are first sorted by depth
// (N keys), then every Gaussian emits one entry per touched tile in rank order,
// and a stable sort on the tile id alone (log2(tiles) bits, two 8-bit digits at
// 1080p and 4K) yields per-tile lists that are already front to back, with
// ties broken by the global index (the depth sort is stable over index order).
// An entry's position in emit order is offsets[r] + (its tile's index among the
// Gaussian's row intervals, binning step 15); the backward pass writes its partial
// gradients there, so each Gaussian's partials are contiguous.
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_tile.cuh"

namespace gc {

namespace {


// One warp emits the entries of 32 consecutive ranks (row by row, see emit_rows_warp).
__global__ void __launch_bounds__(256) k_emit(const float4 *__restrict__ ranked,
                                              const uint32_t *__restrict__ offsets,
                                              const uint32_t *__restrict__ touched_r, int64_t n,
                                              RenderParams rp, int W, int H, uint32_t cap,
                                              uint32_t *__restrict__ keys,
                                              uint32_t *__restrict__ vals, const uint32_t *total,
                                              uint32_t *peak) {
    // the largest key count of a forward that overflowed the capacity it ran with, since the
    // host last looked (so that an overflow in any frame of a multi-frame step shows, and a
    // count that fitted an earlier, larger capacity is not taken for one)
    if (peak && blockIdx.x == 0 && threadIdx.x == 0 && *total > cap) atomicMax(peak, *total);
    const int lane = threadIdx.x & 31;
    const int64_t wbase = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;
    if (wbase >= n) return;
    emit_rows_warp(ranked, wbase, n, offsets, touched_r, 0u, rp, W, H, cap, keys, vals);
}

// Range of every key of a key-sorted array: where a key differs from its predecessor its
// range starts, where it differs from its successor it ends.  Each thread takes four
// consecutive keys (one 16-byte load); the neighbours across threads come by shuffles,
// across warps by a load.  keys must be 16-byte aligned.
__global__ void __launch_bounds__(256) k_tile_ranges(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                                                     int64_t n_max, uint2 *__restrict__ ranges) {
    int64_t n = n_max;
    if (n_dev) {
        int64_t d = (int64_t)*n_dev;
        if (d < n) n = d;
    }
    const int lane = threadIdx.x & 31;
    const int64_t n4 = n >> 2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q - lane < n4;
         q += (int64_t)gridDim.x * blockDim.x) {
        const bool in = q < n4;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (in) v = reinterpret_cast<const uint4 *>(keys)[q];
        uint32_t prev = __shfl_up_sync(0xffffffffu, v.w, 1);
        uint32_t next = __shfl_down_sync(0xffffffffu, v.x, 1);
        if (!in) continue;
        const int64_t p = 4 * q;
        if (lane == 0 && p > 0) prev = keys[p - 1];
        if ((lane == 31 || q + 1 >= n4) && p + 4 < n) next = keys[p + 4];
        const uint32_t k[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t before = i == 0 ? prev : k[i - 1];
            const uint32_t after = i == 3 ? next : k[i + 1];
            if (p + i == 0 || before != k[i]) ranges[k[i]].x = (uint32_t)(p + i);
            if (p + i == n - 1 || after != k[i]) ranges[k[i]].y = (uint32_t)(p + i + 1);
        }
    }
    // the last n mod 4 keys
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) {
        const int64_t p = 4 * n4 + threadIdx.x;
        const uint32_t k = keys[p];
        if (p == 0 || keys[p - 1] != k) ranges[k].x = (uint32_t)p;
        if (p == n - 1 || keys[p + 1] != k) ranges[k].y = (uint32_t)(p + 1);
    }
}

// One CTA per tile of a single image (with the per-pixel blended / walked counts).
template <int TW, int TH>
__global__ void __launch_bounds__(256) k_blend_fwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, int W, int H, int ntx, float bg0, float bg1, float bg2,
    int membership, uint32_t rank_mask, float *__restrict__ image, float *__restrict__ final_T,
    uint32_t *__restrict__ n_contrib, uint32_t *__restrict__ n_blended,
    uint32_t *__restrict__ n_walked) {
    __shared__ __align__(16) FwdSmem sm;
    const int tile = blockIdx.x;
    const TileOut o{image, final_T, n_contrib, n_blended, n_walked, bg0, bg1, bg2, W, H, membership, rank_mask, 0u};
    blend_fwd_tile<TW, TH, true>(tile % ntx, tile / ntx, ranges[tile], sorted_vals, ranked, o, sm);
}

__global__ void k_entries_to_global(const uint32_t *__restrict__ sorted_vals,
                                    const uint32_t *__restrict__ perm, Selection sel, int64_t K,
                                    int64_t *__restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < K;
         e += (int64_t)gridDim.x * blockDim.x)
        out[e] = sel_global(sel, perm[sorted_vals[e]]);
}

}  // namespace

cudaError_t launch_entries_to_global(const uint32_t *sorted_vals, const uint32_t *perm,
                                     const Selection &sel, int64_t K, int64_t *out,
                                     cudaStream_t st) {
    if (K <= 0) return cudaSuccess;
    int64_t blocks = std::min<int64_t>((K + 255) / 256, 148 * 16);
    k_entries_to_global<<<(unsigned)blocks, 256, 0, st>>>(sorted_vals, perm, sel, K, out);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_emit(const float4 *ranked, const uint32_t *offsets, const uint32_t *touched_r,
                        int64_t n, const RenderParams &rp, int W, int H, uint32_t *keys, uint32_t *vals,
                        uint32_t cap, cudaStream_t st, const uint32_t *total, uint32_t *peak) {
    if (n <= 0) return cudaSuccess;
    if (peak && !total) return cudaErrorInvalidValue;
    const int64_t threads = ((n + 31) / 32) * 32;
    k_emit<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(ranked, offsets, touched_r, n, rp, W, H, cap,
                                                                keys, vals, total, peak);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const uint32_t *keys, const uint32_t *n_dev, int64_t n_max,
                               uint2 *ranges, cudaStream_t st) {
    if (n_max <= 0) return cudaSuccess;
    int64_t blocks = (n_max / 4 + 255) / 256;   // four keys per thread
    if (blocks < 1) blocks = 1;
    if (blocks > 148 * 16) blocks = 148 * 16;
    k_tile_ranges<<<(unsigned)blocks, 256, 0, st>>>(keys, n_dev, n_max, ranges);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_blend_fwd(const uint2 *ranges, const uint32_t *sorted_vals,
                             const float4 *ranked, const CamParams &cam, const RenderParams &rp,
                             float *image, float *final_T, uint32_t *n_contrib,
                             uint32_t *n_blended, uint32_t *n_walked, cudaStream_t st) {
    const unsigned tiles = (unsigned)(rp.ntx * rp.nty);
    if (tiles == 0) return cudaSuccess;
#define GC_BLEND_ARGS                                                                          \
    ranges, sorted_vals, ranked, cam.width, cam.height, rp.ntx, rp.bg[0], rp.bg[1], rp.bg[2], \
        rp.membership, list_rank_mask(rp), image, final_T, n_contrib, n_blended, n_walked
    if (rp.tile_w == 16 && rp.tile_h == 16)
        k_blend_fwd<16, 16><<<tiles, 256, 0, st>>>(GC_BLEND_ARGS);
    else if (rp.tile_w == 8 && rp.tile_h == 32)
        k_blend_fwd<8, 32><<<tiles, 256, 0, st>>>(GC_BLEND_ARGS);
    else if (rp.tile_w == 32 && rp.tile_h == 8)
        k_blend_fwd<32, 8><<<tiles, 256, 0, st>>>(GC_BLEND_ARGS);
    else
        return cudaErrorInvalidValue;
    note_launches(1);
#undef GC_BLEND_ARGS
    return cudaGetLastError();
}

}  // namespace gc
