// gc_bucket.cu - binning by tile row for one view (the kernels are in gc_bucket.cuh): one
// image, chunk c = items 32 c .. 32 c + 31 of the depth-ranked Gaussians, cell (row y, chunk
// c) = y * n_chunks + c, global row = tile row, tile (y, x) = y * ntx + x.  Also the export of
// the tile lists without the row padding (diagnostics).
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_bucket.cuh"

namespace gc {

namespace {

struct SingleMap {
    RenderParams rp;
    int W, H;
    int64_t n, n_chunks;
    __device__ __forceinline__ void chunk(int64_t c, BucketChunk &ci) const {
        ci.rp = rp;
        ci.W = W;
        ci.H = H;
        ci.n_rows = rp.nty;
        ci.cell0 = c;
        ci.stride = n_chunks;
        ci.row0 = 0;
        ci.r0 = c * 32;
        ci.v0 = c * 32;
        ci.n_valid = n - c * 32 < 32 ? (int)(n - c * 32) : 32;
    }
    __device__ __forceinline__ void row(int64_t gr, BucketRow &ri) const {
        ri.cell = gr * n_chunks;
        ri.n_cells = n_chunks;
        ri.tile0 = gr * rp.ntx;
        ri.ntx = rp.ntx;
    }
};

SingleMap single_map(int64_t n, const RenderParams &rp, int W, int H) {
    return SingleMap{rp, W, H, n, (n + 31) / 32};
}

// Tile lists without the row padding (diagnostics): per tile its range shifted back by the
// row's pad shift, and the global index of each of its entries (the rank of its list word)
// at the unpadded position.
__global__ void k_row_lists_export(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
                                   const uint32_t *__restrict__ shift, int ntx, int64_t n_tiles,
                                   const uint32_t *__restrict__ perm, Selection sel, int32_t *__restrict__ out_ranges,
                                   int64_t *__restrict__ out_ids) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t sh = shift[t / ntx];
        const bool any = r.y > r.x;
        out_ranges[2 * t] = any ? (int32_t)(r.x - sh) : 0;
        out_ranges[2 * t + 1] = any ? (int32_t)(r.y - sh) : 0;
        for (uint32_t p = r.x; p < r.y; ++p) out_ids[p - sh] = sel_global(sel, perm[sorted_vals[p] & kListRankMask]);
    }
}

}  // namespace

// Column 255 is left to the pad words, so that a tile's range is a digit range of its row;
// ranks take the low 24 bits of a word.
bool bucket_binning_fits(const RenderParams &rp, int64_t n_sel) {
    return rp.ntx >= 1 && rp.ntx <= 255 && rp.nty <= 1 << 16 && n_sel <= (int64_t)kListRankMask + 1;
}

size_t bucket_scratch_words(int64_t n, int n_rows) { return bucket_words((int64_t)n_rows * ((n + 31) / 32), n_rows); }

cudaError_t launch_bucket_place(const float4 *ranked, const uint32_t *total, const uint32_t *touched_r, int64_t n,
                                const RenderParams &rp, int W, int H, uint32_t *keys, uint32_t cap,
                                uint32_t alloc, uint32_t *words, uint32_t *shift, uint32_t *scratch, uint32_t *peak,
                                cudaStream_t st) {
    const SingleMap map = single_map(n, rp, W, H);
    return bucket_place(ranked, total, total, touched_r, map, map.n_chunks, rp.nty, (int64_t)rp.nty * map.n_chunks, keys,
                        cap, alloc, words, shift, scratch, peak, st);
}

cudaError_t launch_bucket_sort(uint32_t *keys[2], uint32_t alloc, uint32_t *words, int64_t n, int n_rows,
                               uint32_t *scratch, uint32_t *sort_scratch, int *out_buf, cudaStream_t st) {
    return bucket_sort(keys, alloc, words, n_rows, (int64_t)n_rows * ((n + 31) / 32), scratch, sort_scratch, out_buf,
                       st);
}

cudaError_t launch_bucket_ranges(int64_t n, uint32_t *scratch, uint32_t *sort_scratch, const RenderParams &rp,
                                 uint2 *ranges, cudaStream_t st) {
    const SingleMap map = single_map(n, rp, 0, 0);
    return bucket_ranges(map, rp.nty, (int64_t)rp.nty * map.n_chunks, scratch, sort_scratch, ranges, st);
}

cudaError_t launch_row_lists_export(const uint2 *ranges, const uint32_t *sorted_vals, const uint32_t *shift,
                                    const RenderParams &rp, const uint32_t *perm, const Selection &sel,
                                    int32_t *out_ranges, int64_t *out_ids, cudaStream_t st) {
    const int64_t n_tiles = (int64_t)rp.ntx * rp.nty;
    if (n_tiles <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n_tiles + 127) / 128, 148 * 8);
    k_row_lists_export<<<(unsigned)blocks, 128, 0, st>>>(ranges, sorted_vals, shift, rp.ntx, n_tiles, perm, sel,
                                                         out_ranges, out_ids);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace gc
