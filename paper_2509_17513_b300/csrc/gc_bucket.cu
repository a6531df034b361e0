// gc_bucket.cu - binning by tile row: the (tile, Gaussian) entries of one view written
// straight into per-row segments, so that one 8-bit radix pass on the tile column finishes
// the stable (tile, depth rank) order.
//
// The entries of a Gaussian are its row intervals (binning step 15): in tile row y the
// columns [a_y, b_y].  Ordered by (tile, rank), the entries of row y are those of every
// Gaussian touching the row, by rank and then by column.  Writing them in that order
// into the segment of row y (rank order within the row, the Gaussian's columns in order)
// and then sorting each segment stably on the column gives (row, column, rank) = (tile,
// rank) order, the order that an LSD radix sort on the tile index gives from the rank-order
// emit.  Its first pass is replaced by direct placement:
//   k_bucket_count  one warp per 32 consecutive ranks (a chunk): entries per tile row,
//                   counts[row * n_chunks + chunk];
//   exclusive scan  of the counts (row-major), so that scanned[row * n_chunks + chunk] is
//                   the number of entries before the chunk's part of the row;
//   k_bucket_segments  each row's segment padded to whole radix tiles (a radix block never
//                   straddles two rows): the shift from the scanned offsets to the padded
//                   positions, the segments in radix-block units, the padded total;
//   k_bucket_pads   pad slots get the key 0xFFFFFFFF (column 255, which no tile uses: sorted
//                   behind the row's entries);
//   k_bucket_place  the chunk's entries of each row written at their positions, key =
//                   (row << 8) | column, value = rank.
// Within a chunk the lanes' entries of a row are laid out lane by lane (rank order); each
// warp computes the per-row lane prefix in a 32-row window of shared memory (column =
// lane, padded to 33 words so that both the lane writes and the row scans hit distinct
// banks).  After the pass, tile (row, column)'s range is the column's digit range in the
// row's segment, read from the pass's scanned digit counts.  At most 255 tile columns.
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_tile.cuh"

namespace gc {

namespace {

constexpr int kBucketWarps = 8;
constexpr int kWin = 32;  // tile rows per window

// Rows of one lane's Gaussian (rank r): [ty0, ty1] (empty: ty1 < ty0) and the interval of
// each row from the packed bytes or, for Gaussians whose rows are not packed, recomputed.
struct LaneRows {
    RowGeom g;
    float4 r4;
    int ty0, ty1, tx0;
    bool packed;
};

__device__ __forceinline__ void lane_rows(const float4 *__restrict__ ranked, int64_t r, bool has,
                                          const RenderParams &rp, LaneRows &L) {
    L.ty0 = 0;
    L.ty1 = -1;
    L.tx0 = 0;
    L.packed = true;
    L.r4 = make_float4(__uint_as_float(0xffu), 0.f, 0.f, 0.f);
    if (!has) return;
    L.r4 = ranked[kRec * r + 4];
    L.packed = rows_packed(L.r4);
    if (L.packed) {
        const float4 r2 = ranked[kRec * r + 2];
        const uint32_t rx = __float_as_uint(r2.z), ry = __float_as_uint(r2.w);
        L.tx0 = (int)(rx & 0xffffu) >> rp.tile_w_log2;
        L.ty0 = (int)(ry & 0xffffu) >> rp.tile_h_log2;
        L.ty1 = (int)(ry >> 16) >> rp.tile_h_log2;
    } else {
        row_geom(ranked[kRec * r], ranked[kRec * r + 2], ranked[kRec * r + 3], rp, L.g);
        L.tx0 = L.g.tx0;
        L.ty0 = L.g.ty0;
        L.ty1 = L.g.ty1;
    }
}

// Columns [a, b] of row y (a > b: no entry in the row); y in [ty0, ty1].
__device__ __forceinline__ void lane_row(const LaneRows &L, int y, const RenderParams &rp, int W, int H, int &a,
                                         int &b) {
    if (L.packed) packed_row(L.r4, y - L.ty0, L.tx0, a, b);
    else row_interval(L.g, y, rp, W, H, a, b);
}

// Entries per tile row of each chunk: counts[row * n_chunks + chunk], every row written.
__global__ void __launch_bounds__(kBucketWarps * 32) k_bucket_count(const float4 *__restrict__ ranked,
                                                                    const uint32_t *__restrict__ touched_r,
                                                                    int64_t n, RenderParams rp, int W, int H,
                                                                    int n_rows, int64_t n_chunks,
                                                                    uint32_t *__restrict__ counts) {
    __shared__ uint32_t m[kBucketWarps][kWin][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kBucketWarps + warp;
    if (c >= n_chunks) return;  // whole warp
    const int64_t r = c * 32 + lane;
    const bool has = r < n && touched_r[r] != 0u;
    LaneRows L;
    lane_rows(ranked, r, has, rp, L);
    uint32_t(*mw)[33] = m[warp];
    for (int w0 = 0; w0 < n_rows; w0 += kWin) {
#pragma unroll 8
        for (int j = 0; j < kWin; ++j) mw[j][lane] = 0u;
        const int y0 = max(L.ty0, w0), y1 = min(L.ty1, w0 + kWin - 1);
        for (int y = y0; y <= y1; ++y) {
            int a, b;
            lane_row(L, y, rp, W, H, a, b);
            if (b >= a) mw[y - w0][lane] = (uint32_t)(b - a + 1);
        }
        __syncwarp();
        uint32_t s = 0u;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) s += mw[lane][l];
        if (w0 + lane < n_rows) counts[(int64_t)(w0 + lane) * n_chunks + c] = s;
        __syncwarp();
    }
}

// One CTA: per row its entry total (from the scanned counts), the padded segment start,
// the shift from scanned offsets to positions, the segments in radix-block units, the pad
// range, and words[3] = padded total.  More entries than the capacity `cap` are recorded
// in *peak (the fixed-capacity check); a padded total beyond the buffers (`alloc`) also
// empties every segment, so that nothing is placed or sorted.
__global__ void __launch_bounds__(1024) k_bucket_segments(const uint32_t *__restrict__ scanned,
                                                          const uint32_t *__restrict__ total, int n_rows,
                                                          int64_t n_chunks, uint32_t tile_keys, uint32_t cap,
                                                          uint32_t alloc, uint32_t *__restrict__ shift,
                                                          uint32_t *__restrict__ seg_block0,
                                                          uint2 *__restrict__ pads, uint32_t *words,
                                                          uint32_t *peak) {
    __shared__ uint32_t ws[33];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < n_rows; base += 1024) {
        const int y = base + (int)threadIdx.x;
        uint32_t start = 0u, tot = 0u, size = 0u;
        if (y < n_rows) {
            start = scanned[(int64_t)y * n_chunks];
            const uint32_t end = y + 1 < n_rows ? scanned[(int64_t)(y + 1) * n_chunks] : *total;
            tot = end - start;
            size = (tot + tile_keys - 1) / tile_keys * tile_keys;
        }
        uint32_t inc = size;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) ws[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t v = lane < 32 ? ws[lane] : 0u;
            uint32_t vi = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, vi, o);
                if (lane >= o) vi += u;
            }
            ws[lane] = vi - v;
            if (lane == 31) ws[32] = vi;
        }
        __syncthreads();
        const uint32_t ps = carry + ws[warp] + inc - size;  // padded start of row y
        if (y < n_rows) {
            shift[y] = ps - start;
            seg_block0[y] = ps / tile_keys;
            pads[y] = make_uint2(ps + tot, size - tot);
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint32_t padded = carry;
        seg_block0[n_rows] = padded / tile_keys;
        words[3] = padded;
        if (peak && *total > cap) atomicMax(peak, *total);
        if (padded > alloc) {
            for (int y = 0; y <= n_rows; ++y) seg_block0[y] = 0u;
            words[3] = 0u;
        }
    }
}

// Pad slots of row y (CTA y): key 0xFFFFFFFF, value 0.
__global__ void __launch_bounds__(256) k_bucket_pads(const uint2 *__restrict__ pads, const uint32_t *words,
                                                     uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    if (words[3] == 0u) return;  // nothing placed (empty frame or overflow)
    const uint2 p = pads[blockIdx.x];
    for (uint32_t i = threadIdx.x; i < p.y; i += 256) {
        keys[p.x + i] = 0xffffffffu;
        vals[p.x + i] = 0u;
    }
}

// The chunk's entries of every row at their positions: scanned[row * n_chunks + chunk] +
// shift[row] + (entries of the lower lanes in the row) + (column - a_row).  Per window of 32
// rows the lanes put their counts and first columns in shared memory, lane j turns row j's
// counts into start positions, then the warp writes each row's contiguous region with
// coalesced stores: element e of the region belongs to the last lane whose start is <= e
// (binary search over the row's 32 starts), at column first + (e - start).
__global__ void __launch_bounds__(kBucketWarps * 32) k_bucket_place(const float4 *__restrict__ ranked,
                                                                    const uint32_t *__restrict__ touched_r,
                                                                    int64_t n, RenderParams rp, int W, int H,
                                                                    int n_rows, int64_t n_chunks,
                                                                    const uint32_t *__restrict__ scanned,
                                                                    const uint32_t *__restrict__ shift,
                                                                    const uint32_t *words, uint32_t alloc,
                                                                    uint32_t *__restrict__ keys,
                                                                    uint32_t *__restrict__ vals) {
    __shared__ uint32_t m[kBucketWarps][kWin][33];   // counts, then start positions
    __shared__ uint8_t col[kBucketWarps][kWin][36];  // first column of each lane's interval
    __shared__ uint32_t rtot[kBucketWarps][kWin];    // entries of the chunk in each row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kBucketWarps + warp;
    if (c >= n_chunks) return;  // whole warp
    if (words[3] == 0u) return;  // overflowed fixed capacity: nothing is placed
    const int64_t r = c * 32 + lane;
    const bool has = r < n && touched_r[r] != 0u;
    LaneRows L;
    lane_rows(ranked, r, has, rp, L);
    const int ylo = (int)__reduce_min_sync(0xffffffffu, (uint32_t)(has ? L.ty0 : 0x7fffffff));
    const int yhi = (int)__reduce_max_sync(0xffffffffu, (uint32_t)(has ? L.ty1 + 1 : 0)) - 1;
    uint32_t(*mw)[33] = m[warp];
    uint8_t(*cw)[36] = col[warp];
    const uint32_t r0 = (uint32_t)(c * 32);
    for (int w0 = (ylo / kWin) * kWin; w0 <= yhi; w0 += kWin) {
#pragma unroll 8
        for (int j = 0; j < kWin; ++j) mw[j][lane] = 0u;
        const int y0 = max(L.ty0, w0), y1 = min(L.ty1, w0 + kWin - 1);
        for (int y = y0; y <= y1; ++y) {
            int a, b;
            lane_row(L, y, rp, W, H, a, b);
            if (b >= a) {
                mw[y - w0][lane] = (uint32_t)(b - a + 1);
                cw[y - w0][lane] = (uint8_t)a;
            }
        }
        __syncwarp();
        {  // lane j: start positions of every lane's entries in row w0 + j
            const int y = w0 + lane;
            uint32_t run = 0u;
            if (y < n_rows) run = scanned[(int64_t)y * n_chunks + c] + shift[y];
            const uint32_t base = run;
#pragma unroll 8
            for (int l = 0; l < 32; ++l) {
                const uint32_t x = mw[lane][l];
                mw[lane][l] = run;
                run += x;
            }
            rtot[warp][lane] = run - base;
        }
        __syncwarp();
        const int jmax = min(kWin, n_rows - w0);
        for (int j = 0; j < jmax; ++j) {
            const uint32_t tot = rtot[warp][j];
            if (tot == 0u) continue;  // warp-uniform
            const uint32_t p0 = mw[j][0];
            const uint32_t key0 = (uint32_t)(w0 + j) << 8;
            for (uint32_t e = lane; e < tot; e += 32) {
                const uint32_t pe = p0 + e;
                int o = 0;  // last lane whose start is <= pe
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (mw[j][o + step] <= pe) o += step;
                const uint32_t x = (uint32_t)cw[j][o] + (pe - mw[j][o]);
                if (pe < alloc) {
                    keys[pe] = key0 | x;
                    vals[pe] = r0 + (uint32_t)o;
                }
            }
        }
        __syncwarp();
    }
}

// Tile lists without the row padding (diagnostics): per tile its range shifted back by the
// row's pad shift, and the global index of each of its entries at the unpadded position.
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
        for (uint32_t p = r.x; p < r.y; ++p) out_ids[p - sh] = sel_global(sel, perm[sorted_vals[p]]);
    }
}

}  // namespace

// Column 255 is left to the pad keys, so that a tile's range is a digit range of its row.
bool bucket_binning_fits(const RenderParams &rp) { return rp.ntx >= 1 && rp.ntx <= 255 && rp.nty <= 1 << 16; }

size_t bucket_scratch_words(int64_t n, int n_rows) {
    const int64_t chunks = (n + 31) / 32;
    const int64_t cells = (int64_t)n_rows * (chunks > 0 ? chunks : 1);
    // counts, scanned counts, scan state (8-byte aligned), segments, pads (uint2, 8-byte aligned)
    return (size_t)(2 * cells + scan_partials_size(cells) + (n_rows + 1) + 2 * (n_rows + 1) + 64);
}

namespace {
struct BucketScratch {
    uint32_t *counts, *scanned, *partials, *segs;
    uint2 *pads;
};
BucketScratch carve(uint32_t *scratch, int64_t n, int n_rows) {
    const int64_t chunks = (n + 31) / 32;
    const int64_t cells = (int64_t)n_rows * (chunks > 0 ? chunks : 1);
    BucketScratch b;
    b.counts = scratch;
    b.scanned = b.counts + cells;
    b.partials = b.counts + 2 * cells;  // an even word offset: the scan's 64-bit status words are 8-byte aligned
    b.segs = b.partials + scan_partials_size(cells);
    size_t off = (size_t)(b.segs - scratch) + (size_t)(n_rows + 1);
    off = (off + 1) & ~(size_t)1;
    b.pads = reinterpret_cast<uint2 *>(scratch + off);
    return b;
}
}  // namespace

cudaError_t launch_bucket_place(const float4 *ranked, const uint32_t *total, const uint32_t *touched_r, int64_t n,
                                const RenderParams &rp, int W, int H, uint32_t *keys, uint32_t *vals, uint32_t cap,
                                uint32_t alloc, uint32_t *words, uint32_t *shift, uint32_t *scratch, uint32_t *peak,
                                cudaStream_t st) {
    const int n_rows = rp.nty;
    const int64_t chunks = (n + 31) / 32;
    const int64_t cells = (int64_t)n_rows * chunks;
    const BucketScratch b = carve(scratch, n, n_rows);
    if ((reinterpret_cast<uintptr_t>(b.pads) | reinterpret_cast<uintptr_t>(b.partials)) & 7)
        return cudaErrorMisalignedAddress;  // 8-byte words must be 8-byte aligned (never launched)
    const unsigned grid = (unsigned)((chunks + kBucketWarps - 1) / kBucketWarps);
    k_bucket_count<<<grid, kBucketWarps * 32, 0, st>>>(ranked, touched_r, n, rp, W, H, n_rows, chunks, b.counts);
    note_launches(1);
    cudaError_t e = launch_exclusive_scan(b.counts, b.scanned, cells, nullptr, b.partials, st, words + 1);
    if (e != cudaSuccess) return e;
    k_bucket_segments<<<1, 1024, 0, st>>>(b.scanned, total, n_rows, chunks, (uint32_t)radix_tile_keys(), cap, alloc,
                                          shift, b.segs, b.pads, words, peak);
    note_launches(1);
    k_bucket_pads<<<(unsigned)n_rows, 256, 0, st>>>(b.pads, words, keys, vals);
    note_launches(1);
    k_bucket_place<<<grid, kBucketWarps * 32, 0, st>>>(ranked, touched_r, n, rp, W, H, n_rows, chunks, b.scanned,
                                                       shift, words, alloc, keys, vals);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bucket_sort(uint32_t *keys[2], uint32_t *vals[2], uint32_t alloc, uint32_t *words, int64_t n,
                               int n_rows, uint32_t *scratch, uint32_t *sort_scratch, int *out_buf, cudaStream_t st) {
    const BucketScratch b = carve(scratch, n, n_rows);
    // the sorted keys are not kept: the ranges come from the pass's digit counts
    return radix_sort_pairs(keys, vals, alloc, words + 3, 8, sort_scratch, out_buf, st, words + 1, false, b.segs,
                            n_rows);
}

cudaError_t launch_bucket_ranges(int64_t n, uint32_t *scratch, uint32_t *sort_scratch, const RenderParams &rp,
                                 uint2 *ranges, cudaStream_t st) {
    const BucketScratch b = carve(scratch, n, rp.nty);
    return launch_segment_digit_ranges(sort_scratch, b.segs, rp.nty, rp.ntx, ranges, st);
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
