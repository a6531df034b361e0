// gc_bucket.cuh - binning by tile row, for one view (gc_bucket.cu) and for a batch of
// requests (gc_batch.cu): the (tile, Gaussian) entries written straight into per-row
// segments, so that one 8-bit radix pass on the tile column finishes the stable (tile,
// depth rank) order.  An entry is one word, column << 24 | rank (the rank within its image:
// at most 2^24 selected Gaussians per image), so the pass moves keys only and the sorted
// words are the tile lists.
//
// The entries of a Gaussian are its row intervals (binning step 15): in tile row y the
// columns [a_y, b_y].  Ordered by (tile, rank), the entries of row y are those of every
// Gaussian touching the row, by rank and then by column.  Writing them in that order into
// the segment of row y and sorting each segment stably on the column gives (row, column,
// rank) = (tile, rank) order, the order an LSD radix sort on the tile index gives from the
// rank-order emit; its first pass is replaced by direct placement:
//   k_bucket_count     one warp per 32 consecutive items of one image (a chunk): entries
//                      per tile row of the image, counts[cell of (row, chunk)];
//   exclusive scan     of the counts in cell order, so that scanned[cell] is the number of
//                      entries before the chunk's part of the row;
//   k_bucket_segments  each row's segment padded to whole radix tiles (a radix block never
//                      straddles two rows): the shift from the scanned offsets to the padded
//                      positions, the segments in radix-block units, the padded total;
//   k_bucket_pads      pad slots get the word 0xFFFFFFFF (column 255, which no tile uses:
//                      sorted behind the row's entries);
//   k_bucket_place     the chunk's entries of each row at their positions, word = column <<
//                      24 | rank;
//   k_bucket_ranges    after the column pass, tile (row, column)'s range is the column's digit
//                      range in the row's segment, read from the pass's scanned digit counts.
// Within a chunk the lanes' entries of a row are laid out lane by lane (rank order); each warp
// computes the per-row lane prefix in a 32-row window of shared memory (column = lane, padded
// to 33 words so that both the lane writes and the row scans hit distinct banks).  At most
// 255 tile columns per image.
//
// The layout is a map (template parameter) with two device methods:
//   chunk(c, BucketChunk &)  the image of chunk c, the cells of its rows, its first item;
//   row(gr, BucketRow &)     the cells of global row gr (all chunks of its image, in order),
//                            the global index of its column-0 tile and its tile columns.
// Cells are numbered image by image, row-major (row, chunk) within an image; global rows image
// by image.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_tile.cuh"

namespace gc {

struct BucketChunk {
    RenderParams rp;
    int W, H, n_rows;
    int64_t cell0;   // cell of (row 0, this chunk)
    int64_t stride;  // cells per row of the image (its chunk count)
    int64_t row0;    // global row of the image's row 0
    int64_t r0;      // first item of the chunk
    int64_t v0;      // rank of the chunk's first item within its image (the list words' rank)
    int n_valid;     // lanes holding an item
};

struct BucketRow {
    int64_t cell;     // cell of (this row, the image's first chunk)
    int64_t n_cells;  // the image's chunk count
    int64_t tile0;    // global tile index of (this row, column 0)
    int ntx;          // tile columns
};

namespace {

constexpr int kBucketWarps = 8;
constexpr int kWin = 32;  // tile rows per window

// Rows of one lane's Gaussian (item r): [ty0, ty1] (empty: ty1 < ty0) and the interval of
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

// Entries per tile row of each chunk: counts[cell0 + row * stride], every row of the image.
template <class Map>
__global__ void __launch_bounds__(kBucketWarps * 32) k_bucket_count(const float4 *__restrict__ ranked,
                                                                    const uint32_t *__restrict__ touched_r, Map map,
                                                                    int64_t n_chunks, uint32_t *__restrict__ counts) {
    __shared__ uint32_t m[kBucketWarps][kWin][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kBucketWarps + warp;
    if (c >= n_chunks) return;  // whole warp
    BucketChunk ci;
    map.chunk(c, ci);
    const int64_t r = ci.r0 + lane;
    const bool has = lane < ci.n_valid && touched_r[r] != 0u;
    LaneRows L;
    lane_rows(ranked, r, has, ci.rp, L);
    uint32_t(*mw)[33] = m[warp];
    for (int w0 = 0; w0 < ci.n_rows; w0 += kWin) {
#pragma unroll 8
        for (int j = 0; j < kWin; ++j) mw[j][lane] = 0u;
        const int y0 = max(L.ty0, w0), y1 = min(L.ty1, w0 + kWin - 1);
        for (int y = y0; y <= y1; ++y) {
            int a, b;
            lane_row(L, y, ci.rp, ci.W, ci.H, a, b);
            if (b >= a) mw[y - w0][lane] = (uint32_t)(b - a + 1);
        }
        __syncwarp();
        uint32_t s = 0u;
#pragma unroll 8
        for (int l = 0; l < 32; ++l) s += mw[lane][l];
        if (w0 + lane < ci.n_rows) counts[ci.cell0 + (int64_t)(w0 + lane) * ci.stride] = s;
        __syncwarp();
    }
}

// One CTA over all n_rows global rows: per row its entry total (from the scanned counts), the
// padded segment start, the shift from scanned offsets to positions, the segment in radix-block
// units and the pad range; words[3] = padded total.  A demand (*demand: one past the largest
// backward partial slot the entries take) above the capacity `cap` is recorded in *peak (the
// fixed-capacity check) and, like a padded total beyond the buffers (`alloc`), empties every
// segment: nothing is placed or sorted, so that no blend reads, and no backward writes, past
// the buffers sized by the capacity.
template <class Map>
__global__ void __launch_bounds__(1024) k_bucket_segments(const uint32_t *__restrict__ scanned,
                                                          const uint32_t *__restrict__ total,
                                                          const uint32_t *__restrict__ demand, Map map, int n_rows,
                                                          int64_t n_cells, uint32_t tile_keys, uint32_t cap,
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
        const int gr = base + (int)threadIdx.x;
        uint32_t start = 0u, tot = 0u, size = 0u;
        if (gr < n_rows) {
            BucketRow ri;
            map.row(gr, ri);
            if (ri.n_cells > 0) {
                start = scanned[ri.cell];
                const int64_t e = ri.cell + ri.n_cells;
                const uint32_t end = e < n_cells ? scanned[e] : *total;
                tot = end - start;
                size = (tot + tile_keys - 1) / tile_keys * tile_keys;
            }
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
            const uint32_t v = ws[lane];
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
        const uint32_t ps = carry + ws[warp] + inc - size;  // padded start of row gr
        if (gr < n_rows) {
            shift[gr] = ps - start;
            seg_block0[gr] = ps / tile_keys;
            pads[gr] = make_uint2(ps + tot, size - tot);
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint32_t padded = carry;
        seg_block0[n_rows] = padded / tile_keys;
        words[3] = padded;
        const uint32_t want = *demand;
        if (peak && want > cap) atomicMax(peak, want);
        if (want > cap || padded > alloc) {
            for (int y = 0; y <= n_rows; ++y) seg_block0[y] = 0u;
            words[3] = 0u;
        }
    }
}

// Pad slots of global row blockIdx.x: word 0xFFFFFFFF.
__global__ void __launch_bounds__(256) k_bucket_pads(const uint2 *__restrict__ pads, const uint32_t *words,
                                                     uint32_t *__restrict__ keys) {
    if (words[3] == 0u) return;  // nothing placed (empty frame or overflow)
    const uint2 p = pads[blockIdx.x];
    for (uint32_t i = threadIdx.x; i < p.y; i += 256) keys[p.x + i] = 0xffffffffu;
}

// The chunk's entries of every row at their positions: scanned[cell0 + row * stride] +
// shift[row0 + row] + (entries of the lower lanes in the row) + (column - a_row).  Per window
// of 32 rows the lanes put their counts and first columns in shared memory, lane j turns row
// j's counts into start positions, then the warp writes each row's contiguous region with
// coalesced stores: element e of the region belongs to the last lane whose start is <= e
// (binary search over the row's 32 starts), at column first + (e - start).  (Writing the
// window's entries as one flat sequence across rows, 32 per step, takes a second binary search
// per element and measured slower: a chunk's entries fall in few rows.)
template <class Map>
__global__ void __launch_bounds__(kBucketWarps * 32) k_bucket_place(const float4 *__restrict__ ranked,
                                                                    const uint32_t *__restrict__ touched_r, Map map,
                                                                    int64_t n_chunks,
                                                                    const uint32_t *__restrict__ scanned,
                                                                    const uint32_t *__restrict__ shift,
                                                                    const uint32_t *words, uint32_t alloc,
                                                                    uint32_t *__restrict__ keys) {
    __shared__ uint32_t m[kBucketWarps][kWin][33];   // counts, then start positions
    __shared__ uint8_t col[kBucketWarps][kWin][36];  // first column of each lane's interval
    __shared__ uint32_t rtot[kBucketWarps][kWin];    // entries of the chunk in each row
    __shared__ uint32_t bw[kBucketWarps][32];         // per owner of a row: its base word
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * kBucketWarps + warp;
    if (c >= n_chunks) return;   // whole warp
    if (words[3] == 0u) return;  // overflowed fixed capacity: nothing is placed
    BucketChunk ci;
    map.chunk(c, ci);
    const int64_t r = ci.r0 + lane;
    const bool has = lane < ci.n_valid && touched_r[r] != 0u;
    LaneRows L;
    lane_rows(ranked, r, has, ci.rp, L);
    const int ylo = (int)__reduce_min_sync(0xffffffffu, (uint32_t)(has ? L.ty0 : 0x7fffffff));
    const int yhi = (int)__reduce_max_sync(0xffffffffu, (uint32_t)(has ? L.ty1 + 1 : 0)) - 1;
    uint32_t(*mw)[33] = m[warp];
    uint8_t(*cw)[36] = col[warp];
    const uint32_t v0 = (uint32_t)ci.v0;
    for (int w0 = (ylo / kWin) * kWin; w0 <= yhi; w0 += kWin) {
#pragma unroll 8
        for (int j = 0; j < kWin; ++j) mw[j][lane] = 0u;
        const int y0 = max(L.ty0, w0), y1 = min(L.ty1, w0 + kWin - 1);
        for (int y = y0; y <= y1; ++y) {
            int a, b;
            lane_row(L, y, ci.rp, ci.W, ci.H, a, b);
            if (b >= a) {
                mw[y - w0][lane] = (uint32_t)(b - a + 1);
                cw[y - w0][lane] = (uint8_t)a;
            }
        }
        __syncwarp();
        {  // lane j: start positions of every lane's entries in row w0 + j
            const int y = w0 + lane;
            uint32_t run = 0u;
            if (y < ci.n_rows) run = scanned[ci.cell0 + (int64_t)y * ci.stride] + shift[ci.row0 + y];
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
        const int jmax = min(kWin, ci.n_rows - w0);
        const uint32_t lane_le = 0xffffffffu >> (31 - lane);  // bits 0..lane
        // not unrolled: a row holds one warp step of the chunk's entries or none, mostly
#pragma unroll 1
        for (int j = 0; j < jmax; ++j) {
            const uint32_t tot = rtot[warp][j];
            if (tot == 0u) continue;  // warp-uniform
            // lane l's entries of the row are [rel, end) of the row's run, in lane order
            const uint32_t p0 = mw[j][0], s = mw[j][lane];
            const uint32_t rel = s - p0, end = lane < 31 ? mw[j][lane + 1] - p0 : tot;
            const bool own = end > rel;
            const uint32_t owners = __ballot_sync(0xffffffffu, own);
            // owner k (k-th lane with entries): word of its element e = base + (e << 24), base =
            // ((first column - rel) << 24) + rank; the column stays in 0..254, so the sum mod 2^32
            // is the word
            if (own)
                bw[warp][__popc(owners & (lane_le >> 1))] =
                    (((uint32_t)cw[j][lane] - rel) << kListRankBits) + v0 + (uint32_t)lane;
            __syncwarp();
#pragma unroll 1
            for (uint32_t e0 = 0; e0 < tot; e0 += 32) {
                // the owners' run starts in this window of 32 elements (bit rel - e0), and the
                // number of owners starting before it: element e's owner is the last start <= e
                const uint32_t starts =
                    __reduce_or_sync(0xffffffffu, (own && rel - e0 < 32u) ? 1u << (rel - e0) : 0u);
                const uint32_t before = __popc(__ballot_sync(0xffffffffu, own && rel < e0));
                const uint32_t e = e0 + lane;
                if (e < tot) {
                    const uint32_t pe = p0 + e;
                    const int k = (int)(before + __popc(starts & lane_le)) - 1;
                    if (pe < alloc) keys[pe] = bw[warp][k] + (e << kListRankBits);
                }
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

// Tile ranges after the column pass: thread per (global row, column < 255).  The segmented pass
// leaves the scanned per-block digit counts at the start of its scratch, segment-major and
// digit-major within a segment (radix_sort_pairs): digit d of the segment with first block b0
// and nb blocks starts at counts[256 b0 + d nb] and ends where digit d + 1 starts.  Empty
// ranges are not written (ranges must be zeroed).
template <class Map>
__global__ void __launch_bounds__(256) k_bucket_ranges(const uint32_t *__restrict__ counts,
                                                       const uint32_t *__restrict__ seg_block0, Map map, int n_rows,
                                                       uint2 *__restrict__ ranges) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_rows * 255) return;
    const int gr = (int)(i / 255), d = (int)(i - (int64_t)gr * 255);
    BucketRow ri;
    map.row(gr, ri);
    if (d >= ri.ntx) return;
    const uint32_t b0 = seg_block0[gr], nb = seg_block0[gr + 1] - b0;
    if (nb == 0u) return;
    const uint32_t a = counts[(int64_t)256 * b0 + (int64_t)d * nb];
    const uint32_t b = counts[(int64_t)256 * b0 + (int64_t)(d + 1) * nb];
    if (b > a) ranges[ri.tile0 + d] = make_uint2(a, b);
}

// Carving of the row-binning scratch: counts and scanned counts (n_cells each), the chained
// scan's state (8-byte aligned), the segments (n_rows + 1) and the pad ranges (uint2).
struct BucketScratch {
    uint32_t *counts, *scanned, *partials, *segs;
    uint2 *pads;
};

inline size_t bucket_words(int64_t n_cells, int n_rows) {
    const int64_t c = n_cells > 0 ? n_cells : 1;
    return (size_t)(2 * c + scan_partials_size(c) + (n_rows + 1) + 2 * (n_rows + 1) + 64);
}

inline BucketScratch bucket_carve(uint32_t *scratch, int64_t n_cells, int n_rows) {
    const int64_t c = n_cells > 0 ? n_cells : 1;
    BucketScratch b;
    b.counts = scratch;
    b.scanned = b.counts + c;
    b.partials = b.counts + 2 * c;  // an even word offset: the scan's 64-bit status words
    b.segs = b.partials + scan_partials_size(c);
    size_t off = (size_t)(b.segs - scratch) + (size_t)(n_rows + 1);
    off = (off + 1) & ~(size_t)1;
    b.pads = reinterpret_cast<uint2 *>(scratch + off);
    return b;
}

// Placement (count, scan, segments, pads, place).  total: device word with the entry count
// (the scan of the Gaussians' tile counts); demand: device word checked against the capacity
// `cap` (the partial slots the entries need); alloc: key capacity of keys / vals; shift: n_rows
// words; words[1] error word, words[3] padded total; peak: fixed-capacity record or NULL.
template <class Map>
cudaError_t bucket_place(const float4 *ranked, const uint32_t *total, const uint32_t *demand,
                         const uint32_t *touched_r, const Map &map,
                         int64_t n_chunks, int n_rows, int64_t n_cells, uint32_t *keys,
                         uint32_t cap, uint32_t alloc, uint32_t *words, uint32_t *shift, uint32_t *scratch,
                         uint32_t *peak, cudaStream_t st) {
    const BucketScratch b = bucket_carve(scratch, n_cells, n_rows);
    if ((reinterpret_cast<uintptr_t>(b.pads) | reinterpret_cast<uintptr_t>(b.partials)) & 7)
        return cudaErrorMisalignedAddress;  // 8-byte words must be 8-byte aligned (never launched)
    if (n_rows <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::max<int64_t>((n_chunks + kBucketWarps - 1) / kBucketWarps, 1);
    if (n_chunks > 0) {
        k_bucket_count<Map><<<grid, kBucketWarps * 32, 0, st>>>(ranked, touched_r, map, n_chunks, b.counts);
        note_launches(1);
    }
    cudaError_t e = launch_exclusive_scan(b.counts, b.scanned, n_cells, nullptr, b.partials, st, words + 1);
    if (e != cudaSuccess) return e;
    k_bucket_segments<Map><<<1, 1024, 0, st>>>(b.scanned, total, demand, map, n_rows, n_cells,
                                               (uint32_t)radix_tile_keys(true), cap, alloc, shift, b.segs, b.pads,
                                               words, peak);
    note_launches(1);
    k_bucket_pads<<<(unsigned)n_rows, 256, 0, st>>>(b.pads, words, keys);
    note_launches(1);
    if (n_chunks > 0) {
        k_bucket_place<Map><<<grid, kBucketWarps * 32, 0, st>>>(ranked, touched_r, map, n_chunks, b.scanned, shift,
                                                                words, alloc, keys);
        note_launches(1);
    }
    return cudaGetLastError();
}

// One segmented stable pass on the column byte of the words (keys only): the sorted words are
// the tile lists, in keys[*out_buf]; the ranges come from the pass's digit counts.
inline cudaError_t bucket_sort(uint32_t *keys[2], uint32_t alloc, uint32_t *words, int n_rows, int64_t n_cells,
                               uint32_t *scratch, uint32_t *sort_scratch, int *out_buf, cudaStream_t st) {
    const BucketScratch b = bucket_carve(scratch, n_cells, n_rows);
    return radix_sort_pairs(keys, nullptr, alloc, words + 3, 32, sort_scratch, out_buf, st, words + 1, true, b.segs,
                            n_rows, kListRankBits);
}

// Tile ranges from the column pass's digit counts (after bucket_sort with the same scratch).
template <class Map>
cudaError_t bucket_ranges(const Map &map, int n_rows, int64_t n_cells, uint32_t *scratch,
                          const uint32_t *sort_scratch, uint2 *ranges, cudaStream_t st) {
    if (n_rows <= 0) return cudaSuccess;
    const BucketScratch b = bucket_carve(scratch, n_cells, n_rows);
    const int64_t threads = (int64_t)n_rows * 255;
    k_bucket_ranges<Map><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(sort_scratch, b.segs, map, n_rows,
                                                                            ranges);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace

}  // namespace gc
