// gc_internal.cuh - device-side types and launchers shared by the kernel files.
//
// Layout of the per-Gaussian projected record (five float4, 80 bytes), written
// by the preprocess kernel at the Gaussian's compact (selected) position and
// gathered into depth-rank order before binning:
//   r0 = { u, v, A, B }                  conic = inverse 2D covariance [[a, b], [b, c]],
//   r1 = { C, opacity, red, green }      stored pre-scaled: A = -a log2e/2, B = -b log2e,
//                                        C = -c log2e/2 (gc_blend.cuh)
//   r2 = { blue, layer, rect_x, rect_y } layer = the Gaussian's layer (int bits);
//                                        rect_* = pixel footprint, int bits: lo16 = first,
//                                        hi16 = last (inclusive)
//   r3 = { a, b, c, tc }                 the conic as computed by the binning spec and the
//                                        alpha-ellipse level (row intervals, step 15)
//   r4 = 16 bytes                        the row intervals packed (row i: start column
//                                        - tx0 in byte 2i, length in byte 2i + 1) when
//                                        the Gaussian has at most 8 tile rows and every
//                                        start offset is below 255; byte 0 = 255 otherwise
// The blends read r0..r2; emit and the reverse pass read a Gaussian's per-row tile
// intervals from r4, or recompute them from r0, r2, r3 when they are not packed.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gc4d.h"

namespace gc {

constexpr int kMaxLayers = 32;
constexpr uint32_t kCulledKey = 0xFFFFFFFFu;
constexpr int kRec = 5;  // float4s per projected record
constexpr int kMaxLevels = 8;  // levels of one multi-level render

// Output images (3 x H x W each) and dL/dimage of the levels of a multi-level render.
struct LevelPtrs {
    float *img[kMaxLevels];
};
struct LevelGrads {
    const float *g[kMaxLevels];
};

// Selected layer ranges: compact index j maps to global index
// range_begin[k] + (j - range_start[k]) for the range k holding j.
struct Selection {
    int n_ranges;
    int64_t range_begin[kMaxLayers];
    int64_t range_start[kMaxLayers + 1];  // prefix sums of range lengths
    int n_layers;
    int64_t layer_off[kMaxLayers + 1];    // the set's layer offsets (layer l = [off[l], off[l+1]))
};

// Layer (0-based) of global Gaussian i.
__host__ __device__ inline int layer_of(const Selection &s, int64_t i) {
    int l = 0;
    while (l + 1 < s.n_layers && i >= s.layer_off[l + 1]) ++l;
    return l;
}

struct CamParams {
    int width, height;
    float fx, fy, cx, cy;
    float R[9], t[3], campos[3];
};

struct RenderParams {
    float near_plane, dilation, frustum_clamp;
    float bg[3];
    int tile_w, tile_h, tile_w_log2, tile_h_log2;
    int ntx, nty;
    int membership;
    int alpha_cull;
    int list_packed;  // tile-list words: 0 = the rank; 1 = column << 24 | rank (row binning)
};

// Rank of a tile-list word: the low 24 bits of a row-binned list (whose top byte holds the
// tile column the lists were sorted on), else the whole word.
constexpr int kListRankBits = 24;
constexpr uint32_t kListRankMask = (1u << kListRankBits) - 1u;
__host__ __device__ __forceinline__ uint32_t list_rank_mask(const RenderParams &rp) {
    return rp.list_packed ? kListRankMask : 0xffffffffu;
}

// Attribute source.  FP32 arrays, or BF16/FP8 planes with per-channel scales.
// Per-Gaussian additive residuals of one frame (Sec. 3.2, Eq. 7): log-scale, opacity logit
// and SH coefficient offsets, FP32 device arrays by global index, NULL = none.
struct Residual {
    const float *ls, *logit, *sh;
};

struct GaussSrc {
    int64_t n;
    int sh_degree, K;
    int precision;
    const float *means, *log_scales, *quats, *opacity_logits, *sh;
    const int32_t *group_id;
    const uint16_t *means_h, *log_scales_h, *quats_h, *opacity_h;
    const uint8_t *sh_q;
    const float *scales;
    const float *group_q, *group_t;  // NULL = identity motion
    int n_groups;
    int per_gaussian;                // 1: group index = global Gaussian index (n_groups = n)
    Residual res;                    // the frame's residual deformation
    // GC_PREC_PLANES (the decoded attribute planes): per-layer plane buffers and offsets
    int n_layers, plane_width, pos_bits, n_channels;
    int64_t plane_pitch, pos_pitch;
    const uint8_t *plane_u8[kMaxLayers];
    const uint8_t *plane_pos[kMaxLayers];
    int64_t layer_off[kMaxLayers + 1];
    const float *dequant;
};

// Runs the statements with the compile-time constant PREC_ equal to the storage format
// `prec` (the preprocess and chain-rule kernels are instantiated per format).
#define GC_DISPATCH_PREC(prec, ...)                                                        \
    switch (prec) {                                                                        \
        case GC_PREC_FP32: { constexpr int PREC_ = GC_PREC_FP32; __VA_ARGS__; } break;           \
        case GC_PREC_BF16_FP8: { constexpr int PREC_ = GC_PREC_BF16_FP8; __VA_ARGS__; } break;   \
        default: { constexpr int PREC_ = GC_PREC_PLANES; __VA_ARGS__; } break;                   \
    }

// Where global Gaussian i sits in the decoded planes: its layer, the layer's row count and
// its row and column.
struct PlaneLoc {
    int l, row, col, rows;
};

__device__ __forceinline__ PlaneLoc plane_loc(const GaussSrc &G, int64_t i) {
    int l = 0;
    while (l + 1 < G.n_layers && i >= G.layer_off[l + 1]) ++l;
    const int j = (int)(i - G.layer_off[l]);
    const int n_l = (int)(G.layer_off[l + 1] - G.layer_off[l]);
    PlaneLoc p;
    p.l = l;
    p.rows = (n_l + G.plane_width - 1) / G.plane_width;
    p.row = j / G.plane_width;
    p.col = j - p.row * G.plane_width;
    return p;
}

// Channel ch (0..2 positions, 3..C-1 the uint8 channels) of the Gaussian at `p`:
// lo + code * step, the product and the sum each rounded once in FP32.
__device__ __forceinline__ float plane_value(const GaussSrc &G, const PlaneLoc &p, int ch) {
    uint32_t code;
    if (ch < 3) {
        const uint8_t *row = G.plane_pos[p.l] + ((int64_t)ch * p.rows + p.row) * G.pos_pitch;
        code = G.pos_bits == 16 ? (uint32_t)reinterpret_cast<const uint16_t *>(row)[p.col]
                                : reinterpret_cast<const uint32_t *>(row)[p.col];
    } else {
        code = G.plane_u8[p.l][((int64_t)(ch - 3) * p.rows + p.row) * G.plane_pitch + p.col];
    }
    const float2 d = reinterpret_cast<const float2 *>(G.dequant)[(int64_t)p.l * G.n_channels + ch];
    return __fadd_rn(__fmul_rn(__uint2float_rn(code), d.y), d.x);
}

__host__ __device__ inline int64_t sel_global(const Selection &s, int64_t j) {
    int k = 0;
    while (k + 1 < s.n_ranges && j >= s.range_start[k + 1]) ++k;
    return s.range_begin[k] + (j - s.range_start[k]);
}

// Kernel launches issued by this library (all contexts), for accounting.
void note_launches(int n);
uint64_t launches_total();

// ---- launchers (host) ----

// Projection of the n_sel selected Gaussians.  Writes the records rec[kRec*j ..], depth
// keys (kCulledKey when culled), values = j, and tiles touched per Gaussian.
cudaError_t launch_preprocess(const GaussSrc &g, const Selection &sel, int64_t n_sel,
                              const CamParams &cam, const RenderParams &rp, float4 *rec,
                              uint32_t *depth_keys, uint32_t *depth_vals, uint32_t *touched,
                              cudaStream_t st);

// rank r -> compact j = perm[r]: ranked[r] = rec[j], touched_r[r] = touched[j]
cudaError_t launch_rank_gather(const uint32_t *perm, const float4 *rec, const uint32_t *touched,
                               int64_t n, float4 *ranked, uint32_t *touched_r, cudaStream_t st);

// Exclusive scan of n uint32 values; writes out[0..n) and, if total != NULL,
// the sum to *total (device).  `partials` needs scan_partials_size(n) words (8-byte
// aligned).  Longer inputs are scanned in one chained pass whose bounded waits set
// kErrTimeout in *err (device word; NULL: a word of `partials`).
size_t scan_partials_size(int64_t n);
cudaError_t launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                                  uint32_t *partials, cudaStream_t st, uint32_t *err = nullptr);

// Stable LSD radix sort of (key, value) pairs on key bits [begin_bit, end_bit), or of keys
// alone (vals NULL: the keys are always written).
// keys[0]/vals[0] hold the input; the sorted output ends in buffer *out_buf.
// n_dev: optional device count (<= n_max) read by the kernels; n_max sizes the grid.
// keys_out = false: the last pass writes only the values (the sorted keys are not kept).
// Buffers must hold n_max rounded up to 4 elements (tiles are copied in 16-byte units).
// A bounded wait that runs out sets kErrTimeout in *err (device word).
// Segmented mode (seg_block0 != NULL, device array of n_seg + 1 block indices in units
// of radix_tile_keys(keys only)): every segment is sorted on its own and stays in place; the last
// pass leaves its scanned per-block digit counts at the start of `scratch`, segment-major
// and digit-major within a segment (digit d of the segment with first block b0 and nb
// blocks starts at scratch[256 b0 + d nb]; gc_bucket.cuh reads tile ranges from them).
size_t radix_scratch_words(int64_t n_max);
// Keys per radix tile: of a sort of (key, value) pairs, or of a keys-only sort (which
// segmented callers pad their segments to).
int radix_tile_keys(bool keys_only = false);
// scratch: radix_scratch_words(n_max) words, 8-byte aligned (the segmented mode keeps a
// per-block table of count-array bases and strides there).
cudaError_t radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max,
                             const uint32_t *n_dev, int end_bit, uint32_t *scratch, int *out_buf,
                             cudaStream_t st, uint32_t *err, bool keys_out = true,
                             const uint32_t *seg_block0 = nullptr, int n_seg = 0, int begin_bit = 0);

// Emit (tile key, rank) for every tile of every row interval of every visible Gaussian,
// in rank order (image W x H).  Entries at positions >= cap are dropped (fixed-capacity
// mode reports the overflow).
cudaError_t launch_emit(const float4 *ranked, const uint32_t *offsets, const uint32_t *touched_r,
                        int64_t n, const RenderParams &rp, int W, int H, uint32_t *keys, uint32_t *vals,
                        uint32_t cap, cudaStream_t st, const uint32_t *total = nullptr,
                        uint32_t *peak = nullptr);

// Binning by tile row (gc_bucket.cu), for images of at most 255 tile columns and at most
// 2^24 selected Gaussians (bucket_binning_fits): the entries placed straight into per-row
// segments padded to whole radix tiles as one word each, column << 24 | rank
// (launch_bucket_place: words[3] = padded total, shift[row] = padded minus unpadded start of
// the row, more than `cap` entries recorded in *peak and nothing placed); one segmented stable
// pass on the column byte (launch_bucket_sort: the sorted words are the tile lists, in
// keys[*out_buf]); tile ranges from its digit counts (launch_bucket_ranges; ranges must be
// zeroed).  Buffers hold `alloc` >= entries + rows x radix_tile_keys(true) words; `scratch` needs
// bucket_scratch_words.
bool bucket_binning_fits(const RenderParams &rp, int64_t n_sel);
size_t bucket_scratch_words(int64_t n, int n_rows);
cudaError_t launch_bucket_place(const float4 *ranked, const uint32_t *total, const uint32_t *touched_r, int64_t n,
                                const RenderParams &rp, int W, int H, uint32_t *keys, uint32_t cap,
                                uint32_t alloc, uint32_t *words, uint32_t *shift, uint32_t *scratch, uint32_t *peak,
                                cudaStream_t st);
cudaError_t launch_bucket_sort(uint32_t *keys[2], uint32_t alloc, uint32_t *words, int64_t n,
                               int n_rows, uint32_t *scratch, uint32_t *sort_scratch, int *out_buf, cudaStream_t st);
cudaError_t launch_bucket_ranges(int64_t n, uint32_t *scratch, uint32_t *sort_scratch, const RenderParams &rp,
                                 uint2 *ranges, cudaStream_t st);
// Unpadded tile lists of a row-binned state: ranges (int32 pairs) and global indices.
cudaError_t launch_row_lists_export(const uint2 *ranges, const uint32_t *sorted_vals, const uint32_t *shift,
                                    const RenderParams &rp, const uint32_t *perm, const Selection &sel,
                                    int32_t *out_ranges, int64_t *out_ids, cudaStream_t st);

// Tile ranges [start, end) from sorted tile keys; ranges must be zeroed.
cudaError_t launch_tile_ranges(const uint32_t *keys, const uint32_t *n_dev, int64_t n_max,
                               uint2 *ranges, cudaStream_t st);

// Front-to-back blend, one CTA per tile.  Per pixel: final transmittance, list
// position after the last blended entry, number blended, number of entries walked.
cudaError_t launch_blend_fwd(const uint2 *ranges, const uint32_t *sorted_vals,
                             const float4 *ranked, const CamParams &cam, const RenderParams &rp,
                             float *image, float *final_T, uint32_t *n_contrib,
                             uint32_t *n_blended, uint32_t *n_walked, cudaStream_t st);

// Multi-level blends (levels 1..L of one view from one list): per-level images, final
// transmittances lv_T[l * H * W + p] and list positions lv_last; the reverse pass writes
// the partials of every entry summed over the levels (layout and flags of launch_blend_bwd).
cudaError_t launch_blend_levels_fwd(const uint2 *ranges, const uint32_t *sorted_vals, const float4 *ranked,
                                    const CamParams &cam, const RenderParams &rp, int L, const LevelPtrs &out,
                                    float *lv_T, uint32_t *lv_last, cudaStream_t st);
cudaError_t launch_blend_levels_bwd(const uint2 *ranges, const uint32_t *sorted_vals, const float4 *ranked,
                                    const uint32_t *offsets, const CamParams &cam, const RenderParams &rp, int L,
                                    const float *lv_T, const uint32_t *lv_last, const LevelGrads &dimg,
                                    float *part, uint8_t *flag, cudaStream_t st);

// sorted list entry (rank) -> global Gaussian index, int64
cudaError_t launch_entries_to_global(const uint32_t *sorted_vals, const uint32_t *perm,
                                     const Selection &sel, int64_t K, int64_t *out,
                                     cudaStream_t st);

// ---- backward ----

// Reverse compositing per tile; writes 9 partial gradients per (tile, Gaussian)
// entry at the entry's emit position e = offsets[r] + (index of the tile among the
// Gaussian's row intervals): part[9 * e + c], c = du, dv, da, db, dc, dopacity,
// dr, dg, db.  Entries behind every pixel's last blended one are not written: the
// buffer must hold zeros there (the reduce leaves it all zero).  flag (one byte per entry,
// all zero on entry, or NULL): only nonzero partials are stored, and their entries' flags
// set to 1.
cudaError_t launch_blend_bwd(const uint2 *ranges, const uint32_t *sorted_vals,
                             const float4 *ranked, const uint32_t *offsets, const CamParams &cam,
                             const RenderParams &rp, const float *final_T,
                             const uint32_t *n_contrib, const float *dL_dimg, float *part, uint8_t *flag,
                             cudaStream_t st);

// Per-rank sum of the partials over the Gaussian's entries -> g2d[9 * j + c] at the
// Gaussian's compact position j = perm[r]; zeroes the partials it read (all of them
// nonzero are reset, so the buffer is all zero afterwards).  cap: buffer capacity in
// entries (Gaussians whose entries pass it contribute zero).  flag (the reverse pass's, or
// NULL): only flagged entries are read, and their flags cleared.
cudaError_t launch_reduce_entries(float *part, const uint32_t *offsets, const uint32_t *touched_r,
                                  const uint32_t *perm, int64_t n, uint32_t cap, uint8_t *flag, float *g2d,
                                  cudaStream_t st);

// Chain rule from the 2D gradients (by compact position) to the attributes (by
// global index) and to per-Gaussian motion terms (7 floats per compact position:
// dq_g[4], dt_g[3]).  touched[j] != 0 marks visible Gaussians.
cudaError_t launch_preprocess_bwd(const GaussSrc &g, const Selection &sel, int64_t n_sel,
                                  const CamParams &cam, const RenderParams &rp, const float *g2d,
                                  const uint32_t *touched, gc_grads out, float *motion_contrib,
                                  cudaStream_t st);

// Deterministic per-group sums of the motion terms.  `partial` needs
// group_partial_floats(n_sel, n_groups) floats.
size_t group_partial_floats(int64_t n_sel, int n_groups);
cudaError_t launch_motion_scatter(const float *motion_contrib, const Selection &sel, int64_t n_sel, float *d_q,
                                  float *d_t, cudaStream_t st);
cudaError_t launch_group_reduce(const float *motion_contrib, const int32_t *group_id,
                                const Selection &sel, int64_t n_sel, int n_groups, float *partial,
                                float *d_group_q, float *d_group_t, cudaStream_t st);

}  // namespace gc
