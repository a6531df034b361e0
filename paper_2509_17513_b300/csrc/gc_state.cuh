// gc_state.cuh - host-side state of the C ABI: library-owned device buffers, the
// context, saved forward states, error reporting and the stage profiler.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "gc_internal.cuh"

struct BatchState;  // gc_batch.cu
struct gc_saved;
gc_status batch_check(gc_context *ctx, const gc_saved &S, cudaStream_t stream);  // gc_batch.cu: errors of a batched forward (synchronises stream)
void batch_invalidate(gc_saved &S);                        // gc_batch.cu: a single-frame forward replaced it

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

inline cudaError_t grow(DevBuf &b, size_t bytes) {
    if (bytes <= b.cap && b.p) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t c = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(&b.p, c);
    if (e != cudaSuccess) {
        b.p = nullptr;
        cudaGetLastError();
        return e;
    }
    b.cap = c;
    return cudaSuccess;
}

inline void release(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

inline int ilog2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return ((1 << l) == v) ? l : -1;
}

inline int bits_for(int64_t max_value) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) <= max_value) ++b;
    return b;
}

struct gc_saved {
    std::shared_ptr<BatchState> batch;  // batched forward state (gc_batch.cu)
    bool valid = false;
    int64_t n = 0, n_sel = 0;
    int sh_degree = 0, n_groups = 1;
    bool has_motion = false;
    int per_gaussian = 0;
    gc::Residual res{nullptr, nullptr, nullptr};  // residual arrays of the forward
    int n_layers = 0;
    int64_t layer_offsets[gc::kMaxLayers + 1] = {};
    uint32_t layer_mask = 0;
    gc::Selection sel{};
    gc::CamParams cam{};
    gc::RenderParams rp{};
    int64_t K = 0;       // keys used (host view; fixed-capacity mode: the capacity)
    bool k_exact = false;
    int depth_buf = 0, tile_buf = 0;
    DevBuf rec, ranked, dkeys[2], dvals[2], touched, touched_r, offsets, tkeys[2], tvals[2], ranges,
        final_T, n_contrib, n_blended, n_walked, words;
    int levels = 0;         // > 0: a multi-level forward of levels 1..levels
    DevBuf lv_T, lv_last;   // its per-level final transmittance and list position
    bool row_binned = false;  // lists binned by tile row: row segments padded to radix tiles
    DevBuf row_shift;         // per tile row: padded minus unpadded start of its segment
    // Working memory of this state's forward (scan and sort scratch) and backward (per-entry
    // partials, per-Gaussian screen-space and motion gradients, group partials): owned by the
    // state, so that distinct states may run on different streams at once.  The backward's
    // buffers are scratch, not results (mutable: a backward reads a const state).
    DevBuf scratch;
    mutable DevBuf bwd_part, bwd_flag, bwd_g2d, bwd_motion, bwd_group;
    // bwd_part holds only zeros and bwd_flag (one byte per entry) too (see the reduce)
    mutable bool bwd_part_clean = false;
    // The sorted tile lists: the keys buffer of the last pass for row-binned lists (one word
    // per entry, column << 24 | rank), else the values of the key sort.
    uint32_t *lists() const {
        return row_binned ? tkeys[tile_buf].as<uint32_t>() : tvals[tile_buf].as<uint32_t>();
    }
};


struct ProfMark {
    int stage;     // -1: end of a call
    int ev_end;    // event closing the previous stage (index into the event pool)
    int ev_start;  // event opening this stage: ev_end, or the event after the L2 flush
};

struct gc_context {
    int device = 0;
    bool prof_on = false;
    bool prof_flush_on = false;     // flush L2 before each stage (outside its events)
    DevBuf prof_flush;              // the buffer written to flush L2
    std::vector<cudaEvent_t> prof_pool;
    std::vector<ProfMark> prof_marks;
    int prof_used = 0;              // events of the pool recorded since the last read
    uint64_t launch_base = 0;
    gc_options opt{};
    gc_saved internal;
    DevBuf field_part;              // per-block partial gradients of the motion source
    DevBuf field_h;                 // hash-grid encodings of the motion source (backward)
    DevBuf kde_scratch;             // KDE training form: histograms, bandwidths, partial sums
    DevBuf loss_part;               // L1 loss: one FP64 partial sum per CTA
    uint32_t *host_word = nullptr;  // pinned
    const gc_saved *last = nullptr; // state written by the most recent forward
    std::string err;
};

inline gc_status fail(gc_context *ctx, gc_status s, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

#define GC_CUDA(ctx, call)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA,    \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Records a stage boundary on the stream when profiling is on.
// GC_ERR_CAPACITY if a forward on S since the last check needed more keys than its fixed
// capacity (synchronises `stream`, the stream of those forwards; S must have a fixed capacity).
gc_status capacity_check(gc_context *ctx, const gc_saved &S, cudaStream_t stream);
// gc_render_levels_backward whose writes into `out` wait for order_wait and are followed by a
// record of order_done (either may be NULL); the reverse blend and reduce before them do not
// wait (gc_api.cu; used by the multi-frame graphs to keep shared gradient sets in frame order).
gc_status levels_backward_ordered(gc_context *ctx, const gc_saved *saved, const gc_gaussians *g,
                                  const gc_motion *motion, const float *const *dL_dimages, gc_grads *out,
                                  cudaStream_t stream, cudaEvent_t order_wait, cudaEvent_t order_done);

inline cudaError_t prof_event(gc_context *ctx, cudaStream_t s, int &idx) {
    idx = ctx->prof_used;
    if ((size_t)idx >= ctx->prof_pool.size()) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        ctx->prof_pool.push_back(e);
    }
    ctx->prof_used++;
    return cudaEventRecord(ctx->prof_pool[idx], s);
}

// With the flush on, a stage boundary records the end of the previous stage, writes the
// flush buffer (larger than L2) and records the start of the next stage after it, so that
// each stage starts with its inputs in HBM and its time excludes the flush.
inline cudaError_t prof_mark(gc_context *ctx, cudaStream_t s, int stage) {
    if (!ctx->prof_on) return cudaSuccess;
    int e0 = 0, e1 = 0;
    cudaError_t err = prof_event(ctx, s, e0);
    if (err != cudaSuccess) return err;
    e1 = e0;
    if (ctx->prof_flush_on && stage >= 0 && ctx->prof_flush.p) {
        err = cudaMemsetAsync(ctx->prof_flush.p, (int)(ctx->prof_marks.size() & 0x7f), ctx->prof_flush.cap, s);
        if (err != cudaSuccess) return err;
        err = prof_event(ctx, s, e1);
        if (err != cudaSuccess) return err;
    }
    ctx->prof_marks.push_back({stage, e0, e1});
    return cudaSuccess;
}

inline gc_status check_options(gc_context *ctx, const gc_options *o) {
    bool shape_ok = (o->tile_w == 16 && o->tile_h == 16) || (o->tile_w == 8 && o->tile_h == 32) ||
                    (o->tile_w == 32 && o->tile_h == 8);
    if (!shape_ok) return fail(ctx, GC_ERR_INVALID_ARG, "tile shape %dx%d not in {16x16, 8x32, 32x8}", o->tile_w, o->tile_h);
    if (!(o->near_plane > 0.f)) return fail(ctx, GC_ERR_INVALID_ARG, "near_plane must be > 0");
    if (!(o->dilation >= 0.f)) return fail(ctx, GC_ERR_INVALID_ARG, "dilation must be >= 0");
    if (!(o->frustum_clamp > 0.f)) return fail(ctx, GC_ERR_INVALID_ARG, "frustum_clamp must be > 0");
    if (o->membership != GC_MEMBER_PIXEL && o->membership != GC_MEMBER_TILE)
        return fail(ctx, GC_ERR_INVALID_ARG, "membership must be GC_MEMBER_PIXEL or GC_MEMBER_TILE");
    if (o->key_capacity < 0 || o->key_capacity > 0xFFFFFFF0ll)
        return fail(ctx, GC_ERR_INVALID_ARG, "key_capacity out of range");
    if (o->alpha_cull != 0 && o->alpha_cull != 1) return fail(ctx, GC_ERR_INVALID_ARG, "alpha_cull must be 0 or 1");
    return GC_OK;
}

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
        dev_ = dev;
    }
    ~DeviceGuard() {
        if (prev_ != dev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0, dev_ = 0;
};

inline gc_status make_source(gc_context *ctx, const gc_gaussians *g, const gc_motion *m, gc::GaussSrc &s) {
    if (!g) return fail(ctx, GC_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0) return fail(ctx, GC_ERR_INVALID_ARG, "n < 0");
    if (g->n > 0x7FFFFFFFll) return fail(ctx, GC_ERR_INVALID_ARG, "n exceeds 2^31 - 1");
    if (g->sh_degree < 0 || g->sh_degree > 3) return fail(ctx, GC_ERR_INVALID_ARG, "sh_degree must be 0..3");
    if (g->n_layers < 1 || g->n_layers > gc::kMaxLayers)
        return fail(ctx, GC_ERR_INVALID_ARG, "n_layers must be 1..32");
    if (!g->layer_offsets) return fail(ctx, GC_ERR_INVALID_ARG, "layer_offsets is NULL");
    if (g->layer_offsets[0] != 0 || g->layer_offsets[g->n_layers] != g->n)
        return fail(ctx, GC_ERR_INVALID_ARG, "layer_offsets must start at 0 and end at n");
    for (int l = 0; l < g->n_layers; ++l)
        if (g->layer_offsets[l + 1] < g->layer_offsets[l])
            return fail(ctx, GC_ERR_INVALID_ARG, "layer_offsets must be nondecreasing");
    memset(&s, 0, sizeof s);
    s.n = g->n;
    s.sh_degree = g->sh_degree;
    s.K = (g->sh_degree + 1) * (g->sh_degree + 1);
    s.precision = g->precision;
    if (g->precision == GC_PREC_FP32) {
        if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
            return fail(ctx, GC_ERR_INVALID_ARG, "an FP32 attribute array is NULL");
    } else if (g->precision == GC_PREC_BF16_FP8) {
        if (g->n > 0 && (!g->means_bf16 || !g->log_scales_bf16 || !g->quats_bf16 ||
                         !g->opacity_bf16 || !g->sh_e4m3 || !g->scales))
            return fail(ctx, GC_ERR_INVALID_ARG, "a reduced-precision plane or the scales are NULL");
    } else if (g->precision == GC_PREC_PLANES) {
        if (g->plane_width < 1) return fail(ctx, GC_ERR_INVALID_ARG, "plane_width must be >= 1");
        if (g->pos_bits != 16 && g->pos_bits != 32) return fail(ctx, GC_ERR_INVALID_ARG, "pos_bits must be 16 or 32");
        const int pb = g->pos_bits / 8;
        if (g->plane_pitch < g->plane_width || g->pos_pitch < (int64_t)g->plane_width * pb || g->pos_pitch % pb)
            return fail(ctx, GC_ERR_INVALID_ARG, "plane pitches too small or misaligned");
        if (g->n > 0 && (!g->planes_u8 || !g->planes_pos || !g->dequant))
            return fail(ctx, GC_ERR_INVALID_ARG, "the decoded planes or the dequantisation table are NULL");
        for (int l = 0; l < g->n_layers; ++l) {
            if (g->layer_offsets[l + 1] == g->layer_offsets[l]) continue;
            if (g->layer_offsets[l + 1] - g->layer_offsets[l] > 0x7FFFFFFFll)
                return fail(ctx, GC_ERR_INVALID_ARG, "a layer holds more than 2^31 - 1 Gaussians");
            if (!g->planes_u8[l] || !g->planes_pos[l])
                return fail(ctx, GC_ERR_INVALID_ARG, "the planes of layer %d are NULL", l);
            if (reinterpret_cast<uintptr_t>(g->planes_pos[l]) % pb)
                return fail(ctx, GC_ERR_INVALID_ARG, "the position planes of layer %d are misaligned", l);
        }
    } else {
        return fail(ctx, GC_ERR_INVALID_ARG, "unknown precision %d", g->precision);
    }
    s.means = g->means; s.log_scales = g->log_scales; s.quats = g->quats;
    s.opacity_logits = g->opacity_logits; s.sh = g->sh; s.group_id = g->group_id;
    s.means_h = g->means_bf16; s.log_scales_h = g->log_scales_bf16; s.quats_h = g->quats_bf16;
    s.opacity_h = g->opacity_bf16; s.sh_q = g->sh_e4m3; s.scales = g->scales;
    s.n_layers = g->n_layers;
    for (int l = 0; l <= g->n_layers; ++l) s.layer_off[l] = g->layer_offsets[l];
    if (g->precision == GC_PREC_PLANES) {
        s.plane_width = g->plane_width;
        s.pos_bits = g->pos_bits;
        s.n_channels = 11 + 3 * s.K;
        s.plane_pitch = g->plane_pitch;
        s.pos_pitch = g->pos_pitch;
        s.dequant = g->dequant;
        for (int l = 0; l < g->n_layers; ++l) {
            s.plane_u8[l] = g->planes_u8 ? g->planes_u8[l] : nullptr;
            s.plane_pos[l] = g->planes_pos ? static_cast<const uint8_t *>(g->planes_pos[l]) : nullptr;
        }
    }
    s.n_groups = 1;
    if (m && m->per_gaussian) {
        if (!m->q || !m->t) return fail(ctx, GC_ERR_INVALID_ARG, "per-Gaussian motion needs q and t arrays");
        s.group_q = m->q;
        s.group_t = m->t;
        s.n_groups = (int)std::max<int64_t>(g->n, 1);
        s.per_gaussian = 1;
        s.group_id = nullptr;
    } else if (m && (m->q || m->t)) {
        if (m->n_groups < 1 || !m->q || !m->t)
            return fail(ctx, GC_ERR_INVALID_ARG, "motion needs n_groups >= 1 and both q and t arrays");
        s.group_q = m->q;
        s.group_t = m->t;
        s.n_groups = m->n_groups;
    } else if (g->group_id) {
        s.group_id = nullptr;  // keyframe: groups are irrelevant
    }
    if (m) {
        if (m->res_sh && s.K == 16 && (reinterpret_cast<uintptr_t>(m->res_sh) & 15))
            return fail(ctx, GC_ERR_INVALID_ARG, "res_sh must be 16-byte aligned");
        s.res = gc::Residual{m->res_log_scales, m->res_opacity_logits, m->res_sh};
    }
    return GC_OK;
}

inline gc::Selection make_selection(const gc_gaussians *g, uint32_t mask, int64_t &n_sel) {
    gc::Selection s{};
    n_sel = 0;
    s.n_layers = g->n_layers;
    for (int l = 0; l <= g->n_layers; ++l) s.layer_off[l] = g->layer_offsets[l];
    s.range_start[0] = 0;
    for (int l = 0; l < g->n_layers; ++l) {
        if (!((mask >> l) & 1u)) continue;
        int64_t a = g->layer_offsets[l], b = g->layer_offsets[l + 1];
        if (b <= a) continue;
        // merge adjacent ranges
        if (s.n_ranges > 0 && s.range_begin[s.n_ranges - 1] + (s.range_start[s.n_ranges] - s.range_start[s.n_ranges - 1]) == a) {
            s.range_start[s.n_ranges] += b - a;
        } else {
            s.range_begin[s.n_ranges] = a;
            s.range_start[s.n_ranges + 1] = s.range_start[s.n_ranges] + (b - a);
            s.n_ranges++;
        }
        n_sel += b - a;
    }
    if (s.n_ranges == 0) s.n_ranges = 1;
    return s;
}
