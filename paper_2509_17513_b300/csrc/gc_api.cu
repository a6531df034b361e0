// gc_api.cu - the C ABI (include/gc4d.h): context, library-owned scratch and the
// orchestration of one frame on the caller's stream.
//
// Forward, one frame (all on `stream`):
//   preprocess (motion + projection + footprint + colour, per selected Gaussian)
//   -> depth sort (32-bit depth keys, stable over index order)
//   -> rank gather (records into depth order) -> exclusive scan of tiles touched
//   -> [key count: one 4-byte device->host read unless the capacity is fixed]
//   -> emit (tile, rank) entries -> stable tile sort -> tile ranges -> blend.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gc_internal.cuh"

#include "gc_state.cuh"

namespace gc {
static std::atomic<uint64_t> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }
uint64_t launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace gc


extern "C" {

const char *gc_version(void) { return "gc4d 0.1 (sm_103a)"; }

gc_status gc_default_options(gc_options *o) {
    if (!o) return GC_ERR_INVALID_ARG;
    memset(o, 0, sizeof *o);
    o->tile_w = 16;
    o->tile_h = 16;
    o->near_plane = 0.2f;
    o->dilation = 0.3f;
    o->frustum_clamp = 1.3f;
    o->membership = GC_MEMBER_PIXEL;
    o->key_capacity = 0;
    o->alpha_cull = 1;
    return GC_OK;
}

gc_status gc_create(gc_context **out, int device, const gc_options *opt) {
    if (!out) return GC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GC_ERR_INVALID_ARG;
    }
    gc_context *ctx = new (std::nothrow) gc_context();
    if (!ctx) return GC_ERR_OOM;
    ctx->device = device;
    gc_default_options(&ctx->opt);
    if (opt) {
        gc_status s = check_options(ctx, opt);
        if (s != GC_OK) {
            delete ctx;
            return s;
        }
        ctx->opt = *opt;
    }
    DeviceGuard dg(device);
    if (cudaHostAlloc(&ctx->host_word, 64, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GC_ERR_OOM;
    }
    *out = ctx;
    return GC_OK;
}

static void saved_release(gc_context *ctx, gc_saved *s) {
    if (ctx && ctx->last == s) ctx->last = nullptr;
    DevBuf *bufs[] = {&s->rec, &s->ranked, &s->dkeys[0], &s->dkeys[1], &s->dvals[0], &s->dvals[1],
                      &s->touched, &s->touched_r, &s->offsets, &s->tkeys[0], &s->tkeys[1],
                      &s->tvals[0], &s->tvals[1], &s->ranges, &s->final_T, &s->n_contrib,
                      &s->n_blended, &s->n_walked, &s->words, &s->lv_T, &s->lv_last, &s->row_shift,
                      &s->scratch, &s->bwd_part, &s->bwd_flag, &s->bwd_g2d, &s->bwd_motion, &s->bwd_group};
    for (DevBuf *b : bufs) release(*b);
    s->valid = false;
}

gc_status gc_destroy(gc_context *ctx) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    {
        DeviceGuard dg(ctx->device);
        saved_release(ctx, &ctx->internal);
        ctx->internal.batch.reset();
        DevBuf *bufs[] = {&ctx->field_part, &ctx->field_h, &ctx->kde_scratch, &ctx->prof_flush,
                          &ctx->loss_part};
        for (DevBuf *b : bufs) release(*b);
        if (ctx->host_word) cudaFreeHost(ctx->host_word);
        for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    }
    delete ctx;
    return GC_OK;
}

gc_status gc_set_options(gc_context *ctx, const gc_options *opt) {
    if (!ctx || !opt) return GC_ERR_INVALID_ARG;
    gc_status s = check_options(ctx, opt);
    if (s != GC_OK) return s;
    ctx->opt = *opt;
    return GC_OK;
}

gc_status gc_saved_create(gc_context *ctx, gc_saved **out) {
    if (!ctx || !out) return GC_ERR_INVALID_ARG;
    *out = new (std::nothrow) gc_saved();
    return *out ? GC_OK : GC_ERR_OOM;
}

gc_status gc_saved_destroy(gc_context *ctx, gc_saved *saved) {
    if (!ctx || !saved) return GC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    saved_release(ctx, saved);
    delete saved;
    return GC_OK;
}

const char *gc_last_error(gc_context *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

}  // extern "C"

// One view: layer_mask selects the layers (levels = 0) or, for levels L > 0, the layers
// 1..L rendered as L images at once (level_images[0..L-1]).
static gc_status render_forward_impl(gc_context *ctx, const gc_gaussians *g, const gc_motion *motion,
                                     uint32_t layer_mask, const gc_camera *cam, float *image, gc_saved *saved,
                                     void *stream, int levels, float *const *level_images) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!cam || (!image && !levels)) return fail(ctx, GC_ERR_INVALID_ARG, "camera or image is NULL");
    if (cam->width <= 0 || cam->height <= 0 || cam->width > 32768 || cam->height > 32768)
        return fail(ctx, GC_ERR_INVALID_ARG, "image size %dx%d out of range (1..32768)", cam->width, cam->height);
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f)) return fail(ctx, GC_ERR_INVALID_ARG, "fx, fy must be > 0");
    gc::GaussSrc src;
    gc_status st = make_source(ctx, g, motion, src);
    if (st != GC_OK) return st;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gc_saved &S = saved ? *saved : ctx->internal;
    S.valid = false;
    if (S.batch) batch_invalidate(S);
    if (levels) {
        if (levels < 1 || levels > gc::kMaxLevels || levels > g->n_layers)
            return fail(ctx, GC_ERR_INVALID_ARG, "levels must be 1..min(8, n_layers)");
        for (int l = 0; l < levels; ++l)
            if (!level_images[l]) return fail(ctx, GC_ERR_INVALID_ARG, "level image %d is NULL", l);
        layer_mask = (1u << levels) - 1u;
    }
    S.levels = levels;

    const gc_options &o = ctx->opt;
    int64_t n_sel = 0;
    S.sel = make_selection(g, layer_mask, n_sel);
    S.n = g->n;
    S.n_sel = n_sel;
    S.sh_degree = g->sh_degree;
    S.n_groups = src.n_groups;
    S.has_motion = src.group_q != nullptr;
    S.per_gaussian = src.per_gaussian;
    S.res = src.res;
    S.n_layers = g->n_layers;
    for (int l = 0; l <= g->n_layers; ++l) S.layer_offsets[l] = g->layer_offsets[l];
    S.layer_mask = layer_mask;
    gc::CamParams &cp = S.cam;
    cp.width = cam->width; cp.height = cam->height;
    cp.fx = cam->fx; cp.fy = cam->fy; cp.cx = cam->cx; cp.cy = cam->cy;
    memcpy(cp.R, cam->R, sizeof cp.R);
    memcpy(cp.t, cam->t, sizeof cp.t);
    memcpy(cp.campos, cam->campos, sizeof cp.campos);
    gc::RenderParams &rp = S.rp;
    rp.near_plane = o.near_plane; rp.dilation = o.dilation; rp.frustum_clamp = o.frustum_clamp;
    memcpy(rp.bg, o.bg, sizeof rp.bg);
    rp.tile_w = o.tile_w; rp.tile_h = o.tile_h;
    rp.tile_w_log2 = ilog2_exact(o.tile_w); rp.tile_h_log2 = ilog2_exact(o.tile_h);
    rp.ntx = (cam->width + o.tile_w - 1) / o.tile_w;
    rp.nty = (cam->height + o.tile_h - 1) / o.tile_h;
    rp.membership = o.membership;
    rp.alpha_cull = o.alpha_cull;
    rp.list_packed = 0;  // set below when the lists are binned by tile row
    const int64_t n_tiles = (int64_t)rp.ntx * rp.nty;
    const int64_t hw = (int64_t)cam->width * cam->height;

    // per-frame buffers sized by the selection and the image
    const int64_t nn = n_sel > 0 ? n_sel : 1;
    GC_CUDA(ctx, grow(S.rec, (size_t)nn * 16 * gc::kRec));
    GC_CUDA(ctx, grow(S.ranked, (size_t)nn * 16 * gc::kRec));
    for (int b = 0; b < 2; ++b) {
        GC_CUDA(ctx, grow(S.dkeys[b], (size_t)nn * 4));
        GC_CUDA(ctx, grow(S.dvals[b], (size_t)nn * 4));
    }
    GC_CUDA(ctx, grow(S.touched, (size_t)nn * 4));
    GC_CUDA(ctx, grow(S.touched_r, (size_t)nn * 4));
    GC_CUDA(ctx, grow(S.offsets, (size_t)(nn + 1) * 4));
    GC_CUDA(ctx, grow(S.ranges, (size_t)n_tiles * 8));
    GC_CUDA(ctx, grow(S.final_T, (size_t)hw * 4));
    GC_CUDA(ctx, grow(S.n_contrib, (size_t)hw * 4));
    GC_CUDA(ctx, grow(S.n_blended, (size_t)hw * 4));
    GC_CUDA(ctx, grow(S.n_walked, (size_t)hw * 4));
    if (!S.words.p) {
        GC_CUDA(ctx, grow(S.words, 64));
        GC_CUDA(ctx, cudaMemsetAsync(S.words.p, 0, 64, s));
    }
    // Tile ranges come from the sorted keys (the last sort pass keeps them): counting entries
    // per tile with a difference grid filled by the preprocess costs ~2.4M contended integer
    // atomics on a few thousand cells per 1080p frame, measured slower than one pass over the
    // sorted keys.
    const int64_t cap_fixed = o.key_capacity;
    const size_t scan_words = gc::scan_partials_size(nn);

    GC_CUDA(ctx, cudaMemsetAsync(S.ranges.p, 0, (size_t)n_tiles * 8, s));
    uint32_t *words = S.words.as<uint32_t>();  // [0] = K, [1] = error flags
    int64_t K = 0;
    if (n_sel > 0) {
        GC_CUDA(ctx, grow(S.scratch, 4 * std::max(gc::radix_scratch_words(nn), scan_words)));
        uint32_t *scratch = S.scratch.as<uint32_t>();
        GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_PREPROCESS));
        GC_CUDA(ctx, gc::launch_preprocess(src, S.sel, n_sel, cp, rp, S.rec.as<float4>(),
                                           S.dkeys[0].as<uint32_t>(), S.dvals[0].as<uint32_t>(),
                                           S.touched.as<uint32_t>(), s));
        uint32_t *dk[2] = {S.dkeys[0].as<uint32_t>(), S.dkeys[1].as<uint32_t>()};
        uint32_t *dv[2] = {S.dvals[0].as<uint32_t>(), S.dvals[1].as<uint32_t>()};
        GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_DEPTH_SORT));
        GC_CUDA(ctx, gc::radix_sort_pairs(dk, dv, n_sel, nullptr, 32, scratch, &S.depth_buf, s, words + 1));
        GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_SCAN));
        GC_CUDA(ctx, gc::launch_rank_gather(dv[S.depth_buf], S.rec.as<float4>(),
                                            S.touched.as<uint32_t>(), n_sel, S.ranked.as<float4>(),
                                            S.touched_r.as<uint32_t>(), s));
        GC_CUDA(ctx, gc::launch_exclusive_scan(S.touched_r.as<uint32_t>(), S.offsets.as<uint32_t>(),
                                               n_sel, words, scratch, s, words + 1));
        if (cap_fixed > 0) {
            K = cap_fixed;
            S.k_exact = false;
        } else {
            GC_CUDA(ctx, cudaMemcpyAsync(ctx->host_word, words, 4, cudaMemcpyDeviceToHost, s));
            GC_CUDA(ctx, cudaStreamSynchronize(s));
            K = (int64_t)ctx->host_word[0];
            S.k_exact = true;
        }
        const int64_t kk = K > 0 ? K : 1;
        // binning by tile row pads every row's segment to whole radix tiles: room for that
        // beyond the entries (the capacity counts entries only)
        const int64_t kpad = (kk + (int64_t)rp.nty * gc::radix_tile_keys(true) + 3) & ~int64_t(3);
        const bool rows = gc::bucket_binning_fits(rp, n_sel) && kpad <= 0xFFFFFFF0ll;
        const int64_t kalloc = rows ? kpad : kk;
        for (int b = 0; b < 2; ++b) {
            GC_CUDA(ctx, grow(S.tkeys[b], (size_t)kalloc * 4));
            if (!rows) GC_CUDA(ctx, grow(S.tvals[b], (size_t)kalloc * 4));  // row-binned lists: one word per entry
        }
        const size_t bucket_words = rows ? ((gc::bucket_scratch_words(n_sel, rp.nty) + 63) & ~size_t(63)) : 0;
        GC_CUDA(ctx, grow(S.scratch, 4 * (bucket_words + std::max(gc::radix_scratch_words(kalloc), scan_words))));
        scratch = S.scratch.as<uint32_t>();
        S.row_binned = false;
        if (K > 0) {
            uint32_t *tk[2] = {S.tkeys[0].as<uint32_t>(), S.tkeys[1].as<uint32_t>()};
            uint32_t *tv[2] = {S.tvals[0].as<uint32_t>(), S.tvals[1].as<uint32_t>()};
            uint32_t *peak = S.k_exact ? nullptr : words + 2;
            GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_EMIT));
            if (rows) {
                GC_CUDA(ctx, grow(S.row_shift, (size_t)(rp.nty + 1) * 4));
                GC_CUDA(ctx, gc::launch_bucket_place(S.ranked.as<float4>(), words, S.touched_r.as<uint32_t>(), n_sel,
                                                     rp, cam->width, cam->height, tk[0],
                                                     (uint32_t)std::min<int64_t>(K, 0xFFFFFFFFll), (uint32_t)kalloc,
                                                     words, S.row_shift.as<uint32_t>(), scratch, peak, s));
                GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_TILE_SORT));
                GC_CUDA(ctx, gc::launch_bucket_sort(tk, (uint32_t)kalloc, words, n_sel, rp.nty, scratch,
                                                    scratch + bucket_words, &S.tile_buf, s));
                GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_RANGES));
                GC_CUDA(ctx, gc::launch_bucket_ranges(n_sel, scratch, scratch + bucket_words, rp,
                                                      S.ranges.as<uint2>(), s));
                S.row_binned = true;
                rp.list_packed = 1;
            } else {
                GC_CUDA(ctx, gc::launch_emit(S.ranked.as<float4>(), S.offsets.as<uint32_t>(),
                                             S.touched_r.as<uint32_t>(), n_sel, rp, cam->width, cam->height,
                                             tk[0], tv[0], (uint32_t)K, s, words, peak));
                const uint32_t *ndev = S.k_exact ? nullptr : words;
                GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_TILE_SORT));
                GC_CUDA(ctx, gc::radix_sort_pairs(tk, tv, K, ndev, bits_for(n_tiles - 1), scratch,
                                                  &S.tile_buf, s, words + 1, /*keys_out=*/true));
                GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_RANGES));
                GC_CUDA(ctx, gc::launch_tile_ranges(tk[S.tile_buf], ndev, K, S.ranges.as<uint2>(), s));
            }
        }
    } else {
        GC_CUDA(ctx, cudaMemsetAsync(words, 0, 4, s));
    }
    S.K = K;
    uint32_t *sorted_vals = (n_sel > 0 && K > 0) ? S.lists() : nullptr;
    GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_BLEND));
    if (levels) {
        GC_CUDA(ctx, grow(S.lv_T, (size_t)levels * hw * 4));
        GC_CUDA(ctx, grow(S.lv_last, (size_t)levels * hw * 4));
        gc::LevelPtrs lp{};
        for (int l = 0; l < levels; ++l) lp.img[l] = level_images[l];
        GC_CUDA(ctx, gc::launch_blend_levels_fwd(S.ranges.as<uint2>(), sorted_vals, S.ranked.as<float4>(), cp, rp,
                                                 levels, lp, S.lv_T.as<float>(), S.lv_last.as<uint32_t>(), s));
    } else {
        GC_CUDA(ctx, gc::launch_blend_fwd(S.ranges.as<uint2>(), sorted_vals, S.ranked.as<float4>(), cp, rp,
                                          image, S.final_T.as<float>(), S.n_contrib.as<uint32_t>(),
                                          S.n_blended.as<uint32_t>(), S.n_walked.as<uint32_t>(), s));
    }
    GC_CUDA(ctx, prof_mark(ctx, s, -1));
    S.valid = true;
    ctx->last = &S;
    return GC_OK;
}

// Fixed key capacity: word 2 holds the largest count of any forward on this state that
// overflowed the capacity it ran with since the last check (kept by the emit kernel), word 0
// the last forward's count; the record is then cleared on `stream`, ordered before the
// stream's next forwards.
gc_status capacity_check(gc_context *ctx, const gc_saved &S, cudaStream_t stream) {
    uint32_t w[3];
    GC_CUDA(ctx, cudaMemcpyAsync(w, S.words.p, 12, cudaMemcpyDeviceToHost, stream));
    GC_CUDA(ctx, cudaStreamSynchronize(stream));
    GC_CUDA(ctx, cudaMemsetAsync(static_cast<uint32_t *>(S.words.p) + 2, 0, 4, stream));
    if (w[2] != 0u)
        return fail(ctx, GC_ERR_CAPACITY, "a frame needed %u keys, more than its fixed capacity (now %lld)",
                    w[2], (long long)S.K);
    if ((int64_t)w[0] > S.K)
        return fail(ctx, GC_ERR_CAPACITY, "a frame needs %u keys, capacity %lld", w[0], (long long)S.K);
    return GC_OK;
}

extern "C" {

gc_status gc_render_forward(gc_context *ctx, const gc_gaussians *g, const gc_motion *motion,
                            uint32_t layer_mask, const gc_camera *cam, float *image,
                            gc_saved *saved, void *stream) {
    return render_forward_impl(ctx, g, motion, layer_mask, cam, image, saved, stream, 0, nullptr);
}

gc_status gc_render_levels_forward(gc_context *ctx, const gc_gaussians *g, const gc_motion *motion,
                                   int32_t levels, const gc_camera *cam, float *const *level_images,
                                   gc_saved *saved, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!level_images) return fail(ctx, GC_ERR_INVALID_ARG, "level_images is NULL");
    if (levels < 1) return fail(ctx, GC_ERR_INVALID_ARG, "levels must be >= 1");
    return render_forward_impl(ctx, g, motion, 0u, cam, nullptr, saved, stream, levels, level_images);
}

gc_status gc_saved_stats(gc_context *ctx, const gc_saved *saved, gc_stats *out, void *stream) {
    if (!ctx || !out) return GC_ERR_INVALID_ARG;
    const gc_saved &S = saved ? *saved : ctx->internal;
    if (!S.valid) return fail(ctx, GC_ERR_STATE, "no forward recorded");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    memset(out, 0, sizeof *out);
    out->n_selected = S.n_sel;
    out->n_tiles = S.rp.ntx * S.rp.nty;
    out->width = S.cam.width;
    out->height = S.cam.height;
    if (S.n_sel > 0) {
        GC_CUDA(ctx, cudaMemcpyAsync(ctx->host_word, S.words.p, 4, cudaMemcpyDeviceToHost, s));
        GC_CUDA(ctx, cudaStreamSynchronize(s));
        out->n_keys = ctx->host_word[0];
        // visible = number of depth keys below the culled sentinel: the sorted keys end with them
        uint32_t *keys = static_cast<uint32_t *>(S.dkeys[S.depth_buf].p);
        int64_t lo = 0, hi = S.n_sel;  // first index with key == culled
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            uint32_t k;
            GC_CUDA(ctx, cudaMemcpy(&k, keys + mid, 4, cudaMemcpyDeviceToHost));
            if (k == gc::kCulledKey) hi = mid; else lo = mid + 1;
        }
        out->n_visible = lo;
    }
    return GC_OK;
}

gc_status gc_saved_tile_lists(gc_context *ctx, const gc_saved *saved, int32_t *ranges,
                              int64_t *gauss_ids, int64_t capacity, void *stream) {
    if (!ctx || !ranges || !gauss_ids) return GC_ERR_INVALID_ARG;
    const gc_saved &S = saved ? *saved : ctx->internal;
    if (!S.valid) return fail(ctx, GC_ERR_STATE, "no forward recorded");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int64_t K = 0;
    if (S.n_sel > 0) {
        GC_CUDA(ctx, cudaMemcpyAsync(ctx->host_word, S.words.p, 4, cudaMemcpyDeviceToHost, s));
        GC_CUDA(ctx, cudaStreamSynchronize(s));
        K = std::min<int64_t>(ctx->host_word[0], S.K);
    }
    if (capacity < K) return fail(ctx, GC_ERR_CAPACITY, "tile lists need %lld entries", (long long)K);
    const int64_t n_tiles = (int64_t)S.rp.ntx * S.rp.nty;
    if (S.row_binned && K > 0) {  // row segments carry padding: export the lists without it
        GC_CUDA(ctx, gc::launch_row_lists_export(S.ranges.as<uint2>(), S.lists(),
                                                 S.row_shift.as<uint32_t>(), S.rp, S.dvals[S.depth_buf].as<uint32_t>(),
                                                 S.sel, ranges, gauss_ids, s));
    } else {
        GC_CUDA(ctx, cudaMemcpyAsync(ranges, S.ranges.p, (size_t)n_tiles * 8, cudaMemcpyDeviceToDevice, s));
        if (K > 0)
            GC_CUDA(ctx, gc::launch_entries_to_global(S.lists(),
                                                      S.dvals[S.depth_buf].as<uint32_t>(), S.sel, K,
                                                      gauss_ids, s));
    }
    GC_CUDA(ctx, cudaStreamSynchronize(s));
    return GC_OK;
}

gc_status gc_saved_pixel_state(gc_context *ctx, const gc_saved *saved, float *final_T,
                               int32_t *n_blended, int32_t *n_walked, int32_t *n_contrib,
                               void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    const gc_saved &S = saved ? *saved : ctx->internal;
    if (!S.valid) return fail(ctx, GC_ERR_STATE, "no forward recorded");
    if (S.levels) return fail(ctx, GC_ERR_STATE, "per-pixel state of a multi-level forward is not kept here");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    size_t hw = (size_t)S.cam.width * S.cam.height;
    if (final_T) GC_CUDA(ctx, cudaMemcpyAsync(final_T, S.final_T.p, hw * 4, cudaMemcpyDeviceToDevice, s));
    if (n_blended) GC_CUDA(ctx, cudaMemcpyAsync(n_blended, S.n_blended.p, hw * 4, cudaMemcpyDeviceToDevice, s));
    if (n_walked) GC_CUDA(ctx, cudaMemcpyAsync(n_walked, S.n_walked.p, hw * 4, cudaMemcpyDeviceToDevice, s));
    if (n_contrib) GC_CUDA(ctx, cudaMemcpyAsync(n_contrib, S.n_contrib.p, hw * 4, cudaMemcpyDeviceToDevice, s));
    return GC_OK;
}

gc_status gc_profile_enable(gc_context *ctx, int enable) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (enable < 0 || enable > 2) return fail(ctx, GC_ERR_INVALID_ARG, "profile mode must be 0, 1 or 2");
    if (enable == 2) {
        DeviceGuard dg(ctx->device);
        GC_CUDA(ctx, grow(ctx->prof_flush, (size_t)256 << 20));  // twice the 126 MB L2
    }
    ctx->prof_on = enable != 0;
    ctx->prof_flush_on = enable == 2;
    return GC_OK;
}

gc_status gc_profile_read(gc_context *ctx, double *stage_ms, int64_t *stage_calls,
                          uint64_t *kernel_launches) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    if (stage_ms) for (int k = 0; k < GC_N_STAGES; ++k) stage_ms[k] = 0.0;
    if (stage_calls) for (int k = 0; k < GC_N_STAGES; ++k) stage_calls[k] = 0;
    if (!ctx->prof_marks.empty()) {
        GC_CUDA(ctx, cudaEventSynchronize(ctx->prof_pool[ctx->prof_marks.back().ev_start]));
        for (size_t i = 0; i + 1 < ctx->prof_marks.size(); ++i) {
            const ProfMark &a = ctx->prof_marks[i], &b = ctx->prof_marks[i + 1];
            if (a.stage < 0) continue;
            float ms = 0.f;
            GC_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->prof_pool[a.ev_start], ctx->prof_pool[b.ev_end]));
            if (stage_ms) stage_ms[a.stage] += ms;
            if (stage_calls) stage_calls[a.stage] += 1;
        }
    }
    ctx->prof_marks.clear();
    ctx->prof_used = 0;
    const uint64_t now = gc::launches_total();
    if (kernel_launches) *kernel_launches = now - ctx->launch_base;
    ctx->launch_base = now;
    return GC_OK;
}

gc_status gc_check(gc_context *ctx, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    GC_CUDA(ctx, cudaStreamSynchronize(s));
    if (!ctx->last) return GC_OK;
    const gc_saved &S = *ctx->last;
    if (S.words.p) {
        uint32_t w[2];
        GC_CUDA(ctx, cudaMemcpyAsync(w, S.words.p, 8, cudaMemcpyDeviceToHost, s));
        GC_CUDA(ctx, cudaStreamSynchronize(s));
        if (w[1]) {
            GC_CUDA(ctx, cudaMemsetAsync(static_cast<uint32_t *>(S.words.p) + 1, 0, 4, s));
            return fail(ctx, GC_ERR_TIMEOUT, "a bounded device wait ran out (error word %#x)", w[1]);
        }
    }
    if (S.batch && S.batch.get() && !S.valid) return batch_check(ctx, S, s);
    if (S.valid && !S.k_exact && S.n_sel > 0) return capacity_check(ctx, S, s);
    return GC_OK;
}

}  // extern "C"

// order_wait / order_done (internal callers; NULL for the public entry points): the
// backward's writes into the caller's gradient buffers (the zeros of unselected layers, the
// chain rule, the motion sums) wait for order_wait and are followed by a record of order_done;
// the reverse blend and the reduce, which touch only the state's own buffers, do not wait.
static gc_status render_backward_impl(gc_context *ctx, const gc_saved *saved, const gc_gaussians *g,
                                      const gc_motion *motion, const float *dL_dimage,
                                      const float *const *dL_levels, gc_grads *out, void *stream,
                                      cudaEvent_t order_wait = nullptr, cudaEvent_t order_done = nullptr) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if ((!dL_dimage && !dL_levels) || !out) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimage or grads is NULL");
    const gc_saved &S = saved ? *saved : ctx->internal;
    if (!S.valid) return fail(ctx, GC_ERR_STATE, "no forward recorded in this saved state");
    if ((S.levels > 0) != (dL_levels != nullptr))
        return fail(ctx, GC_ERR_STATE, S.levels ? "the saved forward is multi-level: use gc_render_levels_backward"
                                                : "the saved forward is single-level: use gc_render_backward");
    if (dL_levels)
        for (int l = 0; l < S.levels; ++l)
            if (!dL_levels[l]) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimages[%d] is NULL", l);
    gc::GaussSrc src;
    gc_status st = make_source(ctx, g, motion, src);
    if (st != GC_OK) return st;
    if (g->n != S.n || g->sh_degree != S.sh_degree || g->n_layers != S.n_layers)
        return fail(ctx, GC_ERR_STATE, "the Gaussian set differs from the one of the saved forward");
    if ((src.group_q != nullptr) != S.has_motion || (S.has_motion && src.n_groups != S.n_groups) ||
        src.per_gaussian != S.per_gaussian)
        return fail(ctx, GC_ERR_STATE, "the motion differs from the one of the saved forward");
    if (src.res.ls != S.res.ls || src.res.logit != S.res.logit || src.res.sh != S.res.sh)
        return fail(ctx, GC_ERR_STATE, "the residual deformation differs from the one of the saved forward");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int K3 = 3 * (g->sh_degree + 1) * (g->sh_degree + 1);

    // Gaussians outside the selected layers receive zero gradient (written after the blend and
    // the reduce, with the other writes into the caller's buffers)
    auto zero_unselected = [&]() -> cudaError_t {
        for (int l = 0; l < S.n_layers; ++l) {
            if ((S.layer_mask >> l) & 1u) continue;
            const int64_t a = S.layer_offsets[l], b = S.layer_offsets[l + 1];
            if (b <= a) continue;
            cudaError_t e = cudaSuccess;
            if (out->d_means && e == cudaSuccess) e = cudaMemsetAsync(out->d_means + 3 * a, 0, (size_t)(b - a) * 12, s);
            if (out->d_log_scales && e == cudaSuccess)
                e = cudaMemsetAsync(out->d_log_scales + 3 * a, 0, (size_t)(b - a) * 12, s);
            if (out->d_quats && e == cudaSuccess) e = cudaMemsetAsync(out->d_quats + 4 * a, 0, (size_t)(b - a) * 16, s);
            if (out->d_opacity_logits && e == cudaSuccess)
                e = cudaMemsetAsync(out->d_opacity_logits + a, 0, (size_t)(b - a) * 4, s);
            if (out->d_sh && e == cudaSuccess)
                e = cudaMemsetAsync(out->d_sh + (int64_t)K3 * a, 0, (size_t)(b - a) * K3 * 4, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    };
    const int G = S.has_motion ? S.n_groups : 0;
    if (S.n_sel == 0) {
        if (order_wait) GC_CUDA(ctx, cudaStreamWaitEvent(s, order_wait, 0));
        GC_CUDA(ctx, zero_unselected());
        if (G && out->d_group_q) GC_CUDA(ctx, cudaMemsetAsync(out->d_group_q, 0, (size_t)G * 16, s));
        if (G && out->d_group_t) GC_CUDA(ctx, cudaMemsetAsync(out->d_group_t, 0, (size_t)G * 12, s));
        if (order_done) GC_CUDA(ctx, cudaEventRecord(order_done, s));
        return GC_OK;
    }
    const int64_t K = S.K > 0 ? S.K : 1;
    {
        void *before = S.bwd_part.p, *before_flag = S.bwd_flag.p;
        GC_CUDA(ctx, grow(S.bwd_part, (size_t)K * 9 * 4));
        GC_CUDA(ctx, grow(S.bwd_flag, (size_t)K));
        if (S.bwd_part.p != before || S.bwd_flag.p != before_flag) S.bwd_part_clean = false;
    }
    if (!S.bwd_part_clean) {
        GC_CUDA(ctx, cudaMemsetAsync(S.bwd_part.p, 0, S.bwd_part.cap, s));
        GC_CUDA(ctx, cudaMemsetAsync(S.bwd_flag.p, 0, S.bwd_flag.cap, s));
    }
    GC_CUDA(ctx, grow(S.bwd_g2d, (size_t)S.n_sel * 9 * 4));
    GC_CUDA(ctx, grow(S.bwd_motion, (size_t)S.n_sel * 7 * 4));
    if (G && !S.per_gaussian) GC_CUDA(ctx, grow(S.bwd_group, gc::group_partial_floats(S.n_sel, G) * 4));
    const uint32_t *sorted_vals = S.K > 0 ? S.lists() : nullptr;

    GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_BLEND_BWD));
    S.bwd_part_clean = false;
    if (dL_levels) {
        gc::LevelGrads lg{};
        for (int l = 0; l < S.levels; ++l) lg.g[l] = dL_levels[l];
        GC_CUDA(ctx, gc::launch_blend_levels_bwd(S.ranges.as<uint2>(), sorted_vals, S.ranked.as<float4>(),
                                                 S.offsets.as<uint32_t>(), S.cam, S.rp, S.levels, S.lv_T.as<float>(),
                                                 S.lv_last.as<uint32_t>(), lg, S.bwd_part.as<float>(),
                                                 S.bwd_flag.as<uint8_t>(), s));
    } else {
        GC_CUDA(ctx, gc::launch_blend_bwd(S.ranges.as<uint2>(), sorted_vals, S.ranked.as<float4>(),
                                          S.offsets.as<uint32_t>(), S.cam, S.rp, S.final_T.as<float>(),
                                          S.n_contrib.as<uint32_t>(), dL_dimage, S.bwd_part.as<float>(),
                                          S.bwd_flag.as<uint8_t>(), s));
    }
    GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_REDUCE));
    GC_CUDA(ctx, gc::launch_reduce_entries(S.bwd_part.as<float>(), S.offsets.as<uint32_t>(),
                                           S.touched_r.as<uint32_t>(), S.dvals[S.depth_buf].as<uint32_t>(),
                                           S.n_sel, (uint32_t)std::min<int64_t>(K, 0xFFFFFFFFll),
                                           S.bwd_flag.as<uint8_t>(), S.bwd_g2d.as<float>(), s));
    S.bwd_part_clean = true;
    GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_PREPROCESS_BWD));
    if (order_wait) GC_CUDA(ctx, cudaStreamWaitEvent(s, order_wait, 0));
    GC_CUDA(ctx, zero_unselected());
    GC_CUDA(ctx, gc::launch_preprocess_bwd(src, S.sel, S.n_sel, S.cam, S.rp, S.bwd_g2d.as<float>(),
                                           S.touched.as<uint32_t>(), *out,
                                           G ? S.bwd_motion.as<float>() : nullptr, s));
    if (G && S.per_gaussian) {
        // one motion per Gaussian: its motion terms are its gradient (zero when not selected)
        GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_GROUP_REDUCE));
        if (out->d_group_q) GC_CUDA(ctx, cudaMemsetAsync(out->d_group_q, 0, (size_t)G * 16, s));
        if (out->d_group_t) GC_CUDA(ctx, cudaMemsetAsync(out->d_group_t, 0, (size_t)G * 12, s));
        GC_CUDA(ctx, gc::launch_motion_scatter(S.bwd_motion.as<float>(), S.sel, S.n_sel, out->d_group_q,
                                               out->d_group_t, s));
    } else if (G) {
        GC_CUDA(ctx, prof_mark(ctx, s, GC_STAGE_GROUP_REDUCE));
        GC_CUDA(ctx, gc::launch_group_reduce(S.bwd_motion.as<float>(), src.group_id, S.sel, S.n_sel, G,
                                             S.bwd_group.as<float>(), out->d_group_q, out->d_group_t, s));
    }
    if (order_done) GC_CUDA(ctx, cudaEventRecord(order_done, s));
    GC_CUDA(ctx, prof_mark(ctx, s, -1));
    return GC_OK;
}

gc_status levels_backward_ordered(gc_context *ctx, const gc_saved *saved, const gc_gaussians *g,
                                  const gc_motion *motion, const float *const *dL_dimages, gc_grads *out,
                                  cudaStream_t stream, cudaEvent_t order_wait, cudaEvent_t order_done) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!dL_dimages) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimages is NULL");
    return render_backward_impl(ctx, saved, g, motion, nullptr, dL_dimages, out, stream, order_wait, order_done);
}

extern "C" gc_status gc_render_backward(gc_context *ctx, const gc_saved *saved, const gc_gaussians *g,
                                        const gc_motion *motion, const float *dL_dimage, gc_grads *out,
                                        void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!dL_dimage) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimage or grads is NULL");
    return render_backward_impl(ctx, saved, g, motion, dL_dimage, nullptr, out, stream);
}

extern "C" gc_status gc_render_levels_backward(gc_context *ctx, const gc_saved *saved, const gc_gaussians *g,
                                               const gc_motion *motion, const float *const *dL_dimages,
                                               gc_grads *out, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!dL_dimages) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimages is NULL");
    return render_backward_impl(ctx, saved, g, motion, nullptr, dL_dimages, out, stream);
}
