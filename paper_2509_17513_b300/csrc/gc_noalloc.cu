// gc_noalloc.cu - gc_render_forward_noalloc: the forward render with every piece of
// scratch taken from one file-scope device array, so the call allocates nothing.
//
// Who needs it: callers that cannot allocate device memory at render time.  A
// decode-and-render playback thread with a hard per-frame deadline must not block
// in the allocator or fail with out-of-memory halfway through a stream; and host
// applications or plugins that run inside someone else's CUDA context under a
// fixed memory budget may neither create a gc_context (which owns grow-only
// scratch) nor allocate after start-up.  This entry point serves them with a
// fixed, stated maximum problem size.
//
// The scratch is g_noalloc_scratch below (kScratchBytes, about 22.5 MiB).  Every GPU
// that loads this module holds it until the process exits.  In host code the
// array's name is only a host-side stand-in, so the device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and
// passed to the kernels.
//
// All calls share the array and it keeps the last call's contents: everything
// that must start at zero (the tile ranges) is cleared on the stream by each
// call, every other buffer is fully written before it is read.  Calls whose work
// overlaps on the GPU (two streams, or two host threads) race on the array and
// give wrong images: serialise them on one stream.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "gc_internal.cuh"

namespace {

constexpr int64_t kMaxSelected = 32768;        // selected Gaussians
constexpr int64_t kMaxKeys = int64_t(1) << 20; // (tile, Gaussian) pairs
constexpr int64_t kMaxPixels = int64_t(1) << 18;  // width * height (e.g. 512 x 512)
constexpr int64_t kMaxTiles = 4096;

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// Carving of the array (byte offsets).
constexpr size_t kOffRec = 0;
constexpr size_t kOffRanked = kOffRec + al(kMaxSelected * 16 * gc::kRec);
constexpr size_t kOffDKeys0 = kOffRanked + al(kMaxSelected * 16 * gc::kRec);
constexpr size_t kOffDKeys1 = kOffDKeys0 + al(kMaxSelected * 4);
constexpr size_t kOffDVals0 = kOffDKeys1 + al(kMaxSelected * 4);
constexpr size_t kOffDVals1 = kOffDVals0 + al(kMaxSelected * 4);
constexpr size_t kOffTouched = kOffDVals1 + al(kMaxSelected * 4);
constexpr size_t kOffTouchedR = kOffTouched + al(kMaxSelected * 4);
constexpr size_t kOffOffsets = kOffTouchedR + al(kMaxSelected * 4);
constexpr size_t kOffTKeys0 = kOffOffsets + al((kMaxSelected + 1) * 4);
constexpr size_t kOffTKeys1 = kOffTKeys0 + al(kMaxKeys * 4);
constexpr size_t kOffTVals0 = kOffTKeys1 + al(kMaxKeys * 4);
constexpr size_t kOffTVals1 = kOffTVals0 + al(kMaxKeys * 4);
constexpr size_t kOffRanges = kOffTVals1 + al(kMaxKeys * 4);
constexpr size_t kOffFinalT = kOffRanges + al(kMaxTiles * 8);
constexpr size_t kOffNContrib = kOffFinalT + al(kMaxPixels * 4);
constexpr size_t kOffWords = kOffNContrib + al(kMaxPixels * 4);
constexpr size_t kOffSortScratch = kOffWords + 256;
// radix histograms (256 per block of at least 2048 keys) + their scan partials, with slack
constexpr size_t kSortScratchBytes = al((4 * (257 + 256 * ((kMaxKeys + 2047) / 2048)) + 1024) * 4);  // one-sweep layout
constexpr size_t kScratchBytes = kOffSortScratch + kSortScratchBytes;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_setup_mutex;
void *g_scratch_addr[128];  // per device ordinal, filled at first use

gc_status say(char *err, size_t len, gc_status s, const char *fmt, ...) {
    if (err && len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, len, fmt, ap);
        va_end(ap);
    }
    return s;
}

// Device address of g_noalloc_scratch on the current device (looked up once).
gc_status scratch_address(unsigned char **out, char *err, size_t len) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 128)
        return say(err, len, GC_ERR_CUDA, "cudaGetDevice failed: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return say(err, len, GC_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) failed: %s",
                       cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return GC_OK;
}

int log2_exact(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return ((1 << l) == v) ? l : -1;
}

int key_bits(int64_t max_value) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) <= max_value) ++b;
    return b;
}

#define NA_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return say(err, err_len, GC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
    } while (0)

}  // namespace

extern "C" GC_API gc_status gc_render_forward_noalloc(const gc_options *opt, const gc_gaussians *g,
                                                      const gc_motion *motion, uint32_t layer_mask,
                                                      const gc_camera *cam, float *image,
                                                      void *stream, char *err, size_t err_len) {
    if (err && err_len) err[0] = '\0';
    gc_options o;
    if (opt) o = *opt;
    else gc_default_options(&o);  // exactly the library defaults (alpha footprint on)
    const bool shape_ok = (o.tile_w == 16 && o.tile_h == 16) || (o.tile_w == 8 && o.tile_h == 32) ||
                          (o.tile_w == 32 && o.tile_h == 8);
    if (!shape_ok || !(o.near_plane > 0.f) || !(o.dilation >= 0.f) || !(o.frustum_clamp > 0.f) ||
        (o.membership != GC_MEMBER_PIXEL && o.membership != GC_MEMBER_TILE))
        return say(err, err_len, GC_ERR_INVALID_ARG, "invalid options");
    if (!g || !cam || !image) return say(err, err_len, GC_ERR_INVALID_ARG, "gaussians, camera or image is NULL");
    if (cam->width <= 0 || cam->height <= 0 || !(cam->fx > 0.f) || !(cam->fy > 0.f))
        return say(err, err_len, GC_ERR_INVALID_ARG, "invalid camera");
    if (g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3 || g->n_layers < 1 ||
        g->n_layers > gc::kMaxLayers || !g->layer_offsets || g->layer_offsets[0] != 0 ||
        g->layer_offsets[g->n_layers] != g->n)
        return say(err, err_len, GC_ERR_INVALID_ARG, "invalid Gaussian set");
    for (int l = 0; l < g->n_layers; ++l)
        if (g->layer_offsets[l + 1] < g->layer_offsets[l])
            return say(err, err_len, GC_ERR_INVALID_ARG, "layer_offsets must be nondecreasing");
    if (g->precision == GC_PREC_PLANES)
        return say(err, err_len, GC_ERR_UNSUPPORTED, "the allocation-free path takes FP32 or BF16/FP8 sets, not decoded planes");
    if (g->precision != GC_PREC_FP32 && g->precision != GC_PREC_BF16_FP8)
        return say(err, err_len, GC_ERR_INVALID_ARG, "unknown precision");
    if (g->n > 0 && g->precision == GC_PREC_FP32 &&
        (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return say(err, err_len, GC_ERR_INVALID_ARG, "an FP32 attribute array is NULL");
    if (g->n > 0 && g->precision == GC_PREC_BF16_FP8 &&
        (!g->means_bf16 || !g->log_scales_bf16 || !g->quats_bf16 || !g->opacity_bf16 ||
         !g->sh_e4m3 || !g->scales))
        return say(err, err_len, GC_ERR_INVALID_ARG, "a reduced-precision plane is NULL");
    if (motion && (motion->q || motion->t || motion->per_gaussian) &&
        ((!motion->per_gaussian && motion->n_groups < 1) || !motion->q || !motion->t))
        return say(err, err_len, GC_ERR_INVALID_ARG, "invalid motion");
    if (motion && motion->res_sh && g->sh_degree == 3 && (reinterpret_cast<uintptr_t>(motion->res_sh) & 15))
        return say(err, err_len, GC_ERR_INVALID_ARG, "res_sh must be 16-byte aligned");

    // selection (host, no allocation)
    gc::Selection sel{};
    int64_t n_sel = 0;
    for (int l = 0; l < g->n_layers; ++l) {
        if (!((layer_mask >> l) & 1u)) continue;
        const int64_t a = g->layer_offsets[l], b = g->layer_offsets[l + 1];
        if (b <= a) continue;
        sel.range_begin[sel.n_ranges] = a;
        sel.range_start[sel.n_ranges + 1] = sel.range_start[sel.n_ranges] + (b - a);
        sel.n_ranges++;
        n_sel += b - a;
    }
    if (sel.n_ranges == 0) sel.n_ranges = 1;

    const int ntx = (cam->width + o.tile_w - 1) / o.tile_w;
    const int nty = (cam->height + o.tile_h - 1) / o.tile_h;
    const int64_t n_tiles = (int64_t)ntx * nty;
    const int64_t hw = (int64_t)cam->width * cam->height;
    if (n_sel > kMaxSelected)
        return say(err, err_len, GC_ERR_CAPACITY,
                   "%lld selected Gaussians exceed the no-allocation maximum of %lld",
                   (long long)n_sel, (long long)kMaxSelected);
    if (hw > kMaxPixels || n_tiles > kMaxTiles)
        return say(err, err_len, GC_ERR_CAPACITY,
                   "a %dx%d image exceeds the no-allocation maximum of %lld pixels and %lld tiles",
                   cam->width, cam->height, (long long)kMaxPixels, (long long)kMaxTiles);
    if (gc::radix_scratch_words(kMaxKeys) * 4 > kSortScratchBytes ||
        gc::scan_partials_size(kMaxSelected) * 4 > kSortScratchBytes)
        return say(err, err_len, GC_ERR_STATE, "internal: sort scratch reservation too small");

    unsigned char *base = nullptr;
    gc_status st = scratch_address(&base, err, err_len);
    if (st != GC_OK) return st;

    gc::GaussSrc src;
    memset(&src, 0, sizeof src);
    src.n = g->n;
    src.sh_degree = g->sh_degree;
    src.K = (g->sh_degree + 1) * (g->sh_degree + 1);
    src.precision = g->precision;
    src.means = g->means; src.log_scales = g->log_scales; src.quats = g->quats;
    src.opacity_logits = g->opacity_logits; src.sh = g->sh;
    src.means_h = g->means_bf16; src.log_scales_h = g->log_scales_bf16; src.quats_h = g->quats_bf16;
    src.opacity_h = g->opacity_bf16; src.sh_q = g->sh_e4m3; src.scales = g->scales;
    src.n_groups = 1;
    if (motion) src.res = gc::Residual{motion->res_log_scales, motion->res_opacity_logits, motion->res_sh};
    if (motion && motion->q) {
        src.group_id = motion->per_gaussian ? nullptr : g->group_id;
        src.group_q = motion->q;
        src.group_t = motion->t;
        src.n_groups = motion->per_gaussian ? (int)(g->n > 0 ? g->n : 1) : motion->n_groups;
        src.per_gaussian = motion->per_gaussian ? 1 : 0;
    }
    gc::CamParams cp;
    cp.width = cam->width; cp.height = cam->height;
    cp.fx = cam->fx; cp.fy = cam->fy; cp.cx = cam->cx; cp.cy = cam->cy;
    memcpy(cp.R, cam->R, sizeof cp.R);
    memcpy(cp.t, cam->t, sizeof cp.t);
    memcpy(cp.campos, cam->campos, sizeof cp.campos);
    gc::RenderParams rp{};  // list_packed = 0: the lists of this path come from the key sort
    rp.near_plane = o.near_plane; rp.dilation = o.dilation; rp.frustum_clamp = o.frustum_clamp;
    memcpy(rp.bg, o.bg, sizeof rp.bg);
    rp.tile_w = o.tile_w; rp.tile_h = o.tile_h;
    rp.tile_w_log2 = log2_exact(o.tile_w); rp.tile_h_log2 = log2_exact(o.tile_h);
    rp.ntx = ntx; rp.nty = nty;
    rp.membership = o.membership;
    rp.alpha_cull = o.alpha_cull;

    cudaStream_t s = (cudaStream_t)stream;
    float4 *rec = reinterpret_cast<float4 *>(base + kOffRec);
    float4 *ranked = reinterpret_cast<float4 *>(base + kOffRanked);
    uint32_t *dk[2] = {reinterpret_cast<uint32_t *>(base + kOffDKeys0), reinterpret_cast<uint32_t *>(base + kOffDKeys1)};
    uint32_t *dv[2] = {reinterpret_cast<uint32_t *>(base + kOffDVals0), reinterpret_cast<uint32_t *>(base + kOffDVals1)};
    uint32_t *touched = reinterpret_cast<uint32_t *>(base + kOffTouched);
    uint32_t *touched_r = reinterpret_cast<uint32_t *>(base + kOffTouchedR);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(base + kOffOffsets);
    uint32_t *tk[2] = {reinterpret_cast<uint32_t *>(base + kOffTKeys0), reinterpret_cast<uint32_t *>(base + kOffTKeys1)};
    uint32_t *tv[2] = {reinterpret_cast<uint32_t *>(base + kOffTVals0), reinterpret_cast<uint32_t *>(base + kOffTVals1)};
    uint2 *ranges = reinterpret_cast<uint2 *>(base + kOffRanges);
    float *final_T = reinterpret_cast<float *>(base + kOffFinalT);
    uint32_t *n_contrib = reinterpret_cast<uint32_t *>(base + kOffNContrib);
    uint32_t *words = reinterpret_cast<uint32_t *>(base + kOffWords);
    uint32_t *sort_scratch = reinterpret_cast<uint32_t *>(base + kOffSortScratch);

    // the tile ranges and the error word must start at zero: the array keeps the previous
    // call's values
    NA_CUDA(cudaMemsetAsync(ranges, 0, (size_t)n_tiles * 8, s));
    NA_CUDA(cudaMemsetAsync(words, 0, 8, s));
    int64_t K = 0;
    int tile_buf = 0;
    if (n_sel > 0) {
        int depth_buf = 0;
        NA_CUDA(gc::launch_preprocess(src, sel, n_sel, cp, rp, rec, dk[0], dv[0], touched, s));
        NA_CUDA(gc::radix_sort_pairs(dk, dv, n_sel, nullptr, 32, sort_scratch, &depth_buf, s, words + 1));
        NA_CUDA(gc::launch_rank_gather(dv[depth_buf], rec, touched, n_sel, ranked, touched_r, s));
        NA_CUDA(gc::launch_exclusive_scan(touched_r, offsets, n_sel, words, sort_scratch, s, words + 1));
        uint32_t w_host[2] = {0u, 0u};  // pair count and error word; stack: no host allocation
        NA_CUDA(cudaMemcpyAsync(w_host, words, 8, cudaMemcpyDeviceToHost, s));
        NA_CUDA(cudaStreamSynchronize(s));
        if (w_host[1] != 0u)
            return say(err, err_len, GC_ERR_TIMEOUT, "a bounded wait of the depth sort ran out");
        K = w_host[0];
        if (K > kMaxKeys)
            return say(err, err_len, GC_ERR_CAPACITY,
                       "the frame needs %lld (tile, Gaussian) pairs; the no-allocation maximum is %lld",
                       (long long)K, (long long)kMaxKeys);
        if (K > 0) {
            NA_CUDA(gc::launch_emit(ranked, offsets, touched_r, n_sel, rp, cam->width, cam->height, tk[0], tv[0], (uint32_t)K, s));
            NA_CUDA(gc::radix_sort_pairs(tk, tv, K, nullptr, key_bits(n_tiles - 1), sort_scratch,
                                         &tile_buf, s, words + 1));
            NA_CUDA(gc::launch_tile_ranges(tk[tile_buf], nullptr, K, ranges, s));
        }
    }
    NA_CUDA(gc::launch_blend_fwd(ranges, K > 0 ? tv[tile_buf] : nullptr, ranked, cp, rp, image,
                                 final_T, n_contrib, nullptr, nullptr, s));
    if (K > 0) {
        // the tile sort's bounded waits report through the same error word
        uint32_t e_host = 0u;
        NA_CUDA(cudaMemcpyAsync(&e_host, words + 1, 4, cudaMemcpyDeviceToHost, s));
        NA_CUDA(cudaStreamSynchronize(s));
        if (e_host != 0u)
            return say(err, err_len, GC_ERR_TIMEOUT, "a bounded wait of the tile sort ran out");
    }
    return GC_OK;
}
