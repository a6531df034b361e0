// gc_raster.cu - binning (emit), tile ranges and the forward blend for sm_103a.
//
// Binning works in depth-rank space: Gaussians are first sorted by depth
// (N keys), then every Gaussian emits one entry per touched tile in rank order,
// and a stable sort on the tile id alone (log2(tiles) bits, two 8-bit digits at
// 1080p and 4K) yields per-tile lists that are already front to back, with
// ties broken by the global index (the depth sort is stable over index order).
// An entry's position in emit order is offsets[r] + (its tile's index in the
// Gaussian's tile rectangle); the backward pass writes its partial gradients
// there, so each Gaussian's partials are contiguous.
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_blend.cuh"
#include "gc_internal.cuh"

namespace gc {

namespace {

__device__ __forceinline__ void unpack_rect(float4 r2, int &x0, int &x1, int &y0, int &y1) {
    const uint32_t rx = __float_as_uint(r2.z), ry = __float_as_uint(r2.w);
    x0 = (int)(rx & 0xffffu);
    x1 = (int)(rx >> 16);
    y0 = (int)(ry & 0xffffu);
    y1 = (int)(ry >> 16);
}

// One warp emits the entries of 32 consecutive ranks, lanes striding over the
// warp's contiguous output range (coalesced writes, balanced across lanes).
__global__ void __launch_bounds__(256) k_emit(const float4 *__restrict__ ranked,
                                              const uint32_t *__restrict__ offsets,
                                              const uint32_t *__restrict__ touched_r, int64_t n,
                                              int tw_log2, int th_log2, int ntx, uint32_t cap,
                                              uint32_t *__restrict__ keys,
                                              uint32_t *__restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const int64_t wbase = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;
    if (wbase >= n) return;
    const int64_t r = wbase + lane;
    const bool valid = r < n;
    uint32_t cnt = valid ? touched_r[r] : 0u;
    uint32_t off = valid ? offsets[r] : 0xffffffffu;
    int tx0 = 0, ty0 = 0, twid = 1;
    if (valid && cnt) {
        int x0, x1, y0, y1;
        unpack_rect(ranked[3 * r + 2], x0, x1, y0, y1);
        tx0 = x0 >> tw_log2;
        ty0 = y0 >> th_log2;
        twid = (x1 >> tw_log2) - tx0 + 1;
    }
    const uint32_t start = __shfl_sync(0xffffffffu, off, 0);
    const uint32_t end = __reduce_max_sync(0xffffffffu, valid ? off + cnt : 0u);
    for (uint32_t e0 = start; e0 < end; e0 += 32) {
        const uint32_t e = e0 + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            uint32_t o = __shfl_sync(0xffffffffu, off, owner + step);
            if (o <= e) owner += step;
        }
        const uint32_t oo = __shfl_sync(0xffffffffu, off, owner);
        const int otw = __shfl_sync(0xffffffffu, twid, owner);
        const int otx = __shfl_sync(0xffffffffu, tx0, owner);
        const int oty = __shfl_sync(0xffffffffu, ty0, owner);
        if (e < end && e < cap) {
            const uint32_t k = e - oo;
            const uint32_t ty = (uint32_t)oty + k / (uint32_t)otw;
            const uint32_t tx = (uint32_t)otx + k % (uint32_t)otw;
            keys[e] = ty * (uint32_t)ntx + tx;
            vals[e] = (uint32_t)(wbase + owner);
        }
    }
}

__global__ void k_tile_ranges(const uint32_t *__restrict__ keys, const uint32_t *n_dev,
                              int64_t n_max, uint2 *__restrict__ ranges) {
    int64_t n = n_max;
    if (n_dev) {
        int64_t d = (int64_t)*n_dev;
        if (d < n) n = d;
    }
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[p];
        if (p == 0 || keys[p - 1] != k) ranges[k].x = (uint32_t)p;
        if (p == n - 1 || keys[p + 1] != k) ranges[k].y = (uint32_t)(p + 1);
    }
}

// Front-to-back compositing (Eq. 2), one CTA per tile of TW x TH = 256 pixels.
// Each batch of up to 256 list entries is staged in shared memory (one entry
// per thread, gathered from the depth-ranked records), then every pixel walks
// the batch.  A pixel stops when blending the next Gaussian would take its
// transmittance below 1e-4; the CTA leaves as soon as all its pixels stopped.
template <int TW, int TH>
__global__ void __launch_bounds__(256) k_blend_fwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, int W, int H, int ntx, float bg0, float bg1, float bg2,
    int membership, float *__restrict__ image, float *__restrict__ final_T,
    uint32_t *__restrict__ n_contrib, uint32_t *__restrict__ n_blended,
    uint32_t *__restrict__ n_walked) {
    static_assert(TW * TH == 256, "tile must hold 256 pixels");
    __shared__ float4 sA[256];  // u, v, conic a, conic b
    __shared__ float4 sB[256];  // conic c, opacity, red, green
    __shared__ float4 sC[256];  // blue, column mask, row mask, -

    const int tile = blockIdx.x;
    const int tx = tile % ntx, ty = tile / ntx;
    const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
    const int px = tx * TW + lx, py = ty * TH + ly;
    const bool inside = px < W && py < H;
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const uint32_t xbit = 1u << lx, ybit = 1u << ly;
    const uint2 range = ranges[tile];
    const int n = (int)(range.y - range.x);

    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    bool done = !inside;
    uint32_t last = 0, nb = 0, walked = 0;

    for (int b = 0; b < n; b += 256) {
        if (__syncthreads_count(done) == 256) break;
        const int idx = b + (int)threadIdx.x;
        if (idx < n) {
            const uint32_t r = sorted_vals[range.x + idx];
            const float4 a = ranked[3 * (size_t)r];
            const float4 bb = ranked[3 * (size_t)r + 1];
            const float4 c = ranked[3 * (size_t)r + 2];
            uint32_t cm = 0xffffffffu, rm = 0xffffffffu;
            if (membership == GC_MEMBER_PIXEL) {
                int x0, x1, y0, y1;
                unpack_rect(c, x0, x1, y0, y1);
                const int lx0 = max(x0 - tx * TW, 0), lx1 = min(x1 - tx * TW, TW - 1);
                const int ly0 = max(y0 - ty * TH, 0), ly1 = min(y1 - ty * TH, TH - 1);
                cm = (lx1 >= lx0) ? ((0xffffffffu >> (31 - lx1)) & (0xffffffffu << lx0)) : 0u;
                rm = (ly1 >= ly0) ? ((0xffffffffu >> (31 - ly1)) & (0xffffffffu << ly0)) : 0u;
            }
            sA[threadIdx.x] = a;
            sB[threadIdx.x] = bb;
            sC[threadIdx.x] = make_float4(c.x, __uint_as_float(cm), __uint_as_float(rm), 0.f);
        }
        __syncthreads();
        const int cnt = min(256, n - b);
        if (!done) {
            for (int k = 0; k < cnt; ++k) {
                const float4 c = sC[k];
                if (!(__float_as_uint(c.y) & xbit) || !(__float_as_uint(c.z) & ybit)) continue;
                const float4 a = sA[k];
                const float4 bb = sB[k];
                const float dx = pcx - a.x, dy = pcy - a.y;
                const float power = blend_power(a.z, a.w, bb.x, dx, dy);
                if (power > 0.f) continue;
                float G;
                const float alpha = fminf(kAlphaMax, blend_raw_alpha(bb.y, power, G));
                if (alpha < kAlphaMin) continue;
                const float Tn = T * (1.f - alpha);
                if (Tn < kTStop) {
                    done = true;
                    walked = (uint32_t)(b + k + 1);
                    break;
                }
                const float w = alpha * T;
                C0 = fmaf(bb.z, w, C0);
                C1 = fmaf(bb.w, w, C1);
                C2 = fmaf(c.x, w, C2);
                T = Tn;
                last = (uint32_t)(b + k + 1);
                ++nb;
            }
        }
    }
    if (inside) {
        const size_t hw = (size_t)W * H, p = (size_t)py * W + px;
        image[p] = fmaf(T, bg0, C0);
        image[hw + p] = fmaf(T, bg1, C1);
        image[2 * hw + p] = fmaf(T, bg2, C2);
        final_T[p] = T;
        n_contrib[p] = last;
        if (n_blended) n_blended[p] = nb;
        if (n_walked) n_walked[p] = done ? walked : (uint32_t)n;
    }
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
                        int64_t n, const RenderParams &rp, uint32_t *keys, uint32_t *vals,
                        uint32_t cap, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t threads = ((n + 31) / 32) * 32;
    k_emit<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        ranked, offsets, touched_r, n, rp.tile_w_log2, rp.tile_h_log2, rp.ntx, cap, keys, vals);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const uint32_t *keys, const uint32_t *n_dev, int64_t n_max,
                               uint2 *ranges, cudaStream_t st) {
    if (n_max <= 0) return cudaSuccess;
    int64_t blocks = (n_max + 255) / 256;
    if (blocks > 148 * 32) blocks = 148 * 32;
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
        rp.membership, image, final_T, n_contrib, n_blended, n_walked
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
