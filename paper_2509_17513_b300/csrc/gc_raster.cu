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

// Per-pixel front-to-back state.
struct FwdPix {
    float T, C0, C1, C2;
    uint32_t last, nb, walked;
    bool done;
};

// One compositing step of Eq. 2 for one pixel and the staged Gaussian (a, bb, blue).
__device__ __forceinline__ void fwd_step(FwdPix &P, float pcx, float pcy, const float4 &a,
                                         const float4 &bb, float blue, uint32_t idx) {
    const float dx = pcx - a.x, dy = pcy - a.y;
    const float p2 = blend_power2(a.z, a.w, bb.x, dx, dy);
    if (p2 > 0.f) return;
    float G;
    const float alpha = fminf(kAlphaMax, blend_raw_alpha(bb.y, p2, G));
    if (alpha < kAlphaMin) return;
    const float Tn = P.T * (1.f - alpha);
    if (Tn < kTStop) {
        P.done = true;
        P.walked = idx + 1;
        return;
    }
    const float w = alpha * P.T;
    P.C0 = fmaf(bb.z, w, P.C0);
    P.C1 = fmaf(bb.w, w, P.C1);
    P.C2 = fmaf(blue, w, P.C2);
    P.T = Tn;
    P.last = idx + 1;
    ++P.nb;
}

#ifndef GC_FWD_PPT
#define GC_FWD_PPT 1  // pixels per thread in the forward blend (1 measured fastest on B300)
#endif

// Front-to-back compositing (Eq. 2), one CTA per tile of TW x TH = 256 pixels with
// 256 / PPT threads; thread t owns the PPT vertically adjacent pixels
// (t % TW, PPT * (t / TW) + i), so each staged Gaussian is read from shared memory
// once per PPT pixels.  Batches of up to 256 list entries are staged in shared
// memory (gathered from the depth-ranked records); a pixel stops when blending the
// next Gaussian would take its transmittance below 1e-4, the CTA as soon as all its
// pixels did.
template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(256 / PPT) k_blend_fwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, int W, int H, int ntx, float bg0, float bg1, float bg2,
    int membership, float *__restrict__ image, float *__restrict__ final_T,
    uint32_t *__restrict__ n_contrib, uint32_t *__restrict__ n_blended,
    uint32_t *__restrict__ n_walked) {
    static_assert(TW * TH == 256, "tile must hold 256 pixels");
    constexpr int NT = 256 / PPT;
    __shared__ float4 sA[256];  // u, v, A, B
    __shared__ float4 sB[256];  // C, opacity, red, green
    __shared__ float4 sC[256];  // blue, column mask, row mask, -

    const int tile = blockIdx.x;
    const int tx = tile % ntx, ty = tile / ntx;
    const int lx = threadIdx.x % TW, lyb = PPT * (threadIdx.x / TW);
    const int px = tx * TW + lx;
    const float pcx = (float)px + 0.5f;
    const uint32_t xbit = 1u << lx;
    const uint2 range = ranges[tile];
    const int n = (int)(range.y - range.x);

    FwdPix P[PPT];
#pragma unroll
    for (int i = 0; i < PPT; ++i) P[i] = {1.f, 0.f, 0.f, 0.f, 0u, 0u, 0u, !(px < W && ty * TH + lyb + i < H)};
    auto all_done = [&]() {
        bool d = true;
#pragma unroll
        for (int i = 0; i < PPT; ++i) d = d && P[i].done;
        return d;
    };

    for (int b = 0; b < n; b += 256) {
        if (__syncthreads_count(all_done()) == NT) break;
#pragma unroll
        for (int h = 0; h < PPT; ++h) {
            const int slot = (int)threadIdx.x + NT * h;
            const int idx = b + slot;
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
                    const int ly0r = max(y0 - ty * TH, 0), ly1r = min(y1 - ty * TH, TH - 1);
                    cm = (lx1 >= lx0) ? ((0xffffffffu >> (31 - lx1)) & (0xffffffffu << lx0)) : 0u;
                    rm = (ly1r >= ly0r) ? ((0xffffffffu >> (31 - ly1r)) & (0xffffffffu << ly0r)) : 0u;
                }
                sA[slot] = a;
                sB[slot] = bb;
                sC[slot] = make_float4(c.x, __uint_as_float(cm), __uint_as_float(rm), 0.f);
            }
        }
        __syncthreads();
        const int cnt = min(256, n - b);
        for (int k = 0; k < cnt; ++k) {
            if (all_done()) break;
            const float4 c = sC[k];
            if (!(__float_as_uint(c.y) & xbit)) continue;
            const uint32_t rm = __float_as_uint(c.z) >> lyb;  // bit i: row lyb + i of the tile
            bool any = false;
#pragma unroll
            for (int i = 0; i < PPT; ++i) any = any || (!P[i].done && ((rm >> i) & 1u));
            if (!any) continue;
            const float4 a = sA[k];
            const float4 bb = sB[k];
            const uint32_t idx = (uint32_t)(b + k);
#pragma unroll
            for (int i = 0; i < PPT; ++i)
                if (!P[i].done && ((rm >> i) & 1u))
                    fwd_step(P[i], pcx, (float)(ty * TH + lyb + i) + 0.5f, a, bb, c.x, idx);
        }
    }
    const size_t hw = (size_t)W * H;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int py = ty * TH + lyb + i;
        if (px < W && py < H) {
            const size_t p = (size_t)py * W + px;
            image[p] = fmaf(P[i].T, bg0, P[i].C0);
            image[hw + p] = fmaf(P[i].T, bg1, P[i].C1);
            image[2 * hw + p] = fmaf(P[i].T, bg2, P[i].C2);
            final_T[p] = P[i].T;
            n_contrib[p] = P[i].last;
            if (n_blended) n_blended[p] = P[i].nb;
            if (n_walked) n_walked[p] = P[i].done ? P[i].walked : (uint32_t)n;
        }
    }
}

// Single CTA: 2D inclusive prefix of the tile difference grid (rows, then columns)
// gives the entry count of every tile; an exclusive scan in tile order gives the
// ranges of the tile-sorted list.
__global__ void __launch_bounds__(1024) k_tile_ranges_from_diff(const int32_t *__restrict__ diff,
                                                                int ntx, int nty,
                                                                const uint32_t *total_dev,
                                                                uint32_t cap,
                                                                uint2 *__restrict__ ranges) {
    extern __shared__ int32_t g[];
    __shared__ uint32_t ws[33];
    const int gw = ntx + 1, gh = nty + 1;
    const int cells = gw * gh;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) g[k] = diff[k];
    __syncthreads();
    for (int r = threadIdx.x; r < gh; r += blockDim.x) {
        int acc = 0;
        for (int c = 0; c < gw; ++c) {
            acc += g[r * gw + c];
            g[r * gw + c] = acc;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < gw; c += blockDim.x) {
        int acc = 0;
        for (int r = 0; r < gh; ++r) {
            acc += g[r * gw + c];
            g[r * gw + c] = acc;
        }
    }
    __syncthreads();
    const bool overflow = total_dev && (*total_dev > cap);
    const int T = ntx * nty;
    const int per = (T + (int)blockDim.x - 1) / (int)blockDim.x;
    const int start = (int)threadIdx.x * per;
    uint32_t s = 0;
    for (int q = 0; q < per; ++q) {
        const int t = start + q;
        if (t < T) s += (uint32_t)g[(t / ntx) * gw + (t % ntx)];
    }
    // block exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = ws[lane];
        uint32_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        ws[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = ws[warp] + inc - s;
    for (int q = 0; q < per; ++q) {
        const int t = start + q;
        if (t < T) {
            const uint32_t c = (uint32_t)g[(t / ntx) * gw + (t % ntx)];
            ranges[t] = overflow ? make_uint2(0u, 0u) : make_uint2(run, run + c);
            run += c;
        }
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

bool tile_diff_fits(int ntx, int nty) {
    return (size_t)(ntx + 1) * (size_t)(nty + 1) * 4 <= 200 * 1024;
}

cudaError_t launch_tile_ranges_from_diff(const int32_t *tile_diff, int ntx, int nty,
                                         const uint32_t *total_dev, uint32_t cap, uint2 *ranges,
                                         cudaStream_t st) {
    if (!tile_diff_fits(ntx, nty)) return cudaErrorNotSupported;
    const size_t smem = (size_t)(ntx + 1) * (nty + 1) * 4;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_ranges_from_diff,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_tile_ranges_from_diff<<<1, 1024, smem, st>>>(tile_diff, ntx, nty, total_dev, cap, ranges);
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
    constexpr int kThreads = 256 / GC_FWD_PPT;
    if (rp.tile_w == 16 && rp.tile_h == 16)
        k_blend_fwd<16, 16, GC_FWD_PPT><<<tiles, kThreads, 0, st>>>(GC_BLEND_ARGS);
    else if (rp.tile_w == 8 && rp.tile_h == 32)
        k_blend_fwd<8, 32, GC_FWD_PPT><<<tiles, kThreads, 0, st>>>(GC_BLEND_ARGS);
    else if (rp.tile_w == 32 && rp.tile_h == 8)
        k_blend_fwd<32, 8, GC_FWD_PPT><<<tiles, kThreads, 0, st>>>(GC_BLEND_ARGS);
    else
        return cudaErrorInvalidValue;
    note_launches(1);
#undef GC_BLEND_ARGS
    return cudaGetLastError();
}

}  // namespace gc
