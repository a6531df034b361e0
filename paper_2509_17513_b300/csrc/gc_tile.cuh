// gc_tile.cuh - the per-tile forward and backward blends, shared by the single-frame
// kernels (one CTA per tile) and the batched persistent kernels (CTAs pull tiles of
// many images from a work counter).
#pragma once
#include <cuda_runtime.h>

#include "gc_blend.cuh"
#include "gc_internal.cuh"

namespace gc {

__device__ __forceinline__ void unpack_rect(float4 r2, int &x0, int &x1, int &y0, int &y1) {
    const uint32_t rx = __float_as_uint(r2.z), ry = __float_as_uint(r2.w);
    x0 = (int)(rx & 0xffffu);
    x1 = (int)(rx >> 16);
    y0 = (int)(ry & 0xffffu);
    y1 = (int)(ry >> 16);
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

// Front-to-back compositing (Eq. 2) of tile (tx, ty) of one image by a CTA of
// 256 / PPT threads; thread t owns the PPT vertically adjacent pixels
// (t % TW, PPT * (t / TW) + i), so each staged Gaussian is read from shared memory
// once per PPT pixels.  Batches of up to 256 list entries are staged in shared
// memory (sA/sB/sC, 256 float4 each), gathered from the depth-ranked records; a
// pixel stops when blending the next Gaussian would take its transmittance below
// 1e-4, the CTA as soon as all its pixels did.  Per-pixel outputs are indexed
// py * W + px from the given image-local pointers.
template <int TW, int TH, int PPT>
__device__ __forceinline__ void blend_fwd_tile(
    int tx, int ty, uint2 range, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, int W, int H, float bg0, float bg1, float bg2,
    int membership, float *__restrict__ image, float *__restrict__ final_T,
    uint32_t *__restrict__ n_contrib, uint32_t *__restrict__ n_blended,
    uint32_t *__restrict__ n_walked, float4 *sA, float4 *sB, float4 *sC) {
    static_assert(TW * TH == 256, "tile must hold 256 pixels");
    constexpr int NT = 256 / PPT;
    const int lx = threadIdx.x % TW, lyb = PPT * (threadIdx.x / TW);
    const int px = tx * TW + lx;
    const float pcx = (float)px + 0.5f;
    const uint32_t xbit = 1u << lx;
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

// Per-pixel reverse state.
struct BwdPix {
    float T, A0, A1, A2, g0, g1, g2;
    uint32_t last;
};

// Reverse step of Eq. 2 for one pixel and list entry k; adds the pixel's nine partial
// derivatives (du, dv, da, db, dc, dopacity, dr, dg, db) to v.  Returns whether the
// entry was blended into the pixel.
__device__ __forceinline__ bool bwd_step(BwdPix &P, float pcx, float pcy, const float4 &a,
                                         const float4 &bb, const float4 &nat, float blue, float *v) {
    const float dx = pcx - a.x, dy = pcy - a.y;
    const float p2 = blend_power2(a.z, a.w, bb.x, dx, dy);
    if (p2 > 0.f) return false;
    float G;
    const float a0 = blend_raw_alpha(bb.y, p2, G);
    const float alpha = fminf(kAlphaMax, a0);
    if (alpha < kAlphaMin) return false;
    P.T = P.T / (1.f - alpha);
    const float w = alpha * P.T;
    v[6] += w * P.g0;
    v[7] += w * P.g1;
    v[8] += w * P.g2;
    const float dal = P.T * (P.g0 * (bb.z - P.A0) + P.g1 * (bb.w - P.A1) + P.g2 * (blue - P.A2));
    P.A0 = fmaf(alpha, bb.z - P.A0, P.A0);
    P.A1 = fmaf(alpha, bb.w - P.A1, P.A1);
    P.A2 = fmaf(alpha, blue - P.A2, P.A2);
    if (!(a0 > kAlphaMax)) {
        v[5] += G * dal;
        const float dp = alpha * dal;  // dL/dpower (natural exponent)
        v[0] += (nat.x * dx + nat.y * dy) * dp;
        v[1] += (nat.y * dx + nat.z * dy) * dp;
        v[2] += -0.5f * dx * dx * dp;
        v[3] += -dx * dy * dp;
        v[4] += -0.5f * dy * dy * dp;
    }
    return true;
}

// Reverse compositing of tile (tx, ty) of one image by a CTA of 256 / PPT
// threads, each owning PPT vertically adjacent pixels.  For every list entry, the
// nine partials are summed over the thread's pixels, then over the warp with a
// transposing butterfly (values 0-7 spread over lane groups, 9 shuffles) plus a
// plain butterfly for value 8, then over the warps in order, and stored at the
// entry's emit position offsets[r] + entry_shift + (index of the tile in the
// Gaussian's tile rectangle).  *tile_rmax receives the largest rank that may have
// contributed (-1: none).  Shared scratch: sA..sD (256 float4 each), wpart_raw
// (32 x warps x 9 floats), s_last_max.
template <int TW, int TH, int PPT>
__device__ __forceinline__ void blend_bwd_tile(
    int tx, int ty, uint2 range, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, const uint32_t *__restrict__ offsets, uint32_t entry_shift,
    int W, int H, int tw_log2, int th_log2, float bg0, float bg1, float bg2, int membership,
    const float *__restrict__ final_T, const uint32_t *__restrict__ n_contrib,
    const float *__restrict__ dimg, float *__restrict__ part, int32_t *tile_rmax, float4 *sA,
    float4 *sB, float4 *sC, float4 *sD, float *wpart_raw, uint32_t *s_last_max) {
    constexpr int NT = 256 / PPT;
    constexpr int NW = NT / 32;
    float (*wpart)[NW][9] = reinterpret_cast<float (*)[NW][9]>(wpart_raw);
    const int lx = threadIdx.x % TW, lyb = PPT * (threadIdx.x / TW);
    const int px = tx * TW + lx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float pcx = (float)px + 0.5f;
    const uint32_t xbit = 1u << lx;
    const size_t hw = (size_t)W * H;

    BwdPix P[PPT];
    uint32_t my_last = 0;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const int py = ty * TH + lyb + i;
        P[i] = {1.f, bg0, bg1, bg2, 0.f, 0.f, 0.f, 0u};
        if (px < W && py < H) {
            const size_t p = (size_t)py * W + px;
            P[i].T = final_T[p];
            P[i].last = n_contrib[p];
            P[i].g0 = dimg[p];
            P[i].g1 = dimg[hw + p];
            P[i].g2 = dimg[2 * hw + p];
        }
        my_last = max(my_last, P[i].last);
    }

    if (threadIdx.x == 0) *s_last_max = 0;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, my_last);
    if (lane == 0) atomicMax(s_last_max, wmax);
    __syncthreads();
    const int n_active = (int)*s_last_max;
    if (threadIdx.x == 0)
        *tile_rmax = n_active > 0 ? (int32_t)sorted_vals[range.x + n_active - 1] : -1;

    for (int hi = n_active; hi > 0; hi -= 256) {
        const int lo = max(hi - 256, 0);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < PPT; ++h) {
            const int slot = (int)threadIdx.x + NT * h;
            const int k = lo + slot;
            if (k < hi) {
                const uint32_t r = sorted_vals[range.x + k];
                const float4 a = ranked[3 * (size_t)r];
                const float4 bb = ranked[3 * (size_t)r + 1];
                const float4 c = ranked[3 * (size_t)r + 2];
                int x0, x1, y0, y1;
                unpack_rect(c, x0, x1, y0, y1);
                uint32_t cm = 0xffffffffu, rm = 0xffffffffu;
                if (membership == GC_MEMBER_PIXEL) {
                    const int lx0 = max(x0 - tx * TW, 0), lx1 = min(x1 - tx * TW, TW - 1);
                    const int ly0r = max(y0 - ty * TH, 0), ly1r = min(y1 - ty * TH, TH - 1);
                    cm = (lx1 >= lx0) ? ((0xffffffffu >> (31 - lx1)) & (0xffffffffu << lx0)) : 0u;
                    rm = (ly1r >= ly0r) ? ((0xffffffffu >> (31 - ly1r)) & (0xffffffffu << ly0r)) : 0u;
                }
                const int tx0 = x0 >> tw_log2, ty0 = y0 >> th_log2, twid = (x1 >> tw_log2) - tx0 + 1;
                const uint32_t e = offsets[r] + entry_shift + (uint32_t)((ty - ty0) * twid + (tx - tx0));
                sA[slot] = a;
                sB[slot] = bb;
                sC[slot] = make_float4(c.x, __uint_as_float(cm), __uint_as_float(rm), __uint_as_float(e));
                sD[slot] = make_float4(a.z * kUnscaleDiag, a.w * kUnscaleOff, bb.x * kUnscaleDiag, 0.f);
            }
        }
        __syncthreads();
        for (int gtop = hi; gtop > lo; gtop -= 32) {
            const int gbot = max(gtop - 32, lo);
            for (int k = gtop - 1; k >= gbot; --k) {
                const int s = k - lo;
                float v[9];
#pragma unroll
                for (int c = 0; c < 9; ++c) v[c] = 0.f;
                const float4 c4 = sC[s];
                const uint32_t rm = __float_as_uint(c4.z) >> lyb;
                const bool col = (__float_as_uint(c4.y) & xbit) != 0;
                bool any = false;
#pragma unroll
                for (int i = 0; i < PPT; ++i) any = any || (col && (uint32_t)k < P[i].last && ((rm >> i) & 1u));
                bool contrib = false;
                if (any) {
                    const float4 a = sA[s], bb = sB[s], nat = sD[s];
#pragma unroll
                    for (int i = 0; i < PPT; ++i)
                        if (col && (uint32_t)k < P[i].last && ((rm >> i) & 1u))
                            contrib |= bwd_step(P[i], pcx, (float)(ty * TH + lyb + i) + 0.5f, a, bb, nat, c4.x, v);
                }
                float out0 = 0.f, out8 = 0.f;
                if (__any_sync(0xffffffffu, contrib)) {
                    // values 0..7: transposing butterfly; lane l ends with value (l >> 2) & 7
                    {
                        const bool up = lane & 16;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float send = up ? v[i] : v[i + 4];
                            const float keep = up ? v[i + 4] : v[i];
                            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
                        }
                    }
                    {
                        const bool up = lane & 8;
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const float send = up ? v[i] : v[i + 2];
                            const float keep = up ? v[i + 2] : v[i];
                            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
                        }
                    }
                    {
                        const bool up = lane & 4;
                        const float send = up ? v[0] : v[1];
                        const float keep = up ? v[1] : v[0];
                        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
                    }
                    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
                    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
                    out0 = v[0];
                    float x = v[8];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                    out8 = x;
                }
                if ((lane & 3) == 0) wpart[k - gbot][warp][lane >> 2] = out0;
                if (lane == 1) wpart[k - gbot][warp][8] = out8;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < (gtop - gbot) * 9; idx += NT) {
                const int q = idx / 9, c = idx - q * 9;
                float acc = wpart[q][0][c];
#pragma unroll
                for (int w2 = 1; w2 < NW; ++w2) acc += wpart[q][w2][c];
                const uint32_t e = __float_as_uint(sC[gbot + q - lo].w);
                part[(int64_t)e * 9 + c] = acc;
            }
            __syncthreads();
        }
    }
}

}  // namespace gc
