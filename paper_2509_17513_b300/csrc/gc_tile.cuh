// gc_tile.cuh - the per-tile forward and backward blends, shared by the single-frame
// kernels (one CTA per tile) and the batched persistent kernels (CTAs pull tiles of
// many images from a work counter).
#pragma once
#include <cuda_runtime.h>

#include "gc_blend.cuh"
#include "gc_internal.cuh"
#include "gc_project.cuh"

namespace gc {

__device__ __forceinline__ void unpack_rect(float4 r2, int &x0, int &x1, int &y0, int &y1) {
    const uint32_t rx = __float_as_uint(r2.z), ry = __float_as_uint(r2.w);
    x0 = (int)(rx & 0xffffu);
    x1 = (int)(rx >> 16);
    y0 = (int)(ry & 0xffffu);
    y1 = (int)(ry >> 16);
}

// Pixel layout of a tile's 256 threads: each warp owns an 8 x 4 block of the tile
// (blocks row-major, TW / 8 per block row), lane l the pixel (l % 8, l / 8) of its
// block.  Square warp footprints keep a small Gaussian inside few warps, so most warps
// skip most list entries with one uniform test.
template <int TW, int TH>
__device__ __forceinline__ void pixel_of_thread(int t, int &lx, int &ly) {
    static_assert(TW % 8 == 0 && TH % 4 == 0 && TW * TH == 256, "tile must be 256 pixels of 8x4 blocks");
    constexpr int BX = TW / 8;
    const int w = t >> 5, l = t & 31;
    lx = (w % BX) * 8 + (l & 7);
    ly = (w / BX) * 4 + (l >> 3);
}

// Membership mask of warp w's 32 pixels for an entry whose footprint covers the tile
// columns in cm and the tile rows in rm (bit i = column / row i).
template <int TW>
__device__ __forceinline__ uint32_t warp_mask(uint32_t cm, uint32_t rm, int w) {
    constexpr int BX = TW / 8;
    const uint32_t cb = (cm >> ((w % BX) * 8)) & 0xffu;
    const uint32_t rb = (rm >> ((w / BX) * 4)) & 0xfu;
    const uint32_t spread = (rb & 1u) | ((rb & 2u) << 7) | ((rb & 4u) << 14) | ((rb & 8u) << 21);
    return cb * spread;  // bit 8 r + c = column c and row r of the block
}

// Column and row masks of an entry's pixel rectangle within tile (tx, ty).
template <int TW, int TH>
__device__ __forceinline__ void rect_masks(float4 r2, int tx, int ty, int membership, uint32_t &cm,
                                           uint32_t &rm) {
    cm = 0xffffffffu;
    rm = 0xffffffffu;
    if (membership == GC_MEMBER_PIXEL) {
        int x0, x1, y0, y1;
        unpack_rect(r2, x0, x1, y0, y1);
        const int lx0 = max(x0 - tx * TW, 0), lx1 = min(x1 - tx * TW, TW - 1);
        const int ly0 = max(y0 - ty * TH, 0), ly1 = min(y1 - ty * TH, TH - 1);
        cm = (lx1 >= lx0) ? ((0xffffffffu >> (31 - lx1)) & (0xffffffffu << lx0)) : 0u;
        rm = (ly1 >= ly0) ? ((0xffffffffu >> (31 - ly1)) & (0xffffffffu << ly0)) : 0u;
    }
}

template <int TW>
__device__ __forceinline__ void store_masks(uint32_t *m8, uint32_t cm, uint32_t rm) {
    uint4 *mo = reinterpret_cast<uint4 *>(m8);
    mo[0] = make_uint4(warp_mask<TW>(cm, rm, 0), warp_mask<TW>(cm, rm, 1), warp_mask<TW>(cm, rm, 2),
                       warp_mask<TW>(cm, rm, 3));
    mo[1] = make_uint4(warp_mask<TW>(cm, rm, 4), warp_mask<TW>(cm, rm, 5), warp_mask<TW>(cm, rm, 6),
                       warp_mask<TW>(cm, rm, 7));
}

// Mask of warp w's 8 x 4 block (bit 8 r + c = pixel (c, r) of the block) that an entry's alpha
// footprint can reach: binning step 15 evaluated on the block's band of four pixel rows
// instead of the tile row (the same FP32 operation sequence; a pixel left out has alpha below
// 1/255, so the blends skip nothing they would have blended), clipped to the pixel rectangle.
// Needs the alpha footprint (g.cull) and pixel-square membership.
template <int TW, int TH>
__device__ __forceinline__ uint32_t block_alpha_mask(const RowGeom &g, int tx, int ty, int w) {
    constexpr int BX = TW / 8;
    const int bx0 = tx * TW + (w % BX) * 8, by0 = ty * TH + (w / BX) * 4;
    const int r0 = max(by0, g.y0), r1 = min(by0 + 3, g.y1);
    if (r0 > r1) return 0u;
    const float d0 = fsub(fadd((float)r0, 0.5f), g.v), d1 = fsub(fadd((float)r1, 0.5f), g.v);
    const float dr = fminf(fmaxf(-g.sy, d0), d1), dl = fminf(fmaxf(g.sy, d0), d1);
    const float qr = fsub(g.at, fmul(fmul(g.detc, dr), dr)), ql = fsub(g.at, fmul(fmul(g.detc, dl), dl));
    const float xr = fmul(fsub(__fsqrt_rn(fmaxf(qr, 0.f)), fmul(g.ib, dr)), g.ria);
    const float xl = fmul(fsub(-fmul(g.ib, dl), __fsqrt_rn(fmaxf(ql, 0.f))), g.ria);
    float fx0 = ceilf(fsub(fadd(g.u, xl), 0.5f)), fx1 = floorf(fsub(fadd(g.u, xr), 0.5f));
    fx0 = fmaxf(fx0, (float)max(g.x0, bx0));
    fx1 = fminf(fx1, (float)min(g.x1, bx0 + 7));
    if (!(fx0 <= fx1)) return 0u;
    const int c0 = (int)fx0 - bx0, c1 = (int)fx1 - bx0;
    const uint32_t cb = (0xffu >> (7 - c1)) & (0xffu << c0);
    const uint32_t rb = (0xfu >> (3 - (r1 - by0))) & (0xfu << (r0 - by0));
    const uint32_t spread = (rb & 1u) | ((rb & 2u) << 7) | ((rb & 4u) << 14) | ((rb & 8u) << 21);
    return cb * spread;
}

// The same masks stored warp-major (m[w * 256 + t] for entry t), so that a warp reads
// the masks of 32 consecutive entries with one conflict-free load.
template <int TW>
__device__ __forceinline__ void store_masks_by_warp(uint32_t *m, int t, uint32_t cm, uint32_t rm) {
#pragma unroll
    for (int w = 0; w < 8; ++w) m[w * 256 + t] = warp_mask<TW>(cm, rm, w);
}

// Warp-major masks of an entry (record words a, c, r3): the alpha-footprint block masks when
// the footprint applies (alpha cull on, pixel-square membership, a proper conic), else the
// pixel rectangle's masks.
template <int TW, int TH>
__device__ __forceinline__ void store_entry_masks(uint32_t *m, int t, const float4 &a, const float4 &c,
                                                  const float4 &r3, int tx, int ty, const RenderParams &rp) {
    uint32_t cm, rm;
    rect_masks<TW, TH>(c, tx, ty, rp.membership, cm, rm);
    if (rp.membership == GC_MEMBER_PIXEL && rp.alpha_cull) {
        RowGeom g;
        row_geom(a, c, r3, rp, g);
        if (g.cull) {
#pragma unroll
            for (int w = 0; w < 8; ++w) m[w * 256 + t] = block_alpha_mask<TW, TH>(g, tx, ty, w);
            return;
        }
    }
    store_masks_by_warp<TW>(m, t, cm, rm);
}

// Shared staging of one batch of up to 256 list entries for the forward blend:
//   a = {u, v, A, B}, b = {C, opacity}  (what every walked pair reads),
//   c = {r, g, b, -}                    (read only when the pair is blended),
//   m = per entry and warp, the mask of the warp's pixels the entry may touch.
struct FwdSmem {
    float4 a[256];
    float2 b[256];
    float4 c[256];
    uint32_t m[256 * 8];
};

// Where a tile's pixels go: image planes (3 x H x W), final transmittance, list position
// after the last blended entry, optional counts, background.  The batched kernels keep it
// in shared memory so that it holds no registers during the blend.
struct TileOut {
    float *image, *final_T;
    uint32_t *n_contrib, *n_blended, *n_walked;
    float bg0, bg1, bg2;
    int W, H, membership;
    uint32_t rank_mask;  // of the tile-list words (list_rank_mask)
    uint32_t rank_base;  // added to a list word's rank: the record index of rank 0
};

// Front-to-back compositing (Eq. 2) of tile (tx, ty) of one image by a CTA of 256
// threads, one pixel each.  Batches of up to 256 list entries are staged in shared
// memory, gathered from the depth-ranked records.  Per walked entry a lane first tests
// the entry's membership mask against its own bit (cleared once its pixel is done), then
// evaluates the Gaussian; the colour is read only for blended pairs.  A pixel stops when
// blending the next Gaussian would take its transmittance below 1e-4, a warp (checked
// every 16 entries) when all its pixels did, the CTA when all warps did.  STATS adds
// the per-pixel blended and walked counts.
template <int TW, int TH, bool STATS>
__device__ __forceinline__ void blend_fwd_tile(int tx, int ty, uint2 range,
                                               const uint32_t *__restrict__ sorted_vals,
                                               const float4 *__restrict__ ranked, const TileOut &o,
                                               FwdSmem &sm) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lx, ly;
    pixel_of_thread<TW, TH>((int)threadIdx.x, lx, ly);
    const int px = tx * TW + lx, py = ty * TH + ly;
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const int n = (int)(range.y - range.x);
    const bool inside = px < o.W && py < o.H;
    const int membership = o.membership;
    uint32_t act = inside ? (1u << lane) : 0u;  // this lane's bit while the pixel is active
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    uint32_t last = 0u, nb = 0u, walked = (uint32_t)n;

    for (int b = 0; b < n; b += 256) {
        if (__syncthreads_count(act != 0u) == 0) break;
        {
            const int idx = b + (int)threadIdx.x;
            if (idx < n) {
                const uint32_t r = (sorted_vals[range.x + idx] & o.rank_mask) + o.rank_base;
                const float4 a = ranked[kRec * (size_t)r];
                const float4 bb = ranked[kRec * (size_t)r + 1];
                const float4 c = ranked[kRec * (size_t)r + 2];
                uint32_t cm, rm;
                rect_masks<TW, TH>(c, tx, ty, membership, cm, rm);
                sm.a[threadIdx.x] = a;
                sm.b[threadIdx.x] = make_float2(bb.x, bb.y);
                sm.c[threadIdx.x] = make_float4(bb.z, bb.w, c.x, 0.f);
                store_masks<TW>(&sm.m[8 * threadIdx.x], cm, rm);
            }
        }
        __syncthreads();
        const int cnt = min(256, n - b);
        for (int k0 = 0; k0 < cnt; k0 += 16) {
            if (__ballot_sync(0xffffffffu, act != 0u) == 0u) break;  // the whole warp is done
            const int k1 = min(k0 + 16, cnt);
#pragma unroll 4
            for (int k = k0; k < k1; ++k) {
                const uint32_t wm = sm.m[8 * k + warp];
                const float4 a = sm.a[k];
                const float2 bb = sm.b[k];
                const float dx = pcx - a.x, dy = pcy - a.y;
                const float p2 = blend_power2(a.z, a.w, bb.x, dx, dy);
                float G;
                const float alpha = fminf(kAlphaMax, blend_raw_alpha(bb.y, p2, G));
                // one test instead of three branches: footprint, exponent, alpha at least 1/255
                if (!(((wm & act) != 0u) & (p2 <= 0.f) & (alpha >= kAlphaMin))) continue;
                const float Tn = T * (1.f - alpha);
                if (Tn < kTStop) {
                    act = 0u;
                    walked = (uint32_t)(b + k + 1);
                    continue;
                }
                const float4 col = sm.c[k];
                const float w = alpha * T;
                C0 = fmaf(col.x, w, C0);
                C1 = fmaf(col.y, w, C1);
                C2 = fmaf(col.z, w, C2);
                T = Tn;
                last = (uint32_t)(b + k + 1);
                if (STATS) ++nb;
            }
        }
    }
    if (inside) {
        const int W = o.W;
        const size_t hw = (size_t)W * o.H;
        const size_t p = (size_t)py * W + px;
        o.image[p] = fmaf(T, o.bg0, C0);
        o.image[hw + p] = fmaf(T, o.bg1, C1);
        o.image[2 * hw + p] = fmaf(T, o.bg2, C2);
        o.final_T[p] = T;
        o.n_contrib[p] = last;
        if (STATS) {
            if (o.n_blended) o.n_blended[p] = nb;
            if (o.n_walked) o.n_walked[p] = walked;
        }
    }
}

// Threads of a reverse-blend CTA: each thread owns two pixels of the tile.
constexpr int kBwdThreads = 128;

// Shared staging for the reverse blend: a, b as in the forward; c = {r, g, b, a_nat} and
// d = {b_nat, c_nat} (colour and natural conic, read only for blended pairs); m the
// membership masks (per entry: two words per warp, the upper and lower 8 x 4 halves of
// its 8 x 8 block); e the entries' emit positions; wpart the per-warp sums of a group of
// 64 entries.
struct BwdSmem {
    float4 a[256];
    float2 b[256];
    float4 c[256];
    float2 d[256];
    uint32_t m[256 * 8];
    uint32_t e[256];
    float wpart[64][4][9];
    uint32_t last_max;
};

// What the reverse blend of a tile reads besides the lists: saved per-pixel state,
// dL/dimage, background, image size, membership rule and entry-position parameters.
struct TileBwd {
    const float *final_T;
    const uint32_t *n_contrib;
    const float *dimg;
    RenderParams rp;  // background, tile shape, membership, alpha cull
    int W, H;
    uint32_t entry_shift;
    uint32_t rank_base;  // added to a list word's rank: the record index of rank 0
    // per entry: 1 where a nonzero partial was written (only those are stored); NULL: every
    // entry of the walked range is stored, zeros included
    uint8_t *flag;
};

// Mask of the 8 x 4 pixel block at tile column c0 and row r0 (bit 8 r + c = pixel
// (c0 + c, r0 + r)) for an entry covering tile columns cm and rows rm.
__device__ __forceinline__ uint32_t block_mask(uint32_t cm, uint32_t rm, int c0, int r0) {
    const uint32_t cb = (cm >> c0) & 0xffu;
    const uint32_t rb = (rm >> r0) & 0xfu;
    const uint32_t spread = (rb & 1u) | ((rb & 2u) << 7) | ((rb & 4u) << 14) | ((rb & 8u) << 21);
    return cb * spread;
}

// Reverse state of one pixel: transmittance, colour behind, dL/dcolour, list position.
struct BwdPix {
    float T, A0, A1, A2, g0, g1, g2;
    uint32_t last;
};

// Reverse step of Eq. 2 for one pixel and a blended entry: undoes the blend
// (T_before = T_after / (1 - alpha) by a fast divide, 1 - alpha >= 0.01; running colour
// behind) and adds the pixel's nine
// partials (du, dv, da, db, dc, dopacity, dr, dg, db) to v.
__device__ __forceinline__ void bwd_blend(BwdPix &P, float dx, float dy, float alpha, float a0, float G,
                                          const float4 &col, const float2 &nd, float *v) {
    P.T = __fdividef(P.T, 1.f - alpha);
    const float w = alpha * P.T;
    v[6] += w * P.g0;
    v[7] += w * P.g1;
    v[8] += w * P.g2;
    const float dal = P.T * (P.g0 * (col.x - P.A0) + P.g1 * (col.y - P.A1) + P.g2 * (col.z - P.A2));
    P.A0 = fmaf(alpha, col.x - P.A0, P.A0);
    P.A1 = fmaf(alpha, col.y - P.A1, P.A1);
    P.A2 = fmaf(alpha, col.z - P.A2, P.A2);
    if (!(a0 > kAlphaMax)) {
        v[5] += G * dal;
        const float dp = alpha * dal;  // dL/dpower (natural exponent)
        v[0] += (col.w * dx + nd.x * dy) * dp;
        v[1] += (nd.x * dx + nd.y * dy) * dp;
        v[2] += -0.5f * dx * dx * dp;
        v[3] += -dx * dy * dp;
        v[4] += -0.5f * dy * dy * dp;
    }
}

// Reverse compositing of tile (tx, ty) of one image by a CTA of 128 threads.  Warp w
// owns an 8 x 8 block of the tile (blocks row-major, TW / 8 per block row); lane l the
// pixels (l % 8, l / 8) and (l % 8, l / 8 + 4) of its block.  Each pixel starts from its
// saved final transmittance T and list position `last` and walks the list back to
// front, undoing one blend per step.  For every entry the nine partials are summed over
// the thread's two pixels (first, second), over the warp with a transposing butterfly
// (values 0-7 spread over lane groups) plus a plain butterfly for value 8 - skipped when
// no pixel of the warp blended the entry - then over the warps in order, and stored at
// the entry's emit position offsets[r] + entry_shift + (index of the tile in the
// Gaussian's row intervals).
template <int TW, int TH>
__device__ __forceinline__ void blend_bwd_tile(int tx, int ty, uint2 range,
                                               const uint32_t *__restrict__ sorted_vals,
                                               const float4 *__restrict__ ranked,
                                               const uint32_t *__restrict__ offsets, const TileBwd &o,
                                               float *__restrict__ part, BwdSmem &sm) {
    static_assert(TW % 8 == 0 && TH % 8 == 0 && TW * TH == 256, "tile must be 256 pixels of 8x8 blocks");
    constexpr int BX = TW / 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int bx = (warp % BX) * 8, by = (warp / BX) * 8;  // block origin in the tile
    const int px = tx * TW + bx + (lane & 7), py0 = ty * TH + by + (lane >> 3);
    const float pcx = (float)px + 0.5f;
    const int membership = o.rp.membership;
    const uint32_t bit = 1u << lane;
    BwdPix P[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int py = py0 + 4 * i;
        P[i] = {1.f, o.rp.bg[0], o.rp.bg[1], o.rp.bg[2], 0.f, 0.f, 0.f, 0u};
        if (px < o.W && py < o.H) {
            const size_t hw = (size_t)o.W * o.H;
            const size_t p = (size_t)py * o.W + px;
            P[i].T = o.final_T[p];
            P[i].last = o.n_contrib[p];
            P[i].g0 = o.dimg[p];
            P[i].g1 = o.dimg[hw + p];
            P[i].g2 = o.dimg[2 * hw + p];
        }
    }
    if (threadIdx.x == 0) sm.last_max = 0u;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, max(P[0].last, P[1].last));
    if (lane == 0) atomicMax(&sm.last_max, wmax);
    __syncthreads();
    const int n_active = (int)sm.last_max;

    for (int hi = n_active; hi > 0; hi -= 256) {
        const int lo = max(hi - 256, 0);
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int slot = (int)threadIdx.x + kBwdThreads * h;
            const int k = lo + slot;
            if (k < hi) {
                const uint32_t r = (sorted_vals[range.x + k] & list_rank_mask(o.rp)) + o.rank_base;
                const float4 a = ranked[kRec * (size_t)r];
                const float4 bb = ranked[kRec * (size_t)r + 1];
                const float4 c = ranked[kRec * (size_t)r + 2];
                uint32_t cm, rm;
                rect_masks<TW, TH>(c, tx, ty, membership, cm, rm);
                RowGeom g;
                row_geom(a, c, ranked[kRec * (size_t)r + 3], o.rp, g);
                const float4 r4 = ranked[kRec * (size_t)r + 4];
                sm.a[slot] = a;
                sm.b[slot] = make_float2(bb.x, bb.y);
                sm.c[slot] = make_float4(bb.z, bb.w, c.x, a.z * kUnscaleDiag);
                sm.d[slot] = make_float2(a.w * kUnscaleOff, bb.x * kUnscaleDiag);
                uint4 *mo = reinterpret_cast<uint4 *>(&sm.m[8 * slot]);
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int w0 = 2 * q, w1 = 2 * q + 1;
                    const int c0a = (w0 % BX) * 8, r0a = (w0 / BX) * 8, c0b = (w1 % BX) * 8, r0b = (w1 / BX) * 8;
                    mo[q] = make_uint4(block_mask(cm, rm, c0a, r0a), block_mask(cm, rm, c0a, r0a + 4),
                                       block_mask(cm, rm, c0b, r0b), block_mask(cm, rm, c0b, r0b + 4));
                }
                sm.e[slot] = offsets[r] + o.entry_shift + entry_index(g, r4, tx, ty, o.rp, o.W, o.H);
            }
        }
        __syncthreads();
        for (int gtop = hi; gtop > lo; gtop -= 64) {
            const int gbot = max(gtop - 64, lo);
            for (int k = gtop - 1; k >= gbot; --k) {
                const int s = k - lo;
                const uint2 wm = *reinterpret_cast<const uint2 *>(&sm.m[8 * s + 2 * warp]);
                const bool m0 = (wm.x & bit) != 0u && (uint32_t)k < P[0].last;
                const bool m1 = (wm.y & bit) != 0u && (uint32_t)k < P[1].last;
                float v[9];
#pragma unroll
                for (int c = 0; c < 9; ++c) v[c] = 0.f;
                bool contrib = false;
                if (m0 || m1) {
                    const float4 a = sm.a[s];
                    const float2 bb = sm.b[s];
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const float dx = pcx - a.x, dy = ((float)(py0 + 4 * i) + 0.5f) - a.y;
                        const float p2 = blend_power2(a.z, a.w, bb.x, dx, dy);
                        float G;
                        const float a0 = blend_raw_alpha(bb.y, p2, G);
                        const float alpha = fminf(kAlphaMax, a0);
                        if (!((i == 0 ? m0 : m1) & (p2 <= 0.f) & (alpha >= kAlphaMin))) continue;
                        contrib = true;
                        bwd_blend(P[i], dx, dy, alpha, a0, G, sm.c[s], sm.d[s], v);
                    }
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
                    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
                    out8 = x;
                }
                if ((lane & 3) == 0) sm.wpart[k - gbot][warp][lane >> 2] = out0;
                if (lane == 1) sm.wpart[k - gbot][warp][8] = out8;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < (gtop - gbot) * 9; idx += kBwdThreads) {
                const int q = idx / 9, c = idx - q * 9;
                const float acc = ((sm.wpart[q][0][c] + sm.wpart[q][1][c]) + sm.wpart[q][2][c]) + sm.wpart[q][3][c];
                const uint32_t e = sm.e[gbot + q - lo];
                if (!o.flag) {
                    part[(int64_t)e * 9 + c] = acc;
                } else if (acc != 0.f) {  // the buffer holds zeros: a zero partial needs no store
                    part[(int64_t)e * 9 + c] = acc;
                    o.flag[e] = 1;
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace gc
