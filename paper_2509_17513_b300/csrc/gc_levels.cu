// gc_levels.cu - single-pass multi-level render: every quality level l = 1..L of one view
// (level l = layers 1..l, Eq. 4) from one sorted list.
//
// The layers are nested prefixes of the significance-sorted set (Sec. 3.1), so the tile
// lists of level L hold every Gaussian that any level needs, in the same (depth, index)
// order.  Each pixel keeps one transmittance and colour per level; an entry of layer m
// is evaluated once (its alpha is the same for every level) and blended into every
// level l >= m that has not stopped.  The image of level l is therefore exactly the
// single-level render of mask 1..l.  The paper's rate-distortion step renders every
// level per iteration (Sec. 3.3); this replaces L renders by one pass.
//
// The reverse pass keeps the per-level state too: per entry, each level that blended it
// is undone in turn, the colour and opacity partials summed over the levels, and the
// power derivative dL/dpower summed over the levels before it is turned into the mean
// and conic partials (they are linear in it).  One warp reduction per entry serves all
// levels.
#include <cuda_runtime.h>

#include "gc_tile.cuh"

namespace gc {

namespace {

// Forward: one CTA of 256 threads per tile, one pixel per thread (the forward layout);
// NL = number of levels (compile time, so that the per-level state fits in registers).
template <int TW, int TH, int NL>
__global__ void __launch_bounds__(256) k_blend_levels_fwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, int W, int H, RenderParams rp, LevelPtrs out, float *__restrict__ lv_T,
    uint32_t *__restrict__ lv_last) {
    constexpr int L = NL;
    const int ntx = rp.ntx;
    const float bg0 = rp.bg[0], bg1 = rp.bg[1], bg2 = rp.bg[2];
    __shared__ __align__(16) FwdSmem sm;
    __shared__ uint8_t lay[256];
    const int tile = blockIdx.x, tx = tile % ntx, ty = tile / ntx;
    const uint2 range = ranges[tile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lx, ly;
    pixel_of_thread<TW, TH>((int)threadIdx.x, lx, ly);
    const int px = tx * TW + lx, py = ty * TH + ly;
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const int n = (int)(range.y - range.x);
    const bool inside = px < W && py < H;
    uint32_t lv = inside ? ((1u << L) - 1u) : 0u;  // levels still blending
    uint32_t act = lv ? (1u << lane) : 0u;
    float T[NL], C0[NL], C1[NL], C2[NL];
    // Transmittance of the highest level still blending.  Level l blends a subset of level
    // l + 1's entries with the same alphas, so T[l] >= T[l + 1]: the levels still blending
    // are always 0..k, only level k can be the first to stop, and an entry that reaches any
    // of them reaches level k.  Ttop follows T[k] with the same operations, so one test
    // decides whether any level stops at an entry; the levels are only walked when one does.
    float Ttop = 1.f;
    uint32_t last[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        T[l] = 1.f;
        C0[l] = C1[l] = C2[l] = 0.f;
        last[l] = 0u;
    }
    for (int b = 0; b < n; b += 256) {
        if (__syncthreads_count(act != 0u) == 0) break;
        {
            const int idx = b + (int)threadIdx.x;
            if (idx < n) {
                const uint32_t r = sorted_vals[range.x + idx] & list_rank_mask(rp);
                const float4 a = ranked[kRec * (size_t)r];
                const float4 bb = ranked[kRec * (size_t)r + 1];
                const float4 c = ranked[kRec * (size_t)r + 2];
                sm.a[threadIdx.x] = a;
                sm.b[threadIdx.x] = make_float2(bb.x, bb.y);
                sm.c[threadIdx.x] = make_float4(bb.z, bb.w, c.x, 0.f);
                store_entry_masks<TW, TH>(sm.m, (int)threadIdx.x, a, c, ranked[kRec * (size_t)r + 3], tx, ty, rp);
                lay[threadIdx.x] = (uint8_t)min(__float_as_int(c.y), 31);
            }
        }
        __syncthreads();
        const int cnt = min(256, n - b);
        for (int k0 = 0; k0 < cnt; k0 += 32) {
            // the entries of this group that can change a pixel of the warp: footprint
            // over one of its active pixels, layer at most the highest level still blending
            const uint32_t wact = __reduce_or_sync(0xffffffffu, act);
            if (wact == 0u) break;  // the whole warp is done
            const uint32_t wlv = __reduce_or_sync(0xffffffffu, lv);
            const int kq = k0 + lane;
            const bool rel = kq < cnt && (sm.m[warp * 256 + kq] & wact) != 0u && (wlv >> lay[kq]) != 0u;
            uint32_t todo = __ballot_sync(0xffffffffu, rel);
            while (todo) {
                const int k = k0 + __ffs(todo) - 1;
                todo &= todo - 1u;
                const uint32_t wm = sm.m[warp * 256 + k];
                const uint32_t lm = lv & (0xffffffffu << lay[k]);  // active levels >= the entry's layer
                const float4 a = sm.a[k];
                const float2 bb = sm.b[k];
                const float dx = pcx - a.x, dy = pcy - a.y;
                const float p2 = blend_power2(a.z, a.w, bb.x, dx, dy);
                float G;
                const float alpha = fminf(kAlphaMax, blend_raw_alpha(bb.y, p2, G));
                // one test instead of four branches: the pixel is in the entry's footprint, a level >= its
                // layer still blends, and the entry's alpha reaches 1/255 there
                const bool ok = ((wm & act) != 0u) & (lm != 0u) & (p2 <= 0.f) & (alpha >= kAlphaMin);
                if (!ok) continue;
                const float4 col = sm.c[k];
                const float om = 1.f - alpha;
                uint32_t bl = lm;  // the levels that blend the entry
                if (Ttop * om < kTStop) {
                    // some levels stop here: those whose transmittance would fall below the
                    // threshold (a top run of lm), then Ttop moves to the new highest level
#pragma unroll
                    for (int l = 0; l < NL; ++l)
                        if (((lm >> l) & 1u) && T[l] * om < kTStop) bl &= ~(1u << l);
                    lv &= ~(lm & ~bl);
#pragma unroll
                    for (int l = 0; l < NL; ++l)
                        if ((lv >> l) & 1u) Ttop = T[l];
                    if (!lv) act = 0u;
                }
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    if (!((bl >> l) & 1u)) continue;
                    const float w = alpha * T[l];
                    C0[l] = fmaf(col.x, w, C0[l]);
                    C1[l] = fmaf(col.y, w, C1[l]);
                    C2[l] = fmaf(col.z, w, C2[l]);
                    T[l] = T[l] * om;
                    last[l] = (uint32_t)(b + k + 1);
                }
                if (bl) Ttop = Ttop * om;
            }
        }
    }
    if (inside) {
        const size_t hw = (size_t)W * H;
        const size_t p = (size_t)py * W + px;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            float *img = out.img[l];
            img[p] = fmaf(T[l], bg0, C0[l]);
            img[hw + p] = fmaf(T[l], bg1, C1[l]);
            img[2 * hw + p] = fmaf(T[l], bg2, C2[l]);
            lv_T[l * hw + p] = T[l];
            lv_last[l * hw + p] = last[l];
        }
    }
}

constexpr int kPartStride = 73;  // words per entry of the reverse pass's partial staging

// Shared memory of the reverse pass (dynamic: past 48 KB at eight levels).
template <int NL>
struct LvBwdSmem {
    float4 a[256];
    float2 b[256];
    float4 c[256];
    float2 d[256];
    uint32_t m[256 * 8];
    uint32_t e[256];
    uint8_t lay[256];
    // per entry of the group: 8 warps x 9 partials at a stride of 73 words, so that the
    // cross-warp sum (thread i reads entry i / 9, partial i % 9) hits bank i mod 32
    float wpart[64 * kPartStride];
    // per entry of the group and warp: partial written; byte (warp & 3) of word
    // wrote[warp >> 2][entry], so that the 32 lanes of a relevance step write 32
    // consecutive words (distinct banks)
    uint32_t wrote[2][64];
    uint32_t last[NL][256];    // per level and pixel: list position after the last blend
    uint32_t wsuf[8][16];      // per warp: max over its pixels and levels l >= m of last[l]
    uint32_t last_max;
};

// Reverse: one CTA of 256 threads per tile, one pixel per thread; NL levels.
//
// Per pixel and level the reverse step of Eq. 2 needs the transmittance T_l before the entry
// and g_l . (c - A_l), with A_l the colour accumulated behind the entry; only the scalar
// B_l = g_l . A_l is kept (B_l <- B_l + alpha (g_l . c - B_l) when the level blends the
// entry, B_l = g_l . bg at the start), so a pixel's state is T_l, B_l and g_l per level.  The
// list positions after each level's last blended entry stay in shared memory (read only when
// the walk passes one of them).  A warp writes its 9 partials of an entry only when the entry
// passed its relevance ballot and records that in one byte per (entry, warp); the cross-warp
// sum adds the written ones in warp order, which gives the same bits as adding every warp
// with zeros for the others.
template <int TW, int TH, int NL>
__global__ void __launch_bounds__(256, 4) k_blend_levels_bwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, const uint32_t *__restrict__ offsets, int W, int H, RenderParams rp,
    const float *__restrict__ lv_T, const uint32_t *__restrict__ lv_last, LevelGrads dimg,
    float *__restrict__ part, uint8_t *__restrict__ flag) {
    extern __shared__ __align__(16) unsigned char lv_bwd_smem[];
    LvBwdSmem<NL> &sm = *reinterpret_cast<LvBwdSmem<NL> *>(lv_bwd_smem);
    const int tile = blockIdx.x, ntx = rp.ntx, tx = tile % ntx, ty = tile / ntx;
    const uint2 range = ranges[tile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int lx, ly;
    pixel_of_thread<TW, TH>((int)threadIdx.x, lx, ly);
    const int px = tx * TW + lx, py = ty * TH + ly;
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const uint32_t bit = 1u << lane;
    float T[NL], B[NL], g0[NL], g1[NL], g2[NL];
    uint32_t my_last = 0u;
    const size_t hw = (size_t)W * H;
    const bool inside = px < W && py < H;
    const size_t p = inside ? (size_t)py * W + px : 0;
    if (threadIdx.x == 0) sm.last_max = 0u;
    {
        uint32_t lastv[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            T[l] = 1.f;
            g0[l] = g1[l] = g2[l] = 0.f;
            lastv[l] = 0u;
            if (inside) {
                T[l] = lv_T[l * hw + p];
                lastv[l] = lv_last[l * hw + p];
                const float *gl = dimg.g[l];
                g0[l] = gl[p];
                g1[l] = gl[hw + p];
                g2[l] = gl[2 * hw + p];
                my_last = max(my_last, lastv[l]);
            }
            B[l] = fmaf(g2[l], rp.bg[2], fmaf(g1[l], rp.bg[1], g0[l] * rp.bg[0]));
            sm.last[l][threadIdx.x] = lastv[l];
        }
        uint32_t suf = 0u;
#pragma unroll
        for (int l = 15; l >= 0; --l) {
            if (l < NL) suf = max(suf, __reduce_max_sync(0xffffffffu, lastv[l < NL ? l : 0]));
            if (lane == 0) sm.wsuf[warp][l] = suf;
        }
    }
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, my_last);
    if (lane == 0) atomicMax(&sm.last_max, wmax);
    const uint32_t wpix = __ballot_sync(0xffffffffu, my_last != 0u);  // pixels of the warp with work
    // levels whose last blended position lies beyond the current entry: entries are visited in
    // decreasing position, so the set only grows; it is refreshed when the position drops below
    // the largest last position of a level not yet in it (at most once per level)
    uint32_t alive = 0u, next_last = my_last;
    __syncthreads();
    const int n_active = (int)sm.last_max;
    for (int hi = n_active; hi > 0; hi -= 256) {
        const int lo = max(hi - 256, 0);
        __syncthreads();
        {
            const int k = lo + (int)threadIdx.x;
            if (k < hi) {
                const uint32_t r = sorted_vals[range.x + k] & list_rank_mask(rp);
                const float4 a = ranked[kRec * (size_t)r];
                const float4 bb = ranked[kRec * (size_t)r + 1];
                const float4 c = ranked[kRec * (size_t)r + 2];
                RowGeom g;
                row_geom(a, c, ranked[kRec * (size_t)r + 3], rp, g);
                const float4 r4 = ranked[kRec * (size_t)r + 4];
                sm.a[threadIdx.x] = a;
                sm.b[threadIdx.x] = make_float2(bb.x, bb.y);
                sm.c[threadIdx.x] = make_float4(bb.z, bb.w, c.x, a.z * kUnscaleDiag);
                sm.d[threadIdx.x] = make_float2(a.w * kUnscaleOff, bb.x * kUnscaleDiag);
                if (rp.membership == GC_MEMBER_PIXEL && g.cull) {  // alpha-footprint block masks
#pragma unroll
                    for (int w = 0; w < 8; ++w)
                        sm.m[w * 256 + threadIdx.x] = block_alpha_mask<TW, TH>(g, tx, ty, w);
                } else {
                    uint32_t cm, rm;
                    rect_masks<TW, TH>(c, tx, ty, rp.membership, cm, rm);
                    store_masks_by_warp<TW>(sm.m, (int)threadIdx.x, cm, rm);
                }
                sm.e[threadIdx.x] = offsets[r] + entry_index(g, r4, tx, ty, rp, W, H);
                sm.lay[threadIdx.x] = (uint8_t)min(__float_as_int(c.y), 15);
            }
        }
        __syncthreads();
        for (int gtop = hi; gtop > lo; gtop -= 64) {
            const int gbot = max(gtop - 64, lo);
            for (int stop = gtop; stop > gbot; stop -= 32) {   // two halves of 32, upper first
                const int sbot = max(stop - 32, gbot);
                // entries of the half that a pixel of the warp blended at some level: footprint
                // over a pixel with work, and a level >= the entry's layer still past it
                const int kq = sbot + lane;
                bool rel = false;
                if (kq < stop) {
                    const int sq = kq - lo;
                    rel = (sm.m[warp * 256 + sq] & wpix) != 0u && (uint32_t)kq < sm.wsuf[warp][sm.lay[sq]];
                    reinterpret_cast<uint8_t *>(&sm.wrote[warp >> 2][kq - gbot])[warp & 3] = rel ? 1 : 0;
                }
                uint32_t todo = __ballot_sync(0xffffffffu, rel);
                while (todo) {
                    const int j = 31 - __clz(todo);
                    todo &= ~(1u << j);
                    const int k = sbot + j;
                    const int s = k - lo;
                    float v[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) v[c] = 0.f;
                    const uint32_t wm = sm.m[warp * 256 + s];
                    if ((uint32_t)k < next_last) {
                        alive = 0u;
                        next_last = 0u;
#pragma unroll
                        for (int l = 0; l < NL; ++l) {
                            const uint32_t ll = sm.last[l][threadIdx.x];
                            if ((uint32_t)k < ll) alive |= 1u << l;
                            else next_last = max(next_last, ll);
                        }
                    }
                    // levels of this pixel that blended entry k: alive ones at or above its layer
                    const uint32_t lm = alive & (0xffffffffu << sm.lay[s]);
                    {
                        const float4 a = sm.a[s];
                        const float2 bb = sm.b[s];
                        const float dx = pcx - a.x, dy = pcy - a.y;
                        const float p2 = blend_power2(a.z, a.w, bb.x, dx, dy);
                        float G;
                        const float a0 = blend_raw_alpha(bb.y, p2, G);
                        const float alpha = fminf(kAlphaMax, a0);
                        // one test instead of nested branches: footprint, a level that blended
                        // it, and alpha at least 1/255
                        const bool blended =
                            ((wm & bit) != 0u) & (lm != 0u) & (p2 <= 0.f) & (alpha >= kAlphaMin);
                        if (blended) {
                            const float4 col = sm.c[s];
                            // sums over the levels that blended the entry; the per-entry factors
                            // alpha and G multiply them once
                            float s0 = 0.f, s1 = 0.f, s2 = 0.f, sal = 0.f;
                            const float inv_oma = __fdividef(1.f, 1.f - alpha);
#pragma unroll
                            for (int l = 0; l < NL; ++l) {
                                if (!((lm >> l) & 1u)) continue;
                                T[l] = T[l] * inv_oma;
                                s0 = fmaf(T[l], g0[l], s0);
                                s1 = fmaf(T[l], g1[l], s1);
                                s2 = fmaf(T[l], g2[l], s2);
                                const float gc = fmaf(g2[l], col.z, fmaf(g1[l], col.y, g0[l] * col.x));
                                const float dl = gc - B[l];
                                sal = fmaf(T[l], dl, sal);
                                B[l] = fmaf(alpha, dl, B[l]);
                            }
                            v[6] = alpha * s0;
                            v[7] = alpha * s1;
                            v[8] = alpha * s2;
                            float dp = 0.f;  // dL/dpower (natural exponent), summed over levels
                            if (!(a0 > kAlphaMax)) {
                                v[5] = G * sal;
                                dp = alpha * sal;
                            }
                            const float2 nd = sm.d[s];
                            v[0] = (col.w * dx + nd.x * dy) * dp;
                            v[1] = (nd.x * dx + nd.y * dy) * dp;
                            v[2] = -0.5f * dx * dx * dp;
                            v[3] = -dx * dy * dp;
                            v[4] = -0.5f * dy * dy * dp;
                        }
                    }
                    // the entry passed the warp's relevance ballot: some pixel nearly always
                    // blended it, so the reduction runs without a vote
                    float out0, out8;
                    {
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
                    float *wp = &sm.wpart[(k - gbot) * kPartStride + warp * 9];
                    if ((lane & 3) == 0) wp[lane >> 2] = out0;
                    if (lane == 1) wp[8] = out8;
                }
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < (gtop - gbot) * 9; idx += 256) {
                const int q = idx / 9, c = idx - q * 9;
                const uint2 wr = make_uint2(sm.wrote[0][q], sm.wrote[1][q]);
                float acc = 0.f;
#pragma unroll
                for (int w2 = 0; w2 < 8; ++w2) {
                    const uint32_t byte = ((w2 < 4 ? wr.x : wr.y) >> (8 * (w2 & 3))) & 0xffu;
                    if (byte) acc += sm.wpart[q * kPartStride + w2 * 9 + c];
                }
                const uint32_t e = sm.e[gbot + q - lo];
                if (!flag) {
                    part[(int64_t)e * 9 + c] = acc;
                } else if (acc != 0.f) {  // the buffer holds zeros: a zero partial needs no store
                    part[(int64_t)e * 9 + c] = acc;
                    flag[e] = 1;
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_blend_levels_fwd(const uint2 *ranges, const uint32_t *sorted_vals, const float4 *ranked,
                                    const CamParams &cam, const RenderParams &rp, int L, const LevelPtrs &out,
                                    float *lv_T, uint32_t *lv_last, cudaStream_t st) {
    const unsigned tiles = (unsigned)(rp.ntx * rp.nty);
    if (tiles == 0) return cudaSuccess;
#define GC_LV_ARGS ranges, sorted_vals, ranked, cam.width, cam.height, rp, out, lv_T, lv_last
#define GC_LV_CASE(NLV)                                                                                       \
    case NLV:                                                                                                 \
        if (rp.tile_w == 16) k_blend_levels_fwd<16, 16, NLV><<<tiles, 256, 0, st>>>(GC_LV_ARGS);             \
        else if (rp.tile_w == 8) k_blend_levels_fwd<8, 32, NLV><<<tiles, 256, 0, st>>>(GC_LV_ARGS);          \
        else k_blend_levels_fwd<32, 8, NLV><<<tiles, 256, 0, st>>>(GC_LV_ARGS);                               \
        break;
    switch (L) {
        GC_LV_CASE(1) GC_LV_CASE(2) GC_LV_CASE(3) GC_LV_CASE(4) GC_LV_CASE(5) GC_LV_CASE(6) GC_LV_CASE(7)
        GC_LV_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef GC_LV_CASE
#undef GC_LV_ARGS
    note_launches(1);
    return cudaGetLastError();
}

namespace {

// One reverse-pass launch; the shared memory is dynamic, with the opt-in where it passes 48 KB.
template <int TW, int TH, int NL>
cudaError_t lv_bwd_launch(unsigned tiles, cudaStream_t st, const uint2 *ranges, const uint32_t *sorted_vals,
                          const float4 *ranked, const uint32_t *offsets, int W, int H, const RenderParams &rp,
                          const float *lv_T, const uint32_t *lv_last, const LevelGrads &dimg, float *part,
                          uint8_t *flag) {
    constexpr size_t bytes = sizeof(LvBwdSmem<NL>);
    if constexpr (bytes > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_blend_levels_bwd<TW, TH, NL>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
    }
    k_blend_levels_bwd<TW, TH, NL><<<tiles, 256, bytes, st>>>(ranges, sorted_vals, ranked, offsets, W, H, rp, lv_T,
                                                               lv_last, dimg, part, flag);
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_blend_levels_bwd(const uint2 *ranges, const uint32_t *sorted_vals, const float4 *ranked,
                                    const uint32_t *offsets, const CamParams &cam, const RenderParams &rp, int L,
                                    const float *lv_T, const uint32_t *lv_last, const LevelGrads &dimg,
                                    float *part, uint8_t *flag, cudaStream_t st) {
    const unsigned tiles = (unsigned)(rp.ntx * rp.nty);
    if (tiles == 0) return cudaSuccess;
#define GC_LV_ARGS ranges, sorted_vals, ranked, offsets, cam.width, cam.height, rp, lv_T, lv_last, dimg, part, flag
#define GC_LV_CASE(NLV)                                                                                       \
    case NLV:                                                                                                 \
        e = rp.tile_w == 16  ? lv_bwd_launch<16, 16, NLV>(tiles, st, GC_LV_ARGS)                              \
            : rp.tile_w == 8 ? lv_bwd_launch<8, 32, NLV>(tiles, st, GC_LV_ARGS)                               \
                             : lv_bwd_launch<32, 8, NLV>(tiles, st, GC_LV_ARGS);                              \
        break;
    cudaError_t e;
    switch (L) {
        GC_LV_CASE(1) GC_LV_CASE(2) GC_LV_CASE(3) GC_LV_CASE(4) GC_LV_CASE(5) GC_LV_CASE(6) GC_LV_CASE(7)
        GC_LV_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef GC_LV_CASE
#undef GC_LV_ARGS
    if (e != cudaSuccess) return e;
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace gc
