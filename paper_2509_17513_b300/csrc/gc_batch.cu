// gc_batch.cu - batched forward and backward over many requests (camera, resolution,
// motion frame, layer mask) of one Gaussian set: the per-step workload of the
// paper's layer-wise rate-distortion training (Sec. 3.3) and of multi-view playback.
//
// Layout.  Requests are concatenated in every index space, each padded to the radix
// tile (radix_tile_keys() keys) so that no sort block straddles two requests:
//   items    (request, selected Gaussian) pairs, request-major, padded;
//   entries  (tile, Gaussian) pairs, request-major, each request padded (pad keys sort
//            last and are never referenced by a tile range);
//   tiles    request-major global tile index; pixels request-major.
// Steps (all on one stream, no host sync with a fixed key capacity):
//   preprocess over all items -> segmented depth sort (each request on its own) ->
//   rank gather -> scan of tiles touched -> per-request entry bases -> emit -> pad fill
//   -> segmented tile sort (local tile ids) -> per-request tile ranges from the sorted
//   keys -> persistent blend: CTAs take tiles of all images from a work counter (an
//   atomic ticket, no waiting on other CTAs).
// Every image equals the single-request render bit for bit: the same projection, the
// same stable orders and the same per-tile blend run on the same data.
#include <cuda_runtime.h>

#include "gc_bucket.cuh"
#include "gc_chain.cuh"
#include "gc_project.cuh"
#include "gc_state.cuh"
#include "gc_tile.cuh"

namespace gc {

struct __align__(16) BatchReq {
    CamParams cam;
    RenderParams rp;
    Selection sel;
    int64_t n_sel;
    int64_t item_base;
    int64_t tile_base;
    int64_t pixel_base;
    int64_t row_base;   // row binning: global tile row of the request's row 0
    int64_t cell_base;  // row binning: first (row, chunk) cell of the request
    int64_t n_chunks;   // row binning: chunks of 32 items (the request's padded items / 32)
    const float *group_q, *group_t;
    int n_groups;
    int frame;
    float *image;
    Residual res;  // the frame's residual deformation
};

namespace {

// Grid of a persistent kernel: every CTA (of `threads`) that fits on the device at once,
// queried once per kernel (the device's SM count times resident CTAs per SM).
template <auto Kernel, int threads>
int64_t persistent_grid() {
    static int64_t cached = 0;
    if (!cached) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, threads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 4;
        cudaGetLastError();
        cached = (int64_t)sms * per_sm;
    }
    return cached;
}

// Last q with base[q] <= x, over q in [0, n).
__device__ __forceinline__ int find_req(const int64_t *base, int n, int64_t x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Row binning over a batch (gc_bucket.cuh): chunk c = items 32 c .. 32 c + 31 (requests are
// padded to radix tiles, so a chunk never straddles two), cells and global rows request by
// request, tiles at the request's tile base.
struct BatchBucketMap {
    const BatchReq *reqs;
    const int64_t *item_base, *row_base;
    int n_req;
    __device__ __forceinline__ void chunk(int64_t c, BucketChunk &ci) const {
        const int64_t item = c * 32;
        const BatchReq &R = reqs[find_req(item_base, n_req, item)];
        ci.rp = R.rp;
        ci.W = R.cam.width;
        ci.H = R.cam.height;
        ci.n_rows = R.rp.nty;
        ci.cell0 = R.cell_base + (item - R.item_base) / 32;
        ci.stride = R.n_chunks;
        ci.row0 = R.row_base;
        ci.r0 = item;
        ci.v0 = item - R.item_base;  // list words hold the rank within the request
        const int64_t left = R.n_sel - (item - R.item_base);
        ci.n_valid = left <= 0 ? 0 : (left < 32 ? (int)left : 32);
    }
    __device__ __forceinline__ void row(int64_t gr, BucketRow &ri) const {
        const BatchReq &R = reqs[find_req(row_base, n_req, gr)];
        const int64_t y = gr - R.row_base;
        ri.cell = R.cell_base + y * R.n_chunks;
        ri.n_cells = R.n_chunks;
        ri.tile0 = R.tile_base + y * R.rp.ntx;
        ri.ntx = R.rp.ntx;
    }
};

// The request-independent activations of every Gaussian (scales, alpha level), once per batch.
template <int PREC>
__global__ void __launch_bounds__(256) k_batch_activate(GaussSrc G, int64_t n, float4 *__restrict__ act) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) act[i] = gaussian_activation<PREC>(G, i);
}

template <int PREC>
__global__ void __launch_bounds__(256, 4) k_batch_preprocess(GaussSrc G, const BatchReq *__restrict__ reqs,
                                                          const int64_t *__restrict__ item_base, int n_req,
                                                          int64_t n_items, float4 *__restrict__ rec,
                                                          uint32_t *__restrict__ keys,
                                                          uint32_t *__restrict__ vals,
                                                          uint32_t *__restrict__ touched,
                                                          const float4 *__restrict__ act) {
    // a block's 256 items belong to one request (requests are padded to the radix tile):
    // its table entry is staged in shared memory once
    __shared__ __align__(16) BatchReq R;
    {
        const int64_t first = (int64_t)blockIdx.x * blockDim.x;
        const int q = find_req(item_base, n_req, first);
        const int4 *src = reinterpret_cast<const int4 *>(&reqs[q]);
        int4 *dst = reinterpret_cast<int4 *>(&R);
        for (int k = threadIdx.x; k < (int)(sizeof(BatchReq) / 16); k += blockDim.x) dst[k] = src[k];
        __syncthreads();
    }
    const int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= n_items) return;
    const int64_t j = item - R.item_base;
    vals[item] = (uint32_t)item;
    Proj P;
    if (j < R.n_sel) {
        project_gaussian<PREC>(G, sel_global(R.sel, j), R.group_q, R.group_t, R.n_groups, R.cam, R.rp, P, act, R.res);
    } else {
        P.key = kCulledKey;
        P.ntouch = 0;
        P.r0 = P.r1 = P.r2 = P.r3 = P.r4 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    rec[kRec * item] = P.r0;
    rec[kRec * item + 1] = P.r1;
    if (j < R.n_sel) P.r2.y = __int_as_float(layer_of(R.sel, sel_global(R.sel, j)));
    rec[kRec * item + 2] = P.r2;
    const uint32_t nt = bin_rows(P, R.rp, R.cam.width, R.cam.height);
    rec[kRec * item + 3] = P.r3;
    rec[kRec * item + 4] = P.r4;
    keys[item] = P.key;
    touched[item] = nt;
}

// Per request: entry count K_q, padded entry base, the shift from the unpadded scan
// offsets, and the entry segments in radix-block units.  words[2] = padded total.
// If the padded total exceeds `cap`, every entry segment is made empty so that the
// tile sort stays inside its buffers (nothing is emitted; gc_check reports it).
__global__ void k_batch_entry_bases(const uint32_t *__restrict__ offsets, const uint32_t *total,
                                    const int64_t *__restrict__ item_base, int n_req, int64_t n_items,
                                    uint32_t tile_keys, uint32_t cap, uint32_t *__restrict__ ebase,
                                    uint32_t *__restrict__ eshift, uint32_t *__restrict__ ecount,
                                    uint32_t *__restrict__ seg_entries, uint32_t *words) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    auto off = [&](int64_t idx) -> uint32_t { return idx < n_items ? offsets[idx] : *total; };
    uint64_t eb = 0;
    for (int q = 0; q < n_req; ++q) {
        const uint32_t a = off(item_base[q]), b = off(item_base[q + 1]);
        const uint64_t kq = b - a;
        ebase[q] = (uint32_t)eb;
        eshift[q] = (uint32_t)(eb - a);
        ecount[q] = (uint32_t)kq;
        seg_entries[q] = (uint32_t)(eb / tile_keys);
        eb += (kq + tile_keys - 1) / tile_keys * tile_keys;
    }
    const uint32_t padded = (uint32_t)(eb > 0xFFFFFFFFull ? 0xFFFFFFFFull : eb);
    ebase[n_req] = padded;
    seg_entries[n_req] = (uint32_t)(eb / tile_keys);
    if (padded > cap)
        for (int q = 0; q <= n_req; ++q) seg_entries[q] = 0u;
    words[2] = padded;
}

// One warp emits the entries of 32 consecutive ranks (one request: requests are
// padded to the radix tile); entry e = offsets[r] + eshift[q] + index of the tile among
// the Gaussian's row intervals; key = the request's local tile id, value = r.
__global__ void __launch_bounds__(256) k_batch_emit(const float4 *__restrict__ ranked,
                                                    const uint32_t *__restrict__ offsets,
                                                    const uint32_t *__restrict__ touched_r,
                                                    const BatchReq *__restrict__ reqs,
                                                    const int64_t *__restrict__ item_base, int n_req,
                                                    const uint32_t *__restrict__ eshift, int64_t n,
                                                    uint32_t cap, const uint32_t *padded_total,
                                                    uint32_t *__restrict__ keys,
                                                    uint32_t *__restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const int64_t wbase = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) - lane;
    if (wbase >= n) return;
    if (*padded_total > cap) return;  // overflow: reported by gc_check, nothing emitted
    const int q = find_req(item_base, n_req, wbase);
    const BatchReq &R = reqs[q];
    emit_rows_warp(ranked, wbase, n, offsets, touched_r, eshift[q], R.rp, R.cam.width, R.cam.height, cap, keys,
                   vals);
}

// Pad keys after every request's entries (they sort to the end of the segment).
__global__ void k_batch_pad_fill(const uint32_t *__restrict__ ebase, const uint32_t *__restrict__ ecount,
                                 uint32_t cap, const uint32_t *padded_total, uint32_t *__restrict__ keys,
                                 uint32_t *__restrict__ vals) {
    if (*padded_total > cap) return;
    const int q = blockIdx.x;
    const uint32_t a = ebase[q] + ecount[q], b = ebase[q + 1];
    for (uint32_t e = a + threadIdx.x; e < b; e += blockDim.x) {
        keys[e] = 0xffffffffu;
        vals[e] = 0u;
    }
}

// Tile ranges from the segment-sorted keys (each request's keys sorted within its segment
// [ebase[q], ebase[q] + ecount[q]), pad keys after it): a key that differs from its
// predecessor in the segment starts its tile's range, one that differs from its successor
// ends it.  Ranges of tiles without entries stay as zeroed.  Nothing when the padded total
// overflowed the capacity.  Each thread takes four consecutive keys (one 16-byte load); a
// warp's 128 keys lie in one segment (segments are 2048-aligned), whose request lane 0
// looks up once.
__global__ void __launch_bounds__(256) k_batch_key_ranges(const uint32_t *__restrict__ keys,
                                                          const uint32_t *__restrict__ ebase,
                                                          const uint32_t *__restrict__ ecount,
                                                          const int64_t *__restrict__ tile_base, int n_req,
                                                          const uint32_t *padded_total, uint32_t cap,
                                                          uint2 *__restrict__ ranges) {
    const uint32_t total = *padded_total;
    if (total > cap) return;
    const int lane = threadIdx.x & 31;
    const int64_t n4 = (int64_t)total >> 2;  // the padded total is a multiple of 2048
    for (int64_t qd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; qd - lane < n4;
         qd += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = 4 * qd;
        int req = 0;
        if (lane == 0) {  // the last request whose segment starts at or before the warp's first key
            int lo = 0, hi = n_req - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int64_t)ebase[mid] <= p) lo = mid; else hi = mid - 1;
            }
            req = lo;
        }
        req = __shfl_sync(0xffffffffu, req, 0);
        const bool in = qd < n4;
        uint4 v = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
        if (in) v = reinterpret_cast<const uint4 *>(keys)[qd];
        uint32_t prev = __shfl_up_sync(0xffffffffu, v.w, 1);
        uint32_t next = __shfl_down_sync(0xffffffffu, v.x, 1);
        if (!in) continue;
        const int64_t a = ebase[req], e = a + ecount[req];
        if (lane == 0 && p > a) prev = keys[p - 1];
        if ((lane == 31 || qd + 1 >= n4) && p + 4 < e) next = keys[p + 4];
        uint2 *out = ranges + tile_base[req];
        const uint32_t k[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t pt = p + t;
            if (pt >= e) break;  // padding
            const uint32_t before = t == 0 ? prev : k[t - 1];
            const uint32_t after = t == 3 ? next : k[t + 1];
            if (pt == a || before != k[t]) out[k[t]].x = (uint32_t)pt;
            if (pt + 1 == e || after != k[t]) out[k[t]].y = (uint32_t)(pt + 1);
        }
    }
}

// Persistent blend: each CTA repeatedly takes the next global tile from the work
// counter (atomic ticket) and blends it with its request's parameters.
template <int TW, int TH>
__global__ void __launch_bounds__(256) k_batch_blend_fwd(const BatchReq *__restrict__ reqs,
                                                         const int64_t *__restrict__ tile_base, int n_req,
                                                         int64_t n_tiles, const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ sorted_vals,
                                                         const float4 *__restrict__ ranked,
                                                         float *__restrict__ final_T,
                                                         uint32_t *__restrict__ n_contrib,
                                                         unsigned long long *counter) {
    __shared__ __align__(16) FwdSmem sm;
    __shared__ TileOut s_out;
    __shared__ int4 s_tile;  // tx, ty, range start, range end (tx < 0: no tile left)
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(counter, 1ull);
            if (t < n_tiles) {
                const int q = find_req(tile_base, n_req, t);
                const BatchReq &R = reqs[q];
                const int local = (int)(t - R.tile_base);
                const uint2 rg = ranges[t];
                s_tile = make_int4(local % R.rp.ntx, local / R.rp.ntx, (int)rg.x, (int)rg.y);
                s_out = TileOut{R.image, final_T + R.pixel_base, n_contrib + R.pixel_base, nullptr, nullptr,
                                R.rp.bg[0], R.rp.bg[1], R.rp.bg[2], R.cam.width, R.cam.height, R.rp.membership,
                                list_rank_mask(R.rp), R.rp.list_packed ? (uint32_t)R.item_base : 0u};
            } else {
                s_tile = make_int4(-1, 0, 0, 0);
            }
        }
        __syncthreads();
        const int4 tl = s_tile;
        if (tl.x < 0) break;
        blend_fwd_tile<TW, TH, false>(tl.x, tl.y, make_uint2((uint32_t)tl.z, (uint32_t)tl.w), sorted_vals, ranked,
                                      s_out, sm);
        __syncthreads();
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(kBwdThreads, 6) k_batch_blend_bwd(const BatchReq *__restrict__ reqs,
                                                         const int64_t *__restrict__ tile_base, int n_req,
                                                         int64_t n_tiles, const uint2 *__restrict__ ranges,
                                                         const uint32_t *__restrict__ sorted_vals,
                                                         const float4 *__restrict__ ranked,
                                                         const uint32_t *__restrict__ offsets,
                                                         const uint32_t *__restrict__ eshift,
                                                         const float *__restrict__ final_T,
                                                         const uint32_t *__restrict__ n_contrib,
                                                         const float *const *__restrict__ dimgs,
                                                         float *__restrict__ part, uint8_t *__restrict__ flag,
                                                         unsigned long long *counter) {
    __shared__ __align__(16) BwdSmem sm;
    __shared__ TileBwd s_in;
    __shared__ int4 s_tile;    // tx, ty, range start, range end (tx < 0: no tile left)
    for (;;) {
        if (threadIdx.x == 0) {
            const long long t = (long long)atomicAdd(counter, 1ull);
            if (t < n_tiles) {
                const int q = find_req(tile_base, n_req, t);
                const BatchReq &R = reqs[q];
                const int local = (int)(t - R.tile_base);
                const uint2 rg = ranges[t];
                s_tile = make_int4(local % R.rp.ntx, local / R.rp.ntx, (int)rg.x, (int)rg.y);
                s_in = TileBwd{final_T + R.pixel_base, n_contrib + R.pixel_base, dimgs[q], R.rp, R.cam.width,
                               R.cam.height, eshift[q], R.rp.list_packed ? (uint32_t)R.item_base : 0u, flag};
            } else {
                s_tile = make_int4(-1, 0, 0, 0);
            }
        }
        __syncthreads();
        const int4 tl = s_tile;
        if (tl.x < 0) break;
        blend_bwd_tile<TW, TH>(tl.x, tl.y, make_uint2((uint32_t)tl.z, (uint32_t)tl.w), sorted_vals, ranked, offsets,
                               s_in, part, sm);
        __syncthreads();
    }
}

// One warp per rank: the Gaussian's partials over its tiles -> g2d at its item.
__global__ void __launch_bounds__(256) k_batch_reduce(float *__restrict__ part,
                                                      const uint32_t *__restrict__ offsets,
                                                      const uint32_t *__restrict__ touched_r,
                                                      const uint32_t *__restrict__ perm,
                                                      const int64_t *__restrict__ item_base, int n_req,
                                                      const uint32_t *__restrict__ eshift, int64_t n, uint32_t cap,
                                                      uint8_t *__restrict__ flag, float *__restrict__ g2d) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    const uint32_t cnt = touched_r[r];
    const uint32_t base = cnt ? offsets[r] + eshift[find_req(item_base, n_req, r)] : 0u;
    float out0, out8;
    reduce_entries_warp(part, base, cnt, cap, flag, out0, out8);
    store_reduced(g2d + 9 * (int64_t)perm[r], out0, out8);
}

// Compact position of global Gaussian i in a selection, or -1.
__device__ __forceinline__ int64_t sel_local(const Selection &s, int64_t i) {
    for (int k = 0; k < s.n_ranges; ++k) {
        const int64_t len = s.range_start[k + 1] - s.range_start[k];
        if (i >= s.range_begin[k] && i < s.range_begin[k] + len) return s.range_start[k] + (i - s.range_begin[k]);
    }
    return -1;
}

// Thread per Gaussian: the chain rule for every request that sees it, summed in
// request order; per-item motion terms for the group sums.
template <int PREC>
__global__ void __launch_bounds__(128) k_batch_preprocess_bwd(GaussSrc G, const BatchReq *__restrict__ reqs,
                                                              int n_req, int64_t n,
                                                              const float *__restrict__ g2d,
                                                              const uint32_t *__restrict__ touched,
                                                              gc_grads out, int accumulate,
                                                              float *__restrict__ mcontrib) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int K3 = 3 * G.K;
    GradAcc acc;
    for (int k = 0; k < 3; ++k) { acc.dmu[k] = 0.f; acc.dls[k] = 0.f; }
    for (int k = 0; k < 4; ++k) acc.dq[k] = 0.f;
    acc.dlogit = 0.f;
    for (int k = 0; k < K3; ++k) acc.dsh[k] = 0.f;
    const int g = G.group_id ? G.group_id[i] : 0;
    for (int q = 0; q < n_req; ++q) {
        const BatchReq &R = reqs[q];
        if (R.n_sel == 0) continue;
        const int64_t j = sel_local(R.sel, i);
        if (j < 0) continue;
        const int64_t item = R.item_base + j;
        float m7[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (touched[item] != 0)
            chain_rule<PREC>(G, i, R.group_q, R.group_t, g, R.cam, R.rp, g2d + 9 * item, acc, m7, R.res);
        if (mcontrib)
            for (int k = 0; k < 7; ++k) mcontrib[7 * item + k] = m7[k];
    }
    auto put = [accumulate](float *p, float v) { *p = accumulate ? __fadd_rn(*p, v) : v; };
    if (out.d_means) for (int k = 0; k < 3; ++k) put(&out.d_means[3 * i + k], acc.dmu[k]);
    if (out.d_log_scales) for (int k = 0; k < 3; ++k) put(&out.d_log_scales[3 * i + k], acc.dls[k]);
    if (out.d_quats) for (int k = 0; k < 4; ++k) put(&out.d_quats[4 * i + k], acc.dq[k]);
    if (out.d_opacity_logits) put(&out.d_opacity_logits[i], acc.dlogit);
    if (out.d_sh) for (int k = 0; k < K3; ++k) put(&out.d_sh[i * K3 + k], acc.dsh[k]);
}

constexpr int kBatchChunk = 256;

// Per chunk of 256 items (one request), per group: the motion terms of the chunk's
// members in item order.  Keyframe requests and padding contribute zero.
__global__ void __launch_bounds__(128) k_batch_group_partial(const float *__restrict__ mcontrib,
                                                             const int32_t *__restrict__ group_id,
                                                             const BatchReq *__restrict__ reqs,
                                                             const int64_t *__restrict__ item_base, int n_req,
                                                             int n_groups, float *__restrict__ partial) {
    __shared__ int s_gid[kBatchChunk];
    __shared__ float s_val[kBatchChunk * 7];
    const int64_t base = (int64_t)blockIdx.x * kBatchChunk;
    const int q = find_req(item_base, n_req, base);
    const BatchReq &R = reqs[q];
    const int64_t j0 = base - R.item_base;
    const bool use = R.frame >= 0;
    for (int k = threadIdx.x; k < kBatchChunk; k += blockDim.x) {
        const int64_t j = j0 + k;
        s_gid[k] = (use && j < R.n_sel) ? (group_id ? group_id[sel_global(R.sel, j)] : 0) : -1;
    }
    for (int k = threadIdx.x; k < kBatchChunk * 7; k += blockDim.x) s_val[k] = mcontrib[base * 7 + k];
    __syncthreads();
    for (int gg = threadIdx.x; gg < n_groups; gg += blockDim.x) {
        float a[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < kBatchChunk; ++k) {
            if (s_gid[k] == gg) {
#pragma unroll
                for (int c = 0; c < 7; ++c) a[c] += s_val[7 * k + c];
            }
        }
        float *o = partial + ((int64_t)blockIdx.x * n_groups + gg) * 7;
#pragma unroll
        for (int c = 0; c < 7; ++c) o[c] = a[c];
    }
}

// Thread per (frame, group, component): requests of that frame in order, their chunks in order.
__global__ void k_batch_group_final(const float *__restrict__ partial, const BatchReq *__restrict__ reqs,
                                    const int64_t *__restrict__ item_base, int n_req, int n_frames,
                                    int n_groups, int accumulate, float *__restrict__ d_gq,
                                    float *__restrict__ d_gt) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_frames * n_groups * 7) return;
    const int f = id / (n_groups * 7), rest = id - f * n_groups * 7;
    const int g = rest / 7, c = rest - g * 7;
    float acc = 0.f;
    for (int q = 0; q < n_req; ++q) {
        if (reqs[q].frame != f) continue;
        const int64_t c0 = item_base[q] / kBatchChunk, c1 = item_base[q + 1] / kBatchChunk;
        for (int64_t ch = c0; ch < c1; ++ch) acc += partial[(ch * n_groups + g) * 7 + c];
    }
    float *p = nullptr;
    if (c < 4) {
        if (d_gq) p = &d_gq[((int64_t)f * n_groups + g) * 4 + c];
    } else if (d_gt) {
        p = &d_gt[((int64_t)f * n_groups + g) * 3 + (c - 4)];
    }
    if (p) *p = accumulate ? __fadd_rn(*p, acc) : acc;
}

}  // namespace
}  // namespace gc


// --------------------------------------------------------------------------- host side

struct BatchState {
    bool valid = false;
    bool bound = false;  // captured into a CUDA graph: buffers and request table are fixed
    int n_req = 0, n_frames = 0, n_groups = 1;
    bool has_motion = false;
    int64_t n = 0;
    int sh_degree = 0, n_layers = 0;
    std::vector<gc::BatchReq> reqs;    // request table on the device (last upload)
    std::vector<const float *> dimgs;  // dL/dimage pointers on the device (last upload)
    gc::BatchReq *staging = nullptr;   // pinned upload buffers
    size_t staging_cap = 0;
    int64_t *staging_base = nullptr;
    size_t staging_base_cap = 0;
    const float **staging_dimg = nullptr;
    size_t staging_dimg_cap = 0;
    cudaEvent_t staged = nullptr;      // last upload from the pinned buffers
    int64_t n_items = 0, n_tiles = 0, n_pixels = 0, K_cap = 0;
    int key_bits = 1, depth_buf = 0, tile_buf = 0;
    bool k_exact = false;
    bool row_binned = false;  // lists binned by tile row (one word per entry, in tkeys)
    gc_options opt{};
    DevBuf reqs_dev, item_base, tile_base, seg_items, ebase, eshift, ecount, seg_entries, dimg_dev;
    DevBuf row_base, row_shift;  // row binning: per request its first global tile row; per row the pad shift
    // The sorted tile lists: one word per entry (column << 24 | rank within the request) in the
    // last pass's keys when binned by tile row, else the values of the key sort.
    uint32_t *lists() const {
        return row_binned ? tkeys[tile_buf].as<uint32_t>() : tvals[tile_buf].as<uint32_t>();
    }
    DevBuf rec, ranked, dkeys[2], dvals[2], touched, touched_r, offsets, tkeys[2], tvals[2], ranges,
        final_T, n_contrib, words, counter, scratch, act;
    DevBuf part, flag, g2d, mcontrib, gpartial;
    bool part_clean = false;  // part and flag (one byte per entry) hold only zeros (see the reduce)

    ~BatchState() {
        DevBuf *bufs[] = {&reqs_dev, &item_base, &tile_base, &seg_items, &ebase, &eshift, &ecount,
                          &seg_entries, &dimg_dev, &row_base, &row_shift, &rec, &ranked, &dkeys[0], &dkeys[1], &dvals[0],
                          &dvals[1], &touched, &touched_r, &offsets, &tkeys[0], &tkeys[1], &tvals[0],
                          &tvals[1], &ranges, &final_T, &n_contrib, &words, &counter, &scratch, &act,
                          &part, &flag, &g2d, &mcontrib, &gpartial};
        for (DevBuf *b : bufs) release(*b);
        if (staging) cudaFreeHost(staging);
        if (staging_base) cudaFreeHost(staging_base);
        if (staging_dimg) cudaFreeHost(staging_dimg);
        if (staged) cudaEventDestroy(staged);
    }
};

namespace {

template <class T>
gc_status grow_pinned(gc_context *ctx, T *&p, size_t &cap, size_t count) {
    if (count <= cap && p) return GC_OK;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    if (cudaHostAlloc((void **)&p, count * sizeof(T), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GC_ERR_OOM, "pinned staging allocation failed");
    }
    cap = count;
    return GC_OK;
}

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusActive;
}

// Buffer sizing: eager calls grow; a captured call or a state bound to a graph may
// only use buffers that are already large enough.
struct Sizer {
    gc_context *ctx;
    bool fixed;
    gc_status st = GC_OK;
    bool operator()(DevBuf &b, size_t bytes) {
        if (st != GC_OK) return false;
        if (b.p && bytes <= b.cap) return true;
        if (fixed) {
            st = fail(ctx, GC_ERR_STATE,
                      "a captured or graph-bound batch needs larger buffers than its eager call sized");
            return false;
        }
        const cudaError_t e = grow(b, bytes);
        if (e != cudaSuccess) {
            st = fail(ctx, e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA, "batch buffer: %s",
                      cudaGetErrorString(e));
            return false;
        }
        return true;
    }
};

gc_status build_table(gc_context *ctx, const gc_gaussians *g, const gc_motion *frames, int n_frames,
                      int n_groups, const gc_request *reqs, int n_req, const gc_options &o,
                      std::vector<gc::BatchReq> &tab, int64_t &items, int64_t &tiles, int64_t &pixels,
                      int &kbits, int64_t &rows, int64_t &cells, bool &rows_fit) {
    const int64_t T = gc::radix_tile_keys();
    tab.assign(n_req, gc::BatchReq{});
    items = tiles = pixels = rows = cells = 0;
    kbits = 1;
    rows_fit = true;
    for (int q = 0; q < n_req; ++q) {
        const gc_request &rq = reqs[q];
        const gc_camera *cam = &rq.camera;
        if (!rq.image) return fail(ctx, GC_ERR_INVALID_ARG, "request %d has no image", q);
        if (cam->width <= 0 || cam->height <= 0 || cam->width > 32768 || cam->height > 32768 ||
            !(cam->fx > 0.f) || !(cam->fy > 0.f))
            return fail(ctx, GC_ERR_INVALID_ARG, "request %d has an invalid camera", q);
        if (rq.frame < -1 || rq.frame >= n_frames)
            return fail(ctx, GC_ERR_INVALID_ARG, "request %d: frame %d out of range", q, rq.frame);
        gc::BatchReq &R = tab[q];
        memset(&R, 0, sizeof R);  // padding bytes too: tables are compared bytewise
        R.cam.width = cam->width;
        R.cam.height = cam->height;
        R.cam.fx = cam->fx;
        R.cam.fy = cam->fy;
        R.cam.cx = cam->cx;
        R.cam.cy = cam->cy;
        memcpy(R.cam.R, cam->R, sizeof R.cam.R);
        memcpy(R.cam.t, cam->t, sizeof R.cam.t);
        memcpy(R.cam.campos, cam->campos, sizeof R.cam.campos);
        R.rp.near_plane = o.near_plane;
        R.rp.dilation = o.dilation;
        R.rp.frustum_clamp = o.frustum_clamp;
        memcpy(R.rp.bg, o.bg, sizeof R.rp.bg);
        R.rp.tile_w = o.tile_w;
        R.rp.tile_h = o.tile_h;
        R.rp.tile_w_log2 = ilog2_exact(o.tile_w);
        R.rp.tile_h_log2 = ilog2_exact(o.tile_h);
        R.rp.ntx = (cam->width + o.tile_w - 1) / o.tile_w;
        R.rp.nty = (cam->height + o.tile_h - 1) / o.tile_h;
        R.rp.membership = o.membership;
        R.rp.alpha_cull = o.alpha_cull;
        int64_t n_sel = 0;
        R.sel = make_selection(g, rq.layer_mask, n_sel);
        R.n_sel = n_sel;
        R.item_base = items;
        const int64_t padded_items = (n_sel + T - 1) / T * T;
        items += padded_items;
        R.row_base = rows;
        rows += R.rp.nty;
        R.n_chunks = padded_items / 32;
        R.cell_base = cells;
        cells += (int64_t)R.rp.nty * R.n_chunks;
        rows_fit = rows_fit && gc::bucket_binning_fits(R.rp, n_sel);
        R.tile_base = tiles;
        tiles += (int64_t)R.rp.ntx * R.rp.nty;
        R.pixel_base = pixels;
        pixels += (int64_t)cam->width * cam->height;
        kbits = std::max(kbits, bits_for((int64_t)R.rp.ntx * R.rp.nty - 1));
        R.frame = rq.frame;
        R.n_groups = 1;
        if (rq.frame >= 0) {
            R.group_q = frames[rq.frame].q;
            R.group_t = frames[rq.frame].t;
            R.n_groups = n_groups;
            R.res = gc::Residual{frames[rq.frame].res_log_scales, frames[rq.frame].res_opacity_logits,
                                 frames[rq.frame].res_sh};
        }
        R.image = rq.image;
    }
    if (items > 0x7FFFFFFFll) return fail(ctx, GC_ERR_INVALID_ARG, "more than 2^31 - 1 (request, Gaussian) pairs");
    if (rows_fit)  // the lists of every request are binned by tile row (rank within the request)
        for (auto &R : tab) R.rp.list_packed = 1;
    return GC_OK;
}

}  // namespace

void batch_invalidate(gc_saved &S) {
    if (S.batch) S.batch->valid = false;
}

gc_status batch_check(gc_context *ctx, const gc_saved &S, cudaStream_t stream) {
    if (!S.batch || !S.batch->valid || !S.batch->words.p) return GC_OK;
    const BatchState &B = *S.batch;
    uint32_t w[3];
    GC_CUDA(ctx, cudaMemcpyAsync(w, B.words.p, 12, cudaMemcpyDeviceToHost, stream));
    GC_CUDA(ctx, cudaStreamSynchronize(stream));
    if (w[1]) {
        GC_CUDA(ctx, cudaMemsetAsync(static_cast<uint32_t *>(B.words.p) + 1, 0, 4, stream));
        return fail(ctx, GC_ERR_TIMEOUT, "a bounded device wait ran out (error word %#x)", w[1]);
    }
    if (!B.k_exact && (int64_t)w[2] > B.K_cap)
        return fail(ctx, GC_ERR_CAPACITY, "batch needs %u keys (padded), capacity %lld", w[2], (long long)B.K_cap);
    return GC_OK;
}

extern "C" gc_status gc_render_batch_forward(gc_context *ctx, const gc_gaussians *g,
                                             const gc_motion *frames, int32_t n_frames,
                                             const gc_request *reqs, int32_t n_req, gc_saved *saved,
                                             void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!reqs || n_req <= 0) return fail(ctx, GC_ERR_INVALID_ARG, "no requests");
    if (n_frames < 0 || (n_frames > 0 && !frames)) return fail(ctx, GC_ERR_INVALID_ARG, "bad motion frames");
    gc::GaussSrc src;
    gc_status st = make_source(ctx, g, n_frames > 0 ? &frames[0] : nullptr, src);
    if (st != GC_OK) return st;
    src.group_id = g->group_id;  // motion applies per request
    const int n_groups = n_frames > 0 ? frames[0].n_groups : 1;
    for (int f = 0; f < n_frames; ++f) {
        if (frames[f].per_gaussian)
            return fail(ctx, GC_ERR_UNSUPPORTED, "per-Gaussian motion is taken by the single-frame and multi-level calls");
        if (frames[f].n_groups != n_groups || !frames[f].q || !frames[f].t)
            return fail(ctx, GC_ERR_INVALID_ARG, "motion frames must share n_groups and have q, t");
    }
    const gc_options &o = ctx->opt;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool capturing = stream_capturing(s);
    if (capturing && o.key_capacity <= 0)
        return fail(ctx, GC_ERR_INVALID_ARG, "graph capture needs a fixed key_capacity");
    gc_saved &S = saved ? *saved : ctx->internal;
    if (!S.batch) S.batch = std::make_shared<BatchState>();
    BatchState &B = *S.batch;
    const int64_t T = gc::radix_tile_keys();

    std::vector<gc::BatchReq> tab;
    int64_t items, tiles, pixels;
    int kbits;
    int64_t rows, cells;
    bool rows_fit;
    if ((st = build_table(ctx, g, frames, n_frames, n_groups, reqs, n_req, o, tab, items, tiles, pixels,
                          kbits, rows, cells, rows_fit)) != GC_OK)
        return st;
    const bool same_table = B.reqs_dev.p && (int)B.reqs.size() == n_req &&
                            memcmp(B.reqs.data(), tab.data(), sizeof(gc::BatchReq) * n_req) == 0;
    const bool fixed = capturing || B.bound;
    if (fixed && !same_table)
        return fail(ctx, GC_ERR_STATE,
                    capturing ? "a captured batch must repeat the requests of the preceding eager call"
                              : "this saved state is bound to a CUDA graph; use the same requests or another state");
    if (fixed && (o.key_capacity != B.K_cap || memcmp(&o, &B.opt, sizeof o) != 0))
        return fail(ctx, GC_ERR_STATE, "options changed since the batch was bound to a graph");
    S.valid = false;  // the single-frame part of this state no longer describes the last forward
    B.valid = false;
    B.n_req = n_req;
    B.n_frames = n_frames;
    B.n_groups = n_groups;
    B.has_motion = n_frames > 0;
    B.n = g->n;
    B.sh_degree = g->sh_degree;
    B.n_layers = g->n_layers;
    B.n_items = items;
    B.n_tiles = tiles;
    B.n_pixels = pixels;
    B.key_bits = kbits;
    B.opt = o;

    Sizer need{ctx, fixed};
    need(B.reqs_dev, sizeof(gc::BatchReq) * n_req);
    need(B.item_base, 8 * (n_req + 1));
    need(B.tile_base, 8 * (n_req + 1));
    need(B.seg_items, 4 * (n_req + 1));
    need(B.row_base, 8 * (n_req + 1));
    need(B.row_shift, 4 * (size_t)(rows + 1));
    const int64_t ni = items > 0 ? items : 1;
    need(B.rec, (size_t)ni * 16 * gc::kRec);
    need(B.ranked, (size_t)ni * 16 * gc::kRec);
    for (int b = 0; b < 2; ++b) {
        need(B.dkeys[b], (size_t)ni * 4);
        need(B.dvals[b], (size_t)ni * 4);
    }
    need(B.touched, (size_t)ni * 4);
    need(B.touched_r, (size_t)ni * 4);
    need(B.offsets, (size_t)(ni + 1) * 4);
    need(B.ebase, 4 * (n_req + 1));
    need(B.eshift, 4 * (n_req + 1));
    need(B.ecount, 4 * (n_req + 1));
    need(B.seg_entries, 4 * (n_req + 1));
    need(B.ranges, (size_t)tiles * 8);
    need(B.final_T, (size_t)pixels * 4);
    need(B.n_contrib, (size_t)pixels * 4);
    need(B.counter, 16);
    need(B.act, (size_t)std::max<int64_t>(g->n, 1) * 16);
    const bool fresh_words = !B.words.p;
    need(B.words, 64);
    need(B.scratch, 4 * std::max(gc::radix_scratch_words(ni), gc::scan_partials_size(ni)));
    if (need.st != GC_OK) return need.st;
    uint32_t *words = B.words.as<uint32_t>();  // [0] unpadded keys, [1] errors, [2] padded keys
    if (fresh_words) GC_CUDA(ctx, cudaMemsetAsync(B.words.p, 0, 64, s));

    if (!same_table) {  // upload the request table and the base arrays (eager calls only)
        if (B.staged) GC_CUDA(ctx, cudaEventSynchronize(B.staged));
        else GC_CUDA(ctx, cudaEventCreateWithFlags(&B.staged, cudaEventDisableTiming));
        if ((st = grow_pinned(ctx, B.staging, B.staging_cap, (size_t)n_req)) != GC_OK) return st;
        if ((st = grow_pinned(ctx, B.staging_base, B.staging_base_cap, (size_t)4 * (n_req + 1))) != GC_OK) return st;
        memcpy(B.staging, tab.data(), sizeof(gc::BatchReq) * n_req);
        int64_t *ib = B.staging_base, *tb = B.staging_base + (n_req + 1);
        uint32_t *si = reinterpret_cast<uint32_t *>(B.staging_base + 2 * (n_req + 1));
        int64_t *rb = B.staging_base + 3 * (n_req + 1);
        for (int q = 0; q < n_req; ++q) {
            ib[q] = tab[q].item_base;
            tb[q] = tab[q].tile_base;
            si[q] = (uint32_t)(tab[q].item_base / T);
            rb[q] = tab[q].row_base;
        }
        ib[n_req] = items;
        tb[n_req] = tiles;
        si[n_req] = (uint32_t)(items / T);
        rb[n_req] = rows;
        GC_CUDA(ctx, cudaMemcpyAsync(B.reqs_dev.p, B.staging, sizeof(gc::BatchReq) * n_req,
                                     cudaMemcpyHostToDevice, s));
        GC_CUDA(ctx, cudaMemcpyAsync(B.item_base.p, ib, 8 * (n_req + 1), cudaMemcpyHostToDevice, s));
        GC_CUDA(ctx, cudaMemcpyAsync(B.tile_base.p, tb, 8 * (n_req + 1), cudaMemcpyHostToDevice, s));
        GC_CUDA(ctx, cudaMemcpyAsync(B.seg_items.p, si, 4 * (n_req + 1), cudaMemcpyHostToDevice, s));
        GC_CUDA(ctx, cudaMemcpyAsync(B.row_base.p, rb, 8 * (n_req + 1), cudaMemcpyHostToDevice, s));
        GC_CUDA(ctx, cudaEventRecord(B.staged, s));
        B.reqs = tab;
    }
    const bool prof = !capturing;
    auto mark = [&](int stage) -> cudaError_t { return prof ? prof_mark(ctx, s, stage) : cudaSuccess; };

    GC_CUDA(ctx, mark(GC_STAGE_PREPROCESS));
    const gc::BatchReq *rq_dev = B.reqs_dev.as<gc::BatchReq>();
    const int64_t *ib_dev = B.item_base.as<int64_t>(), *tb_dev = B.tile_base.as<int64_t>();
    uint32_t *scratch = B.scratch.as<uint32_t>();
    if (items > 0) {
        // the per-Gaussian activation cache holds keyframe values: not with scale or opacity residuals
        bool deformed = false;
        for (const auto &R : tab) deformed = deformed || R.res.ls || R.res.logit;
        if (!deformed) {
            GC_DISPATCH_PREC(src.precision, gc::k_batch_activate<PREC_><<<(unsigned)((g->n + 255) / 256), 256, 0, s>>>(
                                                src, g->n, B.act.as<float4>()))
            gc::note_launches(1);
        }
        GC_DISPATCH_PREC(src.precision, gc::k_batch_preprocess<PREC_><<<(unsigned)((items + 255) / 256), 256, 0, s>>>(
            src, rq_dev, ib_dev, n_req, items, B.rec.as<float4>(), B.dkeys[0].as<uint32_t>(),
            B.dvals[0].as<uint32_t>(), B.touched.as<uint32_t>(), deformed ? nullptr : B.act.as<float4>()))
        gc::note_launches(1);
        GC_CUDA(ctx, cudaGetLastError());
        GC_CUDA(ctx, mark(GC_STAGE_DEPTH_SORT));
        uint32_t *dk[2] = {B.dkeys[0].as<uint32_t>(), B.dkeys[1].as<uint32_t>()};
        uint32_t *dv[2] = {B.dvals[0].as<uint32_t>(), B.dvals[1].as<uint32_t>()};
        GC_CUDA(ctx, gc::radix_sort_pairs(dk, dv, items, nullptr, 32, scratch, &B.depth_buf, s, words + 1, true,
                                          B.seg_items.as<uint32_t>(), n_req));
        GC_CUDA(ctx, mark(GC_STAGE_SCAN));
        GC_CUDA(ctx, gc::launch_rank_gather(dv[B.depth_buf], B.rec.as<float4>(), B.touched.as<uint32_t>(), items,
                                            B.ranked.as<float4>(), B.touched_r.as<uint32_t>(), s));
        GC_CUDA(ctx, gc::launch_exclusive_scan(B.touched_r.as<uint32_t>(), B.offsets.as<uint32_t>(), items, words,
                                               scratch, s, words + 1));
    } else {
        GC_CUDA(ctx, cudaMemsetAsync(words, 0, 4, s));
    }
    const uint32_t cap_hint = o.key_capacity > 0 ? (uint32_t)o.key_capacity : 0xFFFFFFFFu;
    gc::k_batch_entry_bases<<<1, 1, 0, s>>>(B.offsets.as<uint32_t>(), words, ib_dev, n_req, items, (uint32_t)T,
                                            cap_hint, B.ebase.as<uint32_t>(), B.eshift.as<uint32_t>(),
                                            B.ecount.as<uint32_t>(), B.seg_entries.as<uint32_t>(), words);
    gc::note_launches(1);
    GC_CUDA(ctx, cudaGetLastError());
    int64_t K;
    if (o.key_capacity > 0) {
        K = o.key_capacity;
        B.k_exact = false;
    } else {
        GC_CUDA(ctx, cudaMemcpyAsync(ctx->host_word, words + 2, 4, cudaMemcpyDeviceToHost, s));
        GC_CUDA(ctx, cudaStreamSynchronize(s));
        K = ctx->host_word[0];
        if (K >= 0xFFFFFFFFll) return fail(ctx, GC_ERR_CAPACITY, "batch needs more than 2^32 - 1 keys");
        B.k_exact = true;
    }
    const int64_t kk = K > 0 ? K : 1;
    // row binning (every request within 255 tile columns): the lists in per-(request, tile row)
    // segments padded to whole radix tiles, one segmented pass on the column; room for the
    // padding beyond the capacity K (which counts the entries, padded per request)
    const int64_t kpad = (kk + rows * gc::radix_tile_keys(true) + 3) & ~int64_t(3);
    const bool by_rows = rows_fit;
    if (by_rows && kpad > 0xFFFFFFF0ll)
        return fail(ctx, GC_ERR_CAPACITY, "batch needs more than 2^32 - 16 list words with its row padding");
    const int64_t kalloc = by_rows ? kpad : kk;
    for (int b = 0; b < 2; ++b) {
        need(B.tkeys[b], (size_t)kalloc * 4 + 16);
        if (!by_rows) need(B.tvals[b], (size_t)kalloc * 4 + 16);  // row-binned lists: one word per entry
    }
    const size_t bwords = by_rows ? ((gc::bucket_words(cells, (int)rows) + 63) & ~size_t(63)) : 0;
    need(B.scratch, 4 * (bwords + std::max(gc::radix_scratch_words(kalloc), gc::scan_partials_size(ni))));
    if (need.st != GC_OK) return need.st;
    scratch = B.scratch.as<uint32_t>();
    B.K_cap = K;
    B.row_binned = by_rows;
    uint32_t *tk[2] = {B.tkeys[0].as<uint32_t>(), B.tkeys[1].as<uint32_t>()};
    uint32_t *tv[2] = {B.tvals[0].as<uint32_t>(), B.tvals[1].as<uint32_t>()};
    if (by_rows) {
        const gc::BatchBucketMap map{rq_dev, ib_dev, B.row_base.as<int64_t>(), n_req};
        GC_CUDA(ctx, mark(GC_STAGE_EMIT));
        if (K > 0 && items > 0)
            GC_CUDA(ctx, gc::bucket_place(B.ranked.as<float4>(), words, words + 2, B.touched_r.as<uint32_t>(), map, items / 32,
                                          (int)rows, cells, tk[0], (uint32_t)kk, (uint32_t)kalloc, words,
                                          B.row_shift.as<uint32_t>(), scratch, nullptr, s));
        GC_CUDA(ctx, mark(GC_STAGE_TILE_SORT));
        if (K > 0 && items > 0)
            GC_CUDA(ctx, gc::bucket_sort(tk, (uint32_t)kalloc, words, (int)rows, cells, scratch, scratch + bwords,
                                         &B.tile_buf, s));
        GC_CUDA(ctx, mark(GC_STAGE_RANGES));
        if (tiles > 0) GC_CUDA(ctx, cudaMemsetAsync(B.ranges.p, 0, (size_t)tiles * 8, s));
        if (K > 0 && items > 0)
            GC_CUDA(ctx, gc::bucket_ranges(map, (int)rows, cells, scratch, scratch + bwords, B.ranges.as<uint2>(), s));
    } else {
        if (K > 0 && items > 0) {
            GC_CUDA(ctx, mark(GC_STAGE_EMIT));
            const int64_t threads = ((items + 31) / 32) * 32;
            gc::k_batch_emit<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
                B.ranked.as<float4>(), B.offsets.as<uint32_t>(), B.touched_r.as<uint32_t>(), rq_dev, ib_dev, n_req,
                B.eshift.as<uint32_t>(), items, (uint32_t)K, words + 2, tk[0], tv[0]);
            gc::note_launches(1);
            gc::k_batch_pad_fill<<<n_req, 256, 0, s>>>(B.ebase.as<uint32_t>(), B.ecount.as<uint32_t>(), (uint32_t)K,
                                                       words + 2, tk[0], tv[0]);
            gc::note_launches(1);
            GC_CUDA(ctx, cudaGetLastError());
            GC_CUDA(ctx, mark(GC_STAGE_TILE_SORT));
            GC_CUDA(ctx, gc::radix_sort_pairs(tk, tv, K, words + 2, kbits, scratch, &B.tile_buf, s, words + 1,
                                              /*keys_out=*/true, B.seg_entries.as<uint32_t>(), n_req));
        }
        GC_CUDA(ctx, mark(GC_STAGE_RANGES));
        if (tiles > 0) GC_CUDA(ctx, cudaMemsetAsync(B.ranges.p, 0, (size_t)tiles * 8, s));
        if (K > 0 && items > 0) {
            // ranges from the sorted keys: a difference grid filled by the preprocess costs
            // contended integer atomics, measured slower
            const int64_t blocks = std::max<int64_t>(std::min<int64_t>((K / 4 + 255) / 256, 148 * 16), 1);
            gc::k_batch_key_ranges<<<(unsigned)blocks, 256, 0, s>>>(tk[B.tile_buf], B.ebase.as<uint32_t>(),
                                                                    B.ecount.as<uint32_t>(), tb_dev, n_req, words + 2,
                                                                    (uint32_t)K, B.ranges.as<uint2>());
            gc::note_launches(1);
            GC_CUDA(ctx, cudaGetLastError());
        }
    }
    GC_CUDA(ctx, mark(GC_STAGE_BLEND));
    GC_CUDA(ctx, cudaMemsetAsync(B.counter.p, 0, 8, s));
    {
        const uint32_t *sv = (K > 0 && items > 0) ? B.lists() : nullptr;
        unsigned long long *ctr = B.counter.as<unsigned long long>();
        auto grid = [&](int64_t g) { return (unsigned)std::min<int64_t>(std::max<int64_t>(tiles, 1), g); };
#define GC_BB_ARGS rq_dev, tb_dev, n_req, tiles, B.ranges.as<uint2>(), sv, B.ranked.as<float4>(), \
                   B.final_T.as<float>(), B.n_contrib.as<uint32_t>(), ctr
        if (o.tile_w == 16)
            gc::k_batch_blend_fwd<16, 16><<<grid(gc::persistent_grid<gc::k_batch_blend_fwd<16, 16>, 256>()), 256, 0, s>>>(GC_BB_ARGS);
        else if (o.tile_w == 8)
            gc::k_batch_blend_fwd<8, 32><<<grid(gc::persistent_grid<gc::k_batch_blend_fwd<8, 32>, 256>()), 256, 0, s>>>(GC_BB_ARGS);
        else
            gc::k_batch_blend_fwd<32, 8><<<grid(gc::persistent_grid<gc::k_batch_blend_fwd<32, 8>, 256>()), 256, 0, s>>>(GC_BB_ARGS);
#undef GC_BB_ARGS
        gc::note_launches(1);
        GC_CUDA(ctx, cudaGetLastError());
    }
    GC_CUDA(ctx, mark(-1));
    if (capturing) B.bound = true;
    B.valid = true;
    ctx->last = &S;
    return GC_OK;
}

extern "C" gc_status gc_render_batch_backward(gc_context *ctx, const gc_saved *saved,
                                              const gc_gaussians *g, const gc_motion *frames,
                                              int32_t n_frames, const float *const *dL_dimages,
                                              int32_t accumulate, gc_grads *out, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!dL_dimages || !out) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimages or grads is NULL");
    if (accumulate != 0 && accumulate != 1) return fail(ctx, GC_ERR_INVALID_ARG, "accumulate must be 0 or 1");
    const gc_saved &S = saved ? *saved : ctx->internal;
    if (!S.batch || !S.batch->valid) return fail(ctx, GC_ERR_STATE, "no batched forward recorded");
    BatchState &B = *S.batch;
    if (n_frames < 0 || (n_frames > 0 && !frames)) return fail(ctx, GC_ERR_INVALID_ARG, "bad motion frames");
    gc::GaussSrc src;
    gc_status st = make_source(ctx, g, n_frames > 0 ? &frames[0] : nullptr, src);
    if (st != GC_OK) return st;
    src.group_id = g->group_id;
    if (g->n != B.n || g->sh_degree != B.sh_degree || g->n_layers != B.n_layers)
        return fail(ctx, GC_ERR_STATE, "the Gaussian set differs from the one of the batched forward");
    if (n_frames != B.n_frames || (n_frames > 0 && frames[0].n_groups != B.n_groups))
        return fail(ctx, GC_ERR_STATE, "the motion frames differ from the forward's");
    const int n_req = B.n_req;
    for (int q = 0; q < n_req; ++q)
        if (!dL_dimages[q]) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimages[%d] is NULL", q);
    for (int q = 0; q < n_req; ++q) {
        const int f = B.reqs[q].frame;
        if (f >= 0 && (B.reqs[q].group_q != frames[f].q || B.reqs[q].group_t != frames[f].t ||
                       B.reqs[q].res.ls != frames[f].res_log_scales ||
                       B.reqs[q].res.logit != frames[f].res_opacity_logits || B.reqs[q].res.sh != frames[f].res_sh))
            return fail(ctx, GC_ERR_STATE, "the motion frames differ from the forward's");
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const bool capturing = stream_capturing(s);
    const bool fixed = capturing || B.bound;
    const bool same_dimg = B.dimg_dev.p && (int)B.dimgs.size() == n_req &&
                           std::equal(B.dimgs.begin(), B.dimgs.end(), dL_dimages);
    if (fixed && !same_dimg)
        return fail(ctx, GC_ERR_STATE, "a graph-bound batch backward must use the dL_dimages of its eager call");
    const int64_t items = B.n_items, ni = items > 0 ? items : 1, K = B.K_cap > 0 ? B.K_cap : 1;
    const int G = B.has_motion ? B.n_groups : 0;
    const int64_t chunks = items / gc::kBatchChunk;
    Sizer need{ctx, fixed};
    need(B.dimg_dev, sizeof(float *) * n_req);
    {
        void *before = B.part.p, *before_flag = B.flag.p;
        need(B.part, (size_t)K * 9 * 4 + 64);
        need(B.flag, (size_t)K + 64);
        if (B.part.p != before || B.flag.p != before_flag) B.part_clean = false;
    }
    need(B.g2d, (size_t)ni * 9 * 4);
    need(B.mcontrib, (size_t)ni * 7 * 4);
    if (G) need(B.gpartial, (size_t)std::max<int64_t>(chunks, 1) * G * 7 * 4);
    if (need.st != GC_OK) return need.st;
    if (!same_dimg) {
        if (B.staged) GC_CUDA(ctx, cudaEventSynchronize(B.staged));
        else GC_CUDA(ctx, cudaEventCreateWithFlags(&B.staged, cudaEventDisableTiming));
        if ((st = grow_pinned(ctx, B.staging_dimg, B.staging_dimg_cap, (size_t)n_req)) != GC_OK) return st;
        for (int q = 0; q < n_req; ++q) B.staging_dimg[q] = dL_dimages[q];
        GC_CUDA(ctx, cudaMemcpyAsync(B.dimg_dev.p, B.staging_dimg, sizeof(float *) * n_req, cudaMemcpyHostToDevice, s));
        GC_CUDA(ctx, cudaEventRecord(B.staged, s));
        B.dimgs.assign(dL_dimages, dL_dimages + n_req);
    }
    const bool prof = !capturing;
    auto mark = [&](int stage) -> cudaError_t { return prof ? prof_mark(ctx, s, stage) : cudaSuccess; };
    const gc::BatchReq *rq_dev = B.reqs_dev.as<gc::BatchReq>();
    const int64_t *ib_dev = B.item_base.as<int64_t>(), *tb_dev = B.tile_base.as<int64_t>();

    if (!B.part_clean) {
        if (capturing) return fail(ctx, GC_ERR_STATE, "the partials buffer is not clean; run the backward eagerly first");
        GC_CUDA(ctx, cudaMemsetAsync(B.part.p, 0, B.part.cap, s));
        GC_CUDA(ctx, cudaMemsetAsync(B.flag.p, 0, B.flag.cap, s));
    }
    GC_CUDA(ctx, mark(GC_STAGE_BLEND_BWD));
    B.part_clean = false;
    if (G) GC_CUDA(ctx, cudaMemsetAsync(B.mcontrib.p, 0, (size_t)ni * 7 * 4, s));
    GC_CUDA(ctx, cudaMemsetAsync(B.counter.p, 0, 8, s));
    {
        const uint32_t *sv = (B.K_cap > 0 && items > 0) ? B.lists() : nullptr;
        unsigned long long *ctr = B.counter.as<unsigned long long>();
        auto grid = [&](int64_t g) { return (unsigned)std::min<int64_t>(std::max<int64_t>(B.n_tiles, 1), g); };
#define GC_BB_ARGS rq_dev, tb_dev, n_req, B.n_tiles, B.ranges.as<uint2>(), sv, B.ranked.as<float4>(),            \
                   B.offsets.as<uint32_t>(), B.eshift.as<uint32_t>(), B.final_T.as<float>(),                     \
                   B.n_contrib.as<uint32_t>(), B.dimg_dev.as<const float *>(), B.part.as<float>(),          \
                   B.flag.as<uint8_t>(), ctr
        if (B.opt.tile_w == 16)
            gc::k_batch_blend_bwd<16, 16><<<grid(gc::persistent_grid<gc::k_batch_blend_bwd<16, 16>, gc::kBwdThreads>()), gc::kBwdThreads, 0, s>>>(GC_BB_ARGS);
        else if (B.opt.tile_w == 8)
            gc::k_batch_blend_bwd<8, 32><<<grid(gc::persistent_grid<gc::k_batch_blend_bwd<8, 32>, gc::kBwdThreads>()), gc::kBwdThreads, 0, s>>>(GC_BB_ARGS);
        else
            gc::k_batch_blend_bwd<32, 8><<<grid(gc::persistent_grid<gc::k_batch_blend_bwd<32, 8>, gc::kBwdThreads>()), gc::kBwdThreads, 0, s>>>(GC_BB_ARGS);
#undef GC_BB_ARGS
        gc::note_launches(1);
        GC_CUDA(ctx, cudaGetLastError());
    }
    if (items > 0) {
        GC_CUDA(ctx, mark(GC_STAGE_REDUCE));
        gc::k_batch_reduce<<<(unsigned)((items * 32 + 255) / 256), 256, 0, s>>>(
            B.part.as<float>(), B.offsets.as<uint32_t>(), B.touched_r.as<uint32_t>(),
            B.dvals[B.depth_buf].as<uint32_t>(), ib_dev, n_req, B.eshift.as<uint32_t>(), items,
            (uint32_t)std::min<int64_t>(B.K_cap, 0xFFFFFFFFll), B.flag.as<uint8_t>(), B.g2d.as<float>());
        gc::note_launches(1);
        GC_CUDA(ctx, cudaGetLastError());
    }
    B.part_clean = true;
    GC_CUDA(ctx, mark(GC_STAGE_PREPROCESS_BWD));
    if (g->n > 0) {
        GC_DISPATCH_PREC(src.precision, gc::k_batch_preprocess_bwd<PREC_><<<(unsigned)((g->n + 127) / 128), 128, 0, s>>>(
            src, rq_dev, n_req, g->n, B.g2d.as<float>(), B.touched.as<uint32_t>(), *out, accumulate,
            G ? B.mcontrib.as<float>() : nullptr))
        gc::note_launches(1);
        GC_CUDA(ctx, cudaGetLastError());
    }
    if (G) {
        GC_CUDA(ctx, mark(GC_STAGE_GROUP_REDUCE));
        if (chunks > 0) {
            gc::k_batch_group_partial<<<(unsigned)chunks, 128, 0, s>>>(B.mcontrib.as<float>(), g->group_id, rq_dev,
                                                                       ib_dev, n_req, G, B.gpartial.as<float>());
            gc::note_launches(1);
        }
        const int nt = B.n_frames * G * 7;
        gc::k_batch_group_final<<<(nt + 127) / 128, 128, 0, s>>>(B.gpartial.as<float>(), rq_dev, ib_dev, n_req,
                                                                B.n_frames, G, accumulate, out->d_group_q,
                                                                out->d_group_t);
        gc::note_launches(1);
        GC_CUDA(ctx, cudaGetLastError());
    }
    GC_CUDA(ctx, mark(-1));
    return GC_OK;
}

// --------------------------------------------------------------------------- graphs

namespace {
constexpr int kGraphBranches = 4;  // capture streams of a batch graph
}

struct gc_batch_graph {
    gc_context *ctx = nullptr;
    std::vector<gc_saved *> states;  // one per batch of `depth` requests
    int depth = 0, n_req = 0;
    bool backward = false;
    // batch b is captured on branch b mod branches (branch 0: the caller's stream); the
    // backwards are chained in batch order by bwd_done
    int branches = 1;
    cudaStream_t side[kGraphBranches] = {};
    cudaEvent_t fork = nullptr, bwd_done = nullptr, joins[kGraphBranches] = {};
    int64_t key_capacity = 0;
    int64_t kernel_nodes = 0;
    cudaStream_t own_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void graph_free(gc_batch_graph *G) {
    if (!G) return;
    DeviceGuard dg(G->ctx->device);
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    for (gc_saved *s : G->states) gc_saved_destroy(G->ctx, s);
    for (int c = 0; c < kGraphBranches; ++c) {
        if (G->side[c]) cudaStreamDestroy(G->side[c]);
        if (G->joins[c]) cudaEventDestroy(G->joins[c]);
    }
    if (G->fork) cudaEventDestroy(G->fork);
    if (G->bwd_done) cudaEventDestroy(G->bwd_done);
    if (G->own_stream) cudaStreamDestroy(G->own_stream);
    delete G;
}

// One pass over all batches: per batch its forward and, for a training step, its backward
// (the first overwrites the gradients, the others add to them, so the step's gradient is
// summed in batch order: each backward waits for the previous one).  Batch b runs on
// streams[b mod branches]; its state is its own, so the batches of different branches may
// overlap on the GPU.
gc_status graph_pass(gc_batch_graph *G, const gc_gaussians *g, const gc_motion *frames, int n_frames,
                     const gc_request *reqs, const float *const *dL, gc_grads *grads, const cudaStream_t *streams) {
    gc_status st;
    const int nb = (int)G->states.size();
    for (int b = 0; b < nb; ++b) {
        const cudaStream_t s = streams[b % G->branches];
        const int q0 = b * G->depth, cnt = std::min(G->depth, G->n_req - q0);
        if ((st = gc_render_batch_forward(G->ctx, g, frames, n_frames, reqs + q0, cnt, G->states[b], s)) != GC_OK)
            return st;
        if (G->backward) {
            if (G->branches > 1 && b > 0) GC_CUDA(G->ctx, cudaStreamWaitEvent(s, G->bwd_done, 0));
            if ((st = gc_render_batch_backward(G->ctx, G->states[b], g, frames, n_frames, dL + q0, b > 0 ? 1 : 0,
                                               grads, s)) != GC_OK)
                return st;
            if (G->branches > 1) GC_CUDA(G->ctx, cudaEventRecord(G->bwd_done, s));
        }
    }
    return GC_OK;
}

}  // namespace

extern "C" gc_status gc_batch_graph_create(gc_context *ctx, const gc_gaussians *g, const gc_motion *frames,
                                           int32_t n_frames, const gc_request *reqs, int32_t n_req,
                                           int32_t depth, const float *const *dL_dimages, gc_grads *grads,
                                           void *stream, gc_batch_graph **out) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!out) return fail(ctx, GC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!reqs || n_req <= 0) return fail(ctx, GC_ERR_INVALID_ARG, "no requests");
    if (depth <= 0) return fail(ctx, GC_ERR_INVALID_ARG, "depth must be >= 1");
    if (dL_dimages && !grads) return fail(ctx, GC_ERR_INVALID_ARG, "a backward graph needs gradient buffers");
    DeviceGuard dg(ctx->device);
    gc_batch_graph *G = new (std::nothrow) gc_batch_graph();
    if (!G) return fail(ctx, GC_ERR_OOM, "graph handle");
    G->ctx = ctx;
    G->depth = std::min<int>(depth, n_req);
    G->n_req = n_req;
    G->backward = dL_dimages != nullptr;
    const int nb = (n_req + G->depth - 1) / G->depth;
    gc_status st = GC_OK;
    for (int b = 0; b < nb && st == GC_OK; ++b) {
        gc_saved *s = nullptr;
        st = gc_saved_create(ctx, &s);
        if (st == GC_OK) G->states.push_back(s);
    }
    const gc_options saved_opt = ctx->opt;
    cudaStream_t s = (cudaStream_t)stream;
    auto bail = [&](gc_status e) {
        ctx->opt = saved_opt;
        graph_free(G);
        return e;
    };
    if (st != GC_OK) return bail(fail(ctx, st, "saved state allocation failed"));
    if (!s) {  // capture needs a stream other than the legacy default one
        if (cudaStreamCreateWithFlags(&G->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(ctx, GC_ERR_CUDA, "stream creation failed"));
        }
        s = G->own_stream;
    }
    G->branches = std::min(nb, kGraphBranches);
    {
        bool ok = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming) == cudaSuccess &&
                  cudaEventCreateWithFlags(&G->bwd_done, cudaEventDisableTiming) == cudaSuccess;
        for (int c = 1; c < G->branches && ok; ++c)
            ok = cudaStreamCreateWithFlags(&G->side[c], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&G->joins[c], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return bail(fail(ctx, GC_ERR_CUDA, "stream or event creation failed"));
        }
    }
    cudaStream_t eager[kGraphBranches], capture[kGraphBranches];
    for (int c = 0; c < kGraphBranches; ++c) {
        eager[c] = s;
        capture[c] = c == 0 ? s : G->side[c];
    }
    // 1. key capacity: the caller's, or the largest batch's exact need plus 5 %
    int64_t cap = saved_opt.key_capacity;
    if (cap <= 0) {
        ctx->opt.key_capacity = 0;
        for (int b = 0; b < nb; ++b) {
            const int q0 = b * G->depth, cnt = std::min(G->depth, n_req - q0);
            if ((st = gc_render_batch_forward(ctx, g, frames, n_frames, reqs + q0, cnt, G->states[b], s)) != GC_OK)
                return bail(st);
            cap = std::max<int64_t>(cap, G->states[b]->batch->K_cap);
        }
        const int64_t T = gc::radix_tile_keys();
        cap = (cap + cap / 20 + 2 * T + T - 1) / T * T;
        if (cap > 0xFFFFFFF0ll) return bail(fail(ctx, GC_ERR_CAPACITY, "a batch needs more than 2^32 keys"));
        for (gc_saved *x : G->states) {  // re-bind the states to the fixed capacity
            gc_saved *fresh = nullptr;
            if ((st = gc_saved_create(ctx, &fresh)) != GC_OK) return bail(st);
            gc_saved_destroy(ctx, x);
            std::replace(G->states.begin(), G->states.end(), x, fresh);
        }
    }
    G->key_capacity = cap;
    ctx->opt.key_capacity = cap;
    // 2. eager pass on the caller's stream: sizes every buffer, uploads the request tables
    if ((st = graph_pass(G, g, frames, n_frames, reqs, dL_dimages, grads, eager)) != GC_OK) return bail(st);
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(ctx, GC_ERR_CUDA, "eager pass failed"));
    for (gc_saved *x : G->states)
        if ((st = batch_check(ctx, *x, s)) != GC_OK) return bail(st);
    // 3. capture the same pass, branch c on capture[c] (forked from s, joined back into s)
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ctx, GC_ERR_CUDA, "cannot begin stream capture"));
    }
    cudaError_t ce = cudaEventRecord(G->fork, s);
    for (int c = 1; c < G->branches && ce == cudaSuccess; ++c) ce = cudaStreamWaitEvent(G->side[c], G->fork, 0);
    if (ce == cudaSuccess) st = graph_pass(G, g, frames, n_frames, reqs, dL_dimages, grads, capture);
    for (int c = 1; c < G->branches && ce == cudaSuccess; ++c) {
        ce = cudaEventRecord(G->joins[c], G->side[c]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, G->joins[c], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    G->graph = graph;
    if (st != GC_OK) return bail(st);
    if (ce != cudaSuccess || ee != cudaSuccess || !graph) {
        cudaGetLastError();
        return bail(fail(ctx, GC_ERR_CUDA, "stream capture failed: %s",
                         cudaGetErrorString(ce != cudaSuccess ? ce : ee)));
    }
    size_t n_nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes) cudaGraphGetNodes(graph, nodes.data(), &n_nodes);
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) G->kernel_nodes++;
    }
    if (cudaGraphInstantiate(&G->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ctx, GC_ERR_CUDA, "graph instantiation failed"));
    }
    ctx->opt = saved_opt;
    *out = G;
    return GC_OK;
}

extern "C" gc_status gc_batch_graph_launch(gc_batch_graph *G, void *stream) {
    if (!G) return GC_ERR_INVALID_ARG;
    DeviceGuard dg(G->ctx->device);
    GC_CUDA(G->ctx, cudaGraphLaunch(G->exec, (cudaStream_t)stream));
    gc::note_launches((int)G->kernel_nodes);
    return GC_OK;
}

extern "C" gc_status gc_batch_graph_info(const gc_batch_graph *G, int64_t *key_capacity, int64_t *kernel_nodes,
                                         int32_t *n_batches) {
    if (!G) return GC_ERR_INVALID_ARG;
    if (key_capacity) *key_capacity = G->key_capacity;
    if (kernel_nodes) *kernel_nodes = G->kernel_nodes;
    if (n_batches) *n_batches = (int32_t)G->states.size();
    return GC_OK;
}

extern "C" gc_status gc_batch_graph_check(gc_batch_graph *G, void *stream) {
    if (!G) return GC_ERR_INVALID_ARG;
    DeviceGuard dg(G->ctx->device);
    GC_CUDA(G->ctx, cudaStreamSynchronize((cudaStream_t)stream));
    for (gc_saved *x : G->states) {
        const gc_status st = batch_check(G->ctx, *x, (cudaStream_t)stream);
        if (st != GC_OK) return st;
    }
    return GC_OK;
}

extern "C" gc_status gc_batch_graph_destroy(gc_batch_graph *G) {
    if (!G) return GC_ERR_INVALID_ARG;
    graph_free(G);
    return GC_OK;
}

// --------------------------------------------------------------------------- autotuner

extern "C" gc_status gc_tune_batch(gc_context *ctx, const gc_gaussians *g, const gc_motion *frames,
                                   int32_t n_frames, const gc_request *reqs, int32_t n_req,
                                   const float *const *dL_dimages, gc_grads *grads, const int32_t *depths,
                                   int32_t n_depths, int32_t iters, gc_tune_entry *entries,
                                   gc_tune_entry *best, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!depths || n_depths <= 0 || !entries || !best)
        return fail(ctx, GC_ERR_INVALID_ARG, "depths, entries and best are required");
    if (iters <= 0) return fail(ctx, GC_ERR_INVALID_ARG, "iters must be >= 1");
    static const int shapes[3][2] = {{16, 16}, {8, 32}, {32, 8}};
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaStream_t own = nullptr;
    if (!s) {
        GC_CUDA(ctx, cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        s = own;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const gc_options base = ctx->opt;
    gc_status st = GC_OK;
    int n_out = 0, ib = -1;
    for (int sh = 0; sh < 3 && st == GC_OK; ++sh) {
        for (int d = 0; d < n_depths && st == GC_OK; ++d) {
            ctx->opt = base;
            ctx->opt.tile_w = shapes[sh][0];
            ctx->opt.tile_h = shapes[sh][1];
            gc_batch_graph *G = nullptr;
            st = gc_batch_graph_create(ctx, g, frames, n_frames, reqs, n_req, depths[d], dL_dimages, grads, s, &G);
            if (st != GC_OK) break;
            float ms = 0.f;
            if ((st = gc_batch_graph_launch(G, s)) == GC_OK) {  // warm-up
                cudaEventRecord(e0, s);
                for (int it = 0; it < iters && st == GC_OK; ++it) st = gc_batch_graph_launch(G, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    cudaGetLastError();
                    st = fail(ctx, GC_ERR_CUDA, "timing failed");
                }
            }
            if (st == GC_OK) st = gc_batch_graph_check(G, s);
            gc_tune_entry &E = entries[n_out];
            E.tile_w = shapes[sh][0];
            E.tile_h = shapes[sh][1];
            E.depth = std::min<int>(depths[d], n_req);
            E.key_capacity = G->key_capacity;
            E.ms = ms / (float)iters;
            graph_free(G);
            if (st != GC_OK) break;
            if (ib < 0 || E.ms < entries[ib].ms) ib = n_out;
            ++n_out;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (own) cudaStreamDestroy(own);
    ctx->opt = base;
    if (st != GC_OK) return st;
    *best = entries[ib];
    ctx->opt.tile_w = best->tile_w;
    ctx->opt.tile_h = best->tile_h;
    return GC_OK;
}
