// gc_backward.cu - reverse mode of the render (the gradients the paper's
// rate-distortion training needs, Sec. 3.3), atomics-free and deterministic.
//
//  k_blend_bwd        one CTA per tile walks the tile list back to front from each
//                     pixel's saved final transmittance (Eq. 2 reversed), and reduces
//                     the 9 per-pixel partial derivatives of every list entry over the
//                     tile's pixels in a fixed order (warp butterfly, then warps in
//                     order).  The sums go to the entry's emit position, so each
//                     Gaussian's partials are contiguous.  Entries behind the last
//                     blended one of every pixel are not written; the tile records the
//                     largest rank that may have contributed.
//  k_reduce_entries   one warp per Gaussian sums its entries' partials (the flagged ones:
//                     only entries with a nonzero partial are stored and flagged).
//  k_preprocess_bwd   chain rule from (u, v, conic, opacity, rgb) to mean, log-scale,
//                     quaternion, opacity logit, SH and the group motion (Sec. 3.2).
//  k_group_partial /  per-group sums of the motion terms: each thread owns a group and
//  k_group_final      adds its members of a chunk in index order; then one warp per
//                     (group, component) adds the chunks in a fixed order.
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_chain.cuh"
#include "gc_tile.cuh"
#include "gc_sh.cuh"

namespace gc {

namespace {


// One CTA per tile of a single image.
template <int TW, int TH>
__global__ void __launch_bounds__(kBwdThreads) k_blend_bwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, const uint32_t *__restrict__ offsets, int W, int H, RenderParams rp,
    const float *__restrict__ final_T, const uint32_t *__restrict__ n_contrib,
    const float *__restrict__ dimg, float *__restrict__ part, uint8_t *__restrict__ flag) {
    __shared__ __align__(16) BwdSmem sm;
    const int tile = blockIdx.x, ntx = rp.ntx;
    const TileBwd o{final_T, n_contrib, dimg, rp, W, H, 0u, 0u, flag};
    blend_bwd_tile<TW, TH>(tile % ntx, tile / ntx, ranges[tile], sorted_vals, ranked, offsets, o, part, sm);
}

// One warp per rank: sum of the Gaussian's partials over its tiles (entry-major
// partials, nine floats per entry); the result goes to the Gaussian's compact
// position j = perm[r].
__global__ void __launch_bounds__(256) k_reduce_entries(float *__restrict__ part,
                                                        const uint32_t *__restrict__ offsets,
                                                        const uint32_t *__restrict__ touched_r,
                                                        const uint32_t *__restrict__ perm, int64_t n,
                                                        uint32_t cap, uint8_t *__restrict__ flag,
                                                        float *__restrict__ g2d) {
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    float out0, out8;
    reduce_entries_warp(part, offsets[r], touched_r[r], cap, flag, out0, out8);
    store_reduced(g2d + 9 * (int64_t)perm[r], out0, out8);
}

// Thread per selected Gaussian in index order (coalesced attribute reads and
// gradient writes); g2d and touched are by compact position.  The SH gradient (up to 48
// floats per Gaussian) is staged in shared memory, one row per thread at a pitch of 49 words
// (the rows' k-th words of a warp fall on distinct banks), and each warp then writes its 32
// rows with consecutive lanes on consecutive words: a thread storing its own row would put
// one word in each of 32 sectors per store instruction.
constexpr int kShPitch = 49;

template <int PREC>
__global__ void __launch_bounds__(128) k_preprocess_bwd(GaussSrc G, Selection sel, int64_t n_sel,
                                                        CamParams cam, RenderParams rp,
                                                        const float *__restrict__ g2d,
                                                        const uint32_t *__restrict__ touched,
                                                        gc_grads out, float *__restrict__ mcontrib) {
    __shared__ float s_dsh[128 * kShPitch];
    __shared__ int64_t s_row[128];
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = j < n_sel;
    const int64_t i = valid ? sel_global(sel, j) : 0;
    const int K3 = 3 * G.K;
    float *dsh = &s_dsh[threadIdx.x * kShPitch];
    if (valid) {
        GradAcc acc;
        for (int k = 0; k < 3; ++k) { acc.dmu[k] = 0.f; acc.dls[k] = 0.f; }
        for (int k = 0; k < 4; ++k) acc.dq[k] = 0.f;
        acc.dlogit = 0.f;
        float m7[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (touched[j] != 0) {
            const int g = G.per_gaussian ? (int)i : ((G.group_q && G.group_id) ? G.group_id[i] : 0);
            chain_rule<PREC>(G, i, G.group_q, G.group_t, g, cam, rp, g2d + 9 * j, acc, m7, G.res, dsh);
        } else {
            for (int k = 0; k < K3; ++k) dsh[k] = 0.f;
        }
        if (out.d_means) for (int k = 0; k < 3; ++k) out.d_means[3 * i + k] = acc.dmu[k];
        if (out.d_log_scales) for (int k = 0; k < 3; ++k) out.d_log_scales[3 * i + k] = acc.dls[k];
        if (out.d_quats) for (int k = 0; k < 4; ++k) out.d_quats[4 * i + k] = acc.dq[k];
        if (out.d_opacity_logits) out.d_opacity_logits[i] = acc.dlogit;
        if (mcontrib) for (int k = 0; k < 7; ++k) mcontrib[7 * j + k] = m7[k];
    }
    if (!out.d_sh) return;  // uniform over the grid
    s_row[threadIdx.x] = valid ? i : -1;
    __syncwarp();
    const int w0 = threadIdx.x & ~31;
    for (int e = threadIdx.x & 31; e < 32 * K3; e += 32) {
        const int r = e / K3, c = e - r * K3;
        const int64_t row = s_row[w0 + r];
        if (row >= 0) out.d_sh[row * K3 + c] = s_dsh[(w0 + r) * kShPitch + c];
    }
}

// Per-Gaussian motion: scatter each selected Gaussian's motion terms to its own rows.
__global__ void k_motion_scatter(const float *__restrict__ mcontrib, Selection sel, int64_t n_sel,
                                 float *__restrict__ d_q, float *__restrict__ d_t) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_sel) return;
    const int64_t i = sel_global(sel, j);
    if (d_q)
        for (int k = 0; k < 4; ++k) d_q[4 * i + k] = mcontrib[7 * j + k];
    if (d_t)
        for (int k = 0; k < 3; ++k) d_t[3 * i + k] = mcontrib[7 * j + 4 + k];
}

constexpr int kGroupChunk = 256;

// Per chunk of 256 compact positions, each thread sums the motion terms of the
// chunk's members of the groups it owns, in position order.
__global__ void __launch_bounds__(128) k_group_partial(const float *__restrict__ mcontrib,
                                                       const int32_t *__restrict__ group_id,
                                                       Selection sel, int64_t n_sel, int n_groups,
                                                       float *__restrict__ partial) {
    __shared__ int s_gid[kGroupChunk];
    __shared__ float s_val[kGroupChunk * 7];
    const int64_t base = (int64_t)blockIdx.x * kGroupChunk;
    const int cnt = (int)((n_sel - base) < (int64_t)kGroupChunk ? (n_sel - base) : (int64_t)kGroupChunk);
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const int64_t i = sel_global(sel, base + k);
        s_gid[k] = group_id ? group_id[i] : 0;
    }
    for (int k = threadIdx.x; k < cnt * 7; k += blockDim.x) s_val[k] = mcontrib[base * 7 + k];
    __syncthreads();
    for (int g = threadIdx.x; g < n_groups; g += blockDim.x) {
        float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < cnt; ++k) {
            if (s_gid[k] == g) {
#pragma unroll
                for (int c = 0; c < 7; ++c) acc[c] += s_val[7 * k + c];
            }
        }
        float *o = partial + ((int64_t)blockIdx.x * n_groups + g) * 7;
#pragma unroll
        for (int c = 0; c < 7; ++c) o[c] = acc[c];
    }
}

// One warp per (group, component): lane l sums chunks l, l + 32, ... in order, then a fixed
// butterfly adds the lanes (a fixed summation order: deterministic).
__global__ void __launch_bounds__(256) k_group_final(const float *__restrict__ partial, int n_chunks,
                                                     int n_groups, float *__restrict__ d_gq,
                                                     float *__restrict__ d_gt) {
    const int lane = threadIdx.x & 31;
    const int id = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (id >= n_groups * 7) return;  // the whole warp
    const int g = id / 7, c = id - g * 7;
    const int64_t stride = (int64_t)n_groups * 7;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    int b = lane;
    for (; b + 96 < n_chunks; b += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += partial[(int64_t)(b + 32 * u) * stride + id];
    }
    for (; b < n_chunks; b += 32) acc[0] += partial[(int64_t)b * stride + id];
    float v = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane != 0) return;
    if (c < 4) {
        if (d_gq) d_gq[4 * g + c] = v;
    } else if (d_gt) {
        d_gt[3 * g + (c - 4)] = v;
    }
}

}  // namespace

cudaError_t launch_blend_bwd(const uint2 *ranges, const uint32_t *sorted_vals,
                             const float4 *ranked, const uint32_t *offsets, const CamParams &cam,
                             const RenderParams &rp, const float *final_T,
                             const uint32_t *n_contrib, const float *dL_dimg, float *part, uint8_t *flag,
                             cudaStream_t st) {
    const unsigned tiles = (unsigned)(rp.ntx * rp.nty);
    if (tiles == 0) return cudaSuccess;
#define GC_BWD_ARGS                                                                           \
    ranges, sorted_vals, ranked, offsets, cam.width, cam.height, rp, final_T, n_contrib, dL_dimg, part, flag
    if (rp.tile_w == 16 && rp.tile_h == 16)
        k_blend_bwd<16, 16><<<tiles, kBwdThreads, 0, st>>>(GC_BWD_ARGS);
    else if (rp.tile_w == 8 && rp.tile_h == 32)
        k_blend_bwd<8, 32><<<tiles, kBwdThreads, 0, st>>>(GC_BWD_ARGS);
    else if (rp.tile_w == 32 && rp.tile_h == 8)
        k_blend_bwd<32, 8><<<tiles, kBwdThreads, 0, st>>>(GC_BWD_ARGS);
    else
        return cudaErrorInvalidValue;
#undef GC_BWD_ARGS
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reduce_entries(float *part, const uint32_t *offsets, const uint32_t *touched_r,
                                  const uint32_t *perm, int64_t n, uint32_t cap, uint8_t *flag, float *g2d,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t threads = n * 32;
    k_reduce_entries<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(part, offsets, touched_r, perm, n, cap,
                                                                         flag, g2d);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const GaussSrc &g, const Selection &sel, int64_t n_sel,
                                  const CamParams &cam, const RenderParams &rp, const float *g2d,
                                  const uint32_t *touched, gc_grads out, float *motion_contrib,
                                  cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    GC_DISPATCH_PREC(g.precision, k_preprocess_bwd<PREC_><<<(unsigned)((n_sel + 127) / 128), 128, 0, st>>>(
                                      g, sel, n_sel, cam, rp, g2d, touched, out, motion_contrib))
    note_launches(1);
    return cudaGetLastError();
}

size_t group_partial_floats(int64_t n_sel, int n_groups) {
    const int64_t chunks = (n_sel + kGroupChunk - 1) / kGroupChunk;
    return (size_t)std::max<int64_t>(chunks, 1) * n_groups * 7;
}

cudaError_t launch_motion_scatter(const float *motion_contrib, const Selection &sel, int64_t n_sel, float *d_q,
                                  float *d_t, cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    k_motion_scatter<<<(unsigned)((n_sel + 255) / 256), 256, 0, st>>>(motion_contrib, sel, n_sel, d_q, d_t);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_group_reduce(const float *motion_contrib, const int32_t *group_id,
                                const Selection &sel, int64_t n_sel, int n_groups, float *partial,
                                float *d_group_q, float *d_group_t, cudaStream_t st) {
    const int chunks = (int)((n_sel + kGroupChunk - 1) / kGroupChunk);
    if (chunks > 0) {
        k_group_partial<<<chunks, 128, 0, st>>>(motion_contrib, group_id, sel, n_sel, n_groups, partial);
        note_launches(1);
    }
    k_group_final<<<(n_groups * 7 + 7) / 8, 256, 0, st>>>(partial, chunks, n_groups, d_group_q, d_group_t);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace gc
