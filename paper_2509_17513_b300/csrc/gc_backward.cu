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
//  k_reduce_entries   one warp per Gaussian sums its entries' partials.
//  k_preprocess_bwd   chain rule from (u, v, conic, opacity, rgb) to mean, log-scale,
//                     quaternion, opacity logit, SH and the group motion (Sec. 3.2).
//  k_group_partial /  per-group sums of the motion terms: each thread owns a group and
//  k_group_final      adds its members of a chunk in index order; chunks in order.
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_blend.cuh"
#include "gc_internal.cuh"
#include "gc_sh.cuh"

namespace gc {

namespace {

__device__ __forceinline__ void rect_of(float4 r2, int &x0, int &x1, int &y0, int &y1) {
    const uint32_t rx = __float_as_uint(r2.z), ry = __float_as_uint(r2.w);
    x0 = (int)(rx & 0xffffu);
    x1 = (int)(rx >> 16);
    y0 = (int)(ry & 0xffffu);
    y1 = (int)(ry >> 16);
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

#ifndef GC_BWD_PPT
#define GC_BWD_PPT 1  // pixels per thread in the backward blend (1 measured fastest on B300)
#endif

// Reverse compositing, one CTA per tile of TW x TH = 256 pixels with 256 / PPT
// threads, each owning PPT vertically adjacent pixels.  For every list entry, the
// nine partials are summed over the thread's pixels, then over the warp with a
// transposing butterfly (values 0-7 spread over lane groups, 9 shuffles) plus a
// plain butterfly for value 8, then over the warps in order.
template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(256 / PPT) k_blend_bwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, const uint32_t *__restrict__ offsets, int W, int H, int ntx,
    int tw_log2, int th_log2, float bg0, float bg1, float bg2, int membership,
    const float *__restrict__ final_T, const uint32_t *__restrict__ n_contrib,
    const float *__restrict__ dimg, float *__restrict__ part, int64_t K,
    int32_t *__restrict__ tile_rmax) {
    constexpr int NT = 256 / PPT;
    constexpr int NW = NT / 32;
    __shared__ float4 sA[256];   // u, v, A, B (pre-scaled conic)
    __shared__ float4 sB[256];   // C, opacity, red, green
    __shared__ float4 sC[256];   // blue, column mask, row mask, entry index (bits)
    __shared__ float4 sD[256];   // natural conic a, b, c
    __shared__ float wpart[32][NW][9];
    __shared__ uint32_t s_last_max;

    const int tile = blockIdx.x;
    const int tx = tile % ntx, ty = tile / ntx;
    const int lx = threadIdx.x % TW, lyb = PPT * (threadIdx.x / TW);
    const int px = tx * TW + lx;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float pcx = (float)px + 0.5f;
    const uint32_t xbit = 1u << lx;
    const uint2 range = ranges[tile];
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

    if (threadIdx.x == 0) s_last_max = 0;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, my_last);
    if (lane == 0) atomicMax(&s_last_max, wmax);
    __syncthreads();
    const int n_active = (int)s_last_max;
    if (threadIdx.x == 0)
        tile_rmax[tile] = n_active > 0 ? (int32_t)sorted_vals[range.x + n_active - 1] : -1;

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
                rect_of(c, x0, x1, y0, y1);
                uint32_t cm = 0xffffffffu, rm = 0xffffffffu;
                if (membership == GC_MEMBER_PIXEL) {
                    const int lx0 = max(x0 - tx * TW, 0), lx1 = min(x1 - tx * TW, TW - 1);
                    const int ly0r = max(y0 - ty * TH, 0), ly1r = min(y1 - ty * TH, TH - 1);
                    cm = (lx1 >= lx0) ? ((0xffffffffu >> (31 - lx1)) & (0xffffffffu << lx0)) : 0u;
                    rm = (ly1r >= ly0r) ? ((0xffffffffu >> (31 - ly1r)) & (0xffffffffu << ly0r)) : 0u;
                }
                const int tx0 = x0 >> tw_log2, ty0 = y0 >> th_log2, twid = (x1 >> tw_log2) - tx0 + 1;
                const uint32_t e = offsets[r] + (uint32_t)((ty - ty0) * twid + (tx - tx0));
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

// One warp per rank: sum of the Gaussian's partials over its tiles (entry-major
// partials, nine floats per entry); the result goes to the Gaussian's compact
// position j = perm[r].
__global__ void __launch_bounds__(256) k_reduce_entries(
    const float *__restrict__ part, const uint32_t *__restrict__ offsets,
    const uint32_t *__restrict__ touched_r, const float4 *__restrict__ ranked,
    const int32_t *__restrict__ tile_rmax, const uint32_t *__restrict__ perm, int tw_log2,
    int th_log2, int ntx, int64_t n, float *__restrict__ g2d) {
    const int lane = threadIdx.x & 31;
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= n) return;
    const uint32_t cnt = touched_r[r];
    float acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = 0.f;
    if (cnt) {
        const uint32_t off = offsets[r];
        int x0, x1, y0, y1;
        rect_of(ranked[3 * r + 2], x0, x1, y0, y1);
        const int tx0 = x0 >> tw_log2, ty0 = y0 >> th_log2, twid = (x1 >> tw_log2) - tx0 + 1;
        for (uint32_t j = lane; j < cnt; j += 32) {
            const int t = (ty0 + (int)(j / (uint32_t)twid)) * ntx + tx0 + (int)(j % (uint32_t)twid);
            if ((int64_t)r <= (int64_t)tile_rmax[t]) {
                const float *p = part + (int64_t)(off + j) * 9;
#pragma unroll
                for (int c = 0; c < 9; ++c) acc[c] += p[c];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 9; ++c) {
        float x = acc[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        acc[c] = x;
    }
    float mine = 0.f;
#pragma unroll
    for (int c = 0; c < 9; ++c)
        if (lane == c) mine = acc[c];
    if (lane < 9) g2d[9 * (int64_t)perm[r] + lane] = mine;
}

__device__ __forceinline__ float bf16f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// SH coefficient k, channel c of global Gaussian i (dequantised for BF16/FP8 storage).
__device__ __forceinline__ float sh_coeff(const GaussSrc &G, int64_t i, int k, int c) {
    const int64_t idx = (i * G.K + k) * 3 + c;
    if (G.precision == GC_PREC_FP32) return G.sh[idx];
    __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)G.sh_q[idx], __NV_E4M3);
    return __fmul_rn(__half2float(__half(hr)), G.scales[11 + 3 * k + c]);
}

// Thread per selected Gaussian in index order (coalesced attribute reads and
// gradient writes); g2d and touched are by compact position.
__global__ void __launch_bounds__(128) k_preprocess_bwd(GaussSrc G, Selection sel, int64_t n_sel,
                                                        CamParams cam, RenderParams rp,
                                                        const float *__restrict__ g2d,
                                                        const uint32_t *__restrict__ touched,
                                                        gc_grads out, float *__restrict__ mcontrib) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_sel) return;
    const int64_t i = sel_global(sel, j);
    const int K = G.K;
    float mu[3], ls[3], q[4], logit;
    if (G.precision == GC_PREC_FP32) {
        for (int k = 0; k < 3; ++k) { mu[k] = G.means[3 * i + k]; ls[k] = G.log_scales[3 * i + k]; }
        for (int k = 0; k < 4; ++k) q[k] = G.quats[4 * i + k];
        logit = G.opacity_logits[i];
    } else {
        for (int k = 0; k < 3; ++k) {
            mu[k] = __fmul_rn(bf16f(G.means_h[3 * i + k]), G.scales[k]);
            ls[k] = __fmul_rn(bf16f(G.log_scales_h[3 * i + k]), G.scales[3 + k]);
        }
        for (int k = 0; k < 4; ++k) q[k] = __fmul_rn(bf16f(G.quats_h[4 * i + k]), G.scales[6 + k]);
        logit = __fmul_rn(bf16f(G.opacity_h[i]), G.scales[10]);
    }
    const int g = (G.group_q && G.group_id) ? G.group_id[i] : 0;
    const bool visible = touched[j] != 0;
    float dmu[3] = {0.f, 0.f, 0.f}, dls[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
    float dlogit = 0.f, dgq[4] = {0.f, 0.f, 0.f, 0.f};
    if (visible) {
        const float *d = g2d + 9 * j;
        float gq[4] = {1.f, 0.f, 0.f, 0.f}, gt[3] = {0.f, 0.f, 0.f};
        if (G.group_q) {
            for (int k = 0; k < 4; ++k) gq[k] = G.group_q[4 * g + k];
            for (int k = 0; k < 3; ++k) gt[k] = G.group_t[3 * g + k];
        }
        const float m[3] = {mu[0] + gt[0], mu[1] + gt[1], mu[2] + gt[2]};
        const float a0 = gq[0], a1 = gq[1], a2 = gq[2], a3 = gq[3];
        const float b0 = q[0], b1 = q[1], b2 = q[2], b3 = q[3];
        const float p[4] = {a0 * b0 - a1 * b1 - a2 * b2 - a3 * b3, a0 * b1 + a1 * b0 + a2 * b3 - a3 * b2,
                            a0 * b2 - a1 * b3 + a2 * b0 + a3 * b1, a0 * b3 + a1 * b2 - a2 * b1 + a3 * b0};
        const float pn = sqrtf(p[0] * p[0] + p[1] * p[1] + p[2] * p[2] + p[3] * p[3]);
        const float w = p[0] / pn, x = p[1] / pn, y = p[2] / pn, z = p[3] / pn;
        float R[9];
        R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
        R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
        R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
        float s[3];
        for (int k = 0; k < 3; ++k) s[k] = expf(ls[k]);
        float M[9], S[9];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) M[3 * a + c] = R[3 * a + c] * s[c];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
                S[3 * a + c] = M[3 * a] * M[3 * c] + M[3 * a + 1] * M[3 * c + 1] + M[3 * a + 2] * M[3 * c + 2];
        const float *Wm = cam.R;
        float cpt[3];
        for (int a = 0; a < 3; ++a) cpt[a] = Wm[3 * a] * m[0] + Wm[3 * a + 1] * m[1] + Wm[3 * a + 2] * m[2] + cam.t[a];
        const float cz = cpt[2];
        const float xoz = cpt[0] / cz, yoz = cpt[1] / cz;
        const float limx = rp.frustum_clamp * (0.5f * (float)cam.width / cam.fx);
        const float limy = rp.frustum_clamp * (0.5f * (float)cam.height / cam.fy);
        const bool clx = (xoz > limx) || (xoz < -limx), cly = (yoz > limy) || (yoz < -limy);
        const float xt = fminf(limx, fmaxf(-limx, xoz)), yt = fminf(limy, fmaxf(-limy, yoz));
        const float fx = cam.fx, fy = cam.fy;
        const float J00 = fx / cz, J11 = fy / cz, J02 = -fx * xt / cz, J12 = -fy * yt / cz;
        float T[6];
        for (int c = 0; c < 3; ++c) {
            T[c] = J00 * Wm[c] + J02 * Wm[6 + c];
            T[3 + c] = J11 * Wm[3 + c] + J12 * Wm[6 + c];
        }
        float TS[6];  // T Sigma
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 3; ++c) TS[3 * a + c] = T[3 * a] * S[c] + T[3 * a + 1] * S[3 + c] + T[3 * a + 2] * S[6 + c];
        const float A = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2] + rp.dilation;
        const float B = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
        const float Cc = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5] + rp.dilation;
        const float det = A * Cc - B * B;
        const float qa = Cc / det, qb = -B / det, qc = A / det;
        const float op = 1.f / (1.f + expf(-logit));
        // opacity
        dlogit = d[5] * op * (1.f - op);
        // colour
        float dv[3] = {m[0] - cam.campos[0], m[1] - cam.campos[1], m[2] - cam.campos[2]};
        const float dn = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        const float dir[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
        float Y[16];
        sh_basis(G.sh_degree, dir[0], dir[1], dir[2], Y);
        float raw[3] = {0.5f, 0.5f, 0.5f};
        float wsh[16];
        for (int k = 0; k < K; ++k) {
            raw[0] += Y[k] * sh_coeff(G, i, k, 0);
            raw[1] += Y[k] * sh_coeff(G, i, k, 1);
            raw[2] += Y[k] * sh_coeff(G, i, k, 2);
        }
        const float draw[3] = {raw[0] > 0.f ? d[6] : 0.f, raw[1] > 0.f ? d[7] : 0.f, raw[2] > 0.f ? d[8] : 0.f};
        for (int k = 0; k < K; ++k) {
            wsh[k] = sh_coeff(G, i, k, 0) * draw[0] + sh_coeff(G, i, k, 1) * draw[1] +
                     sh_coeff(G, i, k, 2) * draw[2];
            if (out.d_sh) {
                const int64_t idx = (i * K + k) * 3;
                out.d_sh[idx] = Y[k] * draw[0];
                out.d_sh[idx + 1] = Y[k] * draw[1];
                out.d_sh[idx + 2] = Y[k] * draw[2];
            }
        }
        float ddx, ddy, ddz;
        sh_basis_vjp(G.sh_degree, dir[0], dir[1], dir[2], wsh, ddx, ddy, ddz);
        const float dd = dir[0] * ddx + dir[1] * ddy + dir[2] * ddz;
        dmu[0] = (ddx - dir[0] * dd) / dn;
        dmu[1] = (ddy - dir[1] * dd) / dn;
        dmu[2] = (ddz - dir[2] * dd) / dn;
        // conic -> Sigma2: GS = -Q Gc Q, Gc = [[da, db/2], [db/2, dc]]
        const float gca = d[2], gcb = 0.5f * d[3], gcc = d[4];
        const float t00 = qa * gca + qb * gcb, t01 = qa * gcb + qb * gcc;
        const float t10 = qb * gca + qc * gcb, t11 = qb * gcb + qc * gcc;
        const float GS00 = -(t00 * qa + t01 * qb), GS01 = -(t00 * qb + t01 * qc);
        const float GS11 = -(t10 * qb + t11 * qc);
        const float GSm[4] = {GS00, GS01, GS01, GS11};
        // dSigma = T^T GS T, dT = 2 GS T Sigma
        float dSig[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                float acc = 0.f;
                for (int u2 = 0; u2 < 2; ++u2)
                    for (int v2 = 0; v2 < 2; ++v2) acc += T[3 * u2 + a] * GSm[2 * u2 + v2] * T[3 * v2 + b];
                dSig[3 * a + b] = acc;
            }
        float dT[6];
        for (int u2 = 0; u2 < 2; ++u2)
            for (int b = 0; b < 3; ++b) dT[3 * u2 + b] = 2.f * (GSm[2 * u2] * TS[b] + GSm[2 * u2 + 1] * TS[3 + b]);
        float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
        for (int b = 0; b < 3; ++b) {
            dJ00 += dT[b] * Wm[b];
            dJ02 += dT[b] * Wm[6 + b];
            dJ11 += dT[3 + b] * Wm[3 + b];
            dJ12 += dT[3 + b] * Wm[6 + b];
        }
        const float z2 = cz * cz;
        float dc[3] = {0.f, 0.f, 0.f};
        dc[2] += dJ00 * (-fx / z2) + dJ11 * (-fy / z2);
        if (clx) dc[2] += dJ02 * (fx * xt / z2);
        else { dc[0] += dJ02 * (-fx / z2); dc[2] += dJ02 * (2.f * fx * cpt[0] / (z2 * cz)); }
        if (cly) dc[2] += dJ12 * (fy * yt / z2);
        else { dc[1] += dJ12 * (-fy / z2); dc[2] += dJ12 * (2.f * fy * cpt[1] / (z2 * cz)); }
        dc[0] += d[0] * fx / cz; dc[2] += d[0] * (-fx * cpt[0] / z2);
        dc[1] += d[1] * fy / cz; dc[2] += d[1] * (-fy * cpt[1] / z2);
        for (int a = 0; a < 3; ++a) dmu[a] += Wm[a] * dc[0] + Wm[3 + a] * dc[1] + Wm[6 + a] * dc[2];
        // Sigma = M M^T
        float dR[9];
        for (int c = 0; c < 3; ++c) {
            float ds = 0.f;
            for (int a = 0; a < 3; ++a) {
                float dM = 0.f;
                for (int b = 0; b < 3; ++b) dM += (dSig[3 * a + b] + dSig[3 * b + a]) * M[3 * b + c];
                ds += dM * R[3 * a + c];
                dR[3 * a + c] = dM * s[c];
            }
            dls[c] = ds * s[c];
        }
        // R(q^): vjp to the unit quaternion, then through the normalisation and q_g (x) q
        float dqn[4];
        dqn[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        dqn[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - w * dR[5] + z * dR[6] + w * dR[7]) - 4.f * x * (dR[4] + dR[8]);
        dqn[2] = 2.f * (x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7]) - 4.f * y * (dR[0] + dR[8]);
        dqn[3] = 2.f * (-w * dR[1] + x * dR[2] + w * dR[3] + y * dR[5] + x * dR[6] + y * dR[7]) - 4.f * z * (dR[0] + dR[4]);
        const float qd = w * dqn[0] + x * dqn[1] + y * dqn[2] + z * dqn[3];
        const float dp[4] = {(dqn[0] - w * qd) / pn, (dqn[1] - x * qd) / pn, (dqn[2] - y * qd) / pn,
                             (dqn[3] - z * qd) / pn};
        // dq = L(q_g)^T dp ; dq_g = Rm(q)^T dp
        dq[0] = a0 * dp[0] + a1 * dp[1] + a2 * dp[2] + a3 * dp[3];
        dq[1] = -a1 * dp[0] + a0 * dp[1] + a3 * dp[2] - a2 * dp[3];
        dq[2] = -a2 * dp[0] - a3 * dp[1] + a0 * dp[2] + a1 * dp[3];
        dq[3] = -a3 * dp[0] + a2 * dp[1] - a1 * dp[2] + a0 * dp[3];
        dgq[0] = b0 * dp[0] + b1 * dp[1] + b2 * dp[2] + b3 * dp[3];
        dgq[1] = -b1 * dp[0] + b0 * dp[1] - b3 * dp[2] + b2 * dp[3];
        dgq[2] = -b2 * dp[0] + b3 * dp[1] + b0 * dp[2] - b1 * dp[3];
        dgq[3] = -b3 * dp[0] - b2 * dp[1] + b1 * dp[2] + b0 * dp[3];
    } else if (out.d_sh) {
        for (int k = 0; k < 3 * K; ++k) out.d_sh[i * 3 * K + k] = 0.f;
    }
    if (out.d_means) for (int k = 0; k < 3; ++k) out.d_means[3 * i + k] = dmu[k];
    if (out.d_log_scales) for (int k = 0; k < 3; ++k) out.d_log_scales[3 * i + k] = dls[k];
    if (out.d_quats) for (int k = 0; k < 4; ++k) out.d_quats[4 * i + k] = dq[k];
    if (out.d_opacity_logits) out.d_opacity_logits[i] = dlogit;
    if (mcontrib) {
        float *mc = mcontrib + 7 * j;
        for (int k = 0; k < 4; ++k) mc[k] = dgq[k];
        for (int k = 0; k < 3; ++k) mc[4 + k] = dmu[k];
    }
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

// One thread per (group, component): the chunk partials summed in chunk order.
__global__ void k_group_final(const float *__restrict__ partial, int n_chunks, int n_groups,
                              float *__restrict__ d_gq, float *__restrict__ d_gt) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_groups * 7) return;
    const int g = id / 7, c = id - g * 7;
    float acc = 0.f;
    const int64_t stride = (int64_t)n_groups * 7;
    int b = 0;
    for (; b + 8 <= n_chunks; b += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = partial[(int64_t)(b + u) * stride + id];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc += v[u];
    }
    for (; b < n_chunks; ++b) acc += partial[(int64_t)b * stride + id];
    if (c < 4) {
        if (d_gq) d_gq[4 * g + c] = acc;
    } else if (d_gt) {
        d_gt[3 * g + (c - 4)] = acc;
    }
}

}  // namespace

cudaError_t launch_blend_bwd(const uint2 *ranges, const uint32_t *sorted_vals,
                             const float4 *ranked, const uint32_t *offsets, const CamParams &cam,
                             const RenderParams &rp, const float *final_T,
                             const uint32_t *n_contrib, const float *dL_dimg, float *part,
                             int64_t K, int32_t *tile_rmax, cudaStream_t st) {
    const unsigned tiles = (unsigned)(rp.ntx * rp.nty);
    if (tiles == 0) return cudaSuccess;
#define GC_BWD_ARGS                                                                           \
    ranges, sorted_vals, ranked, offsets, cam.width, cam.height, rp.ntx, rp.tile_w_log2,       \
        rp.tile_h_log2, rp.bg[0], rp.bg[1], rp.bg[2], rp.membership, final_T, n_contrib,      \
        dL_dimg, part, K, tile_rmax
    constexpr int kThreads = 256 / GC_BWD_PPT;
    if (rp.tile_w == 16 && rp.tile_h == 16)
        k_blend_bwd<16, 16, GC_BWD_PPT><<<tiles, kThreads, 0, st>>>(GC_BWD_ARGS);
    else if (rp.tile_w == 8 && rp.tile_h == 32)
        k_blend_bwd<8, 32, GC_BWD_PPT><<<tiles, kThreads, 0, st>>>(GC_BWD_ARGS);
    else if (rp.tile_w == 32 && rp.tile_h == 8)
        k_blend_bwd<32, 8, GC_BWD_PPT><<<tiles, kThreads, 0, st>>>(GC_BWD_ARGS);
    else
        return cudaErrorInvalidValue;
#undef GC_BWD_ARGS
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reduce_entries(const float *part, const uint32_t *offsets,
                                  const uint32_t *touched_r, const float4 *ranked,
                                  const int32_t *tile_rmax, const uint32_t *perm,
                                  const RenderParams &rp, int64_t n, float *g2d, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t threads = n * 32;
    k_reduce_entries<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        part, offsets, touched_r, ranked, tile_rmax, perm, rp.tile_w_log2, rp.tile_h_log2, rp.ntx, n, g2d);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const GaussSrc &g, const Selection &sel, int64_t n_sel,
                                  const CamParams &cam, const RenderParams &rp, const float *g2d,
                                  const uint32_t *touched, gc_grads out, float *motion_contrib,
                                  cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    k_preprocess_bwd<<<(unsigned)((n_sel + 127) / 128), 128, 0, st>>>(g, sel, n_sel, cam, rp, g2d, touched,
                                                                       out, motion_contrib);
    note_launches(1);
    return cudaGetLastError();
}

size_t group_partial_floats(int64_t n_sel, int n_groups) {
    const int64_t chunks = (n_sel + kGroupChunk - 1) / kGroupChunk;
    return (size_t)std::max<int64_t>(chunks, 1) * n_groups * 7;
}

cudaError_t launch_group_reduce(const float *motion_contrib, const int32_t *group_id,
                                const Selection &sel, int64_t n_sel, int n_groups, float *partial,
                                float *d_group_q, float *d_group_t, cudaStream_t st) {
    const int chunks = (int)((n_sel + kGroupChunk - 1) / kGroupChunk);
    if (chunks > 0) {
        k_group_partial<<<chunks, 128, 0, st>>>(motion_contrib, group_id, sel, n_sel, n_groups, partial);
        note_launches(1);
    }
    k_group_final<<<(n_groups * 7 + 127) / 128, 128, 0, st>>>(partial, chunks, n_groups, d_group_q, d_group_t);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace gc
