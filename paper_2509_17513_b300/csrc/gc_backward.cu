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

template <int TW, int TH>
__global__ void __launch_bounds__(256) k_blend_bwd(
    const uint2 *__restrict__ ranges, const uint32_t *__restrict__ sorted_vals,
    const float4 *__restrict__ ranked, const uint32_t *__restrict__ offsets, int W, int H, int ntx,
    int tw_log2, int th_log2, float bg0, float bg1, float bg2, int membership,
    const float *__restrict__ final_T, const uint32_t *__restrict__ n_contrib,
    const float *__restrict__ dimg, float *__restrict__ part, int64_t K,
    int32_t *__restrict__ tile_rmax) {
    __shared__ float4 sA[256];   // u, v, conic a, conic b
    __shared__ float4 sB[256];   // conic c, opacity, red, green
    __shared__ float4 sC[256];   // blue, column mask, row mask, entry index (bits)
    __shared__ float wpart[32][8][9];
    __shared__ uint32_t s_last_max;

    const int tile = blockIdx.x;
    const int tx = tile % ntx, ty = tile / ntx;
    const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
    const int px = tx * TW + lx, py = ty * TH + ly;
    const bool inside = px < W && py < H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float pcx = (float)px + 0.5f, pcy = (float)py + 0.5f;
    const uint32_t xbit = 1u << lx, ybit = 1u << ly;
    const uint2 range = ranges[tile];

    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t last = 0;
    if (inside) {
        const size_t hw = (size_t)W * H, p = (size_t)py * W + px;
        T = final_T[p];
        last = n_contrib[p];
        g0 = dimg[p];
        g1 = dimg[hw + p];
        g2 = dimg[2 * hw + p];
    }
    float A0 = bg0, A1 = bg1, A2 = bg2;  // colour behind, normalised by the transmittance

    if (threadIdx.x == 0) s_last_max = 0;
    __syncthreads();
    // max over the tile of the list position after the last blended entry
    uint32_t wmax = __reduce_max_sync(0xffffffffu, last);
    if (lane == 0) atomicMax(&s_last_max, wmax);
    __syncthreads();
    const int n_active = (int)s_last_max;
    if (threadIdx.x == 0)
        tile_rmax[tile] = n_active > 0 ? (int32_t)sorted_vals[range.x + n_active - 1] : -1;

    for (int hi = n_active; hi > 0; hi -= 256) {
        const int lo = max(hi - 256, 0);
        __syncthreads();
        {
            const int k = lo + (int)threadIdx.x;
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
                    const int ly0 = max(y0 - ty * TH, 0), ly1 = min(y1 - ty * TH, TH - 1);
                    cm = (lx1 >= lx0) ? ((0xffffffffu >> (31 - lx1)) & (0xffffffffu << lx0)) : 0u;
                    rm = (ly1 >= ly0) ? ((0xffffffffu >> (31 - ly1)) & (0xffffffffu << ly0)) : 0u;
                }
                const int tx0 = x0 >> tw_log2, ty0 = y0 >> th_log2, twid = (x1 >> tw_log2) - tx0 + 1;
                const uint32_t e = offsets[r] + (uint32_t)((ty - ty0) * twid + (tx - tx0));
                sA[threadIdx.x] = a;
                sB[threadIdx.x] = bb;
                sC[threadIdx.x] = make_float4(c.x, __uint_as_float(cm), __uint_as_float(rm), __uint_as_float(e));
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
                bool contrib = false;
                if ((uint32_t)k < last) {
                    const float4 c4 = sC[s];
                    if ((__float_as_uint(c4.y) & xbit) && (__float_as_uint(c4.z) & ybit)) {
                        const float4 a = sA[s];
                        const float4 bb = sB[s];
                        const float dx = pcx - a.x, dy = pcy - a.y;
                        const float power = blend_power(a.z, a.w, bb.x, dx, dy);
                        if (!(power > 0.f)) {
                            float G;
                            const float a0 = blend_raw_alpha(bb.y, power, G);
                            const float alpha = fminf(kAlphaMax, a0);
                            if (!(alpha < kAlphaMin)) {
                                contrib = true;
                                T = T / (1.f - alpha);
                                const float w = alpha * T;
                                v[6] = w * g0;
                                v[7] = w * g1;
                                v[8] = w * g2;
                                const float dal = T * (g0 * (bb.z - A0) + g1 * (bb.w - A1) + g2 * (c4.x - A2));
                                A0 = alpha * bb.z + (1.f - alpha) * A0;
                                A1 = alpha * bb.w + (1.f - alpha) * A1;
                                A2 = alpha * c4.x + (1.f - alpha) * A2;
                                if (!(a0 > kAlphaMax)) {
                                    v[5] = G * dal;
                                    const float dp = alpha * dal;
                                    v[0] = (a.z * dx + a.w * dy) * dp;
                                    v[1] = (a.w * dx + bb.x * dy) * dp;
                                    v[2] = -0.5f * dx * dx * dp;
                                    v[3] = -dx * dy * dp;
                                    v[4] = -0.5f * dy * dy * dp;
                                }
                            }
                        }
                    }
                }
                if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
                    for (int c = 0; c < 9; ++c) {
                        float x = v[c];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                        v[c] = x;
                    }
                }
                float mine = 0.f;
#pragma unroll
                for (int c = 0; c < 9; ++c)
                    if (lane == c) mine = v[c];
                if (lane < 9) wpart[k - gbot][warp][lane] = mine;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < (gtop - gbot) * 9; idx += 256) {
                const int q = idx / 9, c = idx - q * 9;
                float acc = 0.f;
#pragma unroll
                for (int w = 0; w < 8; ++w) acc += wpart[q][w][c];
                const uint32_t e = __float_as_uint(sC[gbot + q - lo].w);
                part[(int64_t)c * K + e] = acc;
            }
            __syncthreads();
        }
    }
}

// One warp per rank: sum of the Gaussian's partials over its tiles.
__global__ void __launch_bounds__(256) k_reduce_entries(
    const float *__restrict__ part, int64_t K, const uint32_t *__restrict__ offsets,
    const uint32_t *__restrict__ touched_r, const float4 *__restrict__ ranked,
    const int32_t *__restrict__ tile_rmax, int tw_log2, int th_log2, int ntx, int64_t n,
    float *__restrict__ g2d) {
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
#pragma unroll
                for (int c = 0; c < 9; ++c) acc[c] += part[(int64_t)c * K + off + j];
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
    if (lane < 9) g2d[9 * r + lane] = acc[lane];
}

__device__ __forceinline__ float bf16f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// SH coefficient k, channel c of global Gaussian i (dequantised for BF16/FP8 storage).
__device__ __forceinline__ float sh_coeff(const GaussSrc &G, int64_t i, int k, int c) {
    const int64_t idx = (i * G.K + k) * 3 + c;
    if (G.precision == GC_PREC_FP32) return G.sh[idx];
    __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)G.sh_q[idx], __NV_E4M3);
    return __fmul_rn(__half2float(__half(hr)), G.scales[11 + 3 * k + c]);
}

__global__ void __launch_bounds__(128) k_preprocess_bwd(GaussSrc G, Selection sel, int64_t n_sel,
                                                        CamParams cam, RenderParams rp,
                                                        const uint32_t *__restrict__ perm,
                                                        const float *__restrict__ g2d,
                                                        const uint32_t *__restrict__ touched_r,
                                                        gc_grads out, float *__restrict__ mcontrib) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_sel) return;
    const int64_t j = perm[r];
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
    const bool visible = touched_r[r] != 0;
    float dmu[3] = {0.f, 0.f, 0.f}, dls[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
    float dlogit = 0.f, dgq[4] = {0.f, 0.f, 0.f, 0.f};
    if (visible) {
        const float *d = g2d + 9 * r;
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

constexpr int kGroupChunk = 1024;

// Per chunk of 1024 compact positions, each thread sums the motion terms of the
// chunk's members of the groups it owns, in position order.
__global__ void __launch_bounds__(256) k_group_partial(const float *__restrict__ mcontrib,
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

__global__ void k_group_final(const float *__restrict__ partial, int n_chunks, int n_groups,
                              float *__restrict__ d_gq, float *__restrict__ d_gt) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int b = 0; b < n_chunks; ++b) {
        const float *p = partial + ((int64_t)b * n_groups + g) * 7;
#pragma unroll
        for (int c = 0; c < 7; ++c) acc[c] += p[c];
    }
    if (d_gq) for (int c = 0; c < 4; ++c) d_gq[4 * g + c] = acc[c];
    if (d_gt) for (int c = 0; c < 3; ++c) d_gt[3 * g + c] = acc[4 + c];
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
    if (rp.tile_w == 16 && rp.tile_h == 16)
        k_blend_bwd<16, 16><<<tiles, 256, 0, st>>>(GC_BWD_ARGS);
    else if (rp.tile_w == 8 && rp.tile_h == 32)
        k_blend_bwd<8, 32><<<tiles, 256, 0, st>>>(GC_BWD_ARGS);
    else if (rp.tile_w == 32 && rp.tile_h == 8)
        k_blend_bwd<32, 8><<<tiles, 256, 0, st>>>(GC_BWD_ARGS);
    else
        return cudaErrorInvalidValue;
#undef GC_BWD_ARGS
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_reduce_entries(const float *part, int64_t K, const uint32_t *offsets,
                                  const uint32_t *touched_r, const float4 *ranked,
                                  const int32_t *tile_rmax, const RenderParams &rp, int64_t n,
                                  float *g2d, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t threads = n * 32;
    k_reduce_entries<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        part, K, offsets, touched_r, ranked, tile_rmax, rp.tile_w_log2, rp.tile_h_log2, rp.ntx, n, g2d);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const GaussSrc &g, const Selection &sel, int64_t n_sel,
                                  const CamParams &cam, const RenderParams &rp,
                                  const uint32_t *perm, const float *g2d,
                                  const uint32_t *touched_r, gc_grads out, float *motion_contrib,
                                  cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    k_preprocess_bwd<<<(unsigned)((n_sel + 127) / 128), 128, 0, st>>>(g, sel, n_sel, cam, rp, perm, g2d,
                                                                       touched_r, out, motion_contrib);
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
        k_group_partial<<<chunks, 256, 0, st>>>(motion_contrib, group_id, sel, n_sel, n_groups, partial);
        note_launches(1);
    }
    k_group_final<<<(n_groups + 127) / 128, 128, 0, st>>>(partial, chunks, n_groups, d_group_q, d_group_t);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace gc
