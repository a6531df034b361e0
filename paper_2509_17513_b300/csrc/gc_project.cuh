// gc_project.cuh - per-Gaussian motion, activation, EWA projection, footprint and
// SH colour (4DGCPro Sec. 3.1 / 3.2), shared by the single-frame and the batched
// preprocess kernels.
//
// The values that decide integers - visibility, the depth key and the pixel
// footprint - follow the binning specification op by op: every operation is a
// separately rounded IEEE binary32 op (__fmul_rn / __fadd_rn / __fdiv_rn /
// __fsqrt_rn are never fused into FMA), and s = (float)exp((double)log_s).
// Colour (SH) is free arithmetic: it only feeds continuous values.
#pragma once
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "gc_blend.cuh"
#include "gc_exact.cuh"
#include "gc_internal.cuh"
#include "gc_sh.cuh"

namespace gc {

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

__device__ __forceinline__ float e4m3_to_f32(uint8_t b) {
    __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(hr));
}

// Loads the attributes of global Gaussian i (dequantised for BF16/FP8).
struct Attr {
    float mu[3], ls[3], q[4], logit;
    int g;
};

template <int PREC>
__device__ __forceinline__ void load_attr(const GaussSrc &G, int64_t i, Attr &a, const Residual &res) {
    if constexpr (PREC == GC_PREC_FP32) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.mu[k] = G.means[3 * i + k];
            a.ls[k] = G.log_scales[3 * i + k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) a.q[k] = G.quats[4 * i + k];
        a.logit = G.opacity_logits[i];
    } else if constexpr (PREC == GC_PREC_PLANES) {
        const PlaneLoc p = plane_loc(G, i);
#pragma unroll
        for (int k = 0; k < 3; ++k) a.mu[k] = plane_value(G, p, k);
#pragma unroll
        for (int k = 0; k < 4; ++k) a.q[k] = plane_value(G, p, 3 + k);
#pragma unroll
        for (int k = 0; k < 3; ++k) a.ls[k] = plane_value(G, p, 7 + k);
        a.logit = plane_value(G, p, 10);
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a.mu[k] = fmul(bf16_to_f32(G.means_h[3 * i + k]), G.scales[k]);
            a.ls[k] = fmul(bf16_to_f32(G.log_scales_h[3 * i + k]), G.scales[3 + k]);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) a.q[k] = fmul(bf16_to_f32(G.quats_h[4 * i + k]), G.scales[6 + k]);
        a.logit = fmul(bf16_to_f32(G.opacity_h[i]), G.scales[10]);
    }
    // residual deformation (Eq. 7): one FP32 addition per attribute, before activation
    if (res.ls) {
#pragma unroll
        for (int k = 0; k < 3; ++k) a.ls[k] = fadd(a.ls[k], res.ls[3 * i + k]);
    }
    if (res.logit) a.logit = fadd(a.logit, res.logit[i]);
    a.g = G.per_gaussian ? (int)i : (G.group_id ? G.group_id[i] : 0);
}

// SH coefficient k, channel c (FP32 or FP8 storage; decoded planes go through sh_plane).
template <int PREC>
__device__ __forceinline__ float load_sh(const GaussSrc &G, int64_t i, int k, int c, const Residual &res) {
    int64_t idx = (i * G.K + k) * 3 + c;
    const float f = PREC == GC_PREC_FP32 ? G.sh[idx] : fmul(e4m3_to_f32(G.sh_q[idx]), G.scales[11 + 3 * k + c]);
    return res.sh ? fadd(f, res.sh[idx]) : f;
}

template <int PREC>
__device__ __forceinline__ float sh_plane(const GaussSrc &G, const PlaneLoc &p, int64_t i, int k, int c,
                                          const Residual &res) {
    const float f = plane_value(G, p, 11 + 3 * k + c);
    return res.sh ? fadd(f, res.sh[(i * G.K + k) * 3 + c]) : f;
}


// Result of projecting one Gaussian: the three record float4s, the depth key
// (kCulledKey when culled), the number of tiles touched and the tile rectangle.
struct Proj {
    float4 r0, r1, r2, r3, r4;
    uint32_t key, ntouch;
    int tx0, tx1, ty0, ty1;
};

// Projects global Gaussian i under group motion (group_q == NULL: identity) into
// camera `cam` with options `rp`.
// Per-Gaussian values that depend on no camera or motion: the scales
// s = (float)exp((double)log_s) (step 5) and tau = (float)(2 ln(255 / (1 + exp(-logit))))
// (step 14).  A batch computes them once per Gaussian instead of once per request.
template <int PREC>
__device__ __forceinline__ float4 gaussian_activation(const GaussSrc &G, int64_t i) {
    Attr A;
    load_attr<PREC>(G, i, A, Residual{nullptr, nullptr, nullptr});
    return make_float4(exp_f32_of_f64(A.ls[0]), exp_f32_of_f64(A.ls[1]), exp_f32_of_f64(A.ls[2]),
                       tau_f32_of_f64(A.logit));
}

// act: NULL, or the cached gaussian_activation of every Gaussian (bit-identical results;
// only without residuals).  res: the frame's residual deformation.
template <int PREC>
__device__ __forceinline__ void project_gaussian(const GaussSrc &G, int64_t i, const float *group_q,
                                                const float *group_t, int n_groups,
                                                const CamParams &cam, const RenderParams &rp,
                                                Proj &P, const float4 *act, const Residual &res) {
    Attr A;
    load_attr<PREC>(G, i, A, res);
    P.key = kCulledKey;
    P.ntouch = 0;
    P.tx0 = P.tx1 = P.ty0 = P.ty1 = 0;
    P.r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    P.r1 = P.r0;
    P.r2 = P.r0;
    P.r3 = P.r0;
    P.r4 = P.r0;
    do {
        float gq[4] = {1.f, 0.f, 0.f, 0.f}, gt[3] = {0.f, 0.f, 0.f};
        if (group_q && (A.g < 0 || A.g >= n_groups)) break;  // invalid group id: culled
        if (group_q) {
#pragma unroll
            for (int k = 0; k < 4; ++k) gq[k] = group_q[4 * A.g + k];
#pragma unroll
            for (int k = 0; k < 3; ++k) gt[k] = group_t[3 * A.g + k];
        }
        // 1. moved mean
        const float m0 = fadd(A.mu[0], gt[0]), m1 = fadd(A.mu[1], gt[1]), m2 = fadd(A.mu[2], gt[2]);
        // 2. p = q_g (x) q
        const float a0 = gq[0], a1 = gq[1], a2 = gq[2], a3 = gq[3];
        const float b0 = A.q[0], b1 = A.q[1], b2 = A.q[2], b3 = A.q[3];
        float p0 = fmul(a0, b0); p0 = fsub(p0, fmul(a1, b1)); p0 = fsub(p0, fmul(a2, b2)); p0 = fsub(p0, fmul(a3, b3));
        float p1 = fmul(a0, b1); p1 = fadd(p1, fmul(a1, b0)); p1 = fadd(p1, fmul(a2, b3)); p1 = fsub(p1, fmul(a3, b2));
        float p2 = fmul(a0, b2); p2 = fsub(p2, fmul(a1, b3)); p2 = fadd(p2, fmul(a2, b0)); p2 = fadd(p2, fmul(a3, b1));
        float p3 = fmul(a0, b3); p3 = fadd(p3, fmul(a1, b2)); p3 = fsub(p3, fmul(a2, b1)); p3 = fadd(p3, fmul(a3, b0));
        // 3. normalise
        float n2 = fmul(p0, p0); n2 = fadd(n2, fmul(p1, p1)); n2 = fadd(n2, fmul(p2, p2)); n2 = fadd(n2, fmul(p3, p3));
        if (!(n2 > 0.f)) break;
        const float nn = __fsqrt_rn(n2);
        const float w = fdiv(p0, nn), x = fdiv(p1, nn), y = fdiv(p2, nn), z = fdiv(p3, nn);
        // 4. rotation
        const float xx = fmul(x, x), yy = fmul(y, y), zz = fmul(z, z);
        const float xy = fmul(x, y), xz = fmul(x, z), yz = fmul(y, z);
        const float wx = fmul(w, x), wy = fmul(w, y), wz = fmul(w, z);
        float R[9];
        R[0] = fsub(1.f, fmul(2.f, fadd(yy, zz))); R[1] = fmul(2.f, fsub(xy, wz)); R[2] = fmul(2.f, fadd(xz, wy));
        R[3] = fmul(2.f, fadd(xy, wz)); R[4] = fsub(1.f, fmul(2.f, fadd(xx, zz))); R[5] = fmul(2.f, fsub(yz, wx));
        R[6] = fmul(2.f, fsub(xz, wy)); R[7] = fmul(2.f, fadd(yz, wx)); R[8] = fsub(1.f, fmul(2.f, fadd(xx, yy)));
        // 5. scales: the FP32 rounding of the FP64 exponential
        float s[3];
        float4 av;
        if (act) {
            av = act[i];
            s[0] = av.x;
            s[1] = av.y;
            s[2] = av.z;
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) s[k] = exp_f32_of_f64(A.ls[k]);
        }
        // 6-7. M = R diag(s), Sigma = M M^T
        float M[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) M[3 * r + c] = fmul(R[3 * r + c], s[c]);
        float S[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = r; c < 3; ++c) {
                float acc = fmul(M[3 * r], M[3 * c]);
                acc = fadd(acc, fmul(M[3 * r + 1], M[3 * c + 1]));
                acc = fadd(acc, fmul(M[3 * r + 2], M[3 * c + 2]));
                S[3 * r + c] = acc;
                S[3 * c + r] = acc;
            }
        // 8. camera point
        float cp[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float acc = fmul(cam.R[3 * r], m0);
            acc = fadd(acc, fmul(cam.R[3 * r + 1], m1));
            acc = fadd(acc, fmul(cam.R[3 * r + 2], m2));
            cp[r] = fadd(acc, cam.t[r]);
        }
        const float cz = cp[2];
        if (!(cz > rp.near_plane)) break;
        // 9. clamped Jacobian, T = J W, Sigma2 = T Sigma T^T
        const float xoz = fdiv(cp[0], cz), yoz = fdiv(cp[1], cz);
        const float limx = fmul(rp.frustum_clamp, fdiv(fmul(0.5f, (float)cam.width), cam.fx));
        const float limy = fmul(rp.frustum_clamp, fdiv(fmul(0.5f, (float)cam.height), cam.fy));
        const float xt = fminf(limx, fmaxf(-limx, xoz));
        const float yt = fminf(limy, fmaxf(-limy, yoz));
        const float J00 = fdiv(cam.fx, cz), J11 = fdiv(cam.fy, cz);
        const float J02 = -fdiv(fmul(cam.fx, xt), cz), J12 = -fdiv(fmul(cam.fy, yt), cz);
        float T[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T[c] = fadd(fmul(J00, cam.R[c]), fmul(J02, cam.R[6 + c]));
            T[3 + c] = fadd(fmul(J11, cam.R[3 + c]), fmul(J12, cam.R[6 + c]));
        }
        float U[6];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float acc = fmul(T[3 * r], S[c]);
                acc = fadd(acc, fmul(T[3 * r + 1], S[3 + c]));
                acc = fadd(acc, fmul(T[3 * r + 2], S[6 + c]));
                U[3 * r + c] = acc;
            }
        float ca = fmul(U[0], T[0]); ca = fadd(ca, fmul(U[1], T[1])); ca = fadd(ca, fmul(U[2], T[2])); ca = fadd(ca, rp.dilation);
        float cb = fmul(U[0], T[3]); cb = fadd(cb, fmul(U[1], T[4])); cb = fadd(cb, fmul(U[2], T[5]));
        float cc = fmul(U[3], T[3]); cc = fadd(cc, fmul(U[4], T[4])); cc = fadd(cc, fmul(U[5], T[5])); cc = fadd(cc, rp.dilation);
        // 10. conic
        const float det = fsub(fmul(ca, cc), fmul(cb, cb));
        if (!(det > 0.f)) break;
        const float ia = fdiv(cc, det), ib = -fdiv(cb, det), ic = fdiv(ca, det);
        // 11. radius
        const float mid = fmul(0.5f, fadd(ca, cc));
        const float disc = fsub(fmul(mid, mid), det);
        const float lam = fadd(mid, __fsqrt_rn(fmaxf(0.f, disc)));
        const float rf = ceilf(fmul(3.f, __fsqrt_rn(lam)));
        // 12. centre
        const float u = fadd(fmul(cam.fx, xoz), cam.cx);
        const float v = fadd(fmul(cam.fy, yoz), cam.cy);
        if (!isfinite(u) || !isfinite(v) || !isfinite(rf)) break;
        // 13. clipped pixel rectangle
        float fx0 = ceilf(fsub(fsub(u, rf), 0.5f)), fx1 = floorf(fsub(fadd(u, rf), 0.5f));
        float fy0 = ceilf(fsub(fsub(v, rf), 0.5f)), fy1 = floorf(fsub(fadd(v, rf), 0.5f));
        fx0 = fmaxf(fx0, 0.f);
        fy0 = fmaxf(fy0, 0.f);
        fx1 = fminf(fx1, (float)(cam.width - 1));
        fy1 = fminf(fy1, (float)(cam.height - 1));
        if (!(fx0 <= fx1) || !(fy0 <= fy1)) break;
        // 14. alpha footprint: o exp(-Q/2) >= 1/255 needs Q <= tau = 2 ln(255 o); the
        //     ellipse Q <= tau_c (tau plus a margin that covers the blend's FP32 rounding)
        //     has half-extents sqrt(tau_c ic / det_c), sqrt(tau_c ia / det_c)
        float tc_out = 0.f;
        if (rp.alpha_cull) {
            const float tau = act ? av.w : tau_f32_of_f64(A.logit);
            if (!(tau > 0.f)) break;  // opacity <= 1/255: never blended
            const float t1 = fadd(rf, 1.f);
            const float mt = fmul(fadd(fadd(ia, fmul(2.f, fabsf(ib))), ic), fmul(t1, t1));
            const float tc = fadd(fadd(tau, 0.02f), fmul(1e-6f, mt));
            tc_out = tc;
            const float detc = fsub(fmul(ia, ic), fmul(ib, ib));
            if (detc > 0.f) {
                const float xa = __fsqrt_rn(fdiv(fmul(tc, ic), detc));
                const float ya = __fsqrt_rn(fdiv(fmul(tc, ia), detc));
                fx0 = fmaxf(fx0, ceilf(fsub(fsub(u, xa), 0.5f)));
                fx1 = fminf(fx1, floorf(fsub(fadd(u, xa), 0.5f)));
                fy0 = fmaxf(fy0, ceilf(fsub(fsub(v, ya), 0.5f)));
                fy1 = fminf(fy1, floorf(fsub(fadd(v, ya), 0.5f)));
                if (!(fx0 <= fx1) || !(fy0 <= fy1)) break;
            }
        }
        const int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
        const int tx0 = x0 >> rp.tile_w_log2, tx1 = x1 >> rp.tile_w_log2;
        const int ty0 = y0 >> rp.tile_h_log2, ty1 = y1 >> rp.tile_h_log2;
        P.ntouch = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        P.key = __float_as_uint(cz);
        P.tx0 = tx0; P.tx1 = tx1; P.ty0 = ty0; P.ty1 = ty1;

        // colour (free FP32 arithmetic)
        float dxv = m0 - cam.campos[0], dyv = m1 - cam.campos[1], dzv = m2 - cam.campos[2];
        float inv = 1.0f / sqrtf(dxv * dxv + dyv * dyv + dzv * dzv);
        float Y[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) Y[k] = 0.f;
        sh_basis(G.sh_degree, dxv * inv, dyv * inv, dzv * inv, Y);
        float rgb[3];
        if (PREC != GC_PREC_PLANES && G.K == 16) {  // degree 3: 16-byte loads, used as they arrive
            float acc[3] = {0.f, 0.f, 0.f};
            if constexpr (PREC == GC_PREC_FP32) {
                const float4 *p = reinterpret_cast<const float4 *>(G.sh + i * 48);
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    float4 x = p[q];
                    if (res.sh) {
                        const float4 d = reinterpret_cast<const float4 *>(res.sh + i * 48)[q];
                        x = make_float4(fadd(x.x, d.x), fadd(x.y, d.y), fadd(x.z, d.z), fadd(x.w, d.w));
                    }
                    const float v4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int idx = 4 * q + t;  // coefficient k = idx / 3, channel idx % 3
                        acc[idx % 3] = fmaf(Y[idx / 3], v4[t], acc[idx % 3]);
                    }
                }
            } else {
                const uint4 *p = reinterpret_cast<const uint4 *>(G.sh_q + i * 48);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const uint4 x = p[q];
                    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int b = 0; b < 16; ++b) {
                        const int idx = 16 * q + b;
                        float v = fmul(e4m3_to_f32((uint8_t)(w[b >> 2] >> (8 * (b & 3)))), G.scales[11 + idx]);
                        if (res.sh) v = fadd(v, res.sh[i * 48 + idx]);
                        acc[idx % 3] = fmaf(Y[idx / 3], v, acc[idx % 3]);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) rgb[c] = fmaxf(acc[c] + 0.5f, 0.f);
        } else if constexpr (PREC == GC_PREC_PLANES) {
            const PlaneLoc pl = plane_loc(G, i);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < G.K) acc = fmaf(Y[k], sh_plane<PREC>(G, pl, i, k, c, res), acc);
                rgb[c] = fmaxf(acc + 0.5f, 0.f);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (k < G.K) acc = fmaf(Y[k], load_sh<PREC>(G, i, k, c, res), acc);
                rgb[c] = fmaxf(acc + 0.5f, 0.f);
            }
        }
        const float op = 1.0f / (1.0f + expf(-A.logit));
        // conic stored pre-scaled for the blend's base-2 exponent (see gc_blend.cuh)
        P.r0 = make_float4(u, v, __fmul_rn(ia, -0.5f * kLog2e), __fmul_rn(ib, -kLog2e));
        P.r1 = make_float4(__fmul_rn(ic, -0.5f * kLog2e), op, rgb[0], rgb[1]);
        P.r2 = make_float4(rgb[2], cz, __int_as_float(x0 | (x1 << 16)), __int_as_float(y0 | (y1 << 16)));
        P.r3 = make_float4(ia, ib, ic, tc_out);
    } while (0);
}

// Per-Gaussian part of binning step 15: the ellipse Q <= tc (conic a, b, c from r3) and
// its extreme points.  Without the alpha cull, or for a degenerate conic, rows are the
// whole rectangle.
struct RowGeom {
    float u, v, ia, ib, ic, tc, detc, sy, ria, at;
    int x0, x1, y0, y1, tx0, tx1, ty0, ty1;
    bool cull;
};

__device__ __forceinline__ void row_geom(const float4 &r0, const float4 &r2, const float4 &r3,
                                         const RenderParams &rp, RowGeom &g) {
    const uint32_t rx = __float_as_uint(r2.z), ry = __float_as_uint(r2.w);
    g.x0 = (int)(rx & 0xffffu);
    g.x1 = (int)(rx >> 16);
    g.y0 = (int)(ry & 0xffffu);
    g.y1 = (int)(ry >> 16);
    g.tx0 = g.x0 >> rp.tile_w_log2;
    g.tx1 = g.x1 >> rp.tile_w_log2;
    g.ty0 = g.y0 >> rp.tile_h_log2;
    g.ty1 = g.y1 >> rp.tile_h_log2;
    g.u = r0.x;
    g.v = r0.y;
    g.ia = r3.x;
    g.ib = r3.y;
    g.ic = r3.z;
    g.tc = r3.w;
    g.detc = fsub(fmul(g.ia, g.ic), fmul(g.ib, g.ib));
    g.cull = rp.alpha_cull && g.detc > 0.f;
    g.sy = 0.f;
    g.ria = 0.f;
    g.at = 0.f;
    if (g.cull) {
        const float xa = __fsqrt_rn(fdiv(fmul(g.tc, g.ic), g.detc));
        g.sy = fdiv(fmul(g.ib, xa), g.ic);
        g.ria = fdiv(1.f, g.ia);
        g.at = fmul(g.ia, g.tc);
    }
}

// Binning step 15: tile columns [a, b] (a > b: empty) of tile row ty, i.e. the tiles whose
// pixel centres in the row's band of pixel-centre rows can meet the ellipse.  Over dy in
// [d0, d1] the ellipse spans dx in [(-b dy - sqrt(a tc - det dy^2)) / a, (-b dy + sqrt(.)) / a]
// (evaluated as products with ria = 1 / a); the right end is largest at dy = -sy, the left
// end smallest at dy = sy, each clamped into the band.  Every operation is a separately rounded IEEE binary32 operation (the oracle's
// FP32 mirror evaluates the same sequence).
__device__ __forceinline__ void row_interval(const RowGeom &g, int ty, const RenderParams &rp, int W, int H,
                                             int &a, int &b) {
    a = g.tx0;
    b = g.tx1;
    if (!g.cull) return;
    const int TW = rp.tile_w, TH = rp.tile_h;
    int r0, r1, c0, c1;
    if (rp.membership == GC_MEMBER_PIXEL) {
        r0 = max(ty * TH, g.y0);
        r1 = min(ty * TH + TH - 1, g.y1);
        c0 = g.x0;
        c1 = g.x1;
    } else {
        r0 = ty * TH;
        r1 = min(ty * TH + TH - 1, H - 1);
        c0 = g.tx0 * TW;
        c1 = min(g.tx1 * TW + TW - 1, W - 1);
    }
    const float d0 = fsub(fadd((float)r0, 0.5f), g.v), d1 = fsub(fadd((float)r1, 0.5f), g.v);
    const float dr = fminf(fmaxf(-g.sy, d0), d1), dl = fminf(fmaxf(g.sy, d0), d1);
    const float qr = fsub(g.at, fmul(fmul(g.detc, dr), dr)), ql = fsub(g.at, fmul(fmul(g.detc, dl), dl));
    const float xr = fmul(fsub(__fsqrt_rn(fmaxf(qr, 0.f)), fmul(g.ib, dr)), g.ria);
    const float xl = fmul(fsub(-fmul(g.ib, dl), __fsqrt_rn(fmaxf(ql, 0.f))), g.ria);
    float fx0 = ceilf(fsub(fadd(g.u, xl), 0.5f)), fx1 = floorf(fsub(fadd(g.u, xr), 0.5f));
    fx0 = fmaxf(fx0, (float)c0);
    fx1 = fminf(fx1, (float)c1);
    if (!(fx0 <= fx1)) {
        a = 1;
        b = 0;
        return;
    }
    a = (int)fx0 >> rp.tile_w_log2;
    b = (int)fx1 >> rp.tile_w_log2;
}

// Packed row intervals (r4): row i of a Gaussian with tile columns from tx0 has start
// tx0 + byte(2i) and length byte(2i + 1); byte 0 = 255 means "not packed".
__device__ __forceinline__ bool rows_packed(const float4 &r4) {
    return (__float_as_uint(r4.x) & 0xffu) != 0xffu;
}

__device__ __forceinline__ void packed_row(const float4 &r4, int i, int tx0, int &a, int &b) {
    const uint32_t w = __float_as_uint(i < 2 ? r4.x : i < 4 ? r4.y : i < 6 ? r4.z : r4.w);
    const uint32_t h = (w >> (16 * (i & 1))) & 0xffffu;
    a = tx0 + (int)(h & 0xffu);
    b = a + (int)(h >> 8) - 1;
}

// Row interval of row ty: from the packed bytes when present, else recomputed.
__device__ __forceinline__ void row_interval_rec(const RowGeom &g, const float4 &r4, int ty,
                                                 const RenderParams &rp, int W, int H, int &a, int &b) {
    if (rows_packed(r4)) packed_row(r4, ty - g.ty0, g.tx0, a, b);
    else row_interval(g, ty, rp, W, H, a, b);
}

// Emit of one warp: the 32 consecutive ranks wbase .. wbase + 31 (all of one image) write
// their (tile key, rank) entries, entry k of rank r at position offsets[r] + shift + k
// with k running over the Gaussian's tile rows in order and over the columns of each
// row's interval.  Gaussians with packed row intervals (nearly all): the lanes stride
// over the warp's contiguous output range, each finding its entry's Gaussian by a
// search over the lanes' offsets and its row by a scan of the packed lengths (coalesced
// writes).  The others: the warp walks their row index j = 0, 1, ... together; per step
// a warp scan of the lanes' interval lengths spreads the step's entries over the lanes.
// Positions >= cap are dropped.
__device__ __forceinline__ void emit_rows_warp(const float4 *__restrict__ ranked, int64_t wbase, int64_t n,
                                               const uint32_t *__restrict__ offsets,
                                               const uint32_t *__restrict__ touched_r, uint32_t shift,
                                               const RenderParams &rp, int W, int H, uint32_t cap,
                                               uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const int64_t r = wbase + lane;
    const bool in = r < n;
    const uint32_t cnt = in ? touched_r[r] : 0u;
    const uint32_t off = in ? offsets[r] + shift : 0xffffffffu;
    RowGeom g;
    float4 r4 = make_float4(__uint_as_float(0xffu), 0.f, 0.f, 0.f);
    bool packed = false;
    if (cnt) {
        r4 = ranked[kRec * r + 4];
        packed = rows_packed(r4);
        if (packed) {  // only the tile rectangle's origin is needed
            const float4 r2 = ranked[kRec * r + 2];
            g.tx0 = (int)(__float_as_uint(r2.z) & 0xffffu) >> rp.tile_w_log2;
            g.ty0 = (int)(__float_as_uint(r2.w) & 0xffffu) >> rp.tile_h_log2;
            g.ty1 = g.ty0;
        } else {
            row_geom(ranked[kRec * r], ranked[kRec * r + 2], ranked[kRec * r + 3], rp, g);
        }
    } else {
        g.tx0 = g.ty0 = 0;
        g.ty1 = -1;
    }
    // packed Gaussians: contiguous output range of the warp
    const uint32_t start = __shfl_sync(0xffffffffu, off, 0);
    const uint32_t end = __reduce_max_sync(0xffffffffu, in ? off + cnt : 0u);
    for (uint32_t e0 = start; e0 < end; e0 += 32) {
        const uint32_t e = e0 + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t o = __shfl_sync(0xffffffffu, off, owner + step);
            if (o <= e) owner += step;
        }
        const uint32_t oo = __shfl_sync(0xffffffffu, off, owner);
        const bool opk = __shfl_sync(0xffffffffu, (int)packed, owner) != 0;
        const int otx = __shfl_sync(0xffffffffu, g.tx0, owner);
        const int oty = __shfl_sync(0xffffffffu, g.ty0, owner);
        const uint32_t w0 = __shfl_sync(0xffffffffu, __float_as_uint(r4.x), owner);
        const uint32_t w1 = __shfl_sync(0xffffffffu, __float_as_uint(r4.y), owner);
        const uint32_t w2 = __shfl_sync(0xffffffffu, __float_as_uint(r4.z), owner);
        const uint32_t w3 = __shfl_sync(0xffffffffu, __float_as_uint(r4.w), owner);
        if (e < end && opk && e < cap) {
            uint32_t k = e - oo;
            int row = 0, a = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t w = i < 2 ? w0 : i < 4 ? w1 : i < 6 ? w2 : w3;
                const uint32_t h = (w >> (16 * (i & 1))) & 0xffffu, len = h >> 8;
                if (row == i) {
                    if (k < len) {
                        a = otx + (int)(h & 0xffu) + (int)k;
                        row = i + 100;  // found
                    } else {
                        k -= len;
                        row = i + 1;
                    }
                }
            }
            keys[e] = (uint32_t)(oty + row - 100) * (uint32_t)rp.ntx + (uint32_t)a;
            vals[e] = (uint32_t)(wbase + owner);
        }
    }
    // Gaussians whose rows are not packed: row by row
    const int nrows = (cnt && !packed) ? g.ty1 - g.ty0 + 1 : 0;
    const int steps = __reduce_max_sync(0xffffffffu, (uint32_t)nrows);
    uint32_t pos = off;
    for (int j = 0; j < steps; ++j) {
        int a = 0, b = -1, ty = 0;
        if (j < nrows) {
            ty = g.ty0 + j;
            row_interval(g, ty, rp, W, H, a, b);
        }
        const uint32_t c = b >= a ? (uint32_t)(b - a + 1) : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - c;
        for (uint32_t e0 = 0; e0 < total; e0 += 32) {
            const uint32_t e = e0 + lane;
            int owner = 0;  // first lane whose inclusive prefix exceeds e
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint32_t p = __shfl_sync(0xffffffffu, incl, owner + step - 1);
                if (p <= e) owner += step;
            }
            const uint32_t oex = __shfl_sync(0xffffffffu, excl, owner);
            const uint32_t opos = __shfl_sync(0xffffffffu, pos, owner);
            const int oa = __shfl_sync(0xffffffffu, a, owner);
            const int oty = __shfl_sync(0xffffffffu, ty, owner);
            if (e < total) {
                const uint32_t k = e - oex;
                const uint32_t at = opos + k;
                if (at < cap) {
                    keys[at] = (uint32_t)oty * (uint32_t)rp.ntx + (uint32_t)(oa + (int)k);
                    vals[at] = (uint32_t)(wbase + owner);
                }
            }
        }
        pos += c;
    }
}

// Position of tile (tx, ty) among a Gaussian's entries (its rows in order, the columns
// of each row's interval); the tile must be one of them.
__device__ __forceinline__ uint32_t entry_index(const RowGeom &g, const float4 &r4, int tx, int ty,
                                                const RenderParams &rp, int W, int H) {
    uint32_t k = 0u;
    for (int y = g.ty0; y < ty; ++y) {
        int a, b;
        row_interval_rec(g, r4, y, rp, W, H, a, b);
        if (b >= a) k += (uint32_t)(b - a + 1);
    }
    int a, b;
    row_interval_rec(g, r4, ty, rp, W, H, a, b);
    return k + (uint32_t)(tx - a);
}

// One warp sums the partials of one Gaussian's entries (positions base .. base + cnt - 1,
// nine floats each, contiguous) and sets every nonzero one back to zero, so that the
// partials buffer is all zeros again for the next reverse pass (entries the reverse
// blend does not reach are never written and must read as zero).  With the reverse pass's
// flags (one byte per entry, 1 where it stored a nonzero partial), only flagged entries are
// read, and their partials and flags are cleared; without (NULL), every entry is read.
// Entries past `cap`
// (an overflowed fixed capacity) are skipped.  Lanes stride over the entries; the warp
// sum is a transposing butterfly: afterwards lane 4 c holds value c (c < 8) and every
// lane holds value 8.
__device__ __forceinline__ void reduce_entries_warp(float *__restrict__ part, uint32_t base, uint32_t cnt,
                                                    uint32_t cap, uint8_t *__restrict__ flag, float &out0,
                                                    float &out8) {
    const int lane = threadIdx.x & 31;
    float v[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) v[c] = 0.f;
    if ((uint64_t)base + cnt <= cap) {
        for (uint32_t k = lane; k < cnt; k += 32) {
            // with flags, an entry whose partials were not stored holds zeros: adding them
            // changes no sum (no partial sum is -0), so it is skipped unread
            if (flag) {
                if (!flag[base + k]) continue;
                flag[base + k] = 0;
            }
            float *p = part + (int64_t)(base + k) * 9;
            float x[9];
            bool nz = false;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                x[c] = p[c];
                nz |= x[c] != 0.f;
                v[c] += x[c];
            }
            if (nz) {
#pragma unroll
                for (int c = 0; c < 9; ++c) p[c] = 0.f;
            }
        }
    }
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
    float x8 = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x8 += __shfl_xor_sync(0xffffffffu, x8, o);
    out8 = x8;
}

// Writes the nine sums of reduce_entries_warp to g[0..8].
__device__ __forceinline__ void store_reduced(float *g, float out0, float out8) {
    const int lane = threadIdx.x & 31;
    if ((lane & 3) == 0) g[lane >> 2] = out0;
    if (lane == 1) g[8] = out8;
}

// Tiles touched by a projected Gaussian (sum of its row intervals); packs the intervals
// into P.r4 when they fit.
__device__ __forceinline__ uint32_t bin_rows(Proj &P, const RenderParams &rp, int W, int H) {
    P.r4 = make_float4(__uint_as_float(0xffu), 0.f, 0.f, 0.f);
    if (!P.ntouch) return 0u;
    RowGeom g;
    row_geom(P.r0, P.r2, P.r3, rp, g);
    uint32_t total = 0u, pk0 = 0u, pk1 = 0u, pk2 = 0u, pk3 = 0u;
    bool fits = g.ty1 - g.ty0 < 8;
    for (int ty = g.ty0; ty <= g.ty1; ++ty) {
        int a, b;
        row_interval(g, ty, rp, W, H, a, b);
        const int i = ty - g.ty0, len = b >= a ? b - a + 1 : 0;
        const int off = b >= a ? a - g.tx0 : 0;
        if (off > 254 || len > 255) fits = false;
        if (fits) {
            const uint32_t h = ((uint32_t)off | ((uint32_t)len << 8)) << (16 * (i & 1));
            const int w = i >> 1;
            pk0 |= w == 0 ? h : 0u;
            pk1 |= w == 1 ? h : 0u;
            pk2 |= w == 2 ? h : 0u;
            pk3 |= w == 3 ? h : 0u;
        }
        if (a > b) continue;
        total += (uint32_t)len;
    }
    if (fits)
        P.r4 = make_float4(__uint_as_float(pk0), __uint_as_float(pk1), __uint_as_float(pk2), __uint_as_float(pk3));
    return total;
}

}  // namespace gc
