// gc_chain.cuh - chain rule of the preprocess (4DGCPro Sec. 3.1 / 3.2): from the 2D
// gradient of one projected Gaussian (du, dv, d conic a/b/c, d opacity, d rgb) to its
// mean, log-scales, quaternion, opacity logit and SH, and to its group's motion.
// Shared by the single-frame and the batched backward.
#pragma once
#include <cuda_fp8.h>
#include <cuda_runtime.h>

#include "gc_internal.cuh"
#include "gc_sh.cuh"

namespace gc {

__device__ __forceinline__ float bf16f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// SH coefficient k, channel c of global Gaussian i (dequantised for BF16/FP8 storage or
// from the decoded planes at `pl`), plus the frame's residual (Eq. 7).
template <int PREC>
__device__ __forceinline__ float sh_coeff(const GaussSrc &G, int64_t i, int k, int c, const Residual &res,
                                          const PlaneLoc &pl) {
    const int64_t idx = (i * G.K + k) * 3 + c;
    float f;
    if constexpr (PREC == GC_PREC_FP32) {
        f = G.sh[idx];
    } else if constexpr (PREC == GC_PREC_PLANES) {
        f = plane_value(G, pl, 11 + 3 * k + c);
    } else {
        __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)G.sh_q[idx], __NV_E4M3);
        f = __fmul_rn(__half2float(__half(hr)), G.scales[11 + 3 * k + c]);
    }
    return res.sh ? __fadd_rn(f, res.sh[idx]) : f;
}

// Gradient accumulators of one Gaussian (added to, never overwritten).
struct GradAcc {
    float dmu[3], dls[3], dq[4], dlogit, dsh[48];
};

// Adds the gradient of global Gaussian i, seen by camera `cam` under group motion
// (group_q == NULL: identity) and residual deformation `res`, given its 2D gradient d[9],
// to `acc`; writes the Gaussian's motion terms (d q_g[4], d t_g[3]) to motion7.  The
// Gaussian must be visible in that view.  The log-scale, logit and SH gradients are those
// of the deformed attributes (= those of the residuals).
template <int PREC>
__device__ __forceinline__ void chain_rule(const GaussSrc &G, int64_t i, const float *group_q,
                                           const float *group_t, int g, const CamParams &cam,
                                           const RenderParams &rp, const float *d, GradAcc &acc,
                                           float *motion7, const Residual &res, float *dsh_direct = nullptr) {
    const int K = G.K;
    float mu[3], ls[3], q[4], logit;
    PlaneLoc pl{0, 0, 0, 0};
    if constexpr (PREC == GC_PREC_PLANES) {
        pl = plane_loc(G, i);
        for (int k = 0; k < 3; ++k) { mu[k] = plane_value(G, pl, k); ls[k] = plane_value(G, pl, 7 + k); }
        for (int k = 0; k < 4; ++k) q[k] = plane_value(G, pl, 3 + k);
        logit = plane_value(G, pl, 10);
    } else if constexpr (PREC == GC_PREC_FP32) {
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
    if (res.ls)
        for (int k = 0; k < 3; ++k) ls[k] = __fadd_rn(ls[k], res.ls[3 * i + k]);
    if (res.logit) logit = __fadd_rn(logit, res.logit[i]);
    {
        float gq[4] = {1.f, 0.f, 0.f, 0.f}, gt[3] = {0.f, 0.f, 0.f};
        if (group_q) {
            for (int k = 0; k < 4; ++k) gq[k] = group_q[4 * g + k];
            for (int k = 0; k < 3; ++k) gt[k] = group_t[3 * g + k];
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
        acc.dlogit += d[5] * op * (1.f - op);
        // colour
        float dv[3] = {m[0] - cam.campos[0], m[1] - cam.campos[1], m[2] - cam.campos[2]};
        const float dn = sqrtf(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        const float dir[3] = {dv[0] / dn, dv[1] / dn, dv[2] / dn};
        float Y[16];
        sh_basis(G.sh_degree, dir[0], dir[1], dir[2], Y);
        // fully unrolled over the 16 coefficients (guarded by K) so that Y, wsh and the SH
        // gradient stay in registers; dsh_direct: the SH gradient is stored, not accumulated
        float raw[3] = {0.5f, 0.5f, 0.5f};
        float wsh[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (k < K) {
                raw[0] += Y[k] * sh_coeff<PREC>(G, i, k, 0, res, pl);
                raw[1] += Y[k] * sh_coeff<PREC>(G, i, k, 1, res, pl);
                raw[2] += Y[k] * sh_coeff<PREC>(G, i, k, 2, res, pl);
            }
        }
        const float draw[3] = {raw[0] > 0.f ? d[6] : 0.f, raw[1] > 0.f ? d[7] : 0.f, raw[2] > 0.f ? d[8] : 0.f};
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            wsh[k] = 0.f;
            if (k < K) {
                wsh[k] = sh_coeff<PREC>(G, i, k, 0, res, pl) * draw[0] + sh_coeff<PREC>(G, i, k, 1, res, pl) * draw[1] +
                         sh_coeff<PREC>(G, i, k, 2, res, pl) * draw[2];
                if (dsh_direct) {
                    dsh_direct[3 * k] = Y[k] * draw[0];
                    dsh_direct[3 * k + 1] = Y[k] * draw[1];
                    dsh_direct[3 * k + 2] = Y[k] * draw[2];
                } else {
                    acc.dsh[3 * k] += Y[k] * draw[0];
                    acc.dsh[3 * k + 1] += Y[k] * draw[1];
                    acc.dsh[3 * k + 2] += Y[k] * draw[2];
                }
            }
        }
        float ddx, ddy, ddz;
        sh_basis_vjp(G.sh_degree, dir[0], dir[1], dir[2], wsh, ddx, ddy, ddz);
        const float dd = dir[0] * ddx + dir[1] * ddy + dir[2] * ddz;
        float dmu[3];
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
            acc.dls[c] += ds * s[c];
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
        acc.dq[0] += a0 * dp[0] + a1 * dp[1] + a2 * dp[2] + a3 * dp[3];
        acc.dq[1] += -a1 * dp[0] + a0 * dp[1] + a3 * dp[2] - a2 * dp[3];
        acc.dq[2] += -a2 * dp[0] - a3 * dp[1] + a0 * dp[2] + a1 * dp[3];
        acc.dq[3] += -a3 * dp[0] + a2 * dp[1] - a1 * dp[2] + a0 * dp[3];
        motion7[0] = b0 * dp[0] + b1 * dp[1] + b2 * dp[2] + b3 * dp[3];
        motion7[1] = -b1 * dp[0] + b0 * dp[1] - b3 * dp[2] + b2 * dp[3];
        motion7[2] = -b2 * dp[0] + b3 * dp[1] + b0 * dp[2] - b1 * dp[3];
        motion7[3] = -b3 * dp[0] - b2 * dp[1] + b1 * dp[2] + b0 * dp[3];
        for (int a = 0; a < 3; ++a) {
            acc.dmu[a] += dmu[a];
            motion7[4 + a] = dmu[a];
        }
    }
}

}  // namespace gc
