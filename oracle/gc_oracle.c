/*
 * gc_oracle.c - plain, slow, FP64 CPU oracle of the hierarchical 4D Gaussian
 * tile rasterizer.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the CPU-baseline leg of the benchmark call it; the product path never does.
 * It shares no code, header or constant with the CUDA library.
 *
 * What it computes (paper: 4DGCPro, Sec. 3.1 and 3.2):
 *   - per-group rigid motion of the keyframe Gaussians, mu_t = mu + t_g and
 *     R_t = R_g R (Sec. 3.2, "Rigid Transformation"), broadcast per group;
 *   - the 3D Gaussian of Eq. 1 with covariance Sigma = R s s^T R^T (Sec. 3.1);
 *   - EWA projection of Sigma to a 2D conic (3DGS lineage the paper builds on,
 *     Sec. A), a 3-sigma radius and a pixel-square footprint;
 *   - colour from real spherical harmonics in the viewing direction (Sec. 3.1);
 *   - front-to-back alpha compositing over the depth-ordered Gaussians of the
 *     selected layers (Eq. 2 and the progressive form Eq. 4), with
 *     alpha = min(0.99, o exp(power)), skip when alpha < 1/255, stop (without
 *     blending) when the transmittance would drop below 1e-4;
 *   - the reverse-mode gradient of a linear functional of the image.
 *
 * Everything continuous is FP64.  The integer decisions that an FP32 renderer
 * takes - visibility, the depth order and the pixel footprint (radius and
 * rectangle) - are taken by the FP32 "binning mirror" below, in the op order
 * of the written binning specification, and the FP64 renderer consumes them,
 * so both sides decide in the same precision.
 *
 * The brute-force renderer visits, for every pixel, every selected visible
 * Gaussian whose footprint holds the pixel, in (depth, index) order; the only
 * acceleration is an exact per-row bucket of Gaussians by footprint rows.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define API __attribute__((visibility("default")))

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];       /* world -> camera rotation, row major */
    float t[3];       /* world -> camera translation */
    float campos[3];  /* camera centre in world coordinates */
} gco_camera;

typedef struct {
    float near_plane;     /* cull z <= near */
    float dilation;       /* added to the 2D covariance diagonal */
    float frustum_clamp;  /* x/z, y/z clamped to +-clamp * tan(half fov) inside J */
    float bg[3];
    int32_t tile_w, tile_h;
    int32_t membership;   /* 0: pixel square of half-width r; 1: every pixel of a touched tile */
    int32_t alpha_cull;   /* 1: footprint also clipped to the alpha >= 1/255 bounding box */
} gco_options;

typedef struct {
    int64_t n;
    int32_t sh_degree;
    const float *means;          /* n x 3 */
    const float *log_scales;     /* n x 3 */
    const float *quats;          /* n x 4, (w, x, y, z) */
    const float *opacity_logits; /* n */
    const float *sh;             /* n x K x 3, K = (d+1)^2 */
    const int32_t *group_id;     /* n, or NULL: every Gaussian in group 0 */
} gco_scene;

typedef struct {
    int32_t n_groups;
    const float *q;  /* G x 4 unit (w, x, y, z), or NULL: identity motion */
    const float *t;  /* G x 3 */
    /* Residual deformation of this frame (Sec. 3.2, Eq. 7: s_t = s_{t-1} + ds_t,
       alpha_t = alpha_{t-1} + dalpha_t, f_t = f_{t-1} + df_t), cumulative from the
       keyframe and indexed by global Gaussian; each may be NULL (no residual).  Read as
       additive in log-scale, opacity-logit and SH-coefficient space. */
    const float *res_ls;     /* n x 3 */
    const float *res_logit;  /* n */
    const float *res_sh;     /* n x K x 3 */
} gco_motion;

/* Deformed log-scale k, opacity logit and SH coefficient e (= 3 k + channel) of global
   Gaussian i: exact FP64 sums for the FP64 renderer ... */
static double ls_d(const gco_scene *sc, const gco_motion *mo, int64_t i, int k) {
    double v = sc->log_scales[3 * i + k];
    if (mo && mo->res_ls) v += (double)mo->res_ls[3 * i + k];
    return v;
}
static double logit_d(const gco_scene *sc, const gco_motion *mo, int64_t i) {
    double v = sc->opacity_logits[i];
    if (mo && mo->res_logit) v += (double)mo->res_logit[i];
    return v;
}
static double sh_d(const gco_scene *sc, const gco_motion *mo, int64_t i, int K, int e) {
    double v = sc->sh[i * K * 3 + e];
    if (mo && mo->res_sh) v += (double)mo->res_sh[i * K * 3 + e];
    return v;
}
/* ... and single FP32 additions for the binning mirror (binning specification). */
static float ls_f(const gco_scene *sc, const gco_motion *mo, int64_t i, int k) {
    float v = sc->log_scales[3 * i + k];
    if (mo && mo->res_ls) v = v + mo->res_ls[3 * i + k];
    return v;
}
static float logit_f(const gco_scene *sc, const gco_motion *mo, int64_t i) {
    float v = sc->opacity_logits[i];
    if (mo && mo->res_logit) v = v + mo->res_logit[i];
    return v;
}

/* ------------------------------------------------------------------------ */
/* Quaternions and rotations (FP64)                                          */
/* ------------------------------------------------------------------------ */

/* Hamilton product a (x) b, quaternions as (w, x, y, z). */
static void qmul_d(const double a[4], const double b[4], double o[4]) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/* Rotation matrix (row major) of a unit quaternion (w, x, y, z). */
static void quat_to_rot_d(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

/* dL/dq (unit q) given dL/dR, differentiating each entry of quat_to_rot_d. */
static void quat_to_rot_vjp_d(const double q[4], const double gR[9], double gq[4]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    gq[0] = 2 * (-z * gR[1] + y * gR[2] + z * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
    gq[1] = 2 * (y * gR[1] + z * gR[2] + y * gR[3] - w * gR[5] + z * gR[6] + w * gR[7])
          - 4 * x * (gR[4] + gR[8]);
    gq[2] = 2 * (x * gR[1] + w * gR[2] + x * gR[3] + z * gR[5] - w * gR[6] + z * gR[7])
          - 4 * y * (gR[0] + gR[8]);
    gq[3] = 2 * (-w * gR[1] + x * gR[2] + w * gR[3] + y * gR[5] + x * gR[6] + y * gR[7])
          - 4 * z * (gR[0] + gR[4]);
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics from their definition (FP64)                     */
/*                                                                           */
/* Y_l^m with the Condon-Shortley phase, index k = l^2 + l + m:              */
/*   Y_l^0  = K_l^0 P_l(z)                                                   */
/*   Y_l^m  = sqrt2 K_l^m (-1)^m P_l^(m)(z) Re((x + i y)^m),  m > 0          */
/*   Y_l^-m = sqrt2 K_l^m (-1)^m P_l^(m)(z) Im((x + i y)^m),  m > 0          */
/* with K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^(m) the m-th          */
/* derivative of the Legendre polynomial (Rodrigues' formula), and           */
/* (1-z^2)^(m/2) e^(i m phi) = (x + i y)^m on the unit sphere.  Written as a */
/* polynomial in (x, y, z), so its gradient is exact everywhere.             */
/* ------------------------------------------------------------------------ */

#define SH_MAX_DEG 3
static double g_leg[SH_MAX_DEG + 1][SH_MAX_DEG + 1];    /* g_leg[l][p]: coeff of z^p in P_l */
static double g_norm[SH_MAX_DEG + 1][SH_MAX_DEG + 1];   /* sqrt2 K_l^m (-1)^m, or K_l^0 */
static int g_sh_ready = 0;

static double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

static void sh_init(void) {
    if (g_sh_ready) return;
    for (int l = 0; l <= SH_MAX_DEG; ++l) {
        /* (z^2 - 1)^l = sum_j C(l,j) z^(2j) (-1)^(l-j); differentiate l times; / (2^l l!) */
        double c[2 * SH_MAX_DEG + 1];
        memset(c, 0, sizeof c);
        for (int j = 0; j <= l; ++j) c[2 * j] = binom(l, j) * (((l - j) & 1) ? -1.0 : 1.0);
        for (int d = 0; d < l; ++d) {
            for (int p = 0; p < 2 * SH_MAX_DEG; ++p) c[p] = (p + 1) * c[p + 1];
            c[2 * SH_MAX_DEG] = 0.0;
        }
        for (int p = 0; p <= SH_MAX_DEG; ++p)
            g_leg[l][p] = (p <= l) ? c[p] / (pow(2.0, l) * fact(l)) : 0.0;
        for (int m = 0; m <= l; ++m) {
            double K = sqrt((2 * l + 1) / (4 * M_PI) * fact(l - m) / fact(l + m));
            g_norm[l][m] = (m == 0) ? K : sqrt(2.0) * K * ((m & 1) ? -1.0 : 1.0);
        }
    }
    g_sh_ready = 1;
}

/* value and derivative of the m-th derivative of P_l at z */
static void legendre_dm(int l, int m, double z, double *val, double *dval) {
    double c[SH_MAX_DEG + 1];
    for (int p = 0; p <= SH_MAX_DEG; ++p) c[p] = g_leg[l][p];
    for (int d = 0; d < m; ++d) {
        for (int p = 0; p < SH_MAX_DEG; ++p) c[p] = (p + 1) * c[p + 1];
        c[SH_MAX_DEG] = 0.0;
    }
    double v = 0, dv = 0, zp = 1;
    for (int p = 0; p <= SH_MAX_DEG; ++p) { v += c[p] * zp; zp *= z; }
    zp = 1;
    for (int p = 1; p <= SH_MAX_DEG; ++p) { dv += p * c[p] * zp; zp *= z; }
    *val = v; *dval = dv;
}

/* Y[k] for k < (deg+1)^2 and, if dY != NULL, dY[3k..3k+2] = grad wrt (x,y,z). */
static void sh_eval_d(int deg, const double dir[3], double *Y, double *dY) {
    sh_init();
    double x = dir[0], y = dir[1], z = dir[2];
    /* (x + i y)^m and its partials: d/dx = m (x+iy)^(m-1), d/dy = i m (x+iy)^(m-1) */
    double re[SH_MAX_DEG + 1], im[SH_MAX_DEG + 1];
    re[0] = 1; im[0] = 0;
    for (int m = 1; m <= SH_MAX_DEG; ++m) {
        re[m] = re[m - 1] * x - im[m - 1] * y;
        im[m] = re[m - 1] * y + im[m - 1] * x;
    }
    for (int l = 0; l <= deg; ++l) {
        for (int m = 0; m <= l; ++m) {
            double P, dP;
            legendre_dm(l, m, z, &P, &dP);
            double N = g_norm[l][m];
            if (m == 0) {
                int k = l * l + l;
                Y[k] = N * P;
                if (dY) { dY[3 * k] = 0; dY[3 * k + 1] = 0; dY[3 * k + 2] = N * dP; }
            } else {
                int kp = l * l + l + m, kn = l * l + l - m;
                Y[kp] = N * P * re[m];
                Y[kn] = N * P * im[m];
                if (dY) {
                    /* d re_m/dx = m re_{m-1}, d re_m/dy = -m im_{m-1}
                       d im_m/dx = m im_{m-1}, d im_m/dy =  m re_{m-1} */
                    dY[3 * kp] = N * P * m * re[m - 1];
                    dY[3 * kp + 1] = -N * P * m * im[m - 1];
                    dY[3 * kp + 2] = N * dP * re[m];
                    dY[3 * kn] = N * P * m * im[m - 1];
                    dY[3 * kn + 1] = N * P * m * re[m - 1];
                    dY[3 * kn + 2] = N * dP * im[m];
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* FP32 binning mirror: the written binning specification, op by op.         */
/* Every line is one IEEE single operation; compiled with -ffp-contract=off  */
/* so no multiply-add is fused.  s = (float)exp((double)log_s).              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t visible;
    float depth;
    int32_t rect[4];   /* px0, px1, py0, py1 (inclusive) */
    int32_t trect[4];  /* tx0, tx1, ty0, ty1 (inclusive) */
    int32_t radius;
    float u, v, conic[3];
    float tc;          /* alpha-ellipse level of step 14 (0 without the alpha cull) */
} gco_bin;

static void bin_one_f32(const gco_scene *sc, const gco_motion *mo, const gco_camera *cam,
                        const gco_options *op, int64_t i, gco_bin *out) {
    memset(out, 0, sizeof *out);
    const float *mu = sc->means + 3 * i, *qq = sc->quats + 4 * i;
    int g = sc->group_id ? sc->group_id[i] : 0;
    float gq[4] = {1.0f, 0.0f, 0.0f, 0.0f}, gt[3] = {0.0f, 0.0f, 0.0f};
    if (mo && mo->q) {
        for (int k = 0; k < 4; ++k) gq[k] = mo->q[4 * g + k];
        for (int k = 0; k < 3; ++k) gt[k] = mo->t[3 * g + k];
    }
    /* 1. moved mean */
    float m0 = mu[0] + gt[0], m1 = mu[1] + gt[1], m2 = mu[2] + gt[2];
    /* 2. p = gq (x) q */
    float a0 = gq[0], a1 = gq[1], a2 = gq[2], a3 = gq[3];
    float b0 = qq[0], b1 = qq[1], b2 = qq[2], b3 = qq[3];
    float p0 = a0 * b0; p0 = p0 - a1 * b1; p0 = p0 - a2 * b2; p0 = p0 - a3 * b3;
    float p1 = a0 * b1; p1 = p1 + a1 * b0; p1 = p1 + a2 * b3; p1 = p1 - a3 * b2;
    float p2 = a0 * b2; p2 = p2 - a1 * b3; p2 = p2 + a2 * b0; p2 = p2 + a3 * b1;
    float p3 = a0 * b3; p3 = p3 + a1 * b2; p3 = p3 - a2 * b1; p3 = p3 + a3 * b0;
    /* 3. normalise */
    float n2 = p0 * p0; n2 = n2 + p1 * p1; n2 = n2 + p2 * p2; n2 = n2 + p3 * p3;
    if (!(n2 > 0.0f)) return;
    float nn = sqrtf(n2);
    float w = p0 / nn, x = p1 / nn, y = p2 / nn, z = p3 / nn;
    /* 4. rotation */
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float wx = w * x, wy = w * y, wz = w * z;
    float R[9];
    R[0] = 1.0f - 2.0f * (yy + zz); R[1] = 2.0f * (xy - wz); R[2] = 2.0f * (xz + wy);
    R[3] = 2.0f * (xy + wz); R[4] = 1.0f - 2.0f * (xx + zz); R[5] = 2.0f * (yz - wx);
    R[6] = 2.0f * (xz - wy); R[7] = 2.0f * (yz + wx); R[8] = 1.0f - 2.0f * (xx + yy);
    /* 5. scales */
    float s[3];
    for (int k = 0; k < 3; ++k) s[k] = (float)exp((double)ls_f(sc, mo, i, k));
    /* 6. M = R diag(s) */
    float M[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * s[c];
    /* 7. Sigma = M M^T */
    float S[9];
    for (int r = 0; r < 3; ++r)
        for (int c = r; c < 3; ++c) {
            float acc = M[3 * r] * M[3 * c];
            acc = acc + M[3 * r + 1] * M[3 * c + 1];
            acc = acc + M[3 * r + 2] * M[3 * c + 2];
            S[3 * r + c] = acc; S[3 * c + r] = acc;
        }
    /* 8. camera point */
    const float *W = cam->R;
    float cpt[3];
    for (int r = 0; r < 3; ++r) {
        float acc = W[3 * r] * m0;
        acc = acc + W[3 * r + 1] * m1;
        acc = acc + W[3 * r + 2] * m2;
        cpt[r] = acc + cam->t[r];
    }
    float cz = cpt[2];
    if (!(cz > op->near_plane)) return;
    /* 9. Jacobian with the frustum clamp, T = J W, Sigma2 = T Sigma T^T */
    float xoz = cpt[0] / cz, yoz = cpt[1] / cz;
    float limx = op->frustum_clamp * ((0.5f * (float)cam->width) / cam->fx);
    float limy = op->frustum_clamp * ((0.5f * (float)cam->height) / cam->fy);
    float xt = fminf(limx, fmaxf(-limx, xoz));
    float yt = fminf(limy, fmaxf(-limy, yoz));
    float J00 = cam->fx / cz, J11 = cam->fy / cz;
    float J02 = -((cam->fx * xt) / cz), J12 = -((cam->fy * yt) / cz);
    float T[6];
    for (int c = 0; c < 3; ++c) {
        T[c] = J00 * W[c] + J02 * W[6 + c];
        T[3 + c] = J11 * W[3 + c] + J12 * W[6 + c];
    }
    float U[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            float acc = T[3 * r] * S[c];
            acc = acc + T[3 * r + 1] * S[3 + c];
            acc = acc + T[3 * r + 2] * S[6 + c];
            U[3 * r + c] = acc;
        }
    float ca = U[0] * T[0]; ca = ca + U[1] * T[1]; ca = ca + U[2] * T[2]; ca = ca + op->dilation;
    float cb = U[0] * T[3]; cb = cb + U[1] * T[4]; cb = cb + U[2] * T[5];
    float cc = U[3] * T[3]; cc = cc + U[4] * T[4]; cc = cc + U[5] * T[5]; cc = cc + op->dilation;
    /* 10. conic */
    float det = ca * cc - cb * cb;
    if (!(det > 0.0f)) return;
    float ia = cc / det, ib = -(cb / det), ic = ca / det;
    /* 11. radius */
    float mid = 0.5f * (ca + cc);
    float disc = mid * mid - det;
    float lam = mid + sqrtf(fmaxf(0.0f, disc));
    float rf = ceilf(3.0f * sqrtf(lam));
    /* 12. centre */
    float u = cam->fx * xoz + cam->cx;
    float v = cam->fy * yoz + cam->cy;
    if (!isfinite(u) || !isfinite(v) || !isfinite(rf)) return;
    /* 13. pixel rectangle, clipped */
    float fx0 = ceilf((u - rf) - 0.5f), fx1 = floorf((u + rf) - 0.5f);
    float fy0 = ceilf((v - rf) - 0.5f), fy1 = floorf((v + rf) - 0.5f);
    fx0 = fmaxf(fx0, 0.0f); fy0 = fmaxf(fy0, 0.0f);
    fx1 = fminf(fx1, (float)(cam->width - 1)); fy1 = fminf(fy1, (float)(cam->height - 1));
    if (!(fx0 <= fx1) || !(fy0 <= fy1)) return;   /* also rejects NaN */
    /* 14. alpha footprint (binning spec, not in the paper): alpha = o exp(-Q/2) reaches
       1/255 only where Q <= tau = 2 ln(255 o).  The ellipse Q <= tau_c, tau_c = tau +
       0.02 + 1e-6 (ia + 2|ib| + ic)(r + 1)^2 (the second term bounds the rounding of an
       FP32 evaluation of Q over the 3-sigma square), has the half-extents
       sqrt(tau_c ic / det_c) and sqrt(tau_c ia / det_c); the rectangle is clipped to
       them.  Opacity <= 1/255: the Gaussian is never blended and is not binned. */
    if (op->alpha_cull) {
        float tau = (float)(2.0 * log(255.0 / (1.0 + exp(-(double)logit_f(sc, mo, i)))));
        if (!(tau > 0.0f)) return;
        float t1 = rf + 1.0f;
        float mt = ((ia + 2.0f * fabsf(ib)) + ic) * (t1 * t1);
        float tc = (tau + 0.02f) + 1e-6f * mt;
        out->tc = tc;
        float detc = ia * ic - ib * ib;
        if (detc > 0.0f) {
            float xa = sqrtf((tc * ic) / detc), ya = sqrtf((tc * ia) / detc);
            fx0 = fmaxf(fx0, ceilf((u - xa) - 0.5f)); fx1 = fminf(fx1, floorf((u + xa) - 0.5f));
            fy0 = fmaxf(fy0, ceilf((v - ya) - 0.5f)); fy1 = fminf(fy1, floorf((v + ya) - 0.5f));
            if (!(fx0 <= fx1) || !(fy0 <= fy1)) return;
        }
    }
    out->visible = 1;
    out->depth = cz;
    out->rect[0] = (int32_t)fx0; out->rect[1] = (int32_t)fx1;
    out->rect[2] = (int32_t)fy0; out->rect[3] = (int32_t)fy1;
    out->trect[0] = out->rect[0] / op->tile_w; out->trect[1] = out->rect[1] / op->tile_w;
    out->trect[2] = out->rect[2] / op->tile_h; out->trect[3] = out->rect[3] / op->tile_h;
    out->radius = (int32_t)rf;
    out->u = u; out->v = v;
    out->conic[0] = ia; out->conic[1] = ib; out->conic[2] = ic;
}

/* 15. row intervals (binning spec, not in the paper).  With the alpha cull, a tile row
   keeps only the tile columns whose pixel centres can meet the ellipse Q <= tc within
   the row's band of pixel-centre rows: over dy in [d0, d1] the ellipse spans
   dx in [(-ib dy - sqrt(ia tc - det dy^2)) / ia, (-ib dy + sqrt(...)) / ia] (evaluated as
   a product with ria = 1 / ia); its right end is largest at dy = -s and its left end
   smallest at dy = s, s = ib xa / ic (the extreme points), each clamped into the band.  Without the cull, or for a degenerate
   conic, a row is the rectangle's [tx0, tx1].  Writes [*a, *b] (*a > *b: empty). */
static void row_interval_f32(const gco_bin *b, int ty, const gco_options *op, const gco_camera *cam,
                             int32_t *a, int32_t *bb) {
    const int TW = op->tile_w, TH = op->tile_h;
    *a = b->trect[0]; *bb = b->trect[1];
    if (!op->alpha_cull) return;
    const float ia = b->conic[0], ib = b->conic[1], ic = b->conic[2], tc = b->tc, u = b->u, v = b->v;
    const float detc = ia * ic - ib * ib;
    if (!(detc > 0.0f)) return;
    const float xa = sqrtf((tc * ic) / detc);
    const float sy = (ib * xa) / ic;
    const float ria = 1.0f / ia;
    int r0, r1, c0, c1;
    if (op->membership == 0) {
        r0 = ty * TH > b->rect[2] ? ty * TH : b->rect[2];
        r1 = ty * TH + TH - 1 < b->rect[3] ? ty * TH + TH - 1 : b->rect[3];
        c0 = b->rect[0]; c1 = b->rect[1];
    } else {
        r0 = ty * TH;
        r1 = ty * TH + TH - 1 < cam->height - 1 ? ty * TH + TH - 1 : cam->height - 1;
        c0 = b->trect[0] * TW;
        c1 = b->trect[1] * TW + TW - 1 < cam->width - 1 ? b->trect[1] * TW + TW - 1 : cam->width - 1;
    }
    const float d0 = ((float)r0 + 0.5f) - v, d1 = ((float)r1 + 0.5f) - v;
    const float dr = fminf(fmaxf(-sy, d0), d1), dl = fminf(fmaxf(sy, d0), d1);
    const float qr = ia * tc - (detc * dr) * dr, ql = ia * tc - (detc * dl) * dl;
    const float xr = (sqrtf(fmaxf(qr, 0.0f)) - ib * dr) * ria;
    const float xl = (-(ib * dl) - sqrtf(fmaxf(ql, 0.0f))) * ria;
    float fx0 = ceilf((u + xl) - 0.5f), fx1 = floorf((u + xr) - 0.5f);
    fx0 = fmaxf(fx0, (float)c0); fx1 = fminf(fx1, (float)c1);
    if (!(fx0 <= fx1)) { *a = 1; *bb = 0; return; }
    *a = (int32_t)fx0 / TW; *bb = (int32_t)fx1 / TW;
}

/* Binning mirror over the selected Gaussians sel[0..n_sel). */
API void gco_bin_f32(const gco_scene *sc, const gco_motion *mo, const gco_camera *cam,
                     const gco_options *op, const int64_t *sel, int64_t n_sel,
                     int32_t *visible, float *depth, int32_t *rect, int32_t *trect,
                     int32_t *radius, float *uv, float *conic, float *tc) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_sel; ++j) {
        gco_bin b;
        bin_one_f32(sc, mo, cam, op, sel[j], &b);
        visible[j] = b.visible;
        depth[j] = b.depth;
        for (int k = 0; k < 4; ++k) { rect[4 * j + k] = b.rect[k]; trect[4 * j + k] = b.trect[k]; }
        radius[j] = b.radius;
        uv[2 * j] = b.u; uv[2 * j + 1] = b.v;
        for (int k = 0; k < 3; ++k) conic[3 * j + k] = b.conic[k];
        tc[j] = b.tc;
    }
}

/* Row intervals of binned Gaussians: for visible j, its tile rows trect[2..3] are
   entries row_off[j] .. row_off[j+1]-1 of a / b (step 15). */
API void gco_bin_rows(const gco_camera *cam, const gco_options *op, int64_t n_sel,
                      const int32_t *visible, const int32_t *rect, const int32_t *trect,
                      const float *uv, const float *conic, const float *tc, const int64_t *row_off,
                      int32_t *a, int32_t *b) {
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_sel; ++j) {
        if (!visible[j]) continue;
        gco_bin g;
        memset(&g, 0, sizeof g);
        g.visible = 1;
        for (int k = 0; k < 4; ++k) { g.rect[k] = rect[4 * j + k]; g.trect[k] = trect[4 * j + k]; }
        g.u = uv[2 * j]; g.v = uv[2 * j + 1];
        for (int k = 0; k < 3; ++k) g.conic[k] = conic[3 * j + k];
        g.tc = tc[j];
        for (int ty = g.trect[2]; ty <= g.trect[3]; ++ty)
            row_interval_f32(&g, ty, op, cam, &a[row_off[j] + ty - g.trect[2]], &b[row_off[j] + ty - g.trect[2]]);
    }
}

/* ------------------------------------------------------------------------ */
/* FP64 per-Gaussian geometry                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* forward values */
    double mup[3];      /* moved mean */
    double p[4];        /* gq (x) q, unnormalised */
    double qn[4];       /* normalised */
    double pn;          /* |p| */
    double R[9], s[3], M[9], Sig[9];
    double c[3];        /* camera point */
    double xoz, yoz, xt, yt;
    int clampx, clampy; /* 1 when the clamp is active */
    double J00, J02, J11, J12, T[6];
    double A, B, C;     /* Sigma2 entries incl. dilation */
    double det, conic[3];
    double u, v;
    double o;           /* opacity */
    double dir[3], dnorm;  /* view direction and |mu' - campos| */
    double raw[3], rgb[3];
    int K;
    double Y[16];
} gc_geom;

static void geom_d(const gco_scene *sc, const gco_motion *mo, const gco_camera *cam,
                   const gco_options *op, int64_t i, gc_geom *G) {
    const float *mu = sc->means + 3 * i, *qq = sc->quats + 4 * i;
    int g = sc->group_id ? sc->group_id[i] : 0;
    double gq[4] = {1, 0, 0, 0}, gt[3] = {0, 0, 0};
    if (mo && mo->q) {
        for (int k = 0; k < 4; ++k) gq[k] = mo->q[4 * g + k];
        for (int k = 0; k < 3; ++k) gt[k] = mo->t[3 * g + k];
    }
    double q[4] = {qq[0], qq[1], qq[2], qq[3]};
    for (int k = 0; k < 3; ++k) G->mup[k] = (double)mu[k] + gt[k];
    qmul_d(gq, q, G->p);
    G->pn = sqrt(G->p[0] * G->p[0] + G->p[1] * G->p[1] + G->p[2] * G->p[2] + G->p[3] * G->p[3]);
    for (int k = 0; k < 4; ++k) G->qn[k] = G->p[k] / G->pn;
    quat_to_rot_d(G->qn, G->R);
    for (int k = 0; k < 3; ++k) G->s[k] = exp(ls_d(sc, mo, i, k));
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) G->M[3 * r + c] = G->R[3 * r + c] * G->s[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            G->Sig[3 * r + c] = G->M[3 * r] * G->M[3 * c] + G->M[3 * r + 1] * G->M[3 * c + 1]
                              + G->M[3 * r + 2] * G->M[3 * c + 2];
    double W[9];
    for (int k = 0; k < 9; ++k) W[k] = cam->R[k];
    for (int r = 0; r < 3; ++r)
        G->c[r] = W[3 * r] * G->mup[0] + W[3 * r + 1] * G->mup[1] + W[3 * r + 2] * G->mup[2]
                + (double)cam->t[r];
    double z = G->c[2];
    double fx = cam->fx, fy = cam->fy;
    G->xoz = G->c[0] / z; G->yoz = G->c[1] / z;
    double limx = (double)op->frustum_clamp * (0.5 * cam->width / fx);
    double limy = (double)op->frustum_clamp * (0.5 * cam->height / fy);
    G->clampx = (G->xoz > limx) || (G->xoz < -limx);
    G->clampy = (G->yoz > limy) || (G->yoz < -limy);
    G->xt = G->xoz > limx ? limx : (G->xoz < -limx ? -limx : G->xoz);
    G->yt = G->yoz > limy ? limy : (G->yoz < -limy ? -limy : G->yoz);
    G->J00 = fx / z; G->J11 = fy / z;
    G->J02 = -fx * G->xt / z; G->J12 = -fy * G->yt / z;
    for (int c = 0; c < 3; ++c) {
        G->T[c] = G->J00 * W[c] + G->J02 * W[6 + c];
        G->T[3 + c] = G->J11 * W[3 + c] + G->J12 * W[6 + c];
    }
    double S2[4] = {0, 0, 0, 0};
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += G->T[3 * r + a] * G->Sig[3 * a + b] * G->T[3 * c + b];
            S2[2 * r + c] = acc;
        }
    G->A = S2[0] + op->dilation; G->B = S2[1]; G->C = S2[3] + op->dilation;
    G->det = G->A * G->C - G->B * G->B;
    G->conic[0] = G->C / G->det; G->conic[1] = -G->B / G->det; G->conic[2] = G->A / G->det;
    G->u = fx * G->xoz + cam->cx;
    G->v = fy * G->yoz + cam->cy;
    G->o = 1.0 / (1.0 + exp(-logit_d(sc, mo, i)));
    double dv[3];
    for (int k = 0; k < 3; ++k) dv[k] = G->mup[k] - (double)cam->campos[k];
    G->dnorm = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int k = 0; k < 3; ++k) G->dir[k] = dv[k] / G->dnorm;
    G->K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    sh_eval_d(sc->sh_degree, G->dir, G->Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0;
        for (int k = 0; k < G->K; ++k) acc += G->Y[k] * sh_d(sc, mo, i, G->K, 3 * k + ch);
        G->raw[ch] = acc + 0.5;
        G->rgb[ch] = G->raw[ch] > 0 ? G->raw[ch] : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Per-pixel compositing (Eq. 2 / Eq. 4), FP64                               */
/* ------------------------------------------------------------------------ */

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_STOP 1.0e-4
/* Margins within which an FP32 renderer may legitimately decide differently */
#define AMB_ALPHA_REL 1.0e-4
#define AMB_T_REL 1.0e-4
#define AMB_POWER_REL 1.0e-5

typedef struct {
    int64_t nvis;
    int64_t *order;      /* selected positions j of visible Gaussians, (depth, index) order */
    gc_geom *geo;        /* FP64 geometry per selected position j */
    const int32_t *rect; /* per selected position: px0, px1, py0, py1 */
    const int32_t *trect;
    int64_t *row_start;  /* CSR per image row over positions in `order` */
    int64_t *row_list;
} gc_prep;

typedef struct {
    double rgb[3], T;
    int32_t n_blended;
    int32_t ambiguous;
    double signature;    /* weighted sum of blended positions, used to detect decision changes */
} gc_pix;

static const int64_t *g_sort_sel;
static const float *g_sort_depth;
static int cmp_depth_index(const void *a, const void *b) {
    int64_t ja = *(const int64_t *)a, jb = *(const int64_t *)b;
    float da = g_sort_depth[ja], db = g_sort_depth[jb];
    if (da < db) return -1;
    if (da > db) return 1;
    int64_t ia = g_sort_sel[ja], ib = g_sort_sel[jb];
    return (ia < ib) ? -1 : (ia > ib);
}

static int member(const gc_prep *P, const gco_options *op, int64_t j, int px, int py) {
    if (op->membership == 0) {
        const int32_t *r = P->rect + 4 * j;
        return px >= r[0] && px <= r[1] && py >= r[2] && py <= r[3];
    }
    const int32_t *t = P->trect + 4 * j;
    int tx = px / op->tile_w, ty = py / op->tile_h;
    return tx >= t[0] && tx <= t[1] && ty >= t[2] && ty <= t[3];
}

static int prep_build(gc_prep *P, const gco_scene *sc, const gco_motion *mo, const gco_camera *cam,
                      const gco_options *op, const int64_t *sel, int64_t n_sel,
                      const int32_t *visible, const float *depth, const int32_t *rect,
                      const int32_t *trect, int direct) {
    memset(P, 0, sizeof *P);
    P->rect = rect; P->trect = trect;
    int64_t nv = 0;
    for (int64_t j = 0; j < n_sel; ++j) nv += visible[j] != 0;
    P->nvis = nv;
    P->order = (int64_t *)malloc(sizeof(int64_t) * (nv ? nv : 1));
    P->geo = (gc_geom *)malloc(sizeof(gc_geom) * (n_sel ? n_sel : 1));
    if (!P->order || !P->geo) return -1;
    nv = 0;
    for (int64_t j = 0; j < n_sel; ++j) if (visible[j]) P->order[nv++] = j;
    g_sort_sel = sel; g_sort_depth = depth;
    qsort(P->order, (size_t)nv, sizeof(int64_t), cmp_depth_index);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_sel; ++j)
        if (visible[j]) geom_d(sc, mo, cam, op, sel[j], &P->geo[j]);
    /* rows covered: pixel rows of the footprint (square mode) or of the tile rows.
       With direct != 0 no buckets are built: pixels scan the whole sorted list. */
    int H = cam->height;
    if (direct) { P->row_start = NULL; P->row_list = NULL; return 0; }
    P->row_start = (int64_t *)calloc((size_t)H + 1, sizeof(int64_t));
    if (!P->row_start) return -1;
    for (int64_t k = 0; k < nv; ++k) {
        int64_t j = P->order[k];
        int y0, y1;
        if (op->membership == 0) { y0 = rect[4 * j + 2]; y1 = rect[4 * j + 3]; }
        else { y0 = trect[4 * j + 2] * op->tile_h; y1 = (trect[4 * j + 3] + 1) * op->tile_h - 1; if (y1 > H - 1) y1 = H - 1; }
        for (int y = y0; y <= y1; ++y) P->row_start[y + 1]++;
    }
    for (int y = 0; y < H; ++y) P->row_start[y + 1] += P->row_start[y];
    P->row_list = (int64_t *)malloc(sizeof(int64_t) * (P->row_start[H] ? P->row_start[H] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (H ? H : 1));
    if (!P->row_list || !fill) { free(fill); return -1; }
    for (int y = 0; y < H; ++y) fill[y] = P->row_start[y];
    for (int64_t k = 0; k < nv; ++k) {
        int64_t j = P->order[k];
        int y0, y1;
        if (op->membership == 0) { y0 = rect[4 * j + 2]; y1 = rect[4 * j + 3]; }
        else { y0 = trect[4 * j + 2] * op->tile_h; y1 = (trect[4 * j + 3] + 1) * op->tile_h - 1; if (y1 > H - 1) y1 = H - 1; }
        for (int y = y0; y <= y1; ++y) P->row_list[fill[y]++] = j;
    }
    free(fill);
    return 0;
}

static void prep_free(gc_prep *P) {
    free(P->order); free(P->geo); free(P->row_start); free(P->row_list);
}

/* One blended step recorded for the reverse pass. */
typedef struct {
    int64_t j;
    double alpha, G, T, dx, dy;
    int clamped;
} gc_step;

/* Composite pixel (px, py); if `steps` != NULL record blended steps (cap n_cap). */
static void composite_pixel(const gc_prep *P, const gco_options *op, int px, int py,
                            gc_pix *out, gc_step *steps, int64_t n_cap, int64_t *n_steps) {
    double T = 1.0, C[3] = {0, 0, 0};
    int amb = 0;
    int32_t nb = 0;
    double sig = 0;
    double pcx = px + 0.5, pcy = py + 0.5;
    int64_t ns = 0;
    const int64_t kb = P->row_start ? P->row_start[py] : 0;
    const int64_t ke = P->row_start ? P->row_start[py + 1] : P->nvis;
    for (int64_t k = kb; k < ke; ++k) {
        int64_t j = P->row_start ? P->row_list[k] : P->order[k];
        if (!member(P, op, j, px, py)) continue;
        const gc_geom *G = &P->geo[j];
        double dx = pcx - G->u, dy = pcy - G->v;
        double ta = G->conic[0] * dx * dx, tc = G->conic[2] * dy * dy, tb = 2.0 * G->conic[1] * dx * dy;
        double power = -0.5 * (ta + tc) - 0.5 * tb;
        double pmag = 0.5 * (fabs(ta) + fabs(tc) + fabs(tb));
        if (fabs(power) <= AMB_POWER_REL * pmag + 1e-30) amb = 1;
        if (power > 0) continue;
        double gv = exp(power);
        double a0 = G->o * gv;
        int clamped = a0 > ALPHA_MAX;
        double alpha = clamped ? ALPHA_MAX : a0;
        if (fabs(alpha - ALPHA_MIN) <= AMB_ALPHA_REL * ALPHA_MIN) amb = 1;
        if (alpha < ALPHA_MIN) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - T_STOP) <= AMB_T_REL * T_STOP) amb = 1;
        if (Tn < T_STOP) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += G->rgb[ch] * alpha * T;
        if (steps && ns < n_cap) {
            steps[ns].j = j; steps[ns].alpha = alpha; steps[ns].G = gv; steps[ns].T = T;
            steps[ns].dx = dx; steps[ns].dy = dy; steps[ns].clamped = clamped;
        }
        ++ns;
        T = Tn;
        ++nb;
        sig += (double)(j + 1) * (1.0 + 1e-3 * nb);
    }
    for (int ch = 0; ch < 3; ++ch) out->rgb[ch] = C[ch] + T * op->bg[ch];
    out->T = T; out->n_blended = nb; out->ambiguous = amb; out->signature = sig;
    if (n_steps) *n_steps = ns;
}

/*
 * FP64 render.  Decisions from the binning mirror (visible, depth, rect,
 * trect per selected position).  If n_pix > 0, renders only the pixels
 * pix[2k] = x, pix[2k+1] = y into out_*[k]; otherwise the full frame in
 * planar layout (rgb: 3 x H x W, others H x W).
 */
API int gco_render_f64(const gco_scene *sc, const gco_motion *mo, const gco_camera *cam,
                       const gco_options *op, const int64_t *sel, int64_t n_sel,
                       const int32_t *visible, const float *depth, const int32_t *rect,
                       const int32_t *trect, const int32_t *pix, int64_t n_pix,
                       double *out_rgb, double *out_T, int32_t *out_nb, int32_t *out_amb,
                       double *out_sig) {
    gc_prep P;
    sh_init();
    /* sampled pixels over a large scene: scan the sorted list per pixel instead of
       building per-row buckets (same visiting order, same result) */
    int direct = n_pix > 0 && n_pix * 64 < (int64_t)cam->height * cam->width && n_sel > 200000;
    if (prep_build(&P, sc, mo, cam, op, sel, n_sel, visible, depth, rect, trect, direct)) { prep_free(&P); return -1; }
    int64_t W = cam->width, H = cam->height;
    int64_t total = n_pix > 0 ? n_pix : W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < total; ++k) {
        int px, py;
        if (n_pix > 0) { px = pix[2 * k]; py = pix[2 * k + 1]; }
        else { px = (int)(k % W); py = (int)(k / W); }
        gc_pix r;
        composite_pixel(&P, op, px, py, &r, NULL, 0, NULL);
        if (n_pix > 0) {
            for (int ch = 0; ch < 3; ++ch) out_rgb[3 * k + ch] = r.rgb[ch];
        } else {
            for (int ch = 0; ch < 3; ++ch) out_rgb[ch * W * H + k] = r.rgb[ch];
        }
        if (out_T) out_T[k] = r.T;
        if (out_nb) out_nb[k] = r.n_blended;
        if (out_amb) out_amb[k] = r.ambiguous;
        if (out_sig) out_sig[k] = r.signature;
    }
    prep_free(&P);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode, FP64                                                        */
/* ------------------------------------------------------------------------ */

/* Per-Gaussian gradient of a linear functional L = sum dLdimg * image, through
 * compositing (Eq. 2) and then the projection chain back to the attributes.
 * dLdimg: planar 3 x H x W.  Outputs are indexed by selected position j and
 * overwritten: d_means (3), d_log_scales (3), d_quats (4), d_logits (1),
 * d_sh (K x 3), and per group d_gq (4), d_gt (3).  Also returns the 2D
 * per-Gaussian gradient (du, dv, dconic_a, dconic_b, dconic_c, dopacity,
 * dr, dg, db) in d2d (9 per position) when non-NULL. */
API int gco_grad_f64(const gco_scene *sc, const gco_motion *mo, const gco_camera *cam,
                     const gco_options *op, const int64_t *sel, int64_t n_sel,
                     const int32_t *visible, const float *depth, const int32_t *rect,
                     const int32_t *trect, const double *dLdimg,
                     double *d_means, double *d_log_scales, double *d_quats, double *d_logits,
                     double *d_sh, double *d_gq, double *d_gt, double *d2d) {
    gc_prep P;
    sh_init();
    if (prep_build(&P, sc, mo, cam, op, sel, n_sel, visible, depth, rect, trect, 0)) { prep_free(&P); return -1; }
    int64_t W = cam->width, H = cam->height;
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthreads * (size_t)(n_sel ? n_sel : 1) * 9, sizeof(double));
    if (!acc) { prep_free(&P); return -1; }
    const int64_t cap = P.nvis > 0 ? P.nvis : 1;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * (size_t)(n_sel ? n_sel : 1) * 9;
        gc_step *steps = (gc_step *)malloc(sizeof(gc_step) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (int64_t k = 0; k < W * H; ++k) {
            double g[3] = {dLdimg[k], dLdimg[W * H + k], dLdimg[2 * W * H + k]};
            if (g[0] == 0 && g[1] == 0 && g[2] == 0) continue;
            int px = (int)(k % W), py = (int)(k / W);
            gc_pix r;
            int64_t ns = 0;
            composite_pixel(&P, op, px, py, &r, steps, cap, &ns);
            /* reverse: Atil = colour of everything behind step k, normalised by T_{k+1} */
            double At[3] = {op->bg[0], op->bg[1], op->bg[2]};
            for (int64_t s = ns - 1; s >= 0; --s) {
                const gc_step *st = &steps[s];
                const gc_geom *G = &P.geo[st->j];
                double *d = my + 9 * st->j;
                double dalpha = 0;
                for (int ch = 0; ch < 3; ++ch) {
                    d[6 + ch] += st->alpha * st->T * g[ch];
                    dalpha += g[ch] * (G->rgb[ch] - At[ch]);
                }
                dalpha *= st->T;
                for (int ch = 0; ch < 3; ++ch) At[ch] = st->alpha * G->rgb[ch] + (1.0 - st->alpha) * At[ch];
                if (st->clamped) continue;
                d[5] += dalpha * st->G;                       /* d opacity */
                double dpow = dalpha * G->o * st->G;          /* d power */
                double dx = st->dx, dy = st->dy;
                /* power = -0.5 (a dx^2 + c dy^2) - b dx dy, dx = px - u */
                d[2] += -0.5 * dx * dx * dpow;
                d[3] += -dx * dy * dpow;
                d[4] += -0.5 * dy * dy * dpow;
                d[0] += (G->conic[0] * dx + G->conic[1] * dy) * dpow;  /* d u */
                d[1] += (G->conic[1] * dx + G->conic[2] * dy) * dpow;  /* d v */
            }
        }
        free(steps);
    }
    /* reduce thread buffers into thread 0's */
    for (int t = 1; t < nthreads; ++t)
        for (int64_t e = 0; e < n_sel * 9; ++e) acc[e] += acc[(size_t)t * (size_t)n_sel * 9 + e];
    if (d2d) memcpy(d2d, acc, sizeof(double) * (size_t)n_sel * 9);

    int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    int G_n = (mo && mo->q) ? mo->n_groups : 1;
    memset(d_means, 0, sizeof(double) * (size_t)n_sel * 3);
    memset(d_log_scales, 0, sizeof(double) * (size_t)n_sel * 3);
    memset(d_quats, 0, sizeof(double) * (size_t)n_sel * 4);
    memset(d_logits, 0, sizeof(double) * (size_t)n_sel);
    memset(d_sh, 0, sizeof(double) * (size_t)n_sel * K * 3);
    if (d_gq) memset(d_gq, 0, sizeof(double) * (size_t)G_n * 4);
    if (d_gt) memset(d_gt, 0, sizeof(double) * (size_t)G_n * 3);
    double *pg_q = (double *)calloc((size_t)(n_sel ? n_sel : 1) * 4, sizeof(double));
    double *pg_t = (double *)calloc((size_t)(n_sel ? n_sel : 1) * 3, sizeof(double));

#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n_sel; ++j) {
        if (!visible[j]) continue;
        const gc_geom *G = &P.geo[j];
        const double *d = acc + 9 * j;
        double W9[9];
        for (int k = 0; k < 9; ++k) W9[k] = cam->R[k];
        double fx = cam->fx, fy = cam->fy, z = G->c[2];
        /* opacity */
        d_logits[j] = d[5] * G->o * (1.0 - G->o);
        /* colour: rgb = max(0, raw), raw = sum Y_k f_k + 0.5 */
        double draw[3];
        for (int ch = 0; ch < 3; ++ch) draw[ch] = G->raw[ch] > 0 ? d[6 + ch] : 0.0;
        double Y[16], dY[48];
        sh_eval_d(sc->sh_degree, G->dir, Y, dY);
        double ddir[3] = {0, 0, 0};
        for (int k = 0; k < K; ++k) {
            double s_k = 0;
            for (int ch = 0; ch < 3; ++ch) {
                d_sh[(j * K + k) * 3 + ch] = Y[k] * draw[ch];
                s_k += sh_d(sc, mo, sel[j], K, 3 * k + ch) * draw[ch];
            }
            for (int a = 0; a < 3; ++a) ddir[a] += s_k * dY[3 * k + a];
        }
        double dmup[3];
        double dd = G->dir[0] * ddir[0] + G->dir[1] * ddir[1] + G->dir[2] * ddir[2];
        for (int a = 0; a < 3; ++a) dmup[a] = (ddir[a] - G->dir[a] * dd) / G->dnorm;
        /* conic (ia, ib, ic) = inverse of [[A, B], [B, C]] */
        double Qm[4] = {G->conic[0], G->conic[1], G->conic[1], G->conic[2]};
        double Gc[4] = {d[2], 0.5 * d[3], 0.5 * d[3], d[4]};
        double tmp[4], GS[4];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) tmp[2 * r + c] = Qm[2 * r] * Gc[c] + Qm[2 * r + 1] * Gc[2 + c];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c) GS[2 * r + c] = -(tmp[2 * r] * Qm[c] + tmp[2 * r + 1] * Qm[2 + c]);
        /* Sigma2 = T Sigma T^T: dSigma = T^T GS T, dT = 2 GS T Sigma */
        double dSig[9], dT[6];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc2 = 0;
                for (int r = 0; r < 2; ++r)
                    for (int c = 0; c < 2; ++c) acc2 += G->T[3 * r + a] * GS[2 * r + c] * G->T[3 * c + b];
                dSig[3 * a + b] = acc2;
            }
        for (int r = 0; r < 2; ++r)
            for (int b = 0; b < 3; ++b) {
                double acc2 = 0;
                for (int c = 0; c < 2; ++c)
                    for (int a = 0; a < 3; ++a) acc2 += GS[2 * r + c] * G->T[3 * c + a] * G->Sig[3 * a + b];
                dT[3 * r + b] = 2.0 * acc2;
            }
        /* T = J W: dJ = dT W^T (entries 00, 02, 11, 12) */
        double dJ00 = 0, dJ02 = 0, dJ11 = 0, dJ12 = 0;
        for (int b = 0; b < 3; ++b) {
            dJ00 += dT[b] * W9[b];
            dJ02 += dT[b] * W9[6 + b];
            dJ11 += dT[3 + b] * W9[3 + b];
            dJ12 += dT[3 + b] * W9[6 + b];
        }
        /* camera point gradient: through J and through (u, v) */
        double dc[3] = {0, 0, 0};
        double x = G->c[0], y = G->c[1];
        dc[2] += dJ00 * (-fx / (z * z)) + dJ11 * (-fy / (z * z));
        if (G->clampx) dc[2] += dJ02 * (fx * G->xt / (z * z));
        else { dc[0] += dJ02 * (-fx / (z * z)); dc[2] += dJ02 * (2.0 * fx * x / (z * z * z)); }
        if (G->clampy) dc[2] += dJ12 * (fy * G->yt / (z * z));
        else { dc[1] += dJ12 * (-fy / (z * z)); dc[2] += dJ12 * (2.0 * fy * y / (z * z * z)); }
        dc[0] += d[0] * fx / z; dc[2] += d[0] * (-fx * x / (z * z));
        dc[1] += d[1] * fy / z; dc[2] += d[1] * (-fy * y / (z * z));
        for (int a = 0; a < 3; ++a) dmup[a] += W9[a] * dc[0] + W9[3 + a] * dc[1] + W9[6 + a] * dc[2];
        /* Sigma = M M^T, M = R diag(s) */
        double dM[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc2 = 0;
                for (int a = 0; a < 3; ++a) acc2 += (dSig[3 * r + a] + dSig[3 * a + r]) * G->M[3 * a + c];
                dM[3 * r + c] = acc2;
            }
        double dR[9];
        for (int c = 0; c < 3; ++c) {
            double ds = 0;
            for (int r = 0; r < 3; ++r) { ds += dM[3 * r + c] * G->R[3 * r + c]; dR[3 * r + c] = dM[3 * r + c] * G->s[c]; }
            d_log_scales[3 * j + c] = ds * G->s[c];
        }
        double dqn[4];
        quat_to_rot_vjp_d(G->qn, dR, dqn);
        double dot = 0;
        for (int k = 0; k < 4; ++k) dot += G->qn[k] * dqn[k];
        double dp[4];
        for (int k = 0; k < 4; ++k) dp[k] = (dqn[k] - G->qn[k] * dot) / G->pn;
        /* p = gq (x) q: dq = L(gq)^T dp, dgq = Rm(q)^T dp */
        int gi = sc->group_id ? sc->group_id[sel[j]] : 0;
        double a[4] = {1, 0, 0, 0};
        if (mo && mo->q) for (int k = 0; k < 4; ++k) a[k] = mo->q[4 * gi + k];
        const float *qq = sc->quats + 4 * sel[j];
        double b[4] = {qq[0], qq[1], qq[2], qq[3]};
        double Lm[16] = {a[0], -a[1], -a[2], -a[3],
                         a[1], a[0], -a[3], a[2],
                         a[2], a[3], a[0], -a[1],
                         a[3], -a[2], a[1], a[0]};
        double Rm[16] = {b[0], -b[1], -b[2], -b[3],
                         b[1], b[0], b[3], -b[2],
                         b[2], -b[3], b[0], b[1],
                         b[3], b[2], -b[1], b[0]};
        for (int c = 0; c < 4; ++c) {
            double s1 = 0, s2 = 0;
            for (int r = 0; r < 4; ++r) { s1 += Lm[4 * r + c] * dp[r]; s2 += Rm[4 * r + c] * dp[r]; }
            d_quats[4 * j + c] = s1;
            pg_q[4 * j + c] = s2;
        }
        for (int a2 = 0; a2 < 3; ++a2) { d_means[3 * j + a2] = dmup[a2]; pg_t[3 * j + a2] = dmup[a2]; }
    }
    /* per-group sums of the motion gradient */
    if (d_gq && d_gt) {
        for (int64_t j = 0; j < n_sel; ++j) {
            if (!visible[j]) continue;
            int gi = (mo && mo->q && sc->group_id) ? sc->group_id[sel[j]] : 0;
            for (int k = 0; k < 4; ++k) d_gq[4 * gi + k] += pg_q[4 * j + k];
            for (int k = 0; k < 3; ++k) d_gt[3 * gi + k] += pg_t[3 * j + k];
        }
    }
    free(pg_q); free(pg_t);
    free(acc);
    prep_free(&P);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exported primitives for pin tests                                         */
/* ------------------------------------------------------------------------ */

API void gco_quat_to_rot(const double *q, double *R) { quat_to_rot_d(q, R); }
API void gco_quat_mul(const double *a, const double *b, double *o) { qmul_d(a, b, o); }
API void gco_sh_eval(int deg, const double *dirs, int64_t n, double *Y, double *dY) {
    sh_init();
    int K = (deg + 1) * (deg + 1);
    for (int64_t i = 0; i < n; ++i) sh_eval_d(deg, dirs + 3 * i, Y + i * K, dY ? dY + i * 3 * K : NULL);
}

/* FP64 geometry of one Gaussian: u, v, Sigma2 (A, B, C incl. dilation), conic,
 * J (00, 02, 11, 12), opacity, rgb, camera point, 3D covariance (9). */
API void gco_geom_f64(const gco_scene *sc, const gco_motion *mo, const gco_camera *cam,
                      const gco_options *op, int64_t i, double *out) {
    gc_geom G;
    geom_d(sc, mo, cam, op, i, &G);
    out[0] = G.u; out[1] = G.v; out[2] = G.A; out[3] = G.B; out[4] = G.C;
    out[5] = G.conic[0]; out[6] = G.conic[1]; out[7] = G.conic[2];
    out[8] = G.J00; out[9] = G.J02; out[10] = G.J11; out[11] = G.J12;
    out[12] = G.o; out[13] = G.rgb[0]; out[14] = G.rgb[1]; out[15] = G.rgb[2];
    out[16] = G.c[0]; out[17] = G.c[1]; out[18] = G.c[2];
    for (int k = 0; k < 9; ++k) out[19 + k] = G.Sig[k];
}

API int gco_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision decoding from the format definitions                    */
/* ------------------------------------------------------------------------ */

/* bfloat16: the upper 16 bits of an IEEE binary32. */
API void gco_decode_bf16(const uint16_t *in, int64_t n, float *out) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t b = (uint32_t)in[i] << 16;
        float f;
        memcpy(&f, &b, 4);
        out[i] = f;
    }
}

/* float8 e4m3 (OCP "fn" variant): 1 sign, 4 exponent (bias 7), 3 mantissa
 * bits; exponent 0 is subnormal (m/8 * 2^-6); S.1111.111 is NaN; no inf. */
API void gco_decode_e4m3(const uint8_t *in, int64_t n, float *out) {
    for (int64_t i = 0; i < n; ++i) {
        int s = in[i] >> 7, e = (in[i] >> 3) & 15, m = in[i] & 7;
        double v;
        if (e == 15 && m == 7) v = NAN;
        else if (e == 0) v = ldexp((double)m / 8.0, -6);
        else v = ldexp(1.0 + (double)m / 8.0, e - 7);
        out[i] = (float)(s ? -v : v);
    }
}
