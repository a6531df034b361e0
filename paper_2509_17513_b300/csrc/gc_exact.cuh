// gc_exact.cuh - the two FP64-defined quantities of the binning specification, rounded to
// FP32, without the FP64 pipe in the common case:
//   step 5:  s   = (float)exp((double)log_s)
//   step 14: tau = (float)(2 ln(255 / (1 + exp(-logit))))   (evaluated in FP64, rounded once)
//
// Both are first evaluated in float-float arithmetic (an unevaluated sum hi + lo of two
// floats, about 44 significant bits) from their mathematical definitions: e^x by range
// reduction x = k ln2 + r and the Taylor series of e^r, ln y by one Newton step on
// e^z = y from an FP32 start.  If the float-float value lies farther from the nearest
// FP32 rounding boundary than its error bound plus the FP64 evaluation's own error, the
// FP64 expression rounds to the same float, which is returned; otherwise (about one call
// in 2^14) the FP64 expression itself is evaluated.  The result is therefore the FP64
// expression's float in every case.  The FP64 pipe of sm_103a runs at a small fraction of
// the FP32 rate, which made these five transcendental evaluations half of the preprocess.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace gc {
namespace ffx {

struct F2 {
    float hi, lo;
};

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 mul(F2 a, F2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact low part of a.hi * b.hi
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ F2 add(F2 a, F2 b) {
    const F2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// ln 2 = kLn2Hi + kLn2Lo + kLn2Lo2 (each the float nearest to what remains).
constexpr float kLn2Hi = 0.693147182464599609375f;
constexpr float kLn2Lo = -1.9046542121259336e-09f;
constexpr float kLn2Lo2 = -8.78318373858934e-17f;
constexpr float kLog2e = 1.44269502162933349609375f;

// 1/j! as float-float for j <= 6, as float for 7 <= j <= 11.
__device__ __forceinline__ F2 inv_fact(int j) {
    switch (j) {
        case 0: return {1.f, 0.f};
        case 1: return {1.f, 0.f};
        case 2: return {0.5f, 0.f};
        case 3: return {0.1666666716337204f, -4.967053879312289e-09f};
        case 4: return {0.0416666679084301f, -1.2417634698280722e-09f};
        case 5: return {0.008333333767950535f, -4.34617203337595e-10f};
        default: return {0.0013888889225199819f, -3.3631094437103215e-11f};
    }
}

// e^x as float-float for |x| <= 60.  k = rint(x log2e), r = x - k ln2 (|r| <= 0.347):
// k ln2_hi is split exactly by an FMA, x - k ln2_hi is exact (Sterbenz), the two smaller
// parts of ln 2 are subtracted in float-float.  e^r = sum_{j<=11} r^j / j! by Horner
// (terms 7..11 in FP32: they are below 1.3e-7, so their FP32 rounding stays under 2^-46;
// terms 0..6 in float-float); truncation r^12/12! < 2^-47.  Then scaled by 2^k exactly.
__device__ __forceinline__ F2 exp_ff(float x) {
    const float k = rintf(__fmul_rn(x, kLog2e));
    const float kh = __fmul_rn(k, kLn2Hi);
    const float ke = __fmaf_rn(k, kLn2Hi, -kh);    // k ln2_hi = kh + ke
    const float s = __fsub_rn(x, kh);               // exact
    const float pl = __fmul_rn(k, kLn2Lo);
    const float pe = __fmaf_rn(k, kLn2Lo, -pl);     // k ln2_lo = pl + pe
    const F2 c = two_sum(ke, pl);
    const float tiny = __fadd_rn(__fadd_rn(c.lo, pe), __fmul_rn(k, kLn2Lo2));
    F2 r = two_sum(s, -c.hi);
    r = fast_two_sum(r.hi, __fsub_rn(r.lo, tiny));  // r = x - k ln2
    float q = 2.505210838544172e-08f;               // 1/11!
    q = __fmaf_rn(q, r.hi, 2.755731922398589e-07f);  // 1/10!
    q = __fmaf_rn(q, r.hi, 2.7557319223985893e-06f);  // 1/9!
    q = __fmaf_rn(q, r.hi, 2.48015873015873e-05f);   // 1/8!
    q = __fmaf_rn(q, r.hi, 0.0001984126984126984f);  // 1/7!
    F2 p = add(mul({q, 0.f}, r), inv_fact(6));
#pragma unroll
    for (int j = 5; j >= 0; --j) p = add(mul(p, r), inv_fact(j));
    const float scale = __uint_as_float((uint32_t)(127 + (int)k) << 23);  // 2^k, |k| <= 87
    return {__fmul_rn(p.hi, scale), __fmul_rn(p.lo, scale)};
}

// True when the float nearest to v.hi + v.lo (normalised, v.hi > 0 normal with exponent
// field >= 24) is v.hi and every value within `tol` of it rounds to v.hi as well.
__device__ __forceinline__ bool rounds_to_hi(F2 v, float tol) {
    const uint32_t b = __float_as_uint(v.hi);
    const float ulp = __uint_as_float((b & 0x7f800000u) - (23u << 23));
    const bool pow2 = (b & 0x007fffffu) == 0u;
    const float half = (pow2 && v.lo < 0.f) ? 0.25f * ulp : 0.5f * ulp;
    return fabsf(v.lo) < half - tol;
}

}  // namespace ffx

// (float)exp((double)x): the FP64 exponential has an error below one FP64 ulp, the
// float-float one below 2^-43 relative; 2^-40 relative is the margin.
__device__ __forceinline__ float exp_f32_of_f64(float x) {
    if (fabsf(x) <= 60.f) {
        const ffx::F2 e = ffx::exp_ff(x);
        if (ffx::rounds_to_hi(e, e.hi * 0x1p-40f)) return e.hi;
    }
    return (float)exp((double)x);
}

// (float)(2 ln(255 / (1 + exp(-logit)))) in FP64.  Float-float: u = e^-logit, y = 255 / (1 + u)
// (one correction step of the quotient), z0 = logf(y), z = z0 + ln(y e^-z0) with
// ln(1 + w) = w - w^2/2 for the tiny w; absolute error of 2z below 2^-40, the FP64
// expression's below 2^-46; 2^-37 is the margin.  A clearly negative value is returned
// as is: only its sign is used (opacity <= 1/255, never binned).
__device__ __forceinline__ float tau_f32_of_f64(float logit) {
    if (fabsf(logit) <= 60.f) {
        using namespace ffx;
        const F2 u = exp_ff(-logit);
        const F2 d = add({1.f, 0.f}, u);
        const float q1 = __fdiv_rn(255.f, d.hi);
        const float ph = __fmul_rn(q1, d.hi);
        const float pe = __fmaf_rn(q1, d.hi, -ph);
        const float rem = __fsub_rn(__fsub_rn(__fsub_rn(255.f, ph), pe), __fmul_rn(q1, d.lo));
        const F2 y = fast_two_sum(q1, __fdiv_rn(rem, d.hi));
        const float z0 = logf(y.hi);
        F2 w = mul(y, exp_ff(-z0));
        w = add(w, {-1.f, 0.f});
        const float corr = __fsub_rn(w.lo, __fmul_rn(0.5f, __fmul_rn(w.hi, w.hi)));
        F2 z = two_sum(z0, w.hi);
        z = fast_two_sum(z.hi, __fadd_rn(z.lo, corr));
        const F2 t = {__fmul_rn(2.f, z.hi), __fmul_rn(2.f, z.lo)};
        constexpr float kTol = 0x1p-37f;
        if (t.hi < -kTol) return t.hi;
        if (t.hi >= 0x1p-12f && rounds_to_hi(t, kTol)) return t.hi;
    }
    return (float)(2.0 * log(255.0 / (1.0 + exp(-(double)logit))));
}

}  // namespace gc
