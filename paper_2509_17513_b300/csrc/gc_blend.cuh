// gc_blend.cuh - the per-(pixel, Gaussian) evaluation shared by the forward and the
// backward blend.  Written with explicit rounding intrinsics so both kernels compute
// bit-identical exponents and alphas, and therefore take identical skip decisions.
//
// The depth-ranked record stores the conic pre-scaled by -log2(e)/2 (diagonal) and
// -log2(e) (off-diagonal): A = -a log2e / 2, B = -b log2e, C = -c log2e / 2, so that
//   power2 = A dx^2 + B dx dy + C dy^2 = log2(e) * (-(a dx^2 + 2 b dx dy + c dy^2) / 2)
// and the Gaussian's value exp(power) of Eq. 1 in the image plane is 2^power2.
#pragma once

namespace gc {

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;
// natural conic from the pre-scaled one: a = -2 ln2 A, b = -ln2 B, c = -2 ln2 C
constexpr float kUnscaleDiag = -1.3862943611198906f;
constexpr float kUnscaleOff = -0.69314718055994531f;

__device__ __forceinline__ float blend_power2(float A, float B, float C, float dx, float dy) {
    const float t = __fmaf_rn(A, dx, __fmul_rn(B, dy));
    return __fmaf_rn(__fmul_rn(C, dy), dy, __fmul_rn(dx, t));
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// o * 2^power2 (before the 0.99 clamp); G = 2^power2
__device__ __forceinline__ float blend_raw_alpha(float opacity, float power2, float &G) {
    G = ex2_approx(power2);
    return __fmul_rn(opacity, G);
}

}  // namespace gc
