// gc_blend.cuh - the per-(pixel, Gaussian) evaluation shared by the forward and the
// backward blend.  Written with explicit rounding intrinsics so both kernels compute
// bit-identical powers and alphas, and therefore take identical skip decisions.
#pragma once

namespace gc {

// power = -1/2 (a dx^2 + c dy^2) - b dx dy  (the exponent of Eq. 1 in the image plane)
__device__ __forceinline__ float blend_power(float ca, float cb, float cc, float dx, float dy) {
    const float q = __fmaf_rn(ca, __fmul_rn(dx, dx), __fmul_rn(cc, __fmul_rn(dy, dy)));
    return __fmaf_rn(-0.5f, q, -__fmul_rn(cb, __fmul_rn(dx, dy)));
}

// o * exp(power) (before the 0.99 clamp)
__device__ __forceinline__ float blend_raw_alpha(float opacity, float power, float &G) {
    G = __expf(power);
    return __fmul_rn(opacity, G);
}

constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTStop = 1e-4f;

}  // namespace gc
