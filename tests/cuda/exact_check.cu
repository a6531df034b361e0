// exact_check.cu - checks the library's float-float evaluations of the binning
// specification's FP64 quantities (step 5: (float)exp((double)x); step 14: tau) against
// the FP64 expressions themselves, over a uniform grid and over scattered float bit
// patterns of [-60, 60].  Prints one line per (quantity, sampling): sample count,
// mismatches, FP64 fallbacks and the float-float error.
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cmath>
#include "gc_exact.cuh"
using namespace gc;

struct Out { unsigned long long mism, fall, n; double maxrel; };

__device__ double atomicMaxD(double *a, double v) {
    unsigned long long *p = (unsigned long long *)a, old = *p, as;
    do { as = old; if (__longlong_as_double(as) >= v) break; old = atomicCAS(p, as, __double_as_longlong(v)); } while (as != old);
    return __longlong_as_double(old);
}

// sample i of n: mode 0 a uniform grid over [lo, hi]; mode 1 scattered float bit patterns
// of magnitude <= hi (a multiplicative hash over the ordered patterns) with alternating sign
__device__ float xof(uint64_t i, uint64_t n, int mode, float lo, float hi) {
    if (mode == 0) return lo + (hi - lo) * (float)((double)i / (double)n);
    const uint64_t span = (uint64_t)(__float_as_uint(hi) & 0x7fffffffu);
    uint32_t m = (uint32_t)((i * 2654435761ull) % (span + 1));
    float v = __uint_as_float(m);
    return (i & 1) ? -v : v;
}

__global__ void k_exp(uint64_t n, int mode, Out *o) {
    unsigned long long mism = 0, fall = 0, cnt = 0; double mr = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float x = xof(i, n, mode, -60.f, 60.f);
        if (!(fabsf(x) <= 60.f)) continue;
        ++cnt;
        const float got = exp_f32_of_f64(x);
        const double ref = exp((double)x);
        if (got != (float)ref) ++mism;
        const ffx::F2 e = ffx::exp_ff(x);
        if (!ffx::rounds_to_hi(e, e.hi * 0x1p-40f)) ++fall;
        const double rel = fabs(((double)e.hi + (double)e.lo) - ref) / ref;
        if (rel > mr) mr = rel;
    }
    atomicAdd(&o->mism, mism); atomicAdd(&o->fall, fall); atomicAdd(&o->n, cnt); atomicMaxD(&o->maxrel, mr);
}

__global__ void k_tau(uint64_t n, int mode, Out *o) {
    unsigned long long mism = 0, fall = 0, cnt = 0; double mr = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float l = xof(i, n, mode, -60.f, 60.f);
        if (!(fabsf(l) <= 60.f)) continue;
        ++cnt;
        const float got = tau_f32_of_f64(l);
        const double refd = 2.0 * log(255.0 / (1.0 + exp(-(double)l)));
        const float ref = (float)refd;
        // only the sign matters for negative values
        const bool same = (ref > 0.f) ? (got == ref) : !(got > 0.f);
        if (!same) ++mism;
        // float-float error vs the FP64 value (absolute)
        using namespace ffx;
        const F2 u = exp_ff(-l);
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
        const double t = 2.0 * ((double)z.hi + (double)z.lo);
        const double ae = fabs(t - refd);
        if (ae > mr) mr = ae;
        const F2 tt = {2.f * z.hi, 2.f * z.lo};
        if (!(tt.hi < -0x1p-37f) && !(tt.hi >= 0x1p-12f && rounds_to_hi(tt, 0x1p-37f))) ++fall;
    }
    atomicAdd(&o->mism, mism); atomicAdd(&o->fall, fall); atomicAdd(&o->n, cnt); atomicMaxD(&o->maxrel, mr);
}

int main(int argc, char **argv) {
    Out *o; cudaMallocManaged(&o, sizeof(Out));
    const uint64_t N = argc > 1 ? strtoull(argv[1], nullptr, 10) : (1ull << 24);
    for (int mode = 0; mode < 2; ++mode) {
        *o = Out{0, 0, 0, 0.0};
        k_exp<<<148 * 8, 256>>>(N, mode, o); cudaDeviceSynchronize();
        printf("exp %d %llu %llu %llu %.6e\n", mode, o->n, o->mism, o->fall, o->maxrel);
        *o = Out{0, 0, 0, 0.0};
        k_tau<<<148 * 8, 256>>>(N, mode, o); cudaDeviceSynchronize();
        printf("tau %d %llu %llu %llu %.6e\n", mode, o->n, o->mism, o->fall, o->maxrel);
    }
    cudaError_t e = cudaGetLastError();
    printf("%s\n", cudaGetErrorString(e));
    return e != cudaSuccess;
}
