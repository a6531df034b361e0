// gc_kde.cu - the KDE rate estimate of the keyframe RD loss (4DGCPro Sec. 3.3): for each
// attribute channel, the bits per symbol of its quantised symbols s_i = round(y_i) under the
// Gaussian kernel density of those symbols (Silverman-rule bandwidth h = sigma (3N/4)^(-1/5)),
// PMF(k) = CDF(k + 1/2) - CDF(k - 1/2), rate = -(1/N) sum_i log2 max(PMF(s_i), 2^-40).
//
// One CTA per channel.  The symbols are integers, so the PMF at every symbol value is the
// symbol histogram convolved with the kernel taps w(d) = Phi((d + 1/2) / h) - Phi((d - 1/2) / h)
// (the paper's FFT convolution computes the same sum); the histogram lives in shared memory,
// the taps are evaluated in FP64 (tail form, no cancellation) and truncated where they fall
// below 1e-32, and the convolution runs only over the occupied symbol range.
#include <cuda_runtime.h>

#include <cmath>

#include "gc_state.cuh"

namespace gc {

namespace {

constexpr int kKT = 256;
constexpr int kMaxSymbols = 8192;   // symbol values spanned by one channel
constexpr size_t kKdeSmem = (size_t)kMaxSymbols * 4 * 2;   // histogram + taps

template <typename T>
__device__ __forceinline__ T block_reduce(T v, T *ws, bool is_max = false, bool is_min = false) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? (u > v ? u : v) : is_min ? (u < v ? u : v) : v + u;
    }
    __syncthreads();
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    T r = ws[0];
    for (int w = 1; w < kKT / 32; ++w) {
        const T u = ws[w];
        r = is_max ? (u > r ? u : r) : is_min ? (u < r ? u : r) : r + u;
    }
    return r;
}

__global__ void __launch_bounds__(kKT) k_kde_rate(const float *__restrict__ y, int64_t n, int64_t stride,
                                                  float *__restrict__ rate) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *cnt = smem;                                      // kMaxSymbols counts
    float *w = reinterpret_cast<float *>(smem + kMaxSymbols);  // taps w(0..D)
    __shared__ long long ws_i[kKT / 32];
    __shared__ double ws_d[kKT / 32];
    const float *yc = y + (int64_t)blockIdx.x * stride;
    // 1. symbol range (and validity)
    int lo = 0x7fffffff, hi = -0x7fffffff;
    int bad = 0;
    for (int64_t i = threadIdx.x; i < n; i += kKT) {
        const float v = yc[i];
        if (!(fabsf(v) <= 16777216.f)) {
            bad = 1;
            continue;
        }
        const int s = (int)rintf(v);
        lo = min(lo, s);
        hi = max(hi, s);
    }
    const long long gbad = block_reduce<long long>(bad, ws_i);
    const long long glo = block_reduce<long long>(lo, ws_i, false, true);
    const long long ghi = block_reduce<long long>(hi, ws_i, true, false);
    const long long M = ghi - glo + 1;
    if (gbad || M > kMaxSymbols) {
        if (threadIdx.x == 0) rate[blockIdx.x] = __int_as_float(0x7fc00000);  // NaN: unsupported channel
        return;
    }
    // 2. histogram
    for (int k = threadIdx.x; k < (int)M; k += kKT) cnt[k] = 0u;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += kKT) atomicAdd(&cnt[(int)rintf(yc[i]) - (int)glo], 1u);
    __syncthreads();
    // 3. bandwidth from the exact integer moments of the histogram
    long long s1 = 0, s2 = 0;
    for (int k = threadIdx.x; k < (int)M; k += kKT) {
        const long long c = cnt[k];
        s1 += c * k;
        s2 += c * (long long)k * k;
    }
    s1 = block_reduce<long long>(s1, ws_i);
    s2 = block_reduce<long long>(s2, ws_i);
    const double N = (double)n;
    double var = n > 1 ? ((double)s2 - (double)s1 * (double)s1 / N) / (N - 1.0) : 0.0;
    const double h = var > 0.0 ? sqrt(var) * pow(0.75 * N, -0.2) : 1.0;
    int D = (int)ceil(12.0 * h) + 1;  // w(d) < 1e-32 beyond 12 h
    if (D > (int)M - 1) D = (int)M - 1;
    // 4. taps in FP64: upper-tail differences for d >= 1, 1 - 2 Phi(-1/(2h)) at d = 0
    for (int d = threadIdx.x; d <= D; d += kKT) {
        const double t = d == 0 ? 1.0 - 2.0 * normcdf(-0.5 / h) : normcdf(-(d - 0.5) / h) - normcdf(-(d + 0.5) / h);
        w[d] = (float)t;
    }
    __syncthreads();
    // 5. PMF at every occupied symbol and its share of the code length
    double acc = 0.0;
    for (int v = threadIdx.x; v < (int)M; v += kKT) {
        const uint32_t cv = cnt[v];
        if (!cv) continue;
        float p = 0.f;
        const int u0 = max(v - D, 0), u1 = min(v + D, (int)M - 1);
        for (int u = u0; u <= u1; ++u) p = fmaf((float)cnt[u], w[abs(v - u)], p);
        const float pmf = fmaxf(p / (float)n, 9.094947e-13f);   // floor 2^-40
        acc += (double)cv * (double)log2f(pmf);
    }
    acc = block_reduce<double>(acc, ws_d);
    if (threadIdx.x == 0) rate[blockIdx.x] = (float)(-acc / N);
}

}  // namespace

}  // namespace gc

extern "C" gc_status gc_kde_rate(gc_context *ctx, const float *y, int32_t n_channels, int64_t n, int64_t stride,
                                 float *rate, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (n_channels < 0 || n < 1 || stride < n) return fail(ctx, GC_ERR_INVALID_ARG, "need n >= 1 and stride >= n");
    if (n_channels == 0) return GC_OK;
    if (!y || !rate) return fail(ctx, GC_ERR_INVALID_ARG, "y or rate is NULL");
    if (n > 0x7fffffffll) return fail(ctx, GC_ERR_INVALID_ARG, "n exceeds 2^31 - 1");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    GC_CUDA(ctx, cudaFuncSetAttribute(gc::k_kde_rate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)gc::kKdeSmem));
    gc::k_kde_rate<<<n_channels, gc::kKT, gc::kKdeSmem, s>>>(y, n, stride, rate);
    gc::note_launches(1);
    GC_CUDA(ctx, cudaGetLastError());
    return GC_OK;
}
