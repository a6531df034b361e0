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

// Steps shared by both forms, for the channel row yc: symbol range and validity, the symbol
// histogram in shared memory (cnt[k] = count of symbol lo + k) and the bandwidth.  Returns
// false (every thread) for an unsupported channel: a non-finite or huge value, or more than
// kMaxSymbols symbol values.
__device__ bool channel_density(const float *__restrict__ yc, int64_t n, uint32_t *cnt, long long *ws_i,
                                int &lo_out, int &M_out, double &h_out) {
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
    if (gbad || M > kMaxSymbols) return false;
    for (int k = threadIdx.x; k < (int)M; k += kKT) cnt[k] = 0u;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += kKT) atomicAdd(&cnt[(int)rintf(yc[i]) - (int)glo], 1u);
    __syncthreads();
    // bandwidth from the exact integer moments of the histogram
    long long s1 = 0, s2 = 0;
    for (int k = threadIdx.x; k < (int)M; k += kKT) {
        const long long c = cnt[k];
        s1 += c * k;
        s2 += c * (long long)k * k;
    }
    s1 = block_reduce<long long>(s1, ws_i);
    s2 = block_reduce<long long>(s2, ws_i);
    const double N = (double)n;
    const double var = n > 1 ? ((double)s2 - (double)s1 * (double)s1 / N) / (N - 1.0) : 0.0;
    lo_out = (int)glo;
    M_out = (int)M;
    h_out = var > 0.0 ? sqrt(var) * pow(0.75 * N, -0.2) : 1.0;
    return true;
}

__global__ void __launch_bounds__(kKT) k_kde_rate(const float *__restrict__ y, int64_t n, int64_t stride,
                                                  float *__restrict__ rate) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *cnt = smem;                                      // kMaxSymbols counts
    float *w = reinterpret_cast<float *>(smem + kMaxSymbols);  // taps w(0..D)
    __shared__ long long ws_i[kKT / 32];
    __shared__ double ws_d[kKT / 32];
    const float *yc = y + (int64_t)blockIdx.x * stride;
    int lo, M;
    double h;
    if (!channel_density(yc, n, cnt, ws_i, lo, M, h)) {
        if (threadIdx.x == 0) rate[blockIdx.x] = __int_as_float(0x7fc00000);  // NaN: unsupported channel
        return;
    }
    const double N = (double)n;
    int D = (int)ceil(12.0 * h) + 1;  // w(d) < 1e-32 beyond 12 h
    if (D > M - 1) D = M - 1;
    // taps in FP64: upper-tail differences for d >= 1, 1 - 2 Phi(-1/(2h)) at d = 0
    for (int d = threadIdx.x; d <= D; d += kKT) {
        const double t = d == 0 ? 1.0 - 2.0 * normcdf(-0.5 / h) : normcdf(-(d - 0.5) / h) - normcdf(-(d + 0.5) / h);
        w[d] = (float)t;
    }
    __syncthreads();
    // PMF at every occupied symbol and its share of the code length
    double acc = 0.0;
    for (int v = threadIdx.x; v < M; v += kKT) {
        const uint32_t cv = cnt[v];
        if (!cv) continue;
        float p = 0.f;
        const int u0 = max(v - D, 0), u1 = min(v + D, M - 1);
        for (int u = u0; u <= u1; ++u) p = fmaf((float)cnt[u], w[abs(v - u)], p);
        const float pmf = fmaxf(p / (float)n, 9.094947e-13f);   // floor 2^-40
        acc += (double)cv * (double)log2f(pmf);
    }
    acc = block_reduce<double>(acc, ws_d);
    if (threadIdx.x == 0) rate[blockIdx.x] = (float)(-acc / N);
}

// Training form: the rate of the noise-injected values x_i under the fixed density of their
// symbols, and dR/dx_i = -(pdf(x_i + 1/2) - pdf(x_i - 1/2)) / (N ln2 P(x_i)).  Three kernels:
// the channel's histogram and bandwidth (one CTA per channel), the per-value sums (a CTA per
// chunk of kGradChunk values of a channel, the histogram in shared memory), and the channel
// totals (the chunks' partial sums added in chunk order: reproducible).
constexpr int kGradChunk = 2048;

__global__ void __launch_bounds__(kKT) k_kde_density(const float *__restrict__ y, int64_t n, int64_t stride,
                                                     uint32_t *__restrict__ hist, int *__restrict__ ch_lo,
                                                     int *__restrict__ ch_m, double *__restrict__ ch_h) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ long long ws_i[kKT / 32];
    const int c = blockIdx.x;
    int lo, M;
    double h;
    if (!channel_density(y + (int64_t)c * stride, n, smem, ws_i, lo, M, h)) {
        if (threadIdx.x == 0) ch_m[c] = 0;  // unsupported channel
        return;
    }
    for (int k = threadIdx.x; k < M; k += kKT) hist[(size_t)c * kMaxSymbols + k] = smem[k];
    if (threadIdx.x == 0) {
        ch_lo[c] = lo;
        ch_m[c] = M;
        ch_h[c] = h;
    }
}

// For each value x of the chunk the bins k of the symbols within 8 h + 1 are visited in
// order (a bin farther away holds mass below Phi(-8) = 6e-16 of its count, while P(x) >=
// about 1 / (N h) from x's own symbol: the relative truncation error stays below 1e-9); bin k spans the standardised boundaries zu = (x - s_k + 1/2) / h > zl = (x - s_k -
// 1/2) / h, and the lower boundary of bin k is the upper one of bin k + 1, so each boundary
// costs one erfc and one exp.  Phi(zu) - Phi(zl) is taken between upper tails q(|z|) =
// Phi(-|z|) on the side of zero where both boundaries lie (no cancellation).
__global__ void __launch_bounds__(kKT) k_kde_grad_values(
    const float *__restrict__ y, int64_t n, int64_t stride, int nchunks, const uint32_t *__restrict__ hist,
    const int *__restrict__ ch_lo, const int *__restrict__ ch_m, const double *__restrict__ ch_h,
    const float *__restrict__ d_rate, float *__restrict__ d_y, double *__restrict__ partial) {
    extern __shared__ __align__(16) uint32_t cnt[];
    __shared__ double ws_d[kKT / 32];
    const int c = blockIdx.x / nchunks, chunk = blockIdx.x - c * nchunks;
    const int64_t i0 = (int64_t)chunk * kGradChunk, i1 = min(n, i0 + kGradChunk);
    const float *yc = y + (int64_t)c * stride;
    float *dyc = d_y ? d_y + (int64_t)c * stride : nullptr;
    const int M = ch_m[c];
    if (M == 0) {  // unsupported channel: NaN gradients, NaN partial
        if (dyc)
            for (int64_t i = i0 + threadIdx.x; i < i1; i += kKT) dyc[i] = __int_as_float(0x7fc00000);
        if (threadIdx.x == 0) partial[blockIdx.x] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    for (int k = threadIdx.x; k < M; k += kKT) cnt[k] = hist[(size_t)c * kMaxSymbols + k];
    __syncthreads();
    const int lo = ch_lo[c];
    const double h = ch_h[c];
    const float inv_h = (float)(1.0 / h);
    const float span = (float)(8.0 * h + 1.0);
    const float inv_n = (float)(1.0 / (double)n);
    const float gscale = (float)(-1.0 / ((double)n * 0.6931471805599453));  // -1 / (N ln 2)
    const float up = d_rate ? d_rate[c] : 1.f;
    const float kInvSqrt2 = 0.70710678118654752f, kInvSqrt2Pi = 0.39894228040143268f;
    const float floor40 = 9.094947e-13f;  // 2^-40
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += kKT) {
        const float x = yc[i];
        const float rel = x - (float)lo;  // position in histogram index units
        const int k0 = max(0, (int)floorf(rel - span)), k1 = min(M - 1, (int)ceilf(rel + span));
        float P = 0.f, dP = 0.f;
        float zu = (rel - (float)k0 + 0.5f) * inv_h;
        float qu = 0.5f * erfcf(fabsf(zu) * kInvSqrt2), eu = expf(-0.5f * zu * zu);
        for (int k = k0; k <= k1; ++k) {
            const float zl = (rel - (float)k - 0.5f) * inv_h;
            const float ql = 0.5f * erfcf(fabsf(zl) * kInvSqrt2), el = expf(-0.5f * zl * zl);
            const float cf = (float)cnt[k];
            if (cf != 0.f) {
                const float mass = zl >= 0.f ? ql - qu : (zu <= 0.f ? qu - ql : (1.f - qu) - ql);
                P = fmaf(cf, mass, P);
                dP = fmaf(cf, eu - el, dP);
            }
            zu = zl;
            qu = ql;
            eu = el;
        }
        P *= inv_n;
        dP *= inv_n * inv_h * kInvSqrt2Pi;  // pdf(x + 1/2) - pdf(x - 1/2)
        acc += (double)log2f(fmaxf(P, floor40));
        if (dyc) dyc[i] = P > floor40 ? up * gscale * dP / P : 0.f;
    }
    acc = block_reduce<double>(acc, ws_d);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void k_kde_grad_final(const double *__restrict__ partial, int nchunks, int n_channels, int64_t n,
                                 float *__restrict__ rate) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_channels) return;
    double acc = 0.0;
    for (int k = 0; k < nchunks; ++k) acc += partial[(size_t)c * nchunks + k];
    rate[c] = (float)(-acc / (double)n);  // NaN stays NaN
}

}  // namespace

}  // namespace gc

extern "C" gc_status gc_kde_rate_grad(gc_context *ctx, const float *y, int32_t n_channels, int64_t n,
                                      int64_t stride, const float *d_rate, float *rate, float *d_y, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (n_channels < 0 || n < 1 || stride < n) return fail(ctx, GC_ERR_INVALID_ARG, "need n >= 1 and stride >= n");
    if (n_channels == 0) return GC_OK;
    if (!y || !rate) return fail(ctx, GC_ERR_INVALID_ARG, "y or rate is NULL");
    if (n > 0x7fffffffll) return fail(ctx, GC_ERR_INVALID_ARG, "n exceeds 2^31 - 1");
    const int64_t nchunks = (n + gc::kGradChunk - 1) / gc::kGradChunk;
    if ((int64_t)n_channels * nchunks > 0x7fffffffll)
        return fail(ctx, GC_ERR_INVALID_ARG, "n_channels x ceil(n / %d) exceeds 2^31 - 1", gc::kGradChunk);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // scratch: histograms (n_channels x kMaxSymbols), lo, M, h per channel, partials per chunk
    const size_t hist_b = (size_t)n_channels * gc::kMaxSymbols * 4, meta_b = (size_t)n_channels * 16,
                 part_b = (size_t)n_channels * nchunks * 8;
    GC_CUDA(ctx, grow(ctx->kde_scratch, hist_b + meta_b + part_b + 64));
    char *base = static_cast<char *>(ctx->kde_scratch.p);
    uint32_t *hist = reinterpret_cast<uint32_t *>(base);
    double *ch_h = reinterpret_cast<double *>(base + hist_b);
    int *ch_lo = reinterpret_cast<int *>(base + hist_b + (size_t)n_channels * 8);
    int *ch_m = ch_lo + n_channels;
    double *partial = reinterpret_cast<double *>(base + hist_b + meta_b);
    const size_t smem = (size_t)gc::kMaxSymbols * 4;
    GC_CUDA(ctx, cudaFuncSetAttribute(gc::k_kde_density, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GC_CUDA(ctx, cudaFuncSetAttribute(gc::k_kde_grad_values, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    gc::k_kde_density<<<n_channels, gc::kKT, smem, s>>>(y, n, stride, hist, ch_lo, ch_m, ch_h);
    gc::k_kde_grad_values<<<(unsigned)(n_channels * nchunks), gc::kKT, smem, s>>>(
        y, n, stride, (int)nchunks, hist, ch_lo, ch_m, ch_h, d_rate, d_y, partial);
    gc::k_kde_grad_final<<<(n_channels + 127) / 128, 128, 0, s>>>(partial, (int)nchunks, n_channels, n, rate);
    gc::note_launches(3);
    GC_CUDA(ctx, cudaGetLastError());
    return GC_OK;
}

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
