// gc_loss.cu - the L1 photometric distortion of a rendered image against a target image: the
// L1 part of the colour loss of the rate-distortion training (Sec. 3.3, weighted there by
// 1 - lambda_ssim beside a D-SSIM term, which is not built here):
//   loss = scale * sum_i |image_i - target_i|,   dL/dimage_i = scale * sign(image_i - target_i)
// with sign(0) = 0 (scale = 1 / n gives the mean).  One pass reads both images and writes the
// gradient; the loss is summed deterministically: a fixed grid writes one FP64 partial per
// CTA and a single CTA adds the partials in CTA order.
#include <cuda_runtime.h>

#include "gc_state.cuh"

namespace gc {

namespace {

constexpr int kLossThreads = 256;
constexpr int kLossMaxCtas = 148 * 8;

__device__ __forceinline__ float sgn(float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); }

__device__ __forceinline__ double block_sum(double v, double *ws) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kLossThreads / 32; ++w) r += ws[w];
    return r;  // valid in thread 0
}

// vec: image, target and grad are 16-byte aligned, so n / 4 float4 loads cover the bulk
__global__ void __launch_bounds__(kLossThreads) k_l1_loss(const float *__restrict__ img,
                                                          const float *__restrict__ tgt, int64_t n,
                                                          float scale, float *__restrict__ grad, bool vec,
                                                          double *__restrict__ part) {
    __shared__ double ws[kLossThreads / 32];
    const int64_t tid = (int64_t)blockIdx.x * kLossThreads + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * kLossThreads;
    double acc = 0.0;
    int64_t done = 0;
    if (vec) {
        const int64_t n4 = n >> 2;
        const float4 *a4 = reinterpret_cast<const float4 *>(img);
        const float4 *b4 = reinterpret_cast<const float4 *>(tgt);
        for (int64_t i = tid; i < n4; i += stride) {
            const float4 a = a4[i], b = b4[i];
            const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            acc += (double)((fabsf(d0) + fabsf(d1)) + (fabsf(d2) + fabsf(d3)));
            if (grad)
                reinterpret_cast<float4 *>(grad)[i] =
                    make_float4(scale * sgn(d0), scale * sgn(d1), scale * sgn(d2), scale * sgn(d3));
        }
        done = n4 << 2;
    }
    for (int64_t i = done + tid; i < n; i += stride) {
        const float d = img[i] - tgt[i];
        acc += (double)fabsf(d);
        if (grad) grad[i] = scale * sgn(d);
    }
    const double s = block_sum(acc, ws);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kLossThreads) k_l1_loss_final(const double *__restrict__ part, int n_part,
                                                                float scale, float *__restrict__ loss) {
    __shared__ double ws[kLossThreads / 32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n_part; i += kLossThreads) acc += part[i];
    const double s = block_sum(acc, ws);
    if (threadIdx.x == 0) *loss = (float)(s * (double)scale);
}

}  // namespace

}  // namespace gc

extern "C" gc_status gc_l1_loss(gc_context *ctx, const float *image, const float *target, int64_t n, float scale,
                                float *dL_dimage, float *loss, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, GC_ERR_INVALID_ARG, "n must be >= 0");
    if (n > 0 && (!image || !target)) return fail(ctx, GC_ERR_INVALID_ARG, "image or target is NULL");
    if (!dL_dimage && !loss) return GC_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t per_cta = (int64_t)gc::kLossThreads * 4 * 4;  // four float4 per thread
    const int ctas = (int)std::max<int64_t>(1, std::min<int64_t>((n + per_cta - 1) / per_cta, gc::kLossMaxCtas));
    GC_CUDA(ctx, grow(ctx->loss_part, (size_t)gc::kLossMaxCtas * 8));
    const bool vec = ((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(target) |
                       reinterpret_cast<uintptr_t>(dL_dimage)) & 15) == 0;
    gc::k_l1_loss<<<ctas, gc::kLossThreads, 0, s>>>(image, target, n, scale, dL_dimage, vec,
                                                    ctx->loss_part.as<double>());
    GC_CUDA(ctx, cudaGetLastError());
    gc::note_launches(1);
    if (loss) {
        gc::k_l1_loss_final<<<1, gc::kLossThreads, 0, s>>>(ctx->loss_part.as<double>(), ctas, scale, loss);
        GC_CUDA(ctx, cudaGetLastError());
        gc::note_launches(1);
    }
    return GC_OK;
}
