// gc_motion_field.cu - the per-Gaussian motion source of 4DGCPro Sec. 3.2 (rigid
// transformation): a multi-resolution hash grid interpolated at the frame t-1 positions and
// two MLPs of one hidden layer (64 ReLU units) giving each Gaussian's translation and
// rotation.  Forward and backward, one thread per Gaussian.
//
// The cell of each level (an integer) is decided in FP32 with every operation rounded once,
// as the oracle does; interpolation and the MLPs are free FP32 arithmetic.  The MLPs are
// FP32 SIMT: their contraction (per Gaussian 2 x 64 x 32 + 7 x 64 multiply-adds) is small,
// and FP32 keeps the forward within FP32 rounding of the FP64 oracle.
//
// Backward: per block of 128 Gaussians the hidden activations and their gradients are
// staged in shared memory and the weight gradients summed over the block; the per-block sums
// are added over the blocks in block order by a second kernel (deterministic).  The table
// gradient is scattered with atomic additions.
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_state.cuh"

namespace gc {

namespace {

constexpr int kHidden = 64;
constexpr int kMaxLv = 16;
constexpr int kIn = 2 * kMaxLv;   // MLP input, zero-padded to 16 levels
constexpr int kFT = 128;          // threads per block
// per-block partial gradient layout: net 0 (translation) then net 1 (rotation), each
// w1 (kHidden x kIn, padded), b1 (kHidden), w2 (outs x kHidden), b2 (outs)
constexpr int kNetOff1 = kHidden * kIn + kHidden + 3 * kHidden + 3;
constexpr int kPartials = kNetOff1 + kHidden * kIn + kHidden + 4 * kHidden + 4;

struct Field {
    int L, log2T;
    int res[kMaxLv];
    float lo[3], hi[3];
    const float *table;
    const float *w1[2], *b1[2], *w2[2], *b2[2];
};

struct FieldSmem {
    float w1[2][kHidden][kIn];
    float b1[2][kHidden];
    float w2[7][kHidden];   // rows 0..2 translation, 3..6 rotation
    float b2[7];
};

__device__ void stage_weights(const Field &F, FieldSmem &s) {
    const int din = 2 * F.L;
    for (int e = threadIdx.x; e < 2 * kHidden * kIn; e += blockDim.x) {
        const int net = e / (kHidden * kIn), r = (e / kIn) % kHidden, c = e % kIn;
        s.w1[net][r][c] = c < din ? F.w1[net][r * din + c] : 0.f;
    }
    for (int e = threadIdx.x; e < 2 * kHidden; e += blockDim.x) s.b1[e / kHidden][e % kHidden] = F.b1[e / kHidden][e % kHidden];
    for (int e = threadIdx.x; e < 7 * kHidden; e += blockDim.x)
        s.w2[e / kHidden][e % kHidden] = e < 3 * kHidden ? F.w2[0][e] : F.w2[1][e - 3 * kHidden];
    if (threadIdx.x < 7) s.b2[threadIdx.x] = threadIdx.x < 3 ? F.b2[0][threadIdx.x] : F.b2[1][threadIdx.x - 3];
}

__device__ __forceinline__ uint32_t vertex_index(int i, int j, int k, int n_l, bool dense, uint32_t T) {
    if (dense) return (uint32_t)(i + (n_l + 1) * (j + (n_l + 1) * k));
    return ((uint32_t)i ^ ((uint32_t)j * 2654435761u) ^ ((uint32_t)k * 805459861u)) & (T - 1u);
}

// Normalised position (FP32, each operation rounded once, clamped to [0, 1]).
__device__ __forceinline__ void unit_pos(const Field &F, const float *mu, float x[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float v = __fdiv_rn(__fsub_rn(mu[a], F.lo[a]), __fsub_rn(F.hi[a], F.lo[a]));
        x[a] = fminf(fmaxf(v, 0.f), 1.f);
    }
}

// Cell and weights of level l.
__device__ __forceinline__ void level_cell(const Field &F, int l, const float x[3], int c[3], float w[3]) {
    const int n = F.res[l];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float p = __fmul_rn(x[a], (float)n);
        int ci = (int)floorf(p);
        ci = min(max(ci, 0), n - 1);
        c[a] = ci;
        w[a] = __fsub_rn(p, (float)ci);
    }
}

__device__ __forceinline__ bool level_dense(int n, int log2T) {
    const int64_t v = (int64_t)(n + 1) * (n + 1) * (n + 1);
    return v <= ((int64_t)1 << log2T);
}

__device__ __forceinline__ void encode(const Field &F, const float *mu, float h[kIn]) {
    float x[3];
    unit_pos(F, mu, x);
    const uint32_t T = 1u << F.log2T;
#pragma unroll
    for (int l = 0; l < kMaxLv; ++l) {
        float f0 = 0.f, f1 = 0.f;
        if (l < F.L) {
            int c[3];
            float w[3];
            level_cell(F, l, x, c, w);
            const bool dense = level_dense(F.res[l], F.log2T);
            const float2 *tab = reinterpret_cast<const float2 *>(F.table) + (size_t)l * T;
#pragma unroll
            for (int corner = 0; corner < 8; ++corner) {
                const int o0 = corner & 1, o1 = (corner >> 1) & 1, o2 = (corner >> 2) & 1;
                const float wt = (o0 ? w[0] : 1.f - w[0]) * (o1 ? w[1] : 1.f - w[1]) * (o2 ? w[2] : 1.f - w[2]);
                const float2 v = tab[vertex_index(c[0] + o0, c[1] + o1, c[2] + o2, F.res[l], dense, T)];
                f0 = fmaf(wt, v.x, f0);
                f1 = fmaf(wt, v.y, f1);
            }
        }
        h[2 * l] = f0;
        h[2 * l + 1] = f1;
    }
}

__global__ void __launch_bounds__(kFT) k_field_fwd(Field F, const float *__restrict__ means, int64_t n,
                                                   float *__restrict__ q, float *__restrict__ t) {
    __shared__ __align__(16) FieldSmem s;
    stage_weights(F, s);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float h[kIn];
    encode(F, mu, h);
    float o[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) o[c] = s.b2[c];
    for (int j = 0; j < kHidden; ++j) {
        float zt = s.b1[0][j], zr = s.b1[1][j];
#pragma unroll
        for (int k = 0; k < kIn; ++k) {
            zt = fmaf(s.w1[0][j][k], h[k], zt);
            zr = fmaf(s.w1[1][j][k], h[k], zr);
        }
        const float at = zt > 0.f ? zt : 0.f, ar = zr > 0.f ? zr : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = fmaf(s.w2[c][j], at, o[c]);
#pragma unroll
        for (int c = 3; c < 7; ++c) o[c] = fmaf(s.w2[c][j], ar, o[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) t[3 * i + c] = o[c];
    q[4 * i] = o[3] + 1.f;
#pragma unroll
    for (int c = 1; c < 4; ++c) q[4 * i + c] = o[3 + c];
}

// Backward.  Dynamic shared memory: H[kIn][kFT], A[kHidden][kFT], DZ[kHidden][kFT], DO[7][kFT].
constexpr size_t kBwdDyn = (size_t)(kIn + 2 * kHidden + 7) * kFT * 4;

__global__ void __launch_bounds__(kFT) k_field_bwd(Field F, const float *__restrict__ means, int64_t n,
                                                   const float *__restrict__ d_q, const float *__restrict__ d_t,
                                                   float *__restrict__ partial, float *__restrict__ d_table) {
    __shared__ __align__(16) FieldSmem s;
    extern __shared__ __align__(16) float dyn[];
    float *H = dyn, *A = H + kIn * kFT, *DZ = A + kHidden * kFT, *DO = DZ + kHidden * kFT;
    stage_weights(F, s);
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kFT + tid;
    const bool valid = i < n;
    float mu[3] = {0.f, 0.f, 0.f};
    float h[kIn], dout[7];
#pragma unroll
    for (int k = 0; k < kIn; ++k) h[k] = 0.f;
#pragma unroll
    for (int c = 0; c < 7; ++c) dout[c] = 0.f;
    if (valid) {
        for (int a = 0; a < 3; ++a) mu[a] = means[3 * i + a];
        encode(F, mu, h);
        for (int c = 0; c < 3; ++c) dout[c] = d_t[3 * i + c];
        for (int c = 0; c < 4; ++c) dout[3 + c] = d_q[4 * i + c];
    }
#pragma unroll
    for (int k = 0; k < kIn; ++k) H[k * kFT + tid] = h[k];
#pragma unroll
    for (int c = 0; c < 7; ++c) DO[c * kFT + tid] = dout[c];
    __syncthreads();
    float dh[kIn];
#pragma unroll
    for (int k = 0; k < kIn; ++k) dh[k] = 0.f;
    float *blk = partial + (size_t)blockIdx.x * kPartials;
    for (int net = 0; net < 2; ++net) {
        const int o0 = net ? 3 : 0, no = net ? 4 : 3;
        for (int j = 0; j < kHidden; ++j) {
            float z = s.b1[net][j];
#pragma unroll
            for (int k = 0; k < kIn; ++k) z = fmaf(s.w1[net][j][k], h[k], z);
            float da = 0.f;
            for (int c = 0; c < no; ++c) da = fmaf(s.w2[o0 + c][j], dout[o0 + c], da);
            const float dz = z > 0.f ? da : 0.f;
            A[j * kFT + tid] = z > 0.f ? z : 0.f;
            DZ[j * kFT + tid] = dz;
#pragma unroll
            for (int k = 0; k < kIn; ++k) dh[k] = fmaf(s.w1[net][j][k], dz, dh[k]);
        }
        __syncthreads();
        // this block's weight gradients of the net (rows of invalid threads are zero)
        float *P = blk + (net ? kNetOff1 : 0);
        for (int e = tid; e < kHidden * kIn; e += kFT) {
            const int j = e / kIn, k = e % kIn;
            const float4 *a4 = reinterpret_cast<const float4 *>(DZ + j * kFT);
            const float4 *b4 = reinterpret_cast<const float4 *>(H + k * kFT);
            float acc = 0.f;
            for (int r = 0; r < kFT / 4; ++r) {
                const float4 a = a4[r], b = b4[r];
                acc = fmaf(a.x, b.x, acc); acc = fmaf(a.y, b.y, acc); acc = fmaf(a.z, b.z, acc); acc = fmaf(a.w, b.w, acc);
            }
            P[e] = acc;
        }
        for (int j = tid; j < kHidden; j += kFT) {
            float acc = 0.f;
            for (int r = 0; r < kFT; ++r) acc += DZ[j * kFT + r];
            P[kHidden * kIn + j] = acc;
        }
        for (int e = tid; e < no * kHidden; e += kFT) {
            const int c = e / kHidden, j = e % kHidden;
            float acc = 0.f;
            for (int r = 0; r < kFT; ++r) acc = fmaf(DO[(o0 + c) * kFT + r], A[j * kFT + r], acc);
            P[kHidden * kIn + kHidden + e] = acc;
        }
        for (int c = tid; c < no; c += kFT) {
            float acc = 0.f;
            for (int r = 0; r < kFT; ++r) acc += DO[(o0 + c) * kFT + r];
            P[kHidden * kIn + kHidden + no * kHidden + c] = acc;
        }
        __syncthreads();
    }
    // table gradient: each corner's weight times the feature gradient
    if (valid && d_table) {
        float x[3];
        unit_pos(F, mu, x);
        const uint32_t T = 1u << F.log2T;
        for (int l = 0; l < F.L; ++l) {
            int c[3];
            float w[3];
            level_cell(F, l, x, c, w);
            const bool dense = level_dense(F.res[l], F.log2T);
            float2 *tab = reinterpret_cast<float2 *>(d_table) + (size_t)l * T;
            for (int corner = 0; corner < 8; ++corner) {
                const int o0 = corner & 1, o1 = (corner >> 1) & 1, o2 = (corner >> 2) & 1;
                const float wt = (o0 ? w[0] : 1.f - w[0]) * (o1 ? w[1] : 1.f - w[1]) * (o2 ? w[2] : 1.f - w[2]);
                const uint32_t idx = vertex_index(c[0] + o0, c[1] + o1, c[2] + o2, F.res[l], dense, T);
                atomicAdd(tab + idx, make_float2(wt * dh[2 * l], wt * dh[2 * l + 1]));  // one vector atomic
            }
        }
    }
}

struct FieldGrads {
    float *w1[2], *b1[2], *w2[2], *b2[2];
};

// Sum of the per-block partials in block order; one thread per parameter slot.
__global__ void k_field_reduce(const float *__restrict__ partial, int nblocks, int din, FieldGrads g) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kPartials) return;
    const int net = e >= kNetOff1 ? 1 : 0;
    int r = e - (net ? kNetOff1 : 0);
    const int no = net ? 4 : 3;
    float *dst = nullptr;
    if (r < kHidden * kIn) {
        const int j = r / kIn, k = r % kIn;
        if (k < din && g.w1[net]) dst = g.w1[net] + j * din + k;
    } else if ((r -= kHidden * kIn) < kHidden) {
        if (g.b1[net]) dst = g.b1[net] + r;
    } else if ((r -= kHidden) < no * kHidden) {
        if (g.w2[net]) dst = g.w2[net] + r;
    } else {
        r -= no * kHidden;
        if (g.b2[net]) dst = g.b2[net] + r;
    }
    if (!dst) return;
    float acc = 0.f;
    for (int b = 0; b < nblocks; ++b) acc += partial[(size_t)b * kPartials + e];
    *dst = acc;
}

gc_status make_field(gc_context *ctx, const gc_motion_field *f, Field &F) {
    if (!f) return fail(ctx, GC_ERR_INVALID_ARG, "field is NULL");
    if (f->n_levels < 1 || f->n_levels > kMaxLv) return fail(ctx, GC_ERR_INVALID_ARG, "n_levels must be 1..16");
    if (f->log2_table < 4 || f->log2_table > 26) return fail(ctx, GC_ERR_INVALID_ARG, "log2_table must be 4..26");
    if (!f->table || !f->w1t || !f->b1t || !f->w2t || !f->b2t || !f->w1r || !f->b1r || !f->w2r || !f->b2r)
        return fail(ctx, GC_ERR_INVALID_ARG, "a motion-source parameter array is NULL");
    if (reinterpret_cast<uintptr_t>(f->table) & 7) return fail(ctx, GC_ERR_INVALID_ARG, "table must be 8-byte aligned");
    memset(&F, 0, sizeof F);
    F.L = f->n_levels;
    F.log2T = f->log2_table;
    for (int l = 0; l < F.L; ++l) {
        if (f->resolution[l] < 1 || f->resolution[l] > (1 << 20))
            return fail(ctx, GC_ERR_INVALID_ARG, "resolution[%d] must be 1..2^20", l);
        F.res[l] = f->resolution[l];
    }
    for (int a = 0; a < 3; ++a) {
        if (!(f->hi[a] > f->lo[a])) return fail(ctx, GC_ERR_INVALID_ARG, "hi must exceed lo on every axis");
        F.lo[a] = f->lo[a];
        F.hi[a] = f->hi[a];
    }
    F.table = f->table;
    F.w1[0] = f->w1t; F.b1[0] = f->b1t; F.w2[0] = f->w2t; F.b2[0] = f->b2t;
    F.w1[1] = f->w1r; F.b1[1] = f->b1r; F.w2[1] = f->w2r; F.b2[1] = f->b2r;
    return GC_OK;
}

}  // namespace

}  // namespace gc

extern "C" gc_status gc_motion_field_forward(gc_context *ctx, const gc_motion_field *field, const float *means,
                                             int64_t n, float *q, float *t, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    gc::Field F;
    gc_status st = gc::make_field(ctx, field, F);
    if (st != GC_OK) return st;
    if (n < 0) return fail(ctx, GC_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return GC_OK;
    if (!means || !q || !t) return fail(ctx, GC_ERR_INVALID_ARG, "means, q or t is NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gc::k_field_fwd<<<(unsigned)((n + gc::kFT - 1) / gc::kFT), gc::kFT, 0, s>>>(F, means, n, q, t);
    gc::note_launches(1);
    GC_CUDA(ctx, cudaGetLastError());
    return GC_OK;
}

extern "C" gc_status gc_motion_field_backward(gc_context *ctx, const gc_motion_field *field, const float *means,
                                              int64_t n, const float *d_q, const float *d_t,
                                              gc_motion_field_grads *out, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    gc::Field F;
    gc_status st = gc::make_field(ctx, field, F);
    if (st != GC_OK) return st;
    if (!out) return fail(ctx, GC_ERR_INVALID_ARG, "grads is NULL");
    if (reinterpret_cast<uintptr_t>(out->table) & 7) return fail(ctx, GC_ERR_INVALID_ARG, "the table gradient must be 8-byte aligned");
    if (n < 0) return fail(ctx, GC_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!means || !d_q || !d_t)) return fail(ctx, GC_ERR_INVALID_ARG, "means, d_q or d_t is NULL");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int din = 2 * F.L;
    const size_t T = (size_t)1 << F.log2T;
    if (out->table) GC_CUDA(ctx, cudaMemsetAsync(out->table, 0, (size_t)F.L * T * 2 * 4, s));
    float *zero[] = {out->w1t, out->b1t, out->w2t, out->b2t, out->w1r, out->b1r, out->w2r, out->b2r};
    const size_t sizes[] = {(size_t)64 * din, 64, 3 * 64, 3, (size_t)64 * din, 64, 4 * 64, 4};
    if (n == 0) {
        for (int k = 0; k < 8; ++k)
            if (zero[k]) GC_CUDA(ctx, cudaMemsetAsync(zero[k], 0, sizes[k] * 4, s));
        return GC_OK;
    }
    const int nblocks = (int)((n + gc::kFT - 1) / gc::kFT);
    GC_CUDA(ctx, grow(ctx->field_part, (size_t)nblocks * gc::kPartials * 4));
    GC_CUDA(ctx, cudaFuncSetAttribute(gc::k_field_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)gc::kBwdDyn));
    gc::k_field_bwd<<<nblocks, gc::kFT, gc::kBwdDyn, s>>>(F, means, n, d_q, d_t, ctx->field_part.as<float>(),
                                                          out->table);
    gc::FieldGrads g{{out->w1t, out->w1r}, {out->b1t, out->b1r}, {out->w2t, out->w2r}, {out->b2t, out->b2r}};
    gc::k_field_reduce<<<(gc::kPartials + 255) / 256, 256, 0, s>>>(ctx->field_part.as<float>(), nblocks, din, g);
    gc::note_launches(2);
    GC_CUDA(ctx, cudaGetLastError());
    return GC_OK;
}
