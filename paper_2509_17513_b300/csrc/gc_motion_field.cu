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
// Backward: persistent blocks; per chunk of 128 Gaussians the encodings, hidden activations
// and their gradients are staged in shared memory, the weight gradients accumulated in
// registers over the block's chunks and the per-block sums added over the blocks in block
// order by a second kernel (deterministic).  The table gradient is scattered with atomic
// additions.
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

// hrows: NULL, or the encodings to keep for the backward (kIn floats per Gaussian, as written
// by k_field_encode).
__global__ void __launch_bounds__(kFT) k_field_fwd(Field F, const float *__restrict__ means, int64_t n,
                                                   float *__restrict__ q, float *__restrict__ t,
                                                   float4 *__restrict__ hrows) {
    __shared__ __align__(16) FieldSmem s;
    stage_weights(F, s);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float h[kIn];
    encode(F, mu, h);
    if (hrows) {
        float4 *row = hrows + (size_t)i * (kIn / 4);
#pragma unroll
        for (int q4 = 0; q4 < kIn / 4; ++q4)
            row[q4] = make_float4(h[4 * q4], h[4 * q4 + 1], h[4 * q4 + 2], h[4 * q4 + 3]);
    }
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

// Backward, first pass: the hash-grid encoding of every Gaussian, kIn floats per row (levels
// beyond F.L zero).  Its table gathers are latency-bound; this kernel keeps many warps per SM
// to hide them, which the backward proper (large shared rows) cannot.
__global__ void __launch_bounds__(kFT) k_field_encode(Field F, const float *__restrict__ means, int64_t n,
                                                      float4 *__restrict__ hrows) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    float h[kIn];
    encode(F, mu, h);
    float4 *row = hrows + (size_t)i * (kIn / 4);
#pragma unroll
    for (int q4 = 0; q4 < kIn / 4; ++q4) row[q4] = make_float4(h[4 * q4], h[4 * q4 + 1], h[4 * q4 + 2], h[4 * q4 + 3]);
}

// Backward, persistent: block b takes the chunks of kFT Gaussians c = b, b + grid, ... in
// order.  Per chunk the block copies the chunk's encodings (from k_field_encode) into padded
// shared rows, each thread recomputes its Gaussian's hidden layers and stages one padded row
// per Gaussian in shared memory (encoding, output gradient, hidden
// activation, hidden pre-activation gradient; row pitches chosen so that 16-byte row accesses
// of eight consecutive threads fall on distinct banks).  The weight gradients are sums over
// the Gaussians of outer products; each thread accumulates, in registers and over all of its
// block's chunks, a 4 x 4 tile of dW1 per net and one column of dW2 / db1 (and one entry of
// db2).  Each block writes one partial vector at the end, summed over the blocks in block
// order by k_field_reduce, so the weight gradients are reproducible bit for bit for a given n.
// The table gradient is scattered with atomic additions.
// 16-byte global -> shared copy that completes asynchronously (src_bytes 0: zero fill).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, uint32_t src_bytes) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int kHP = kIn + 4;       // 36 floats: row pitch of the encodings
constexpr int kOP = 8;             // row pitch of the output gradients (7 used)
constexpr int kAP = kHidden + 4;   // 68 floats: row pitch of the hidden rows
constexpr size_t kBwdDyn = (size_t)kFT * (kHP + kOP + 2 * kAP) * 4;
constexpr int kBwdBlocksPerSm = 2;
constexpr int kBwdGrid = 148 * kBwdBlocksPerSm;

__global__ void __launch_bounds__(kFT, kBwdBlocksPerSm) k_field_bwd(
    Field F, const float *__restrict__ means, const float4 *__restrict__ hrows, int64_t n,
    const float *__restrict__ d_q, const float *__restrict__ d_t, float *__restrict__ partial,
    float *__restrict__ d_table) {
    __shared__ __align__(16) FieldSmem s;
    extern __shared__ __align__(16) float dyn[];
    float *HT = dyn, *DOT = HT + kFT * kHP, *AT = DOT + kFT * kOP, *DZT = AT + kFT * kAP;
    stage_weights(F, s);
    const int tid = threadIdx.x;
    const int tj = tid >> 3, tk = tid & 7;    // dW1 tile: rows 4 tj .. 4 tj + 3, columns 4 tk .. 4 tk + 3
    const int cj = tid & 63, ch = tid >> 6;  // dW2 column j = cj, outputs 2 ch and 2 ch + 1; db1 (ch = 0)
    float g1[2][4][4], g2[2][2], gb1[2], gb2 = 0.f;
#pragma unroll
    for (int net = 0; net < 2; ++net) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) g1[net][a][b] = 0.f;
        g2[net][0] = g2[net][1] = gb1[net] = 0.f;
    }
    const int64_t nchunks = (n + kFT - 1) / kFT;
    // A chunk's inputs: its encodings into the padded shared rows by asynchronous copies (zero
    // rows past n), its means and output gradients into registers.  The next chunk's are
    // fetched before this chunk's table atomics are issued, so they do not queue behind them.
    auto fetch = [&](int64_t ch, float *mu_n, float *dout_n) {
        const int64_t row0 = ch * kFT;
#pragma unroll
        for (int e = tid; e < kFT * (kIn / 4); e += kFT) {
            const int r = e / (kIn / 4), q4 = e % (kIn / 4);
            const bool in = row0 + r < n;
            cp_async16(HT + r * kHP + 4 * q4, hrows + (in ? (size_t)(row0 + r) * (kIn / 4) + q4 : 0), in ? 16u : 0u);
        }
        cp_async_commit();
        const int64_t i = ch * kFT + tid;
#pragma unroll
        for (int a = 0; a < 3; ++a) mu_n[a] = 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) dout_n[c] = 0.f;
        if (i < n) {
            for (int a = 0; a < 3; ++a) mu_n[a] = means[3 * i + a];
            for (int c = 0; c < 3; ++c) dout_n[c] = d_t[3 * i + c];
            for (int c = 0; c < 4; ++c) dout_n[3 + c] = d_q[4 * i + c];
        }
    };
    float mu[3], dout[8];
    if ((int64_t)blockIdx.x < nchunks) fetch(blockIdx.x, mu, dout);
    for (int64_t chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int64_t i = chunk * kFT + tid;
        const bool valid = i < n;
        float h[kIn];
        cp_async_wait_all();
        {
            float4 *orow = reinterpret_cast<float4 *>(DOT + tid * kOP);
            orow[0] = make_float4(dout[0], dout[1], dout[2], dout[3]);
            orow[1] = make_float4(dout[4], dout[5], dout[6], 0.f);
        }
        __syncthreads();  // the chunk's encodings and output gradients are in shared memory
        {
            const float4 *hr = reinterpret_cast<const float4 *>(HT + tid * kHP);
#pragma unroll
            for (int q4 = 0; q4 < kIn / 4; ++q4) {
                const float4 v = hr[q4];
                h[4 * q4] = v.x;
                h[4 * q4 + 1] = v.y;
                h[4 * q4 + 2] = v.z;
                h[4 * q4 + 3] = v.w;
            }
        }
        float dh[kIn];
#pragma unroll
        for (int k = 0; k < kIn; ++k) dh[k] = 0.f;
#pragma unroll
        for (int net = 0; net < 2; ++net) {
            const int o0 = net ? 3 : 0, no = net ? 4 : 3;
            if (net) __syncthreads();  // net 0's readers of the hidden rows are done
            for (int j0 = 0; j0 < kHidden; j0 += 4) {
                float av[4], dz[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u;
                    float z = s.b1[net][j];
#pragma unroll
                    for (int k = 0; k < kIn; ++k) z = fmaf(s.w1[net][j][k], h[k], z);
                    float da = 0.f;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (c < no) da = fmaf(s.w2[o0 + c][j], dout[o0 + c], da);
                    dz[u] = z > 0.f ? da : 0.f;
                    av[u] = z > 0.f ? z : 0.f;
                }
                *reinterpret_cast<float4 *>(AT + tid * kAP + j0) = make_float4(av[0], av[1], av[2], av[3]);
                *reinterpret_cast<float4 *>(DZT + tid * kAP + j0) = make_float4(dz[0], dz[1], dz[2], dz[3]);
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int k = 0; k < kIn; ++k) dh[k] = fmaf(s.w1[net][j0 + u][k], dz[u], dh[k]);
            }
            __syncthreads();
            // dW1[j][k] += sum over the chunk's Gaussians r of DZ[r][j] H[r][k]
#pragma unroll 4
            for (int r = 0; r < kFT; ++r) {
                const float4 d4 = *reinterpret_cast<const float4 *>(DZT + r * kAP + 4 * tj);
                const float4 h4 = *reinterpret_cast<const float4 *>(HT + r * kHP + 4 * tk);
                const float dv[4] = {d4.x, d4.y, d4.z, d4.w}, hv[4] = {h4.x, h4.y, h4.z, h4.w};
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) g1[net][a][b] = fmaf(dv[a], hv[b], g1[net][a][b]);
            }
            // dW2[c][j] += DO[r][c] A[r][j]; db1[j] += DZ[r][j]; db2[c] += DO[r][c]
            if (ch == 0) {
#pragma unroll 4
                for (int r = 0; r < kFT; ++r) {
                    const float a = AT[r * kAP + cj];
                    g2[net][0] = fmaf(DOT[r * kOP + o0], a, g2[net][0]);
                    g2[net][1] = fmaf(DOT[r * kOP + o0 + 1], a, g2[net][1]);
                    gb1[net] += DZT[r * kAP + cj];
                }
            } else {
#pragma unroll 4
                for (int r = 0; r < kFT; ++r) {
                    const float a = AT[r * kAP + cj];
                    g2[net][0] = fmaf(DOT[r * kOP + o0 + 2], a, g2[net][0]);
                    if (no == 4) g2[net][1] = fmaf(DOT[r * kOP + o0 + 3], a, g2[net][1]);
                }
            }
            if (net == 0 && tid < 7)
                for (int r = 0; r < kFT; ++r) gb2 += DOT[r * kOP + tid];
        }
        __syncthreads();  // every reader of this chunk's shared rows is done
        const float mu_c[3] = {mu[0], mu[1], mu[2]};
        if (chunk + (int64_t)gridDim.x < nchunks) fetch(chunk + gridDim.x, mu, dout);
        // table gradient: each corner's weight times the feature gradient
        if (valid && d_table) {
            float x[3];
            unit_pos(F, mu_c, x);
            const uint32_t T = 1u << F.log2T;
#pragma unroll
            for (int l = 0; l < kMaxLv; ++l) {
                if (l >= F.L) break;
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
    // this block's partial: per net w1 (kHidden x kIn), b1, w2 (no x kHidden), b2
    float *blk = partial + (size_t)blockIdx.x * kPartials;
#pragma unroll
    for (int net = 0; net < 2; ++net) {
        const int no = net ? 4 : 3;
        float *P = blk + (net ? kNetOff1 : 0);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) P[(4 * tj + a) * kIn + 4 * tk + b] = g1[net][a][b];
        if (ch == 0) P[kHidden * kIn + cj] = gb1[net];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int c = 2 * ch + u;
            if (c < no) P[kHidden * kIn + kHidden + c * kHidden + cj] = g2[net][u];
        }
    }
    if (tid < 7) {
        const int net = tid < 3 ? 0 : 1, c = tid < 3 ? tid : tid - 3, no = net ? 4 : 3;
        blk[(net ? kNetOff1 : 0) + kHidden * kIn + kHidden + no * kHidden + c] = gb2;
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

static gc_status field_forward(gc_context *ctx, const gc_motion_field *field, const float *means, int64_t n,
                               float *q, float *t, float *encodings, void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    gc::Field F;
    gc_status st = gc::make_field(ctx, field, F);
    if (st != GC_OK) return st;
    if (n < 0) return fail(ctx, GC_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return GC_OK;
    if (!means || !q || !t) return fail(ctx, GC_ERR_INVALID_ARG, "means, q or t is NULL");
    if (reinterpret_cast<uintptr_t>(encodings) & 15) return fail(ctx, GC_ERR_INVALID_ARG, "encodings must be 16-byte aligned");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    gc::k_field_fwd<<<(unsigned)((n + gc::kFT - 1) / gc::kFT), gc::kFT, 0, s>>>(F, means, n, q, t,
                                                                              reinterpret_cast<float4 *>(encodings));
    gc::note_launches(1);
    GC_CUDA(ctx, cudaGetLastError());
    return GC_OK;
}

extern "C" gc_status gc_motion_field_forward(gc_context *ctx, const gc_motion_field *field, const float *means,
                                             int64_t n, float *q, float *t, void *stream) {
    return field_forward(ctx, field, means, n, q, t, nullptr, stream);
}

extern "C" gc_status gc_motion_field_forward_save(gc_context *ctx, const gc_motion_field *field, const float *means,
                                                  int64_t n, float *q, float *t, float *encodings, void *stream) {
    if (ctx && !encodings) return fail(ctx, GC_ERR_INVALID_ARG, "encodings is NULL");
    return field_forward(ctx, field, means, n, q, t, encodings, stream);
}

static gc_status field_backward(gc_context *ctx, const gc_motion_field *field, const float *means, int64_t n,
                                const float *encodings, const float *d_q, const float *d_t,
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
    const int64_t nchunks = (n + gc::kFT - 1) / gc::kFT;
    const int nblocks = (int)std::min<int64_t>(nchunks, gc::kBwdGrid);
    GC_CUDA(ctx, grow(ctx->field_part, (size_t)nblocks * gc::kPartials * 4));
    GC_CUDA(ctx, cudaFuncSetAttribute(gc::k_field_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)gc::kBwdDyn));
    const float4 *hrows = reinterpret_cast<const float4 *>(encodings);
    if (!hrows) {  // recompute the encodings (latency-bound table gathers)
        GC_CUDA(ctx, grow(ctx->field_h, (size_t)n * gc::kIn * 4));
        gc::k_field_encode<<<(unsigned)nchunks, gc::kFT, 0, s>>>(F, means, n, ctx->field_h.as<float4>());
        gc::note_launches(1);
        hrows = ctx->field_h.as<float4>();
    }
    gc::k_field_bwd<<<nblocks, gc::kFT, gc::kBwdDyn, s>>>(F, means, hrows, n, d_q, d_t,
                                                          ctx->field_part.as<float>(), out->table);
    gc::FieldGrads g{{out->w1t, out->w1r}, {out->b1t, out->b1r}, {out->w2t, out->w2r}, {out->b2t, out->b2r}};
    gc::k_field_reduce<<<(gc::kPartials + 255) / 256, 256, 0, s>>>(ctx->field_part.as<float>(), nblocks, din, g);
    gc::note_launches(2);
    GC_CUDA(ctx, cudaGetLastError());
    return GC_OK;
}

extern "C" gc_status gc_motion_field_backward(gc_context *ctx, const gc_motion_field *field, const float *means,
                                              int64_t n, const float *d_q, const float *d_t,
                                              gc_motion_field_grads *out, void *stream) {
    return field_backward(ctx, field, means, n, nullptr, d_q, d_t, out, stream);
}

extern "C" gc_status gc_motion_field_backward_saved(gc_context *ctx, const gc_motion_field *field,
                                                    const float *means, int64_t n, const float *encodings,
                                                    const float *d_q, const float *d_t, gc_motion_field_grads *out,
                                                    void *stream) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (n > 0 && !encodings) return fail(ctx, GC_ERR_INVALID_ARG, "encodings is NULL");
    if (reinterpret_cast<uintptr_t>(encodings) & 15) return fail(ctx, GC_ERR_INVALID_ARG, "encodings must be 16-byte aligned");
    return field_backward(ctx, field, means, n, encodings, d_q, d_t, out, stream);
}
