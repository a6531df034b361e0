// gc_preprocess.cu - single-frame preprocess (one thread per selected Gaussian,
// projection in gc_project.cuh) and the gather of records into depth order.
#include <cuda_runtime.h>

#include "gc_project.cuh"

namespace gc {

namespace {

template <int PREC>
__global__ void __launch_bounds__(256) k_preprocess(GaussSrc G, Selection sel, int64_t n_sel,
                                                    CamParams cam, RenderParams rp,
                                                    float4 *__restrict__ rec,
                                                    uint32_t *__restrict__ depth_keys,
                                                    uint32_t *__restrict__ depth_vals,
                                                    uint32_t *__restrict__ touched) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_sel) return;
    const int64_t i = sel_global(sel, j);
    Proj P;
    project_gaussian<PREC>(G, i, G.group_q, G.group_t, G.n_groups, cam, rp, P, nullptr, G.res);
    rec[kRec * j] = P.r0;
    rec[kRec * j + 1] = P.r1;
    P.r2.y = __int_as_float(layer_of(sel, i));
    rec[kRec * j + 2] = P.r2;
    const uint32_t nt = bin_rows(P, rp, cam.width, cam.height);
    rec[kRec * j + 3] = P.r3;
    rec[kRec * j + 4] = P.r4;
    depth_keys[j] = P.key;
    depth_vals[j] = (uint32_t)j;
    touched[j] = nt;
}

__global__ void __launch_bounds__(256) k_rank_gather(const uint32_t *__restrict__ perm,
                                                     const float4 *__restrict__ rec,
                                                     const uint32_t *__restrict__ touched,
                                                     int64_t n, float4 *__restrict__ ranked,
                                                     uint32_t *__restrict__ touched_r) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const uint32_t j = perm[r];
#pragma unroll
    for (int k = 0; k < kRec; ++k) ranked[kRec * r + k] = rec[kRec * (int64_t)j + k];
    touched_r[r] = touched[j];
}

}  // namespace

cudaError_t launch_preprocess(const GaussSrc &g, const Selection &sel, int64_t n_sel,
                              const CamParams &cam, const RenderParams &rp, float4 *rec,
                              uint32_t *depth_keys, uint32_t *depth_vals, uint32_t *touched,
                              cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((n_sel + 255) / 256);
    GC_DISPATCH_PREC(g.precision, k_preprocess<PREC_><<<blocks, 256, 0, st>>>(
                                      g, sel, n_sel, cam, rp, rec, depth_keys, depth_vals, touched))
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rank_gather(const uint32_t *perm, const float4 *rec, const uint32_t *touched,
                               int64_t n, float4 *ranked, uint32_t *touched_r, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_rank_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(perm, rec, touched, n, ranked,
                                                              touched_r);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace gc
