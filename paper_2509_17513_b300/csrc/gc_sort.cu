// gc_sort.cu - exclusive scan and stable LSD radix sort of (uint32 key, uint32 value)
// pairs, written for sm_103a.
//
// Neither routine waits on another CTA: the scan is reduce-then-scan (three
// launches) and each radix digit is histogram -> scan -> scatter.  So no kernel
// can hang on a missing predecessor, and every result is deterministic.
//
// Scatter stability: each warp owns a contiguous 512-key segment of its CTA's
// 4096-key tile and ranks its keys row by row with __match_any_sync, so the
// global order of equal digits is (CTA, warp, row, lane) = input order.
#include <cuda_runtime.h>

#include "gc_internal.cuh"

namespace gc {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanRows = 16;
constexpr int kScanChunk = kScanThreads * kScanRows;  // 4096

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread across the CTA; returns the prefix,
// writes the CTA total to *total (all threads).
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_sums,
                                                         uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < THREADS / 32) ? warp_sums[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < THREADS / 32) warp_sums[lane] = wi - w;  // exclusive
        if (lane == THREADS / 32 - 1) warp_sums[32] = wi;
    }
    __syncthreads();
    uint32_t res = warp_sums[warp] + inc - x;
    *total = warp_sums[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in,
                                                              int64_t n,
                                                              uint32_t *__restrict__ partials) {
    __shared__ uint32_t red[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    uint32_t s = 0;
#pragma unroll 4
    for (int r = 0; r < kScanRows; ++r) {
        int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// One CTA scans the partials in chunks of 1024 with a running carry.
__global__ void __launch_bounds__(1024) k_scan_partials(uint32_t *partials, int64_t nb,
                                                        uint32_t *total) {
    __shared__ uint32_t ws[33];
    uint32_t carry = 0;
    for (int64_t b = 0; b < nb; b += 1024) {
        int64_t i = b + threadIdx.x;
        uint32_t x = (i < nb) ? partials[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan<1024>(x, ws, &tot);
        if (i < nb) partials[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *in, uint32_t *out,
                                                            int64_t n,
                                                            const uint32_t *__restrict__ partials) {
    __shared__ uint32_t ws[33];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    uint32_t carry = partials[blockIdx.x];
    for (int r = 0; r < kScanRows; ++r) {
        int64_t i = base + (int64_t)r * kScanThreads + threadIdx.x;
        uint32_t x = (i < n) ? in[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan<kScanThreads>(x, ws, &tot);
        if (i < n) out[i] = carry + ex;
        carry += tot;
    }
}

__device__ __forceinline__ int64_t device_count(const uint32_t *n_dev, int64_t n_max) {
    if (!n_dev) return n_max;
    int64_t n = (int64_t)(*n_dev);
    return n < n_max ? n : n_max;
}

// Per-CTA digit histogram, digit-major: counts[d * nblocks + b].
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ keys,
                                                             const uint32_t *n_dev, int64_t n_max,
                                                             int shift, uint32_t mask,
                                                             uint32_t *__restrict__ counts,
                                                             int nblocks) {
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n = device_count(n_dev, n_max);
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const uint32_t lt = lanemask_lt();
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
        bool valid = i < n;
        uint32_t d = valid ? ((keys[i] >> shift) & mask) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt) == 0) atomicAdd(&hist[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = hist[threadIdx.x];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const uint32_t *n_dev,
    int64_t n_max, int shift, uint32_t mask, const uint32_t *__restrict__ scanned, int nblocks) {
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t dstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t ws[33];
    __shared__ uint32_t skeys[kSortTile];
    __shared__ uint32_t svals[kSortTile];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = device_count(n_dev, n_max);
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    if (base >= n) return;
    const int nvalid = (int)((n - base) < kSortTile ? (n - base) : kSortTile);
    for (int k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wcnt[0][0])[k] = 0;
    __syncthreads();

    const uint32_t lt = lanemask_lt();
    uint32_t key[kSortItems], val[kSortItems], loc[kSortItems];
    const int64_t wbase = base + (int64_t)warp * (32 * kSortItems);
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = wbase + r * 32 + lane;
        bool valid = i < n;
        key[r] = valid ? keys_in[i] : 0u;
        val[r] = valid ? vals_in[i] : 0u;
        uint32_t d = valid ? ((key[r] >> shift) & mask) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
        loc[r] = before + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            uint32_t c = wcnt[w][d];
            wcnt[w][d] = s;
            s += c;
        }
        uint32_t tot;
        uint32_t st = block_exclusive_scan<kSortThreads>(s, ws, &tot);
        dstart[d] = st;
        gbase[d] = scanned[(int64_t)d * nblocks + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = wbase + r * 32 + lane;
        if (i < n) {
            uint32_t d = (key[r] >> shift) & mask;
            uint32_t pos = dstart[d] + wcnt[warp][d] + loc[r];
            skeys[pos] = key[r];
            svals[pos] = val[r];
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < nvalid; p += kSortThreads) {
        uint32_t k = skeys[p];
        uint32_t d = (k >> shift) & mask;
        uint32_t o = gbase[d] + (uint32_t)p - dstart[d];
        keys_out[o] = k;
        vals_out[o] = svals[p];
    }
}

}  // namespace

size_t scan_partials_size(int64_t n) { return (size_t)((n + kScanChunk - 1) / kScanChunk) + 1; }

cudaError_t launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                                  uint32_t *partials, cudaStream_t st) {
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, partials);
    note_launches(1);
    k_scan_partials<<<1, 1024, 0, st>>>(partials, nb, total);
    note_launches(1);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, partials);
    note_launches(1);
    return cudaGetLastError();
}

size_t radix_scratch_words(int64_t n_max) {
    int64_t nb = (n_max + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    return (size_t)(256 * nb) + scan_partials_size(256 * nb);
}

cudaError_t radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max,
                             const uint32_t *n_dev, int end_bit, uint32_t *scratch, int *out_buf,
                             cudaStream_t st) {
    int cur = 0;
    if (n_max <= 0 || end_bit <= 0) {
        *out_buf = 0;
        return cudaSuccess;
    }
    int nblocks = (int)((n_max + kSortTile - 1) / kSortTile);
    uint32_t *counts = scratch;
    uint32_t *partials = scratch + (size_t)256 * nblocks;
    for (int shift = 0; shift < end_bit; shift += 8) {
        int bits = end_bit - shift < 8 ? end_bit - shift : 8;
        uint32_t mask = (1u << bits) - 1u;
        k_radix_hist<<<nblocks, kSortThreads, 0, st>>>(keys[cur], n_dev, n_max, shift, mask, counts,
                                                       nblocks);
        note_launches(1);
        cudaError_t e = launch_exclusive_scan(counts, counts, (int64_t)256 * nblocks, nullptr,
                                              partials, st);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<nblocks, kSortThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                          vals[cur ^ 1], n_dev, n_max, shift, mask,
                                                          counts, nblocks);
        note_launches(1);
        cur ^= 1;
    }
    *out_buf = cur;
    return cudaGetLastError();
}

}  // namespace gc
