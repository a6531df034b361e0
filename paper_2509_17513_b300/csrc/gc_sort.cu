// gc_sort.cu - exclusive scan and stable LSD radix sort of (uint32 key, uint32 value)
// pairs, written for sm_103a.
//
// Two radix sorts share the tile ranking:
//  * one-sweep (unsegmented sorts of up to 2^21 keys): one histogram kernel counts the digits of every pass
//    in one read of the keys, then each pass is a single scatter launch in which a CTA
//    takes the next tile from a ticket counter, publishes its digit counts and finds its
//    global offsets by decoupled look-back over the tiles before it.  A CTA waits only on
//    tiles with smaller tickets, which were taken by CTAs already running and which
//    publish their counts before they wait themselves, so the waits always end; each is
//    still bounded, and a wait that runs out sets the error word.
//  * histogram -> scan -> scatter per digit (longer sorts, and the segmented sorts of the
//    batched path, whose segments need per-segment offsets), where no CTA waits on another.
// The scan is one chained pass (decoupled look-back), or one CTA for short inputs.
//
// Scatter stability: each warp owns a contiguous segment of its CTA's tile
// (kSortItems rows of 32 keys) and ranks its keys row by row (ballot multisplit),
// so the global order of equal digits is (tile, warp, row, lane) = input order.
#include <cuda_runtime.h>

#include <algorithm>

#include "gc_async.cuh"
#include "gc_internal.cuh"

namespace gc {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanChunk = kScanThreads * 16;  // 4096, 16 contiguous elements per thread

#ifndef GC_KEYS_MINB
#define GC_KEYS_MINB 3  // CTAs per SM of the keys-only scatter (80 registers, 75 KB of shared memory)
#endif
#ifndef GC_SORT_ITEMS
#define GC_SORT_ITEMS 8  // keys per thread in a radix tile
#endif
constexpr int kSortThreads = 256;
constexpr int kSortItems = GC_SORT_ITEMS;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048: sorts of (key, value) pairs
// keys-only sorts (the column pass of the row-binned lists) take four times the keys per
// tile: a quarter of the per-tile work (digit scan, offsets, barriers) per key and four times
// the length of the runs written per digit.  Measured on B300 (column pass of 180 batched
// 1080p renders): 2,048 keys 10.45 ms, 4,096 8.18, 6,144 8.00, 8,192 7.40, 12,288 7.47,
// 16,384 9.05 (occupancy falls to one CTA per SM).
#ifndef GC_KEYS_ITEMS
#define GC_KEYS_ITEMS (4 * GC_SORT_ITEMS)
#endif
constexpr int kKeysItems = GC_KEYS_ITEMS;
constexpr int kKeysTile = kSortThreads * kKeysItems;  // 8192
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

// Thread-contiguous chunk layout: thread t of a chunk owns elements
// [16 t, 16 t + 16), read with 16-byte loads when the chunk is full and aligned.
__device__ __forceinline__ void load16(const uint32_t *in, int64_t start, int64_t n, bool vec,
                                       uint32_t *x) {
    if (vec && start + 16 <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(in + start);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = p[q];
            x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = (start + q < n) ? in[start + q] : 0u;
    }
}

__device__ __forceinline__ void store16(uint32_t *out, int64_t start, int64_t n, bool vec,
                                        const uint32_t *x) {
    if (vec && start + 16 <= n) {
        uint4 *p = reinterpret_cast<uint4 *>(out + start);
#pragma unroll
        for (int q = 0; q < 4; ++q) p[q] = make_uint4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (start + q < n) out[start + q] = x[q];
    }
}

// Whole scan in one CTA of 1024 threads for n <= kSmallScan: chunks of 16384
// elements, 16 contiguous per thread (16-byte loads), one block scan per chunk.
constexpr int64_t kSmallScan = 1024 * 16 * 8;

__global__ void __launch_bounds__(1024) k_scan_single(const uint32_t *in, uint32_t *out, int64_t n,
                                                      bool vec, uint32_t *total) {
    __shared__ uint32_t ws[33];
    uint32_t carry = 0;
    for (int64_t base = 0; base < n; base += 16 * 1024) {
        const int64_t start = base + 16 * (int64_t)threadIdx.x;
        uint32_t x[16];
        load16(in, start, n, vec, x);
        uint32_t s = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const uint32_t v = x[q];
            x[q] = s;
            s += v;
        }
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan<1024>(s, ws, &tot) + carry;
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] += ex;
        store16(out, start, n, vec, x);
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// Single-pass chained scan for n > kSmallScan: CTAs take chunks of kScanChunk by ticket,
// scan them, publish the chunk's sum (flag 1) and, once the sum of every chunk before it is
// known, the inclusive prefix (flag 2): one warp looks back over 32 predecessors per round
// trip, adding sums until it meets an inclusive prefix.  A chunk waits only on chunks with
// smaller tickets, taken by CTAs already running, so every wait ends; each is still bounded
// and a wait that runs out sets the error word.  status (one 64-bit word per chunk, flag in
// the high half) and the ticket must be zero before the launch.
constexpr uint32_t kScanWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kScanThreads) k_scan_onepass(const uint32_t *in, uint32_t *out, int64_t n,
                                                               bool vec, uint32_t *ticket,
                                                               unsigned long long *status, uint32_t *total,
                                                               uint32_t *err) {
    __shared__ uint32_t ws[33];
    __shared__ uint32_t s_chunk, s_excl;
    if (threadIdx.x == 0) s_chunk = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t c = (int64_t)s_chunk;
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (c >= nb) return;  // CTA-uniform
    const int64_t start = c * kScanChunk + 16 * (int64_t)threadIdx.x;
    uint32_t x[16];
    load16(in, start, n, vec, x);
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint32_t v = x[q];
        x[q] = s;
        s += v;
    }
    uint32_t agg;
    const uint32_t ex = block_exclusive_scan<kScanThreads>(s, ws, &agg);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        uint32_t excl = 0u;
        if (c == 0) {
            if (lane == 0) st_relaxed64(&status[0], (2ull << 32) | agg);
        } else {
            if (lane == 0) st_relaxed64(&status[c], (1ull << 32) | agg);
            int64_t q = c - 1;
            for (;;) {
                const int64_t idx = q - lane;
                unsigned long long v = idx >= 0 ? ld_relaxed64(&status[idx]) : (2ull << 32);
                for (uint32_t it = 0; (v >> 32) == 0ull; ++it) {
                    if (it >= kScanWaitLimit) {
                        atomicOr(err, kErrTimeout);
                        v = 2ull << 32;
                        break;
                    }
                    v = ld_relaxed64(&status[idx]);
                }
                const uint32_t inc = __ballot_sync(0xffffffffu, (v >> 32) == 2ull);
                const uint32_t upto = inc ? (2u << (__ffs(inc) - 1)) - 1u : 0xffffffffu;  // lanes 0..first inclusive
                uint32_t part = ((upto >> lane) & 1u) ? (uint32_t)v : 0u;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                excl += part;
                if (inc) break;
                q -= 32;
            }
            if (lane == 0) st_relaxed64(&status[c], (2ull << 32) | (excl + agg));
        }
        if (lane == 0) {
            s_excl = excl;
            if (c == nb - 1 && total) *total = excl + agg;
        }
    }
    __syncthreads();
    const uint32_t base = s_excl + ex;
#pragma unroll
    for (int q = 0; q < 16; ++q) x[q] += base;
    store16(out, start, n, vec, x);
}

__device__ __forceinline__ int64_t device_count(const uint32_t *n_dev, int64_t n_max) {
    if (!n_dev) return n_max;
    int64_t n = (int64_t)(*n_dev);
    return n < n_max ? n : n_max;
}

// Index of (digit d, block b) in the histogram array: base + d * stride.  Without segments
// the layout is digit-major over all blocks (base b, stride nblocks).  With segments
// (seg_block0: S+1 nondecreasing block indices, segment s = blocks [seg_block0[s],
// seg_block0[s+1])), each segment owns a contiguous digit-major region in segment order, so
// one exclusive scan over the array yields offsets that keep every segment within its own
// range: block b of the segment starting at b0 with nb blocks has base 256 b0 + (b - b0) and
// stride nb, read from the per-block table blk (k_block_segments); blocks past the last
// segment hold zero counts after all segments (base 256 b, stride 1).  Both loads are
// independent, so a block pays one memory round trip for its index.
struct SegIndex {
    const uint32_t *seg_block0;  // NULL: unsegmented
    const uint2 *blk;
    int n_seg;
};

__device__ __forceinline__ uint2 count_index(int b, int nblocks, const SegIndex &sg) {
    if (!sg.seg_block0) return make_uint2((uint32_t)b, (uint32_t)nblocks);
    const int total = (int)sg.seg_block0[sg.n_seg];
    const uint2 e = sg.blk[b];  // the table has a word pair for every block (unset past the last segment)
    return b < total ? e : make_uint2(256u * (uint32_t)b, 1u);
}

// The per-block table of a segmented sort: CTA s writes (base, stride) of every block of
// segment s.
__global__ void __launch_bounds__(128) k_block_segments(const uint32_t *__restrict__ seg_block0,
                                                        uint2 *__restrict__ blk) {
    const uint32_t b0 = seg_block0[blockIdx.x], nb = seg_block0[blockIdx.x + 1] - b0;
    for (uint32_t i = threadIdx.x; i < nb; i += 128) blk[b0 + i] = make_uint2(256u * b0 + i, nb);
}

// Peers of this lane: the lanes of the warp whose digit equals this lane's, among the
// lanes in `valid` (warp multisplit by one ballot per digit bit).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, int bits, uint32_t valid) {
    uint32_t peers = valid;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        if (b < bits) {
            const uint32_t bit = (d >> b) & 1u;
            const uint32_t t = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? t : ~t;
        }
    }
    return peers;
}

// The same for 8-bit digits (the bit count known at compile time).
__device__ __forceinline__ uint32_t digit_peers8(uint32_t d, uint32_t valid) {
    uint32_t peers = valid;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t t = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? t : ~t;
    }
    return peers;
}

// Per-CTA digit histogram, digit-major: counts[d * nblocks + b].  Keys are read with
// 16-byte loads when the tile is full; each warp counts into its own shared row.
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t *__restrict__ keys,
                                                             const uint32_t *n_dev, int64_t n_max,
                                                             int shift, uint32_t mask,
                                                             uint32_t *__restrict__ counts,
                                                             int nblocks, SegIndex sg) {
    __shared__ uint32_t wh[kWarps][256];
    const int warp = threadIdx.x >> 5;
    const uint2 ci = count_index((int)blockIdx.x, nblocks, sg);  // in flight while the keys load
    for (int k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wh[0][0])[k] = 0;
    __syncthreads();
    const int64_t n = device_count(n_dev, n_max);
    constexpr int kTile = kSortThreads * ITEMS;
    const int64_t base = (int64_t)blockIdx.x * kTile;
    if (base + kTile <= n) {
        const uint4 *k4 = reinterpret_cast<const uint4 *>(keys + base);
#pragma unroll
        for (int r = 0; r < ITEMS / 4; ++r) {
            const uint4 q = k4[r * kSortThreads + threadIdx.x];
            atomicAdd(&wh[warp][(q.x >> shift) & mask], 1u);
            atomicAdd(&wh[warp][(q.y >> shift) & mask], 1u);
            atomicAdd(&wh[warp][(q.z >> shift) & mask], 1u);
            atomicAdd(&wh[warp][(q.w >> shift) & mask], 1u);
        }
    } else {
        for (int r = 0; r < ITEMS; ++r) {
            const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
            if (i < n) atomicAdd(&wh[warp][(keys[i] >> shift) & mask], 1u);
        }
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tot += wh[w][threadIdx.x];
    counts[ci.x + threadIdx.x * ci.y] = tot;
}

// Stable scatter, persistent: each CTA walks tiles t = blockIdx.x, + gridDim.x, ...
// A tile's keys and values arrive in shared memory by two bulk asynchronous copies
// (cp.async.bulk, completed on an mbarrier), double-buffered so the next tile streams
// in while this one is ranked.  Every warp ranks its contiguous 256-key segment row by
// row (match.any or ballot multisplit), the CTA turns warp counts into each warp's tile
// positions per digit, places the (key, value) pairs digit-sorted back into the tile's
// buffer as 8-byte pairs and writes them out in contiguous runs.  keys_out may be NULL
// (last pass of a sort whose keys are not kept).  Without kPairs the keys alone are moved
// (vals_in and vals_out unused; half the shared staging).
template <bool kPairs, int ITEMS>
__global__ void __launch_bounds__(kSortThreads, kPairs ? 5 : GC_KEYS_MINB) k_radix_scatter(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const uint32_t *n_dev,
    int64_t n_max, int shift, uint32_t mask, const uint32_t *__restrict__ scanned, int nblocks,
    uint32_t *err, SegIndex sg) {
    constexpr int kTile = kSortThreads * ITEMS;
    // per stage: keys, values (then key-value pairs); keys only without kPairs
    __shared__ __align__(128) uint32_t skv[2][kPairs ? 2 : 1][kTile];
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t ws[33];
    __shared__ __align__(8) uint64_t bar[2];

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = device_count(n_dev, n_max);
    const int ntiles = (int)((n + kTile - 1) / kTile);
    const int bits = __popc(mask);
    const uint32_t lt = lanemask_lt();
    if ((int)blockIdx.x >= ntiles) return;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int t, int stage) {  // one thread
        const int64_t base = (int64_t)t * kTile;
        const int nv = (int)((n - base) < kTile ? (n - base) : kTile);
        const uint32_t bytes = (uint32_t)((nv * 4 + 15) & ~15);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bar[stage], (kPairs ? 2 : 1) * bytes);
        bulk_copy_g2s(skv[stage][0], keys_in + base, bytes, &bar[stage]);
        if (kPairs) bulk_copy_g2s(skv[stage][kPairs ? 1 : 0], vals_in + base, bytes, &bar[stage]);
    };
    if (threadIdx.x == 0) issue(blockIdx.x, 0);

    int it = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int stage = it & 1;
        const int64_t base = (int64_t)t * kTile;
        const int nvalid = (int)((n - base) < kTile ? (n - base) : kTile);
        const bool has_next = t + (int)gridDim.x < ntiles;
        if (threadIdx.x == 0 && has_next) issue(t + gridDim.x, stage ^ 1);
        const uint2 ci = count_index(t, nblocks, sg);  // in flight while the tile is ranked
        for (int k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wcnt[0][0])[k] = 0;
        const bool ok = mbar_wait_bounded(&bar[stage], (uint32_t)(it >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            // a copy did not complete in time: record it, let in-flight copies land, leave
            if (threadIdx.x == 0) {
                atomicOr(err, kErrTimeout);
                mbar_wait_bounded(&bar[stage], (uint32_t)(it >> 1) & 1u);
                if (has_next) mbar_wait_bounded(&bar[stage ^ 1], (uint32_t)((it + 1) >> 1) & 1u);
            }
            __syncthreads();
            return;
        }
        uint32_t key[ITEMS], val[ITEMS], loc[ITEMS];
        const int wseg = warp * (32 * ITEMS);
        if (nvalid == kTile && bits == 8) {
            // full tile of 8-bit digits (every key valid, the bit count fixed): the common case
#pragma unroll
            for (int r = 0; r < ITEMS; ++r) {
                const int li = wseg + r * 32 + lane;
                key[r] = skv[stage][0][li];
                if (kPairs) val[r] = skv[stage][kPairs ? 1 : 0][li];
                const uint32_t d = (key[r] >> shift) & 0xffu;
                const uint32_t peers = digit_peers8(d, 0xffffffffu);
                const uint32_t before = wcnt[warp][d];
                __syncwarp();
                if ((peers & lt) == 0) wcnt[warp][d] = before + (uint32_t)__popc(peers);
                __syncwarp();
                loc[r] = before + (uint32_t)__popc(peers & lt);
            }
        } else {
#pragma unroll
            for (int r = 0; r < ITEMS; ++r) {
                const int li = wseg + r * 32 + lane;
                const bool valid = li < nvalid;
                key[r] = valid ? skv[stage][0][li] : 0xffffffffu;
                if (kPairs) val[r] = valid ? skv[stage][kPairs ? 1 : 0][li] : 0u;
                const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
                const uint32_t d = (key[r] >> shift) & mask;
                // narrow digits: one match instruction; 8-bit digits: ballots per digit bit
                const uint32_t peers =
                    bits < 8 ? __match_any_sync(0xffffffffu, d) & vmask : digit_peers(d, bits, vmask);
                const uint32_t before = valid ? wcnt[warp][d] : 0u;
                __syncwarp();
                if (valid && (peers & lt) == 0) wcnt[warp][d] = before + (uint32_t)__popc(peers);
                __syncwarp();
                loc[r] = before + (uint32_t)__popc(peers & lt);
            }
        }
        __syncthreads();
        {
            const int d = threadIdx.x;
            uint32_t s = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = wcnt[w][d];
                wcnt[w][d] = s;
                s += c;
            }
            uint32_t tot;
            const uint32_t st = block_exclusive_scan<kSortThreads>(s, ws, &tot);
#pragma unroll
            for (int w = 0; w < kWarps; ++w) wcnt[w][d] += st;   // tile position of warp w's first digit d
            gbase[d] = scanned[ci.x + (uint32_t)d * ci.y] - st;  // output = gbase + tile position
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const int li = wseg + r * 32 + lane;
            if (li < nvalid) {
                const uint32_t d = (key[r] >> shift) & mask;
                const uint32_t pos = wcnt[warp][d] + loc[r];
                if (kPairs) reinterpret_cast<uint2 *>(&skv[stage][0][0])[pos] = make_uint2(key[r], val[r]);
                else skv[stage][0][pos] = key[r];
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < nvalid; p += kSortThreads) {
            if (kPairs) {
                const uint2 kv = reinterpret_cast<const uint2 *>(&skv[stage][0][0])[p];
                const uint32_t o = gbase[(kv.x >> shift) & mask] + (uint32_t)p;
                if (keys_out) keys_out[o] = kv.x;
                vals_out[o] = kv.y;
            } else {
                const uint32_t kk = skv[stage][0][p];
                keys_out[gbase[(kk >> shift) & mask] + (uint32_t)p] = kk;
            }
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------- one-sweep sort

constexpr int kMaxPasses = 4;
constexpr uint32_t kFlagAgg = 1u << 30;   // status word: tile's own digit count published
constexpr uint32_t kFlagInc = 2u << 30;   // status word: inclusive prefix over tiles <= t
constexpr uint32_t kValueMask = (1u << 30) - 1u;
constexpr uint32_t kLookbackLimit = 1u << 22;  // polls per status word
// One-sweep pays a look-back per tile; beyond this many keys the per-digit histogram
// path is faster (its scatter is bound by shared-memory traffic either way).
constexpr int64_t kOnesweepMaxKeys = int64_t(1) << 21;
#ifndef GC_LOOK_WINDOW
#define GC_LOOK_WINDOW 4
#endif
constexpr int kLookWindow = GC_LOOK_WINDOW;  // status words read per look-back round trip

struct DigitPlan {
    int passes;
    int shift[kMaxPasses];
    uint32_t mask[kMaxPasses];
};

// The status words carry their own payload (flag and count in one 32-bit word), so the
// look-back needs no ordering beyond the word's own coherence: relaxed accesses suffice.
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t *p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Digit counts of every pass over all keys: ghist[pass * 256 + digit].  Per-warp shared
// histograms, grid-stride over 16-byte groups of keys.
__global__ void __launch_bounds__(kSortThreads) k_onesweep_hist(const uint32_t *__restrict__ keys,
                                                                const uint32_t *n_dev, int64_t n_max,
                                                                DigitPlan plan, uint32_t *__restrict__ ghist) {
    __shared__ uint32_t wh[kWarps][kMaxPasses][256];
    const int warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kWarps * kMaxPasses * 256; k += kSortThreads) (&wh[0][0][0])[k] = 0;
    __syncthreads();
    const int64_t n = device_count(n_dev, n_max);
    const int64_t n4 = n >> 2;
    const uint4 *k4 = reinterpret_cast<const uint4 *>(keys);
    auto count = [&](uint32_t key) {
#pragma unroll
        for (int p = 0; p < kMaxPasses; ++p)
            if (p < plan.passes) atomicAdd(&wh[warp][p][(key >> plan.shift[p]) & plan.mask[p]], 1u);
    };
    for (int64_t i = (int64_t)blockIdx.x * kSortThreads + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * kSortThreads) {
        const uint4 q = k4[i];
        count(q.x);
        count(q.y);
        count(q.z);
        count(q.w);
    }
    if (blockIdx.x == 0 && threadIdx.x < (n & 3)) count(keys[(n4 << 2) + threadIdx.x]);
    __syncthreads();
    for (int p = 0; p < plan.passes; ++p) {
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) tot += wh[w][p][threadIdx.x];
        if (tot) atomicAdd(&ghist[p * 256 + threadIdx.x], tot);
    }
}

// One pass: a CTA per tile of kSortTile keys, tiles taken in ticket order.  status holds
// one word per (tile, digit), zero before the pass.
__global__ void __launch_bounds__(kSortThreads) k_onesweep_scatter(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const uint32_t *n_dev,
    int64_t n_max, int shift, uint32_t mask, const uint32_t *__restrict__ ghist, uint32_t *status,
    uint32_t *ticket, uint32_t *err) {
    __shared__ __align__(128) uint32_t sk[kSortTile];
    __shared__ __align__(128) uint32_t sv[kSortTile];
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t dstart[256];
    __shared__ uint32_t gbase[256];
    __shared__ uint32_t ws[33];
    __shared__ int s_tile;
    __shared__ __align__(8) uint64_t bar;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = device_count(n_dev, n_max);
    const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
    const int bits = __popc(mask);
    const uint32_t lt = lanemask_lt();
    if (threadIdx.x == 0) {
        s_tile = (int)atomicAdd(ticket, 1u);
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const int t = s_tile;
    if (t >= ntiles) return;
    const int64_t base = (int64_t)t * kSortTile;
    const int nvalid = (int)((n - base) < kSortTile ? (n - base) : kSortTile);
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)((nvalid * 4 + 15) & ~15);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bar, 2 * bytes);
        bulk_copy_g2s(sk, keys_in + base, bytes, &bar);
        bulk_copy_g2s(sv, vals_in + base, bytes, &bar);
    }
    for (int k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wcnt[0][0])[k] = 0;
    // global start of every digit (exclusive scan of the pass histogram), while the tile lands
    uint32_t gtot;
    const uint32_t gstart = block_exclusive_scan<kSortThreads>(ghist[threadIdx.x], ws, &gtot);
    const bool ok = mbar_wait_bounded(&bar, 0u);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(err, kErrTimeout);
            mbar_wait_bounded(&bar, 0u);
        }
        // publish an (empty) inclusive prefix so that no later tile waits on this one
        status[(size_t)t * 256 + threadIdx.x] = kFlagInc;
        return;
    }
    uint32_t key[kSortItems], val[kSortItems], loc[kSortItems];
    const int wseg = warp * (32 * kSortItems);
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int li = wseg + r * 32 + lane;
        const bool valid = li < nvalid;
        key[r] = valid ? sk[li] : 0xffffffffu;
        val[r] = valid ? sv[li] : 0u;
        const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        const uint32_t d = (key[r] >> shift) & mask;
        const uint32_t peers = bits < 8 ? __match_any_sync(0xffffffffu, d) & vmask : digit_peers(d, bits, vmask);
        const uint32_t before = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) wcnt[warp][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
        loc[r] = before + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t x = wcnt[w][d];
            wcnt[w][d] = c;
            c += x;
        }
        // publish this tile's count of digit d, then look back for the tiles before it
        uint32_t *my = status + (size_t)t * 256 + d;
        uint32_t excl = 0;
        if (t == 0) {
            st_relaxed(my, kFlagInc | c);
        } else {
            st_relaxed(my, kFlagAgg | c);
            // kLookWindow predecessors per round trip, nearest first; before tile 0 the
            // sentinel (inclusive, count 0) ends the walk
            bool done = false;
            for (int q = t - 1; !done; q -= kLookWindow) {
                uint32_t v[kLookWindow];
#pragma unroll
                for (int i = 0; i < kLookWindow; ++i)
                    v[i] = q - i >= 0 ? ld_relaxed(status + (size_t)(q - i) * 256 + d) : kFlagInc;
#pragma unroll
                for (int i = 0; i < kLookWindow; ++i) {
                    if (done) break;
                    uint32_t x = v[i];
                    for (uint32_t it = 0; (x & ~kValueMask) == 0u; ++it) {
                        if (it >= kLookbackLimit) {
                            atomicOr(err, kErrTimeout);
                            x = kFlagInc;
                            break;
                        }
                        x = ld_relaxed(status + (size_t)(q - i) * 256 + d);
                    }
                    excl += x & kValueMask;
                    done = (x & kFlagInc) != 0u;
                }
            }
            st_relaxed(my, kFlagInc | (excl + c));
        }
        uint32_t tot;
        dstart[d] = block_exclusive_scan<kSortThreads>(c, ws, &tot);
        gbase[d] = gstart + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int li = wseg + r * 32 + lane;
        if (li < nvalid) {
            const uint32_t d = (key[r] >> shift) & mask;
            const uint32_t pos = dstart[d] + wcnt[warp][d] + loc[r];
            sk[pos] = key[r];
            sv[pos] = val[r];
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < nvalid; p += kSortThreads) {
        const uint32_t k = sk[p];
        const uint32_t d = (k >> shift) & mask;
        const uint32_t o = gbase[d] + (uint32_t)p - dstart[d];
        if (keys_out) keys_out[o] = k;
        vals_out[o] = sv[p];
    }
}

}  // namespace

// Chained scan state: ticket, pad word, one 64-bit status word per chunk, error word.
size_t scan_partials_size(int64_t n) { return (size_t)2 * ((n + kScanChunk - 1) / kScanChunk) + 4; }

cudaError_t launch_exclusive_scan(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total,
                                  uint32_t *partials, cudaStream_t st, uint32_t *err) {
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (n <= kSmallScan) {
        k_scan_single<<<1, 1024, 0, st>>>(in, out, n, vec, total);
        note_launches(1);
        return cudaGetLastError();
    }
    const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
    if (reinterpret_cast<uintptr_t>(partials) & 7) return cudaErrorMisalignedAddress;  // 64-bit status words
    uint32_t *ticket = partials;
    unsigned long long *status = reinterpret_cast<unsigned long long *>(partials + 2);
    uint32_t *own_err = partials + 2 + 2 * nb;
    cudaError_t e = cudaMemsetAsync(partials, 0, 4 * scan_partials_size(n), st);
    if (e != cudaSuccess) return e;
    k_scan_onepass<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, vec, ticket, status, total,
                                                          err ? err : own_err);
    note_launches(1);
    return cudaGetLastError();
}

int radix_tile_keys(bool keys_only) { return keys_only ? kKeysTile : kSortTile; }

// Grid of the persistent scatter: every CTA that fits at once with the shared-memory carveout
// at its maximum (pairs: 48 registers and 42 KB of shared memory, five CTAs per SM), queried
// once per variant.
template <bool kPairs, int ITEMS>
static int scatter_grid() {
    static int cached = 0;
    if (!cached) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 148;
        cudaFuncSetAttribute(k_radix_scatter<kPairs, ITEMS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_radix_scatter<kPairs, ITEMS>, kSortThreads, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 4;
        cudaGetLastError();
        cached = sms * per_sm;
    }
    return cached;
}

// Classic layout: per-block digit counts + scan partials.  One-sweep layout: per pass
// 256 digit counts, a ticket and 256 status words per tile.
static size_t onesweep_words(int64_t nb, int passes) {
    return (size_t)passes * (256 + 1 + (size_t)256 * nb);
}

size_t radix_scratch_words(int64_t n_max) {
    int64_t nb = (n_max + kSortTile - 1) / kSortTile;
    if (nb < 1) nb = 1;
    // counts, scan state, per-block segment table (two words per block, 8-byte aligned)
    const size_t classic = (size_t)(256 * nb) + scan_partials_size(256 * nb) + 2 * (size_t)nb + 2;
    return n_max <= kOnesweepMaxKeys ? std::max(classic, onesweep_words(nb, kMaxPasses)) : classic;
}

cudaError_t radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max,
                             const uint32_t *n_dev, int end_bit, uint32_t *scratch, int *out_buf,
                             cudaStream_t st, uint32_t *err, bool keys_out,
                             const uint32_t *seg_block0, int n_seg, int begin_bit) {
    int cur = 0;
    if (n_max <= 0 || end_bit <= begin_bit) {
        *out_buf = 0;
        return cudaSuccess;
    }
    const bool pairs = vals != nullptr && vals[0] != nullptr;
    if (!pairs) keys_out = true;
    const int tile = pairs ? kSortTile : kKeysTile;
    const int nblocks = (int)((n_max + tile - 1) / tile);
    const int passes = (end_bit - begin_bit + 7) / 8;
    if (pairs && begin_bit == 0 && !seg_block0 && n_max <= kOnesweepMaxKeys && passes <= kMaxPasses) {
        // one-sweep: zero the counts, tickets and status words; one histogram kernel;
        // one scatter launch per pass
        DigitPlan plan;
        plan.passes = passes;
        int sh = 0;
        for (int p = 0; p < kMaxPasses; ++p) {
            const int bits = p < passes ? (end_bit - sh + (passes - p) - 1) / (passes - p) : 0;
            plan.shift[p] = sh;
            plan.mask[p] = bits ? (1u << bits) - 1u : 0u;
            sh += bits;
        }
        uint32_t *ghist = scratch;
        uint32_t *tickets = ghist + 256 * passes;
        uint32_t *status = tickets + passes;
        cudaError_t e = cudaMemsetAsync(scratch, 0, 4 * onesweep_words(nblocks, passes), st);
        if (e != cudaSuccess) return e;
        const int64_t groups = (n_max + 3) / 4;
        int hgrid = (int)std::min<int64_t>((groups + kSortThreads * 4 - 1) / (kSortThreads * 4), 148 * 4);
        if (hgrid < 1) hgrid = 1;
        k_onesweep_hist<<<hgrid, kSortThreads, 0, st>>>(keys[cur], n_dev, n_max, plan, ghist);
        note_launches(1);
        for (int p = 0; p < passes; ++p) {
            const bool last = p == passes - 1;
            k_onesweep_scatter<<<nblocks, kSortThreads, 0, st>>>(
                keys[cur], vals[cur], (last && !keys_out) ? nullptr : keys[cur ^ 1], vals[cur ^ 1], n_dev, n_max,
                plan.shift[p], plan.mask[p], ghist + 256 * p, status + (size_t)256 * nblocks * p, tickets + p, err);
            note_launches(1);
            cur ^= 1;
        }
        *out_buf = cur;
        return cudaGetLastError();
    }
    const int grid = std::min(nblocks, pairs ? scatter_grid<true, kSortItems>() : scatter_grid<false, kKeysItems>());
    uint32_t *counts = scratch;
    uint32_t *partials = scratch + (size_t)256 * nblocks;
    SegIndex sg{seg_block0, nullptr, n_seg};
    if (seg_block0) {
        size_t off = (size_t)256 * nblocks + scan_partials_size((int64_t)256 * nblocks);
        off = (off + 1) & ~(size_t)1;
        uint2 *blk = reinterpret_cast<uint2 *>(scratch + off);
        if (reinterpret_cast<uintptr_t>(blk) & 7) return cudaErrorMisalignedAddress;
        if (n_seg > 0) {
            k_block_segments<<<(unsigned)n_seg, 128, 0, st>>>(seg_block0, blk);
            note_launches(1);
        }
        sg.blk = blk;
    }
    // balanced digit widths: ceil((end_bit - begin_bit) / 8) passes of nearly equal width
    int shift = begin_bit;
    for (int pass = 0; pass < passes; ++pass) {
        const int bits = (end_bit - shift + (passes - pass) - 1) / (passes - pass);
        const uint32_t mask = (1u << bits) - 1u;
        if (pairs)
            k_radix_hist<kSortItems><<<nblocks, kSortThreads, 0, st>>>(keys[cur], n_dev, n_max, shift, mask, counts,
                                                                       nblocks, sg);
        else
            k_radix_hist<kKeysItems><<<nblocks, kSortThreads, 0, st>>>(keys[cur], n_dev, n_max, shift, mask, counts,
                                                                       nblocks, sg);
        note_launches(1);
        cudaError_t e = launch_exclusive_scan(counts, counts, (int64_t)256 * nblocks, nullptr,
                                              partials, st, err);
        if (e != cudaSuccess) return e;
        const bool last = pass == passes - 1;
        if (pairs)
            k_radix_scatter<true, kSortItems><<<grid, kSortThreads, 0, st>>>(keys[cur], vals[cur],
                                                                 (last && !keys_out) ? nullptr : keys[cur ^ 1],
                                                                 vals[cur ^ 1], n_dev, n_max, shift, mask, counts,
                                                                 nblocks, err, sg);
        else
            k_radix_scatter<false, kKeysItems><<<grid, kSortThreads, 0, st>>>(keys[cur], nullptr, keys[cur ^ 1], nullptr, n_dev,
                                                                  n_max, shift, mask, counts, nblocks, err, sg);
        note_launches(1);
        cur ^= 1;
        shift += bits;
    }
    *out_buf = cur;
    return cudaGetLastError();
}

}  // namespace gc
