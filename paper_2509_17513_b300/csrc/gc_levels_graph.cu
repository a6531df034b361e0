// gc_levels_graph.cu - a multi-frame step of the single-pass multi-level render (every
// quality level of each frame from one sorted list, Eq. 4 / Sec. 3.3) as one CUDA graph.
//
// Per frame, in order: gc_render_levels_forward and, for a training step,
// gc_render_levels_backward, on a saved state that the graph owns.  With a fixed key
// capacity neither call synchronises, allocates or copies to the host once the buffers are
// sized, so the whole step is captured after one eager pass and replayed with no host work:
// the launch gaps between the ~15 kernels of every frame disappear.  The binning keeps
// the largest key count of any frame on the state, which gc_levels_graph_check compares
// with the capacity.
//
// Chains: frame f runs on chain f mod C, each chain with its own saved state (its own
// lists, scratch and backward buffers) and its own capture stream forked from the caller's,
// so the graph holds C independent sequences of frames.  A frame's preprocess, sorts and
// binning are short, latency-bound kernels that leave most of the GPU idle; with C > 1 they
// run beside another frame's blend.  The backwards' writes into the gradient sets stay in frame
// order (frame f's wait for frame f-1's; its reverse blend and reduce do not wait), so gradient
// sets shared by several frames are written exactly as by one chain; images and gradients equal
// those of C = 1.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gc_state.cuh"

namespace {
constexpr int kMaxChains = 4;
}

struct gc_levels_graph {
    gc_context *ctx = nullptr;
    int chains = 1;
    gc_saved *states[kMaxChains] = {};
    cudaStream_t side[kMaxChains] = {};  // capture streams of chains 1..chains-1
    cudaEvent_t fork = nullptr, bwd_done = nullptr, joins[kMaxChains] = {};
    int64_t key_capacity = 0;
    int64_t kernel_nodes = 0;
    cudaStream_t own_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void levels_graph_free(gc_levels_graph *G) {
    if (!G) return;
    DeviceGuard dg(G->ctx->device);
    if (G->exec) cudaGraphExecDestroy(G->exec);
    if (G->graph) cudaGraphDestroy(G->graph);
    for (int c = 0; c < kMaxChains; ++c) {
        if (G->states[c]) gc_saved_destroy(G->ctx, G->states[c]);
        if (G->side[c]) cudaStreamDestroy(G->side[c]);
        if (G->joins[c]) cudaEventDestroy(G->joins[c]);
    }
    if (G->fork) cudaEventDestroy(G->fork);
    if (G->bwd_done) cudaEventDestroy(G->bwd_done);
    if (G->own_stream) cudaStreamDestroy(G->own_stream);
    delete G;
}

struct LevelsStep {
    const gc_gaussians *g;
    const gc_motion *motions;
    int n_frames;
    const gc_camera *cams;
    int levels;
    float *const *images;
    const float *const *dL;
    gc_grads *grads;
};

// Every frame on its chain's state and stream (streams[c]; all the caller's stream outside
// capture).  The backwards' gradient writes are ordered by bwd_done.
gc_status levels_pass(gc_levels_graph *G, const LevelsStep &P, const cudaStream_t *streams, int64_t *max_keys) {
    for (int f = 0; f < P.n_frames; ++f) {
        const int c = f % G->chains;
        const cudaStream_t s = streams[c];
        gc_saved *state = G->states[c];
        const gc_motion *m = P.motions ? &P.motions[f] : nullptr;
        gc_status st = gc_render_levels_forward(G->ctx, P.g, m, P.levels, &P.cams[f], P.images + (size_t)f * P.levels,
                                                state, s);
        if (st != GC_OK) return st;
        if (max_keys) *max_keys = std::max<int64_t>(*max_keys, state->K);
        if (P.dL) {
            // the writes into the gradient set wait for the previous frame's; the reverse blend
            // and the reduce run as soon as this chain reaches them
            const bool ordered = G->chains > 1;
            st = levels_backward_ordered(G->ctx, state, P.g, m, P.dL + (size_t)f * P.levels, &P.grads[f], s,
                                         ordered && f > 0 ? G->bwd_done : nullptr, ordered ? G->bwd_done : nullptr);
            if (st != GC_OK) return st;
        }
    }
    return GC_OK;
}

}  // namespace

extern "C" gc_status gc_levels_graph_create(gc_context *ctx, const gc_gaussians *g, const gc_motion *motions,
                                            int32_t n_frames, const gc_camera *cameras, int32_t levels,
                                            float *const *level_images, const float *const *dL_dimages,
                                            gc_grads *grads, int32_t chains, void *stream, gc_levels_graph **out) {
    if (!ctx) return GC_ERR_INVALID_ARG;
    if (!out) return fail(ctx, GC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_frames < 1 || !cameras || !level_images || levels < 1)
        return fail(ctx, GC_ERR_INVALID_ARG, "need n_frames >= 1, cameras, levels >= 1 and level_images");
    if (dL_dimages && !grads) return fail(ctx, GC_ERR_INVALID_ARG, "dL_dimages without grads");
    if (chains < 1 || chains > kMaxChains) return fail(ctx, GC_ERR_INVALID_ARG, "chains must be 1..%d", kMaxChains);
    DeviceGuard dg(ctx->device);
    gc_levels_graph *G = new gc_levels_graph;
    G->ctx = ctx;
    G->chains = std::min<int>(chains, n_frames);
    const gc_options saved_opt = ctx->opt;
    const bool saved_prof = ctx->prof_on;
    auto bail = [&](gc_status e) {
        ctx->opt = saved_opt;
        ctx->prof_on = saved_prof;
        levels_graph_free(G);
        return e;
    };
    for (int c = 0; c < G->chains; ++c) {
        gc_status st = gc_saved_create(ctx, &G->states[c]);
        if (st != GC_OK) return bail(st);
    }
    bool ok = cudaEventCreateWithFlags(&G->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&G->bwd_done, cudaEventDisableTiming) == cudaSuccess;
    for (int c = 1; c < G->chains && ok; ++c)
        ok = cudaStreamCreateWithFlags(&G->side[c], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&G->joins[c], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return bail(fail(ctx, GC_ERR_CUDA, "stream or event creation failed"));
    }
    gc_status st = GC_OK;
    ctx->prof_on = false;  // no profiling events inside a graph
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) {  // capture needs a stream other than the legacy default one
        if (cudaStreamCreateWithFlags(&G->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(ctx, GC_ERR_CUDA, "stream creation failed"));
        }
        s = G->own_stream;
    }
    cudaStream_t eager[kMaxChains], capture[kMaxChains];
    for (int c = 0; c < kMaxChains; ++c) {
        eager[c] = s;
        capture[c] = c == 0 ? s : G->side[c];
    }
    const LevelsStep P{g, motions, n_frames, cameras, levels, level_images, dL_dimages, grads};
    // 1. key capacity: the caller's, or the largest frame's exact need plus 5 %
    int64_t cap = saved_opt.key_capacity;
    if (cap <= 0) {
        ctx->opt.key_capacity = 0;
        int64_t kmax = 0;
        const LevelsStep fwd{g, motions, n_frames, cameras, levels, level_images, nullptr, nullptr};
        if ((st = levels_pass(G, fwd, eager, &kmax)) != GC_OK) return bail(st);
        const int64_t T = gc::radix_tile_keys();
        cap = (kmax + kmax / 20 + 2 * T + T - 1) / T * T;
        if (cap > 0xFFFFFFF0ll) return bail(fail(ctx, GC_ERR_CAPACITY, "a frame needs more than 2^32 keys"));
    }
    G->key_capacity = cap;
    ctx->opt.key_capacity = cap;
    // 2. eager pass at the fixed capacity on the caller's stream: sizes every chain's buffers
    if ((st = levels_pass(G, P, eager, nullptr)) != GC_OK) return bail(st);
    if (cudaStreamSynchronize(s) != cudaSuccess) return bail(fail(ctx, GC_ERR_CUDA, "eager pass failed"));
    for (int c = 0; c < G->chains; ++c)
        if ((st = capacity_check(ctx, *G->states[c], s)) != GC_OK) return bail(st);
    // 3. capture the same pass, chain c on capture[c] (forked from s, joined back into s)
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ctx, GC_ERR_CUDA, "cannot begin stream capture"));
    }
    cudaError_t ce = cudaEventRecord(G->fork, s);
    for (int c = 1; c < G->chains && ce == cudaSuccess; ++c) ce = cudaStreamWaitEvent(G->side[c], G->fork, 0);
    if (ce == cudaSuccess) st = levels_pass(G, P, capture, nullptr);
    for (int c = 1; c < G->chains && ce == cudaSuccess; ++c) {
        ce = cudaEventRecord(G->joins[c], G->side[c]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s, G->joins[c], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s, &graph);
    G->graph = graph;
    if (st != GC_OK) return bail(st);
    if (ce != cudaSuccess || ee != cudaSuccess || !graph) {
        cudaGetLastError();
        return bail(fail(ctx, GC_ERR_CUDA, "stream capture failed: %s",
                         cudaGetErrorString(ce != cudaSuccess ? ce : ee)));
    }
    size_t n_nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes) cudaGraphGetNodes(graph, nodes.data(), &n_nodes);
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) G->kernel_nodes++;
    }
    if (cudaGraphInstantiate(&G->exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(ctx, GC_ERR_CUDA, "graph instantiation failed"));
    }
    ctx->opt = saved_opt;
    ctx->prof_on = saved_prof;
    *out = G;
    return GC_OK;
}

extern "C" gc_status gc_levels_graph_launch(gc_levels_graph *G, void *stream) {
    if (!G) return GC_ERR_INVALID_ARG;
    DeviceGuard dg(G->ctx->device);
    GC_CUDA(G->ctx, cudaGraphLaunch(G->exec, (cudaStream_t)stream));
    gc::note_launches((int)G->kernel_nodes);
    return GC_OK;
}

extern "C" gc_status gc_levels_graph_info(const gc_levels_graph *G, int64_t *key_capacity, int64_t *kernel_nodes) {
    if (!G) return GC_ERR_INVALID_ARG;
    if (key_capacity) *key_capacity = G->key_capacity;
    if (kernel_nodes) *kernel_nodes = G->kernel_nodes;
    return GC_OK;
}

extern "C" gc_status gc_levels_graph_check(gc_levels_graph *G, void *stream) {
    if (!G) return GC_ERR_INVALID_ARG;
    gc_context *ctx = G->ctx;
    DeviceGuard dg(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    for (int c = 0; c < G->chains; ++c) {
        const gc_saved &S = *G->states[c];
        uint32_t err = 0;
        GC_CUDA(ctx, cudaMemcpyAsync(&err, static_cast<uint32_t *>(S.words.p) + 1, 4, cudaMemcpyDeviceToHost, s));
        GC_CUDA(ctx, cudaStreamSynchronize(s));
        if (err) {
            GC_CUDA(ctx, cudaMemsetAsync(static_cast<uint32_t *>(S.words.p) + 1, 0, 4, s));
            return fail(ctx, GC_ERR_TIMEOUT, "a bounded device wait ran out (error word %#x)", err);
        }
        const gc_status st = capacity_check(ctx, S, s);
        if (st != GC_OK) return st;
    }
    return GC_OK;
}

extern "C" gc_status gc_levels_graph_destroy(gc_levels_graph *G) {
    if (!G) return GC_ERR_INVALID_ARG;
    levels_graph_free(G);
    return GC_OK;
}
