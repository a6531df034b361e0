/*
 * gc4d.h - C ABI of a B300 (sm_103a) differentiable tile rasterizer for
 * hierarchical 4D Gaussians (4DGCPro, arXiv 2509.17513).
 *
 * One call renders one frame of a layer-selected Gaussian set:
 *   per-group rigid motion of the keyframe Gaussians (Sec. 3.2, "Rigid
 *   Transformation": mu_t = mu + t_g, R_t = R_g R), the 3D Gaussian of Eq. 1
 *   with Sigma = R s s^T R^T (Sec. 3.1), EWA projection to a 2D conic, tile
 *   binning with an on-device radix sort on (tile, depth), and front-to-back
 *   alpha compositing with spherical-harmonic colour (Eq. 2) restricted to the
 *   selected layers (progressive rendering, Eq. 4).  The backward pass returns
 *   the gradient of a loss w.r.t. every Gaussian attribute and the per-group
 *   motion, as the paper's rate-distortion training needs (Sec. 3.3).
 *
 * Conventions
 *   - Every buffer pointer marked "device" is CUDA global memory on the
 *     context's device, owned by the caller, row-major, tightly packed, and
 *     must stay valid until the work queued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - A context serialises its calls: use it from one host thread and one
 *     stream at a time.
 *   - Every entry point returns a gc_status; nothing throws across the ABI and
 *     no kernel traps.  gc_last_error() describes the last failure.
 *   - Images are planar FP32, 3 x height x width (channel, row, column).
 *   - Quaternions are Hamilton (w, x, y, z).  Camera: pinhole, x right, y down,
 *     z forward; pixel (i, j) has its centre at (i + 0.5, j + 0.5).
 */
#ifndef GC4D_H
#define GC4D_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GC_API __attribute__((visibility("default")))
#else
#define GC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GC_OK = 0,
    GC_ERR_INVALID_ARG = 1,  /* a pointer, size or option is out of range */
    GC_ERR_OOM = 2,          /* device allocation of library scratch failed */
    GC_ERR_CAPACITY = 3,     /* fixed key capacity too small; gc_last_error gives the need */
    GC_ERR_TIMEOUT = 4,      /* a bounded device wait ran out */
    GC_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    GC_ERR_STATE = 6,        /* backward without a matching forward, or a mismatched saved state */
    GC_ERR_UNSUPPORTED = 7   /* a valid request this build does not support */
} gc_status;

enum { GC_PREC_FP32 = 0, GC_PREC_BF16_FP8 = 1, GC_PREC_PLANES = 2 };
enum { GC_MEMBER_PIXEL = 0, GC_MEMBER_TILE = 1 };

typedef struct gc_context gc_context;
typedef struct gc_saved gc_saved;

/* Renderer options.  Defaults (gc_default_options): 16x16 tiles, near 0.2,
 * dilation 0.3, frustum clamp 1.3, black background, pixel-square
 * membership, key capacity 0 (grow on demand).  The near plane, dilation,
 * clamp and the +0.5 SH offset follow the 3DGS lineage the paper builds on
 * (Sec. A); the paper itself does not state them. */
typedef struct {
    int32_t tile_w, tile_h;   /* tile shape in pixels: 16x16, 8x32 or 32x8 */
    float near_plane;         /* Gaussians with camera z <= near are culled */
    float dilation;           /* added to both diagonal entries of the 2D covariance */
    float frustum_clamp;      /* x/z and y/z are clamped to +-clamp*tan(half fov) inside J */
    float bg[3];              /* background colour added with the final transmittance */
    int32_t membership;       /* GC_MEMBER_PIXEL: pixel centre within r of (u, v) in both axes;
                                 GC_MEMBER_TILE: every pixel of a touched tile */
    int64_t key_capacity;     /* 0: size the (tile, Gaussian) list per frame, one host sync per
                                 frame; > 0: fixed capacity, no host sync, GC_ERR_CAPACITY is
                                 reported by gc_check() when a frame needs more */
    int32_t alpha_cull;       /* 1 (default): the footprint is also clipped to the bounding box
                                 of the region where the Gaussian's alpha can reach 1/255
                                 (with a safety margin), and Gaussians with opacity <= 1/255
                                 are dropped; the image and the gradients are unchanged, the
                                 lists are shorter.  0: 3-sigma footprint only. */
} gc_options;

/* The Gaussian set, in layer order: layer l is [layer_offsets[l], layer_offsets[l+1]). */
typedef struct {
    int64_t n;                    /* number of Gaussians in the arrays */
    int32_t n_layers;             /* L, at most 32 */
    const int64_t *layer_offsets; /* HOST array of L+1 nondecreasing offsets, [0] = 0, [L] = n */
    int32_t sh_degree;            /* 0..3; K = (sh_degree+1)^2 coefficients per colour channel */
    int32_t precision;            /* GC_PREC_FP32, GC_PREC_BF16_FP8 or GC_PREC_PLANES */
    /* GC_PREC_FP32 attributes (device) */
    const float *means;           /* n x 3 */
    const float *log_scales;      /* n x 3, s = exp(log_scales) */
    const float *quats;           /* n x 4 (w, x, y, z), any nonzero norm */
    const float *opacity_logits;  /* n, opacity = sigmoid(logit) */
    const float *sh;              /* n x K x 3 (coefficient-major, then r, g, b) */
    const int32_t *group_id;      /* n motion-group ids in [0, G), or NULL: all in group 0 */
    /* GC_PREC_BF16_FP8 attributes (device): value = float(stored) * scale, one FP32 multiply */
    const uint16_t *means_bf16;      /* n x 3 bfloat16 bit patterns */
    const uint16_t *log_scales_bf16; /* n x 3 */
    const uint16_t *quats_bf16;      /* n x 4 */
    const uint16_t *opacity_bf16;    /* n */
    const uint8_t *sh_e4m3;          /* n x K x 3 float8 e4m3 ("fn") bit patterns */
    const float *scales;             /* device, 3 + 3 + 4 + 1 + 3K per-channel FP32 scales in the
                                        order means, log_scales, quats, opacity, sh (k-major, rgb) */
    /* GC_PREC_PLANES: the paper's decoded attribute planes (Sec. 3.4).  C = 11 + 3K channels in
     * the order x, y, z | quaternion w, x, y, z | log-scales 3 | opacity logit | SH (k-major,
     * rgb).  Per layer l (n_l Gaussians, rows_l = ceil(n_l / plane_width)) one device buffer of
     * uint8 codes for channels 3..C-1, channel c occupying rows [(c-3) rows_l, (c-2) rows_l) of
     * plane_pitch bytes each, and one buffer of pos_bits-bit codes (uint16 or uint32, native
     * byte order) for channels 0..2, rows of pos_pitch bytes; Gaussian j of the layer is at row
     * j / plane_width, column j % plane_width of its channel's plane.  value = lo + code * step
     * in FP32 (the product and the sum each rounded once), (lo, step) = dequant[(l C + c) 2 + 0/1]. */
    int32_t plane_width;             /* Gaussians per plane row, >= 1 */
    int32_t pos_bits;                /* 16 or 32 */
    int64_t plane_pitch;             /* bytes per row of the uint8 planes, >= plane_width */
    int64_t pos_pitch;               /* bytes per row of the position planes, >= plane_width * pos_bits / 8,
                                        a multiple of pos_bits / 8 */
    const uint8_t *const *planes_u8; /* HOST array of n_layers device pointers (may be NULL for empty layers) */
    const void *const *planes_pos;   /* HOST array of n_layers device pointers (aligned to pos_bits / 8) */
    const float *dequant;            /* device, n_layers x C x 2 FP32 */
} gc_gaussians;

/* One frame (device arrays): the cumulative per-group rigid motion (Sec. 3.2, rigid
 * transformation) and, optionally, the frame's residual deformation (Sec. 3.2, Eq. 7:
 * s_t = s_{t-1} + ds_t, alpha_t = alpha_{t-1} + dalpha_t, f_t = f_{t-1} + df_t), cumulative
 * from the keyframe.  The residuals are added, one FP32 addition each, to the log-scales,
 * the opacity logits and the SH coefficients before activation; each array may be NULL
 * (no residual for that attribute), and q, t may both be NULL (no group motion).  A
 * backward with residuals returns the gradients of the deformed attributes, which are
 * also the gradients of the residuals (they enter additively). */
typedef struct {
    int32_t n_groups;   /* G >= 1 */
    const float *q;     /* G x 4 unit quaternions; q' = q_g (x) q */
    const float *t;     /* G x 3 translations; mu' = mu + t_g */
    const float *res_log_scales;     /* n x 3 FP32, or NULL */
    const float *res_opacity_logits; /* n FP32, or NULL */
    const float *res_sh;             /* n x K x 3 FP32 (the set's K), or NULL */
    int32_t per_gaussian;            /* 1: one rigid motion per Gaussian (Sec. 3.2: dmu and dR from
                                        the motion source, e.g. gc_motion_field_forward): q is n x 4,
                                        t is n x 3, indexed by global Gaussian index; group ids and
                                        n_groups are ignored and the backward's d_group_q / d_group_t
                                        are n x 4 / n x 3.  Single-frame and multi-level calls only. */
} gc_motion;

/* Pinhole camera (host, by value). X_cam = R X_world + t. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];         /* row major */
    float t[3];
    float campos[3];    /* camera centre in world coordinates (view direction origin) */
} gc_camera;

/* Gradient outputs (device).  Overwritten (gc_render_batch_backward can also add
 * into them).  Gaussians that are not selected or not visible receive 0.  Any pointer may be NULL to skip
 * that output. */
typedef struct {
    float *d_means;          /* n x 3 */
    float *d_log_scales;     /* n x 3 */
    float *d_quats;          /* n x 4 */
    float *d_opacity_logits; /* n */
    float *d_sh;             /* n x K x 3 */
    float *d_group_q;        /* G x 4 */
    float *d_group_t;        /* G x 3 */
} gc_grads;

/* Per-Gaussian motion source (Sec. 3.2, rigid transformation): the positions of frame t-1
 * are encoded by a multi-resolution hash grid and two small MLPs give each Gaussian's
 * translation dmu and rotation dR.  Sizes the paper leaves open are fixed as: 2 features per
 * level, MLPs of one hidden layer of 64 ReLU units, translation = W2t relu(W1t h + b1t) + b2t,
 * rotation quaternion = W2r relu(W1r h + b1r) + b2r + (1, 0, 0, 0) (not normalised; the
 * renderer normalises q_g (x) q).  Level l: x = (mu - lo) / (hi - lo) clamped to [0, 1] per
 * axis, p = x N_l, cell = floor(p) clamped to [0, N_l - 1], w = p - cell (FP32, each
 * operation rounded once); vertex (i, j, k) is table entry i + (N_l + 1)(j + (N_l + 1) k) when
 * (N_l + 1)^3 <= T, else (i xor 2654435761 j xor 805459861 k) mod 2^32 mod T; h = per level the
 * trilinear blend of the cell's 8 vertex features. */
typedef struct {
    int32_t n_levels;          /* L_h, 1..16; the MLP input width is 2 L_h */
    int32_t log2_table;        /* T = 2^log2_table entries per level, 4..26 */
    int32_t resolution[16];    /* N_l >= 1 per level (first n_levels used) */
    float lo[3], hi[3];        /* box mapped to [0, 1]^3, hi > lo per axis */
    const float *table;        /* device, n_levels x T x 2 */
    const float *w1t, *b1t, *w2t, *b2t; /* device, row-major (out x in): 64 x 2L_h, 64, 3 x 64, 3 */
    const float *w1r, *b1r, *w2r, *b2r; /* device: 64 x 2L_h, 64, 4 x 64, 4 */
} gc_motion_field;

/* Gradients of a motion source (device, overwritten; any NULL is skipped).  The table
 * gradient is accumulated with atomic additions (its summation order is not fixed); the
 * weight gradients are summed per block and then over blocks in a fixed order. */
typedef struct {
    float *table, *w1t, *b1t, *w2t, *b2t, *w1r, *b1r, *w2r, *b2r;
} gc_motion_field_grads;

/* Per-frame statistics of a saved forward. */
typedef struct {
    int64_t n_selected;      /* Gaussians in the selected layers */
    int64_t n_visible;       /* of those, visible (non-empty footprint) */
    int64_t n_keys;          /* (tile, Gaussian) pairs, K */
    int32_t n_tiles;
    int32_t width, height;
} gc_stats;

/* Fills *out with the defaults listed at gc_options. */
GC_API gc_status gc_default_options(gc_options *out);

/* Creates a context on CUDA device `device`.  opt may be NULL (defaults).
 * The context owns grow-only device scratch; it is freed by gc_destroy. */
GC_API gc_status gc_create(gc_context **out, int device, const gc_options *opt);
GC_API gc_status gc_destroy(gc_context *ctx);

/* Replaces the context's options (takes effect from the next call). */
GC_API gc_status gc_set_options(gc_context *ctx, const gc_options *opt);

/* A saved forward state: the sorted tile lists, per-Gaussian projections
 * and per-pixel final transmittance that the backward pass reads.  Owned by
 * the library, reused across forwards, freed by gc_saved_destroy. */
GC_API gc_status gc_saved_create(gc_context *ctx, gc_saved **out);
GC_API gc_status gc_saved_destroy(gc_context *ctx, gc_saved *saved);

/*
 * Forward render of one frame (Eq. 2 / Eq. 4 over the layers in layer_mask).
 *   g          the Gaussian set (host struct; its arrays are device memory)
 *   motion     this frame's cumulative group motion, or NULL for the keyframe
 *   layer_mask bit l selects layer l (bit 0 = L1); level l is (1 << l) - 1
 *   cam        the camera (host)
 *   image      device, 3 x height x width, written
 *   saved      NULL for inference; else filled for gc_render_backward
 * An empty selection (n = 0 or no layer bit set) writes the background.
 */
GC_API gc_status gc_render_forward(gc_context *ctx, const gc_gaussians *g, const gc_motion *motion,
                            uint32_t layer_mask, const gc_camera *cam, float *image,
                            gc_saved *saved, void *stream);

/*
 * Forward render that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * render - a playback thread with a hard per-frame deadline (an allocation can
 * block or fail with out-of-memory mid-stream), and plugins running in another
 * application's CUDA context under a fixed memory budget that cannot hold a
 * gc_context.
 *
 * Same image as gc_render_forward with the same options, bit for bit (opt may
 * be NULL for exactly the gc_default_options values; key_capacity is ignored),
 * no saved state.  All scratch lives in
 * one static device array of about 22.5 MiB inside the library, which every GPU
 * that loads the library holds until the process exits.  Limits: at most
 * 32,768 selected Gaussians, 1,048,576 (tile, Gaussian) pairs, 262,144 pixels
 * and 4,096 tiles; larger requests return GC_ERR_CAPACITY with a message in
 * err (a caller buffer of err_len bytes, may be NULL) and write nothing.
 * The pair limit is checked after the depth sort and scan have run on the
 * GPU; the image is still left untouched.  The first call on each device
 * looks up the array's device address with cudaGetSymbolAddress (with that
 * device current).  Each call synchronises `stream`: once to read the pair
 * count and the error word into stack variables, and, when the frame has any
 * pairs, once more after the blend, so the call returns with the image
 * complete.  GC_ERR_TIMEOUT if a bounded wait of either sort ran out.  Calls
 * share the array: calls whose work overlaps on the GPU (other streams, other
 * threads) race and corrupt each other's images; serialise them on one stream.
 */
GC_API gc_status gc_render_forward_noalloc(const gc_options *opt, const gc_gaussians *g,
                                           const gc_motion *motion, uint32_t layer_mask,
                                           const gc_camera *cam, float *image, void *stream,
                                           char *err, size_t err_len);

/*
 * Backward of the forward recorded in `saved`: given dL/dimage (device,
 * 3 x height x width), writes dL/d(every attribute) and dL/d(group motion).
 * g and motion must be the same arrays that the forward read.  Reverse
 * compositing starts from each pixel's saved final transmittance; the
 * per-tile gradient reduction is atomics-free, so the result is bitwise
 * reproducible.
 */
GC_API gc_status gc_render_backward(gc_context *ctx, const gc_saved *saved, const gc_gaussians *g,
                             const gc_motion *motion, const float *dL_dimage, gc_grads *out,
                             void *stream);

/*
 * Multi-level render: all quality levels l = 1..levels of one view (level l = layers
 * 1..l, the paper's progressive render, Eq. 4) in one pass.  The layers are nested, so
 * the tile lists of the top level hold everything; every pixel keeps one transmittance
 * and colour per level and an entry of layer m is blended into the levels >= m.
 * level_images: host array of `levels` device pointers (3 x height x width each);
 * image l - 1 equals gc_render_forward with layer mask 1..l bit for bit.  levels <=
 * min(8, n_layers).  The paper's rate-distortion step renders every level per iteration
 * (Sec. 3.3); this replaces those renders by one.  `saved` then holds a multi-level
 * state for gc_render_levels_backward.
 */
GC_API gc_status gc_render_levels_forward(gc_context *ctx, const gc_gaussians *g, const gc_motion *motion,
                                          int32_t levels, const gc_camera *cam, float *const *level_images,
                                          gc_saved *saved, void *stream);

/*
 * Backward of a multi-level forward: dL_dimages is a host array of `levels` device
 * pointers (3 x height x width); the gradients of L = sum_l <dL_dimages[l], image_l>
 * (one pass; the per-level reverse steps share each entry's evaluation and reduction).
 */
GC_API gc_status gc_render_levels_backward(gc_context *ctx, const gc_saved *saved, const gc_gaussians *g,
                                           const gc_motion *motion, const float *const *dL_dimages,
                                           gc_grads *out, void *stream);

/* One render of a batch (host struct). */
typedef struct {
    gc_camera camera;     /* its own pose, intrinsics and resolution */
    int32_t frame;        /* index into the batch's motion frames, or -1 for the keyframe */
    uint32_t layer_mask;  /* layers rendered (bit l = layer l + 1), as in gc_render_forward */
    float *image;         /* device, 3 x height x width, written */
} gc_request;

/*
 * Batched forward: renders n_req requests of one Gaussian set, each with its own
 * camera, resolution, motion frame and layer mask - the many views, frames and
 * uneven levels that the paper's layer-wise rate-distortion training renders per
 * step (Sec. 3.3) and that multi-view playback needs.  Work is merged across the
 * requests: one preprocess launch over all (request, Gaussian) pairs, segmented
 * depth and tile sorts (each request sorted on its own, in shared launches), and one
 * persistent blend kernel whose CTAs pull tiles of all images from a work counter.
 * Each image equals what gc_render_forward returns for that request alone, bit for
 * bit.  frames: host array of n_frames motion tables (device arrays inside), may be
 * NULL when every request uses frame -1.  saved: NULL, or a state for
 * gc_render_batch_backward.  With key_capacity 0 the call reads one count from the
 * device (a host sync); with a fixed capacity it does not (overflow is reported by
 * gc_check).
 *
 * CUDA graphs: with a fixed capacity the call may be captured on `stream`.  The
 * capture must follow an eager call with the same requests, options and saved
 * state (it sizes the buffers and uploads the request table; the captured call
 * allocates, copies and synchronises nothing).  From then on that saved state is
 * bound to the graph: later calls on it must use the same requests, and it must
 * outlive the graph.  A captured call with other requests or sizes fails with
 * GC_ERR_STATE.
 */
GC_API gc_status gc_render_batch_forward(gc_context *ctx, const gc_gaussians *g,
                                         const gc_motion *frames, int32_t n_frames,
                                         const gc_request *reqs, int32_t n_req, gc_saved *saved,
                                         void *stream);

/*
 * Batched backward of the batch recorded in `saved`.  dL_dimages: host array of
 * n_req device pointers (3 x height x width each).  Attribute gradients are summed
 * over the requests in request order (deterministic); the motion gradient is per
 * (frame, group): out->d_group_q is n_frames x G x 4, out->d_group_t n_frames x G x 3.
 * accumulate = 0 overwrites the gradient buffers; 1 adds this batch's gradients to
 * them (one addition per element), so that a step split into several batches sums
 * its gradients in batch order.  Graph capture follows the rules of the forward
 * (the same dL_dimages pointers as the preceding eager call).
 */
GC_API gc_status gc_render_batch_backward(gc_context *ctx, const gc_saved *saved,
                                          const gc_gaussians *g, const gc_motion *frames,
                                          int32_t n_frames, const float *const *dL_dimages,
                                          int32_t accumulate, gc_grads *out, void *stream);

/*
 * Batch graphs: a whole training or playback step over many requests as one CUDA
 * graph.  The requests are split into consecutive batches of `depth` (the batch
 * depth); the graph holds, per batch, one gc_render_batch_forward and, when
 * dL_dimages is not NULL, one gc_render_batch_backward (the first batch overwrites
 * `grads`, the others add to them, so the gradient is summed over all requests in
 * order).  Each batch has a saved state of its own; batch b is captured on branch
 * b mod min(batches, 4) of the graph, so the batches of different branches overlap on
 * the GPU (one batch's sorts beside another's blend), while the backwards stay in batch
 * order.  Creation runs the step eagerly (with key_capacity 0 it first measures
 * every batch's key count and fixes the capacity at the largest plus 5 %), then
 * captures it; launching replays every kernel with no host work.  The graph reads
 * and writes the same device arrays as at creation (Gaussians, motion, images,
 * dL_dimages, grads): update their contents in place.  It owns its saved states and
 * must be destroyed before the context.  Overflow and bounded-wait timeouts are
 * reported by gc_batch_graph_check.  The context's options (tile shape, ...) are
 * read at creation and restored afterwards.
 */
typedef struct gc_batch_graph gc_batch_graph;

GC_API gc_status gc_batch_graph_create(gc_context *ctx, const gc_gaussians *g, const gc_motion *frames,
                                       int32_t n_frames, const gc_request *reqs, int32_t n_req,
                                       int32_t depth, const float *const *dL_dimages, gc_grads *grads,
                                       void *stream, gc_batch_graph **out);
GC_API gc_status gc_batch_graph_launch(gc_batch_graph *graph, void *stream);
/* Key capacity per batch, kernel nodes in the graph, number of batches; any may be NULL. */
GC_API gc_status gc_batch_graph_info(const gc_batch_graph *graph, int64_t *key_capacity,
                                     int64_t *kernel_nodes, int32_t *n_batches);
/* Synchronises `stream`; GC_ERR_CAPACITY or GC_ERR_TIMEOUT if a replay overflowed or timed out. */
GC_API gc_status gc_batch_graph_check(gc_batch_graph *graph, void *stream);
GC_API gc_status gc_batch_graph_destroy(gc_batch_graph *graph);

/*
 * Multi-level graphs: a multi-frame step of the single-pass multi-level render (every
 * quality level of each frame, Eq. 4; the paper's per-level rate-distortion renders,
 * Sec. 3.3) as one CUDA graph.  Per frame f = 0..n_frames-1, in order, the graph holds
 * gc_render_levels_forward(motions[f] (or no motion when motions is NULL), cameras[f],
 * levels, level_images + f * levels) and, when dL_dimages is not NULL,
 * gc_render_levels_backward(dL_dimages + f * levels, &grads[f]) - so a training step
 * renders and differentiates every frame; grads is a host array of n_frames gradient
 * sets (entries may name the same buffers; each frame overwrites what it names).
 * cameras: host array of n_frames; level_images and dL_dimages: host arrays of
 * n_frames * levels device pointers (3 x height x width each).  Creation fixes the key
 * capacity (the context's option, or with 0 the largest frame's exact need plus 5 %,
 * measured by one eager forward pass), runs the step eagerly once at that capacity
 * (sizing every buffer), then captures it; launching replays every kernel with no host
 * work, images identical to the eager calls.  chains (1..4): frame f runs on chain
 * f mod chains, each chain with a saved state of its own, as an independent branch of
 * the graph, so that the short sort and binning kernels of one frame run beside another
 * frame's blend; the backwards stay in frame order, so images and gradients equal those
 * of chains = 1 (chains > n_frames counts as n_frames).  The graph reads and writes the
 * same device arrays as at creation: update their contents in place.  It owns its saved
 * states and must be destroyed before the context.  An overflow of any frame and
 * bounded-wait timeouts are reported by gc_levels_graph_check.  The context's options
 * are read at creation and restored afterwards; profiling is off inside the graph.
 * Errors: GC_ERR_INVALID_ARG (missing arrays, n_frames or levels < 1), any error of the
 * captured calls, GC_ERR_CUDA if capture or instantiation fails; nothing is created
 * then.
 */
typedef struct gc_levels_graph gc_levels_graph;

GC_API gc_status gc_levels_graph_create(gc_context *ctx, const gc_gaussians *g, const gc_motion *motions,
                                        int32_t n_frames, const gc_camera *cameras, int32_t levels,
                                        float *const *level_images, const float *const *dL_dimages,
                                        gc_grads *grads, int32_t chains, void *stream, gc_levels_graph **out);
GC_API gc_status gc_levels_graph_launch(gc_levels_graph *graph, void *stream);
/* Key capacity per frame and kernel nodes in the graph; either may be NULL. */
GC_API gc_status gc_levels_graph_info(const gc_levels_graph *graph, int64_t *key_capacity,
                                      int64_t *kernel_nodes);
/* Synchronises `stream`; GC_ERR_CAPACITY if a frame of a replay since the last check
 * needed more keys than the capacity, GC_ERR_TIMEOUT if a bounded wait ran out. */
GC_API gc_status gc_levels_graph_check(gc_levels_graph *graph, void *stream);
GC_API gc_status gc_levels_graph_destroy(gc_levels_graph *graph);

/* One measured configuration of the autotuner. */
typedef struct {
    int32_t tile_w, tile_h;  /* tile shape */
    int32_t depth;           /* requests per batch */
    int64_t key_capacity;    /* per-batch key capacity the graph used */
    float ms;                /* mean time of one graph launch (the whole step) */
} gc_tune_entry;

/*
 * Autotuner over tile shape {16x16, 8x32, 32x8} x batch depth (depths[0..n_depths)):
 * builds the batch graph of every configuration, times `iters` launches after one
 * warm-up with CUDA events on `stream`, and writes 3 * n_depths entries (shape-major).
 * The fastest is returned in *best and its tile shape is set in the context's
 * options.  Images and gradients are written as a side effect.
 */
GC_API gc_status gc_tune_batch(gc_context *ctx, const gc_gaussians *g, const gc_motion *frames,
                               int32_t n_frames, const gc_request *reqs, int32_t n_req,
                               const float *const *dL_dimages, gc_grads *grads, const int32_t *depths,
                               int32_t n_depths, int32_t iters, gc_tune_entry *entries,
                               gc_tune_entry *best, void *stream);

/* Motion source forward: for the n Gaussians at means (device, n x 3, the frame t-1
 * positions) writes q (device, n x 4, dR) and t (device, n x 3, dmu), which a gc_motion with
 * per_gaussian = 1 applies to the frame t-1 Gaussians (mu_t = mu + dmu, R_t = dR R). */
GC_API gc_status gc_motion_field_forward(gc_context *ctx, const gc_motion_field *field, const float *means,
                                         int64_t n, float *q, float *t, void *stream);

/* Motion source backward: given dL/dq (n x 4) and dL/dt (n x 3) - the d_group_q / d_group_t of
 * a per-Gaussian render backward - writes the gradients of the table and the MLP weights. */
GC_API gc_status gc_motion_field_backward(gc_context *ctx, const gc_motion_field *field, const float *means,
                                          int64_t n, const float *d_q, const float *d_t,
                                          gc_motion_field_grads *out, void *stream);

/* The same pair with the hash-grid encodings kept between them (a training step): the forward
 * also writes every Gaussian's encoding to `encodings` (device, n x 32 FP32 rows, levels
 * beyond n_levels zero, 16-byte aligned, caller-owned), and the backward reads them instead of
 * gathering the table again.  The backward's results equal gc_motion_field_backward's bit for
 * bit when `encodings` holds the forward's for the same means and table.  Errors: those of
 * the pair above, GC_ERR_INVALID_ARG for a NULL or unaligned `encodings`. */
GC_API gc_status gc_motion_field_forward_save(gc_context *ctx, const gc_motion_field *field, const float *means,
                                              int64_t n, float *q, float *t, float *encodings, void *stream);
GC_API gc_status gc_motion_field_backward_saved(gc_context *ctx, const gc_motion_field *field,
                                                const float *means, int64_t n, const float *encodings,
                                                const float *d_q, const float *d_t, gc_motion_field_grads *out,
                                                void *stream);

/* KDE rate estimate of the keyframe RD loss (Sec. 3.3, the PMF equation): for each of
 * n_channels channels of n FP32 values (channel c at y + c * stride, device), the bits per
 * symbol of its quantised symbols s_i = round(y_i) (half to even) under the Gaussian kernel
 * density of those symbols with the Silverman-rule bandwidth h = sigma (3n/4)^(-1/5) (sigma
 * the symbols' sample standard deviation, h = 1 when it is 0):
 *   PMF(k) = CDF(k + 1/2) - CDF(k - 1/2),  rate = -(1/n) sum_i log2 max(PMF(s_i), 2^-40).
 * Writes rate[c] (device).  A channel whose symbols span more than 8192 consecutive integers,
 * or that holds a value that is not finite or beyond 2^24 in magnitude, gets NaN. */
GC_API gc_status gc_kde_rate(gc_context *ctx, const float *y, int32_t n_channels, int64_t n, int64_t stride,
                             float *rate, void *stream);

/* Training form of the KDE rate (Sec. 3.3: differentiable quantisation by injected uniform
 * noise).  y holds the noise-injected values y~_i = y_i + u_i in units of the quantisation
 * step (the caller draws u), n per channel at y + c * stride.  The density is the one of
 * gc_kde_rate, built from the symbols s_i = round(y~_i) and held fixed; the rate is taken at
 * the continuous values and differentiated through them:
 *   P(x) = CDF(x + 1/2) - CDF(x - 1/2),  R_c = -(1/n) sum_i log2 max(P(y~_i), 2^-40),
 *   dR_c/dy~_i = -(pdf(y~_i + 1/2) - pdf(y~_i - 1/2)) / (n ln 2 P(y~_i))  (0 at the floor),
 *   pdf(x) = (1/(n h)) sum_j phi((x - s_j) / h).
 * For integer inputs R_c equals gc_kde_rate.  d_rate: device array of n_channels upstream
 * gradients dL/dR_c, or NULL for ones.  Writes rate[c] (device) and, when d_y is not NULL,
 * d_y[c * stride + i] = dL/dR_c * dR_c/dy~_i (device, the layout of y).  Unsupported channels
 * (as in gc_kde_rate) get NaN in rate and in their d_y row.  Symbols farther than 8 h + 1
 * from a value are left out of its sums: their mass is below Phi(-8) = 6e-16 of their count,
 * while P of a value is at least about 1 / (n h) from its own symbol (relative error < 1e-9). */
GC_API gc_status gc_kde_rate_grad(gc_context *ctx, const float *y, int32_t n_channels, int64_t n,
                                  int64_t stride, const float *d_rate, float *rate, float *d_y, void *stream);

/* Statistics of the last forward recorded in `saved` (synchronises `stream`). */
GC_API gc_status gc_saved_stats(gc_context *ctx, const gc_saved *saved, gc_stats *out, void *stream);

/*
 * Copies the sorted tile lists of `saved` (synchronises `stream`):
 *   ranges    device, n_tiles x 2 int32 [start, end) into gauss_ids
 *   gauss_ids device, capacity entries: global Gaussian index of each entry,
 *             tile by tile, front to back (depth, then index)
 * Returns GC_ERR_CAPACITY if capacity < n_keys.
 */
GC_API gc_status gc_saved_tile_lists(gc_context *ctx, const gc_saved *saved, int32_t *ranges,
                              int64_t *gauss_ids, int64_t capacity, void *stream);

/* Per-pixel diagnostics of `saved` (device buffers, H x W, any may be NULL):
 * final transmittance (FP32), number of Gaussians blended into the pixel,
 * number of tile-list entries the pixel walked before it stopped, and the
 * list position just after its last blended entry (where the backward pass
 * starts; int32). */
GC_API gc_status gc_saved_pixel_state(gc_context *ctx, const gc_saved *saved, float *final_T,
                                      int32_t *n_blended, int32_t *n_walked, int32_t *n_contrib,
                                      void *stream);

/*
 * L1 photometric distortion of a rendered image against a target (the L1 part of the colour
 * loss of the rate-distortion training, Sec. 3.3; its D-SSIM part is not built):
 *   loss = scale * sum_i |image_i - target_i|,  dL_dimage_i = scale * sign(image_i - target_i),
 * sign(0) = 0; scale = 1 / n gives the mean.  image, target, dL_dimage: device, n floats
 * each (any layout, the same for all three); loss: device, one float.  Either output may be
 * NULL (both NULL: nothing runs).  The sum is deterministic (one FP64 partial per CTA of a
 * fixed grid, added in CTA order).  The first call grows a small context-owned buffer of
 * partial sums; later calls allocate nothing, so a training step that calls it can be
 * captured into a graph after one eager step.
 */
GC_API gc_status gc_l1_loss(gc_context *ctx, const float *image, const float *target, int64_t n, float scale,
                            float *dL_dimage, float *loss, void *stream);

/* Stages timed by the profiler (CUDA events recorded on the call's stream
 * between stages). */
enum {
    GC_STAGE_PREPROCESS = 0,   /* motion + projection + footprint + colour */
    GC_STAGE_DEPTH_SORT = 1,   /* radix sort of the depth keys */
    GC_STAGE_SCAN = 2,         /* rank gather + exclusive scan of tiles touched */
    GC_STAGE_EMIT = 3,         /* (tile, rank) entries */
    GC_STAGE_TILE_SORT = 4,    /* radix sort of the tile keys */
    GC_STAGE_RANGES = 5,       /* per-tile [start, end) */
    GC_STAGE_BLEND = 6,        /* forward compositing */
    GC_STAGE_BLEND_BWD = 7,    /* reverse compositing + per-tile reduction */
    GC_STAGE_REDUCE = 8,       /* per-Gaussian sum of the tile partials */
    GC_STAGE_PREPROCESS_BWD = 9, /* chain rule to the attributes */
    GC_STAGE_GROUP_REDUCE = 10,  /* per-group motion gradient */
    GC_N_STAGES = 11
};

/* Per-stage event timing on this context: 0 off, 1 on, 2 on with L2 flushed before
 * every stage (a 256 MB context-owned buffer is written between the event that closes
 * one stage and the event that opens the next, so each stage reads its inputs from
 * HBM and its time excludes the flush). */
GC_API gc_status gc_profile_enable(gc_context *ctx, int enable);

/* Reads and resets the profile: per stage the summed milliseconds and the
 * number of timed calls (arrays of GC_N_STAGES; either may be NULL), and the
 * number of kernels the library launched since the last read on this
 * context.  Waits for the recorded events. */
GC_API gc_status gc_profile_read(gc_context *ctx, double *stage_ms, int64_t *stage_calls,
                                 uint64_t *kernel_launches);

/* Reports errors recorded on the device by fixed-capacity or bounded-wait
 * work since the last check (synchronises `stream`): GC_OK,
 * GC_ERR_CAPACITY or GC_ERR_TIMEOUT. */
GC_API gc_status gc_check(gc_context *ctx, void *stream);

/* Text of the last error on this context (valid until the next call). */
GC_API const char *gc_last_error(gc_context *ctx);

/* Library version string. */
GC_API const char *gc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GC4D_H */
