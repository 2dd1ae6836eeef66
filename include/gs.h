/*
 * gs.h - C ABI of libgs, the GB300 (sm_103a) hot path of 3D Gaussian
 * Splatting training (arXiv 2406.18533, "On Scaling Up 3D Gaussian Splatting
 * Training").
 *
 * The paper splits one training iteration into four steps (Sec. 2.1):
 * Gaussian transformation, rendering, loss calculation and backpropagation,
 * followed by the Adam update of every Gaussian (Sec. 4, Eq. 1-2 for batched
 * training).  Each entry point below is one of those steps, or the whole
 * iteration (gs_train_step), or a forward-only batch of novel views
 * (gs_render).
 *
 * Conventions shared by every call
 *  - Pointers inside gs_scene, gs_proj, gs_proj_grad, gs_bins and the image
 *    arguments are DEVICE pointers owned by the caller (the library never
 *    frees them).  gs_camera and gs_hparams arrays are HOST memory, read
 *    during the call only.
 *  - Every call is asynchronous on the caller's CUDA stream (cudaStream_t
 *    passed as void*; NULL = legacy default stream) unless it says otherwise.
 *  - The library owns only scratch memory inside the opaque gs_ctx, grown on
 *    demand with cudaMalloc (which synchronises the device) or reserved up
 *    front with gs_reserve.  Calls on one context must not overlap on the GPU
 *    (one stream per context).
 *  - Every call returns a gs_status.  Host-side argument errors return at
 *    once.  Errors found by kernels (fragment capacity overflow, non-finite
 *    parameters in strict mode) are written to a device status word and
 *    reported by gs_get_status.  gs_last_error gives a text for the last
 *    non-OK status.  No exception or abort crosses the ABI.
 *  - Camera model (a reading of the 3DGS projection the paper builds on):
 *    OpenCV axes (x right, y down, z forward), p_cam = R p_world + t, pixel
 *    (i, j) has centre (i + 0.5, j + 0.5), u = fx x/z + cx, v = fy y/z + cy.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GS_ABI_VERSION 5   /* 5: gs_count_work, gs_preprocess_bwd_scaled; work counters on request */
#define GS_MAX_VIEWS 32   /* views per call (training batch or render batch) */
#define GS_MAX_FRAGMENTS 1073741823ull  /* 2^30 - 1: largest fragment capacity of one call */

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,  /* null pointer, bad size, B outside 1..GS_MAX_VIEWS, ... */
    GS_ERR_CAPACITY = 2,     /* fragment buffer too small; the needed count is reported */
    GS_ERR_CUDA = 3,         /* a CUDA runtime call failed (text in gs_last_error) */
    GS_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    GS_ERR_NONFINITE = 5,    /* non-finite parameters met in strict mode */
    GS_ERR_OOM = 6           /* scratch allocation failed */
} gs_status;

/* Pinhole camera; 80 bytes. */
typedef struct gs_camera {
    float R[9];        /* world -> camera rotation, row-major */
    float t[3];        /* translation: p_cam = R p_world + t */
    float fx, fy;      /* focal lengths in pixels */
    float cx, cy;      /* principal point in pixels */
    int32_t W, H;      /* image size in pixels, each >= 1 */
    float near_z;      /* a Gaussian with z_cam <= near_z is culled (> 0) */
    int32_t reserved;
} gs_camera;

/*
 * Gaussian parameters (Sec. 2: position x in R^3, scale s in R^3, rotation
 * q in R^4, opacity, 48 SH coefficients), structure-of-arrays float4 planes,
 * 60 floats per Gaussian.  The same struct describes gradients and the two
 * Adam moments (same layout).  All four planes must be 16-byte aligned.
 */
typedef struct gs_scene {
    float *mo;         /* [N] float4: x, y, z, opacity logit (opacity = sigmoid) */
    float *ls;         /* [N] float4: log sx, log sy, log sz, unused (kept 0) */
    float *q;          /* [N] float4: w, x, y, z (normalised inside) */
    float *sh;         /* [12][N] float4: SH coefficient k (0..15), channel c at flat
                          index j = 3k + c, stored in plane j/4, lane j%4 */
    int64_t N;         /* number of Gaussians, >= 0 */
    int32_t sh_degree; /* 0..3 */
    int32_t reserved;
} gs_scene;

/* Hyperparameters (host struct, copied into the context). */
typedef struct gs_hparams {
    int32_t tile;             /* screen tile edge: 8, 16 (paper's 16x16 blocks) or 32 */
    int32_t smem_batch;       /* list entries a warp stages per shared-memory refill: 32, 64
                                 or 128 (tile 32 with one pixel per thread: 32 or 64) */
    int32_t strict_nonfinite; /* 1: report GS_ERR_NONFINITE; 0: cull silently */
    float alpha_min;          /* skip a Gaussian at a pixel below this alpha (1/255) */
    float alpha_max;          /* alpha is clamped to this (0.99) */
    float T_min;              /* stop before a Gaussian that would take T below this (1e-4) */
    float bg[3];              /* background colour added as T_final * bg (0) */
    float lr[6];              /* Adam learning rates: mean, scale, quat, opacity, sh_dc, sh_rest */
    float beta1, beta2, eps;  /* Adam (0.9, 0.999, 1e-15) */
    int32_t scale_lr_sqrt_b;  /* Eq. 1: lr' = lr * sqrt(B) */
    int32_t scale_beta_pow_b; /* Eq. 2: beta' = beta^B */
    float lambda_dssim;       /* loss = (1-l) L1 + l (1 - SSIM), l = 0.2 */
    int32_t px_per_thread;    /* pixels a blending thread owns: 1 (a warp blends an 8x4 block),
                                 2 (8x8) or 4 (8x16, tile 16 or 32) */
    int32_t sparse_adam;      /* 0: Adam over every Gaussian (the paper's optimizer, default);
                                 1: gs_train_step updates only the Gaussians some view of the
                                 batch sees (visible-only Adam, see gs_adam_step_sparse) */
    int32_t schedule;         /* blending schedule of gs_train_step: 0 (default) one CTA per tile,
                                 longest lists first where that pays; 1 Algorithm 1: the tiles are
                                 split into contiguous ranges of equal cost, measured per tile in
                                 the previous step (list lengths before the first), one range per
                                 resident persistent CTA (see gs_division_points); 2 a persistent
                                 pool: one CTA per resident slot pulls tiles from a device queue
                                 counter, heaviest cost of the previous step first */
} gs_hparams;

/*
 * Per (view, Gaussian) output of the Gaussian transformation (Sec. 2.1 step
 * 1: projected centre x_{v,i}, depth, footprint radius, colour c_{v,i}),
 * index v * N + g.  Caller-owned device arrays of B * N entries.
 */
typedef struct gs_proj {
    float *xy;         /* float2 (u, v) pixel centre */
    float *conic_o;    /* float4 (a, b, c, opacity): inverse 2D covariance [[a,b],[b,c]] */
    float *rgb_d;      /* float4 (r, g, b, depth): view-dependent colour, camera-space z */
    int32_t *radius;   /* footprint radius in whole pixels; 0 = touches no tile */
    int64_t N;
    int32_t B;
    int32_t reserved;
} gs_proj;

/* Gradients with respect to gs_proj entries (float4 each, B * N entries). */
typedef struct gs_proj_grad {
    float *d_xy_o;     /* (dL/du, dL/dv, dL/dopacity, 0) */
    float *d_conic;    /* (dL/da, dL/db, dL/dc, 0) */
    float *d_rgb;      /* (dL/dr, dL/dg, dL/db, 0) */
} gs_proj_grad;

/*
 * Depth-sorted fragments ("Z-buffer", Appendix A.2): one entry per
 * (view, tile, Gaussian) whose footprint rectangle covers the tile, sorted by
 * key = (tile_id << 32) | float_bits(depth); equal keys keep ascending
 * Gaussian index.  tile_id = sum of tile counts of earlier views + ty * TX + tx.
 */
typedef struct gs_bins {
    uint64_t *keys;    /* [capacity] sorted keys */
    uint32_t *vals;    /* [capacity] Gaussian index within its view */
    uint32_t *ranges;  /* [2 * total_tiles] uint2 [start, end) per tile_id */
    uint32_t *count;   /* [1] device: number of fragments F */
    uint64_t capacity; /* entries allocated in keys / vals */
} gs_bins;

typedef struct gs_ctx gs_ctx;

/* Context: hyperparameters, scratch, device status word.  hp == NULL takes the
 * 3DGS defaults.  Returns GS_ERR_INVALID_ARG for an unsupported tile size. */
gs_status gs_create(gs_ctx **ctx, const gs_hparams *hp);
gs_status gs_destroy(gs_ctx *ctx);
gs_status gs_default_hparams(gs_hparams *hp);
gs_status gs_set_hparams(gs_ctx *ctx, const gs_hparams *hp);
const char *gs_last_error(const gs_ctx *ctx);
int32_t gs_abi_version(void);

/* Pre-size the context scratch for gs_train_step / gs_render so that no later
 * call allocates (needed before stream capture into a CUDA graph). */
gs_status gs_reserve(gs_ctx *ctx, int64_t N, const gs_camera *cams, int32_t B, uint64_t frag_capacity);

/* Bytes of workspace that gs_reserve with these arguments takes from a fresh
 * caller workspace (gs_set_workspace): the scratch of gs_train_step and
 * gs_render for these sizes.  Computed on the host (a dry run of gs_reserve
 * that only adds up the buffers), so it is exact for that call sequence. */
gs_status gs_workspace_size(const gs_hparams *hp, int64_t N, const gs_camera *cams, int32_t B,
                            uint64_t frag_capacity, size_t *bytes);

/* Caller workspace.  After this call the context takes all its scratch from
 * [ws, ws + bytes) (device memory the caller allocated and owns, 256-byte
 * aligned) instead of cudaMalloc: buffers are carved in order and never
 * freed by the library; a buffer that has to grow takes a new region, so
 * size the workspace with gs_workspace_size and call gs_reserve once with
 * the same arguments.  A call whose scratch no longer fits returns
 * GS_ERR_OOM (gs_last_error says how many bytes were missing) and launches
 * nothing.  The call synchronises `stream` and drops every buffer the
 * context held (their contents are lost); ws = NULL returns the context to
 * cudaMalloc.  The workspace must outlive its use by the context. */
gs_status gs_set_workspace(gs_ctx *ctx, void *ws, size_t bytes, void *stream);

/* The context's device-side Adam step counter (the number of updates made by
 * calls with step == 0 since creation, or since gs_set_step), for
 * checkpoint and resume.  Both synchronise `stream` and must not be called
 * while it is being captured.  gs_set_step: step >= 0, else
 * GS_ERR_INVALID_ARG; the next step == 0 update then uses step + 1. */
gs_status gs_get_step(gs_ctx *ctx, int64_t *step, void *stream);
gs_status gs_set_step(gs_ctx *ctx, int64_t step, void *stream);

/* Synchronise `stream`, then read and clear the device status word.
 * *status gets GS_OK or the first device-side error; *needed (optional) the
 * fragment count the last binning asked for. */
gs_status gs_get_status(gs_ctx *ctx, void *stream, int32_t *status, uint64_t *needed);

/* Counters of the last binning / forward / backward render (synchronises):
 * out[0] = fragments F, out[1] = (pixel, fragment) evaluations in the
 * forward, out[2] = (pixel, Gaussian) pairs blended in the backward,
 * out[3] = (pixel, list position) pairs the backward walked (out[1],
 * out[2], out[3] and out[5] only while gs_count_work is on), out[4] =
 * Gaussians culled for non-finite parameters (cumulative), out[5] = the sum
 * of n_contrib over the forward's pixels (list positions the backward
 * covers, before any culling).  out holds 6 values (ABI version 2). */
gs_status gs_get_counters(gs_ctx *ctx, void *stream, uint64_t out[6]);

/* Work counting of the compositing kernels (profiling aid, no paper
 * counterpart).  out[1], out[2], out[3] and out[5] of gs_get_counters are
 * counted only while it is on (on != 0); off (the default) they read 0 after
 * each binning.  Counting takes a few percent of the blending kernels' issued
 * instructions, so timed runs leave it off and count in a separate step.  Takes effect at the next
 * backward launch; a CUDA graph captured before keeps the setting it was
 * captured with. */
gs_status gs_count_work(gs_ctx *ctx, int32_t on);

/*
 * Tracing (profiling aid, no paper counterpart): when enabled with
 * gs_trace_enable(ctx, max_steps) (> 0; 0 disables), every gs_train_step
 * records CUDA events on its stream around its GS_TRACE_STAGES stages, for
 * up to max_steps steps.  gs_trace_read synchronises and writes, for each
 * recorded step s and stage k, the elapsed milliseconds to
 * ms[s * GS_TRACE_STAGES + k] (ms holds max_steps * GS_TRACE_STAGES floats),
 * sets *steps to the number of recorded steps and restarts recording.
 * Stage order: preprocess, order (pairs sorted by depth + offsets scan),
 * emit, sort (fragments by tile), ranges, blend_fwd, loss, zero_grad,
 * blend_bwd, preprocess_bwd, adam.
 */
#define GS_TRACE_STAGES 11
gs_status gs_trace_enable(gs_ctx *ctx, int32_t max_steps);
gs_status gs_trace_read(gs_ctx *ctx, float *ms, int32_t *steps);

/* Number of CUDA kernels this library has launched in this process so far
 * (all contexts); differences count the kernels of a region. */
uint64_t gs_kernel_launches(void);

/*
 * Test hooks for the failure paths (no paper counterpart).  Both settings are
 * process-wide (all contexts, all threads) and meant for tests only.
 *
 * gs_debug_set_lookback: a tile of the radix sort waits for the digit counts
 * of earlier tiles (decoupled look-back).  Each such wait polls at most
 * spin_limit times (0 = the default, 2^22) and then gives up, setting
 * GS_ERR_TIMEOUT in the device status word.  withhold_first_tile != 0 makes
 * tile 0 of every sort pass keep its counts to itself, so the waits of later
 * tiles run out: the binning then finishes with wrong but in-bounds results
 * (every store of the sort, and every read of the kernels after it, is
 * checked against its buffer), gs_get_status reports GS_ERR_TIMEOUT, and the
 * context stays usable.  Reset with (0, 0).
 *
 * gs_debug_fail_alloc: after = -1 turns the injection off; after = n >= 0
 * lets the library's next n device allocations succeed and fails the one
 * after that with GS_ERR_OOM, without calling cudaMalloc, then turns itself
 * off.  after < -1 returns GS_ERR_INVALID_ARG.  The call that meets the
 * failure returns GS_ERR_OOM; the context keeps what it had and can retry.
 */
gs_status gs_debug_set_lookback(uint32_t spin_limit, int32_t withhold_first_tile);
gs_status gs_debug_fail_alloc(int64_t after);

/*
 * Sec. 2.1 step 1 (Gaussian transformation), fused over B views: reads each
 * Gaussian's parameters once, writes gs_proj for every view.  A Gaussian is
 * culled in a view (radius 0) when z_cam <= near_z, its 2D covariance is
 * singular, or its footprint rectangle misses the image.
 */
gs_status gs_preprocess(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cams, int32_t B,
                        gs_proj *out, void *stream);

/*
 * Sec. 2.1 step 2, first half (Fig. 2 16x16 blocks; "iterates over
 * intersecting Gaussians in increasing depth"): counts the tiles each
 * (view, Gaussian) footprint rectangle covers; sorts the visible pairs by
 * depth (stable LSD radix sort, 8-bit digits); emits one key per covered tile,
 * pair by pair in that order; sorts the keys stably on their tile bits; and
 * writes per-tile ranges.  If F > out->capacity nothing beyond capacity is written,
 * the status word gets GS_ERR_CAPACITY and *needed_host (if given: this call
 * then synchronises the stream) gets F and the call returns GS_ERR_CAPACITY.
 */
gs_status gs_bin(gs_ctx *ctx, const gs_proj *proj, const gs_camera *cams, int32_t B, gs_bins *out,
                 uint64_t *needed_host, void *stream);

/*
 * gs_bin_noalloc: the binning of gs_bin (tile counts, scan, key emission,
 * radix sort, tile ranges) without any device memory allocation.  The paper
 * has no counterpart; this entry point exists for callers that cannot call
 * cudaMalloc: code that owns a fixed device-memory budget handed out by a
 * host application's own allocator, latency-critical loops that cannot
 * afford cudaMalloc/cudaFree (both synchronise the device), and callers
 * without a gs_ctx (creating one allocates).
 *
 * All scratch lives in one static device array of 20.63 MiB that every GPU on
 * which the library's kernels are loaded holds until the process exits.
 * Limits: B * proj->N <= 262144 (view, Gaussian) pairs and out->capacity <=
 * 1048576 fragments; larger sizes, an unsupported tile (8, 16, 32) or a bad
 * pointer return GS_ERR_INVALID_ARG before any work.  Inputs and outputs are
 * the caller's, exactly as for gs_bin; a capacity overflow is handled as in
 * gs_bin (nothing written past capacity; with needed_host the call
 * synchronises the stream and returns GS_ERR_CAPACITY with the needed count).
 * There is no status word a caller can read: without needed_host an overflow
 * leaves *count == 0, which cannot be told from a binning with no fragments,
 * so a caller whose fragments may exceed out->capacity must pass needed_host.
 * The array's device address is looked up on every call made outside stream
 * capture (so a cudaDeviceReset between calls is harmless); a call during
 * stream capture reuses the address of the last call outside capture on that
 * device, so make a first call on each device before any capture.  Every
 * call uses the same array: calls that overlap on the GPU (other streams,
 * other threads) race and corrupt each other's results.
 */
gs_status gs_bin_noalloc(const gs_proj *proj, const gs_camera *cams, int32_t B, int32_t tile, gs_bins *out,
                         uint64_t *needed_host, void *stream);

/*
 * Sec. 2.1 step 2, second half: per pixel, front-to-back alpha compositing
 * over its tile's sorted list until transmittance would fall below T_min.
 * img: [B][3][H][W] float; T_final: [B][H][W] float; n_contrib: [B][H][W]
 * uint32 (1 + list position of the last blended Gaussian).  All views of one
 * call must share W and H here (mixed sizes: gs_render).
 */
gs_status gs_render_fwd(gs_ctx *ctx, const gs_proj *proj, const gs_bins *bins, const gs_camera *cams,
                        int32_t B, float *img, float *T_final, uint32_t *n_contrib, void *stream);

/*
 * Backward of the compositing (the paper's "standard approaches to
 * backpropagation", Sec. 2.1): walks each pixel's contributors back to front,
 * recovering transmittance from T_final by division (no per-fragment state),
 * and accumulates dL/d(gs_proj) for every (view, Gaussian).  `out` is
 * overwritten.  d_img has the layout of img.
 */
gs_status gs_render_bwd(gs_ctx *ctx, const gs_proj *proj, const gs_bins *bins, const gs_camera *cams,
                        int32_t B, const float *T_final, const uint32_t *n_contrib, const float *d_img,
                        gs_proj_grad *out, void *stream);

/*
 * Backward of the Gaussian transformation: chain rule from dL/d(gs_proj) to
 * the 59 parameters of every Gaussian, summed over the B views and divided by
 * B (the batch gradient is the mean of the per-view gradients, Sec. 4).
 * `grad` is overwritten (its unused lane ls.w is written 0).
 */
gs_status gs_preprocess_bwd(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cams, int32_t B,
                            const gs_proj *proj, const gs_proj_grad *dproj, gs_scene *grad, void *stream);

/*
 * gs_preprocess_bwd with an explicit factor: grad = scale * (sum over the B
 * views of the per-view chain rule).  scale = 1/B is gs_preprocess_bwd (the
 * paper's batch mean, Sec. 4); scale = 1 gives the sum, the gradient of a
 * loss that adds the views' losses (what an autograd engine expects from a
 * function of B images).  scale must be finite and >= 0, else
 * GS_ERR_INVALID_ARG.
 */
gs_status gs_preprocess_bwd_scaled(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cams, int32_t B,
                                   const gs_proj *proj, const gs_proj_grad *dproj, gs_scene *grad, float scale,
                                   void *stream);

/*
 * Sec. 2.1 step 3: loss = (1 - l) mean|I - I*| + l (1 - mean SSIM(I, I*)),
 * SSIM with an 11x11 Gaussian window (sigma 1.5), zero padding, per view.
 * img, target, d_img: [B][3][H][W]; loss_out: [B] float (device).  d_img is
 * dL_v/dI_v for each view v (not divided by B).
 */
gs_status gs_loss(gs_ctx *ctx, const float *img, const float *target, int32_t B, int32_t W, int32_t H,
                  float *loss_out, float *d_img, void *stream);

/*
 * Adam over all 60 N floats (Sec. 4): m = b1' m + (1-b1') g, v = b2' v +
 * (1-b2') g^2, p -= lr' m_hat / (sqrt(v_hat) + eps), bias correction with
 * b' at `step` (>= 1), lr' = lr sqrt(B) (Eq. 1) and b' = b^B (Eq. 2) when the
 * hyperparameter flags ask for them.  In place on p, m, v.  step == 0 takes
 * the step from the context's device-side counter, incremented by the call
 * itself (first call: step 1), so a call captured in a CUDA graph advances the
 * step on every replay.  A pending GS_ERR_CAPACITY or GS_ERR_TIMEOUT in the
 * device status word skips the update (and the device step counter).
 */
gs_status gs_adam_step(gs_ctx *ctx, gs_scene *p, const gs_scene *g, gs_scene *m, gs_scene *v,
                       int64_t step, int32_t B, void *stream);

/*
 * Visible-only ("sparse") Adam: the update of gs_adam_step applied only to
 * the Gaussians with visible[i] != 0; the others keep p, m and v exactly as
 * they were (their moments do not decay).  The paper observes that the
 * gradient of a batch is sparse, each view seeing a small part of the scene
 * (Sec. 4); a Gaussian no view of the batch sees has a zero gradient, and
 * dense Adam spends its 1652 bytes of traffic per Gaussian on it anyway.
 * visible: device array of p->N bytes (caller-owned).  The step's bias
 * correction is the batch count as in gs_adam_step (step == 0: the device
 * counter); a pending GS_ERR_CAPACITY or GS_ERR_TIMEOUT skips the update.
 */
gs_status gs_adam_step_sparse(gs_ctx *ctx, gs_scene *p, const gs_scene *g, gs_scene *m, gs_scene *v,
                              const uint8_t *visible, int64_t step, int32_t B, void *stream);

/*
 * One whole training iteration over a batch of B views (Fig. 1(a) pipeline,
 * batched as in Sec. 4): transformation, binning, compositing, loss,
 * backward, Adam.  targets: [B][3][H][W] float device; loss_out: [B] float
 * device.  Scratch comes from the context.  g receives the batch gradient.
 * step as in gs_adam_step (0: device counter).  With hp.sparse_adam = 1 the
 * optimizer is gs_adam_step_sparse with visible = "some view of the batch has
 * the Gaussian's radius > 0", and g's rows of the unseen Gaussians are left
 * as they were (not written).  Once the context has sized its
 * scratch (a first call, or gs_reserve), the call allocates nothing and never
 * synchronises, so it can be captured in a CUDA graph; the graph replays the
 * captured cameras.
 */
gs_status gs_train_step(gs_ctx *ctx, gs_scene *p, gs_scene *g, gs_scene *m, gs_scene *v, int64_t step,
                        const gs_camera *cams, int32_t B, const float *targets, float *loss_out,
                        void *stream);

/*
 * Densification (App. A.1: Gaussians whose projected position keeps moving
 * across training steps are cloned or split, by whether their scale exceeds a
 * threshold; Gaussians of low opacity are pruned; opacity is reset now and
 * then).  The paper states the rule in words and defers its details to 3DGS;
 * the readings below fix them.
 *
 * gs_set_densify_stats: when grad_acc / grad_cnt (caller-owned device arrays
 * of N float / uint32) are set, every gs_train_step adds, for each view of its
 * batch in which a Gaussian is visible (radius > 0), the length of that
 * view's position gradient |dL_v/d(u, v)| (pixels; the view's own loss, before
 * the batch mean) to grad_acc and 1 to grad_cnt (a step that overflows its
 * fragment buffer or whose sort gives up adds nothing).  NULL pointers stop
 * it.  Steps on a scene of another N add nothing.  The arrays must hold the
 * scene's N; the caller zeroes them after densifying.
 *
 * gs_densify: one densification of N Gaussians (p, m, v) into p_out, m_out,
 * v_out (caller-owned, capacity Gaussians each; their N field must equal
 * capacity).  Per Gaussian g, with mean gradient decided in float32 as
 * grad_acc[g] >= grad_threshold * (float)grad_cnt[g] (and grad_cnt[g] > 0):
 *   - prune when its opacity logit < logit(min_opacity) (float32 compare);
 *   - else clone when the gradient test passes and its largest log-scale
 *     <= log(scale_threshold): the Gaussian and an exact copy (the copy's
 *     Adam moments zero);
 *   - else split when the gradient test passes: two children replace it,
 *     child k at mean + Rq diag(s) xi_k (xi_k = normals[6g + 3k .. +2],
 *     caller-drawn standard normals), log-scale = log-scale - ln(split_div),
 *     same rotation, opacity and SH, moments zero;
 *   - else keep it with its moments.
 * Outputs keep the input order, each Gaussian's results together (the
 * original or first child, then the copy or second child).  The new count
 * goes to *n_out (the call synchronises the stream); if it exceeds capacity
 * nothing is written and the call returns GS_ERR_CAPACITY with *n_out set.
 * normals: device float[6 N].
 *
 * gs_reset_opacity: every opacity becomes min(opacity, max_opacity) (on the
 * logit), and the opacity lane of both Adam moments is zeroed.
 */
typedef struct gs_densify_params {
    float grad_threshold;   /* mean |dL/d(u, v)| per visible view, pixels (3DGS-like: 0.2 px order) */
    float scale_threshold;  /* world units: clone at or below, split above */
    float min_opacity;      /* prune below (0.005) */
    float split_div;        /* child scale = parent scale / split_div (1.6) */
} gs_densify_params;

gs_status gs_set_densify_stats(gs_ctx *ctx, float *grad_acc, uint32_t *grad_cnt, int64_t N);
gs_status gs_densify(gs_ctx *ctx, const gs_scene *p, const gs_scene *m, const gs_scene *v, const float *grad_acc,
                     const uint32_t *grad_cnt, const float *normals, const gs_densify_params *dp, gs_scene *p_out,
                     gs_scene *m_out, gs_scene *v_out, int64_t capacity, int64_t *n_out, void *stream);
gs_status gs_reset_opacity(gs_ctx *ctx, gs_scene *p, gs_scene *m, gs_scene *v, float max_opacity, void *stream);

/*
 * Algorithm 1 ("Calculation of Division Points", Sec. 3.3): the paper splits
 * an image's sequence of pixel blocks among G GPUs by the blocks' runtimes
 * measured in the previous iteration: CT = cumsum(ET), ET_gpu = CT[B-1] / G,
 * DP = searchsorted(CT, arange(0, G) * ET_gpu).  Here the blocks are the
 * batch's tiles and the GPUs are persistent CTAs (hp.schedule = 1).
 * gs_division_points computes DP for T costs (device uint32, caller-owned,
 * read only) and P ranges: div[k] (device uint32[P]) is the first tile of
 * range k, i.e. the first i with CT[i] >= k CT[T-1] / P, compared exactly as
 * P CT[i] >= k CT[T-1] in 64-bit integers; range k is [div[k], div[k+1]) and
 * the last ends at T.  Each cost is first capped at (2^32 - 1) / T (so the
 * 32-bit prefix sums cannot wrap).  T >= 1, 1 <= P <= 2^20.
 */
gs_status gs_division_points(gs_ctx *ctx, const uint32_t *cost, int64_t T, int32_t P, uint32_t *div,
                             void *stream);

/*
 * Storage order of the Gaussians (a data-layout step, no paper counterpart as
 * an algorithm: the paper's Gaussian-wise distribution decides which GPU
 * holds a Gaussian, Sec. 3.1 and App. B.2; this decides where in one GPU's
 * memory it lives).  Every (view, Gaussian) record the compositing kernels
 * gather is indexed by Gaussian, so Gaussians that meet the same screen
 * tiles should sit next to each other in memory.  gs_spatial_order writes
 * perm[N]: the Gaussian indices sorted stably by the Morton (Z-order) code of
 * their positions, each axis quantised to 10 bits over the bounding box of
 * the finite positions as floor((x - lo) * (1024 / (hi - lo))) with each
 * float32 operation rounded separately, clamped to 1023 (a non-finite
 * position, or a flat axis, gives cell 0).  gs_permute then writes
 * dst[i] = src[perm[i]] for all 60 floats (out of place: no plane of dst may
 * be a plane of src); apply it to the parameters and, in training, to the
 * Adam moments.  Renders do not depend on the order (ties of equal depth go
 * to the lower index).  Both calls are asynchronous; perm is caller-owned
 * device memory of N uint32 (N < 2^31).  gs_spatial_order grows the
 * context's scratch (12 bytes per Gaussian plus the sort's).
 */
gs_status gs_spatial_order(gs_ctx *ctx, const gs_scene *scene, uint32_t *perm, void *stream);
gs_status gs_permute(gs_ctx *ctx, const gs_scene *src, const uint32_t *perm, gs_scene *dst, void *stream);

/*
 * Forward-only render of B novel views of possibly different sizes (serving):
 * imgs[b] (host array of device pointers) receives view b as [3][H_b][W_b].
 */
gs_status gs_render(gs_ctx *ctx, const gs_scene *scene, const gs_camera *cams, int32_t B,
                    float *const *imgs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
