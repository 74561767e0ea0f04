/*
 * di.h -- C ABI of the GB300 homogeneous diffusion inpainting decoder.
 *
 * The decoder solves, per colour channel, the discrete inpainting problem of
 * Section 2.2 (eq. 2.6):
 *     (C + (I - C) L) u = C f,
 * c the binary mask (known pixels), L the 5-point negated Laplacian with
 * reflecting image boundaries and unit grid spacing.  The solver is the
 * reduced full multigrid of Section 4.2 with the optimized restricted additive
 * Schwarz smoother of Section 3 (Algorithm 2) and the grid transfers of
 * Sections 4.3 and 4.4.  Everything runs in hand-written CUDA kernels for
 * sm_103a on one GPU.
 *
 * Conventions for every entry point:
 *  - Images are planar float32 [channels][height][width], row-major, in DEVICE
 *    memory; masks are uint8 [height][width] in DEVICE memory, nonzero = known
 *    pixel, shared by all channels.  Channels are 1..4.
 *  - The caller owns every pointer it passes; the library never frees them.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    enqueue their kernels on it; argument errors are reported synchronously
 *    and nothing is enqueued then.  DI_ERR_CUDA reports a failed launch or
 *    allocation error from the CUDA runtime.
 *  - Values of f at unknown pixels are never used in arithmetic (they may be
 *    NaN or Inf).
 *  - A context may be used from one host thread at a time.
 */
#ifndef DI_H
#define DI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct di_ctx di_ctx;

typedef enum {
    DI_OK = 0,
    DI_ERR_INVALID_ARG = 1,   /* null pointer, size < 1, channels not in 1..4,
                                 tol <= 0, aliasing buffers, bad config */
    DI_ERR_EMPTY_MASK = 2,    /* no known pixel: the problem has no unique solution */
    DI_ERR_OOM = 3,           /* device workspace could not be allocated */
    DI_ERR_NOT_CONVERGED = 4, /* max_cycles reached first; u holds the last iterate */
    DI_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    DI_ERR_TIMEOUT = 6        /* a bounded device-side wait ran out: a tile copy of the
                                 32x32 block kernel did not arrive; every output of the
                                 call (u included) is undefined */
} di_status;

/* Stop rules of di_inpaint.  DI_STOP_ERROR_ESTIMATE: after every V-cycle the
 * error is estimated from the size of the cycle's updates and their decay
 * (est = U_k q/(1-q), q the larger of the last two ratios U_k/U_{k-1}, U_k the
 * sum of the largest pre-smoothing, coarse-correction and post-smoothing
 * updates on the finest grid); the solve stops when est <= tol/2.
 * DI_STOP_RELATIVE_RESIDUAL: the paper's criterion
 * (Section 5.2), ||b - A u||_2 / ||b||_2 <= tol, per channel.
 * DI_STOP_FIXED_CYCLES: exactly max_cycles V-cycles. */
enum { DI_STOP_ERROR_ESTIMATE = 0, DI_STOP_RELATIVE_RESIDUAL = 1, DI_STOP_FIXED_CYCLES = 2 };

/* Precision modes.  DI_PREC_FP32: everything FP32.  DI_PREC_FP16 /
 * DI_PREC_BF16: (1) the block-local CG iterates -- vectors, stencil and
 * updates of every local solve -- in packed 16-bit arithmetic with FP32 dot
 * products (the block residual is normalised before it is narrowed); (2) the
 * coarse levels' iterates and restricted residuals, i.e. the coarse-grid
 * corrections of Section 4.1, stored in that 16-bit type (read, widened and
 * computed in FP32, rounded once when stored).  The finest grid keeps FP32
 * iterates and FP32 residuals, so the outer FP32 iteration refines whatever
 * the narrow parts leave (cfg.refine_fp64 adds FP64 residuals there).
 * Requires 32x32 blocks and the block smoother. */
enum { DI_PREC_FP32 = 0, DI_PREC_FP16 = 1, DI_PREC_BF16 = 2 };

/* Schedules (Sections 4.2 and 5).  REDUCED_FMG: the cascade with one
 * smoothing step per level, then V-cycles on the finest level (the paper's
 * method).  FULL_FMG: a V-cycle on every level of the cascade (Fig. 3), then
 * V-cycles.  MULTILEVEL: the cascade, then smoothing steps on the finest level
 * without coarse corrections (the multilevel solver of the comparison).
 * SINGLE: no hierarchy; smoothing steps on the finest level from u = f on the
 * mask, 0 elsewhere.  For the last two a "cycle" of the stop rule is one
 * smoothing step. */
enum { DI_SCHED_REDUCED_FMG = 0, DI_SCHED_FULL_FMG = 1, DI_SCHED_MULTILEVEL = 2,
       DI_SCHED_SINGLE = 3 };

/* Smoothers.  ORAS: one ORAS iteration (Algorithm 2).  CG: local_iters steps
 * of global conjugate gradients on the level's reduced system (the CG
 * counterparts of Section 5).  With DI_SCHED_SINGLE and DI_SCHED_MULTILEVEL
 * one CG run continues across the steps on the finest level (global CG from
 * the cascade's guess); inside V-cycles every smoothing call starts afresh.
 * The single-block solve of the coarsest level always uses the block solver. */
enum { DI_SMOOTH_ORAS = 0, DI_SMOOTH_CG = 1 };

/* Launch of the decode.  ON: CUDA graphs -- the whole decode as one
 * device-driven graph (see di_inpaint) where the configuration allows it;
 * otherwise (profiling on, the full-FMG schedule) one finest-level V-cycle
 * captured per call and replayed once per cycle with the stop rule on the
 * host; the multilevel and single-level schedules launch kernel by kernel.
 * If a capture fails the kernels are launched one by one.  OFF: always one
 * by one, stop rule on the host.  The results are identical. */
enum { DI_GRAPH_ON = 0, DI_GRAPH_OFF = 1 };

/* Initial iterate.  CASCADE: the coarse-to-fine cascade of the schedule (or,
 * single level, u = f on the mask and 0 elsewhere).  GIVEN: the values in u
 * on entry (finite everywhere) are the initial iterate off the mask, u = f on
 * the mask; the cascade is skipped and the cycles start at once.  A decoder
 * of video frames with a fixed mask passes the previous frame's result: the
 * temporal coherence that Section 1 names as a way to make the method faster
 * on videos. */
enum { DI_START_CASCADE = 0, DI_START_GIVEN = 1 };

/* Solver configuration; a zero field takes the default in brackets. */
typedef struct {
    int block;        /* B, square ORAS block side: 8, 16 or 32 [32] (Section 3.1) */
    int overlap;      /* o, overlap of neighbouring blocks, 1..B/2 [6] (Section 3.1) */
    int local_iters;  /* CG steps of each local block solve [8] (Section 3.1) */
    int coarse_iters; /* cap on the CG steps of the single-block solve of the coarsest
                         level, which otherwise runs to a relative residual of ~1e-6 [2048] */
    int pre;          /* ORAS pre-smoothing iterations per V-cycle [1] (Section 4.4) */
    int post;         /* ORAS post-smoothing iterations per V-cycle [1] (Section 4.4) */
    int max_cycles;   /* cap on V-cycles after the cascade [16] */
    int min_cycles;   /* V-cycles always run [1] */
    float alpha;      /* Robin parameter of the inner block boundaries, > 0 [0.5] (Section 3) */
    int downsample;   /* mask-value downsampling: 0 modified [default], 1 naive (Section 4.3) */
    int stop_rule;    /* DI_STOP_* [DI_STOP_ERROR_ESTIMATE] */
    int profile;      /* 1: time every finest-level ORAS block launch with CUDA events
                         recorded on the call's stream (see di_get_profile) [0] */
    int precision;    /* DI_PREC_*: the local CG iterates and the coarse levels' storage
                         [DI_PREC_FP32]; the residual that starts each local solve and
                         the update of u are computed in FP32 in every mode */
    int schedule;     /* DI_SCHED_* [DI_SCHED_REDUCED_FMG] */
    int smoother;     /* DI_SMOOTH_* [DI_SMOOTH_ORAS] */
    int graph;        /* DI_GRAPH_*: replay of the finest-level V-cycle [DI_GRAPH_ON] */
    int start;        /* DI_START_*: initial iterate [DI_START_CASCADE] */
    int local_iters_coarse; /* CG steps of the local solves on the levels below the finest
                               (smoothing of the error equations and the cascade) [local_iters] */
    float local_stop; /* with DI_STOP_ERROR_ESTIMATE: a block's local CG stops early once the
                         2-norm of its residual (per channel, over the block's pixels) is at
                         most local_stop * tol gray -- a local correction that small is
                         below what the stop rule resolves (Section 3.1 stops the local
                         solves on their residual too); < 0 disables [0.2] */
    int refine_fp64;  /* 1: the residuals of the finest grid (the block solves' start, the
                         restriction to the first coarse level, the relative-residual stop
                         rule) are formed in FP64 from the FP32 iterate and rounded once --
                         the outer refinement for tolerances near FP32's resolution of
                         values up to 255; FP64 is used nowhere else [0] */
    int local_iters_cascade; /* CG steps of the local solves of the cascade's iteration on the
                                finest level, the one after the interpolation from the first
                                coarse level (its start has the decode's largest residual, so
                                the local stop ends none of them early) [local_iters] */
} di_config;

/* Statistics of the last di_inpaint call on a context. */
typedef struct {
    int levels;            /* levels of the full pyramid (coarsest fits one block) */
    int levels_used;       /* levels down to the first one without unknown pixels */
    int cycles;            /* V-cycles run after the cascade */
    int converged;         /* 1 if the stop rule was met */
    float est_error;       /* last error estimate (gray levels), DI_STOP_ERROR_ESTIMATE */
    float rel_residual[4]; /* final ||b - A u||_2 / ||b||_2 per channel (if computed) */
    long long unknowns;    /* unknown pixels on the finest level */
    int status;            /* di_status of the call */
} di_stats;

/* Static plan of a solve, computed on the host without touching a GPU. */
typedef struct {
    int levels;                /* pyramid depth: halve (rounding up) until max(w, h) <= B */
    int width[24], height[24]; /* level sizes, level 0 = the image */
    int blocks_x[24], blocks_y[24]; /* ORAS blocks per axis: ceil((n - o) / (B - o)), >= 1 */
    long long local_problems;  /* blocks x channels on level 0 (36852 for 4K RGB, B=32, o=6,
                                  Section 3.1) */
    long long workspace_bytes; /* device bytes di_inpaint allocates for this image */
} di_plan_info;

/* Fill *out for an image of width x height x channels under cfg (NULL =
 * defaults).  Pure host code; usable to size device memory before a solve. */
di_status di_plan(const di_config *cfg, int width, int height, int channels,
                  di_plan_info *out);

/* Create a context bound to CUDA device `device`.  cfg may be NULL (all
 * defaults).  Workspace (pyramids, block-weight buffers) is allocated lazily
 * by di_inpaint and grows with the largest image seen; it is freed by
 * di_destroy. */
di_status di_create(const di_config *cfg, int device, di_ctx **out);

/* Destroy a context and free its workspace; NULL is allowed. */
void di_destroy(di_ctx *ctx);

/* Inpaint f (known where c != 0) into u: the full decoder path.
 *  f: device [channels][height][width] float32, read only at mask pixels.
 *  c: device [height][width] uint8.
 *  u: device output, same layout as f; must not overlap f.  On DI_OK and on
 *     DI_ERR_NOT_CONVERGED it holds the solution (mask pixels equal f
 *     exactly).
 *  tol: target of the stop rule (gray levels for the error estimate, a ratio
 *     for the relative residual), > 0.
 * How it runs.  Device-driven (the default: cfg.graph = DI_GRAPH_ON with the
 * reduced-FMG schedule, no profiling, pre + post even and an image larger
 * than one block): the whole decode is one CUDA graph launch on `stream` --
 * pyramid, cascade and the V-cycle loop, with the stop rule evaluated on the
 * device after every cycle (a WHILE node) and the levels in use and the
 * cascade's start chosen on the device from the mask (IF / SWITCH nodes), so
 * no host round trip happens during the decode.  The graph is captured on
 * the first call with a given (f, c, u, size, tol) and replayed by later
 * calls with the same buffers (a context keeps the last 16); the buffers'
 * contents may change between calls.  di_inpaint then waits for the stream
 * once, at the end.  Host-driven (every other configuration): the host
 * evaluates the stop rule, waiting for the stream after the pyramid and once
 * per V-cycle.  Both give bit-identical results.  The call returns with the
 * work finished. */
di_status di_inpaint(di_ctx *ctx, const float *f, const uint8_t *c, int width, int height,
                     int channels, float tol, float *u, void *stream);

/* di_inpaint without the final wait: on the device-driven path the call
 * enqueues the decode on `stream` and returns DI_OK at once (argument errors
 * are still reported synchronously); the decode's status (DI_OK,
 * DI_ERR_NOT_CONVERGED, DI_ERR_EMPTY_MASK, DI_ERR_TIMEOUT) is in
 * di_stats.status, which di_get_stats waits for.  On the host-driven path it
 * behaves like di_inpaint.  The context's workspace serves one decode at a
 * time: enqueue the calls of one context on one stream (or order them), and
 * keep f, c and u valid until the work is done. */
di_status di_inpaint_async(di_ctx *ctx, const float *f, const uint8_t *c, int width,
                           int height, int channels, float tol, float *u, void *stream);

/* Statistics of the last di_inpaint / di_inpaint_async call (after an
 * asynchronous call, this waits for its work first). */
di_status di_get_stats(const di_ctx *ctx, di_stats *out);

/* Kernel counters of a context, accumulated over di_inpaint calls since the
 * last di_reset_profile.  launches counts every kernel the library enqueued
 * (all contexts of the process, since the library has one launch counter).
 * The oras_* fields are filled only when cfg.profile = 1: number of
 * finest-level ORAS block-kernel launches, their summed duration (from CUDA
 * events on the launching stream, so they include nothing but that kernel),
 * the image pixel-channels they processed, their local problems (blocks x
 * channels) and the local CG steps those problems completed (a block stops
 * before the step limit at its residual floor or the cfg.local_stop level).
 * Read after the decoding stream's work has completed. */
typedef struct {
    long long launches;
    long long oras_l0_launches;
    double oras_l0_ms;
    long long oras_l0_pixel_channels;
    long long oras_l0_cg_steps;  /* local CG steps completed, summed over the local problems */
    long long oras_l0_tasks;     /* local problems (blocks x channels) of those launches */
    long long device_decodes;    /* decodes run as one device-driven graph (see di_inpaint) */
    long long oras_l0_prolong;   /* of the oras_l0 launches, those that also formed the
                                    prolonged start (see di_prolong_oras_iteration) */
    long long reserved[1];
} di_profile;

di_status di_get_profile(const di_ctx *ctx, di_profile *out);
di_status di_reset_profile(di_ctx *ctx);

/* Human-readable name of a status code (static storage). */
const char *di_status_string(di_status s);

/* Last CUDA error text seen by the context (static per context, may be ""). */
const char *di_last_error(const di_ctx *ctx);

/* ------------------------------------------------------------------------
 * Batched and served decoding.  The paper decodes one image at a time; these
 * schedule many di_inpaint calls over a pool of worker slots, each with its
 * own context (resident pyramids and workspace), CUDA stream and host thread,
 * so frames overlap on the GPU.  A frame's result does not depend on what
 * else runs: it is bit-identical to decoding it alone.
 * ------------------------------------------------------------------------ */

/* One image of a batch: device pointers as for di_inpaint; status and cycles
 * are written back. */
typedef struct {
    const float *f;
    const uint8_t *c;
    int width, height, channels;
    float tol;
    float *u;
    int status; /* out: di_status of this image */
    int cycles; /* out: V-cycles used */
} di_image;

/* Decode n images.  When the configuration allows the batched form (see
 * di_batch_create) the batch runs as one di_batch graph; otherwise the images
 * are spread over up to `concurrency` worker slots (0 = 4), largest first.
 * The work starts after what is already queued on `stream` and the call
 * returns when every image is done (`stream` then also waits for it).
 * Returns DI_OK, or the first non-OK image status. */
di_status di_inpaint_batch(const di_config *cfg, int device, di_image *imgs, int n,
                           int concurrency, void *stream);

/* The batched form: the n images of a batch (device pointers, uneven sizes,
 * 1..4 channels, each with its own tol) decoded together, with ONE kernel
 * launch per step of the method over every image -- the pyramid level by
 * level, the cascade level by level, then per V(1,1)-cycle one restriction,
 * one block-kernel and one prolongation launch per level -- and the whole
 * batch captured once into one CUDA graph whose V-cycle loop (a WHILE node)
 * ends when every image's stop rule holds; an image drops out of the cycles
 * as soon as its own rule holds.  The block kernel is persistent over a task
 * list of (image, block, channel) units of all images.  di_batch_create
 * plans the workspace of these images and captures the graph (the buffers,
 * sizes and tolerances become part of it; their contents may change between
 * runs).  Configurations: 32x32 blocks, overlap 2, FP32, the reduced FMG
 * with V(1,1)-cycles, the error-estimate or fixed-cycle stop rule, images of
 * at least two levels; other configurations return DI_ERR_INVALID_ARG (use
 * di_pool_inpaint).  Each image's result equals its single-image decode. */
typedef struct di_batch di_batch;
di_status di_batch_create(const di_config *cfg, int device, const di_image *imgs, int n,
                          di_batch **out);
/* One decode of the batch: imgs must be the images it was created for; their
 * status and cycles are filled.  Waits for the work; returns DI_OK or the
 * first non-OK image status, or DI_ERR_TIMEOUT (every image's status too)
 * when a bounded device-side wait of the block kernel ran out, in which case
 * every output of the run is undefined. */
di_status di_batch_run(di_batch *b, di_image *imgs, int n, void *stream);
void di_batch_destroy(di_batch *b);

/* A persistent pool of `concurrency` decoder slots (0 = 4), each with its own
 * context, stream and host thread, reused by every di_pool_inpaint call, so
 * the slots' workspaces and graphs stay resident between batches.
 * di_inpaint_batch is create + one call + destroy.  One batch at a time per
 * pool (concurrent calls on one pool serialise). */
typedef struct di_pool di_pool;
di_status di_pool_create(const di_config *cfg, int device, int concurrency, di_pool **out);
di_status di_pool_inpaint(di_pool *pool, di_image *imgs, int n, void *stream);
void di_pool_destroy(di_pool *pool);

/* Search space of the autotuner: candidate values per parameter (an empty
 * list, count 0, keeps the base configuration's value).  blocks: B;
 * overlaps: o; local_iters: CG steps of each local solve on the finest level;
 * smoothing: the V-cycle type V(k, k) -- k pre- and k post-smoothing steps;
 * schedules: DI_SCHED_REDUCED_FMG or DI_SCHED_FULL_FMG (the cycle scheme). */
typedef struct {
    const int *blocks;      int nblocks;
    const int *overlaps;    int noverlaps;
    const int *local_iters; int nlocal_iters;
    const int *smoothing;   int nsmoothing;
    const int *schedules;   int nschedules;
} di_tune_space;

/* Time every combination of the search space on the sample images (`reps`
 * timed passes after one warm-up pass, CUDA events) and return the fastest
 * configuration whose decodes all converge, with its mean time per pass.
 * Combinations that are not valid configurations are skipped.  Returns
 * DI_ERR_NOT_CONVERGED if none qualifies. */
di_status di_autotune_space(const di_config *base, int device, const di_image *sample, int n,
                            const di_tune_space *space, int reps, di_config *best,
                            double *best_ms);

/* di_autotune_space over (block, overlap) pairs only. */
di_status di_autotune(const di_config *base, int device, const di_image *sample, int n,
                      const int *blocks, int nblocks, const int *overlaps, int noverlaps,
                      int reps, di_config *best, double *best_ms);

/* Serving loop: requests with HOST buffers (f, c in; u out) are queued FIFO
 * and started on a free slot once their device footprint (di_plan workspace
 * plus device copies of f, c, u) fits within `mem_budget` bytes next to the
 * requests in flight (0 = no limit; a lone request always starts).  Each
 * slot is a pipeline of three host threads -- copy in, decode, copy out --
 * on streams of its own, with three device buffer sets, so a slot's copies
 * of the next and the previous request overlap its decode.  Host buffers in
 * page-locked memory (cudaMallocHost / cudaHostRegister) are copied by DMA at
 * full speed; pageable buffers work too, with the runtime's slower staged
 * copies.  A request is taken by a slot whose decoder has nothing waiting. */
typedef struct di_server di_server;

typedef struct {
    int status;               /* di_status of the request */
    int cycles;               /* V-cycles used */
    double latency_ms;        /* submit to completion */
    double queue_ms;          /* submit to start */
    long long footprint_bytes; /* device bytes charged against the budget */
    /* the slot's stages after the start (their sum with queue_ms is latency_ms): */
    double copy_in_ms;        /* host-to-device copy of f and c */
    double wait_decode_ms;    /* until the slot's decoder takes it */
    double decode_ms;         /* the decode, its status and statistics */
    double wait_out_ms;       /* until the slot's output stage takes it */
    double copy_out_ms;       /* device-to-host copy of u */
} di_request_info;

di_status di_server_create(const di_config *cfg, int device, int slots, long long mem_budget,
                           di_server **out);
/* Queue one request; the host buffers must stay valid until di_server_wait
 * returns for its ticket. */
di_status di_server_submit(di_server *srv, const float *f, const uint8_t *c, int width,
                           int height, int channels, float tol, float *u, long long *ticket);
/* Block until the request finished; fills *info (nullable).  Each ticket can
 * be waited for once. */
di_status di_server_wait(di_server *srv, long long ticket, di_request_info *info);
/* Finish the queued requests, stop the workers and free everything. */
void di_server_destroy(di_server *srv);

/* ------------------------------------------------------------------------
 * Single steps of the path.  Each runs one kernel (or one kernel pair) of the
 * solver on caller buffers; di_inpaint composes them.  They exist so each step
 * can be checked on its own.
 * ------------------------------------------------------------------------ */

/* Mask downsampling by 2x2 max pooling (Section 4.3, "Mask Downsampling").
 * c: [h][w]; cH: [ceil(h/2)][ceil(w/2)] output.  A coarse pixel is known iff
 * any of its (up to four, fewer on odd edges) fine children is. */
di_status di_mask_downsample(const uint8_t *c, int width, int height, uint8_t *cH,
                             void *stream);

/* Mask-value downsampling (Section 4.3).  b: [ch][h][w] values, read only
 * where c != 0; cH: the downsampled mask; bH: [ch][ceil(h/2)][ceil(w/2)]
 * output, 0 where cH == 0.  modified = 1: weights c (4 - masks of the four
 * direct neighbours; fine masks inside the coarse cell, coarse masks across
 * it, out-of-image neighbours unmasked), falling back to the naive average
 * where a masked coarse cell gets total weight 0; modified = 0: the naive
 * average of the masked children. */
di_status di_values_downsample(const uint8_t *c, const float *b, int width, int height,
                               int channels, const uint8_t *cH, float *bH, int modified,
                               void *stream);

/* One level of the pyramid in one pass, as the decoder runs it (Section 4.3):
 * cH = the 2x2 max pooling of c (as di_mask_downsample), bH = the mask-value
 * downsampling of (c, b) with the modified (1) or naive (0) weights (as
 * di_values_downsample; b and bH NULL: masks only), bits = cH bit-packed,
 * ceil(ceil(w/2) / 32) + 1 uint32 words per coarse row (bit x of word k = column
 * 32k + x known or beyond the image; the last word of a row all ones), and
 * *unknown (device, nullable; not cleared) gains the coarse level's unknown
 * pixels.  Bit-identical to the separate steps. */
di_status di_pyramid_level(const uint8_t *c, const float *b, int width, int height, int channels,
                           uint8_t *cH, float *bH, uint32_t *bits, int modified,
                           unsigned long long *unknown, void *stream);

/* Residual r = b - A u with A = C + (I - C) L (Algorithm 2 step 1, eq. 2.6),
 * and its squared 2-norm per channel.
 *  b: [ch][h][w]: at mask pixels the Dirichlet value, at unknown pixels the
 *     right-hand side of L u = b; if rhs_zero != 0 the right-hand side at
 *     unknown pixels is taken as 0 and b is read only at mask pixels.
 *  r: [ch][h][w] output, may be NULL (norm only).
 *  norm2: device double[channels] output.
 * Needs a context for its reduction workspace; the sums are formed in a fixed
 * order (deterministic). */
di_status di_residual_norm(di_ctx *ctx, const float *u, const float *b, int rhs_zero,
                           const uint8_t *c, int width, int height, int channels, float *r,
                           double *norm2, void *stream);

/* The residual and squared norm of di_residual_norm, for callers that cannot
 * allocate device memory when they call: real-time decoders that fix their
 * device footprint before they start, code running while another component
 * owns the device allocator, or paths that cannot afford the device-wide
 * synchronisation cudaFree implies.  It takes no context and allocates
 * nothing (no cudaMalloc, no cudaFree, no allocating library routine).
 * The paper has no counterpart; this is a deployment variant.
 *  Scratch: the per-CTA partial sums live in one array of
 *    DI_NOALLOC_PARTIALS doubles (1 MiB) compiled into the library, which
 *    every GPU that loads the library keeps until the process exits.
 *  Limit: ceil(width/32) * ceil(height/8) * channels <= DI_NOALLOC_PARTIALS
 *    (3840x2160 with up to 4 channels fits); a larger call returns
 *    DI_ERR_INVALID_ARG before touching the GPU.
 *  Device and set-up: the kernels run on the calling thread's current
 *    device, so `stream` must belong to that device (a stream of another
 *    device makes the launch fail with DI_ERR_CUDA).  The first call on a
 *    device (and the first after its context was destroyed and created
 *    again, e.g. by a device reset) looks up the array's device address with
 *    that device current, so make that first call before any stream capture
 *    on the device.
 *  Sharing: every call uses the same array and leaves its partial sums
 *    there; nothing in it needs to start at zero.  Calls whose kernels
 *    overlap on the GPU (different streams or host threads without ordering)
 *    race on the array and can return wrong norms: order them on one stream
 *    or synchronise between them.
 * Other arguments and results as for di_residual_norm. */
#define DI_NOALLOC_PARTIALS 131072
di_status di_residual_norm_noalloc(const float *u, const float *b, int rhs_zero,
                                   const uint8_t *c, int width, int height, int channels,
                                   float *r, double *norm2, void *stream);

/* Residual restriction (Algorithm 3 steps 2-3, Section 4.4): for every coarse
 * cell with cH == 0, rH = 4 * mean over its fine children of (b - A u) (the
 * factor 4 = (H/h)^2 rescales the unit-spacing stencil to the coarse
 * spacing); rH = 0 where cH == 1.  fp64 = 1: the children's residuals are
 * formed and summed in FP64 and rounded once (the finest-grid refinement
 * residual of cfg.refine_fp64).  Other arguments as for di_residual_norm. */
di_status di_restrict_residual(const float *u, const float *b, int rhs_zero,
                               const uint8_t *c, int width, int height, int channels,
                               const uint8_t *cH, float *rH, int fp64, void *stream);

/* Cell-centred bilinear prolongation (Section 4.4) from uH
 * [ch][ceil(h/2)][ceil(w/2)] to the fine grid [ch][h][w] (weights 9/16, 3/16,
 * 3/16, 1/16, coarse indices clamped at the border).
 *  mode 0 (cascadic): u = b at mask pixels, P uH elsewhere (b read only at
 *         mask pixels).
 *  mode 1 (correction): u += P uH at unknown pixels, u unchanged at mask
 *         pixels (b unused, may be NULL). */
di_status di_prolong(const float *uH, const float *b, const uint8_t *c, int width, int height,
                     int channels, float *u, int mode, void *stream);

/* One ORAS iteration (Algorithm 2) with the context's block size, overlap
 * and alpha: r = b - A u_in; on every block i, `local_iters` steps of plain
 * (unpreconditioned) conjugate gradients (from 0, Section 3.1) on A_i v_i = R_i r, A_i = A restricted to the block with Robin rows
 * on inner block edges (Section 3); u_out = u_in + sum_i R_i^T D_i v_i with
 * the separable linear partition-of-unity weights of Section 3.1.
 *  u_in: [ch][h][w]; must equal b at mask pixels (then r = 0 there).
 *  b, rhs_zero: as for di_residual_norm.
 *  u_out: [ch][h][w] output; must not overlap u_in.
 * Deterministic: overlapping contributions are summed in a fixed order. */
di_status di_oras_iteration(di_ctx *ctx, const float *u_in, const float *b, int rhs_zero,
                            const uint8_t *c, int width, int height, int channels,
                            int local_iters, float *u_out, void *stream);

/* A prolongation (Section 4.4) fused with the ORAS iteration (Algorithm 2)
 * that follows it in the method: u_out = ORAS(s) with the start s formed from
 * u_in and P uH inside the block kernel, which the decoder does whenever this
 * form applies.
 *  mode 1 (the V-cycle's correction step before the first post-smoothing):
 *         s = u_in + P uH at unknown pixels, u_in at mask pixels; equals
 *         di_prolong (mode 1) on a copy of u_in followed by
 *         di_oras_iteration, bit for bit.
 *  mode 0 (the cascade's interpolation before its smoothing step, u_in = b):
 *         s = u_in at mask pixels, P uH elsewhere (u_in not read there);
 *         equals di_prolong (mode 0, b = u_in) followed by
 *         di_oras_iteration, bit for bit.
 *  uH: [ch][ceil(h/2)][ceil(w/2)] coarse field (FP32).  u_in is not modified.
 *  Other arguments as for di_oras_iteration.
 * Requires the context's block size 32, FP32 precision and an even block
 * stride (32 - overlap); DI_ERR_INVALID_ARG otherwise. */
di_status di_prolong_oras_iteration(di_ctx *ctx, const float *uH, int mode, const float *u_in,
                                    const float *b, int rhs_zero, const uint8_t *c, int width,
                                    int height, int channels, int local_iters, float *u_out,
                                    void *stream);

/* Fault-path self test (no counterpart in the paper): launches one CTA that
 * waits, with the same bounded mbarrier wait as the 32x32 block kernel
 * (`limit` polls), on a barrier that nothing completes, and reports what the
 * decoder would: DI_ERR_TIMEOUT when the wait ran out (the expected result),
 * DI_OK if it completed, DI_ERR_CUDA on a runtime error.  Nothing faults and
 * nothing stays in flight; the device stays usable.  Exists so that tests can
 * exercise the timeout path on a GPU. */
di_status di_selftest_bounded_wait(int device, int limit, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DI_H */
