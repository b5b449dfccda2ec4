/*
 * rgbid.h - C ABI of the GB300 (sm_103a) library for RGBiD-SLAM's dense
 * frame-to-keyframe alignment in inverse-depth parametrisation and keyframe
 * fusion (Gutierrez-Gomez & Guerrero, arXiv 1807.08271).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Notation is the paper's: A (the reference, normally the keyframe) and B
 *    (the current frame); a pose T = A_T_B is a row-major 4x4 double matrix
 *    that maps B's coordinates into A's (X_A = R X_B + t).
 *  - Images are row-major.  I is intensity in [0, 1]; W is inverse depth in
 *    1/m with W == 0 (or any W <= 0) meaning "no measurement" (a hole).  A
 *    pixel whose I or W is not a finite number (NaN, +-inf) is a hole too: the
 *    pyramid and the keyframe initialisation store it with W = 0 (and I = 0
 *    where I is not finite), and fusion never reads it as a measurement.
 *    `pitch` arguments count ELEMENTS per row (>= width).
 *  - Ownership: the caller allocates and owns every buffer (planes, pyramid
 *    storage, workspace, results).  The library keeps no global state and
 *    never allocates device memory.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *    default stream).  Every call only enqueues work on that stream and
 *    returns; results are valid once the stream reaches that point.
 *  - Errors: argument errors are reported synchronously as the return value
 *    (nothing is enqueued).  A failed kernel launch returns RGBID_ERR_CUDA.
 *    Numerical outcomes (degenerate steps) are written to the result struct's
 *    `status` field on the device.  No C++ exception crosses this ABI.
 *  - Alignment: every device pointer must be a multiple of its element size
 *    (float planes 4 bytes; an interleaved pyramid level its pixel size, 8 or
 *    4 bytes; doubles, result records and batch items 8 bytes); workspaces and
 *    pyramid storage 256 bytes.  A misaligned argument is rejected before
 *    anything is enqueued (RGBID_ERR_INVALID_ARG, or RGBID_ERR_WORKSPACE for a
 *    workspace).  Pointers inside device-resident batch items are checked on
 *    the device: the item reports RGBID_ERR_INVALID_ARG (a misaligned result
 *    record is skipped like NULL).
 *  - Intrinsics must be finite with fx, fy > 0 (else RGBID_ERR_INVALID_ARG).
 */
#ifndef RGBID_H
#define RGBID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RGBID_MAX_LEVELS 6
#define RGBID_MAX_SAMPLES 19200   /* N of the paper's systematic sample ("Error distribution and robust optimisation") */

typedef enum {
    RGBID_OK = 0,
    RGBID_ERR_INVALID_ARG = 1,
    RGBID_ERR_CUDA = 2,
    RGBID_ERR_WORKSPACE = 3,     /* workspace / storage too small or misaligned */
    RGBID_ERR_DEGENERATE = 4,    /* device status: a step was skipped (too few residuals or H not SPD) */
    RGBID_ERR_TIMEOUT = 5,       /* device status: a bounded device-side wait gave up */
    RGBID_ERR_UNSUPPORTED = 6
} rgbid_status;

/* Pinhole intrinsics (level 0 unless stated). */
typedef struct {
    double fx, fy, cx, cy;
} rgbid_intrinsics;

/* Storage precision of pyramid levels. */
typedef enum {
    RGBID_PLANES_F32 = 0,        /* (float I, float W) pairs: 8 bytes per pixel */
    RGBID_PLANES_BF16_F16 = 1    /* (bf16 I, fp16 W) pairs: 4 bytes per pixel */
} rgbid_precision;

/* One pyramid level: an interleaved (I, W) plane in device memory. */
typedef struct {
    int width, height;
    int pitch;                   /* pixels per row */
    int pad_;
    rgbid_intrinsics K;          /* intrinsics at this level */
    void* IW;                    /* device pointer, layout per rgbid_precision */
} rgbid_level;

/* Pyramid descriptor (host struct; the pixel data lives in caller storage). */
typedef struct {
    int levels;
    int precision;               /* rgbid_precision */
    rgbid_level lv[RGBID_MAX_LEVELS];   /* index 0 = finest */
} rgbid_pyramid;

/* Optional per-kernel timing of rgbid_align: the library records the caller's
 * CUDA events (cudaEvent_t passed as void*) on the call's stream immediately
 * before and after every launch of the selected kernel, appending after the
 * `count` pairs already used (at most `capacity`), and adds the algorithmic
 * units those launches process to `units` (pixels of the level for the sweep,
 * systematic-sample pixels for the robust-scale kernel). */
typedef enum {
    RGBID_KERNEL_SWEEP = 0,      /* fused warp + residual + Jacobian + weight + reduce (+ solve) */
    RGBID_KERNEL_ROBUST = 1,     /* systematic sample + (mu, sigma, nu) */
    RGBID_KERNEL_BATCH = 2,      /* the persistent kernel of rgbid_align_batched (units are not counted) */
    RGBID_KERNEL_LEVEL = 3,      /* the persistent level kernel of rgbid_align (units: level pixels x iterations) */
    RGBID_KERNEL_SPLIT = 4       /* the split level kernel of rgbid_align (units: level pixels x iterations) */
} rgbid_kernel_id;

typedef struct {
    void** ev_start;             /* cudaEvent_t[capacity] */
    void** ev_end;               /* cudaEvent_t[capacity] */
    int capacity;
    int kernel;                  /* rgbid_kernel_id */
    int count;                   /* in/out: event pairs used so far */
    int pad_;
    long long units;             /* in/out: algorithmic units of the timed launches */
} rgbid_timing;

/* Where B is warped ("Iterative optimisation": the maps of B warped towards A
 * are downsampled to the level of the current iteration).
 * RGBID_WARP_PER_LEVEL warps B's level-l map with K_l at level l (the default).
 * RGBID_WARP_FULL_RESOLUTION warps B at level 0 for every iteration and reduces
 * the warped maps to level l by the pyramid's rule, each with its own validity
 * (a level-l value is the mean of its valid children and is valid when one
 * child is); a level-l pixel's masks are A's conditions there plus that
 * validity.  Every iteration then warps all level-0 pixels.  rgbid_align and
 * rgbid_eval_step take both; the batched form takes the default only. */
typedef enum {
    RGBID_WARP_PER_LEVEL = 0,
    RGBID_WARP_FULL_RESOLUTION = 1
} rgbid_warp_mode;

/* Alignment schedule and robust-estimation constants. */
typedef struct {
    int levels;                  /* levels used, coarse to fine (<= pyramid levels) */
    int iters[RGBID_MAX_LEVELS]; /* Gauss-Newton iterations per level, index 0 = finest */
    int scale_iters;             /* fixed-point iterations for (mu, sigma); default 10 */
    int bisect_steps;            /* bisection halvings for nu; default 20 */
    int sample_cap;              /* systematic sample size cap, 1..RGBID_MAX_SAMPLES; default 19200 */
    int estimate_nu;             /* 1: bisection for nu per channel; 0: nu = nu0 */
    int min_valid;               /* minimum count of valid residuals (I and W together) for a step */
    int warp_mode;               /* rgbid_warp_mode; default RGBID_WARP_PER_LEVEL */
    double nu0, nu_lo, nu_hi;    /* 5, 2, 10; needs (nu_lo + nu_hi) >= 1.4 (nu_hi - nu_lo) */
    rgbid_timing* timing;        /* optional kernel timing (NULL: none) */
    const int* level_iters;      /* optional DEVICE array of RGBID_MAX_LEVELS ints read by the kernels
                                    (rgbid_align only): level l runs min(iters[l], level_iters[l])
                                    iterations; the launches of the others exit at once.  NULL: iters. */
    int no_level_kernel;         /* 0 (default): rgbid_align runs each level in one launch where it can.
                                    A level whose systematic sample is every pixel (w h <= sample_cap,
                                    and <= 20480 pixels) runs in one persistent 16-CTA cluster: each
                                    iteration warps the level once, takes its residuals as the sample,
                                    and solves inside the cluster.  A larger level runs in the split
                                    kernel, a cooperative launch of one such cluster (solve, sample,
                                    robust parameters) and helper CTAs that evaluate every pixel's
                                    terms while the cluster estimates the parameters; consecutive
                                    such levels share one launch.  1: every level
                                    by the per-iteration robust-scale and sweep kernels.  All compute
                                    the same steps (sums in another order). */
    int pad2_;
} rgbid_align_params;

/* Result of an alignment (or of one evaluated step).  Lives in device memory
 * (or mapped pinned host memory) and is written by the device. */
typedef struct {
    double T[16];                /* final A_T_B (for rgbid_eval_step: the input pose) */
    double H[36];                /* normal matrix of the last step (full, symmetric) */
    double g[6];                 /* sum w J^T r(p,0) of the last step; the step solves H xi = -g */
    double mu[2], sigma[2], nu[2];  /* robust parameters of the last step: [I, W] */
    double cost;                 /* sum w r^2 of the last step */
    int n_valid[2];              /* residuals that passed mask_I / mask_W in the last step */
    int iters_done;
    int iters_skipped;           /* steps skipped as degenerate */
    int status;                  /* rgbid_status: RGBID_OK or RGBID_ERR_DEGENERATE */
    int pad_;
} rgbid_align_result;

/* Human-readable name of a status code (static string, never NULL). */
const char* rgbid_status_string(int status);

/* Fill `p` with the defaults: 3 levels, iters {5, 5, 10} (finest first),
 * 10 scale iterations, 20 bisection steps, sample cap 19200, nu estimated,
 * nu0 = 5, nu in [2, 10], min_valid 60. */
void rgbid_default_params(rgbid_align_params* p);

/* ---------------------------------------------------------------- pyramid
 * Image pyramid ("Dense motion estimation", "Iterative optimisation": the
 * maps are downsampled at each level and their gradients taken there).
 * Level l+1 is the 2x2 box mean of level l (odd sizes drop the last
 * row/column); W averages only its valid children and is 0 if none; the
 * intrinsics follow f <- f/2, c <- (c + 0.5)/2 - 0.5.  Gradients are not
 * stored: the alignment takes central differences on the fly.
 */

/* Bytes of caller storage needed for a pyramid. */
size_t rgbid_pyramid_bytes(int width, int height, int levels, int precision);

/* Build a pyramid from planar float I0/W0 (device, `pitch0` elements per row)
 * into `storage` (device, >= rgbid_pyramid_bytes, 256-byte aligned) and fill
 * the host descriptor `out`.  Levels need width, height >= 4.
 * Errors: INVALID_ARG (sizes, levels, NULL pointers), WORKSPACE (storage). */
int rgbid_build_pyramid(const float* I0, const float* W0, int pitch0, int width, int height,
                        rgbid_intrinsics K0, int levels, int precision,
                        void* storage, size_t storage_bytes, rgbid_pyramid* out, void* stream);

/* ---------------------------------------------------------------- alignment
 * Coarse-to-fine IRLS Gauss-Newton alignment ("Dense motion estimation"):
 * per iteration B is warped towards A with the current estimate (inverse
 * geometric warping, eq. 3d_registration), the Student-t location, scale and
 * robustness (mu, sigma, nu) of the photometric and inverse-depth residuals
 * are estimated on the <= 19200-pixel systematic sample, every pixel's
 * residuals (eqs. res_int, res_depth), Jacobians and weights (eq.
 * minimisationIRLS with the normal weight lambda_n) are reduced into H xi = -g,
 * and T <- exp(xi)^-1 T with the decoupled SE(3) exponential.
 */

/* Workspace bytes needed by rgbid_align / rgbid_eval_step for this reference
 * (more with RGBID_WARP_FULL_RESOLUTION, whose sweeps take one row per thread
 * on every level). */
size_t rgbid_align_workspace_bytes(const rgbid_pyramid* ref, const rgbid_align_params* params);

/* Kernel launches one rgbid_align call with these arguments enqueues on the
 * current device (the initialisation, the per-iteration robust-scale and sweep
 * kernels or one level kernel per level, and the closing launch), or -1 when
 * the arguments are invalid.  Host only. */
int rgbid_align_launches(const rgbid_pyramid* ref, const rgbid_align_params* params);

/* Align `cur` (B) to `ref` (A).  Both pyramids must have the same size,
 * precision and intrinsics.  `T_init` is 16 doubles (row-major A_T_B): a host
 * pointer read during the call when `T_init_on_device` is 0, a device pointer
 * read by the first kernel when it is 1, or NULL for the identity.
 * `workspace` (device, >= rgbid_align_workspace_bytes, 256-byte aligned) is
 * scratch for the duration of the call.  `d_result` is device memory written
 * by the device; on a degenerate step the pose is kept, iters_skipped grows
 * and status becomes RGBID_ERR_DEGENERATE.  Calls sharing a workspace must
 * not overlap on the device. */
int rgbid_align(const rgbid_pyramid* ref, const rgbid_pyramid* cur,
                const double* T_init, int T_init_on_device,
                const rgbid_align_params* params, void* workspace, size_t workspace_bytes,
                rgbid_align_result* d_result, void* stream);

/* Allocation-free variant of rgbid_align, for callers that cannot allocate device
 * memory or keep a workspace: code running under a no-allocation policy (a
 * real-time tracking loop, a plugin inside a host application that owns every
 * device allocation) and callers without a CUDA allocator of their own.  The
 * paper has no counterpart to this entry point.
 * It behaves as rgbid_align but takes its scratch from a fixed device array
 * inside the library (RGBID_NOALLOC_SCRATCH_BYTES, 1 MiB, held by every GPU
 * that loads the library until the process exits) and calls no allocator.
 * Inputs and outputs are still the caller's.  The first call on a device,
 * with that device current, looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Returns RGBID_ERR_WORKSPACE when the reference's finest level needs more
 * scratch than the array holds (about 4 million pixels; about 1 million with
 * RGBID_WARP_FULL_RESOLUTION), RGBID_ERR_CUDA if the
 * look-up fails.  Every call shares the one array: calls whose work overlaps on
 * the GPU (other streams, other host threads) race and must be serialised by
 * the caller.  Each call resets the scratch fields that must start at zero. */
#define RGBID_NOALLOC_SCRATCH_BYTES (1024u * 1024u)
int rgbid_align_noalloc(const rgbid_pyramid* ref, const rgbid_pyramid* cur,
                        const double* T_init, int T_init_on_device,
                        const rgbid_align_params* params,
                        rgbid_align_result* d_result, void* stream);

/* ---------------------------------------------------------------- batched alignment
 * Many independent alignments in ONE persistent kernel launch: the
 * verification of loop-closure candidates ("Loop closure": the current frame
 * is aligned densely against each candidate keyframe from the RANSAC pose),
 * or the frame-to-keyframe alignments of several concurrent sequences.  Each
 * alignment runs the same coarse-to-fine IRLS Gauss-Newton iteration as
 * rgbid_align; pairs may differ in resolution, levels and iteration counts.
 *
 * Execution: a thread-block cluster of `cluster` CTAs takes one pair at a time
 * from a device work queue (array order; put the largest pairs first) and
 * keeps the whole alignment on chip: sample residuals in shared memory, every
 * reduction (robust scale, the 27 normal-equation terms) exchanged between the
 * cluster's CTAs through distributed shared memory, and the 6x6 solve and pose
 * update repeated identically in every CTA, so no grid-wide synchronisation
 * and no host round trip occurs.  The call is a single kernel launch and can
 * be captured in a CUDA graph.  Device-side waits are bounded in time; a
 * pair whose waits ran out reports RGBID_ERR_TIMEOUT in its result.
 */

/* One pair of a batch.  The array of items lives in DEVICE memory (the caller
 * copies these host descriptors there) and must stay valid until the batch
 * completes; the kernel validates each item and writes RGBID_ERR_INVALID_ARG
 * into the status of an item that fails the rgbid_align argument rules. */
typedef struct {
    rgbid_pyramid ref;           /* A: the keyframe / candidate */
    rgbid_pyramid cur;           /* B: the current frame */
    double T_init[16];           /* initial A_T_B, row-major */
    int levels;                  /* levels used, coarse to fine (<= both pyramids' levels) */
    int iters[RGBID_MAX_LEVELS]; /* Gauss-Newton iterations per level, index 0 = finest (0..10000) */
    int pad_;
    rgbid_align_result* result;  /* device pointer, 8-byte aligned; an item with a NULL or
                                    misaligned result is skipped */
} rgbid_batch_item;

/* Launch shape of the persistent kernel (see rgbid_batch_autotune). */
typedef struct {
    int cluster;                 /* CTAs (256 threads each) per alignment: 4, 8 or 16; 0 = 8 */
    int rows_per_warp;           /* sweep tile height per warp: 1, 2 or 4 (tiles are 32 pixels wide); 0 = 2 */
    int n_clusters;              /* persistent clusters launched; 0 = as many as are resident at once.
                                    Always capped at the resident maximum and at n_items. */
    int pad_;
} rgbid_batch_config;

/* Workspace of rgbid_align_batched: 256 bytes of device memory holding the
 * queue head.  It must be zero before its first use (e.g. cudaMemset once);
 * every completed batch leaves it zero again.  Batches sharing a workspace
 * must not overlap on the device. */
size_t rgbid_align_batched_workspace_bytes(void);

/* Host-side check of one item (a host copy of the descriptor) against the
 * rules the kernel applies: returns RGBID_OK or RGBID_ERR_INVALID_ARG. */
int rgbid_batch_check_item(const rgbid_batch_item* item, int precision);

/* Number of clusters of this shape that are resident on the current device at
 * once (0 if none fit).  The first query of a shape on a device also sets the
 * kernel's attributes; make it (or rgbid_batch_autotune) before capturing a
 * batch into a CUDA graph.  Errors: INVALID_ARG (shape), CUDA. */
int rgbid_batch_resident_clusters(int precision, const rgbid_batch_config* cfg, int* n_resident);

/* Align every item of `d_items` (device array of n_items; all pyramids of
 * `precision`).  `params` supplies the robust-estimation constants
 * (scale_iters, bisect_steps, sample_cap, estimate_nu, min_valid, nu0, nu_lo,
 * nu_hi) and the optional timing hook; its `levels`/`iters` are ignored (each
 * item carries its own).  `cfg` may be NULL (defaults).  `workspace` is
 * device memory of rgbid_align_batched_workspace_bytes(), 256-byte aligned.
 * Errors: INVALID_ARG (params, cfg, NULL items with n_items > 0), WORKSPACE,
 * UNSUPPORTED (precision, or no cluster of this shape fits), CUDA. */
int rgbid_align_batched(const rgbid_batch_item* d_items, int n_items, int precision,
                        const rgbid_align_params* params, const rgbid_batch_config* cfg,
                        void* workspace, size_t workspace_bytes, void* stream);

/* The project's autotuner for the batched kernel: runs the batch once per
 * candidate shape (cluster 4/8/16 x rows_per_warp 1/2/4 x all or half of the
 * resident clusters) as a warm-up, then `reps` timed runs each (CUDA events on
 * `stream`, synchronising), and returns the shape with the lowest median time
 * in *best and that time in *best_ms.  The items' results hold the last
 * candidate's output afterwards.  Not for use during stream capture. */
int rgbid_batch_autotune(const rgbid_batch_item* d_items, int n_items, int precision,
                         const rgbid_align_params* params, void* workspace, size_t workspace_bytes,
                         int reps, rgbid_batch_config* best, float* best_ms, void* stream);

/* ---------------------------------------------------------------- learned initialiser
 * A small network that proposes the initial twist of an alignment from the
 * 80x60 pyramid level of both frames, with a log-variance saying how far to
 * trust it.  The paper has no learned part; this is the project's extension.
 * When the proposal is confident, the alignment starts from it and skips the
 * coarsest levels; otherwise the plain coarse-to-fine alignment runs
 * unchanged, and in both cases the Gauss-Newton alignment decides the pose.
 *
 * Network (activations NHWC bfloat16, batch first):
 *   x   [B, 60, 80, 4]  I_A - 0.5, W_A, I_B - 0.5, W_B of the 80x60 level
 *   c1..c4  3x3 convolutions (cross-correlation), stride 2, zero padding 1,
 *           4 -> 32 -> 32 -> 64 -> 64 channels, ReLU: 30x40, 15x20, 8x10, 4x5
 *   f1  fully connected 1280 -> 256 (c4 flattened in NHWC order), ReLU
 *   f2  fully connected 256 -> 7: y[0..5] = twist / RGBID_NET_TWIST_SCALE
 *       (translation t then rotation vector w of T = [exp([w]x), t; 0, 1]),
 *       y[6] = s, the log-variance of the scaled twist
 * Loss (mean over the batch): 0.5 exp(-s) |y[0..5] - target|^2 + 3 s.
 * Parameters: one float32 array (master copy); layer l's weights start at
 * rgbid_net_param_offset(l, 0) stored [kh][kw][c_in][c_out] (convolutions)
 * or [in][out] (fully connected), its biases at rgbid_net_param_offset(l, 1);
 * every tensor starts on a multiple of 64 floats.  The forward and backward
 * passes compute on the fifth-generation tensor cores (tcgen05.mma, bfloat16
 * operands in shared memory, FP32 accumulators in tensor memory): weights,
 * inputs, hidden activations and back-propagated activation gradients are
 * rounded to bfloat16 where they are stored; the output, biases and parameter
 * gradients are float32.  The first rgbid_net_workspace_bytes call on a device
 * sets the GEMM kernels' shared-memory attribute there: make it before any
 * stream capture of the passes.
 */
#define RGBID_NET_IN_H 60
#define RGBID_NET_IN_W 80
#define RGBID_NET_IN_C 4
#define RGBID_NET_OUT 7
#define RGBID_NET_LAYERS 6
#define RGBID_NET_TWIST_SCALE 0.1

/* Number of floats of the parameter (and gradient / Adam moment) arrays. */
size_t rgbid_net_param_count(void);

/* Offset (in floats) of layer `layer`'s weights (what = 0) or biases (what = 1); (size_t)-1 if out of range. */
size_t rgbid_net_param_offset(int layer, int what);

/* Workspace bytes for batches of up to `batch` inputs (bfloat16 weights,
 * activations kept for the backward pass, activation gradients). */
size_t rgbid_net_workspace_bytes(int batch);

/* Waits of the network's GEMM kernels on their tensor-core operations that ran
 * out of their ~2 s budget on the current device since the library was loaded
 * (0 in a healthy run; a CTA whose wait runs out still finishes, with a wrong
 * tile).  Synchronises the device; returns (unsigned)-1 if it cannot be read. */
unsigned int rgbid_net_wait_timeouts(void);

/* Fill `params` (device, rgbid_net_param_count floats) with He-uniform weights
 * U(-sqrt(6/fan_in), sqrt(6/fan_in)) drawn from splitmix64(seed, index), biases 0. */
int rgbid_net_init(float* params, unsigned long long seed, void* stream);

/* Network inputs of n batch items (device array, as for rgbid_align_batched):
 * for each item, the level of its ref and cur pyramids that is 80x60 is
 * packed into x (device, n * 60 * 80 * 4 bfloat16, NHWC).  An item without
 * an 80x60 level gets zeros.  Errors: INVALID_ARG. */
int rgbid_net_inputs(const rgbid_batch_item* d_items, int n, int precision, void* x, void* stream);

/* y[batch][7] (float32) of the inputs x (bfloat16 NHWC).  The activations stay
 * in the workspace for a following rgbid_net_backward on the same inputs. */
int rgbid_net_forward(const float* params, const void* x, int batch, float* y,
                      void* workspace, size_t workspace_bytes, void* stream);

/* Parameter gradients (overwritten, float32) for the upstream gradient dy =
 * dL/dy [batch][7], using the activations of the preceding rgbid_net_forward
 * with the same params, x, batch and workspace. */
int rgbid_net_backward(const float* params, const void* x, int batch, const float* dy, float* grad,
                       void* workspace, size_t workspace_bytes, void* stream);

/* The loss above: writes dy = dL/dy [batch][7] and *loss (device float). */
int rgbid_net_loss(const float* y, const float* target, int batch, float* dy, float* loss, void* stream);

/* One Adam step (Kingma & Ba 2015, with bias correction; `step` counts from 1)
 * on params, in place, with moments m and v (device, zero before step 1). */
int rgbid_net_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                   float beta1, float beta2, float eps, void* stream);

/* Turn the network's outputs y [n][7] into the alignments' starting points:
 * item i of `d_out` = item i of `d_in` (device arrays, may not alias), except
 * that an item whose log-variance y[i][6] is below max_log_var[k - 1] (host
 * array of n_tiers thresholds; tier k skips k levels) for some k gets the
 * proposed pose as T_init and zero iterations on its k coarsest levels, for
 * the largest such k (at least the finest level is always kept).  Items in no
 * tier are left as they are (the plain alignment).  skipped (device, n ints,
 * may be NULL) receives the number of levels skipped per item. */
#define RGBID_NET_MAX_TIERS 4
int rgbid_net_plan(const float* y, int n, const float* max_log_var, int n_tiers,
                   const rgbid_batch_item* d_in, rgbid_batch_item* d_out, int* skipped, void* stream);

/* One step at a fixed pose and level, for inspection and parity testing.
 * `T` (host, 16 doubles) is the pose; `robust` (host, 6 doubles
 * mu_I, sigma_I, nu_I, mu_W, sigma_W, nu_W) fixes the robust parameters, or
 * NULL estimates them on the sample as rgbid_align does.  Optional device
 * outputs of width*height elements of that level (row-major, pitch = width):
 * r_I, r_W (residuals r(p, 0), 0 where masked out), mask_I, mask_W (0/1).
 * `d_result` receives H, g, cost, n_valid and the robust parameters used;
 * its pose is `T` and no update is applied. */
int rgbid_eval_step(const rgbid_pyramid* ref, const rgbid_pyramid* cur, int level,
                    const double* T, const double* robust, const rgbid_align_params* params,
                    void* workspace, size_t workspace_bytes,
                    float* r_I, float* r_W, uint8_t* mask_I, uint8_t* mask_W,
                    rgbid_align_result* d_result, void* stream);

/* ---------------------------------------------------------------- covariance
 * Covariance of a motion estimate ("Dense motion estimation", the paragraph
 * after the update rule): one more iteration at the final pose, which does not
 * update it, in which the reference's level 0 {I_A, W_A} is bilateral-filtered
 * before its gradients are taken; Sigma = H_filt^-1.  The iteration estimates
 * (mu, sigma, nu) on the systematic sample at that pose like any other; only
 * the central differences (the Jacobians and the normal weight) read the
 * filtered planes, while the warp, residuals and masks use the unfiltered
 * ones.  The filter's parameters are not given by the paper. */
#define RGBID_BILATERAL_MAX_RADIUS 5
typedef struct {
    int radius;                  /* window half-width in pixels, 0..RGBID_BILATERAL_MAX_RADIUS (0: no filtering) */
    int pad_;
    double sigma_s;              /* spatial sigma, pixels */
    double sigma_r_I;            /* range sigma of intensity */
    double sigma_r_W;            /* range sigma of inverse depth, 1/m */
} rgbid_bilateral;

/* Defaults: radius 2, sigma_s 1.5 px, sigma_r_I 0.1, sigma_r_W 0.01 1/m. */
void rgbid_default_bilateral(rgbid_bilateral* f);

/* Workspace bytes of rgbid_covariance: the alignment workspace plus a float
 * (I, W) plane of the reference's level 0. */
size_t rgbid_covariance_workspace_bytes(const rgbid_pyramid* ref);

/* The covariance iteration of `cur` (B) against `ref` (A) at pose `T` (16
 * doubles, host when `T_on_device` is 0, device when 1, e.g. &d_result->T of
 * the alignment), level 0, with the robust-estimation constants of `params`.
 * Each output pixel of the filter is the mean of its (2r+1)^2 window inside
 * the image weighted by exp(-d^2 / 2 sigma_s^2) exp(-(f(p) - f(q))^2 / 2 sigma_r^2);
 * inverse depth only over valid neighbours, and holes stay holes.
 * Writes `d_result` (device: T, H = H_filt, g, cost, robust parameters and
 * counts of that iteration; status RGBID_ERR_DEGENERATE when H_filt is not
 * positive definite or fewer than params->min_valid residuals are valid) and
 * `d_sigma` (device, 36 doubles row-major: H_filt^-1 in the twist coordinates
 * (t, theta) of the update, or zeros when degenerate).
 * Errors: INVALID_ARG (pyramids and params as rgbid_align; filter values),
 * WORKSPACE, CUDA. */
int rgbid_covariance(const rgbid_pyramid* ref, const rgbid_pyramid* cur, const double* T, int T_on_device,
                     const rgbid_align_params* params, const rgbid_bilateral* filter,
                     void* workspace, size_t workspace_bytes, rgbid_align_result* d_result,
                     double* d_sigma, void* stream);

/* Chebyshev series (in tau = (nu - m)/h over [nu_lo, nu_hi], m and h the
 * interval's centre and half-width) of the sample-independent part of the
 * degrees-of-freedom equation ("Error distribution and robust optimisation",
 * eq. robustnessValue).  With w_i = (nu + 1)/(nu + x_i^2) the equation
 * f(nu) = n c(nu) + sum_i (ln w_i - w_i) reads
 * f(nu) = n g(nu) - sum_i [ln(nu + x_i^2) + w_i], where
 * g(nu) = psi((nu+1)/2) - psi(nu/2) + 1 + ln nu; the alignment adds g's series
 * to the series of the sample sums and bisects on the result.  Computed on the host in FP64 (22 terms, interpolation at 64 Chebyshev
 * nodes) and used by every alignment entry point; exposed so it can be
 * checked.  Writes min(n_out, 22) coefficients g_0.. (plain convention,
 * g = sum_k g_k T_k(tau)) to host memory `out` and returns their number, or
 * -RGBID_ERR_INVALID_ARG, or -RGBID_ERR_UNSUPPORTED for an interval the
 * alignment rejects too ((lo + hi)/(hi - lo) < 1.4). */
int rgbid_nu_constant_series(double nu_lo, double nu_hi, float* out, int n_out);

/* Diagnostic of the device-side failure detection (the paper has no
 * counterpart).  Launches one 4-CTA cluster that runs one round of the
 * alignment's cluster reduction with every CTA withholding its partials, so
 * each CTA's wait runs out of `budget_cycles` (clock64 cycles, <= 2e10), adds 1 to
 * *d_timeouts (device int, not reset) and ends; nothing faults or hangs and the
 * context stays usable.  The alignment kernels use the same wait with a budget
 * of about 2 s and report RGBID_ERR_TIMEOUT in their results.
 * Errors: INVALID_ARG, CUDA. */
int rgbid_probe_wait_timeout(long long budget_cycles, int* d_timeouts, void* stream);

/* Diagnostic of the bounds-checked test build (the paper has no counterpart): a
 * library compiled with -DRGBID_BOUNDS_CHECK checks every index it gathers from an
 * image plane (level planes, frames, keyframes, the filtered plane) against the
 * plane's allocation, counts an index outside it and reads element 0 instead.  Writes
 * the count since the library was loaded, over every kernel, to *count (host) after a
 * device synchronisation.  The product build does not check: it writes 0 and returns
 * RGBID_ERR_UNSUPPORTED.  Errors: INVALID_ARG (NULL count), CUDA. */
int rgbid_debug_bounds_violations(unsigned long long* count);

/* Diagnostic of the phase-stamped build (the paper has no counterpart): a library
 * compiled with -DRGBID_PHASE_STAMPS has thread 0 of the split kernel's cluster CTA 0
 * and of its first helper CTA record the global timer (ns) as each phase of an
 * iteration ends: out[(level * 16 + iteration) * 16 + phase], iterations < 16 of every
 * pyramid level, the phases 0-8 of the cluster (iteration start, partials arrived,
 * solved, pose published, sample residuals, counts, fixed-point rounds, nu sums,
 * parameters published) and 9-12 of the helper (pose seen, pixel pass done,
 * parameters seen, partial posted).  Copies RGBID_MAX_LEVELS * 256 values (n at least
 * that) to host memory after a device synchronisation.  The product build returns
 * RGBID_ERR_UNSUPPORTED.  Errors: INVALID_ARG, CUDA. */
int rgbid_debug_phase_stamps(long long* out, int n);

/* Diagnostic of the split level kernel's failure detection (the paper has no
 * counterpart).  The split kernel's roles wait on counters in the workspace's
 * mailbox; this launches one CTA that clears a mailbox in `d_scratch` (device,
 * 16-byte aligned, >= 1024 bytes, owned by the caller and not in use by an
 * alignment) and waits on a counter nothing advances: the first wait runs out of
 * `budget_cycles` (clock64 cycles, <= 2e10), counts a timeout and raises the
 * mailbox's error flag; the second wait, with the kernels' full ~2 s budget, must
 * give up at once because the flag is raised.  Writes 4 ints to d_out (device):
 * the timeouts counted, the two waits' verdicts (1 = the counter arrived), and the
 * error flag; then clears the mailbox.  Nothing faults or hangs.
 * Errors: INVALID_ARG, CUDA. */
int rgbid_probe_mailbox_timeout(long long budget_cycles, void* d_scratch, size_t scratch_bytes, int* d_out,
                                void* stream);

/* ---------------------------------------------------------------- fusion
 * Keyframe fusion ("Keyframe fusion", section "RGB-ID SLAM system"): every
 * keyframe pixel with W_kf > 0 is warped into frame k with T_kf_k = kf_T_k
 * (inverse geometric warping); where the four bilinear taps of W_k are valid,
 * both depths are positive and |W_k(p_k) - w_k| < 3 sigma_W (the visibility
 * test of "Dense frame covisibility ratio"), W_kf <- (W_kf C_kf + C_k W_k*) /
 * (C_kf + C_k) and C_kf <- C_kf + C_k, with W_k^* the transferred inverse depth
 * and C_k = (d W_k^* / d W_k(p_k))^-2.  With `fuse_intensity` the intensity is
 * averaged with the same weights.  Planes are float, updated in place.
 * `T_kf_k` (16 doubles) and `sigma_W` (1 double) are host pointers read during
 * the call when `params_on_device` is 0, or device pointers read by the kernel
 * when it is 1 (e.g. &d_result->T and &d_result->sigma[1] of the alignment).
 */
int rgbid_fuse_keyframe(float* I_kf, float* W_kf, float* C_kf, int pitch_kf,
                        const float* I_k, const float* W_k, int pitch_k,
                        int width, int height, rgbid_intrinsics K,
                        const double* T_kf_k, const double* sigma_W, int params_on_device,
                        int fuse_intensity, void* stream);

/* Initialise a keyframe from a frame: I_kf = I_k, W_kf = W_k, C_kf = 1. */
int rgbid_init_keyframe(float* I_kf, float* W_kf, float* C_kf, int pitch_kf,
                        const float* I_k, const float* W_k, int pitch_k,
                        int width, int height, void* stream);

/* Fusion or keyframe switch decided on the device: as rgbid_fuse_keyframe with
 * its pose and sigma_W read from device memory, except that when the device
 * int *d_switch is non-zero (written by rgbid_keyframe_decide) the keyframe is
 * re-initialised from frame k as rgbid_init_keyframe does ("Keyframe fusion":
 * the frame that fails the covisibility test starts the next keyframe).  Lets
 * a tracking loop be enqueued, or replayed as one CUDA graph, without reading
 * the decision back.  Errors: INVALID_ARG (as rgbid_fuse_keyframe; d_switch
 * NULL or misaligned), CUDA. */
int rgbid_fuse_or_switch_keyframe(float* I_kf, float* W_kf, float* C_kf, int pitch_kf,
                                  const float* I_k, const float* W_k, int pitch_k,
                                  int width, int height, rgbid_intrinsics K,
                                  const double* T_kf_k, const double* sigma_W,
                                  int fuse_intensity, const int* d_switch, void* stream);

/* ---------------------------------------------------------------- covisibility
 * Dense covisibility ratio ("Dense frame covisibility ratio"): every pixel of A
 * with a measurement (S_H: W_A > 0, I_A and W_A finite) is transferred into B
 * with T_AB = A_T_B (eq. 3d_registration); it is visible (S_V) when it lies in
 * front of B, its nearest pixel of B, floor(p_B + 1/2), is inside the image and
 * holds a measurement, and |W_B - w_B| < 3 sigma_W with w_B = 1 / Z_B of the
 * transferred point (otherwise it is occluded or out of view).  The same is
 * done from B to A with T_AB^-1, and the ratio is
 * min(|S_V(A->B)| / |S_H(A)|, |S_V(B->A)| / |S_H(B)|).
 * Planes are planar float (device, `pitch` elements per row) of equal size,
 * seen with the same intrinsics K.  `T_AB` (16 doubles) and `sigma_W`
 * (1 double) are host pointers read during the call (`params_on_device` 0) or
 * device pointers read by the kernel (1, e.g. &d_result->T and
 * &d_result->sigma[1] of the alignment).  Writes d_counts[4] (device unsigned
 * ints, zeroed by the call) = {|S_V(A->B)|, |S_H(A)|, |S_V(B->A)|, |S_H(B)|}
 * and, when d_ratio is not NULL, the ratio to the device float *d_ratio.
 * Errors: INVALID_ARG (NULL or misaligned pointers, sizes, intrinsics), CUDA. */
int rgbid_covisibility(const float* I_A, const float* W_A, int pitch_A,
                       const float* I_B, const float* W_B, int pitch_B,
                       int width, int height, rgbid_intrinsics K,
                       const double* T_AB, const double* sigma_W, int params_on_device,
                       unsigned int* d_counts, float* d_ratio, void* stream);

/* Keyframe decision of the tracking front-end by covisibility ("Keyframe
 * fusion": a new keyframe is started when the covisibility ratio of the
 * current frame with the keyframe falls below a threshold, 0.7 in the paper).
 * Reads the counts of rgbid_covisibility (keyframe = A, frame k = B), writes
 * *d_switch = (ratio < threshold) and, when d_ratio is not NULL, the ratio, and
 * advances the constant-velocity model's poses (device, 16 doubles each):
 * on a switch T2 <- T_k^-1 T1 (frame k-1 in the new keyframe) and T1 <- I,
 * else T2 <- T1 and T1 <- T_k.  T_k, T1 and T2 must not alias.
 * Errors: INVALID_ARG (NULL, misaligned or aliased pointers, threshold
 * outside [0, 1]), CUDA. */
int rgbid_keyframe_decide(const unsigned int* d_counts, double threshold, const double* T_k,
                          double* T1, double* T2, int* d_switch, float* d_ratio, void* stream);

/* ---------------------------------------------------------------- tracking helper
 * Constant-velocity initial guess of the tracking front-end ("Camera
 * tracking"): rf_T_k(0) = rf_T_{k-1} (rf_T_{k-2})^-1 rf_T_{k-1}, computed on the
 * device so that a sequence can be enqueued without host round trips.
 * All three pointers are device arrays of 16 doubles; `T_km2` may equal
 * `T_km1` (no motion model yet). */
int rgbid_predict_pose(const double* T_km1, const double* T_km2, double* T_out, void* stream);

/* Pose composition on the device: T_out = A^-1 B when `invert_A` is 1, else
 * A B (rigid transforms; the inverse is [R^T, -R^T t]).  Device arrays of 16
 * doubles; T_out may alias B but not A. */
int rgbid_compose_pose(const double* A, int invert_A, const double* B, double* T_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RGBID_H */
