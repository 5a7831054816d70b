/*
 * cslsm: GB300-native PnP-ADMM reconstruction for compressive light-sheet
 * microscopy (Gong, Zhang, Chai, Ding, Lou, arXiv 2511.03093).
 *
 * C ABI.  Plain pointers and sizes only.  Conventions shared by every call:
 *
 *  - Layout.  Volumes (v, u, d, denoiser in/out) are float32 [Z][H][W],
 *    row-major with W fastest; Z = n_shots * R and slice n = j*R + r belongs
 *    to shot j, plane r (Sec. III-A).  Measurements b are float32
 *    [n_shots][H][W].  Masks are uint8 [R][H][W] (one pattern set shared by
 *    every shot, phi_r of Eq. model-slice) or [Z][H][W] (one pattern per
 *    slice); any nonzero byte is an open DMD mirror.
 *  - Memory.  Every data pointer is DEVICE memory owned by the caller, on the
 *    current CUDA device, unless the argument says "host".  The library keeps
 *    no pointer to caller memory after a call returns; a plan owns its own
 *    device workspace.
 *  - Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).
 *    Work is enqueued asynchronously on it; a call returns before the GPU has
 *    finished unless its comment says it synchronises.  Caller buffers must
 *    stay valid until the stream reaches the enqueued work.
 *  - Errors.  Every call returns a cslsm_status and never throws or exits.
 *    Argument checks happen before any GPU work is enqueued (nothing is
 *    launched on CSLSM_ERR_INVALID_ARG / CSLSM_ERR_UNSUPPORTED);
 *    cslsm_last_error() gives a per-thread message for the last failure.
 *  - Limits.  1 <= R <= CSLSM_MAX_R planes per shot; H, W >= 1;
 *    Z * H * W < 2^31.
 */
#ifndef CSLSM_H
#define CSLSM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSLSM_MAX_R 32
#define CSLSM_ABI_VERSION 4

typedef enum {
    CSLSM_OK = 0,
    CSLSM_ERR_INVALID_ARG = 1, /* bad pointer, size, parameter or shape */
    CSLSM_ERR_CUDA = 2,        /* a CUDA runtime call or kernel launch failed */
    CSLSM_ERR_TIMEOUT = 3,     /* a bounded device-side wait gave up */
    CSLSM_ERR_UNSUPPORTED = 4, /* valid request this build does not implement */
    CSLSM_ERR_OOM = 5          /* device allocation failed */
} cslsm_status;

/* The plug-in priors of the u-step (Eq. u-sub, Sec. III-B). */
typedef enum {
    CSLSM_DEN_TIKHONOV = 0, /* psi(u) = ||u||^2, closed form (Sec. III-B, III-C) */
    CSLSM_DEN_TV = 1,       /* isotropic TV, Chambolle dual projection */
    CSLSM_DEN_BM3D = 2,     /* block matching + 3D collaborative filtering */
    CSLSM_DEN_WNNM = 3      /* weighted nuclear norm minimisation on the BM3D groups
                               (listed in Sec. III-B; one pass per u-step, noise level
                               bm3d_sigma) */
} cslsm_denoiser;

/* Element type of the ADMM state u, d and of the plan's w = v + d workspace
 * (arithmetic is always FP32; the x-update division by rho + diag(Phi Phi^T),
 * the residuals and v_out stay FP32). */
typedef enum {
    CSLSM_STORE_FP32 = 0,
    CSLSM_STORE_BF16 = 1, /* bfloat16, round to nearest even on store */
    CSLSM_STORE_FP16 = 2  /* IEEE half, round to nearest even on store */
} cslsm_storage;

/* Parameters of Algorithm 1 and of its denoiser.
 *   rho     > 0   ADMM penalty (augmented Lagrangian of Sec. III-B).
 *   lambda  >= 0  prior weight (Eq. model-slice).  Ignored by BM3D, whose
 *                 strength is bm3d_sigma (the paper's "noise level" lambda).
 *   gamma   >= 0  z-smoothness weight (Sec. III-C); 0 = slice-based model.
 *                 Ignored when Z == 1.
 *   iters   >= 0  maximum number of ADMM iterations.
 *   tol     >= 0  stop once ||v^{k+1}-v^k|| / ||v^k|| < tol (Sec. IV-B), checked
 *                 every check_every iterations ON THE DEVICE: all `iters`
 *                 iterations are enqueued without any host synchronisation and
 *                 every kernel after the check that met the tolerance returns
 *                 at once; the call synchronises `stream` once at its end to
 *                 report the outcome.
 *                 0 runs exactly `iters` iterations without synchronising.
 *   check_every   >= 1, used only when tol > 0.
 *   denoiser      a cslsm_denoiser.
 *   tv_inner      TV: Chambolle steps per prox (>= 1).
 *   tv_tau        TV: dual step, 0 < tv_tau <= 0.25 (1/8 is the convergent
 *                 bound of Chambolle 2004).
 *   bm3d_sigma    BM3D: noise standard deviation on the volume's scale (> 0).
 *   init_user     0: u^0 = d^0 = 0.  1: u_io / d_io hold u^0, d^0.
 *   storage       a cslsm_storage: element type of u_io / d_io and of the
 *                 plan's state and workspace. */
typedef struct {
    float rho;
    float lambda;
    float gamma;
    int iters;
    float tol;
    int check_every;
    int denoiser;
    int tv_inner;
    float tv_tau;
    float bm3d_sigma;
    int init_user;
    int storage;
} cslsm_admm_params;

/* Filled by cslsm_admm_solve when non-NULL (host memory). */
typedef struct {
    int iters_done;    /* ADMM iterations executed */
    double rel_change; /* last ||v^{k+1}-v^k||/||v^k|| when tol > 0, else -1 */
} cslsm_admm_stats;

typedef struct cslsm_plan_s *cslsm_plan;

/* Create a plan for one acquisition geometry and DMD pattern set (Sec. III-A).
 *   plan      out (host): receives the opaque handle.
 *   H, W      image size; n_shots >= 1 coded images of R planes each.
 *   masks     device uint8, [R][H][W] if per_slice == 0 or [Z][H][W] if 1.
 * The plan packs the patterns into one R-bit word per pixel and shot (bit r
 * = mirror open for plane r; diag(Phi Phi^T) is its popcount, Sec. III-B) and
 * allocates its workspace (about 3 * Z*H*W floats).  Synchronises `stream`. */
cslsm_status cslsm_plan_create(cslsm_plan *plan, int H, int W, int n_shots, int R,
                               const uint8_t *masks, int per_slice, void *stream);

/* Replace the plan's DMD patterns (same geometry): re-packs the bit words.
 * Asynchronous; later calls on the same stream see the new patterns. */
cslsm_status cslsm_plan_set_masks(cslsm_plan plan, const uint8_t *masks, int per_slice,
                                  void *stream);

/* Release the plan and its device memory.  Synchronises the device first.
 * NULL is accepted. */
cslsm_status cslsm_plan_destroy(cslsm_plan plan);

/* Forward operator (Sec. III-A, Eq. model-slice):
 *   b_j = sum_r phi_r (.) v_{jR+r}.   v: [Z][H][W] in, b: [n_shots][H][W] out. */
cslsm_status cslsm_forward(cslsm_plan plan, const float *v, float *b, void *stream);

/* Adjoint (Phi^T of Eq. v-update): v_{jR+r} = phi_r (.) b_j.
 *   b: [n_shots][H][W] in, v: [Z][H][W] out. */
cslsm_status cslsm_adjoint(cslsm_plan plan, const float *b, float *v, void *stream);

/* Algorithm 1 (CS LSM temporal reconstruction; gamma = 0 is the slice-based
 * method): per iteration the Woodbury-form v-update of Eq. (v-update), the
 * Gauss-Seidel u-sweep of Eq. (u-update) with the chosen denoiser, and the
 * dual update d <- d + v - u (Eq. ADMM).
 *   b       device [n_shots][H][W] measurement.
 *   v_out   device [Z][H][W]: receives v^K, Algorithm 1's output.
 *   u_io, d_io  device [Z][H][W] arrays of params->storage elements, or
 *           NULL.  When given they are the ADMM state (read as u^0, d^0 if
 *           init_user, always written with u^K, d^K), which lets a caller
 *           resume a solve; when NULL the plan's own state buffers are used
 *           (then init_user must be 0).
 *   stats   host, optional.
 * v_out must not overlap u_io, d_io or b. */
cslsm_status cslsm_admm_solve(cslsm_plan plan, const float *b, const cslsm_admm_params *params,
                              float *v_out, void *u_io, void *d_io, cslsm_admm_stats *stats,
                              void *stream);

/* The u-step denoiser alone, slice by slice, without z coupling (Eq. u-sub):
 *   Tikhonov: out = rho * in / (2 lambda + rho);
 *   TV:       out = argmin theta*TV(u) + 1/2||u - in||^2, theta = lambda / rho,
 *             by params->tv_inner Chambolle steps from p = 0;
 *   BM3D:     out = BM3D(in) at noise level params->bm3d_sigma (stage 1 then
 *             stage 2, see cslsm_bm3d_stage; scratch from cudaMallocAsync).
 * in, out: device [Z][H][W]; they must not overlap (neighbour reads). */
cslsm_status cslsm_denoise(int denoiser, const float *in, float *out, int Z, int H, int W,
                           const cslsm_admm_params *params, void *stream);

/* ---- BM3D stages (the u-step denoiser of Sec. III-B / IV-C, by stage) ------
 * The variant built here, applied to each 2-D slice: 8 x 8 patches, reference
 * patches every 3 pixels plus the last position, a 39 x 39 search window,
 * matching on the 8-bit codes clamp(rint(x * 255), 0, 255) by exact integer
 * SSD with thresholds 64 * 2500 (stage 1) and 64 * 400 (stage 2), groups of
 * the reference plus up to 15 others in (SSD, y * W + x) order cut to a power
 * of two, an orthonormal 8 x 8 DCT-II + Haar group transform, hard threshold
 * 2.7 sigma (stage 1) or Wiener shrinkage guided by the basic estimate
 * (stage 2), and Kaiser-window (beta = 2) weighted aggregation.  Slices
 * smaller than 8 x 8 are returned unchanged.  These calls allocate their
 * scratch with cudaMallocAsync on `stream`. */

/* Reference patches of one H x W slice (0 if H < 8 or W < 8). */
int cslsm_bm3d_num_refs(int H, int W);

/* Block matching of stage 1 or 2 on each slice of img (device [Z][H][W]):
 * lists (device int32 [Z][nref][16]) receives, per reference in row-major
 * order of the reference grid, the patch positions y * W + x of its group
 * (reference first, -1 padding); counts (device int32 [Z][nref]) the group
 * sizes before the power-of-two cut.  Needs H, W >= 8. */
cslsm_status cslsm_bm3d_match(const float *img, int Z, int H, int W, int stage, int *lists,
                              int *counts, void *stream);

/* One BM3D stage on every slice: stage 1 (hard threshold) of noisy, or
 * stage 2 (Wiener) of noisy guided by the basic estimate `guide` (device
 * [Z][H][W], matched on).  out: device [Z][H][W], not overlapping the inputs. */
cslsm_status cslsm_bm3d_stage(int stage, const float *noisy, const float *guide, float *out,
                              int Z, int H, int W, float sigma, void *stream);

/* cslsm_bm3d_stage with its decisions exposed, for checking them one by one:
 * lists (device int32 [Z][nref][16]) and counts ([Z][nref]) receive the
 * stage's groups as cslsm_bm3d_match gives them, group_stat (device float
 * [Z][nref]) per group the number of coefficients the hard threshold kept
 * (stage 1) or the sum of the squared Wiener factors (stage 2), the quantity
 * each group's aggregation weight is formed from.  Needs H, W >= 8. */
cslsm_status cslsm_bm3d_stage_groups(int stage, const float *noisy, const float *guide,
                                     float *out, int Z, int H, int W, float sigma, int *lists,
                                     int *counts, float *group_stat, void *stream);

/* ---- batched solver --------------------------------------------------------
 * Many independent measurements (each with its own plan: size, slice count,
 * patterns) reconstructed by Algorithm 1 with the TV prior (and the z term
 * when gamma > 0) in one persistent kernel launch, recorded once into a CUDA
 * graph at creation and replayed by every run.  Per measurement the result
 * is bit-identical to cslsm_admm_solve with the same parameters and storage
 * type.  The persistent kernel schedules per-measurement phase chains
 * (x-update, then the TV u-step of each slice in Gauss-Seidel order) from a
 * global work counter; each dependency wait is bounded (4 s by default) and a
 * wait that runs out makes cslsm_batch_wait return CSLSM_ERR_TIMEOUT. */
typedef struct cslsm_batch_s *cslsm_batch;

typedef struct {
    cslsm_plan plan; /* geometry, DMD patterns; its state buffers hold u, d */
    const float *b;  /* device [n_shots][H][W] measurement */
    float *v_out;    /* device [Z][H][W]: receives v^K */
} cslsm_batch_item;

/* Create a batch over n_items items (plans on the current device) with one
 * parameter set: denoiser TV, tol 0, init_user 0.  b and v_out pointers are
 * recorded: every run reads and writes the same buffers, and u^0 = d^0 = 0 in
 * each run.  The TV proxes run in phases of at most 10 Chambolle steps whose
 * tiles hand the dual field over through device memory the batch owns
 * (5 floats per pixel of every item with gamma > 0 and Z > 1, else 4 floats
 * per voxel).  With
 * cslsm_set_autotune(1) the steps per phase are chosen by timing
 * one-iteration runs of a few candidates (this synchronises `stream` and
 * overwrites the items' state and v_out).  Synchronises `stream`. */
cslsm_status cslsm_batch_create(cslsm_batch *batch, const cslsm_batch_item *items, int n_items,
                                const cslsm_admm_params *params, void *stream);

/* Route of slice-independent TV solves (process-wide setting).  A
 * cslsm_admm_solve with denoiser TV, lambda > 0, gamma = 0 (or Z = 1), tol = 0,
 * init_user = 0 and no u_io / d_io gives the same bits on two paths: per-launch
 * TV tiles (an x-update launch and a prox launch per iteration, each prox tile
 * recomputing a halo of T + 1 pixels), or a one-item persistent batch (see
 * cslsm_batch_create; phases of k steps with the dual field handed over through
 * memory), which the plan creates on such a call and keeps while the
 * parameters and the alignment class of b and v_out stay the same (other b and
 * v_out are pointed to by a small copy on `stream`; recreating the batch
 * synchronises the device).
 *   mode 0 (default): the batch when one phase level holds at least 4 tiles
 *          per SM (large volumes), else the per-launch tiles; a batch that does
 *          not fit in device memory leaves the solve to the per-launch tiles;
 *   mode 1: always the per-launch tiles;   mode 2: always the batch.
 * On the batch path a non-NULL stats makes the call synchronise `stream` and
 * report a device-side wait that ran out (CSLSM_ERR_TIMEOUT).  Returns
 * CSLSM_ERR_INVALID_ARG for other modes. */
cslsm_status cslsm_set_tv_route(int mode);

/* Chambolle steps per phase of batches created from now on (process-wide
 * setting).  k = 0 (default): the fixed default, or the timed choice under
 * cslsm_set_autotune(1).  k >= 1: exactly min(k, tv_inner, the largest phase
 * whose halo fits the batch's tile region) steps, without timing (for
 * profiling a small batch with the schedule a larger one chose).  Returns
 * CSLSM_ERR_INVALID_ARG for k < 0. */
cslsm_status cslsm_set_batch_steps_per_phase(int k);

/* The batch's schedule: Chambolle steps per phase (chosen by cslsm_set_autotune(1)
 * timing, else the default), CTAs of the persistent launch, and work units per
 * ADMM iteration.  Any output pointer may be NULL.  Host-only; no stream work. */
cslsm_status cslsm_batch_info(cslsm_batch batch, int *steps_per_phase, int *grid,
                              long long *units_per_iteration);

/* Enqueue one whole batched solve on `stream` (one graph launch). */
cslsm_status cslsm_batch_run(cslsm_batch batch, void *stream);

/* Synchronise `stream` and report the last run's outcome: CSLSM_OK, or
 * CSLSM_ERR_TIMEOUT if a bounded device-side wait gave up (every CTA then
 * stops and the outputs are incomplete). */
cslsm_status cslsm_batch_wait(cslsm_batch batch, void *stream);

/* Set the wait limit (seconds) of later runs.  test_stall = 1 makes every
 * dependency wait target a count that never arrives, so that the next run
 * exercises the time-out path (for tests); 0 restores normal waits.
 * Synchronises the device. */
cslsm_status cslsm_batch_set_wait_limit(cslsm_batch batch, double seconds, int test_stall);

/* Release the batch (synchronises the device).  NULL is accepted. */
cslsm_status cslsm_batch_destroy(cslsm_batch batch);

/* ---- differentiable unrolled solver ----------------------------------------
 * K iterations of Algorithm 1 unrolled into a differentiable map, for learning
 * the DMD patterns and the parameters (rho, lambda, gamma) end to end.  The
 * paper's method with two relaxations: the binary patterns become
 * m = sigmoid(logits) (continuous, D = sum_r m_r^2 in the Woodbury x-update),
 * and TV becomes the Huber-smoothed TV (|x| - eps/2 beyond eps, |x|^2/(2 eps)
 * below), whose prox is taken by tv_steps projected-gradient steps on its
 * dual from p = 0: q = div p - h/theta, a = p + tau (grad q - (eps/theta) p),
 * p <- a / max(1, |a|), u = h - theta div p; h is the Gauss-Seidel input of
 * Eq. (u-update), theta = lambda / (rho + 2 gamma).  One shot per volume
 * (R = Z), u^0 = d^0 = 0, output v^K.
 * Layouts: logits, v_out, logits_bar [B][Z][H][W]; b [B][H][W]; ckpt holds
 * ceil(iters / ckpt_every) checkpoints of (u, d): [n_ckpt][2][B][Z][H][W]
 * floats; ws is caller-owned device scratch of cslsm_unrolled_workspace_bytes
 * bytes (the same params for the workspace size, the forward and the
 * backward).  The backward recomputes each checkpoint segment and runs the
 * hand-written adjoint; it synchronises `stream` (to combine the scalar
 * gradients) and writes dL/dlogits and scalar_bar (device double[3]) =
 * {dL/drho, dL/dlambda, dL/dgamma} for the given v_bar = dL/dv^K.
 * keep_duals = 1 trades memory for time: the segment recompute keeps every
 * slice's prox input and its tv_steps + 1 dual iterates, so the reverse sweep
 * reads them instead of recomputing them (same results bit for bit).  The
 * workspace then grows by ckpt_every x Z x (2 tv_steps + 3) x B x H x W
 * floats (29 GB for batch 8 x 512 x 512 x 16, 20 steps, checkpoints every 5
 * iterations). */
typedef struct {
    float rho, lambda, gamma; /* rho > 0, lambda > 0, gamma >= 0 */
    int iters;                /* K */
    int tv_steps;             /* dual steps per prox */
    float tv_tau;             /* dual step, (0, 1/8] */
    float huber_eps;          /* >= 0 (0: plain TV) */
    int ckpt_every;           /* checkpoint period in iterations */
    int keep_duals;           /* 0: recompute the dual iterates in the reverse sweep; 1: keep */
} cslsm_unrolled_params;

size_t cslsm_unrolled_workspace_bytes(int B, int Z, int H, int W,
                                      const cslsm_unrolled_params *params);
cslsm_status cslsm_unrolled_forward(const float *logits, const float *b, int B, int Z, int H,
                                    int W, const cslsm_unrolled_params *params, float *v_out,
                                    float *ckpt, void *ws, void *stream);
cslsm_status cslsm_unrolled_backward(const float *logits, const float *b, int B, int Z, int H,
                                     int W, const cslsm_unrolled_params *params,
                                     const float *ckpt, const float *v_bar, float *logits_bar,
                                     double *scalar_bar, void *ws, void *stream);

/* ---- allocation-free BM3D ------------------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they denoise (under a fixed memory
 * budget owned by the host application, or in a loop where an allocation's
 * latency or failure is not acceptable).
 *
 * cslsm_denoise_bm3d_noalloc computes exactly what cslsm_denoise does with
 * the BM3D prior at noise level sigma (in, out: device [Z][H][W], not
 * overlapping), but its scratch is a fixed array inside the library instead
 * of cudaMallocAsync memory: it calls no cudaMalloc, cudaFree or other
 * allocating routine.  The array holds cslsm_bm3d_noalloc_capacity() bytes
 * (64 MiB) on every GPU that loads the library, until the process exits.  A
 * call whose scratch (cslsm_bm3d_scratch_bytes(Z, H, W): about 33 bytes per
 * voxel, e.g. 8.5 MB for one 512 x 512 slice) exceeds it returns
 * CSLSM_ERR_INVALID_ARG before any GPU work, and so does a call whose in or
 * out is not device (or managed) memory of the current device (the array
 * used is the current device's).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.  Every call on a device
 * shares the one array and clears the part it uses at its start, so calls
 * whose GPU work overlaps (on different streams, or from different host
 * threads) race and give wrong results; serialise them on one stream. */
size_t cslsm_bm3d_noalloc_capacity(void);
size_t cslsm_bm3d_scratch_bytes(int Z, int H, int W);
cslsm_status cslsm_denoise_bm3d_noalloc(const float *in, float *out, int Z, int H, int W,
                                        float sigma, void *stream);

/* Volume PSNR of Sec. IV (all voxels as one array): writes
 * 10 log10(n V^2 / ||x - ref||^2), V = max(ref), as a double to out (device).
 * Deterministic two-level reduction; uses a stream-ordered scratch buffer. */
cslsm_status cslsm_psnr(const float *x, const float *ref, size_t n, double *out, void *stream);

/* Volume SSIM of Sec. IV: the local ssim of Wang et al. (means, variances and
 * covariance over an 11 x 11 x 11 Gaussian window with standard deviation 1.5,
 * clipped to the volume and renormalised; c1 = 0.01^2, c2 = 0.03^2 for data
 * on [0, 1]) averaged over every voxel.  x, ref: device, FP32 [Z][H][W];
 * writes the mean as a double to out (device).  Deterministic (fixed-order
 * FP64 reduction of FP32 local values).  Uses a stream-ordered scratch buffer
 * of 20 bytes per voxel. */
cslsm_status cslsm_ssim3d(const float *x, const float *ref, int Z, int H, int W, double *out,
                          void *stream);

/* Human-readable name of a status code (static string). */
const char *cslsm_status_string(cslsm_status status);

/* Message describing the calling thread's most recent failure ("" if none). */
const char *cslsm_last_error(void);

/* CSLSM_ABI_VERSION of the loaded library. */
int cslsm_abi_version(void);

/* TV prox tile shapes (process-wide setting).  The TV kernel comes in four
 * variants (column chunks x row bands) with a tile shape chosen per launch
 * geometry.  mode 0 (default): shapes from a cost model of the work per SM.
 * mode 1: on the first launch of each (device, H, W, steps, slices) key that
 * is not being captured into a CUDA graph, time every variant on the actual
 * launch (three runs each; the prox is idempotent, so this only costs time)
 * with a synchronisation of the stream, and keep the fastest for later
 * launches.  modes 2..5: force variant mode - 2 (for tests).  Changing the
 * mode clears the kept choices. */
cslsm_status cslsm_set_autotune(int mode);

/* The TV tile shape a prox launch of this geometry would use now (on the
 * current device): shape4 (host int[4]) = {variant, tile rows, tile columns,
 * region rows}.  steps <= 24 (longer proxes run in chunks). */
cslsm_status cslsm_tv_shape(int H, int W, int steps, int nslices, int *shape4);

/* Persistent z sweep (process-wide setting).  With gamma > 0 the TV u-step
 * of cslsm_admm_solve (the Gauss-Seidel sweep over slices of Sec. III-C) runs
 * in ONE cooperative launch per ADMM iteration (enable = 1, the default):
 * every CTA owns one tile of every slice and trades the dual field of its
 * tile with its neighbours every few Chambolle steps.  enable = 0 runs one
 * tile-kernel launch per slice instead; the two give bit-identical results.
 * tiling < 0: the tiling is chosen per (device, H, W, Z, steps, storage) key
 * by a cost model, or under cslsm_set_autotune(1) by timing every tiling once
 * on scratch copies of u and d (outside stream capture; synchronises the
 * stream).  0 <= tiling < cslsm_zsweep_num_tilings(): force that tiling
 * (tests).  wait_limit_s (> 0, default 2) bounds every device-side wait of the
 * sweep; when one gives up, every CTA stops and the solve returns
 * CSLSM_ERR_TIMEOUT.  test_stall != 0 makes one CTA wait for an epoch that is
 * never published (tests of the timeout path only).  A solve that used the
 * sweep reads the error word at its end (synchronising `stream` unless it is
 * being captured). */
cslsm_status cslsm_zsweep_config(int enable, int tiling, double wait_limit_s, int test_stall);

/* Number of sweep tilings (steps per phase x target CTAs per SM x row shape:
 * warps per CTA and rows per warp). */
int cslsm_zsweep_num_tilings(void);

/* The tiling a sweep of this geometry would use now (on the current device):
 * out8 (host int[8]) = {tiling, steps per phase, rows per warp, warps per CTA,
 * tile rows, tile columns, region rows, tiles}. */
cslsm_status cslsm_zsweep_shape(int H, int W, int Z, int steps, int storage, int *out8);

/* ---- instrumentation (benchmarks, tracing) ------------------------------ */

/* Number of kernels the library has launched in this process so far. */
unsigned long long cslsm_launch_count(void);

/* Sampled kernel timing.  period > 0: from now on every period-th launch of
 * each kernel is bracketed by two CUDA events recorded on its stream (the
 * events add a little GPU time of their own); 0 switches sampling off.
 * Kernel names: "pack_masks", "forward", "adjoint", "xupdate_w",
 * "tikhonov_iter", "tikhonov_prox", "tv_tile", "psnr_partials",
 * "reduce_finish", "bm3d_prep", "bm3d_match", "bm3d_filter", "bm3d_finish",
 * "batch_persistent", "unrolled", "tvz_sweep", "ssim3d". */
cslsm_status cslsm_timing_enable(int period);

/* Waits for the recorded events of `kernel` and returns how many launches
 * were timed and their summed device time in milliseconds (host pointers).
 * reset != 0 then discards every record of every kernel and restarts the
 * sampling counters. */
cslsm_status cslsm_timing_read(const char *kernel, long long *launches_timed, double *total_ms,
                               int reset);

#ifdef __cplusplus
}
#endif
#endif /* CSLSM_H */
