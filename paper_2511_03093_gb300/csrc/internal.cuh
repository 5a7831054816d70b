// Internal declarations shared by the cslsm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "cslsm.h"

namespace cslsm {

// Per-thread error message (set by the API layer and the launchers).
void set_error(const char *fmt, ...);

// Evaluates a CUDA runtime call; on failure records the message and returns
// CSLSM_ERR_CUDA (or CSLSM_ERR_OOM) from the enclosing function.
#define CSLSM_CUDA(call)                                                                    \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            ::cslsm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                               __FILE__, __LINE__);                                         \
            return e_ == cudaErrorMemoryAllocation ? CSLSM_ERR_OOM : CSLSM_ERR_CUDA;        \
        }                                                                                   \
    } while (0)

#define CSLSM_LAUNCHED() CSLSM_CUDA(cudaGetLastError())

// Kernels of the library, for launch accounting and sampled timing (timing.cu).
enum KernelId {
    K_PACK = 0, K_FORWARD, K_ADJOINT, K_XUPDATE, K_TIK_ITER, K_TIK_PROX, K_TV_TILE, K_PSNR,
    K_REDUCE, K_BM3D_PREP, K_BM3D_MATCH, K_BM3D_FILTER, K_BM3D_FINISH, K_BATCH, K_DIFF, K_TVZ,
    K_SSIM, K_WNNM, K_COUNT
};

// Wrap every kernel launch: counts it and, when timing is on, records CUDA
// events around it on its stream (constructor before, destructor after).
class LaunchScope {
  public:
    LaunchScope(int kernel, cudaStream_t s);
    ~LaunchScope();
    LaunchScope(const LaunchScope &) = delete;
    LaunchScope &operator=(const LaunchScope &) = delete;

  private:
    int rec_;
    cudaStream_t s_;
};

// Geometry of one acquisition (Sec. III-A).
struct Geom {
    int H, W, N, R;  // image, shots, planes per shot
    int Z() const { return N * R; }
    int HW() const { return H * W; }
    long long voxels() const { return (long long)N * R * H * W; }
};

// Packed DMD patterns: one 32-bit word per pixel and shot; bit r = plane r.
// wstride = H*W when every shot has its own patterns, 0 when all shots share.
struct Masks {
    const uint32_t *words;
    int wstride;
};

// ---- pointwise kernels (kernels_pointwise.cu) -----------------------------
cslsm_status launch_pack_masks(const uint8_t *masks, uint32_t *words, int HW, int R, int nsets,
                               cudaStream_t s);
cslsm_status launch_forward(const Geom &g, Masks m, const float *v, float *b, cudaStream_t s);
cslsm_status launch_adjoint(const Geom &g, Masks m, const float *b, float *v, cudaStream_t s);

// w = v^{k+1} + d^k with v^{k+1} from the Woodbury update; optionally writes
// v^{k+1} to v_out.  When vprev != nullptr it also accumulates, per block,
// sum (v^{k+1}-vprev)^2 and sum vprev^2 into partials[2*block] and then
// stores v^{k+1} into vprev.
// u, d, w have the element type of `storage` (a cslsm_storage value).
// stop: device flag of a tolerance-stopped solve (the kernel returns at once
// when it is set), or nullptr; the same for launch_tikhonov_iter.
cslsm_status launch_xupdate_w(const Geom &g, Masks m, int storage, const void *u, const void *d,
                              const float *b, float rho, void *w, float *v_out, float *vprev,
                              double *partials, int nblocks_red, cudaStream_t s,
                              const int *stop = nullptr);

// One whole ADMM iteration with the Tikhonov prior fused into one pass:
// v-update, Gauss-Seidel Tikhonov sweep along z (gamma > 0) and dual update.
cslsm_status launch_tikhonov_iter(const Geom &g, Masks m, int storage, void *u, void *d,
                                  const float *b, float rho, float lam, float gam, float *v_out,
                                  float *vprev, double *partials, int nblocks_red, cudaStream_t s,
                                  const int *stop = nullptr);

// Device-side tolerance stop (Sec. IV-B stopping rule without a host sync per
// check).  state: {int stop; int iters_done; double rel}.  tol_check: unless
// already stopped, rel = sqrt(red[0] / red[1]) and, when rel < tol, stop = 1 and
// iters_done = k + 1.  copy_if_stopped: dst = src when the solve stopped.
struct TolState {
    int stop;  // first member: kernels take its address as the stop flag
    int iters_done;
    double rel;
};
static_assert(offsetof(TolState, stop) == 0, "the stop flag leads TolState");
cslsm_status launch_tol_check(const double *red, float tol, int k, TolState *state,
                              cudaStream_t s);
cslsm_status launch_copy_if_stopped(const TolState *state, const float *src, float *dst,
                                    size_t n, cudaStream_t s);

// Slice-wise Tikhonov prox out = rho*in/(2 lam + rho).
cslsm_status launch_tikhonov_prox(const float *in, float *out, long long n, float rho, float lam,
                                  cudaStream_t s);

// Deterministic reductions.
int reduction_blocks();
cslsm_status launch_psnr_partials(const float *x, const float *ref, size_t n, double *partials,
                                  int nblocks, cudaStream_t s);
cslsm_status launch_psnr_finish(const double *partials, int nblocks, size_t n, double *out,
                                cudaStream_t s);
cslsm_status launch_sum_pairs(const double *partials, int nblocks, double *out2,
                              cudaStream_t s);

// ---- TV prox (kernels_tv.cu) ----------------------------------------------
struct TvSlices {
    int storage;         // element type of w, u, d (cslsm_storage)
    const void *w;       // [Z][H][W] prox input source (w = v + d)
    void *u;             // [Z][H][W] output u_n (and u_{n-1}, u_{n+1} source)
    void *d;             // [Z][H][W] output d_n = w_n - u_n, or nullptr
    int H, W, Z;
    int n0, nslices;     // slices n0 .. n0+nslices-1
    float rho, gamma;    // g = (rho w + gamma (u_{n-1} + u_{n+1})) / (rho + 2 gamma)
    float theta;         // TV weight of the prox
    float tau;
    int T;               // Chambolle steps
    const int *stop = nullptr;  // device flag of a tolerance-stopped solve: skip when set
};
// Chambolle TV prox of every listed slice.  Uses the plan-provided dual
// buffers pbuf (4 * nslices * H * W floats) only when T exceeds the largest
// step count one launch covers; pbuf may be nullptr otherwise.
cslsm_status tv_prox_slices(const TvSlices &a, float *pbuf, cudaStream_t s);
int tv_max_steps_per_launch();
// 0: tile shapes from the cost model; 1: time the kernel variants on the first
// launch of every shape key (outside stream capture) and keep the fastest;
// 2 + k: force variant k (tests).
void tv_set_mode(int mode);
int tv_get_mode();
// The shape (variant, TH, TW, RH) a launch of this geometry would use now.
cslsm_status tv_query_shape(int H, int W, int T, int nslices, int *out4);

// ---- persistent z sweep of the TV u-step (kernels_tvz.cu) -----------------
// Workspace of a plan: the dual field handed between phases ([2][2][H][W]
// floats), per-tile epoch flags, the error word, and the next epoch base.
struct ZsweepWs {
    float *pbuf = nullptr;
    size_t pbuf_floats = 0;
    unsigned *flags = nullptr;
    int *err = nullptr;
    int max_tiles = 0;
    unsigned next_base = 0;
};
// True when the sweep handles this u-step: TV with gamma > 0 over all slices
// and the sweep enabled.
bool zsweep_applies(const TvSlices &a);
cslsm_status zsweep_reserve(ZsweepWs &ws, int H, int W);
void zsweep_release(ZsweepWs &ws);
// The whole Gauss-Seidel sweep n = 0 .. Z-1 in one cooperative launch.
cslsm_status zsweep_run(const TvSlices &a, ZsweepWs &ws, cudaStream_t s);
// Reads and clears the error word (synchronises s unless it is capturing).
cslsm_status zsweep_check(ZsweepWs &ws, cudaStream_t s);
void zsweep_config(int enable, int force, double wait_s, int stall);
bool zsweep_forced();  // a tiling is forced (tests): no silent per-slice path
cslsm_status zsweep_query(int H, int W, int Z, int T, int storage, int *out8);
int zsweep_num_candidates();

// ---- 3-D SSIM (kernels_ssim.cu) ---------------------------------------------
// Scratch bytes of one call (five FP32 planes of the volume and the block
// partials); *nblocks receives the partial count launch_ssim3d expects.
size_t ssim3d_workspace_bytes(int Z, int H, int W, int *nblocks);
cslsm_status launch_ssim3d(const float *x, const float *ref, int Z, int H, int W, void *ws,
                           int nblocks, double *out, cudaStream_t s);

// ---- BM3D (kernels_bm3d.cu) -------------------------------------------------
struct Bm3dSlices {
    int storage;       // element type of src, u, out, dual (cslsm_storage)
    const void *src;   // [Z][H][W] u-step input source: w = v + d (ADMM) or the image
    const void *u;     // [Z][H][W] z neighbours when gamma > 0
    void *out;         // [Z][H][W] receives the denoised slices n0 .. n0+nslices-1
    void *dual;        // [Z][H][W] receives src - out for those slices, or nullptr
    int Z, H, W, n0, nslices;
    float rho, gamma, sigma;
    const int *stop = nullptr;  // device flag of a tolerance-stopped solve: skip when set
};
int bm3d_nref(int H, int W);
// Device workspace for nslices slices; it must be zero-filled before its first
// use (the accumulators are cleared again by every call).
size_t bm3d_workspace_bytes(int nslices, int H, int W);
cslsm_status bm3d_slices(const Bm3dSlices &b, void *ws, cudaStream_t s);
// WNNM u-step on the same groups and workspace (hard-stage matching, one pass).
cslsm_status wnnm_slices(const Bm3dSlices &b, void *ws, cudaStream_t s);
// One stage; when lists / counts / stat are not null they receive the stage's
// match lists [ns][nref][16], group sizes [ns][nref] and per-group statistic
// (hard: kept coefficients; Wiener: sum of squared shrinkage factors).
cslsm_status bm3d_stage_only(int stage, const float *noisy, const float *guide, float *out,
                             int nslices, int H, int W, float sigma, void *ws, cudaStream_t s,
                             int *lists = nullptr, int *counts = nullptr, float *stat = nullptr);
cslsm_status bm3d_match_only(const float *img, int nslices, int H, int W, int stage, int *lists,
                             int *counts, void *ws, cudaStream_t s);

// ---- persistent batched solver (kernels_batch.cu) ------------------------------
struct BatchItemSpec {
    void *u, *d, *w;  // state and workspace of the item's plan (storage type)
    const float *b;
    float *v_out;
    const uint32_t *words;
    int wstride;
    int H, W, N, R;
};
struct BatchSpec {
    std::vector<BatchItemSpec> items;
    int iters, T, storage, stall_test;
    int k;  // Chambolle steps per phase (the TV tiles trade p through L2 between phases)
    float rho, lam, gamma, tau;
    double wait_limit_s;
};
// Largest number of Chambolle steps per phase whose halo fits the batched
// solver's region.
int batch_max_steps_per_phase();
// TV tiles per slice of the batched solver's regions at k steps per phase (0 if
// no tile fits).
long long batch_tiles_per_slice(int H, int W, int k);

struct BatchRun {
    void *mem = nullptr;     // one device allocation (descriptors, tables, counters)
    void *desc = nullptr;
    void *counters = nullptr;
    size_t counters_bytes = 0;
    int *error = nullptr;
    size_t smem = 0;
    int grid = 0, storage = 0;
    int k = 0;                  // Chambolle steps per phase
    long long units_iter = 0;   // work units per iteration
};

// ---- differentiable unrolled solver (kernels_diff.cu) -------------------------
size_t unrolled_workspace_bytes(int B, int Z, int H, int W, int T, int S, int keep);
cslsm_status unrolled_forward(int B, int Z, int H, int W, float rho, float lam, float gam,
                              int K, int T, float tau, float eps, int S, const float *logits,
                              const float *b, float *vout, float *ckpt, void *ws, cudaStream_t s);
cslsm_status unrolled_backward(int B, int Z, int H, int W, float rho, float lam, float gam,
                               int K, int T, float tau, float eps, int S, int keep,
                               const float *logits, const float *b, const float *ckpt,
                               const float *vbar, float *logits_bar, double *scal_bar, void *ws,
                               cudaStream_t s);
cslsm_status batch_build(const BatchSpec &spec, BatchRun &run);
cslsm_status batch_set_wait(const BatchRun &run, double limit_s, int stall_test);
// Points item `item` of a built batch at another measurement and output
// (same alignment class as at build time), ordered on `s`.
cslsm_status batch_set_io(const BatchRun &run, int item, const float *b, float *v_out,
                          cudaStream_t s);
// Enqueues the counter reset and the persistent launch (no state reset).
cslsm_status batch_enqueue(const BatchRun &run, cudaStream_t s);

}  // namespace cslsm
