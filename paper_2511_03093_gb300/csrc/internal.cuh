// Internal declarations shared by the cslsm translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

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
    K_REDUCE, K_COUNT
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
cslsm_status launch_xupdate_w(const Geom &g, Masks m, const float *u, const float *d,
                              const float *b, float rho, float *w, float *v_out, float *vprev,
                              double *partials, int nblocks_red, cudaStream_t s);

// One whole ADMM iteration with the Tikhonov prior fused into one pass:
// v-update, Gauss-Seidel Tikhonov sweep along z (gamma > 0) and dual update.
cslsm_status launch_tikhonov_iter(const Geom &g, Masks m, float *u, float *d, const float *b,
                                  float rho, float lam, float gam, float *v_out, float *vprev,
                                  double *partials, int nblocks_red, cudaStream_t s);

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
    const float *w;      // [Z][H][W] prox input source (w = v + d)
    float *u;            // [Z][H][W] output u_n (and u_{n-1}, u_{n+1} source)
    float *d;            // [Z][H][W] output d_n = w_n - u_n, or nullptr
    int H, W, Z;
    int n0, nslices;     // slices n0 .. n0+nslices-1
    float rho, gamma;    // g = (rho w + gamma (u_{n-1} + u_{n+1})) / (rho + 2 gamma)
    float theta;         // TV weight of the prox
    float tau;
    int T;               // Chambolle steps
};
// Chambolle TV prox of every listed slice.  Uses the plan-provided dual
// buffers pbuf (4 * nslices * H * W floats) only when T exceeds the largest
// step count one launch covers; pbuf may be nullptr otherwise.
cslsm_status tv_prox_slices(const TvSlices &a, float *pbuf, cudaStream_t s);
int tv_max_steps_per_launch();

}  // namespace cslsm
