// C ABI of libcslsm: argument checking, plan / workspace ownership and the
// host-side schedule of Algorithm 1.  All arithmetic runs in the kernels of
// kernels_pointwise.cu and kernels_tv.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <new>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace cslsm {

namespace {
thread_local char g_last_error[512] = "";
}

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

}  // namespace cslsm

using namespace cslsm;

struct cslsm_plan_s {
    Geom g;
    int device;
    int per_slice;
    uint32_t *words = nullptr;  // [nsets][H][W]
    int nsets = 0;
    float *u = nullptr, *d = nullptr, *w = nullptr;  // [Z][H][W] state and workspace
    float *vprev = nullptr;                          // [Z][H][W], tolerance checks only
    float *pbuf = nullptr;                           // TV dual buffers for long proxes
    size_t pbuf_floats = 0;
    double *partials = nullptr;  // reduction partials (2 doubles per block)
    int npartials = 0;
    double *red_out = nullptr;  // 2 doubles
    TolState *tol = nullptr;    // device-side stopping state of tolerance solves
    void *bm3d_ws = nullptr;     // BM3D workspace (zero-filled on allocation)
    size_t bm3d_ws_bytes = 0;
    ZsweepWs zs;                 // persistent z sweep (TV, gamma > 0)
    // slice-independent TV solves run as a one-item persistent batch, kept while
    // the parameters (and the alignment class of b and v_out) stay the same
    cslsm_batch route = nullptr;
    struct RouteKey {
        int io_align;  // 16, 8 or 4: alignment of the call's b and v_out
        float rho, lambda, tau;
        int T, iters, storage, tune, k;
        bool operator==(const RouteKey &o) const
        {
            return io_align == o.io_align && rho == o.rho && lambda == o.lambda &&
                   tau == o.tau && T == o.T && iters == o.iters && storage == o.storage &&
                   tune == o.tune && k == o.k;
        }
    } route_key{};
};

namespace {

#define CHECK_ARG(cond, ...)                    \
    do {                                        \
        if (!(cond)) {                          \
            set_error(__VA_ARGS__);             \
            return CSLSM_ERR_INVALID_ARG;       \
        }                                       \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

std::atomic<int> g_batch_k{0};   // cslsm_set_batch_steps_per_phase
std::atomic<int> g_tv_route{0};  // cslsm_set_tv_route

bool finite_f(float x) { return std::isfinite(x); }

cslsm_status check_geometry(int H, int W, int N, int R)
{
    CHECK_ARG(H >= 1 && W >= 1, "H and W must be >= 1 (got %d, %d)", H, W);
    CHECK_ARG(N >= 1, "n_shots must be >= 1 (got %d)", N);
    CHECK_ARG(R >= 1 && R <= CSLSM_MAX_R, "R must be in [1, %d] (got %d)", CSLSM_MAX_R, R);
    const long long v = (long long)N * R * H * W;
    CHECK_ARG(v < (1ll << 31), "Z*H*W must be < 2^31 (got %lld)", v);
    return CSLSM_OK;
}

cslsm_status check_params(const cslsm_admm_params *p, bool for_denoise)
{
    CHECK_ARG(p != nullptr, "params is NULL");
    CHECK_ARG(finite_f(p->rho) && p->rho > 0.f, "rho must be finite and > 0");
    CHECK_ARG(finite_f(p->lambda) && p->lambda >= 0.f, "lambda must be finite and >= 0");
    CHECK_ARG(p->denoiser >= CSLSM_DEN_TIKHONOV && p->denoiser <= CSLSM_DEN_WNNM,
              "unknown denoiser %d", p->denoiser);
    if (p->denoiser == CSLSM_DEN_TV) {
        CHECK_ARG(p->tv_inner >= 1, "tv_inner must be >= 1");
        CHECK_ARG(finite_f(p->tv_tau) && p->tv_tau > 0.f && p->tv_tau <= 0.25f,
                  "tv_tau must be in (0, 0.25]");
    }
    if (p->denoiser == CSLSM_DEN_BM3D || p->denoiser == CSLSM_DEN_WNNM)
        CHECK_ARG(finite_f(p->bm3d_sigma) && p->bm3d_sigma > 0.f, "bm3d_sigma must be > 0");
    if (for_denoise) return CSLSM_OK;
    CHECK_ARG(finite_f(p->gamma) && p->gamma >= 0.f, "gamma must be finite and >= 0");
    CHECK_ARG(p->iters >= 0, "iters must be >= 0");
    CHECK_ARG(finite_f(p->tol) && p->tol >= 0.f, "tol must be finite and >= 0");
    if (p->tol > 0.f) CHECK_ARG(p->check_every >= 1, "check_every must be >= 1 when tol > 0");
    CHECK_ARG(p->init_user == 0 || p->init_user == 1, "init_user must be 0 or 1");
    CHECK_ARG(p->storage >= CSLSM_STORE_FP32 && p->storage <= CSLSM_STORE_FP16,
              "unknown storage type %d", p->storage);
    return CSLSM_OK;
}

cslsm_status check_device(const cslsm_plan_s *plan)
{
    int dev = -1;
    CSLSM_CUDA(cudaGetDevice(&dev));
    CHECK_ARG(dev == plan->device, "plan belongs to device %d, current device is %d",
              plan->device, dev);
    return CSLSM_OK;
}

Masks masks_of(const cslsm_plan_s *p) { return Masks{p->words, p->nsets > 1 ? p->g.HW() : 0}; }

void free_plan(cslsm_plan_s *p)
{
    if (p->route) cslsm_batch_destroy(p->route);
    cudaFree(p->words);
    cudaFree(p->u);
    cudaFree(p->d);
    cudaFree(p->w);
    cudaFree(p->vprev);
    cudaFree(p->pbuf);
    zsweep_release(p->zs);
    cudaFree(p->partials);
    cudaFree(p->red_out);
    cudaFree(p->tol);
    cudaFree(p->bm3d_ws);
    delete p;
}

cslsm_status pack(cslsm_plan_s *p, const uint8_t *masks, int per_slice, cudaStream_t s)
{
    const int nsets = per_slice ? p->g.N : 1;
    CHECK_ARG(nsets == p->nsets || p->nsets == 0,
              "per_slice changes the number of pattern sets; create a new plan");
    return launch_pack_masks(masks, p->words, p->g.HW(), p->g.R, nsets, s);
}

}  // namespace

extern "C" {

int cslsm_abi_version(void) { return CSLSM_ABI_VERSION; }

const char *cslsm_status_string(cslsm_status st)
{
    switch (st) {
    case CSLSM_OK: return "CSLSM_OK";
    case CSLSM_ERR_INVALID_ARG: return "CSLSM_ERR_INVALID_ARG";
    case CSLSM_ERR_CUDA: return "CSLSM_ERR_CUDA";
    case CSLSM_ERR_TIMEOUT: return "CSLSM_ERR_TIMEOUT";
    case CSLSM_ERR_UNSUPPORTED: return "CSLSM_ERR_UNSUPPORTED";
    case CSLSM_ERR_OOM: return "CSLSM_ERR_OOM";
    }
    return "CSLSM_STATUS_UNKNOWN";
}

const char *cslsm_last_error(void) { return g_last_error; }

cslsm_status cslsm_plan_create(cslsm_plan *out, int H, int W, int n_shots, int R,
                               const uint8_t *masks, int per_slice, void *stream)
{
    CHECK_ARG(out != nullptr, "plan output pointer is NULL");
    *out = nullptr;
    cslsm_status st = check_geometry(H, W, n_shots, R);
    if (st) return st;
    CHECK_ARG(masks != nullptr, "masks is NULL");
    CHECK_ARG(per_slice == 0 || per_slice == 1, "per_slice must be 0 or 1");
    cslsm_plan_s *p = new (std::nothrow) cslsm_plan_s();
    CHECK_ARG(p != nullptr, "host allocation failed");
    p->g = Geom{H, W, n_shots, R};
    p->per_slice = per_slice;
    p->nsets = per_slice ? n_shots : 1;
    const size_t nv = (size_t)p->g.voxels();
    const dim3 grid_px((p->g.HW() + 255) / 256, n_shots);
    p->npartials = (int)(grid_px.x * grid_px.y);
    cudaStream_t s = as_stream(stream);
#define TRY(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            set_error("%s failed: %s", #call, cudaGetErrorString(e_));                      \
            free_plan(p);                                                                   \
            return e_ == cudaErrorMemoryAllocation ? CSLSM_ERR_OOM : CSLSM_ERR_CUDA;        \
        }                                                                                   \
    } while (0)
    TRY(cudaGetDevice(&p->device));
    TRY(cudaMalloc(&p->words, sizeof(uint32_t) * (size_t)p->nsets * p->g.HW()));
    TRY(cudaMalloc(&p->u, sizeof(float) * nv));
    TRY(cudaMalloc(&p->d, sizeof(float) * nv));
    TRY(cudaMalloc(&p->w, sizeof(float) * nv));
    TRY(cudaMalloc(&p->partials, sizeof(double) * 2 * (size_t)p->npartials));
    TRY(cudaMalloc(&p->red_out, sizeof(double) * 2));
#undef TRY
    st = pack(p, masks, per_slice, s);
    if (st == CSLSM_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("plan_create: %s", cudaGetErrorString(cudaGetLastError()));
        st = CSLSM_ERR_CUDA;
    }
    if (st) {
        free_plan(p);
        return st;
    }
    *out = p;
    return CSLSM_OK;
}

cslsm_status cslsm_plan_set_masks(cslsm_plan plan, const uint8_t *masks, int per_slice,
                                  void *stream)
{
    CHECK_ARG(plan != nullptr, "plan is NULL");
    CHECK_ARG(masks != nullptr, "masks is NULL");
    CHECK_ARG(per_slice == 0 || per_slice == 1, "per_slice must be 0 or 1");
    CHECK_ARG((per_slice ? plan->g.N : 1) == plan->nsets,
              "per_slice changes the number of pattern sets; create a new plan");
    cslsm_status st = check_device(plan);
    if (st) return st;
    plan->per_slice = per_slice;
    return pack(plan, masks, per_slice, as_stream(stream));
}

cslsm_status cslsm_plan_destroy(cslsm_plan plan)
{
    if (!plan) return CSLSM_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(plan->device);
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(plan);
    cudaSetDevice(cur);
    if (e != cudaSuccess) {
        set_error("plan_destroy: %s", cudaGetErrorString(e));
        return CSLSM_ERR_CUDA;
    }
    return CSLSM_OK;
}

cslsm_status cslsm_forward(cslsm_plan plan, const float *v, float *b, void *stream)
{
    CHECK_ARG(plan != nullptr, "plan is NULL");
    CHECK_ARG(v != nullptr && b != nullptr, "v and b must be non-NULL");
    cslsm_status st = check_device(plan);
    if (st) return st;
    return launch_forward(plan->g, masks_of(plan), v, b, as_stream(stream));
}

cslsm_status cslsm_adjoint(cslsm_plan plan, const float *b, float *v, void *stream)
{
    CHECK_ARG(plan != nullptr, "plan is NULL");
    CHECK_ARG(v != nullptr && b != nullptr, "v and b must be non-NULL");
    cslsm_status st = check_device(plan);
    if (st) return st;
    return launch_adjoint(plan->g, masks_of(plan), b, v, as_stream(stream));
}

namespace {

// A TV solve whose prox is slice-independent (gamma = 0 or Z = 1), with a fixed
// iteration count from u = d = 0 in the plan's own state, can run as a one-item
// persistent batch (the same bits as the per-launch tiles, which recompute a
// halo of T + 1 pixels in every launch).  Auto mode takes that path when one
// phase level holds enough tiles to fill the GPU twice over.
bool tv_route_applies(const cslsm_plan_s *plan, const cslsm_admm_params *prm, float gam,
                      bool use_tol, const void *u_io)
{
    const int mode = g_tv_route.load();
    if (mode == 1) return false;
    if (prm->denoiser != CSLSM_DEN_TV || !(prm->lambda > 0.f) || gam != 0.f || use_tol ||
        prm->init_user || u_io != nullptr || prm->iters < 1)
        return false;
    if (mode == 2) return true;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return false;
    const int k = std::min(prm->tv_inner, 10);
    return (long long)plan->g.Z() * batch_tiles_per_slice(plan->g.H, plan->g.W, k) >=
           4ll * sms;  // two CTAs per SM, twice over
}

cslsm_status batch_repoint(cslsm_batch bt, const float *b, float *v_out, cudaStream_t s);

cslsm_status routed_tv_solve(cslsm_plan plan, const float *b, const cslsm_admm_params *prm,
                             float *v_out, cslsm_admm_stats *stats, cudaStream_t s)
{
    const uintptr_t bv = (uintptr_t)b | (uintptr_t)v_out;
    const int io_align = bv % 16 == 0 ? 16 : bv % 8 == 0 ? 8 : 4;
    const cslsm_plan_s::RouteKey key{io_align,    prm->rho,     prm->lambda,
                                     prm->tv_tau, prm->tv_inner, prm->iters,
                                     prm->storage, tv_get_mode(), g_batch_k.load()};
    if (plan->route && !(plan->route_key == key)) {
        const cslsm_status st = cslsm_batch_destroy(plan->route);
        plan->route = nullptr;
        if (st) return st;
    }
    if (!plan->route) {
        const cslsm_batch_item it{plan, b, v_out};
        cslsm_admm_params p = *prm;
        p.gamma = 0.f;
        const cslsm_status st = cslsm_batch_create(&plan->route, &it, 1, &p, s);
        if (st) {
            plan->route = nullptr;
            return st;
        }
        plan->route_key = key;
    }
    cslsm_status st = batch_repoint(plan->route, b, v_out, s);
    if (st) return st;
    st = cslsm_batch_run(plan->route, s);
    if (st) return st;
    if (stats) {  // reports a device-side wait that ran out (synchronises `stream`)
        st = cslsm_batch_wait(plan->route, s);
        if (st) return st;
        stats->iters_done = prm->iters;
        stats->rel_change = -1.0;
    }
    return CSLSM_OK;
}

}  // namespace

cslsm_status cslsm_admm_solve(cslsm_plan plan, const float *b, const cslsm_admm_params *prm,
                              float *v_out, void *u_io, void *d_io, cslsm_admm_stats *stats,
                              void *stream)
{
    CHECK_ARG(plan != nullptr, "plan is NULL");
    CHECK_ARG(b != nullptr && v_out != nullptr, "b and v_out must be non-NULL");
    cslsm_status st = check_params(prm, false);
    if (st) return st;
    CHECK_ARG((u_io == nullptr) == (d_io == nullptr), "give both u_io and d_io or neither");
    CHECK_ARG(!prm->init_user || u_io != nullptr, "init_user needs u_io and d_io");
    st = check_device(plan);
    if (st) return st;

    const Geom &g = plan->g;
    const size_t nv = (size_t)g.voxels();
    cudaStream_t s = as_stream(stream);
    void *u = u_io ? u_io : (void *)plan->u;
    void *d = d_io ? d_io : (void *)plan->d;
    const int store = prm->storage;
    const size_t esz = store == CSLSM_STORE_FP32 ? 4 : 2;
    const float gam = g.Z() > 1 ? prm->gamma : 0.f;
    const bool use_tol = prm->tol > 0.f;
    if (tv_route_applies(plan, prm, gam, use_tol, u_io)) {
        st = routed_tv_solve(plan, b, prm, v_out, stats, s);
        // auto mode: a batch that does not fit (memory) leaves the solve to the
        // per-launch tiles; a forced batch reports it
        if (st != CSLSM_ERR_OOM || g_tv_route.load() == 2) return st;
        cudaGetLastError();  // the failed allocation's (non-sticky) error
    }
    if (!prm->init_user) {
        CSLSM_CUDA(cudaMemsetAsync(u, 0, esz * nv, s));
        CSLSM_CUDA(cudaMemsetAsync(d, 0, esz * nv, s));
    }
    if (use_tol) {
        if (!plan->vprev) CSLSM_CUDA(cudaMalloc(&plan->vprev, sizeof(float) * nv));
        if (!plan->tol) CSLSM_CUDA(cudaMalloc(&plan->tol, sizeof(TolState)));
        CSLSM_CUDA(cudaMemsetAsync(plan->vprev, 0, sizeof(float) * nv, s));
        CSLSM_CUDA(cudaMemsetAsync(plan->tol, 0, sizeof(TolState), s));
    }
    // tolerance solves stop on the device: every kernel of the iteration reads
    // this flag and returns at once after the check that met the tolerance
    const int *stop = use_tol ? reinterpret_cast<const int *>(plan->tol) : nullptr;  // .stop
    int checks = 0;
    const bool tv = prm->denoiser == CSLSM_DEN_TV;
    if (tv && prm->lambda > 0.f && prm->tv_inner > tv_max_steps_per_launch()) {
        const size_t need = 4 * (gam > 0.f ? 1 : (size_t)g.Z()) * (size_t)g.HW();
        if (plan->pbuf_floats < need) {
            CSLSM_CUDA(cudaStreamSynchronize(s));
            cudaFree(plan->pbuf);
            plan->pbuf = nullptr;
            plan->pbuf_floats = 0;
            CSLSM_CUDA(cudaMalloc(&plan->pbuf, sizeof(float) * need));
            plan->pbuf_floats = need;
        }
    }
    const bool patchwise = prm->denoiser == CSLSM_DEN_BM3D || prm->denoiser == CSLSM_DEN_WNNM;
    if (patchwise) {
        const size_t need = bm3d_workspace_bytes(gam > 0.f ? 1 : g.Z(), g.H, g.W);
        if (plan->bm3d_ws_bytes < need) {
            CSLSM_CUDA(cudaStreamSynchronize(s));
            cudaFree(plan->bm3d_ws);
            plan->bm3d_ws = nullptr;
            plan->bm3d_ws_bytes = 0;
            CSLSM_CUDA(cudaMalloc(&plan->bm3d_ws, need));
            CSLSM_CUDA(cudaMemsetAsync(plan->bm3d_ws, 0, need, s));
            plan->bm3d_ws_bytes = need;
        }
    }
    const Masks m = masks_of(plan);
    int k = 0;
    double rel = -1.0;
    bool stopped = false;
    bool used_zsweep = false;
    for (k = 0; k < prm->iters; ++k) {
        const bool last = (k == prm->iters - 1);
        const bool check = use_tol && k > 0 && ((k + 1) % prm->check_every == 0 || last);
        float *vo = last ? v_out : nullptr;
        float *vp = use_tol ? plan->vprev : nullptr;
        double *part = check ? plan->partials : nullptr;
        if (prm->denoiser == CSLSM_DEN_TIKHONOV) {
            st = launch_tikhonov_iter(g, m, store, u, d, b, prm->rho, prm->lambda, gam, vo, vp,
                                      part, plan->npartials, s, stop);
            if (st) return st;
        } else if (patchwise) {
            st = launch_xupdate_w(g, m, store, u, d, b, prm->rho, plan->w, vo, vp, part,
                                  plan->npartials, s, stop);
            if (st) return st;
            Bm3dSlices a{};
            a.stop = stop;
            a.storage = store;
            a.src = plan->w;
            a.u = u;
            a.out = u;
            a.dual = d;
            a.Z = g.Z();
            a.H = g.H;
            a.W = g.W;
            a.rho = prm->rho;
            a.gamma = gam;
            a.sigma = prm->bm3d_sigma;
            if (gam == 0.f) {
                a.n0 = 0;
                a.nslices = g.Z();
                st = prm->denoiser == CSLSM_DEN_WNNM ? wnnm_slices(a, plan->bm3d_ws, s)
                                                     : bm3d_slices(a, plan->bm3d_ws, s);
                if (st) return st;
            } else {
                a.nslices = 1;
                for (int n = 0; n < g.Z(); ++n) {
                    a.n0 = n;
                    st = prm->denoiser == CSLSM_DEN_WNNM ? wnnm_slices(a, plan->bm3d_ws, s)
                                                         : bm3d_slices(a, plan->bm3d_ws, s);
                    if (st) return st;
                }
            }
        } else {
            st = launch_xupdate_w(g, m, store, u, d, b, prm->rho, plan->w, vo, vp, part,
                                  plan->npartials, s, stop);
            if (st) return st;
            TvSlices a{};
            a.stop = stop;
            a.storage = store;
            a.w = plan->w;
            a.u = u;
            a.d = d;
            a.H = g.H;
            a.W = g.W;
            a.Z = g.Z();
            a.rho = prm->rho;
            a.gamma = gam;
            a.theta = prm->lambda / (prm->rho + 2.f * gam);
            a.tau = prm->tv_tau;
            a.T = prm->tv_inner;
            if (gam == 0.f) {
                a.n0 = 0;
                a.nslices = g.Z();
                st = tv_prox_slices(a, plan->pbuf, s);
                if (st) return st;
            } else {
                a.n0 = 0;
                a.nslices = g.Z();
                bool swept = false;
                if (zsweep_applies(a)) {
                    if (!plan->zs.pbuf) {
                        CSLSM_CUDA(cudaStreamSynchronize(s));
                        st = zsweep_reserve(plan->zs, g.H, g.W);
                        if (st) return st;
                    }
                    st = zsweep_run(a, plan->zs, s);
                    if (st && !(st == CSLSM_ERR_UNSUPPORTED && !zsweep_forced())) return st;
                    swept = st == CSLSM_OK;  // else: no tiling fits; per-slice launches
                    used_zsweep = used_zsweep || swept;
                }
                if (!swept) {
                    a.nslices = 1;
                    for (int n = 0; n < g.Z(); ++n) {
                        a.n0 = n;
                        st = tv_prox_slices(a, plan->pbuf, s);
                        if (st) return st;
                    }
                }
            }
        }
        if (check) {
            const int nblk = prm->denoiser == CSLSM_DEN_TIKHONOV ? (g.HW() + 255) / 256
                                                                 : plan->npartials;
            st = launch_sum_pairs(plan->partials, nblk, plan->red_out, s);
            if (st) return st;
            st = launch_tol_check(plan->red_out, prm->tol, k, plan->tol, s);
            if (st) return st;
            ++checks;
        }
    }
    if (used_zsweep) {
        st = zsweep_check(plan->zs, s);
        if (st) return st;
    }
    if (use_tol && prm->iters > 0) {
        // a stopped solve's v^{k} is in vprev; then read the outcome (one sync)
        st = launch_copy_if_stopped(plan->tol, plan->vprev, v_out, nv, s);
        if (st) return st;
        TolState h{};
        CSLSM_CUDA(cudaMemcpyAsync(&h, plan->tol, sizeof(h), cudaMemcpyDeviceToHost, s));
        CSLSM_CUDA(cudaStreamSynchronize(s));
        stopped = h.stop != 0;
        k = stopped ? h.iters_done : prm->iters;
        rel = checks > 0 ? h.rel : -1.0;
    }
    if (prm->iters == 0) {  // v^0: nothing computed; report zeros
        CSLSM_CUDA(cudaMemsetAsync(v_out, 0, sizeof(float) * nv, s));
    }
    if (stats) {
        stats->iters_done = k;
        stats->rel_change = use_tol ? rel : -1.0;
    }
    return CSLSM_OK;
}

cslsm_status cslsm_denoise(int denoiser, const float *in, float *out, int Z, int H, int W,
                           const cslsm_admm_params *prm, void *stream)
{
    CHECK_ARG(in != nullptr && out != nullptr, "in and out must be non-NULL");
    CHECK_ARG(Z >= 1 && H >= 1 && W >= 1, "Z, H, W must be >= 1");
    CHECK_ARG((long long)Z * H * W < (1ll << 31), "Z*H*W must be < 2^31");
    cslsm_status st = check_params(prm, true);
    if (st) return st;
    CHECK_ARG(denoiser == prm->denoiser, "denoiser argument and params->denoiser differ");
    const size_t nv = (size_t)Z * H * W;
    if (denoiser != CSLSM_DEN_TIKHONOV) {
        const char *a = (const char *)in, *o = (const char *)out;
        CHECK_ARG(o + nv * sizeof(float) <= a || a + nv * sizeof(float) <= o,
                  "in and out must not overlap");
    }
    cudaStream_t s = as_stream(stream);
    if (denoiser == CSLSM_DEN_TIKHONOV)
        return launch_tikhonov_prox(in, out, (long long)nv, prm->rho, prm->lambda, s);
    if (denoiser == CSLSM_DEN_BM3D || denoiser == CSLSM_DEN_WNNM) {
        const size_t need = bm3d_workspace_bytes(Z, H, W);
        void *ws = nullptr;
        CSLSM_CUDA(cudaMallocAsync(&ws, need, s));
        cudaError_t e = cudaMemsetAsync(ws, 0, need, s);
        if (e != cudaSuccess) {
            cudaFreeAsync(ws, s);
            set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
            return CSLSM_ERR_CUDA;
        }
        Bm3dSlices a{};
        a.storage = CSLSM_STORE_FP32;
        a.src = in;
        a.u = nullptr;
        a.out = out;
        a.dual = nullptr;
        a.Z = Z;
        a.H = H;
        a.W = W;
        a.n0 = 0;
        a.nslices = Z;
        a.rho = 1.f;
        a.gamma = 0.f;
        a.sigma = prm->bm3d_sigma;
        st = denoiser == CSLSM_DEN_WNNM ? wnnm_slices(a, ws, s) : bm3d_slices(a, ws, s);
        cudaFreeAsync(ws, s);
        return st;
    }
    TvSlices a{};
    a.storage = CSLSM_STORE_FP32;
    a.w = in;
    a.u = out;
    a.d = nullptr;
    a.H = H;
    a.W = W;
    a.Z = Z;
    a.n0 = 0;
    a.nslices = Z;
    a.rho = prm->rho;
    a.gamma = 0.f;
    a.theta = prm->lambda / prm->rho;
    a.tau = prm->tv_tau;
    a.T = prm->tv_inner;
    float *pbuf = nullptr;
    if (a.theta > 0.f && a.T > tv_max_steps_per_launch())
        CSLSM_CUDA(cudaMallocAsync(&pbuf, sizeof(float) * 4 * nv, s));
    st = tv_prox_slices(a, pbuf, s);
    if (pbuf) cudaFreeAsync(pbuf, s);
    return st;
}

}  // extern "C"

struct cslsm_batch_s {
    int device;
    BatchRun run;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<std::pair<void *, size_t>> zero;  // state buffers zeroed by each run
};

namespace {

cslsm_status batch_repoint(cslsm_batch bt, const float *b, float *v_out, cudaStream_t s)
{
    return batch_set_io(bt->run, 0, b, v_out, s);
}

}  // namespace

namespace {

void free_batch(cslsm_batch_s *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->run.mem);
    delete b;
}

cslsm_status build_and_capture(cslsm_batch_s *bt, const BatchSpec &spec)
{
    cslsm_status st = batch_build(spec, bt->run);
    if (st) return st;
    cudaStream_t cs = nullptr;
    CSLSM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (auto &z : bt->zero)
            if ((e = cudaMemsetAsync(z.first, 0, z.second, cs)) != cudaSuccess) break;
        if (e == cudaSuccess) st = batch_enqueue(bt->run, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
        bt->graph = g;
    }
    if (e == cudaSuccess && !st) e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
    cudaStreamDestroy(cs);
    if (st) return st;
    if (e != cudaSuccess) {
        set_error("batch graph capture: %s", cudaGetErrorString(e));
        return CSLSM_ERR_CUDA;
    }
    return CSLSM_OK;
}

}  // namespace

extern "C" {

cslsm_status cslsm_batch_create(cslsm_batch *out, const cslsm_batch_item *items, int n_items,
                                const cslsm_admm_params *prm, void *stream)
{
    CHECK_ARG(out != nullptr, "batch output pointer is NULL");
    *out = nullptr;
    CHECK_ARG(items != nullptr && n_items >= 1, "need at least one item");
    cslsm_status st = check_params(prm, false);
    if (st) return st;
    CHECK_ARG(prm->denoiser == CSLSM_DEN_TV, "the batched solver runs the TV prior");
    CHECK_ARG(prm->tol == 0.f, "the batched solver runs a fixed iteration count (tol = 0)");
    CHECK_ARG(prm->init_user == 0, "the batched solver starts from u = d = 0");
    CHECK_ARG(prm->iters >= 1, "iters must be >= 1");
    int dev = 0;
    for (int i = 0; i < n_items; ++i) {
        CHECK_ARG(items[i].plan && items[i].b && items[i].v_out, "item %d is incomplete", i);
        if (i == 0) dev = items[i].plan->device;
        CHECK_ARG(items[i].plan->device == dev, "items on different devices");
    }
    int cur = -1;
    CSLSM_CUDA(cudaGetDevice(&cur));
    CHECK_ARG(cur == dev, "the items' plans belong to device %d, current device is %d", dev, cur);
    cudaStream_t s = as_stream(stream);
    CSLSM_CUDA(cudaStreamSynchronize(s));
    cslsm_batch_s *bt = new (std::nothrow) cslsm_batch_s();
    CHECK_ARG(bt != nullptr, "host allocation failed");
    bt->device = dev;
    const int T = prm->lambda > 0.f ? prm->tv_inner : 0;
    BatchSpec spec;
    spec.iters = prm->iters;
    spec.T = prm->tv_inner;
    spec.storage = prm->storage;
    spec.stall_test = 0;
    spec.rho = prm->rho;
    spec.lam = prm->lambda;
    spec.gamma = prm->gamma;
    spec.tau = prm->tv_tau;
    spec.wait_limit_s = 4.0;
    const size_t esz = prm->storage == CSLSM_STORE_FP32 ? 4 : 2;
    for (int i = 0; i < n_items; ++i) {
        const cslsm_plan_s *p = items[i].plan;
        BatchItemSpec it{};
        it.u = p->u;
        it.d = p->d;
        it.w = p->w;
        it.b = items[i].b;
        it.v_out = items[i].v_out;
        it.words = p->words;
        it.wstride = p->nsets > 1 ? p->g.HW() : 0;
        it.H = p->g.H;
        it.W = p->g.W;
        it.N = p->g.N;
        it.R = p->g.R;
        spec.items.push_back(it);
        bt->zero.push_back({p->u, esz * (size_t)p->g.voxels()});
        bt->zero.push_back({p->d, esz * (size_t)p->g.voxels()});
    }
    // steps per phase: a fixed default unless a phase length is set or timing
    // a few candidates on the batch itself is asked for (autotune mode 1)
    int kbest = std::min(std::max(T, 1), 10);
    const int kset = g_batch_k;
    if (kset > 0) {
        kbest = std::min({kset, std::max(T, 1), batch_max_steps_per_phase()});
    } else if (tv_get_mode() == 1 && T > 0) {
        float best = 1e30f;
        // balanced phases: ceil(T / P) steps for P = 1, 2, ... phases (a short
        // trailing phase pays a unit's fixed loads for little work), no more
        // than fit the region's halo, none below 5 unless T is, four at most
        std::vector<int> cand;
        for (int P = 1; P <= T && cand.size() < 4; ++P) {
            const int c = (T + P - 1) / P;
            if (c > batch_max_steps_per_phase() || c < std::min(5, T)) continue;
            if (std::find(cand.begin(), cand.end(), c) == cand.end()) cand.push_back(c);
        }
        for (int c : cand) {
            BatchSpec trial = spec;
            trial.iters = 1;
            trial.k = c;
            cslsm_batch_s probe;
            probe.device = dev;
            probe.zero = bt->zero;
            st = batch_build(trial, probe.run);
            float ms = 1e30f;
            if (!st) {
                cudaEvent_t e0, e1;
                cudaEventCreate(&e0);
                cudaEventCreate(&e1);
                // two runs, the faster one counts: the first launch of a
                // candidate may carry one-time costs
                for (int rep = 0; rep < 2 && !st; ++rep) {
                    for (auto &z : probe.zero) cudaMemsetAsync(z.first, 0, z.second, s);
                    cudaEventRecord(e0, s);
                    st = batch_enqueue(probe.run, s);
                    cudaEventRecord(e1, s);
                    float t = 1e30f;
                    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1))
                        t = 1e30f;
                    ms = std::min(ms, t);
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
            }
            cudaFree(probe.run.mem);
            probe.run.mem = nullptr;
            if (st) {
                free_batch(bt);
                return st;
            }
            if (ms < best) {
                best = ms;
                kbest = c;
            }
        }
    }
    spec.k = kbest;
    st = build_and_capture(bt, spec);
    if (st) {
        free_batch(bt);
        return st;
    }
    *out = bt;
    return CSLSM_OK;
}

cslsm_status cslsm_batch_info(cslsm_batch batch, int *steps_per_phase, int *grid,
                              long long *units_per_iteration)
{
    CHECK_ARG(batch != nullptr, "batch is NULL");
    if (steps_per_phase) *steps_per_phase = batch->run.k;
    if (grid) *grid = batch->run.grid;
    if (units_per_iteration) *units_per_iteration = batch->run.units_iter;
    return CSLSM_OK;
}

cslsm_status cslsm_batch_run(cslsm_batch batch, void *stream)
{
    CHECK_ARG(batch != nullptr, "batch is NULL");
    int cur = -1;
    CSLSM_CUDA(cudaGetDevice(&cur));
    CHECK_ARG(cur == batch->device, "batch belongs to device %d", batch->device);
    LaunchScope ls(K_BATCH, as_stream(stream));
    CSLSM_CUDA(cudaGraphLaunch(batch->exec, as_stream(stream)));
    return CSLSM_OK;
}

cslsm_status cslsm_batch_wait(cslsm_batch batch, void *stream)
{
    CHECK_ARG(batch != nullptr, "batch is NULL");
    CSLSM_CUDA(cudaStreamSynchronize(as_stream(stream)));
    int err = 0;
    CSLSM_CUDA(cudaMemcpy(&err, batch->run.error, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        set_error("a device-side wait of the batched solver ran out of time");
        return CSLSM_ERR_TIMEOUT;
    }
    return CSLSM_OK;
}

cslsm_status cslsm_batch_set_wait_limit(cslsm_batch batch, double seconds, int test_stall)
{
    CHECK_ARG(batch != nullptr, "batch is NULL");
    CHECK_ARG(seconds > 0.0 && seconds <= 600.0, "seconds must be in (0, 600]");
    CHECK_ARG(test_stall == 0 || test_stall == 1, "test_stall must be 0 or 1");
    CSLSM_CUDA(cudaDeviceSynchronize());
    return batch_set_wait(batch->run, seconds, test_stall);
}

cslsm_status cslsm_batch_destroy(cslsm_batch batch)
{
    if (!batch) return CSLSM_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(batch);
    if (e != cudaSuccess) {
        set_error("batch_destroy: %s", cudaGetErrorString(e));
        return CSLSM_ERR_CUDA;
    }
    return CSLSM_OK;
}

namespace {
cslsm_status check_unrolled(int B, int Z, int H, int W, const cslsm_unrolled_params *p)
{
    CHECK_ARG(p != nullptr, "params is NULL");
    CHECK_ARG(B >= 1 && Z >= 1 && H >= 1 && W >= 1, "B, Z, H, W must be >= 1");
    CHECK_ARG((long long)B * Z * H * W < (1ll << 31), "B*Z*H*W must be < 2^31");
    CHECK_ARG(std::isfinite(p->rho) && p->rho > 0.f, "rho must be > 0");
    CHECK_ARG(std::isfinite(p->lambda) && p->lambda > 0.f, "lambda must be > 0");
    CHECK_ARG(std::isfinite(p->gamma) && p->gamma >= 0.f, "gamma must be >= 0");
    CHECK_ARG(p->iters >= 1 && p->tv_steps >= 1 && p->ckpt_every >= 1,
              "iters, tv_steps, ckpt_every must be >= 1");
    CHECK_ARG(std::isfinite(p->tv_tau) && p->tv_tau > 0.f && p->tv_tau <= 0.125f,
              "tv_tau must be in (0, 1/8]");
    CHECK_ARG(std::isfinite(p->huber_eps) && p->huber_eps >= 0.f, "huber_eps must be >= 0");
    CHECK_ARG(p->keep_duals == 0 || p->keep_duals == 1, "keep_duals must be 0 or 1");
    return CSLSM_OK;
}
}  // namespace

size_t cslsm_unrolled_workspace_bytes(int B, int Z, int H, int W, const cslsm_unrolled_params *p)
{
    if (check_unrolled(B, Z, H, W, p)) return 0;
    return unrolled_workspace_bytes(B, Z, H, W, p->tv_steps, p->ckpt_every, p->keep_duals);
}

cslsm_status cslsm_unrolled_forward(const float *logits, const float *b, int B, int Z, int H,
                                    int W, const cslsm_unrolled_params *p, float *v_out,
                                    float *ckpt, void *ws, void *stream)
{
    cslsm_status st = check_unrolled(B, Z, H, W, p);
    if (st) return st;
    CHECK_ARG(logits && b && v_out && ckpt && ws, "logits, b, v_out, ckpt, ws must be non-NULL");
    return unrolled_forward(B, Z, H, W, p->rho, p->lambda, p->gamma, p->iters, p->tv_steps,
                            p->tv_tau, p->huber_eps, p->ckpt_every, logits, b, v_out, ckpt, ws,
                            as_stream(stream));
}

cslsm_status cslsm_unrolled_backward(const float *logits, const float *b, int B, int Z, int H,
                                     int W, const cslsm_unrolled_params *p, const float *ckpt,
                                     const float *v_bar, float *logits_bar, double *scalar_bar,
                                     void *ws, void *stream)
{
    cslsm_status st = check_unrolled(B, Z, H, W, p);
    if (st) return st;
    CHECK_ARG(logits && b && ckpt && v_bar && logits_bar && scalar_bar && ws,
              "every pointer must be non-NULL");
    return unrolled_backward(B, Z, H, W, p->rho, p->lambda, p->gamma, p->iters, p->tv_steps,
                             p->tv_tau, p->huber_eps, p->ckpt_every, p->keep_duals, logits, b,
                             ckpt, v_bar, logits_bar, scalar_bar, ws, as_stream(stream));
}

cslsm_status cslsm_set_tv_route(int mode)
{
    CHECK_ARG(mode >= 0 && mode <= 2, "TV route mode must be 0, 1 or 2");
    g_tv_route = mode;
    return CSLSM_OK;
}

cslsm_status cslsm_set_batch_steps_per_phase(int k)
{
    CHECK_ARG(k >= 0, "steps per phase must be >= 0 (0: default / timed)");
    g_batch_k = k;
    return CSLSM_OK;
}

cslsm_status cslsm_set_autotune(int mode)
{
    CHECK_ARG(mode >= 0 && mode <= 5, "autotune mode must be in [0, 5]");
    tv_set_mode(mode);
    return CSLSM_OK;
}

cslsm_status cslsm_tv_shape(int H, int W, int steps, int nslices, int *shape4)
{
    CHECK_ARG(shape4 != nullptr, "shape4 is NULL");
    CHECK_ARG(H >= 1 && W >= 1 && nslices >= 1, "H, W, nslices must be >= 1");
    CHECK_ARG(steps >= 0 && steps <= tv_max_steps_per_launch(), "steps must be in [0, %d]",
              tv_max_steps_per_launch());
    return tv_query_shape(H, W, steps, nslices, shape4);
}

cslsm_status cslsm_zsweep_config(int enable, int tiling, double wait_limit_s, int test_stall)
{
    CHECK_ARG(enable == 0 || enable == 1, "enable must be 0 or 1");
    CHECK_ARG(tiling < zsweep_num_candidates(), "tiling must be < %d", zsweep_num_candidates());
    CHECK_ARG(std::isfinite(wait_limit_s) && wait_limit_s > 0.0 && wait_limit_s <= 3600.0,
              "wait_limit_s must be in (0, 3600]");
    zsweep_config(enable, tiling < 0 ? -1 : tiling, wait_limit_s, test_stall != 0);
    return CSLSM_OK;
}

int cslsm_zsweep_num_tilings(void) { return zsweep_num_candidates(); }

cslsm_status cslsm_zsweep_shape(int H, int W, int Z, int steps, int storage, int *out8)
{
    CHECK_ARG(out8 != nullptr, "out8 is NULL");
    CHECK_ARG(H >= 1 && W >= 1 && Z >= 2 && steps >= 1, "need H, W >= 1, Z >= 2, steps >= 1");
    CHECK_ARG(storage >= CSLSM_STORE_FP32 && storage <= CSLSM_STORE_FP16, "bad storage");
    return zsweep_query(H, W, Z, steps, storage, out8);
}

int cslsm_bm3d_num_refs(int H, int W) { return (H >= 1 && W >= 1) ? bm3d_nref(H, W) : 0; }

cslsm_status cslsm_bm3d_match(const float *img, int Z, int H, int W, int stage, int *lists,
                              int *counts, void *stream)
{
    CHECK_ARG(img != nullptr && lists != nullptr && counts != nullptr,
              "img, lists and counts must be non-NULL");
    CHECK_ARG(Z >= 1 && H >= 8 && W >= 8, "need Z >= 1 and H, W >= 8");
    CHECK_ARG((long long)Z * H * W < (1ll << 31), "Z*H*W must be < 2^31");
    CHECK_ARG(stage == 1 || stage == 2, "stage must be 1 or 2");
    cudaStream_t s = as_stream(stream);
    const size_t need = bm3d_workspace_bytes(Z, H, W);
    void *ws = nullptr;
    CSLSM_CUDA(cudaMallocAsync(&ws, need, s));
    cslsm_status st = bm3d_match_only(img, Z, H, W, stage, lists, counts, ws, s);
    cudaFreeAsync(ws, s);
    return st;
}

cslsm_status cslsm_bm3d_stage(int stage, const float *noisy, const float *guide, float *out,
                              int Z, int H, int W, float sigma, void *stream)
{
    CHECK_ARG(noisy != nullptr && out != nullptr, "noisy and out must be non-NULL");
    CHECK_ARG(stage == 1 || (stage == 2 && guide != nullptr),
              "stage must be 1, or 2 with a guide");
    CHECK_ARG(Z >= 1 && H >= 1 && W >= 1, "Z, H, W must be >= 1");
    CHECK_ARG((long long)Z * H * W < (1ll << 31), "Z*H*W must be < 2^31");
    CHECK_ARG(std::isfinite(sigma) && sigma > 0.f, "sigma must be > 0");
    cudaStream_t s = as_stream(stream);
    const size_t need = bm3d_workspace_bytes(Z, H, W);
    void *ws = nullptr;
    CSLSM_CUDA(cudaMallocAsync(&ws, need, s));
    cudaError_t e = cudaMemsetAsync(ws, 0, need, s);
    cslsm_status st = CSLSM_OK;
    if (e != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
        st = CSLSM_ERR_CUDA;
    } else {
        st = bm3d_stage_only(stage, noisy, guide, out, Z, H, W, sigma, ws, s);
    }
    cudaFreeAsync(ws, s);
    return st;
}

cslsm_status cslsm_bm3d_stage_groups(int stage, const float *noisy, const float *guide,
                                     float *out, int Z, int H, int W, float sigma, int *lists,
                                     int *counts, float *group_stat, void *stream)
{
    CHECK_ARG(noisy != nullptr && out != nullptr, "noisy and out must be non-NULL");
    CHECK_ARG(lists != nullptr && counts != nullptr && group_stat != nullptr,
              "lists, counts and group_stat must be non-NULL");
    CHECK_ARG(stage == 1 || (stage == 2 && guide != nullptr),
              "stage must be 1, or 2 with a guide");
    CHECK_ARG(Z >= 1 && H >= 8 && W >= 8, "need Z >= 1 and H, W >= 8");
    CHECK_ARG((long long)Z * H * W < (1ll << 31), "Z*H*W must be < 2^31");
    CHECK_ARG(std::isfinite(sigma) && sigma > 0.f, "sigma must be > 0");
    cudaStream_t s = as_stream(stream);
    const size_t need = bm3d_workspace_bytes(Z, H, W);
    void *ws = nullptr;
    CSLSM_CUDA(cudaMallocAsync(&ws, need, s));
    cudaError_t e = cudaMemsetAsync(ws, 0, need, s);
    cslsm_status st = CSLSM_OK;
    if (e != cudaSuccess) {
        set_error("cudaMemsetAsync: %s", cudaGetErrorString(e));
        st = CSLSM_ERR_CUDA;
    } else {
        st = bm3d_stage_only(stage, noisy, guide, out, Z, H, W, sigma, ws, s, lists, counts,
                             group_stat);
    }
    cudaFreeAsync(ws, s);
    return st;
}

cslsm_status cslsm_psnr(const float *x, const float *ref, size_t n, double *out, void *stream)
{
    CHECK_ARG(x != nullptr && ref != nullptr && out != nullptr, "x, ref, out must be non-NULL");
    CHECK_ARG(n >= 1, "n must be >= 1");
    cudaStream_t s = as_stream(stream);
    const int nb = reduction_blocks();
    double *partials = nullptr;
    CSLSM_CUDA(cudaMallocAsync(&partials, sizeof(double) * 2 * nb, s));
    cslsm_status st = launch_psnr_partials(x, ref, n, partials, nb, s);
    if (!st) st = launch_psnr_finish(partials, nb, n, out, s);
    cudaFreeAsync(partials, s);
    return st;
}

cslsm_status cslsm_ssim3d(const float *x, const float *ref, int Z, int H, int W, double *out,
                          void *stream)
{
    CHECK_ARG(x != nullptr && ref != nullptr && out != nullptr, "x, ref, out must be non-NULL");
    CHECK_ARG(Z >= 1 && H >= 1 && W >= 1, "Z, H, W must be >= 1");
    CHECK_ARG((long long)Z * H * W < (1ll << 31), "Z*H*W must be < 2^31");
    cudaStream_t s = as_stream(stream);
    int nb = 0;
    const size_t bytes = ssim3d_workspace_bytes(Z, H, W, &nb);
    void *ws = nullptr;
    CSLSM_CUDA(cudaMallocAsync(&ws, bytes, s));
    cslsm_status st = launch_ssim3d(x, ref, Z, H, W, ws, nb, out, s);
    cudaFreeAsync(ws, s);
    return st;
}

}  // extern "C"
