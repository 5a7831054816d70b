// Isotropic-TV prox of the u-step (Eq. u-sub / u-update) by Chambolle's dual
// projection, with the z-smoothness Gauss-Seidel input of Sec. III-C folded
// into the tile load.
//
//   g  = (rho w_n + gamma (u_{n-1} + u_{n+1})) / (rho + 2 gamma)   (gamma > 0)
//      = w_n                                                        (gamma = 0)
//   p^0 = 0,  q^t = div p^t - g / theta,
//   p^{t+1} = (p^t + tau grad q^t) / (1 + tau |grad q^t|),
//   u_n = g - theta div p^T,  d_n = w_n - u_n.
// grad: forward differences, zero on the last row / column; div = -grad^T.
//
// GB300 design: temporal blocking in shared memory.  One CTA owns a TH x TW
// output tile of one slice and loads g on the tile plus a halo of T+1 pixels
// (the dependence cone of T Chambolle steps), so all T steps run on chip and
// the dual field p never touches HBM; one launch performs the whole prox of
// every slice it covers.  HBM/L2 traffic per prox is one read of w (plus the
// two neighbouring u slices when gamma > 0) and one write of u and d.
//
// Inside a step every warp walks a band of rows top to bottom, one row per
// iteration; each lane owns two adjacent columns (float2 shared accesses).
// q of the next row is computed once and carried in registers, the right
// neighbour's q comes from a warp shuffle and the left neighbour's p from the
// float2 holding the two columns to the left (no lane-divergent load), so a
// pixel-step costs 2 shared loads and 1 store.  A warp spans 64 columns
// and owns 62 of them (column chunks overlap by two so that every chunk
// starts on an even column; the last lane only supplies q and p to its
// neighbours).  p is double-buffered in shared memory,
// so one __syncthreads per step suffices, and the row bands are re-balanced
// every step as the valid region shrinks by one pixel per side.  The Neumann
// boundary and the outside of the image are handled without branches:
// gradient components are multiplied by a 0/1 row / column mask, which keeps
// p = 0 wherever the discrete gradient vanishes.
//
// Step counts above kMaxSteps are split into chunks that hand p over through
// a double-buffered global array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "internal.cuh"
#include "storage.cuh"
#include "tv_body.cuh"

namespace cslsm {
namespace {

constexpr int kMaxSteps = 24;

inline size_t smem_bytes(int C, int RH) { return tv_smem_bytes(C, RH); }

constexpr size_t kSmemLimit = 227 * 1024;  // per CTA
constexpr size_t kSmemPerSm = 228 * 1024;

// Kernel variants: (column chunks, row bands).
struct Variant {
    int C, B;
};
constexpr Variant kVariants[] = {{1, 12}, {1, 24}, {2, 12}, {2, 16}};
constexpr int kNumVariants = 4;

struct Shape {
    int v, TH, TW, RH;  // variant index, tile rows / columns, region rows
};

std::mutex g_mu;
struct DeviceInfo {
    int sms = 0;
    bool ready = false;
};
std::vector<DeviceInfo> g_dev;
int g_mode = 0;  // 0: cost model, 1: timed autotuning, 2 + k: force variant k
struct Key {
    int dev, H, W, T, ns;
    bool operator<(const Key &o) const
    {
        return std::tie(dev, H, W, T, ns) < std::tie(o.dev, o.H, o.W, o.T, o.ns);
    }
};
std::map<Key, Shape> g_tuned;

template <int C, int B>
cslsm_status set_attr()
{
    const int lim = (int)kSmemLimit;
    CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel<C, B, float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel<C, B, __nv_bfloat16>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel<C, B, __half>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
    return CSLSM_OK;
}

cslsm_status device_info(int &dev, int &sms)
{
    CSLSM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DeviceInfo &di = g_dev[dev];
    if (!di.ready) {
        CSLSM_CUDA(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev));
        cslsm_status e;
        if ((e = set_attr<1, 12>()) || (e = set_attr<1, 24>()) || (e = set_attr<2, 12>()) ||
            (e = set_attr<2, 16>()))
            return e;
        di.ready = true;
    }
    sms = di.sms;
    return CSLSM_OK;
}

// Best tile rows for one variant under the cost model: waves of CTAs times the
// pixel-steps of one CTA's shrinking region, with a latency penalty when fewer
// than 32 warps share an SM.  Returns the modelled cost (inf if nothing fits).
double model_shape(int vi, int H, int W, int T, int nslices, int sms, Shape &out)
{
    const int C = kVariants[vi].C, B = kVariants[vi].B;
    const int RW = 62 * C + 2, TW = RW - 2 * T - 2;
    double best = 1e300;
    if (TW < 4) return best;
    const int tiles_w = (W + TW - 1) / TW, threads = C * B * 32;
    for (int TH = 4; TH <= 1024; TH += 2) {
        const int RH = TH + 2 * T + 2;
        const size_t sm = smem_bytes(C, RH);
        if (sm > kSmemLimit) break;
        const int per_sm = (int)std::min<size_t>(kSmemPerSm / (sm + 1024), 2048 / threads);
        if (per_sm < 1) break;
        const long long ctas = (long long)tiles_w * ((H + TH - 1) / TH) * nslices;
        const int resident = (int)std::min<long long>(per_sm, (ctas + sms - 1) / sms);
        const double waves = std::ceil((double)ctas / ((double)sms * per_sm));
        double work = 2.0 * RW * RH;  // pixel-steps of one CTA plus its load
        for (int s = 0; s < T; ++s) work += (double)(RW - 2 * s - 3) * (RH - 2 * s - 3);
        const double warps = (double)resident * C * B;
        const double cost = waves * work * per_sm * std::max(1.0, 32.0 / warps);
        if (cost < best) {
            best = cost;
            out = Shape{vi, TH, TW, RH};
        }
        if (TH >= H) break;
    }
    return best;
}

template <typename S>
void launch_variant(int v, dim3 grid, int nt, size_t sm, cudaStream_t st, const TvLaunch &b)
{
    switch (v) {
    case 0: tv_tile_kernel<1, 12, S><<<grid, nt, sm, st>>>(b); break;
    case 1: tv_tile_kernel<1, 24, S><<<grid, nt, sm, st>>>(b); break;
    case 2: tv_tile_kernel<2, 12, S><<<grid, nt, sm, st>>>(b); break;
    default: tv_tile_kernel<2, 16, S><<<grid, nt, sm, st>>>(b); break;
    }
}

cslsm_status launch_tile(const TvLaunch &a, const Shape &sh, cudaStream_t st)
{
    if (sh.RH <= 0) {
        set_error("no TV tile shape fits shared memory for %d steps", a.T);
        return CSLSM_ERR_UNSUPPORTED;
    }
    TvLaunch b = a;
    b.TH = sh.TH;
    b.TW = sh.TW;
    b.RH = sh.RH;
    const Variant v = kVariants[sh.v];
    const dim3 grid((a.W + sh.TW - 1) / sh.TW, (a.H + sh.TH - 1) / sh.TH, a.nslices);
    const size_t sm = smem_bytes(v.C, sh.RH);
    const int nt = v.C * v.B * 32;
    LaunchScope ls(K_TV_TILE, st);
    if (a.storage == CSLSM_STORE_BF16) launch_variant<__nv_bfloat16>(sh.v, grid, nt, sm, st, b);
    else if (a.storage == CSLSM_STORE_FP16) launch_variant<__half>(sh.v, grid, nt, sm, st, b);
    else launch_variant<float>(sh.v, grid, nt, sm, st, b);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

// Shape for this launch: forced variant, cached tuning result, cost model, or
// (mode 1, outside stream capture, first use of the key) timed candidates.
cslsm_status choose_shape(const TvLaunch &a, int dev, int sms, cudaStream_t st, bool may_time,
                          Shape &sh)
{
    int mode;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        mode = g_mode;
        if (mode == 1 && !may_time) mode = 0;
        if (mode == 1) {
            auto it = g_tuned.find(Key{dev, a.H, a.W, a.T, a.nslices});
            if (it != g_tuned.end()) {
                sh = it->second;
                return CSLSM_OK;
            }
        }
    }
    Shape cand[kNumVariants];
    double cost[kNumVariants];
    int best = -1;
    for (int v = 0; v < kNumVariants; ++v) {
        cand[v] = Shape{v, 0, 0, 0};
        cost[v] = model_shape(v, a.H, a.W, a.T, a.nslices, sms, cand[v]);
        if (cost[v] < 1e300 && (best < 0 || cost[v] < cost[best])) best = v;
    }
    if (mode >= 2) {
        const int v = (mode - 2) % kNumVariants;
        if (cost[v] < 1e300) best = v;
    }
    if (best < 0) {
        set_error("no TV tile shape fits shared memory for %d steps", a.T);
        return CSLSM_ERR_UNSUPPORTED;
    }
    sh = cand[best];
    if (mode != 1) return CSLSM_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CSLSM_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return CSLSM_OK;
    // time every variant (the launch is idempotent: same inputs, same outputs)
    cudaEvent_t e0, e1;
    CSLSM_CUDA(cudaEventCreate(&e0));
    CSLSM_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    for (int v = 0; v < kNumVariants; ++v) {
        if (cost[v] >= 1e300) continue;
        float ms_min = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, st);
            cslsm_status e = launch_tile(a, cand[v], st);
            cudaEventRecord(e1, st);
            if (e) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return e;
            }
            float ms = 0.f;
            if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) ==
                                                               cudaSuccess)
                ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            sh = cand[v];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_mu);
    g_tuned[Key{dev, a.H, a.W, a.T, a.nslices}] = sh;
    return CSLSM_OK;
}

}  // namespace

int tv_max_steps_per_launch() { return kMaxSteps; }

cslsm_status tv_query_shape(int H, int W, int T, int nslices, int *out4)
{
    int dev = 0, sms = 0;
    cslsm_status e = device_info(dev, sms);
    if (e) return e;
    TvLaunch a{};
    a.H = H;
    a.W = W;
    a.T = T;
    a.nslices = nslices;
    Shape sh{};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_mode == 1) {
            auto it = g_tuned.find(Key{dev, H, W, T, nslices});
            if (it != g_tuned.end()) {
                sh = it->second;
                out4[0] = sh.v;
                out4[1] = sh.TH;
                out4[2] = sh.TW;
                out4[3] = sh.RH;
                return CSLSM_OK;
            }
        }
    }
    if ((e = choose_shape(a, dev, sms, nullptr, false, sh))) return e;
    out4[0] = sh.v;
    out4[1] = sh.TH;
    out4[2] = sh.TW;
    out4[3] = sh.RH;
    return CSLSM_OK;
}

int tv_get_mode()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_mode;
}

void tv_set_mode(int mode)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_mode = mode;
    if (mode != 1) g_tuned.clear();
}

cslsm_status tv_prox_slices(const TvSlices &s, float *pbuf, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cslsm_status e = device_info(dev, sms);
    if (e) return e;
    TvLaunch a{};
    a.storage = s.storage;
    a.stop = s.stop;
    a.w = s.w;
    a.u = s.u;
    a.d = s.d;
    a.H = s.H;
    a.W = s.W;
    a.Z = s.Z;
    a.n0 = s.n0;
    a.nslices = s.nslices;
    a.rho = s.rho;
    a.gamma = s.Z > 1 ? s.gamma : 0.f;
    a.inv_rho2g = 1.f / (s.rho + 2.f * a.gamma);
    a.theta = s.theta;
    a.inv_theta = s.theta > 0.f ? 1.f / s.theta : 0.f;
    a.tau = s.tau;
    const int T = s.theta > 0.f ? s.T : 0;  // zero weight: the prox is the identity
    if (T <= kMaxSteps) {
        a.T = T;
        a.write_final = 1;
        Shape sh{};
        if ((e = choose_shape(a, dev, sms, st, true, sh))) return e;
        return launch_tile(a, sh, st);
    }
    if (!pbuf) {
        set_error("TV prox with %d steps needs the dual buffers", T);
        return CSLSM_ERR_INVALID_ARG;
    }
    const int nch = (T + kMaxSteps - 1) / kMaxSteps;
    const size_t half = 2ull * s.nslices * s.H * s.W;
    const float *pin = nullptr;
    int done = 0;
    for (int c = 0; c < nch; ++c) {
        const int steps = (T - done) / (nch - c);
        a.T = steps;
        a.pin = pin;
        a.write_final = (c == nch - 1);
        a.pout = a.write_final ? nullptr : pbuf + (c % 2) * half;
        Shape sh{};
        if ((e = choose_shape(a, dev, sms, st, false, sh))) return e;
        e = launch_tile(a, sh, st);
        if (e) return e;
        pin = a.pout;
        done += steps;
    }
    return CSLSM_OK;
}

}  // namespace cslsm
