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
// iteration, with lane = column: q of the next row is computed once and
// carried in a register, the right neighbour's q comes from a warp shuffle,
// so a pixel-step costs 4 shared loads and 2 stores.  Warps own 31 of their
// 32 columns (column chunks overlap by one, the 32nd lane only supplies q to
// its left neighbour).  p is double-buffered in shared memory, so one
// __syncthreads per step suffices, and the row bands are re-balanced every
// step as the valid region shrinks by one pixel per side.  The Neumann
// boundary and the outside of the image are handled without branches:
// gradient components are multiplied by a 0/1 row / column mask, which keeps
// p = 0 wherever the discrete gradient vanishes.
//
// Step counts above kMaxSteps are split into chunks that hand p over through
// a double-buffered global array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace cslsm {
namespace {

constexpr int kMaxSteps = 24;
constexpr int kBands = 8;  // row bands per CTA (warps per column chunk)

struct TvLaunch {
    const float *w;
    float *u;
    float *d;
    const float *pin;  // [2][nslices][H][W] dual field entering this launch, or null (p = 0)
    float *pout;       // [2][nslices][H][W] dual field leaving it (write_final == 0)
    int H, W, Z, n0, nslices;
    int T;             // steps in this launch
    int TH, TW, RH;    // tile rows / columns, region rows (region columns: 31 C + 1)
    float rho, gamma, inv_rho2g;
    float theta, inv_theta, tau;
    int write_final;
};

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int C>
__global__ void __launch_bounds__(C * kBands * 32) tv_tile_kernel(const TvLaunch a)
{
    constexpr int RW = 31 * C + 1;
    constexpr int NT = C * kBands * 32;
    extern __shared__ float smem[];
    const int T = a.T, RH = a.RH, RA = RW * RH;
    float *sg = smem;
    float *A1 = sg + RA, *A2 = A1 + RA;  // p^t   (components along rows / columns)
    float *B1 = A2 + RA, *B2 = B1 + RA;  // p^t+1
    const int sl = blockIdx.z;
    const int n = a.n0 + sl;
    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    const int gi0 = blockIdx.y * a.TH - (T + 1);
    const int gj0 = blockIdx.x * a.TW - (T + 1);

    const float *wn = a.w + (size_t)n * HW;
    const float *um = a.u + (size_t)((n + a.Z - 1) % a.Z) * HW;
    const float *up = a.u + (size_t)((n + 1) % a.Z) * HW;
    const float *p1in = a.pin ? a.pin + (size_t)sl * HW : nullptr;
    const float *p2in = a.pin ? a.pin + (size_t)(a.nslices + sl) * HW : nullptr;

    for (int idx = threadIdx.x; idx < RA; idx += NT) {
        const int li = idx / RW, lj = idx - li * RW;
        const int gi = gi0 + li, gj = gj0 + lj;
        float g = 0.f, p1 = 0.f, p2 = 0.f;
        if (gi >= 0 && gi < H && gj >= 0 && gj < W) {
            const size_t o = (size_t)gi * W + gj;
            const float wv = wn[o];
            g = a.gamma > 0.f ? (a.rho * wv + a.gamma * (um[o] + up[o])) * a.inv_rho2g : wv;
            if (p1in) {
                p1 = p1in[o];
                p2 = p2in[o];
            }
        }
        sg[idx] = g;
        A1[idx] = p1;
        A2[idx] = p2;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunk = warp % C, band = warp / C;
    const int j = chunk * 31 + lane;   // local column, 0 .. RW-1
    const int jl = j > 0 ? j - 1 : 0;  // left neighbour (clamped for column 0, never updated)
    const int gj = gj0 + j;
    const float mc = (gj >= 0 && gj < W - 1) ? 1.f : 0.f;
    const float inv_theta = a.inv_theta, tau = a.tau;

    for (int s = 0; s < T; ++s) {
        const int lo = s + 1, len = RH - 2 * s - 3;  // p^{s+1} rows [s+1, RH-s-2)
        const int r0 = lo + (band * len) / kBands;
        const int r1 = lo + ((band + 1) * len) / kBands;
        const bool upd = lane < 31 && j >= lo && j < RW - s - 2;
        if (r0 < r1) {
            float p1c = A1[r0 * RW + j], p2c = A2[r0 * RW + j];
            float qc = fmaf(-sg[r0 * RW + j], inv_theta,
                            (p1c - A1[(r0 - 1) * RW + j]) + (p2c - A2[r0 * RW + jl]));
            int gi = gi0 + r0;
            for (int i = r0; i < r1; ++i, ++gi) {
                const int o = (i + 1) * RW;
                const float p1n = A1[o + j], p2n = A2[o + j];
                const float qn = fmaf(-sg[o + j], inv_theta, (p1n - p1c) + (p2n - A2[o + jl]));
                const float qr = __shfl_down_sync(0xffffffffu, qc, 1);
                const float mr = (gi >= 0 && gi < H - 1) ? 1.f : 0.f;
                const float gx = (qn - qc) * mr;
                const float gy = (qr - qc) * mc;
                const float inv = rcp_approx(fmaf(tau, sqrt_approx(fmaf(gx, gx, gy * gy)), 1.f));
                if (upd) {
                    B1[i * RW + j] = fmaf(tau, gx, p1c) * inv;
                    B2[i * RW + j] = fmaf(tau, gy, p2c) * inv;
                }
                qc = qn;
                p1c = p1n;
                p2c = p2n;
            }
        }
        __syncthreads();
        float *t1 = A1, *t2 = A2;
        A1 = B1;
        A2 = B2;
        B1 = t1;
        B2 = t2;
    }

    // interior: local rows [T+1, T+1+TH), columns [T+1, T+1+TW)
    const int TH = a.TH, TW = a.TW;
    for (int idx = threadIdx.x; idx < TH * TW; idx += NT) {
        const int ti = idx / TW, tj = idx - ti * TW;
        const int gi = gi0 + T + 1 + ti, gjj = gj0 + T + 1 + tj;
        if (gi >= H || gjj >= W) continue;
        const int l = (T + 1 + ti) * RW + (T + 1 + tj);
        const size_t o = (size_t)gi * W + gjj;
        if (a.write_final) {
            const float divp = (A1[l] - A1[l - RW]) + (A2[l] - A2[l - 1]);
            const float uv = sg[l] - a.theta * divp;
            a.u[(size_t)n * HW + o] = uv;
            if (a.d) a.d[(size_t)n * HW + o] = wn[o] - uv;
        } else {
            a.pout[(size_t)sl * HW + o] = A1[l];
            a.pout[(size_t)(a.nslices + sl) * HW + o] = A2[l];
        }
    }
}

inline size_t smem_bytes(int C, int RH) { return 5ull * (31 * C + 1) * RH * sizeof(float); }

constexpr size_t kSmemLimit = 227 * 1024;  // per CTA
constexpr size_t kSmemPerSm = 228 * 1024;

struct Shape {
    int C, TH, TW, RH;
};

// Per-device state: SM count and the kernels' shared-memory opt-in.
struct DeviceInfo {
    int sms = 0;
    bool ready = false;
};
std::mutex g_mu;
std::vector<DeviceInfo> g_dev;

cslsm_status device_info(int &sms)
{
    int dev = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_dev.size() <= dev) g_dev.resize(dev + 1);
    DeviceInfo &di = g_dev[dev];
    if (!di.ready) {
        CSLSM_CUDA(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev));
        const int lim = (int)kSmemLimit;
        CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel<1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel<2>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel<3>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel<4>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
        di.ready = true;
    }
    sms = di.sms;
    return CSLSM_OK;
}

// Tile shape with the least estimated time: waves of CTAs over the SMs times
// the pixel-steps one CTA performs on its shrinking region.
Shape pick_shape(int H, int W, int T, int nslices, int sms)
{
    Shape best{0, 0, 0, 0};
    double best_cost = 1e300;
    for (int C = 1; C <= 4; ++C) {
        const int RW = 31 * C + 1;
        const int TW = RW - 2 * T - 2;
        if (TW < 8) continue;
        const int tiles_w = (W + TW - 1) / TW;
        const int threads = C * kBands * 32;
        for (int TH = 8; TH <= 512; TH += 2) {
            const int RH = TH + 2 * T + 2;
            const size_t sm = smem_bytes(C, RH);
            if (sm > kSmemLimit) break;
            const int per_sm = (int)std::min<size_t>(kSmemPerSm / (sm + 1024), 2048 / threads);
            if (per_sm < 1) break;
            const long long ctas = (long long)tiles_w * ((H + TH - 1) / TH) * nslices;
            const double waves = std::ceil((double)ctas / ((double)sms * per_sm));
            double work = 2.0 * RW * RH;  // pixel-steps of one CTA plus its load
            for (int s = 0; s < T; ++s) work += (double)(RW - 2 * s - 3) * (RH - 2 * s - 3);
            const double cost = waves * work * per_sm;
            if (cost < best_cost) {
                best_cost = cost;
                best = Shape{C, TH, TW, RH};
            }
            if (TH >= H) break;
        }
    }
    return best;
}

cslsm_status launch_tile(const TvLaunch &a, const Shape &sh, cudaStream_t st)
{
    if (sh.C < 1) {
        set_error("no TV tile shape fits shared memory for %d steps", a.T);
        return CSLSM_ERR_UNSUPPORTED;
    }
    const dim3 grid((a.W + sh.TW - 1) / sh.TW, (a.H + sh.TH - 1) / sh.TH, a.nslices);
    const size_t sm = smem_bytes(sh.C, sh.RH);
    LaunchScope ls(K_TV_TILE, st);
    switch (sh.C) {
    case 1: tv_tile_kernel<1><<<grid, 1 * kBands * 32, sm, st>>>(a); break;
    case 2: tv_tile_kernel<2><<<grid, 2 * kBands * 32, sm, st>>>(a); break;
    case 3: tv_tile_kernel<3><<<grid, 3 * kBands * 32, sm, st>>>(a); break;
    default: tv_tile_kernel<4><<<grid, 4 * kBands * 32, sm, st>>>(a); break;
    }
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

}  // namespace

int tv_max_steps_per_launch() { return kMaxSteps; }

cslsm_status tv_prox_slices(const TvSlices &s, float *pbuf, cudaStream_t st)
{
    int sms = 0;
    cslsm_status e = device_info(sms);
    if (e) return e;
    TvLaunch a{};
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
        const Shape sh = pick_shape(s.H, s.W, T, s.nslices, sms);
        a.T = T;
        a.TH = sh.TH;
        a.TW = sh.TW;
        a.RH = sh.RH;
        a.write_final = 1;
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
        const Shape sh = pick_shape(s.H, s.W, steps, s.nslices, sms);
        a.T = steps;
        a.TH = sh.TH;
        a.TW = sh.TW;
        a.RH = sh.RH;
        a.pin = pin;
        a.write_final = (c == nch - 1);
        a.pout = a.write_final ? nullptr : pbuf + (c % 2) * half;
        e = launch_tile(a, sh, st);
        if (e) return e;
        pin = a.pout;
        done += steps;
    }
    return CSLSM_OK;
}

}  // namespace cslsm
