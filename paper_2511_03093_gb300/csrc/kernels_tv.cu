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
// GB300 design: temporal blocking in shared memory.  One CTA owns a 32 x 32
// output tile of one slice and loads g on the tile plus a halo of T+1 pixels
// (the dependence cone of T Chambolle steps).  All T steps then run out of
// shared memory on a region that shrinks by one pixel per side per step, so
// the dual field p never touches HBM and one launch performs the whole prox
// of every slice it covers.  HBM traffic per prox is one read of w (plus the
// two neighbouring u slices when gamma > 0) and one write of u and d; the
// halo re-reads of neighbouring tiles are served by L2.  Pixels outside the
// image hold p = 0, which reproduces the Neumann boundary exactly.
//
// Step counts above kMaxSteps are split into chunks of at most kMaxSteps
// steps that hand p over through a double-buffered global array.
#include <cuda_runtime.h>

#include <atomic>

#include "internal.cuh"

namespace cslsm {
namespace {

constexpr int kTile = 32;
constexpr int kTvThreads = 256;
constexpr int kMaxSteps = 40;

struct TvLaunch {
    const float *w;
    float *u;
    float *d;
    const float *pin;  // [2][nslices][H][W] dual field entering this launch, or null (p = 0)
    float *pout;       // [2][nslices][H][W] dual field leaving it (write_final == 0)
    int H, W, Z, n0, nslices;
    int T;
    float rho, gamma, inv_rho2g;
    float theta, inv_theta, tau;
    int write_final;
};

__host__ __device__ constexpr int region_edge(int T) { return kTile + 2 * T + 2; }
inline size_t smem_bytes(int T)
{
    return 4ull * region_edge(T) * region_edge(T) * sizeof(float);
}

__global__ void __launch_bounds__(kTvThreads, 2) tv_tile_kernel(const TvLaunch a)
{
    extern __shared__ float smem[];
    const int T = a.T;
    const int RE = region_edge(T);
    const int RA = RE * RE;
    float *sg = smem;      // g
    float *s1 = sg + RA;   // p, component along rows (i)
    float *s2 = s1 + RA;   // p, component along columns (j)
    float *sq = s2 + RA;   // q = div p - g / theta
    const int sl = blockIdx.z;
    const int n = a.n0 + sl;
    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    const int gi0 = blockIdx.y * kTile - (T + 1);
    const int gj0 = blockIdx.x * kTile - (T + 1);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = kTvThreads / 32;

    const float *wn = a.w + (size_t)n * HW;
    const float *um = a.u + (size_t)((n + a.Z - 1) % a.Z) * HW;
    const float *up = a.u + (size_t)((n + 1) % a.Z) * HW;
    const float *p1in = a.pin ? a.pin + (size_t)sl * HW : nullptr;
    const float *p2in = a.pin ? a.pin + (size_t)(a.nslices + sl) * HW : nullptr;

    for (int li = wid; li < RE; li += NW) {
        const int gi = gi0 + li;
        for (int lj = lane; lj < RE; lj += 32) {
            const int gj = gj0 + lj;
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
            const int idx = li * RE + lj;
            sg[idx] = g;
            s1[idx] = p1;
            s2[idx] = p2;
        }
    }
    __syncthreads();

    for (int s = 0; s < T; ++s) {
        // q^s on local rows/cols [s+1, RE-s-1)
        const int lo = s + 1, hq = RE - s - 1, hp = RE - s - 2;
        for (int li = lo + wid; li < hq; li += NW)
            for (int lj = lo + lane; lj < hq; lj += 32) {
                const int idx = li * RE + lj;
                sq[idx] = ((s1[idx] - s1[idx - RE]) + (s2[idx] - s2[idx - 1])) -
                          sg[idx] * a.inv_theta;
            }
        __syncthreads();
        // p^{s+1} on [s+1, RE-s-2)
        for (int li = lo + wid; li < hp; li += NW) {
            const int gi = gi0 + li;
            if (gi < 0 || gi >= H) continue;
            for (int lj = lo + lane; lj < hp; lj += 32) {
                const int gj = gj0 + lj;
                if (gj < 0 || gj >= W) continue;
                const int idx = li * RE + lj;
                const float qc = sq[idx];
                const float gx = gi < H - 1 ? sq[idx + RE] - qc : 0.f;
                const float gy = gj < W - 1 ? sq[idx + 1] - qc : 0.f;
                const float den = 1.f + a.tau * sqrtf(gx * gx + gy * gy);
                s1[idx] = (s1[idx] + a.tau * gx) / den;
                s2[idx] = (s2[idx] + a.tau * gy) / den;
            }
        }
        __syncthreads();
    }

    // interior: local [T+1, T+1+kTile)
    for (int li = T + 1 + wid; li < T + 1 + kTile; li += NW) {
        const int gi = gi0 + li;
        if (gi >= H) break;
        const int lj = T + 1 + lane;
        const int gj = gj0 + lj;
        if (gj >= W) continue;
        const int idx = li * RE + lj;
        const size_t o = (size_t)gi * W + gj;
        if (a.write_final) {
            const float divp = (s1[idx] - s1[idx - RE]) + (s2[idx] - s2[idx - 1]);
            const float uv = sg[idx] - a.theta * divp;
            a.u[(size_t)n * HW + o] = uv;
            if (a.d) a.d[(size_t)n * HW + o] = wn[o] - uv;
        } else {
            a.pout[(size_t)sl * HW + o] = s1[idx];
            a.pout[(size_t)(a.nslices + sl) * HW + o] = s2[idx];
        }
    }
}

// cudaFuncSetAttribute is per device: remember which devices are set up.
std::atomic<unsigned long long> g_attr_devices{0};

}  // namespace

int tv_max_steps_per_launch() { return kMaxSteps; }

cslsm_status tv_prox_slices(const TvSlices &s, float *pbuf, cudaStream_t st)
{
    int dev = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    const unsigned long long bitm = 1ull << (dev & 63);
    if (!(g_attr_devices.load() & bitm)) {
        CSLSM_CUDA(cudaFuncSetAttribute(tv_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem_bytes(kMaxSteps)));
        g_attr_devices.fetch_or(bitm);
    }
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
    const dim3 grid((s.W + kTile - 1) / kTile, (s.H + kTile - 1) / kTile, s.nslices);
    if (T <= kMaxSteps) {
        a.T = T;
        a.write_final = 1;
        {
            LaunchScope ls(K_TV_TILE, st);
            tv_tile_kernel<<<grid, kTvThreads, smem_bytes(T), st>>>(a);
        }
        CSLSM_LAUNCHED();
        return CSLSM_OK;
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
        {
            LaunchScope ls(K_TV_TILE, st);
            tv_tile_kernel<<<grid, kTvThreads, smem_bytes(steps), st>>>(a);
        }
        CSLSM_LAUNCHED();
        pin = a.pout;
        done += steps;
    }
    return CSLSM_OK;
}

}  // namespace cslsm
