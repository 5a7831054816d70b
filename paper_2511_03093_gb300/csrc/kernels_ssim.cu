// 3-D SSIM of Sec. IV (evaluation metrics): the local ssim of Wang et al. with
// means, variances and the covariance over an 11 x 11 x 11 Gaussian window
// (standard deviation 1.5) centred on every voxel, c1 = 0.01^2, c2 = 0.03^2
// (L = 1), averaged over the volume.  The window is clipped to the volume and
// renormalised (the paper does not say how it meets the faces).  Gaussian
// weights and box clipping are separable, so every window mean is three 1-D
// normalised passes:
//
//   ssim_xy_kernel  one slice tile in shared memory: the five fields x, y,
//                   x^2, y^2, x y filtered along x then y -> five FP32 planes;
//   ssim_z_kernel   one thread per (row, column): the z pass of the five
//                   fields, the local ssim, FP64 block partial sums;
//   finish          the partials summed in a fixed order, / n.
//
// Bytes per voxel: read x, y (8), write and read back the five planes (40):
// 48 B; the z pass re-reads each plane from L1/L2 for its 11 taps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace cslsm {
namespace {

constexpr int kR = 5;                      // window radius
constexpr int kTX = 64, kTY = 32;          // output tile of the xy pass
constexpr int kRX = kTX + 2 * kR, kRY = kTY + 2 * kR;
constexpr int kXYThreads = 256;
constexpr int kZThreads = 256;

__constant__ float c_g[2 * kR + 1];  // exp(-k^2 / (2 * 1.5^2)), k = -5..5

// Sum of the window weights whose taps fall inside [0, n) around position c.
__device__ __forceinline__ float wsum(int c, int n)
{
    float s = 0.f;
#pragma unroll
    for (int k = -kR; k <= kR; ++k) s += (c + k >= 0 && c + k < n) ? c_g[k + kR] : 0.f;
    return s;
}

__global__ void __launch_bounds__(kXYThreads) ssim_xy_kernel(const float *__restrict__ x,
                                                            const float *__restrict__ y,
                                                            float *__restrict__ fields, int H,
                                                            int W, size_t N)
{
    extern __shared__ float smem[];  // sx[kRY][kRX], sy[kRY][kRX], hf[5][kRY][kTX]
    float(*sx)[kRX] = reinterpret_cast<float(*)[kRX]>(smem);
    float(*sy)[kRX] = reinterpret_cast<float(*)[kRX]>(smem + kRY * kRX);
    float(*hf)[kRY][kTX] = reinterpret_cast<float(*)[kRY][kTX]>(smem + 2 * kRY * kRX);
    const int z = blockIdx.z;
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;
    const size_t zo = (size_t)z * H * W;
    for (int idx = threadIdx.x; idx < kRY * kRX; idx += kXYThreads) {
        const int li = idx / kRX, lj = idx - li * kRX;
        const int gi = i0 - kR + li, gj = j0 - kR + lj;
        const bool in = gi >= 0 && gi < H && gj >= 0 && gj < W;
        const size_t o = zo + (size_t)gi * W + gj;
        sx[li][lj] = in ? x[o] : 0.f;
        sy[li][lj] = in ? y[o] : 0.f;
    }
    __syncthreads();
    // along x (out-of-volume taps hold zeros), normalised by the clipped weight sum
    for (int idx = threadIdx.x; idx < kRY * kTX; idx += kXYThreads) {
        const int li = idx / kTX, tj = idx - li * kTX;
        float a[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k <= 2 * kR; ++k) {
            const float g = c_g[k], vx = sx[li][tj + k], vy = sy[li][tj + k];
            a[0] += g * vx;
            a[1] += g * vy;
            a[2] += g * (vx * vx);
            a[3] += g * (vy * vy);
            a[4] += g * (vx * vy);
        }
        const float inv = 1.f / wsum(j0 + tj, W);
#pragma unroll
        for (int f = 0; f < 5; ++f) hf[f][li][tj] = a[f] * inv;
    }
    __syncthreads();
    // along y
    for (int idx = threadIdx.x; idx < kTY * kTX; idx += kXYThreads) {
        const int ti = idx / kTX, tj = idx - ti * kTX;
        const int gi = i0 + ti, gj = j0 + tj;
        if (gi >= H || gj >= W) continue;
        const float inv = 1.f / wsum(gi, H);
        const size_t o = zo + (size_t)gi * W + gj;
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kR; ++k) {
                const int li = ti + k, gr = gi - kR + k;
                a += (gr >= 0 && gr < H) ? c_g[k] * hf[f][li][tj] : 0.f;
            }
            fields[f * N + o] = a * inv;
        }
    }
}

__global__ void __launch_bounds__(kZThreads) ssim_z_kernel(const float *__restrict__ fields,
                                                          int Z, int HW, size_t N,
                                                          double *__restrict__ partials)
{
    const float c1 = 0.01f * 0.01f, c2 = 0.03f * 0.03f;
    double acc = 0.0;
    for (int p = blockIdx.x * kZThreads + threadIdx.x; p < HW; p += gridDim.x * kZThreads) {
        for (int z = 0; z < Z; ++z) {
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            const int k0 = max(-kR, -z), k1 = min(kR, Z - 1 - z);
            float ws = 0.f;
            for (int k = k0; k <= k1; ++k) {
                const float g = c_g[k + kR];
                const size_t o = (size_t)(z + k) * HW + p;
                ws += g;
#pragma unroll
                for (int f = 0; f < 5; ++f) m[f] += g * __ldg(fields + f * N + o);
            }
            const float inv = 1.f / ws;
            const float mx = m[0] * inv, my = m[1] * inv;
            const float vx = m[2] * inv - mx * mx, vy = m[3] * inv - my * my;
            const float cxy = m[4] * inv - mx * my;
            const float s = (2.f * mx * my + c1) * (2.f * cxy + c2) /
                            ((mx * mx + my * my + c1) * (vx + vy + c2));
            acc += (double)s;
        }
    }
    __shared__ double sa[kZThreads];
    sa[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kZThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sa[threadIdx.x] += sa[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sa[0];
}

__global__ void ssim_finish_kernel(const double *__restrict__ partials, int nblocks, size_t n,
                                   double *__restrict__ out)
{
    __shared__ double sa[kZThreads];
    double a = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += kZThreads) a += partials[k];
    sa[threadIdx.x] = a;
    __syncthreads();
    for (int s = kZThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sa[threadIdx.x] += sa[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sa[0] / (double)n;
}

bool g_weights_set[64] = {};

cslsm_status set_weights(int dev)
{
    if (dev >= 0 && dev < 64 && g_weights_set[dev]) return CSLSM_OK;
    float g[2 * kR + 1];
    for (int k = -kR; k <= kR; ++k) g[k + kR] = (float)std::exp(-(double)(k * k) / 4.5);
    CSLSM_CUDA(cudaMemcpyToSymbol(c_g, g, sizeof(g)));
    if (dev >= 0 && dev < 64) g_weights_set[dev] = true;
    return CSLSM_OK;
}

}  // namespace

size_t ssim3d_workspace_bytes(int Z, int H, int W, int *nblocks)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long HW = (long long)H * W;
    const int nb = (int)std::max(1ll, std::min<long long>((HW + kZThreads - 1) / kZThreads,
                                                           8ll * std::max(sms, 1)));
    *nblocks = nb;
    return 5 * sizeof(float) * (size_t)Z * H * W + sizeof(double) * (size_t)nb;
}

cslsm_status launch_ssim3d(const float *x, const float *ref, int Z, int H, int W, void *ws,
                           int nblocks, double *out, cudaStream_t s)
{
    int dev = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    cslsm_status st = set_weights(dev);
    if (st) return st;
    const size_t N = (size_t)Z * H * W;
    float *fields = (float *)ws;
    double *partials = (double *)(fields + 5 * N);
    {
        LaunchScope ls(K_SSIM, s);
        const dim3 grid((W + kTX - 1) / kTX, (H + kTY - 1) / kTY, Z);
        constexpr size_t smem = sizeof(float) * (2 * kRY * kRX + 5 * kRY * kTX);
        CSLSM_CUDA(cudaFuncSetAttribute(ssim_xy_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ssim_xy_kernel<<<grid, kXYThreads, smem, s>>>(x, ref, fields, H, W, N);
        CSLSM_LAUNCHED();
    }
    {
        LaunchScope ls(K_SSIM, s);
        ssim_z_kernel<<<nblocks, kZThreads, 0, s>>>(fields, Z, H * W, N, partials);
        CSLSM_LAUNCHED();
    }
    {
        LaunchScope ls(K_REDUCE, s);
        ssim_finish_kernel<<<1, kZThreads, 0, s>>>(partials, nblocks, N, out);
        CSLSM_LAUNCHED();
    }
    return CSLSM_OK;
}

}  // namespace cslsm
