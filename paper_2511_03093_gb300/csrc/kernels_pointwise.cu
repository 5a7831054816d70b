// Pixel-local kernels of the PnP-ADMM iteration: DMD pattern packing, the
// forward / adjoint operators, the Woodbury x-update and the fused Tikhonov
// iteration, plus deterministic reductions.
//
// Layout: volumes [Z][H][W] float32, one thread per pixel column (h, w); the
// thread walks the R planes of a shot, so every global access of a warp is a
// contiguous 128-byte row segment of one plane.  The DMD patterns of a shot
// are one 32-bit word per pixel (bit r = plane r), so diag(Phi Phi^T) at the
// pixel is __popc(word) (Sec. III-B: Phi Phi^T is diagonal).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"
#include "storage.cuh"

namespace cslsm {
namespace {

constexpr int kThreads = 256;
constexpr int kRedBlocks = 1024;

__device__ __forceinline__ bool bit(uint32_t word, int r) { return (word >> r) & 1u; }

__global__ void __launch_bounds__(kThreads) pack_masks_kernel(const uint8_t *__restrict__ masks,
                                                              uint32_t *__restrict__ words,
                                                              int HW, int R)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const int j = blockIdx.y;
    if (p >= HW) return;
    uint32_t word = 0;
    const uint8_t *m = masks + (size_t)j * R * HW + p;
    for (int r = 0; r < R; ++r)
        word |= (m[(size_t)r * HW] != 0 ? 1u : 0u) << r;
    words[(size_t)j * HW + p] = word;
}

// b_j = sum_r phi_r v_{jR+r}  (Sec. III-A)
__global__ void __launch_bounds__(kThreads) forward_kernel(const float *__restrict__ v,
                                                           float *__restrict__ b,
                                                           const uint32_t *__restrict__ words,
                                                           int wstride, int HW, int R)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const int j = blockIdx.y;
    if (p >= HW) return;
    const uint32_t word = words[(size_t)j * wstride + p];
    const float *vj = v + (size_t)j * R * HW + p;
    float s = 0.f;
    for (int r = 0; r < R; ++r)
        if (bit(word, r)) s += __ldg(vj + (size_t)r * HW);
    b[(size_t)j * HW + p] = s;
}

// v_{jR+r} = phi_r b_j
__global__ void __launch_bounds__(kThreads) adjoint_kernel(const float *__restrict__ b,
                                                           float *__restrict__ v,
                                                           const uint32_t *__restrict__ words,
                                                           int wstride, int HW, int R)
{
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const int j = blockIdx.y;
    if (p >= HW) return;
    const uint32_t word = words[(size_t)j * wstride + p];
    const float bj = b[(size_t)j * HW + p];
    float *vj = v + (size_t)j * R * HW + p;
    for (int r = 0; r < R; ++r)
        vj[(size_t)r * HW] = bit(word, r) ? bj : 0.f;
}

// Block-wide sum of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double &a, double &c)
{
    __shared__ double sa[kThreads / 32], sc[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sa[wid] = a; sc[wid] = c; }
    __syncthreads();
    if (wid == 0) {
        a = lane < kThreads / 32 ? sa[lane] : 0.0;
        c = lane < kThreads / 32 ? sc[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            c += __shfl_down_sync(0xffffffffu, c, o);
        }
    }
}

// Woodbury x-update (Eq. v-update): for shot j at pixel p,
//   g_r = u_r - d_r,  e = (b_j - sum_r phi_r g_r) / (rho + popc),
//   v_r = g_r + phi_r e,  w_r = v_r + d_r.
template <int RMAX, typename S>
__global__ void __launch_bounds__(kThreads, RMAX >= 32 ? 2 : 4)
xupdate_w_kernel(const S *__restrict__ u, const S *__restrict__ d,
                 const float *__restrict__ b, const uint32_t *__restrict__ words, int wstride,
                 int HW, int R, float rho, S *__restrict__ w, float *__restrict__ v_out,
                 float *__restrict__ vprev, double *__restrict__ partials,
                 const int *__restrict__ stop)
{
    if (stop && *stop) return;  // a tolerance-stopped solve: nothing more to do
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const int j = blockIdx.y;
    double sdv = 0.0, sv = 0.0;
    if (p < HW) {
        const uint32_t word = words[j * wstride + p];
        const int base = j * R * HW + p;
        float g[RMAX], dr[RMAX];
        float s = 0.f;
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            if (r < R) {
                dr[r] = ld<S>(d + base + r * HW);
                g[r] = ld<S>(u + base + r * HW) - dr[r];
                if (bit(word, r)) s += g[r];
            }
        }
        const float e = (__ldg(b + j * HW + p) - s) / (rho + (float)__popc(word));
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
            if (r < R) {
                const int o = base + r * HW;
                const float v = bit(word, r) ? g[r] + e : g[r];
                st<S>(w + o, keep<S>(v + dr[r], (size_t)o, kKeyW));
                if (v_out) v_out[o] = v;
                if (vprev) {
                    const double vp = vprev[o];
                    sdv += ((double)v - vp) * ((double)v - vp);
                    sv += vp * vp;
                    vprev[o] = v;
                }
            }
        }
    }
    if (partials) {
        block_sum2(sdv, sv);
        if (threadIdx.x == 0) {
            const int blk = blockIdx.y * gridDim.x + blockIdx.x;
            partials[2 * blk] = sdv;
            partials[2 * blk + 1] = sv;
        }
    }
}

// One fused ADMM iteration with the Tikhonov prior (psi = ||u||^2):
// x-update as above (with w = v + d = u + phi_r e, one rounding), then along z
// in order n = 0..Z-1 (Gauss-Seidel, cyclic, always the newest neighbour values)
//   u_n = (rho w_n + gam (u_{n-1} + u_{n+1})) / (2 lam + rho + 2 gam),
// and d_n = w_n - u_n  (= d + v - u).  One thread owns a pixel column for all
// shots, so the in-place sweep needs no synchronisation.
template <int RMAX, typename S>
__global__ void __launch_bounds__(kThreads, 2)
tikhonov_iter_kernel(S *__restrict__ u, S *__restrict__ d, const float *__restrict__ b,
                     const uint32_t *__restrict__ words, int wstride, int HW, int R, int N,
                     float rho, float lam, float gam, float *__restrict__ v_out,
                     float *__restrict__ vprev, double *__restrict__ partials,
                     const int *__restrict__ stop)
{
    if (stop && *stop) return;
    const int p = blockIdx.x * kThreads + threadIdx.x;
    const int Z = N * R;
    // one reciprocal per thread: the per-voxel divisions cost more issue slots
    // than the kernel's memory traffic leaves (the u-update multiplies by it)
    const float inv_den = 1.f / (2.f * lam + rho + 2.f * gam);
    double sdv = 0.0, sv = 0.0;
    if (p < HW) {
        float prev = gam > 0.f ? ld<S>(u + (Z - 1) * HW + p) : 0.f;  // u_{Z-1}, not yet updated
        float first_new = 0.f;
        for (int j = 0; j < N; ++j) {
            const uint32_t word = words[j * wstride + p];
            const int base = j * R * HW + p;
            float ur[RMAX], dr[RMAX];
            float s = 0.f;
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (r < R) {
                    ur[r] = ld<S>(u + base + r * HW);
                    dr[r] = ld<S>(d + base + r * HW);
                    if (bit(word, r)) s += ur[r] - dr[r];
                }
            }
            const float e = (b[j * HW + p] - s) / (rho + (float)__popc(word));
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (r < R) {
                    const int n = j * R + r;
                    const int o = base + r * HW;
                    const float g = ur[r] - dr[r];
                    const float v = bit(word, r) ? g + e : g;
                    const float w = bit(word, r) ? ur[r] + e : ur[r];  // v + d
                    float un;
                    if (gam > 0.f) {
                        float next;
                        if (n == Z - 1) next = first_new;
                        else if (r + 1 < R) next = ur[r + 1 < RMAX ? r + 1 : r];
                        else next = ld<S>(u + o + HW);  // next shot's first plane, still old
                        un = keep<S>((rho * w + gam * (prev + next)) * inv_den, (size_t)o, kKeyU);
                        prev = un;
                        if (n == 0) first_new = un;
                    } else {
                        un = keep<S>(rho * w * inv_den, (size_t)o, kKeyU);
                    }
                    st<S>(u + o, un);
                    st<S>(d + o, keep<S>(w - un, (size_t)o, kKeyD));
                    if (v_out) v_out[o] = v;
                    if (vprev) {
                        const double vp = vprev[o];
                        sdv += ((double)v - vp) * ((double)v - vp);
                        sv += vp * vp;
                        vprev[o] = v;
                    }
                }
            }
        }
    }
    if (partials) {
        block_sum2(sdv, sv);
        if (threadIdx.x == 0) partials[2 * blockIdx.x] = sdv, partials[2 * blockIdx.x + 1] = sv;
    }
}

// The same fused Tikhonov iteration, two adjacent pixel columns per thread
// (8-byte accesses for FP32).  The first pass over a shot's planes reads u and
// d once from HBM, accumulates sum_r phi_r (u_r - d_r) and parks u_r in shared
// memory; the second pass takes u_r (and the next plane's u for the z term)
// from shared memory, so HBM sees exactly one read of u, d and one write of
// u, d per voxel.  The arithmetic per pixel is that of tikhonov_iter_kernel.
template <typename S>
__global__ void __launch_bounds__(kThreads)
tikhonov_iter_v2_kernel(S *__restrict__ u, S *__restrict__ d, const float *__restrict__ b,
                        const uint32_t *__restrict__ words, int wstride, int HW, int R, int N,
                        float rho, float lam, float gam, float *__restrict__ v_out)
{
    extern __shared__ float2 su[];  // [R][kThreads]
    const int t = threadIdx.x;
    const int p = 2 * (blockIdx.x * kThreads + t);
    if (p >= HW) return;
    const int Z = N * R;
    // one reciprocal per thread: the per-voxel divisions cost more issue slots
    // than the kernel's memory traffic leaves (the u-update multiplies by it)
    const float inv_den = 1.f / (2.f * lam + rho + 2.f * gam);
    float2 prev = gam > 0.f ? ld2<S>(u + (size_t)(Z - 1) * HW + p) : make_float2(0.f, 0.f);
    float2 first_new = make_float2(0.f, 0.f);
    for (int j = 0; j < N; ++j) {
        const uint2 wd = *reinterpret_cast<const uint2 *>(words + (size_t)j * wstride + p);
        const float2 bj = *reinterpret_cast<const float2 *>(b + (size_t)j * HW + p);
        const size_t base = (size_t)j * R * HW + p;
        float2 s = make_float2(0.f, 0.f);
        if constexpr (sizeof(S) == 4) {
            // FP32: the loads of 16 planes issued together, then summed in
            // plane order (more bytes in flight per thread; measured 0.82 ->
            // 0.88 of HBM at 1024 x 1024 x 32; for 16-bit storage it was slower)
            constexpr int C = 16;
            for (int r0 = 0; r0 < R; r0 += C) {
                float2 uu[C], dd[C];
#pragma unroll
                for (int q = 0; q < C; ++q)
                    if (r0 + q < R) {
                        uu[q] = ld2<S>(u + base + (size_t)(r0 + q) * HW);
                        dd[q] = ld2<S>(d + base + (size_t)(r0 + q) * HW);
                    }
#pragma unroll
                for (int q = 0; q < C; ++q)
                    if (r0 + q < R) {
                        const int r = r0 + q;
                        su[r * kThreads + t] = uu[q];
                        if ((wd.x >> r) & 1u) s.x += uu[q].x - dd[q].x;
                        if ((wd.y >> r) & 1u) s.y += uu[q].y - dd[q].y;
                    }
            }
        } else {
#pragma unroll 8
            for (int r = 0; r < R; ++r) {
                const float2 uu = ld2<S>(u + base + (size_t)r * HW);
                const float2 dd = ld2<S>(d + base + (size_t)r * HW);
                su[r * kThreads + t] = uu;
                if ((wd.x >> r) & 1u) s.x += uu.x - dd.x;
                if ((wd.y >> r) & 1u) s.y += uu.y - dd.y;
            }
        }
        const float ex = (bj.x - s.x) / (rho + (float)__popc(wd.x));
        const float ey = (bj.y - s.y) / (rho + (float)__popc(wd.y));
#pragma unroll 4
        for (int r = 0; r < R; ++r) {
            const int n = j * R + r;
            const size_t o = base + (size_t)r * HW;
            const float2 uu = su[r * kThreads + t];
            const bool bx = (wd.x >> r) & 1u, by = (wd.y >> r) & 1u;
            const float2 w = make_float2(bx ? uu.x + ex : uu.x, by ? uu.y + ey : uu.y);
            float2 un;
            if (gam > 0.f) {
                float2 nx;
                if (n == Z - 1) nx = first_new;
                else if (r + 1 < R) nx = su[(r + 1) * kThreads + t];
                else nx = ld2<S>(u + o + HW);  // next shot's first plane, still old
                un.x = keep<S>((rho * w.x + gam * (prev.x + nx.x)) * inv_den, o, kKeyU);
                un.y = keep<S>((rho * w.y + gam * (prev.y + nx.y)) * inv_den, o + 1, kKeyU);
                prev = un;
                if (n == 0) first_new = un;
            } else {
                un = make_float2(keep<S>(rho * w.x * inv_den, o, kKeyU),
                                 keep<S>(rho * w.y * inv_den, o + 1, kKeyU));
            }
            if (v_out) {  // v = (u - d) + phi e, with d before this iteration's store
                const float2 dd = ld2<S>(d + o);
                const float gx = uu.x - dd.x, gy = uu.y - dd.y;
                *reinterpret_cast<float2 *>(v_out + o) = make_float2(bx ? gx + ex : gx,
                                                                     by ? gy + ey : gy);
            }
            st2<S>(u + o, un);
            st2<S>(d + o, make_float2(keep<S>(w.x - un.x, o, kKeyD), keep<S>(w.y - un.y, o + 1, kKeyD)));
        }
    }
}

__global__ void __launch_bounds__(kThreads) tikhonov_prox_kernel(const float *__restrict__ in,
                                                                 float *__restrict__ out,
                                                                 long long n, float rho,
                                                                 float lam)
{
    const float den = 2.f * lam + rho;
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kThreads)
        out[i] = rho * in[i] / den;
}

// PSNR partials: per block max(ref) and sum (x - ref)^2 over a grid-stride range.
__global__ void __launch_bounds__(kThreads) psnr_partials_kernel(const float *__restrict__ x,
                                                                 const float *__restrict__ ref,
                                                                 size_t n,
                                                                 double *__restrict__ partials)
{
    double e = 0.0, mx = -INFINITY;
    for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
         i += (size_t)gridDim.x * kThreads) {
        const float r = ref[i];
        const double t = (double)x[i] - (double)r;
        e += t * t;
        mx = fmax(mx, (double)r);
    }
    __shared__ double se[kThreads / 32], sm[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { se[wid] = e; sm[wid] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = -INFINITY;
        for (int k = 0; k < kThreads / 32; ++k) { a += se[k]; m = fmax(m, sm[k]); }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = m;
    }
}

// Sums `nblocks` pairs in a fixed order (one block): out = {sum a, sum c} or,
// for PSNR, {sum e, max m} -> 10 log10(n V^2 / e).
// The stopping rule of Sec. IV-B on the device: rel = ||v^{k+1} - v^k|| / ||v^k||
// from the reduced sums red = {sum (v^{k+1} - v^k)^2, sum (v^k)^2}; below tol the
// solve stops (every later kernel of the solve returns at once).
__global__ void tol_check_kernel(const double *__restrict__ red, float tol, int k,
                                 TolState *__restrict__ state)
{
    if (threadIdx.x != 0 || state->stop) return;
    const double rel = red[1] > 0.0 ? sqrt(red[0] / red[1]) : INFINITY;
    state->rel = rel;
    if (rel < (double)tol) {
        state->stop = 1;
        state->iters_done = k + 1;
    }
}

__global__ void __launch_bounds__(kThreads) copy_if_stopped_kernel(
    const TolState *__restrict__ state, const float *__restrict__ src, float *__restrict__ dst,
    size_t n)
{
    if (!state->stop) return;
    for (size_t i = blockIdx.x * (size_t)kThreads + threadIdx.x; i < n;
         i += (size_t)gridDim.x * kThreads)
        dst[i] = src[i];
}

template <bool kPsnr>
__global__ void __launch_bounds__(kThreads) finish_pairs_kernel(const double *__restrict__ partials,
                                                                int nblocks, size_t n,
                                                                double *__restrict__ out)
{
    double a = 0.0, c = kPsnr ? -INFINITY : 0.0;
    for (int k = threadIdx.x; k < nblocks; k += kThreads) {
        a += partials[2 * k];
        c = kPsnr ? fmax(c, partials[2 * k + 1]) : c + partials[2 * k + 1];
    }
    __shared__ double sa[kThreads], sc[kThreads];
    sa[threadIdx.x] = a;
    sc[threadIdx.x] = c;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sc[threadIdx.x] = kPsnr ? fmax(sc[threadIdx.x], sc[threadIdx.x + s])
                                    : sc[threadIdx.x] + sc[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (kPsnr) {
            out[0] = 10.0 * log10((double)n * sc[0] * sc[0] / sa[0]);
        } else {
            out[0] = sa[0];
            out[1] = sc[0];
        }
    }
}

inline dim3 pixel_grid(int HW, int ny) { return dim3((HW + kThreads - 1) / kThreads, ny); }

}  // namespace

int reduction_blocks() { return kRedBlocks; }

cslsm_status launch_pack_masks(const uint8_t *masks, uint32_t *words, int HW, int R, int nsets,
                               cudaStream_t s)
{
    LaunchScope ls(K_PACK, s);
    pack_masks_kernel<<<pixel_grid(HW, nsets), kThreads, 0, s>>>(masks, words, HW, R);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_forward(const Geom &g, Masks m, const float *v, float *b, cudaStream_t s)
{
    LaunchScope ls(K_FORWARD, s);
    forward_kernel<<<pixel_grid(g.HW(), g.N), kThreads, 0, s>>>(v, b, m.words, m.wstride, g.HW(),
                                                                g.R);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_adjoint(const Geom &g, Masks m, const float *b, float *v, cudaStream_t s)
{
    LaunchScope ls(K_ADJOINT, s);
    adjoint_kernel<<<pixel_grid(g.HW(), g.N), kThreads, 0, s>>>(b, v, m.words, m.wstride, g.HW(),
                                                                g.R);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

template <typename S>
cslsm_status xupdate_typed(const Geom &g, Masks m, const void *u_, const void *d_, const float *b,
                           float rho, void *w_, float *v_out, float *vprev, double *partials,
                           cudaStream_t s, const int *stop)
{
    const S *u = (const S *)u_, *d = (const S *)d_;
    S *w = (S *)w_;
    const dim3 grid = pixel_grid(g.HW(), g.N);
#define XU(RM)                                                                          \
    xupdate_w_kernel<RM, S><<<grid, kThreads, 0, s>>>(u, d, b, m.words, m.wstride, g.HW(), \
                                                      g.R, rho, w, v_out, vprev, partials, stop)
    LaunchScope ls(K_XUPDATE, s);
    if (g.R <= 4) XU(4);
    else if (g.R <= 8) XU(8);
    else if (g.R <= 16) XU(16);
    else XU(32);
#undef XU
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

template <typename S>
cslsm_status tikhonov_typed(const Geom &g, Masks m, void *u_, void *d_, const float *b,
                            float rho, float lam, float gam, float *v_out, float *vprev,
                            double *partials, cudaStream_t s, const int *stop)
{
    S *u = (S *)u_, *d = (S *)d_;
    const uintptr_t al = (uintptr_t)u | (uintptr_t)d | (uintptr_t)b | (uintptr_t)m.words |
                         (uintptr_t)v_out;
    if (!vprev && !partials && !stop && g.HW() % 2 == 0 && (al & 7) == 0) {
        const int pairs = g.HW() / 2;
        const size_t sm = sizeof(float2) * kThreads * (size_t)g.R;
        static_assert(sizeof(float2) * kThreads * CSLSM_MAX_R <= 227 * 1024, "staging too large");
        CSLSM_CUDA(cudaFuncSetAttribute(tikhonov_iter_v2_kernel<S>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)(sizeof(float2) * kThreads * CSLSM_MAX_R)));
        LaunchScope ls(K_TIK_ITER, s);
        tikhonov_iter_v2_kernel<S><<<(pairs + kThreads - 1) / kThreads, kThreads, sm, s>>>(
            u, d, b, m.words, m.wstride, g.HW(), g.R, g.N, rho, lam, gam, v_out);
        CSLSM_LAUNCHED();
        return CSLSM_OK;
    }
    const dim3 grid = pixel_grid(g.HW(), 1);
#define TK(RM)                                                                            \
    tikhonov_iter_kernel<RM, S><<<grid, kThreads, 0, s>>>(u, d, b, m.words, m.wstride,   \
                                                          g.HW(), g.R, g.N, rho, lam, gam, \
                                                          v_out, vprev, partials, stop)
    LaunchScope ls(K_TIK_ITER, s);
    if (g.R <= 4) TK(4);
    else if (g.R <= 8) TK(8);
    else if (g.R <= 16) TK(16);
    else TK(32);
#undef TK
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_xupdate_w(const Geom &g, Masks m, int storage, const void *u, const void *d,
                              const float *b, float rho, void *w, float *v_out, float *vprev,
                              double *partials, int nblocks_red, cudaStream_t s, const int *stop)
{
    const dim3 grid = pixel_grid(g.HW(), g.N);
    if (partials && (int)(grid.x * grid.y) > nblocks_red) {
        set_error("reduction buffer too small");
        return CSLSM_ERR_INVALID_ARG;
    }
    switch (storage) {
    case CSLSM_STORE_BF16:
        return xupdate_typed<__nv_bfloat16>(g, m, u, d, b, rho, w, v_out, vprev, partials, s, stop);
    case CSLSM_STORE_FP16:
        return xupdate_typed<__half>(g, m, u, d, b, rho, w, v_out, vprev, partials, s, stop);
    default:
        return xupdate_typed<float>(g, m, u, d, b, rho, w, v_out, vprev, partials, s, stop);
    }
}

cslsm_status launch_tikhonov_iter(const Geom &g, Masks m, int storage, void *u, void *d,
                                  const float *b, float rho, float lam, float gam, float *v_out,
                                  float *vprev, double *partials, int nblocks_red, cudaStream_t s,
                                  const int *stop)
{
    const dim3 grid = pixel_grid(g.HW(), 1);
    if (partials && (int)grid.x > nblocks_red) {
        set_error("reduction buffer too small");
        return CSLSM_ERR_INVALID_ARG;
    }
    switch (storage) {
    case CSLSM_STORE_BF16:
        return tikhonov_typed<__nv_bfloat16>(g, m, u, d, b, rho, lam, gam, v_out, vprev,
                                             partials, s, stop);
    case CSLSM_STORE_FP16:
        return tikhonov_typed<__half>(g, m, u, d, b, rho, lam, gam, v_out, vprev, partials, s,
                                      stop);
    default:
        return tikhonov_typed<float>(g, m, u, d, b, rho, lam, gam, v_out, vprev, partials, s,
                                     stop);
    }
}

cslsm_status launch_tikhonov_prox(const float *in, float *out, long long n, float rho, float lam,
                                  cudaStream_t s)
{
    long long blocks = (n + kThreads - 1) / kThreads;
    if (blocks > 8192) blocks = 8192;
    if (blocks < 1) blocks = 1;
    LaunchScope ls(K_TIK_PROX, s);
    tikhonov_prox_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(in, out, n, rho, lam);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_psnr_partials(const float *x, const float *ref, size_t n, double *partials,
                                  int nblocks, cudaStream_t s)
{
    LaunchScope ls(K_PSNR, s);
    psnr_partials_kernel<<<nblocks, kThreads, 0, s>>>(x, ref, n, partials);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_psnr_finish(const double *partials, int nblocks, size_t n, double *out,
                                cudaStream_t s)
{
    LaunchScope ls(K_REDUCE, s);
    finish_pairs_kernel<true><<<1, kThreads, 0, s>>>(partials, nblocks, n, out);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_tol_check(const double *red, float tol, int k, TolState *state,
                              cudaStream_t s)
{
    LaunchScope ls(K_REDUCE, s);
    tol_check_kernel<<<1, 32, 0, s>>>(red, tol, k, state);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_copy_if_stopped(const TolState *state, const float *src, float *dst,
                                    size_t n, cudaStream_t s)
{
    long long blocks = ((long long)n + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    LaunchScope ls(K_REDUCE, s);
    copy_if_stopped_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(state, src, dst, n);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status launch_sum_pairs(const double *partials, int nblocks, double *out2, cudaStream_t s)
{
    LaunchScope ls(K_REDUCE, s);
    finish_pairs_kernel<false><<<1, kThreads, 0, s>>>(partials, nblocks, 0, out2);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

}  // namespace cslsm
