// TV prox tile body shared by the per-launch kernel (kernels_tv.cu) and the
// persistent batched solver (kernels_batch.cu); the algorithm and the
// shared-memory design are described at the top of kernels_tv.cu.
#pragma once

#include <cuda_runtime.h>

#include "storage.cuh"

namespace cslsm {

struct TvLaunch {
    const void *w;  // element type S of the kernel instantiation
    void *u;
    void *d;
    const float *pin;  // [2][nslices][H][W] dual field entering this launch, or null (p = 0)
    float *pout;       // [2][nslices][H][W] dual field leaving it (write_final == 0)
    int H, W, Z, n0, nslices;
    int T;             // steps in this launch
    int TH, TW, RH;    // tile rows / columns, region rows (region columns: 62 C + 2)
    float rho, gamma, inv_rho2g;
    float theta, inv_theta, tau;
    int write_final;
    int storage;
    const int *stop;  // device flag of a tolerance-stopped solve (skip when set), or null
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

// Region of RH rows x RW = 62 C + 2 columns, rows stored with pitch PW = 64 C
// floats (the columns beyond RW stay zero).  Every array starts 2 floats into its allocation so that column -1
// (read as the left neighbour of column 0, never updated) is addressable.
template <int C, int B>
struct Region {
    static constexpr int RW = 62 * C + 2;
    static constexpr int PW = 64 * C;
    static constexpr int NT = C * B * 32;
    __host__ __device__ static size_t array_floats(int RH) { return (size_t)PW * RH + 4; }
};

// One Chambolle update of the two columns a lane owns at row i.
__device__ __forceinline__ float2 chambolle_pair(float2 qc, float2 qn, float qr, float2 pc,
                                                 float mr, float mc0, float mc1, float tau,
                                                 float2 &p2c)
{
    const float gx0 = (qn.x - qc.x) * mr, gy0 = (qc.y - qc.x) * mc0;
    const float gx1 = (qn.y - qc.y) * mr, gy1 = (qr - qc.y) * mc1;
    const float i0 = rcp_approx(fmaf(tau, sqrt_approx(fmaf(gx0, gx0, gy0 * gy0)), 1.f));
    const float i1 = rcp_approx(fmaf(tau, sqrt_approx(fmaf(gx1, gx1, gy1 * gy1)), 1.f));
    p2c = make_float2(fmaf(tau, gy0, p2c.x) * i0, fmaf(tau, gy1, p2c.y) * i1);
    return make_float2(fmaf(tau, gx0, pc.x) * i0, fmaf(tau, gx1, pc.y) * i1);
}

// chambolle_pair with every mask equal to one (a tile whose region lies inside
// the image); multiplying by one is exact, so the results are bit-identical.
__device__ __forceinline__ float2 chambolle_pair_interior(float2 qc, float2 qn, float qr,
                                                          float2 pc, float tau, float2 &p2c)
{
    const float gx0 = qn.x - qc.x, gy0 = qc.y - qc.x;
    const float gx1 = qn.y - qc.y, gy1 = qr - qc.y;
    const float i0 = rcp_approx(fmaf(tau, sqrt_approx(fmaf(gx0, gx0, gy0 * gy0)), 1.f));
    const float i1 = rcp_approx(fmaf(tau, sqrt_approx(fmaf(gx1, gx1, gy1 * gy1)), 1.f));
    p2c = make_float2(fmaf(tau, gy0, p2c.x) * i0, fmaf(tau, gy1, p2c.y) * i1);
    return make_float2(fmaf(tau, gx0, pc.x) * i0, fmaf(tau, gx1, pc.y) * i1);
}

// Boundary rows exchanged between the warps of a CTA each step (double-
// buffered by step parity): p1 of the row above warp w's rows, p1 and p2 of
// the row below.
template <int B>
struct Bnd {
    float2 up[2][B][32];
    float2 dn1[2][B][32];
    float2 dn2[2][B][32];
};

// ns Chambolle steps on the warp's rows (registers) with one barrier per step.
// INTERIOR: the CTA's whole region lies inside the image, all masks are one.
template <bool INTERIOR, int B, int RPW>
__device__ __forceinline__ void sweep_steps(Bnd<B> &sb, float2 (&p1)[RPW], float2 (&p2)[RPW],
                                            const float2 (&g)[RPW], float2 gdn,
                                            const float (&mr)[RPW], float mc0, float mc1,
                                            float inv_theta, float tau, int ns, int wp, int lane)
{
    constexpr unsigned FULL = 0xffffffffu;
    for (int t = 0; t < ns; ++t) {
        const int par = t & 1, nxt = par ^ 1;
        const float2 pu0 = sb.up[par][wp][lane];
        const float2 dn1 = sb.dn1[par][wp][lane], dn2 = sb.dn2[par][wp][lane];
        float2 q[RPW + 1];
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const float p2l = __shfl_up_sync(FULL, p2[i].y, 1);
            const float2 pu = i == 0 ? pu0 : p1[i - 1];
            q[i].x = fmaf(-g[i].x, inv_theta, (p1[i].x - pu.x) + (p2[i].x - p2l));
            q[i].y = fmaf(-g[i].y, inv_theta, (p1[i].y - pu.y) + (p2[i].y - p2[i].x));
        }
        {
            const float p2l = __shfl_up_sync(FULL, dn2.y, 1);
            q[RPW].x = fmaf(-gdn.x, inv_theta, (dn1.x - p1[RPW - 1].x) + (dn2.x - p2l));
            q[RPW].y = fmaf(-gdn.y, inv_theta, (dn1.y - p1[RPW - 1].y) + (dn2.y - dn2.x));
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const float qr = __shfl_down_sync(FULL, q[i].x, 1);
            float2 p2n = p2[i];
            const float2 p1n =
                INTERIOR ? chambolle_pair_interior(q[i], q[i + 1], qr, p1[i], tau, p2n)
                         : chambolle_pair(q[i], q[i + 1], qr, p1[i], mr[i], mc0, mc1, tau, p2n);
            p1[i] = p1n;
            p2[i] = p2n;
        }
        if (wp + 1 < B) sb.up[nxt][wp + 1][lane] = p1[RPW - 1];
        if (wp > 0) {
            sb.dn1[nxt][wp - 1][lane] = p1[0];
            sb.dn2[nxt][wp - 1][lane] = p2[0];
        }
        __syncthreads();
    }
}

// One Chambolle step on rows [r0, r1) of a band: reads p^t (A1, A2) and g
// (sg) at rows r0-1 .. r1, writes p^{t+1} (B1, B2) at rows [r0, r1).  Arrays
// have row pitch PW; the lane owns local columns j0, j0 + 1; gi is the image
// row of r0 (unsigned, so rows above the image fail gi < H-1).
template <int PW>
__device__ __forceinline__ void tv_band_rows(const float *A1, const float *A2, const float *sg,
                                             float *B1, float *B2, int r0, int r1, int j0,
                                             unsigned gi, unsigned Hm1, float mc0, float mc1,
                                             float inv_theta, float tau, int lane)
{
    const float *a1 = A1 + r0 * PW + j0, *a2 = A2 + r0 * PW + j0, *gg = sg + r0 * PW + j0;
    float *b1 = B1 + r0 * PW + j0, *b2 = B2 + r0 * PW + j0;
    float2 p1c = *reinterpret_cast<const float2 *>(a1);
    float2 p2c = *reinterpret_cast<const float2 *>(a2);
    float2 qc;
    {
        const float2 p1u = *reinterpret_cast<const float2 *>(a1 - PW);
        const float2 gc = *reinterpret_cast<const float2 *>(gg);
        const float p2l = reinterpret_cast<const float2 *>(a2 - 2)->y;
        qc.x = fmaf(-gc.x, inv_theta, (p1c.x - p1u.x) + (p2c.x - p2l));
        qc.y = fmaf(-gc.y, inv_theta, (p1c.y - p1u.y) + (p2c.y - p2c.x));
    }
    for (int i = r0; i < r1; ++i, ++gi) {
        a1 += PW;
        a2 += PW;
        gg += PW;
        const float2 p1n = *reinterpret_cast<const float2 *>(a1);
        const float2 p2n = *reinterpret_cast<const float2 *>(a2);
        const float2 gn = *reinterpret_cast<const float2 *>(gg);
        const float p2l = reinterpret_cast<const float2 *>(a2 - 2)->y;
        float2 qn;
        qn.x = fmaf(-gn.x, inv_theta, (p1n.x - p1c.x) + (p2n.x - p2l));
        qn.y = fmaf(-gn.y, inv_theta, (p1n.y - p1c.y) + (p2n.y - p2n.x));
        const float qr = __shfl_down_sync(0xffffffffu, qc.x, 1);
        const float mr = gi < Hm1 ? 1.f : 0.f;
        float2 p2new = p2c;
        const float2 p1new = chambolle_pair(qc, qn, qr, p1c, mr, mc0, mc1, tau, p2new);
        if (lane < 31) {  // lane 31's columns belong to the next chunk
            *reinterpret_cast<float2 *>(b1) = p1new;
            *reinterpret_cast<float2 *>(b2) = p2new;
        }
        b1 += PW;
        b2 += PW;
        qc = qn;
        p1c = p1n;
        p2c = p2n;
    }
}

// One CTA's work: the tile (bx, by) of launch slice sl.  C column chunks of 62
// owned columns, B row bands: C * B warps; smem holds Region<C, B> arrays.
template <int C, int B, typename S>
__device__ __forceinline__ void tv_tile_body(const TvLaunch &a, int bx, int by, int sl,
                                             float *smem)
{
    constexpr int kBands = B;
    using Rg = Region<C, B>;
    constexpr int RW = Rg::RW, PW = Rg::PW, NT = Rg::NT;
    const int T = a.T, RH = a.RH;
    const size_t AF = Rg::array_floats(RH);
    float *sg = smem + 2;
    float *A1 = sg + AF, *A2 = A1 + AF;  // p^t   (components along rows / columns)
    float *B1 = A2 + AF, *B2 = B1 + AF;  // p^t+1
    const int n = a.n0 + sl;
    const int H = a.H, W = a.W;
    const size_t HW = (size_t)H * W;
    const int gi0 = by * a.TH - (T + 1);
    const int gj0 = bx * a.TW - (T + 1);

    const S *wn = (const S *)a.w + (size_t)n * HW;
    const S *um = (const S *)a.u + (size_t)((n + a.Z - 1) % a.Z) * HW;
    const S *up = (const S *)a.u + (size_t)((n + 1) % a.Z) * HW;
    const float *p1in = a.pin ? a.pin + (size_t)sl * HW : nullptr;
    const float *p2in = a.pin ? a.pin + (size_t)(a.nslices + sl) * HW : nullptr;

    if (threadIdx.x < 2)  // column -1 of row 0 .. and the pads: zero
        for (int k = 0; k < 5; ++k) smem[k * AF + threadIdx.x] = 0.f;
    for (int idx = threadIdx.x; idx < RH * PW; idx += NT) {
        const int li = idx / PW, lj = idx - li * PW;
        const int gi = gi0 + li, gj = gj0 + lj;
        float g = 0.f, p1 = 0.f, p2 = 0.f;
        if (lj < RW && gi >= 0 && gi < H && gj >= 0 && gj < W) {
            const size_t o = (size_t)gi * W + gj;
            const float wv = ld_l2<S>(wn + o);
            g = a.gamma > 0.f ? (a.rho * wv + a.gamma * (ld_l2<S>(um + o) + ld_l2<S>(up + o))) *
                                    a.inv_rho2g
                              : wv;
            if (p1in) {
                p1 = __ldcg(p1in + o);
                p2 = __ldcg(p2in + o);
            }
        }
        sg[idx] = g;
        A1[idx] = p1;
        A2[idx] = p2;
        B1[idx] = 0.f;
        B2[idx] = 0.f;
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int chunk = warp % C, band = warp / C;
    const int j0 = chunk * 62 + 2 * lane;  // local columns j0, j0 + 1 (even: float2)
    const int gj = gj0 + j0;
    const float mc0 = (gj >= 0 && gj < W - 1) ? 1.f : 0.f;
    const float mc1 = (gj + 1 >= 0 && gj + 1 < W - 1) ? 1.f : 0.f;
    const float inv_theta = a.inv_theta, tau = a.tau;
    const unsigned Hm1 = (unsigned)(H - 1);

    for (int s = 0; s < T; ++s) {
        const int lo = s + 1, len = RH - 2 * s - 3;  // p^{s+1} rows [s+1, RH-s-2)
        const int r0 = lo + (band * len) / kBands;
        const int r1 = lo + ((band + 1) * len) / kBands;
        if (r0 < r1)
            tv_band_rows<PW>(A1, A2, sg, B1, B2, r0, r1, j0, (unsigned)(gi0 + r0), Hm1, mc0, mc1,
                             inv_theta, tau, lane);
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
        const int l = (T + 1 + ti) * PW + (T + 1 + tj);
        const size_t o = (size_t)gi * W + gjj;
        if (a.write_final) {
            const float divp = (A1[l] - A1[l - PW]) + (A2[l] - A2[l - 1]);
            const float uv = sg[l] - a.theta * divp;
            st<S>((S *)a.u + (size_t)n * HW + o, uv);
            if (a.d) st<S>((S *)a.d + (size_t)n * HW + o, ld_l2<S>(wn + o) - rnd<S>(uv));
        } else {
            a.pout[(size_t)sl * HW + o] = A1[l];
            a.pout[(size_t)(a.nslices + sl) * HW + o] = A2[l];
        }
    }
}

template <int C, int B, typename S>
__global__ void __launch_bounds__(C * B * 32) tv_tile_kernel(const TvLaunch a)
{
    if (a.stop && *a.stop) return;
    extern __shared__ float smem[];
    tv_tile_body<C, B, S>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}


inline size_t tv_smem_bytes(int C, int RH)
{
    return 5ull * ((size_t)64 * C * RH + 4) * sizeof(float);
}

}  // namespace cslsm
