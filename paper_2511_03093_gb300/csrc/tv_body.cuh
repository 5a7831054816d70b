// TV prox tile body shared by the per-launch kernel (kernels_tv.cu) and the
// persistent batched solver (kernels_batch.cu); the algorithm and the
// shared-memory design are described at the top of kernels_tv.cu.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

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

// Packed pairs of FP32 operations (PTX .f32x2): each half is computed and
// rounded to nearest even exactly as the scalar instruction would, so the
// pair forms below give the same bits as two scalar operations in half the
// instructions.
__device__ __forceinline__ unsigned long long f2_pack(float2 v)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}

__device__ __forceinline__ float2 f2_unpack(unsigned long long r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}

__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
    return f2_unpack(r);
}

// Shared tail of one Chambolle update of a lane's two columns from the
// gradients (gx, gy) of q: |grad q| per column, then
// p <- (p + tau grad q) / (1 + tau |grad q|) for both components.
__device__ __forceinline__ float2 chambolle_tail(float2 gx, float2 gy, float2 pc, float tau,
                                                 float2 &p2c)
{
    const float2 s = fma2(gx, gx, mul2(gy, gy));
    const float2 t2 = make_float2(tau, tau);
    const float2 den = fma2(t2, make_float2(sqrt_approx(s.x), sqrt_approx(s.y)),
                            make_float2(1.f, 1.f));
    const float2 inv = make_float2(rcp_approx(den.x), rcp_approx(den.y));
    p2c = mul2(fma2(t2, gy, p2c), inv);
    return mul2(fma2(t2, gx, pc), inv);
}

// One Chambolle update of the two columns a lane owns at row i.
__device__ __forceinline__ float2 chambolle_pair(float2 qc, float2 qn, float qr, float2 pc,
                                                 float mr, float mc0, float mc1, float tau,
                                                 float2 &p2c)
{
    const float2 gx = mul2(sub2(qn, qc), make_float2(mr, mr));
    const float2 gy = mul2(sub2(make_float2(qc.y, qr), qc), make_float2(mc0, mc1));
    return chambolle_tail(gx, gy, pc, tau, p2c);
}

// chambolle_pair with every mask equal to one (a tile whose region lies inside
// the image); multiplying by one is exact, so the results are bit-identical.
__device__ __forceinline__ float2 chambolle_pair_interior(float2 qc, float2 qn, float qr,
                                                          float2 pc, float tau, float2 &p2c)
{
    return chambolle_tail(sub2(qn, qc), sub2(make_float2(qc.y, qr), qc), pc, tau, p2c);
}

// q = div p - g / theta at a lane's two columns of one row, from p1 of the row
// (p1c) and of the row above (pu), p2 of the row (p2c) and p2 of the column to
// the left of the lane's first column (p2l).
__device__ __forceinline__ float2 q_pair(float2 p1c, float2 pu, float2 p2c, float p2l, float2 g,
                                         float inv_theta)
{
    const float2 dv = add2(sub2(p1c, pu), sub2(p2c, make_float2(p2l, p2c.x)));
    return fma2(g, make_float2(-inv_theta, -inv_theta), dv);
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

// Row i of g for a lane: from a register array of the warp's rows, or from the
// warp's rows in shared memory ([RPW][32] float2), which frees 2 RPW registers
// for taller regions at one shared load per row and step.
// Row mask of row i (1 where the row has a row below it in the image): from an
// array of the warp's rows, or from bit i of a word (fewer registers).
template <int RPW>
__device__ __forceinline__ float mr_at(const float (&mr)[RPW], int i) { return mr[i]; }
template <int RPW>
__device__ __forceinline__ float mr_at(unsigned mr, int i) { return (mr >> i) & 1u ? 1.f : 0.f; }

template <typename G>
__device__ __forceinline__ float2 g_row(const G &g, int i, int lane)
{
    if constexpr (std::is_pointer<G>::value)
        return g[i * 32 + lane];
    else
        return g[i];
}

// ns Chambolle steps on the warp's rows (registers) with one barrier per step.
// INTERIOR: the CTA's whole region lies inside the image, all masks are one.
//
// Only the local rows [lo, hi) must be exact after the last step.  p^{t+1} of
// a row depends on p^t of the rows above and below, so step t (of ns) must be
// exact on [lo - e, hi + e) with e = ns - 1 - t, a band that narrows by one
// row per side and step.  A warp whose rows (local rows 1 + wp RPW ..
// (wp + 1) RPW) miss that band skips the step (it still takes the barrier);
// the stale rows it leaves, in registers and in the boundary-row buffers, are
// read only by rows outside the band of the next step, so the rows that
// matter get exactly the values of a full update.
//
// g (constant over the steps) is read through g_row.  ROLL: q of row i + 1 is
// formed just before row i's update instead of q of every row first, so two q
// values are live instead of RPW + 1 (the shuffles keep their order, so the
// compiler cannot interleave the other way round); the same operations on the
// same values, so the same bits.
template <bool INTERIOR, int B, int RPW, bool ROLL = false, typename G, typename MR>
__device__ __forceinline__ void sweep_steps(Bnd<B> &sb, float2 (&p1)[RPW], float2 (&p2)[RPW],
                                            const G &g, float2 gdn,
                                            const MR &mr, float mc0, float mc1,
                                            float inv_theta, float tau, int ns, int wp, int lane,
                                            int lo, int hi)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int r0 = 1 + wp * RPW;
    for (int t = 0; t < ns; ++t) {
        const int par = t & 1, nxt = par ^ 1;
        const int e = ns - 1 - t;
        if (r0 + RPW > lo - e && r0 < hi + e) {
            const float2 pu0 = sb.up[par][wp][lane];
            const float2 dn1 = sb.dn1[par][wp][lane], dn2 = sb.dn2[par][wp][lane];
            if (ROLL) {
                // row by row: q of row i + 1 (from the old p1 of row i), then row
                // i's update; two q values live instead of RPW + 1
                float2 qc = q_pair(p1[0], pu0, p2[0], __shfl_up_sync(FULL, p2[0].y, 1),
                                   g_row(g, 0, lane), inv_theta);
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    const float2 qn =
                        i + 1 < RPW
                            ? q_pair(p1[i + 1], p1[i], p2[i + 1],
                                     __shfl_up_sync(FULL, p2[i + 1].y, 1),
                                     g_row(g, i + 1, lane), inv_theta)
                            : q_pair(dn1, p1[RPW - 1], dn2, __shfl_up_sync(FULL, dn2.y, 1), gdn,
                                     inv_theta);
                    const float qr = __shfl_down_sync(FULL, qc.x, 1);
                    float2 p2n = p2[i];
                    const float2 p1n =
                        INTERIOR ? chambolle_pair_interior(qc, qn, qr, p1[i], tau, p2n)
                                 : chambolle_pair(qc, qn, qr, p1[i], mr_at<RPW>(mr, i), mc0, mc1, tau, p2n);
                    p1[i] = p1n;
                    p2[i] = p2n;
                    qc = qn;
                }
            } else {
            float2 q[RPW + 1];
#pragma unroll
            for (int i = 0; i < RPW; ++i)
                q[i] = q_pair(p1[i], i == 0 ? pu0 : p1[i - 1], p2[i],
                              __shfl_up_sync(FULL, p2[i].y, 1), g_row(g, i, lane), inv_theta);
            q[RPW] = q_pair(dn1, p1[RPW - 1], dn2, __shfl_up_sync(FULL, dn2.y, 1), gdn, inv_theta);
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                const float qr = __shfl_down_sync(FULL, q[i].x, 1);
                float2 p2n = p2[i];
                const float2 p1n =
                    INTERIOR ? chambolle_pair_interior(q[i], q[i + 1], qr, p1[i], tau, p2n)
                             : chambolle_pair(q[i], q[i + 1], qr, p1[i], mr_at<RPW>(mr, i), mc0, mc1, tau,
                                              p2n);
                p1[i] = p1n;
                p2[i] = p2n;
            }
            }
            if (wp + 1 < B) sb.up[nxt][wp + 1][lane] = p1[RPW - 1];
            if (wp > 0) {
                sb.dn1[nxt][wp - 1][lane] = p1[0];
                sb.dn2[nxt][wp - 1][lane] = p2[0];
            }
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
        qc = q_pair(p1c, p1u, p2c, p2l, gc, inv_theta);
    }
    for (int i = r0; i < r1; ++i, ++gi) {
        a1 += PW;
        a2 += PW;
        gg += PW;
        const float2 p1n = *reinterpret_cast<const float2 *>(a1);
        const float2 p2n = *reinterpret_cast<const float2 *>(a2);
        const float2 gn = *reinterpret_cast<const float2 *>(gg);
        const float p2l = reinterpret_cast<const float2 *>(a2 - 2)->y;
        const float2 qn = q_pair(p1n, p1c, p2n, p2l, gn, inv_theta);
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
            const size_t vi = (size_t)n * HW + o;
            const float ur = keep<S>(uv, vi, kKeyU);
            st<S>((S *)a.u + vi, ur);
            if (a.d) st<S>((S *)a.d + vi, keep<S>(ld_l2<S>(wn + o) - ur, vi, kKeyD));
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
