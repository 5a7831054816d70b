// Persistent Gauss-Seidel sweep of the TV u-step along z (Sec. III-C: the
// u-update of slice n takes the newest u_{n-1} and the previous u_{n+1}).
//
// The sweep is a chain of Z proxes: slice n cannot start before slice n-1 is
// finished around it.  Launching one kernel per slice leaves every launch with
// one 2-D slice of work and makes each CTA recompute a halo of T + 1 pixels
// (the dependence cone of T Chambolle steps); at 512 x 512 and T = 20 that
// halo is most of the work.  Here ONE cooperative launch runs the whole sweep.
// Every CTA owns the same output tile in every slice and keeps its tile, a
// halo of k + 1 pixels and g in shared memory.  The T steps of a slice are cut
// into phases of at most k steps; between phases a CTA publishes the dual
// field p of its own tile to global memory (L2) and reads the halo ring from
// its eight neighbours' tiles, so the halo is k + 1 instead of T + 1.
//
// Ordering: every (slice, phase) pair is an epoch e = n * P + j.  A CTA
// starts epoch e only after its eight neighbours have completed epoch e - 1
// (a per-tile flag holding the id of the last completed epoch, written by one
// thread with release semantics after a CTA barrier, polled with acquire
// loads).  Neighbours are
// therefore never more than one epoch apart, which makes the reuse of the two
// parity buffers of p and the in-place update of u safe: the data a CTA
// overwrites in epoch e was last read by its neighbours in epoch e - 1 or
// earlier.  Data written in the launch is read with L2-only loads (__ldcg).
// Epoch ids grow across launches (a per-workspace base), so flags are never
// reset.  All CTAs are resident (cooperative launch), so the waits cannot
// deadlock; every wait is still bounded by a wall-clock limit (%globaltimer),
// after which the CTA raises the workspace's error word, every CTA returns, and
// the host reports CSLSM_ERR_TIMEOUT.
//
// Arithmetic per pixel is exactly that of the per-slice tile kernel
// (tv_band_rows, same g, same final u and d), so the two paths give
// bit-identical results.
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

constexpr int kPW = 64;  // region columns: one warp of 32 lanes x 2 columns

struct ZsArgs {
    const void *w;  // [Z][H][W] element type S
    void *u, *d;
    float *pbuf;      // [2 parities][2 components][H][W]
    unsigned *flags;  // [tiles] id of the last completed epoch
    int *err;
    unsigned base;  // epoch e of this launch has id base + 1 + e
    int H, W, Z, T, k, P, hh, TH, TW, RH, tx, ty;
    float rho, gamma, inv_rho2g, theta, inv_theta, tau;
    long long limit_ns;
    int stall;        // test hook: tile 0 waits in epoch 1 for an id nobody publishes
    const int *stop;  // device flag of a tolerance-stopped solve (skip when set), or null
};

__device__ __forceinline__ unsigned long long zs_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spins until *f >= target (modulo 2^32); false on timeout or a raised error.
__device__ bool wait_ge(const unsigned *f, unsigned target, int *err, long long limit_ns)
{
    unsigned long long t0 = 0;
    for (unsigned spins = 1;; ++spins) {
        if ((int)(ld_acquire(f) - target) >= 0) return true;
        if ((spins & 127u) == 0) {
            if (*(volatile int *)err) return false;
            const unsigned long long now = zs_ns();
            if (t0 == 0) {
                t0 = now;
            } else if ((long long)(now - t0) > limit_ns) {
                atomicExch(err, 1);
                return false;
            }
        }
    }
}

// Dual field of one warp's rows in registers: the warp owns RPW consecutive
// local rows (from 1 + warp * RPW), each lane two adjacent columns.  Per step
// a warp needs, from other warps, p1 of the row above its first row and p1, p2
// of the row below its last row; these boundary rows go through shared memory.
// Local rows 0 and RH - 1 are never updated within a phase (their staleness
// stays in the halo), nor are wrong neighbours of columns 0 and 63.
template <int B, int RPW, typename S>
__global__ void __launch_bounds__(B * 32) tvz_sweep_kernel(const ZsArgs a)
{
    if (a.stop && *a.stop) return;  // every CTA reads the same flag: all return
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int RH = B * RPW + 2;
    __shared__ Bnd<B> sb;
    __shared__ int s_abort;
    const int hh = a.hh, TH = a.TH, TW = a.TW, H = a.H, W = a.W;
    const int tile = blockIdx.x;
    const int bx = tile % a.tx, by = tile / a.tx;
    const int gi0 = by * TH - hh, gj0 = bx * TW - hh;
    const size_t HW = (size_t)H * W;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int j0 = 2 * lane;      // local columns j0, j0 + 1
    const int r0 = 1 + wp * RPW;  // local rows r0 .. r0 + RPW - 1
    const int gc = gj0 + j0;
    const float mc0 = (gc >= 0 && gc < W - 1) ? 1.f : 0.f;
    const float mc1 = (gc + 1 >= 0 && gc + 1 < W - 1) ? 1.f : 0.f;
    const bool inc[2] = {gc >= 0 && gc < W, gc + 1 >= 0 && gc + 1 < W};
    const bool ownc[2] = {inc[0] && j0 >= hh && j0 < hh + TW,
                          inc[1] && j0 + 1 >= hh && j0 + 1 < hh + TW};
    // every row and column mask of the region is one
    const bool interior = gi0 >= 0 && gi0 + RH < H && gj0 >= 0 && gj0 + kPW < W;
    const unsigned Hm1 = (unsigned)(H - 1);
    float mr[RPW];
    bool inr[RPW + 1], ownr[RPW];
    int off[RPW + 1];  // image offset of (row, column gc); used only inside the image
#pragma unroll
    for (int i = 0; i <= RPW; ++i) {
        const int gi = gi0 + r0 + i;
        inr[i] = gi >= 0 && gi < H;
        off[i] = gi * W + gc;
        if (i < RPW) {
            mr[i] = (unsigned)gi < Hm1 ? 1.f : 0.f;
            ownr[i] = inr[i] && r0 + i >= hh && r0 + i < hh + TH;
        }
    }
    const float inv_theta = a.inv_theta, tau = a.tau;

    const unsigned *nflag = nullptr;  // neighbour polled by this thread
    if (threadIdx.x < 9 && threadIdx.x != 4) {
        const int ny = by + (int)threadIdx.x / 3 - 1, nx = bx + (int)threadIdx.x % 3 - 1;
        if (ny >= 0 && ny < a.ty && nx >= 0 && nx < a.tx) nflag = a.flags + ny * a.tx + nx;
    }
    if (threadIdx.x == 0) s_abort = 0;

    float2 p1[RPW], p2[RPW], g[RPW], gdn;
    float2 wo[RPW];  // w_n of the warp's rows, kept for d_n = w_n - u_n at the slice end
    for (int n = 0; n < a.Z; ++n) {
        const S *wn = (const S *)a.w + (size_t)n * HW;
        const S *um = (const S *)a.u + (size_t)((n + a.Z - 1) % a.Z) * HW;
        const S *up = (const S *)a.u + (size_t)((n + 1) % a.Z) * HW;
        for (int j = 0; j < a.P; ++j) {
            const int e = n * a.P + j;
            // w_n and u_{n+1} do not depend on the neighbours' current epoch:
            // fetch them before waiting (held in p1 / p2, dead here).  u_{n+1}
            // of the last slice is the u_0 of this sweep, written in epoch
            // P - 1; it is complete for the neighbours from epoch P + 1 on.
            const bool pre_up = n + 1 < a.Z || e >= a.P + 1;
            if (j == 0) {
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    p1[i].x = inr[i] && inc[0] ? ld_l2<S>(wn + (size_t)off[i]) : 0.f;
                    p1[i].y = inr[i] && inc[1] ? ld_l2<S>(wn + (size_t)off[i] + 1) : 0.f;
                    if (pre_up) {
                        p2[i].x = inr[i] && inc[0] ? ld_l2<S>(up + (size_t)off[i]) : 0.f;
                        p2[i].y = inr[i] && inc[1] ? ld_l2<S>(up + (size_t)off[i] + 1) : 0.f;
                    }
                }
                gdn.x = inr[RPW] && inc[0] ? ld_l2<S>(wn + (size_t)off[RPW]) : 0.f;
                gdn.y = inr[RPW] && inc[1] ? ld_l2<S>(wn + (size_t)off[RPW] + 1) : 0.f;
            }
            if (e > 0) {
                if (nflag || (a.stall && tile == 0 && e == 1 && threadIdx.x == 0)) {
                    const unsigned target = (a.stall && tile == 0 && e == 1)
                                                ? a.base + 0x40000000u
                                                : a.base + (unsigned)e;  // id of epoch e - 1
                    if (!wait_ge(nflag ? nflag : a.flags + tile, target, a.err, a.limit_ns))
                        s_abort = 1;
                }
                __syncthreads();
                if (s_abort) return;
            }
            if (j == 0) {  // g of slice n on the warp's rows and the row below; p^0 = 0
                if (!pre_up) {
#pragma unroll
                    for (int i = 0; i < RPW; ++i) {
                        p2[i].x = inr[i] && inc[0] ? ld_l2<S>(up + (size_t)off[i]) : 0.f;
                        p2[i].y = inr[i] && inc[1] ? ld_l2<S>(up + (size_t)off[i] + 1) : 0.f;
                    }
                }
#pragma unroll
                for (int i = 0; i <= RPW; ++i) {
                    const bool in0 = inr[i] && inc[0], in1 = inr[i] && inc[1];
                    const float m0 = in0 ? ld_l2<S>(um + (size_t)off[i]) : 0.f;
                    const float m1 = in1 ? ld_l2<S>(um + (size_t)off[i] + 1) : 0.f;
                    const float u0 = in0 ? ld_l2<S>(up + (size_t)off[i]) : 0.f;
                    const float u1 = in1 ? ld_l2<S>(up + (size_t)off[i] + 1) : 0.f;
                    const float w0 = i < RPW ? p1[i < RPW ? i : 0].x : gdn.x;
                    const float w1 = i < RPW ? p1[i < RPW ? i : 0].y : gdn.y;
                    const float2 gv = make_float2(
                        in0 ? (a.rho * w0 + a.gamma * (m0 + (i < RPW ? p2[i < RPW ? i : 0].x : u0))) *
                                  a.inv_rho2g
                            : 0.f,
                        in1 ? (a.rho * w1 + a.gamma * (m1 + (i < RPW ? p2[i < RPW ? i : 0].y : u1))) *
                                  a.inv_rho2g
                            : 0.f);
                    if (i < RPW) g[i < RPW ? i : 0] = gv;
                    else gdn = gv;
                }
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    wo[i] = p1[i];
                    p1[i] = make_float2(0.f, 0.f);
                    p2[i] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    sb.up[q][wp][lane] = make_float2(0.f, 0.f);
                    sb.dn1[q][wp][lane] = make_float2(0.f, 0.f);
                    sb.dn2[q][wp][lane] = make_float2(0.f, 0.f);
                }
            } else {  // p on the ring from the neighbours; the own tile is in registers
                const float *P1 = a.pbuf + (size_t)((e - 1) & 1) * 2 * HW, *P2 = P1 + HW;
                float v1[RPW][2], v2[RPW][2];
#pragma unroll
                for (int i = 0; i < RPW; ++i)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const bool ring = !(ownr[i] && ownc[c]);
                        const bool in = inr[i] && inc[c];
                        v1[i][c] = ring && in ? __ldcg(P1 + (size_t)(off[i] + c)) : 0.f;
                        v2[i][c] = ring && in ? __ldcg(P2 + (size_t)(off[i] + c)) : 0.f;
                    }
                // frozen rows 0 and RH - 1 of the region
                float2 f1 = make_float2(0.f, 0.f), f2 = make_float2(0.f, 0.f);
                if (wp == 0 || wp == B - 1) {
                    const int gi = gi0 + (wp == 0 ? 0 : RH - 1);
                    if (gi >= 0 && gi < H) {
                        const size_t o = (size_t)(gi * W + gc);
                        if (inc[0]) {
                            f1.x = __ldcg(P1 + o);
                            f2.x = __ldcg(P2 + o);
                        }
                        if (inc[1]) {
                            f1.y = __ldcg(P1 + o + 1);
                            f2.y = __ldcg(P2 + o + 1);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    if (!(ownr[i] && ownc[0])) {
                        p1[i].x = v1[i][0];
                        p2[i].x = v2[i][0];
                    }
                    if (!(ownr[i] && ownc[1])) {
                        p1[i].y = v1[i][1];
                        p2[i].y = v2[i][1];
                    }
                }
                if (wp == 0) {
                    sb.up[0][0][lane] = f1;
                    sb.up[1][0][lane] = f1;
                }
                if (wp == B - 1) {
                    sb.dn1[0][B - 1][lane] = f1;
                    sb.dn1[1][B - 1][lane] = f1;
                    sb.dn2[0][B - 1][lane] = f2;
                    sb.dn2[1][B - 1][lane] = f2;
                }
                if (wp + 1 < B) sb.up[0][wp + 1][lane] = p1[RPW - 1];
                if (wp > 0) {
                    sb.dn1[0][wp - 1][lane] = p1[0];
                    sb.dn2[0][wp - 1][lane] = p2[0];
                }
            }
            __syncthreads();
            const int ns = min(a.k, a.T - j * a.k);
            // rows that must be exact after the phase: the own tile (published, or
            // kept for the next phase), plus the row above it when u_n = g - theta
            // div p is formed at the slice end
            const int lo = hh - (j == a.P - 1 ? 1 : 0), hi = hh + TH;
            if (interior)
                sweep_steps<true, B, RPW>(sb, p1, p2, g, gdn, mr, mc0, mc1, inv_theta, tau, ns,
                                          wp, lane, lo, hi);
            else
                sweep_steps<false, B, RPW>(sb, p1, p2, g, gdn, mr, mc0, mc1, inv_theta, tau, ns,
                                           wp, lane, lo, hi);
            if (j < a.P - 1) {  // publish p of the own tile
                float *Q1 = a.pbuf + (size_t)(e & 1) * 2 * HW, *Q2 = Q1 + HW;
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    if (ownr[i] && ownc[0]) {
                        Q1[(size_t)off[i]] = p1[i].x;
                        Q2[(size_t)off[i]] = p2[i].x;
                    }
                    if (ownr[i] && ownc[1]) {
                        Q1[(size_t)off[i] + 1] = p1[i].y;
                        Q2[(size_t)off[i] + 1] = p2[i].y;
                    }
                }
            } else {  // u_n = g - theta div p^T and d_n = w_n - u_n on the own tile
                S *un = (S *)a.u + (size_t)n * HW;
                S *dn = a.d ? (S *)a.d + (size_t)n * HW : nullptr;
                const float2 pu0 = sb.up[ns & 1][wp][lane];
#pragma unroll
                for (int i = 0; i < RPW; ++i) {
                    const float p2l = __shfl_up_sync(FULL, p2[i].y, 1);
                    const float2 pu = i == 0 ? pu0 : p1[i - 1];
                    const float dx = (p1[i].x - pu.x) + (p2[i].x - p2l);
                    const float dy = (p1[i].y - pu.y) + (p2[i].y - p2[i].x);
                    const float ux = g[i].x - a.theta * dx;
                    const float uy = g[i].y - a.theta * dy;
                    if (ownr[i] && ownc[0]) {
                        const size_t vi = (size_t)n * HW + (size_t)off[i];
                        const float ur = keep<S>(ux, vi, kKeyU);
                        st<S>(un + (size_t)off[i], ur);
                        if (dn) st<S>(dn + (size_t)off[i], keep<S>(wo[i].x - ur, vi, kKeyD));
                    }
                    if (ownr[i] && ownc[1]) {
                        const size_t vi = (size_t)n * HW + (size_t)off[i] + 1;
                        const float ur = keep<S>(uy, vi, kKeyU);
                        st<S>(un + (size_t)off[i] + 1, ur);
                        if (dn) st<S>(dn + (size_t)off[i] + 1, keep<S>(wo[i].y - ur, vi, kKeyD));
                    }
                }
            }
            __syncthreads();
            // the barrier orders every thread's stores before thread 0's release
            // store, whose release semantics make them visible (at gpu scope) to a
            // neighbour that acquires the flag
            if (threadIdx.x == 0) st_release(a.flags + tile, a.base + 1u + (unsigned)e);
        }
    }
}

// ---- host side ----------------------------------------------------------------

struct Cfg {
    int cand;      // candidate index
    int k, shape;  // steps per phase, row shape index
    int B, RPW;    // warps per CTA, rows per warp
    int hh, TH, TW, RH, tx, ty;
};

// Row shapes (warps, rows per warp): the region is B * RPW + 2 rows high.
constexpr int kShapes[][2] = {{16, 3}, {8, 6}, {16, 2}, {8, 4}, {12, 4}, {16, 4}, {8, 16}, {16, 8}};
constexpr int kNumShapes = 8;
constexpr int kKs[] = {4, 5, 6, 8, 10, 20};
constexpr int kNumK = 6;
constexpr int kNumCand = kNumShapes * kNumK * 2;  // x target CTAs per SM (1, 2)

template <int B, int RPW>
const void *kernel_for(int storage)
{
    if (storage == CSLSM_STORE_BF16) return (const void *)tvz_sweep_kernel<B, RPW, __nv_bfloat16>;
    if (storage == CSLSM_STORE_FP16) return (const void *)tvz_sweep_kernel<B, RPW, __half>;
    return (const void *)tvz_sweep_kernel<B, RPW, float>;
}

const void *kernel_of(int shape, int storage)
{
    switch (shape) {
    case 0: return kernel_for<16, 3>(storage);
    case 1: return kernel_for<8, 6>(storage);
    case 2: return kernel_for<16, 2>(storage);
    case 3: return kernel_for<8, 4>(storage);
    case 4: return kernel_for<12, 4>(storage);
    case 5: return kernel_for<16, 4>(storage);
    case 6: return kernel_for<8, 16>(storage);
    default: return kernel_for<16, 8>(storage);
    }
}

// Tiling of candidate c for an H x W slice with T steps; false if it does not
// fit (halo wider than a tile, more tiles than can be resident).
bool make_cfg(int c, int H, int W, int T, int sms, int storage, Cfg &f)
{
    f.cand = c;
    f.shape = c % kNumShapes;
    const int m = 1 + (c / kNumShapes) % 2;  // target CTAs per SM
    f.k = std::min(kKs[c / (2 * kNumShapes)], T);
    f.B = kShapes[f.shape][0];
    f.RPW = kShapes[f.shape][1];
    f.hh = f.k + 1;
    f.RH = f.B * f.RPW + 2;
    f.TW = kPW - 2 * f.hh;
    const int th_max = f.RH - 2 * f.hh;
    if (f.TW < 1 || th_max < 1) return false;
    f.tx = (W + f.TW - 1) / f.TW;
    // the shortest tiles that keep the grid within m CTAs per SM: the tile
    // count is then close to a multiple of the SM count
    const int ty_max = m * sms / f.tx;
    if (ty_max < 1) return false;
    f.TH = std::max((H + ty_max - 1) / ty_max, std::min(f.hh, H));
    if (f.TH > th_max) return false;
    f.ty = (H + f.TH - 1) / f.TH;
    if ((f.tx > 1 && f.TW < f.hh) || (f.ty > 1 && f.TH < f.hh)) return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel_of(f.shape, storage),
                                                      f.B * 32, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return f.tx * f.ty <= occ * sms;
}

// Model in SM cycles per slice: every region row is updated in every step
// (about 0.25 cycles per pixel on an SM at full issue, scaled down when fewer
// than 16 warps share the SM), plus a fixed cost per phase boundary.
double model(const Cfg &f, int T, int sms)
{
    const int tiles = f.tx * f.ty;
    const int per_sm = (tiles + sms - 1) / sms;
    const double warps = (double)f.B * per_sm;
    const double eff = std::min(1.0, warps / 16.0);
    const int P = (T + f.k - 1) / f.k;
    return per_sm * (double)T * f.RH * kPW * 0.25 / eff + 4000.0 * P;
}

std::mutex g_mu;
int g_enable = 1;
int g_force = -1;
double g_wait_s = 2.0;
int g_stall = 0;
using Key = std::tuple<int, int, int, int, int, int>;  // device, H, W, Z, T, storage
std::map<Key, Cfg> g_tuned;  // timed choice
std::map<Key, Cfg> g_model;  // model choice

int sm_count(int &dev)
{
    int sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cslsm_status launch(const TvSlices &s, const Cfg &f, ZsweepWs &ws, void *u, void *d,
                    cudaStream_t st)
{
    ZsArgs a{};
    a.w = s.w;
    a.u = u;
    a.d = d;
    a.pbuf = ws.pbuf;
    a.flags = ws.flags;
    a.err = ws.err;
    a.H = s.H;
    a.W = s.W;
    a.Z = s.Z;
    a.T = s.T;
    a.k = f.k;
    a.P = (s.T + f.k - 1) / f.k;
    a.hh = f.hh;
    a.TH = f.TH;
    a.TW = f.TW;
    a.RH = f.RH;
    a.tx = f.tx;
    a.ty = f.ty;
    a.rho = s.rho;
    a.gamma = s.gamma;
    a.inv_rho2g = 1.f / (s.rho + 2.f * s.gamma);
    a.theta = s.theta;
    a.inv_theta = s.theta > 0.f ? 1.f / s.theta : 0.f;
    a.tau = s.tau;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        a.limit_ns = (long long)(g_wait_s * 1e9);
        a.stall = g_stall;
    }
    a.stop = s.stop;
    a.base = ws.next_base;
    ws.next_base += (unsigned)(a.Z * a.P);

    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(f.tx * f.ty);
    cfg.blockDim = dim3(f.B * 32);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LaunchScope ls(K_TVZ, st);
    void *args[] = {(void *)&a};
    const cudaError_t e = cudaLaunchKernelExC(&cfg, kernel_of(f.shape, s.storage), args);
    if (e != cudaSuccess) {
        set_error("z-sweep cooperative launch failed: %s", cudaGetErrorString(e));
        return CSLSM_ERR_CUDA;
    }
    return CSLSM_OK;
}

// Reads (and clears) the error word; synchronises the stream.
cslsm_status check_err(ZsweepWs &ws, cudaStream_t st)
{
    int h = 0;
    CSLSM_CUDA(cudaMemcpyAsync(&h, ws.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CSLSM_CUDA(cudaStreamSynchronize(st));
    if (h) {
        CSLSM_CUDA(cudaMemsetAsync(ws.err, 0, sizeof(int), st));
        set_error("z-sweep: a neighbour wait exceeded its limit");
        return CSLSM_ERR_TIMEOUT;
    }
    return CSLSM_OK;
}

// Candidate for this geometry: forced, tuned, timed now (mode 1, outside
// capture, on scratch copies of u and d), or the model's best.
cslsm_status choose(const TvSlices &s, ZsweepWs &ws, cudaStream_t st, Cfg &out)
{
    int dev = 0;
    const int sms = sm_count(dev);
    int force;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        force = g_force;
    }
    if (force >= 0) {
        if (force >= kNumCand || !make_cfg(force, s.H, s.W, s.T, sms, s.storage, out)) {
            set_error("z-sweep candidate %d does not fit this geometry", force);
            return CSLSM_ERR_UNSUPPORTED;
        }
        return CSLSM_OK;
    }
    const auto key = std::make_tuple(dev, s.H, s.W, s.Z, s.T, s.storage);
    const bool timed = tv_get_mode() == 1;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            out = it->second;
            return CSLSM_OK;
        }
        if (!timed) {
            auto im = g_model.find(key);
            if (im != g_model.end()) {
                out = im->second;
                return CSLSM_OK;
            }
        }
    }
    std::vector<int> ok;
    int best = -1;
    double best_cost = 1e300;
    for (int c = 0; c < kNumCand; ++c) {
        Cfg f;
        if (!make_cfg(c, s.H, s.W, s.T, sms, s.storage, f)) continue;
        ok.push_back(c);
        const double m = model(f, s.T, sms);
        if (m < best_cost) {
            best_cost = m;
            best = c;
        }
    }
    if (best < 0) {
        set_error("no z-sweep tiling fits %d x %d with %d steps", s.H, s.W, s.T);
        return CSLSM_ERR_UNSUPPORTED;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CSLSM_CUDA(cudaStreamIsCapturing(st, &cap));
    if (timed && cap == cudaStreamCaptureStatusNone) {
        const size_t esz = s.storage == CSLSM_STORE_FP32 ? 4 : 2;
        const size_t bytes = esz * (size_t)s.Z * s.H * s.W;
        void *tu = nullptr, *td = nullptr;
        CSLSM_CUDA(cudaMallocAsync(&tu, bytes, st));
        CSLSM_CUDA(cudaMallocAsync(&td, bytes, st));
        CSLSM_CUDA(cudaMemcpyAsync(tu, s.u, bytes, cudaMemcpyDeviceToDevice, st));
        cudaEvent_t e0, e1;
        CSLSM_CUDA(cudaEventCreate(&e0));
        CSLSM_CUDA(cudaEventCreate(&e1));
        float best_ms = 1e30f;
        cslsm_status rs = CSLSM_OK;
        for (int c : ok) {
            Cfg f;
            make_cfg(c, s.H, s.W, s.T, sms, s.storage, f);
            float ms_min = 1e30f;
            for (int rep = 0; rep < 3 && rs == CSLSM_OK; ++rep) {
                cudaEventRecord(e0, st);
                rs = launch(s, f, ws, tu, td, st);
                cudaEventRecord(e1, st);
                if (rs == CSLSM_OK) {
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms_min = std::min(ms_min, ms);
                }
            }
            if (rs != CSLSM_OK) break;
            if (ms_min < best_ms) {
                best_ms = ms_min;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFreeAsync(tu, st);
        cudaFreeAsync(td, st);
        if (rs != CSLSM_OK) return rs;
        CSLSM_CUDA(cudaGetLastError());
        rs = check_err(ws, st);
        if (rs != CSLSM_OK) return rs;
        make_cfg(best, s.H, s.W, s.T, sms, s.storage, out);
        std::lock_guard<std::mutex> lk(g_mu);
        g_tuned[key] = out;
        return CSLSM_OK;
    }
    make_cfg(best, s.H, s.W, s.T, sms, s.storage, out);
    std::lock_guard<std::mutex> lk(g_mu);
    g_model[key] = out;
    return CSLSM_OK;
}

}  // namespace

bool zsweep_applies(const TvSlices &s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_enable && s.gamma > 0.f && s.theta > 0.f && s.T >= 1 && s.Z > 1 && s.n0 == 0;
}

cslsm_status zsweep_reserve(ZsweepWs &ws, int H, int W)
{
    const size_t need = 4 * (size_t)H * W;
    int dev = 0;
    const int sms = sm_count(dev);
    const int tiles = 16 * sms;  // at most 16 resident CTAs per SM
    if (ws.pbuf_floats >= need && ws.max_tiles >= tiles) return CSLSM_OK;
    cudaFree(ws.pbuf);
    cudaFree(ws.flags);
    ws.pbuf = nullptr;
    ws.flags = nullptr;
    ws.err = nullptr;
    ws.pbuf_floats = 0;
    ws.max_tiles = 0;
    CSLSM_CUDA(cudaMalloc(&ws.pbuf, sizeof(float) * need));
    CSLSM_CUDA(cudaMalloc(&ws.flags, sizeof(unsigned) * (tiles + 32)));
    CSLSM_CUDA(cudaMemset(ws.flags, 0, sizeof(unsigned) * (tiles + 32)));
    ws.err = (int *)(ws.flags + tiles);
    ws.pbuf_floats = need;
    ws.max_tiles = tiles;
    ws.next_base = 0;
    return CSLSM_OK;
}

void zsweep_release(ZsweepWs &ws)
{
    cudaFree(ws.pbuf);
    cudaFree(ws.flags);
    ws = ZsweepWs{};
}

cslsm_status zsweep_run(const TvSlices &s, ZsweepWs &ws, cudaStream_t st)
{
    Cfg f;
    cslsm_status r = choose(s, ws, st, f);
    if (r != CSLSM_OK) return r;
    if (f.tx * f.ty > ws.max_tiles) {
        set_error("z-sweep workspace holds %d tiles, %d needed", ws.max_tiles, f.tx * f.ty);
        return CSLSM_ERR_UNSUPPORTED;
    }
    return launch(s, f, ws, s.u, s.d, st);
}

cslsm_status zsweep_check(ZsweepWs &ws, cudaStream_t st)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CSLSM_CUDA(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return CSLSM_OK;
    return check_err(ws, st);
}

void zsweep_config(int enable, int force, double wait_s, int stall)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_enable = enable;
    g_force = force;
    g_wait_s = wait_s;
    g_stall = stall;
}

cslsm_status zsweep_query(int H, int W, int Z, int T, int storage, int *out8)
{
    (void)Z;
    int dev = 0;
    const int sms = sm_count(dev);
    int force, cand = -1;
    Cfg f;
    bool have = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        force = g_force;
        auto it = g_tuned.find(std::make_tuple(dev, H, W, Z, T, storage));
        if (it != g_tuned.end()) {
            f = it->second;
            have = true;
        }
    }
    if (force >= 0) {
        cand = force;
        have = false;
    }
    if (!have && cand < 0) {
        double bc = 1e300;
        for (int c = 0; c < kNumCand; ++c) {
            Cfg g;
            if (!make_cfg(c, H, W, T, sms, storage, g)) continue;
            const double m = model(g, T, sms);
            if (m < bc) {
                bc = m;
                cand = c;
            }
        }
    }
    if (!have && (cand < 0 || !make_cfg(cand, H, W, T, sms, storage, f))) {
        set_error("no z-sweep tiling fits %d x %d with %d steps", H, W, T);
        return CSLSM_ERR_UNSUPPORTED;
    }
    out8[0] = f.cand;
    out8[1] = f.k;
    out8[2] = f.RPW;
    out8[3] = f.B;
    out8[4] = f.TH;
    out8[5] = f.TW;
    out8[6] = f.RH;
    out8[7] = f.tx * f.ty;
    return CSLSM_OK;
}

int zsweep_num_candidates() { return kNumCand; }

bool zsweep_forced()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return g_force >= 0;
}

}  // namespace cslsm
