// Batched reconstruction: many independent measurements of uneven size and
// slice count solved by Algorithm 1 (TV prior, optional z smoothness) in ONE
// persistent kernel launch, captured once in a CUDA graph and replayed.
//
// Work decomposition.  For every item (measurement) an iteration is a chain of
// phases: the x-update (Eq. v-update, units of 256 threads of 1, 2 or 4 adjacent
// pixel columns, as the alignment of H W and the caller's buffers allows), then the
// TV u-step cut into phases of at most k Chambolle steps.  A TV unit is one
// tile of one slice for one phase: it forms g on its region (the tile plus a
// halo of k + 1 pixels; with gamma > 0 from the newest u_{n-1} and the previous
// u_{n+1}, Sec. III-C; the first phase then keeps g of its own tile in the
// item's exchange buffer and the later phases load it), loads the dual field
// p that the previous phase left in the exchange buffer (p = 0 in the first
// phase), runs the steps with the dual field of every warp's rows in registers
// and g in shared memory, and stores p of its own tile for the next phase,
// or, in the last phase, u = g - theta div p and d = w - u.  With gamma > 0
// the slices follow one another in
// Gauss-Seidel order (one level per slice and phase); with gamma = 0 a level
// holds one phase of every slice.  Units of a level are independent; a level
// may start when every unit of the item's previous levels is done.  All units
// of all items and iterations are numbered in one global order: iteration-
// major, then level, then item - so every unit a unit waits for has a smaller
// number.  Many items in flight hide the exchange latency that bounds the
// single-volume sweep.
//
// Scheduling.  The grid is exactly as many CTAs as fit on the GPU at once
// (three 256-thread CTAs per SM at 80 registers a thread, so that one CTA's
// loads and barriers overlap the others' Chambolle steps; measured faster than
// two CTAs at 128 registers despite the spills).  Each CTA holds a current
// unit number and reserves the next one from a global ticket counter while it
// works (the atomic's latency hides behind the unit); a unit number is decoded by one
// lookup in a per-iteration table of (item, level, index).  Before it starts
// a unit the CTA waits until the item's completed-unit counter (read with
// acquire semantics) reaches the count the unit depends on; it increments the
// counter with release semantics after a CTA barrier.  Units are numbered so
// that every unit waited for has a smaller number, and a CTA finishes its
// current unit before it waits for its reserved one, so the smallest unfinished
// number can always proceed: the schedule cannot deadlock.  Every wait is bounded
// (a wall-clock limit read from %globaltimer); on expiry the CTA raises the
// batch's error word, every CTA stops taking units, and the host reports
// CSLSM_ERR_TIMEOUT.  Data produced inside the launch is read with L2-only
// loads (__ldcg) after an acquire fence, never from a possibly stale L1.
//
// The arithmetic per pixel is that of the per-slice tile kernel and the z
// sweep, so results are bit-identical to per-volume solves.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <vector>

#include "internal.cuh"
#include "storage.cuh"
#include "tv_body.cuh"

namespace cslsm {
namespace {

constexpr int kBW = 8, kBR = 11;     // warps per CTA, rows of the region per warp
constexpr int kBNT = kBW * 32;       // 256 threads per CTA, three CTAs per SM
constexpr int kBRH = kBW * kBR + 2;  // region rows
// a warp's row masks hold 2 bits (columns) for each of its kBR + 1 rows
static_assert(2 * (kBR + 1) <= 32, "row masks are 32-bit");
constexpr int kBPW = 64;             // region columns

struct BItem {
    void *u, *d, *w;
    const float *b;
    float *v_out;
    const uint32_t *words;
    float *pbuf;  // [2 parities][2 components][slots][H][W], slots = 1 (gamma > 0) or Z;
                  // with gamma > 0 then g [H][W] of the slice in progress
    int wstride;
    int H, W, N, R, Z;
    int hh, hc, TH, TW, tiles_x, tiles;  // row / column halo, tile rows / columns
    int units_x;
    int xvec;             // x-update pixels per thread: 1, 2 (H W even), 4 (H W % 4 == 0)
    long long units_lvl;  // TV units per level
    long long units_iter;
};

// Unit of an iteration: item (16 bits), level (16 bits), index within the
// item's level (32 bits).
__host__ __device__ inline unsigned long long pack_unit(int item, int level, int idx)
{
    return ((unsigned long long)item << 48) | ((unsigned long long)level << 32) | (unsigned)idx;
}

struct BDesc {
    const BItem *items;
    int n, iters, levels;
    const unsigned long long *unit_tab;  // [units_iter] units of one iteration, in order
    long long units_iter, total;
    unsigned long long *ticket;
    unsigned long long *done;  // [n]
    int *error;
    long long timeout_ns;
    int stall_test;
    float rho, lam, gam, tau;
    int T, k, P;  // steps per prox, steps per phase, phases per prox
};

// Completed-unit counters: read with acquire, incremented with release (gpu scope).
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Units of item it before level p of an iteration.
__device__ __forceinline__ long long level_prefix(const BItem &it, int p)
{
    return p == 0 ? 0 : it.units_x + (long long)(p - 1) * it.units_lvl;
}

template <typename S>
__device__ void xupdate_unit(const BItem &it, int unit, float rho, bool last)
{
    const int HW = it.H * it.W;
    const int pix = unit * kBNT + threadIdx.x;
    if (pix >= HW) return;
    const S *u = (const S *)it.u, *d = (const S *)it.d;
    S *w = (S *)it.w;
    for (int j = 0; j < it.N; ++j) {
        const uint32_t word = __ldcg(it.words + (size_t)j * it.wstride + pix);
        const size_t base = (size_t)j * it.R * HW + pix;
        float s = 0.f;
#pragma unroll 8
        for (int r = 0; r < it.R; ++r) {
            if ((word >> r) & 1u) {
                const size_t o = base + (size_t)r * HW;
                s += ld_l2<S>(u + o) - ld_l2<S>(d + o);
            }
        }
        const float e = (__ldcg(it.b + (size_t)j * HW + pix) - s) / (rho + (float)__popc(word));
#pragma unroll 8
        for (int r = 0; r < it.R; ++r) {
            const size_t o = base + (size_t)r * HW;
            const float dr = ld_l2<S>(d + o);
            const float g = ld_l2<S>(u + o) - dr;
            const float v = ((word >> r) & 1u) ? g + e : g;
            st<S>(w + o, keep<S>(v + dr, o, kKeyW));
            if (last) it.v_out[o] = v;
        }
    }
}

// The same x-update, two adjacent pixels per thread (H W even: the pairs are
// aligned), one access per field and plane for both; per pixel the same
// operations in the same order.
template <typename S>
__device__ void xupdate_unit2(const BItem &it, int unit, float rho, bool last)
{
    const int HW = it.H * it.W;
    const int pix = 2 * (unit * kBNT + threadIdx.x);
    if (pix >= HW) return;
    const S *u = (const S *)it.u, *d = (const S *)it.d;
    S *w = (S *)it.w;
    for (int j = 0; j < it.N; ++j) {
        const uint2 word = __ldcg(reinterpret_cast<const uint2 *>(it.words + (size_t)j * it.wstride + pix));
        const size_t base = (size_t)j * it.R * HW + pix;
        float sx = 0.f, sy = 0.f;
#pragma unroll 8
        for (int r = 0; r < it.R; ++r) {
            const size_t o = base + (size_t)r * HW;
            const float2 uu = ld2_l2<S>(u + o), dd = ld2_l2<S>(d + o);
            if ((word.x >> r) & 1u) sx += uu.x - dd.x;
            if ((word.y >> r) & 1u) sy += uu.y - dd.y;
        }
        const float2 bb = __ldcg(reinterpret_cast<const float2 *>(it.b + (size_t)j * HW + pix));
        const float ex = (bb.x - sx) / (rho + (float)__popc(word.x));
        const float ey = (bb.y - sy) / (rho + (float)__popc(word.y));
#pragma unroll 8
        for (int r = 0; r < it.R; ++r) {
            const size_t o = base + (size_t)r * HW;
            const float2 dd = ld2_l2<S>(d + o), uu = ld2_l2<S>(u + o);
            const float gx = uu.x - dd.x, gy = uu.y - dd.y;
            const float vx = ((word.x >> r) & 1u) ? gx + ex : gx;
            const float vy = ((word.y >> r) & 1u) ? gy + ey : gy;
            st2<S>(w + o, make_float2(keep<S>(vx + dd.x, o, kKeyW), keep<S>(vy + dd.y, o + 1, kKeyW)));
            if (last) *reinterpret_cast<float2 *>(it.v_out + o) = make_float2(vx, vy);
        }
    }
}

// The same x-update, four adjacent pixels per thread (H W a multiple of 4: the
// quads are aligned), one access per field and plane for all four; per pixel
// the same operations in the same order.
template <typename S>
__device__ void xupdate_unit4(const BItem &it, int unit, float rho, bool last)
{
    const int HW = it.H * it.W;
    const int pix = 4 * (unit * kBNT + threadIdx.x);
    if (pix >= HW) return;
    const S *u = (const S *)it.u, *d = (const S *)it.d;
    S *w = (S *)it.w;
    for (int j = 0; j < it.N; ++j) {
        const uint4 word = __ldcg(reinterpret_cast<const uint4 *>(it.words + (size_t)j * it.wstride + pix));
        const size_t base = (size_t)j * it.R * HW + pix;
        float4 sm = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
        for (int r = 0; r < it.R; ++r) {
            const size_t o = base + (size_t)r * HW;
            const float4 uu = ld4_l2<S>(u + o), dd = ld4_l2<S>(d + o);
            if ((word.x >> r) & 1u) sm.x += uu.x - dd.x;
            if ((word.y >> r) & 1u) sm.y += uu.y - dd.y;
            if ((word.z >> r) & 1u) sm.z += uu.z - dd.z;
            if ((word.w >> r) & 1u) sm.w += uu.w - dd.w;
        }
        const float4 bb = __ldcg(reinterpret_cast<const float4 *>(it.b + (size_t)j * HW + pix));
        const float ex = (bb.x - sm.x) / (rho + (float)__popc(word.x));
        const float ey = (bb.y - sm.y) / (rho + (float)__popc(word.y));
        const float ez = (bb.z - sm.z) / (rho + (float)__popc(word.z));
        const float ew = (bb.w - sm.w) / (rho + (float)__popc(word.w));
#pragma unroll 4
        for (int r = 0; r < it.R; ++r) {
            const size_t o = base + (size_t)r * HW;
            const float4 dd = ld4_l2<S>(d + o), uu = ld4_l2<S>(u + o);
            const float gx = uu.x - dd.x, gy = uu.y - dd.y, gz = uu.z - dd.z, gw = uu.w - dd.w;
            const float vx = ((word.x >> r) & 1u) ? gx + ex : gx;
            const float vy = ((word.y >> r) & 1u) ? gy + ey : gy;
            const float vz = ((word.z >> r) & 1u) ? gz + ez : gz;
            const float vw = ((word.w >> r) & 1u) ? gw + ew : gw;
            st4<S>(w + o, make_float4(keep<S>(vx + dd.x, o, kKeyW), keep<S>(vy + dd.y, o + 1, kKeyW),
                                      keep<S>(vz + dd.z, o + 2, kKeyW), keep<S>(vw + dd.w, o + 3, kKeyW)));
            if (last) *reinterpret_cast<float4 *>(it.v_out + o) = make_float4(vx, vy, vz, vw);
        }
    }
}

// Phase j (of D.P) of slice n's TV prox on tile `tile` of item it: g on the
// region, p from the previous phase (or 0), ns Chambolle steps with the rows
// in registers, then p of the own tile (or the final u, d) back to memory.
template <typename S>
__device__ void tv_unit(const BItem &it, const BDesc &D, int n, int j, int tile, Bnd<kBW> &sb,
                        float2 *s_g)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int B = kBW, RPW = kBR, NR = kBR + 1, RH = kBRH;
    const int H = it.H, W = it.W, hh = it.hh, hc = it.hc, TH = it.TH, TW = it.TW;
    const int bx = tile % it.tiles_x, by = tile / it.tiles_x;
    const int gi0 = by * TH - hh, gj0 = bx * TW - hc;  // gj0 even: a lane's columns pair up
    const size_t HW = (size_t)H * W;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int j0 = 2 * lane, r0 = 1 + wp * RPW, gc = gj0 + j0;
    const float mc0 = (gc >= 0 && gc < W - 1) ? 1.f : 0.f;
    const float mc1 = (gc + 1 >= 0 && gc + 1 < W - 1) ? 1.f : 0.f;
    const bool inc[2] = {gc >= 0 && gc < W, gc + 1 >= 0 && gc + 1 < W};
    const bool ownc[2] = {inc[0] && j0 >= hc && j0 < hc + TW,
                          inc[1] && j0 + 1 >= hc && j0 + 1 < hc + TW};
    const bool interior = gi0 >= 0 && gi0 + RH < H && gj0 >= 0 && gj0 + kBPW < W;
    const unsigned Hm1 = (unsigned)(H - 1);
    unsigned mr = 0;  // bit i: row i has a row below it in the image
    int off[NR];
    unsigned inm = 0, ownm = 0, pairm = 0;  // pairm: both columns in, pair aligned
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int gi = gi0 + r0 + i;
        const bool inr = gi >= 0 && gi < H;
        off[i] = gi * W + gc;
        if (inr && inc[0] && inc[1] && !(off[i] & 1)) pairm |= 1u << i;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (inr && inc[c]) inm |= 1u << (2 * i + c);
            if (i < RPW && inr && ownc[c] && r0 + i >= hh && r0 + i < hh + TH)
                ownm |= 1u << (2 * i + c);
        }
        if (i < RPW && (unsigned)gi < Hm1) mr |= 1u << i;
    }
    const float gam = it.Z > 1 ? D.gam : 0.f;
    const float rho = D.rho, inv_rho2g = 1.f / (D.rho + 2.f * gam);
    const float theta = D.lam / (D.rho + 2.f * gam);
    const float inv_theta = theta > 0.f ? 1.f / theta : 0.f;
    const S *wn = (const S *)it.w + (size_t)n * HW;
    const S *um = (const S *)it.u + (size_t)((n + it.Z - 1) % it.Z) * HW;
    const S *up = (const S *)it.u + (size_t)((n + 1) % it.Z) * HW;

    float2 g[RPW], gdn;
    // with gamma > 0 and several phases, phase 0 stores g of its own tile and the
    // later phases load it (the same FP32 values) instead of forming it again
    const int Zp = gam > 0.f ? 1 : it.Z, slot = gam > 0.f ? 0 : n;
    const bool gkeep = gam > 0.f && D.P > 1;
    float *Gp = gkeep ? it.pbuf + (size_t)4 * Zp * HW : nullptr;
    if (gkeep && j > 0) {
        float gv[2 * NR];
        if (pairm == (1u << NR) - 1) {
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const float2 v2 = __ldcg(reinterpret_cast<const float2 *>(Gp + off[i]));
                gv[2 * i] = v2.x;
                gv[2 * i + 1] = v2.y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2 * NR; ++q)
                gv[q] = (inm & (1u << q)) ? __ldcg(Gp + off[q >> 1] + (q & 1)) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) g[i] = make_float2(gv[2 * i], gv[2 * i + 1]);
        gdn = make_float2(gv[2 * RPW], gv[2 * RPW + 1]);
    } else {
        float gv[2 * NR];
        if (pairm == (1u << NR) - 1) {  // every row: one load per field for both columns
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const size_t o = (size_t)off[i];
                const float2 w2 = ld2_l2<S>(wn + o);
                if (gam > 0.f) {
                    const float2 a2 = ld2_l2<S>(um + o), b2 = ld2_l2<S>(up + o);
                    gv[2 * i] = (rho * w2.x + gam * (a2.x + b2.x)) * inv_rho2g;
                    gv[2 * i + 1] = (rho * w2.y + gam * (a2.y + b2.y)) * inv_rho2g;
                } else {
                    gv[2 * i] = w2.x;
                    gv[2 * i + 1] = w2.y;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2 * NR; ++q) {
                gv[q] = 0.f;
                if (inm & (1u << q)) {
                    const size_t o = (size_t)(off[q >> 1] + (q & 1));
                    const float wv = ld_l2<S>(wn + o);
                    gv[q] = gam > 0.f
                                ? (rho * wv + gam * (ld_l2<S>(um + o) + ld_l2<S>(up + o))) * inv_rho2g
                                : wv;
                }
            }
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) g[i] = make_float2(gv[2 * i], gv[2 * i + 1]);
        gdn = make_float2(gv[2 * RPW], gv[2 * RPW + 1]);
        if (gkeep) {
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                if (ownm & (1u << (2 * i))) Gp[off[i]] = g[i].x;
                if (ownm & (1u << (2 * i + 1))) Gp[off[i] + 1] = g[i].y;
            }
        }
    }
    float2 *sgw = s_g + wp * RPW * 32;
    float2 p1[RPW], p2[RPW];
    float2 f1 = make_float2(0.f, 0.f), f2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
        p1[i] = make_float2(0.f, 0.f);
        p2[i] = make_float2(0.f, 0.f);
    }
    if (j > 0) {
        const float *P1 = it.pbuf + ((size_t)((j - 1) & 1) * 2 * Zp + slot) * HW;
        const float *P2 = P1 + (size_t)Zp * HW;
        if (pairm == (1u << NR) - 1) {
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                p1[i] = __ldcg(reinterpret_cast<const float2 *>(P1 + off[i]));
                p2[i] = __ldcg(reinterpret_cast<const float2 *>(P2 + off[i]));
            }
        } else {
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            if (inm & (1u << (2 * i))) {
                p1[i].x = __ldcg(P1 + off[i]);
                p2[i].x = __ldcg(P2 + off[i]);
            }
            if (inm & (1u << (2 * i + 1))) {
                p1[i].y = __ldcg(P1 + off[i] + 1);
                p2[i].y = __ldcg(P2 + off[i] + 1);
            }
        }
        }
        if (wp == 0 || wp == B - 1) {  // frozen rows 0 and RH - 1 of the region
            const int gi = gi0 + (wp == 0 ? 0 : RH - 1);
            if (gi >= 0 && gi < H) {
                const size_t o = (size_t)gi * W + gc;
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
    }
    // g of the warp's rows stays in shared memory over the steps (registers go
    // to the dual field); each warp reads only its own rows.  Stored after the p
    // loads are issued, so that both loads are in flight together.
#pragma unroll
    for (int i = 0; i < RPW; ++i) sgw[i * 32 + lane] = g[i];
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
    __syncthreads();
    const int ns = min(D.k, D.T - j * D.k);
    // rows exact after the phase: the own tile, and the row above it for u_n
    const int lo = hh - (j == D.P - 1 ? 1 : 0), hi = hh + TH;
    const float2 *sgr = sgw;
    if (interior)
        sweep_steps<true, B, RPW, true>(sb, p1, p2, sgr, gdn, mr, mc0, mc1, inv_theta, D.tau, ns, wp,
                                  lane, lo, hi);
    else
        sweep_steps<false, B, RPW, true>(sb, p1, p2, sgr, gdn, mr, mc0, mc1, inv_theta, D.tau, ns, wp,
                                   lane, lo, hi);
    // Every row pairs up (pairm full) only when W is even, so every plane and
    // buffer offset is even and a lane's two columns take one aligned access.
    // The column halo and the tile width are even, so the two columns are then
    // owned together: bit 2i of ownm stands for both.
    const bool pairs = pairm == (1u << NR) - 1;
    if (j < D.P - 1) {  // p of the own tile for the next phase
        float *Q1 = it.pbuf + ((size_t)(j & 1) * 2 * Zp + slot) * HW;
        float *Q2 = Q1 + (size_t)Zp * HW;
        if (pairs) {
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                if (ownm & (1u << (2 * i))) {
                    *reinterpret_cast<float2 *>(Q1 + off[i]) = p1[i];
                    *reinterpret_cast<float2 *>(Q2 + off[i]) = p2[i];
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < RPW; ++i) {
                if (ownm & (1u << (2 * i))) {
                    Q1[off[i]] = p1[i].x;
                    Q2[off[i]] = p2[i].x;
                }
                if (ownm & (1u << (2 * i + 1))) {
                    Q1[off[i] + 1] = p1[i].y;
                    Q2[off[i] + 1] = p2[i].y;
                }
            }
        }
    } else {  // u_n = g - theta div p^T and d_n = w_n - u_n on the own tile
        S *un = (S *)it.u + (size_t)n * HW;
        S *dn = (S *)it.d + (size_t)n * HW;
        const float2 pu0 = sb.up[ns & 1][wp][lane];
        float wv[RPW][2];
#pragma unroll
        for (int i = 0; i < RPW; ++i)
#pragma unroll
            for (int c = 0; c < 2; ++c)
                wv[i][c] =
                    (ownm & (1u << (2 * i + c))) ? ld_l2<S>(wn + (size_t)off[i] + c) : 0.f;
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const float p2l = __shfl_up_sync(FULL, p2[i].y, 1);
            const float2 pu = i == 0 ? pu0 : p1[i - 1];
            const float dx = (p1[i].x - pu.x) + (p2[i].x - p2l);
            const float dy = (p1[i].y - pu.y) + (p2[i].y - p2[i].x);
            const float2 gi = sgw[i * 32 + lane];
            const float uu[2] = {gi.x - theta * dx, gi.y - theta * dy};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (!(ownm & (1u << (2 * i + c)))) continue;
                const size_t o = (size_t)off[i] + c;
                const size_t vi = (size_t)n * HW + o;
                const float ur = keep<S>(uu[c], vi, kKeyU);
                st<S>(un + o, ur);
                st<S>(dn + o, keep<S>(wv[i][c] - ur, vi, kKeyD));
            }
        }
    }
}

template <typename S>
__global__ void __launch_bounds__(kBNT, 3) batch_persistent_kernel(const BDesc *__restrict__ dp)
{
    __shared__ Bnd<kBW> sb;
    __shared__ float2 s_g[kBW * kBR * 32];  // g of each warp's rows during a TV unit
    __shared__ long long s_t;
    __shared__ int s_abort;
    const BDesc D = *dp;
    const bool zsweep = D.gam > 0.f;
    unsigned long long next = 0;  // thread 0: the reserved unit number
    if (threadIdx.x == 0) next = atomicAdd(D.ticket, 1ull);
    for (;;) {
        if (threadIdx.x == 0) {
            s_abort = *(volatile int *)D.error;
            s_t = s_abort ? D.total : (long long)next;
        }
        __syncthreads();
        const long long t = s_t;
        if (t >= D.total) break;
        // reserve the following unit now; the value is read after this unit
        if (threadIdx.x == 0) next = atomicAdd(D.ticket, 1ull);
        const int k = (int)(t / D.units_iter);
        const unsigned long long ent = __ldg(D.unit_tab + (t - (long long)k * D.units_iter));
        const int i = (int)(ent >> 48), p = (int)((ent >> 32) & 0xffffu);
        const int unit = (int)(ent & 0xffffffffu);
        const BItem &it = D.items[i];
        // wait for the item's previous levels (and iteration)
        if (threadIdx.x == 0) {
            const unsigned long long need =
                D.stall_test ? ~0ull
                             : (unsigned long long)((long long)k * it.units_iter +
                                                    level_prefix(it, p));
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u64(D.done + i) < need) {
                if (*(volatile int *)D.error) {
                    s_abort = 1;
                    break;
                }
                if ((long long)(global_ns() - t0) > D.timeout_ns) {
                    atomicExch(D.error, 1);
                    s_abort = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        __syncthreads();
        if (s_abort) break;
        if (p == 0) {
            if (it.xvec == 4) xupdate_unit4<S>(it, unit, D.rho, k == D.iters - 1);
            else if (it.xvec == 2) xupdate_unit2<S>(it, unit, D.rho, k == D.iters - 1);
            else xupdate_unit<S>(it, unit, D.rho, k == D.iters - 1);
        } else {
            // level p: slice n, phase j (gamma > 0), or phase j of every slice
            const int q = p - 1;
            int n, j, tile;
            if (zsweep && it.Z > 1) {
                n = q / D.P;
                j = q - n * D.P;
                tile = unit;
            } else {
                j = q;
                n = unit / it.tiles;
                tile = unit - n * it.tiles;
            }
            tv_unit<S>(it, D, n, j, tile, sb, s_g);
        }
        // the barrier orders every thread's stores before thread 0's release
        // add; a unit that acquires the count sees them
        __syncthreads();
        if (threadIdx.x == 0) red_release_add_u64(D.done + i, 1ull);
    }
}

template <typename S>
cslsm_status launch_persistent(const BDesc *dp, int grid, cudaStream_t s)
{
    LaunchScope ls(K_BATCH, s);
    batch_persistent_kernel<S><<<grid, kBNT, 0, s>>>(dp);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

template <typename S>
cslsm_status occupancy(int &per_sm)
{
    CSLSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<S>,
                                                             kBNT, 0));
    return CSLSM_OK;
}

}  // namespace

cslsm_status batch_build(const BatchSpec &spec, BatchRun &run)
{
    const int n = (int)spec.items.size();
    const bool zs = spec.gamma > 0.f;
    const int T = spec.lam > 0.f ? spec.T : 0;
    const int k = T > 0 ? std::max(1, std::min(spec.k, T)) : 0;
    const int P = T > 0 ? (T + k - 1) / k : 1;
    const int hh = k + 1;
    if (kBRH - 2 * hh < 1 || kBPW - 2 * (hh + (hh & 1)) < 2) {
        set_error("batched TV: %d steps per phase leave no tile", k);
        return CSLSM_ERR_UNSUPPORTED;
    }
    std::vector<BItem> items(n);
    int levels = 1;
    size_t pbytes = 0;
    std::vector<size_t> poff(n);
    for (int i = 0; i < n; ++i) {
        const BatchItemSpec &s = spec.items[i];
        BItem &b = items[i];
        b.u = s.u;
        b.d = s.d;
        b.w = s.w;
        b.b = s.b;
        b.v_out = s.v_out;
        b.words = s.words;
        b.wstride = s.wstride;
        b.H = s.H;
        b.W = s.W;
        b.N = s.N;
        b.R = s.R;
        b.Z = s.N * s.R;
        b.hh = hh;
        b.hc = hh + (hh & 1);  // even column halo: regions start on even columns
        b.TH = kBRH - 2 * hh;
        b.TW = kBPW - 2 * b.hc;
        b.tiles_x = (s.W + b.TW - 1) / b.TW;
        b.tiles = b.tiles_x * ((s.H + b.TH - 1) / b.TH);
        // pairs need H W even and the caller's b and v_out 8-byte aligned (the
        // plan's buffers are)
        {
            const int hw = s.H * s.W;
            const uintptr_t bv = (uintptr_t)s.b | (uintptr_t)s.v_out;
            b.xvec = hw % 4 == 0 && bv % 16 == 0 ? 4 : hw % 2 == 0 && bv % 8 == 0 ? 2 : 1;
            b.units_x = (hw / b.xvec + kBNT - 1) / kBNT;
        }
        const bool chain = zs && b.Z > 1;  // Gauss-Seidel: one level per slice and phase
        b.units_lvl = chain ? b.tiles : (long long)b.tiles * b.Z;
        const int lv = chain ? b.Z * P : P;
        b.units_iter = b.units_x + b.units_lvl * lv;
        levels = std::max(levels, 1 + lv);
        poff[i] = pbytes;
        // p: 2 parities x 2 components x slots planes; with gamma > 0 one more plane for g
        const size_t planes = 4 * (size_t)(chain ? 1 : b.Z) + (chain ? 1 : 0);
        if (P > 1) pbytes += (planes * s.H * s.W * sizeof(float) + 255) & ~size_t(255);
    }
    // the units of one iteration in order: level-major, then item, then index
    std::vector<unsigned long long> tab;
    for (int p = 0; p < levels; ++p)
        for (int i = 0; i < n; ++i) {
            const BItem &b = items[i];
            const long long lv = (b.units_iter - b.units_x) / b.units_lvl;
            const long long c = p == 0 ? b.units_x : (p - 1 < lv ? b.units_lvl : 0);
            for (long long u = 0; u < c; ++u) tab.push_back(pack_unit(i, p, (int)u));
        }
    const long long units_iter = (long long)tab.size();
    // one device allocation for descriptors, tables, counters and the items'
    // dual-field exchange buffers
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t sz_items = al(sizeof(BItem) * n), sz_tab = al(sizeof(unsigned long long) * tab.size()),
                 sz_cnt = al(8 * (n + 1)), sz_err = 256, sz_desc = al(sizeof(BDesc));
    const size_t total = sz_items + sz_tab + sz_cnt + sz_err + sz_desc + pbytes;
    char *base = nullptr;
    CSLSM_CUDA(cudaMalloc(&base, total));
    run.mem = base;
    char *q = base;
    BItem *d_items = (BItem *)q;
    q += sz_items;
    unsigned long long *d_tab = (unsigned long long *)q;
    q += sz_tab;
    unsigned long long *d_cnt = (unsigned long long *)q;  // [0] ticket, [1..n] done
    q += sz_cnt;
    int *d_err = (int *)q;
    q += sz_err;
    BDesc *d_desc = (BDesc *)q;
    q += sz_desc;
    for (int i = 0; i < n; ++i) items[i].pbuf = P > 1 ? (float *)(q + poff[i]) : nullptr;
    BDesc D{};
    D.items = d_items;
    D.n = n;
    D.iters = spec.iters;
    D.levels = levels;
    D.unit_tab = d_tab;
    D.units_iter = units_iter;
    D.total = units_iter * spec.iters;
    D.ticket = d_cnt;
    D.done = d_cnt + 1;
    D.error = d_err;
    D.timeout_ns = (long long)(spec.wait_limit_s * 1e9);
    D.stall_test = spec.stall_test;
    D.rho = spec.rho;
    D.lam = spec.lam;
    D.gam = spec.gamma;
    D.tau = spec.tau;
    D.T = T;
    D.k = k;
    D.P = P;
    CSLSM_CUDA(cudaMemcpy(d_items, items.data(), sizeof(BItem) * n, cudaMemcpyHostToDevice));
    CSLSM_CUDA(cudaMemcpy(d_tab, tab.data(), sizeof(unsigned long long) * tab.size(),
                          cudaMemcpyHostToDevice));
    CSLSM_CUDA(cudaMemcpy(d_desc, &D, sizeof(BDesc), cudaMemcpyHostToDevice));
    run.desc = d_desc;
    run.counters = d_cnt;
    run.counters_bytes = 8 * (n + 1);
    run.error = d_err;
    run.smem = 0;
    int per_sm = 0, dev = 0, sms = 0;
    cslsm_status e;
    if (spec.storage == CSLSM_STORE_BF16) e = occupancy<__nv_bfloat16>(per_sm);
    else if (spec.storage == CSLSM_STORE_FP16) e = occupancy<__half>(per_sm);
    else e = occupancy<float>(per_sm);
    if (e) return e;
    CSLSM_CUDA(cudaGetDevice(&dev));
    CSLSM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) {
        set_error("persistent batch kernel does not fit on an SM");
        return CSLSM_ERR_UNSUPPORTED;
    }
    run.grid = per_sm * sms;
    run.storage = spec.storage;
    run.k = k;
    run.units_iter = units_iter;
    return CSLSM_OK;
}

cslsm_status batch_set_io(const BatchRun &run, int item, const float *b, float *v_out,
                          cudaStream_t s)
{
    // the item's measurement and output pointers in the device copy of its
    // descriptor, ordered on `s` before the next launch (host values are staged
    // by the copy, so the locals may go out of scope)
    BItem *d_items = reinterpret_cast<BItem *>(run.mem);
    const float *bp = b;
    float *vp = v_out;
    CSLSM_CUDA(cudaMemcpyAsync(&d_items[item].b, &bp, sizeof(bp), cudaMemcpyHostToDevice, s));
    CSLSM_CUDA(cudaMemcpyAsync(&d_items[item].v_out, &vp, sizeof(vp), cudaMemcpyHostToDevice, s));
    return CSLSM_OK;
}

long long batch_tiles_per_slice(int H, int W, int k)
{
    const int hh = k + 1, hc = hh + (hh & 1);
    const int TH = kBRH - 2 * hh, TW = kBPW - 2 * hc;
    if (TH < 1 || TW < 2) return 0;
    return (long long)((W + TW - 1) / TW) * ((H + TH - 1) / TH);
}

int batch_max_steps_per_phase()
{
    int k = 1;
    for (;;) {
        const int hh = k + 2;  // the halo k + 1 steps would need
        if (kBRH - 2 * hh < 1 || kBPW - 2 * (hh + (hh & 1)) < 2) return k;
        ++k;
    }
}

cslsm_status batch_set_wait(const BatchRun &run, double limit_s, int stall_test)
{
    BDesc D{};
    CSLSM_CUDA(cudaMemcpy(&D, run.desc, sizeof(BDesc), cudaMemcpyDeviceToHost));
    D.timeout_ns = (long long)(limit_s * 1e9);
    D.stall_test = stall_test;
    CSLSM_CUDA(cudaMemcpy(run.desc, &D, sizeof(BDesc), cudaMemcpyHostToDevice));
    return CSLSM_OK;
}

cslsm_status batch_enqueue(const BatchRun &run, cudaStream_t s)
{
    CSLSM_CUDA(cudaMemsetAsync(run.counters, 0, run.counters_bytes, s));
    CSLSM_CUDA(cudaMemsetAsync(run.error, 0, sizeof(int), s));
    const BDesc *dp = (const BDesc *)run.desc;
    if (run.storage == CSLSM_STORE_BF16) return launch_persistent<__nv_bfloat16>(dp, run.grid, s);
    if (run.storage == CSLSM_STORE_FP16) return launch_persistent<__half>(dp, run.grid, s);
    return launch_persistent<float>(dp, run.grid, s);
}

}  // namespace cslsm
