// Differentiable unrolled PnP-ADMM (relaxed DMD masks, Huber-smoothed TV with
// the z-smoothness Gauss-Seidel sweep) and its hand-written reverse pass.
//
// Forward, K iterations of Algorithm 1 on a batch of B volumes [Z][H][W]
// (one shot, R = Z), from u = d = 0:
//   m     = sigmoid(logits)                             relaxed DMD patterns
//   x-update (Eq. v-update, Woodbury with D = sum_r m_r^2):
//         g = u - d,  e = (b - sum_r m_r g_r) / (rho + D),  v_r = g_r + m_r e,
//         w = v + d
//   u-step, n = 0..Z-1 in order (Eq. u-update, newest neighbours, cyclic):
//         h_n = (rho w_n + gamma (u_{n-1} + u_{n+1})) / (rho + 2 gamma)
//         u_n = prox of theta * HuberTV_eps at h_n, theta = lambda/(rho+2gamma),
//               by T steps of projected gradient on its dual from p = 0:
//               q = div p - h/theta,  a = p + tau (grad q - kappa p),
//               p <- a / max(1, |a|),  kappa = eps / theta,
//               u_n = h - theta div p
//   d = w - u.
// The Huber function |x| - eps/2 (|x| > eps), |x|^2/(2 eps) (|x| <= eps) has the
// conjugate eps/2 |p|^2 on |p| <= 1, which is the -kappa p damping above.
// grad: forward differences, zero on the last row / column; div = -grad^T.
//
// Reverse.  The caller gives vbar = dL/dv^K.  The state (u^k, d^k) is stored
// every `ckpt_every` iterations by the forward; the reverse walks the
// segments backwards, recomputes each segment's states from its checkpoint,
// and backpropagates one iteration at a time: the dual update, the
// Gauss-Seidel sweep in reverse slice order (each prox recomputes its T dual
// iterates and runs their adjoint), the x-update.  Gradients: dL/dlogits and
// the three scalars dL/drho, dL/dlambda, dL/dgamma (FP64 accumulators).
//
// Kernels are one-thread-per-pixel passes (a block row of the grid per batch
// item); the stencils read their neighbours from global memory (L1/L2), except
// that the forward dual step forms q once per tile in shared memory and the
// reverse dual step works on shared-memory tiles.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace cslsm {
namespace {

constexpr int kT = 256;
// The three scalar gradients are accumulated in kAccCopies FP64 copies each
// (one atomic per block into copy blockIdx % kAccCopies), summed at the end:
// one address per scalar would serialise tens of thousands of atomics a launch.
constexpr int kAccCopies = 64;

// Adds the block's sum of v to acc[idx][blockIdx.x % kAccCopies].  Every thread
// of the block must call it.
__device__ __forceinline__ void block_acc(double v, double *acc, int idx)
{
    __shared__ double s_part[kT / 32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kT / 32; ++w) t += s_part[w];
        atomicAdd(acc + idx * kAccCopies + blockIdx.x % kAccCopies, t);
    }
    __syncthreads();
}

struct Geo {
    int B, Z, H, W;
    __host__ __device__ size_t HW() const { return (size_t)H * W; }
    __host__ __device__ size_t NV() const { return (size_t)Z * H * W; }  // per batch item
};

__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

// div of a dual field (components along rows p1, along columns p2) with the
// Neumann boundary of the forward differences.
__device__ __forceinline__ float divp(const float *p1, const float *p2, int i, int j, int H, int W)
{
    const size_t o = (size_t)i * W + j;
    const float a = (i < H - 1 ? p1[o] : 0.f) - (i > 0 ? p1[o - W] : 0.f);
    const float c = (j < W - 1 ? p2[o] : 0.f) - (j > 0 ? p2[o - 1] : 0.f);
    return a + c;
}

// ---- x-update ----------------------------------------------------------------
__global__ void ux_fwd_kernel(const float *__restrict__ U, const float *__restrict__ Dl,
                              const float *__restrict__ logits, const float *__restrict__ b,
                              Geo g, float rho, float *__restrict__ Wb, float *__restrict__ vout)
{
    const size_t p = blockIdx.x * (size_t)kT + threadIdx.x;
    const int bi = blockIdx.y;
    if (p >= g.HW()) return;
    const size_t base = bi * g.NV() + p, HW = g.HW();
    float s = 0.f, D = 0.f;
    for (int r = 0; r < g.Z; ++r) {
        const size_t o = base + r * HW;
        const float m = sigm(logits[o]);
        s += m * (U[o] - Dl[o]);
        D += m * m;
    }
    const float e = (b[bi * HW + p] - s) / (rho + D);
    for (int r = 0; r < g.Z; ++r) {
        const size_t o = base + r * HW;
        const float m = sigm(logits[o]);
        const float v = (U[o] - Dl[o]) + m * e;
        Wb[o] = v + Dl[o];
        if (vout) vout[o] = v;
    }
}

// Reverse of ux_fwd: given vbar (may be null) and wbar = dL/dw, accumulates
// dL/du^k into Uold_bar, writes dL/dd^k into Dbar, adds dL/dlogits into
// lbar, and dL/drho (direct) into acc[0].
__global__ void ux_bwd_kernel(const float *__restrict__ U, const float *__restrict__ Dl,
                              const float *__restrict__ logits, const float *__restrict__ b,
                              Geo g, float rho, const float *__restrict__ vbar,
                              const float *__restrict__ Wbar, float *__restrict__ Uold_bar,
                              float *__restrict__ Dbar, float *__restrict__ lbar,
                              double *__restrict__ acc)
{
    const size_t p = blockIdx.x * (size_t)kT + threadIdx.x;
    const int bi = blockIdx.y;
    double rho_bar = 0.0;
    if (p < g.HW()) {
        const size_t base = bi * g.NV() + p, HW = g.HW();
        float s = 0.f, D = 0.f, ebar = 0.f;
        for (int r = 0; r < g.Z; ++r) {
            const size_t o = base + r * HW;
            const float m = sigm(logits[o]);
            s += m * (U[o] - Dl[o]);
            D += m * m;
            const float vb = Wbar[o] + (vbar ? vbar[o] : 0.f);  // v feeds w = v + d and v^K
            ebar += m * vb;
        }
        const float den = rho + D;
        const float e = (b[bi * HW + p] - s) / den;
        const float sbar = -ebar / den;
        const float Dbarv = -ebar * e / den;
        rho_bar = (double)(-ebar * e / den);
        for (int r = 0; r < g.Z; ++r) {
            const size_t o = base + r * HW;
            const float m = sigm(logits[o]);
            const float gr = U[o] - Dl[o];
            const float vb = Wbar[o] + (vbar ? vbar[o] : 0.f);
            const float gbar = vb + sbar * m;
            const float mbar = e * vb + sbar * gr + 2.f * m * Dbarv;
            Uold_bar[o] += gbar;
            Dbar[o] = Wbar[o] - gbar;
            lbar[o] += mbar * m * (1.f - m);
        }
    }
    block_acc(rho_bar, acc, 0);
}

// ---- u-step: g formation -----------------------------------------------------
// h = (rho w_n + gamma (A + C)) / (rho + 2 gamma), A, C the neighbour slices.
__global__ void hform_kernel(const float *__restrict__ Wn, const float *A, const float *C, Geo g,
                             float rho, float gam,
                             float *__restrict__ Hb)
{
    const size_t p = blockIdx.x * (size_t)kT + threadIdx.x;
    const int bi = blockIdx.y;
    if (p >= g.HW()) return;
    const size_t o = bi * g.NV() + p;
    const float s = gam > 0.f ? A[o] + C[o] : 0.f;
    Hb[bi * g.HW() + p] = (rho * Wn[o] + gam * s) / (rho + 2.f * gam);
}

// Reverse of hform: hbar -> w_n, neighbours; direct dL/drho, dL/dgamma.
__global__ void hform_bwd_kernel(const float *__restrict__ Hbar, const float *__restrict__ Wn,
                                 const float *A, const float *C, Geo g,
                                 float rho, float gam, float *__restrict__ Wn_bar,
                                 float *A_bar, float *C_bar,  // may be the same slice (Z = 2)
                                 double *__restrict__ acc)
{
    const size_t p = blockIdx.x * (size_t)kT + threadIdx.x;
    const int bi = blockIdx.y;
    double rb = 0.0, gb = 0.0;
    if (p < g.HW()) {
        const size_t o = bi * g.NV() + p;
        const float den = rho + 2.f * gam;
        const float hb = Hbar[bi * g.HW() + p];
        const float s = gam > 0.f ? A[o] + C[o] : 0.f;
        const float h = (rho * Wn[o] + gam * s) / den;
        Wn_bar[o] += rho / den * hb;
        if (gam > 0.f) {
            A_bar[o] += gam / den * hb;
            C_bar[o] += gam / den * hb;
            gb = (double)(hb * (s - 2.f * h) / den);
        }
        rb = (double)(hb * (Wn[o] - h) / den);
    }
    block_acc(rb, acc, 0);
    block_acc(gb, acc, 1);
}

// ---- Huber-TV prox: dual projected gradient ----------------------------------
// q at (i, j) from p (both components, [bi] planes) and h.
__device__ __forceinline__ float qval(const float *p1, const float *p2, const float *h, int i,
                                      int j, int H, int W, float inv_theta)
{
    return divp(p1, p2, i, j, H, W) - h[(size_t)i * W + j] * inv_theta;
}

struct DualArgs {
    const float *P;  // [B][2][H][W] p^t
    float *Pn;       // [B][2][H][W] p^{t+1}
    const float *Hb; // [B][H][W]
    Geo g;
    float inv_theta, tau, kappa;
};

// One step p <- proj(p + tau (grad q - kappa p)) on a 2-D grid: blocks of 32
// columns x 8 rows (row chunks grid-strided), z = batch item.  q is formed once
// per pixel of the chunk, plus the row below and the column to the right that
// grad q reads, into shared memory (by qval, as everywhere, so the same bits),
// instead of three times per pixel.
__global__ void __launch_bounds__(kT) dual_fwd_kernel(const DualArgs A)
{
    constexpr int R = kT / 32;  // rows per chunk
    __shared__ float s_q[R + 1][33];
    const Geo &g = A.g;
    const int lane = (int)(threadIdx.x & 31), wr = (int)(threadIdx.x >> 5);
    const int j0 = (int)blockIdx.x * 32, j = j0 + lane;
    const int bi = blockIdx.z;
    const float *p1 = A.P + (size_t)bi * 2 * g.HW(), *p2 = p1 + g.HW();
    const float *h = A.Hb + (size_t)bi * g.HW();
    float *n1 = A.Pn + (size_t)bi * 2 * g.HW(), *n2 = n1 + g.HW();
    for (int i0 = (int)blockIdx.y * R; i0 < g.H; i0 += (int)gridDim.y * R) {
        for (int t = (int)threadIdx.x; t < (R + 1) * 33; t += kT) {
            const int r = t / 33, c = t - r * 33;
            const int qi = i0 + r, qj = j0 + c;
            if (qi < g.H && qj < g.W) s_q[r][c] = qval(p1, p2, h, qi, qj, g.H, g.W, A.inv_theta);
        }
        __syncthreads();
        const int i = i0 + wr;
        if (i < g.H && j < g.W) {
            const float qc = s_q[wr][lane];
            const float gx = i < g.H - 1 ? s_q[wr + 1][lane] - qc : 0.f;
            const float gy = j < g.W - 1 ? s_q[wr][lane + 1] - qc : 0.f;
            const size_t o = (size_t)i * g.W + j;
            const float a1 = p1[o] + A.tau * (gx - A.kappa * p1[o]);
            const float a2 = p2[o] + A.tau * (gy - A.kappa * p2[o]);
            const float sc = 1.f / fmaxf(1.f, sqrtf(a1 * a1 + a2 * a2));
            n1[o] = a1 * sc;
            n2[o] = a2 * sc;
        }
        __syncthreads();
    }
}

// u_n = h - theta div p; d_n = w_n - u_n.
__global__ void prox_out_kernel(const float *__restrict__ P, const float *__restrict__ Hb, Geo g,
                                float theta, const float *__restrict__ Wn, float *__restrict__ Un,
                                float *__restrict__ Dn)
{
    const size_t p = blockIdx.x * (size_t)kT + threadIdx.x;
    const int bi = blockIdx.y;
    if (p >= g.HW()) return;
    const int i = (int)(p / g.W), j = (int)(p % g.W);
    const float *p1 = P + (size_t)bi * 2 * g.HW(), *p2 = p1 + g.HW();
    const float u = Hb[bi * g.HW() + p] - theta * divp(p1, p2, i, j, g.H, g.W);
    const size_t o = bi * g.NV() + p;
    Un[o] = u;
    if (Dn) Dn[o] = Wn[o] - u;
}

// Reverse of prox_out: ubar -> hbar (set), pbar^T = theta grad ubar; theta
// partial -<ubar, div p^T> into acc[2].
__global__ void prox_out_bwd_kernel(const float *__restrict__ P, Geo g, float theta,
                                    const float *__restrict__ Ubar_n, float *__restrict__ Hbar,
                                    float *__restrict__ Pbar, double *__restrict__ acc)
{
    const size_t p = blockIdx.x * (size_t)kT + threadIdx.x;
    const int bi = blockIdx.y;
    double tb = 0.0;
    if (p < g.HW()) {
        const int i = (int)(p / g.W), j = (int)(p % g.W);
        const float *p1 = P + (size_t)bi * 2 * g.HW(), *p2 = p1 + g.HW();
        const float *ub = Ubar_n + (size_t)bi * g.NV();
        const float uc = ub[p];
        Hbar[bi * g.HW() + p] = uc;
        tb = (double)(-uc * divp(p1, p2, i, j, g.H, g.W));
        // d/dp of -theta <ubar, div p> = theta grad ubar (div = -grad^T)
        float *b1 = Pbar + (size_t)bi * 2 * g.HW(), *b2 = b1 + g.HW();
        b1[p] = i < g.H - 1 ? theta * (ub[p + g.W] - uc) : 0.f;
        b2[p] = j < g.W - 1 ? theta * (ub[p + 1] - uc) : 0.f;
    }
    block_acc(tb, acc, 2);
}

// Reverse of one dual step p^{t+1} = proj(a), a = p^t + tau (grad q - kappa
// p^t), q = div p^t - h / theta.  Given pbar^{t+1}:
//   abar  = J_proj(a)^T pbar^{t+1}   (J = (I - a a^T / |a|^2) / |a| if |a| > 1)
//   qbar  = tau grad^T abar = -tau div abar
//   pbar^t = (1 - tau kappa) abar - grad qbar,  hbar -= qbar / theta,
// and the theta partials: kappa = eps / theta gives -tau <abar, p^t> (-eps /
// theta^2), the h / theta term gives <qbar, h> / theta^2.
// One pass: a CTA owns a 28 x 28 tile of one batch item and keeps a 32 x 32
// region (2 pixels of halo on every side) in shared memory, one region column
// per lane and kRB rows per warp: q on the region, abar where qbar needs it,
// qbar one row / column beyond the tile, then pbar^t and hbar on the tile;
// abar never leaves the chip.  The theta partials are summed over the tile's
// own pixels only (in FP32 per thread, FP64 from the block sum on).
constexpr int kBT = 28;              // tile side
constexpr int kDR = kBT + 4;         // region side: one warp's 32 lanes
constexpr int kDP = kDR + 1;         // row pitch
static_assert(kDR == 32, "one region column per lane");

__global__ void __launch_bounds__(kT) dual_bwd_kernel(const DualArgs A,
                                                      const float *__restrict__ Pbar_next,
                                                      float *__restrict__ Pbar,
                                                      float *__restrict__ Hbar, float eps,
                                                      double *__restrict__ acc)
{
    // p^t, overwritten by abar where it is formed (each pixel reads only its own
    // p there); q, then qbar
    __shared__ float sp1[kDR][kDP], sp2[kDR][kDP], sh[kDR][kDP], sq[kDR][kDP];
    float(&sa1)[kDR][kDP] = sp1;
    float(&sa2)[kDR][kDP] = sp2;
    float(&sqb)[kDR][kDP] = sq;
    constexpr int kW = kT / 32;  // warps
    const Geo &g = A.g;
    const int H = g.H, W = g.W;
    const int tx = (W + kBT - 1) / kBT;
    const int i0 = (int)(blockIdx.x / tx) * kBT, j0 = (int)(blockIdx.x % tx) * kBT;
    const int bi = blockIdx.y;
    const int lj = (int)(threadIdx.x & 31), wr = (int)(threadIdx.x >> 5);
    const int j = j0 - 2 + lj;  // the lane's image column
    const bool cin = j >= 0 && j < W;
    const size_t HW = g.HW();
    const float *p1 = A.P + (size_t)bi * 2 * HW, *p2 = p1 + HW;
    const float *h = A.Hb + (size_t)bi * HW;
    const float *n1 = Pbar_next + (size_t)bi * 2 * HW, *n2 = n1 + HW;
    // local (li, lj) is image (i0 - 2 + li, j0 - 2 + lj); outside the image 0
    for (int li = wr; li < kDR; li += kW) {
        const int i = i0 - 2 + li;
        const bool in = cin && i >= 0 && i < H;
        const int o = in ? i * W + j : 0;  // H W < 2^31
        sp1[li][lj] = in ? p1[o] : 0.f;
        sp2[li][lj] = in ? p2[o] : 0.f;
        sh[li][lj] = in ? h[o] : 0.f;
    }
    __syncthreads();
    // q = div p - h / theta on local rows / columns 1 .. 31 (boundaries as divp)
    if (lj >= 1) {
        for (int li = 1 + wr; li < kDR; li += kW) {
            const int i = i0 - 2 + li;
            const float a = (i < H - 1 ? sp1[li][lj] : 0.f) - (i > 0 ? sp1[li - 1][lj] : 0.f);
            const float c = (j < W - 1 ? sp2[li][lj] : 0.f) - (j > 0 ? sp2[li][lj - 1] : 0.f);
            sq[li][lj] = (a + c) - sh[li][lj] * A.inv_theta;
        }
    }
    __syncthreads();
    const float theta = 1.f / A.inv_theta;
    const float kfac = -A.tau * (-eps / (theta * theta));
    const bool ctile = lj >= 2 && lj < kBT + 2 && j < W;
    float tk = 0.f, tq = 0.f;  // this thread's theta partials (tile pixels)
    // abar on local rows / columns 1 .. 30
    if (lj >= 1 && lj < kDR - 1) {
        for (int li = 1 + wr; li < kDR - 1; li += kW) {
            const int i = i0 - 2 + li;
            const float qc = sq[li][lj];
            const float gx = i < H - 1 ? sq[li + 1][lj] - qc : 0.f;
            const float gy = j < W - 1 ? sq[li][lj + 1] - qc : 0.f;
            const float pc1 = sp1[li][lj], pc2 = sp2[li][lj];
            const float a1 = pc1 + A.tau * (gx - A.kappa * pc1);
            const float a2 = pc2 + A.tau * (gy - A.kappa * pc2);
            const bool in = cin && i >= 0 && i < H;
            const int o = in ? i * W + j : 0;
            const float b1 = in ? n1[o] : 0.f, b2 = in ? n2[o] : 0.f;
            const float na = sqrtf(a1 * a1 + a2 * a2);
            float o1 = b1, o2 = b2;
            if (na > 1.f) {  // J = (I - a a^T / |a|^2) / |a|, symmetric
                const float inv = 1.f / na;
                const float dot = (a1 * b1 + a2 * b2) * inv * inv;
                o1 = (b1 - a1 * dot) * inv;
                o2 = (b2 - a2 * dot) * inv;
            }
            sa1[li][lj] = o1;
            sa2[li][lj] = o2;
            // kappa = eps / theta: d/dtheta of -tau kappa <abar, p>
            if (ctile && li >= 2 && li < kBT + 2 && i < H) tk += o1 * pc1 + o2 * pc2;
        }
    }
    __syncthreads();
    // qbar = -tau div abar on local rows / columns 2 .. 30
    if (lj >= 2 && lj < kDR - 1) {
        for (int li = 2 + wr; li < kDR - 1; li += kW) {
            const int i = i0 - 2 + li;
            const float a = (i < H - 1 ? sa1[li][lj] : 0.f) - (i > 0 ? sa1[li - 1][lj] : 0.f);
            const float c = (j < W - 1 ? sa2[li][lj] : 0.f) - (j > 0 ? sa2[li][lj - 1] : 0.f);
            sqb[li][lj] = -A.tau * (a + c);
        }
    }
    __syncthreads();
    // pbar^t = (1 - tau kappa) abar - grad qbar; hbar -= qbar / theta (tile)
    const float damp = 1.f - A.tau * A.kappa;
    float *pb1 = Pbar + (size_t)bi * 2 * HW, *pb2 = pb1 + HW;
    float *hb = Hbar + (size_t)bi * HW;
    if (ctile) {
        for (int li = 2 + wr; li < kBT + 2; li += kW) {
            const int i = i0 - 2 + li;
            if (i >= H) break;
            const int o = i * W + j;
            const float qc = sqb[li][lj];
            const float gx = i < H - 1 ? sqb[li + 1][lj] - qc : 0.f;
            const float gy = j < W - 1 ? sqb[li][lj + 1] - qc : 0.f;
            pb1[o] = damp * sa1[li][lj] - gx;
            pb2[o] = damp * sa2[li][lj] - gy;
            hb[o] -= qc * A.inv_theta;
            tq += qc * sh[li][lj];
        }
    }
    block_acc((double)tk * (double)kfac + (double)tq * ((double)A.inv_theta * A.inv_theta), acc,
              2);
}

// lbar -> dL/dlogits already includes m (1 - m); Uold_bar etc. are plain adds.
__global__ void axpy_kernel(float *__restrict__ y, const float *__restrict__ x, float a,
                            size_t n)
{
    for (size_t i = blockIdx.x * (size_t)kT + threadIdx.x; i < n; i += (size_t)gridDim.x * kT)
        y[i] += a * x[i];
}

// ---- host side ---------------------------------------------------------------
struct Ws {
    float *U, *D, *Wb, *Hb, *Pa, *Pb, *PH, *Useg, *Dseg;
    float *Ubar_new, *Ubar_old, *Wbar, *Dbar, *Hbar, *Pbar_a, *Pbar_b;
    double *acc;  // [3]: rho (direct), gamma (direct), theta (total)
    // keep_duals: the prox inputs h and dual iterates p^0..p^T of every slice of
    // a checkpoint segment, recorded by the segment's recompute:
    // Hall [S][Z][B][H][W], PHall [S][Z][T + 1][B][2][H][W]; else null
    float *Hall, *PHall;
};

inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

size_t ws_bytes(const Geo &g, int T, int S, int keep)
{
    const size_t nv = (size_t)g.B * g.NV() * 4, hw = (size_t)g.B * g.HW() * 4;
    size_t n = al(nv) * 3 + al(hw) + 2 * al(2 * hw) + al((size_t)(T + 1) * 2 * hw) +
               2 * al((size_t)(S + 1) * nv) + al(nv) * 4 + al(hw) + 2 * al(2 * hw) +
               al(3 * kAccCopies * sizeof(double));
    if (keep)
        n += al((size_t)S * g.Z * hw) + al((size_t)S * g.Z * (T + 1) * 2 * hw);
    return n;
}

Ws carve(void *base, const Geo &g, int T, int S, int keep)
{
    const size_t nv = (size_t)g.B * g.NV() * 4, hw = (size_t)g.B * g.HW() * 4;
    char *p = (char *)base;
    auto take = [&](size_t n) {
        char *r = p;
        p += al(n);
        return (float *)r;
    };
    Ws w;
    w.U = take(nv);
    w.D = take(nv);
    w.Wb = take(nv);
    w.Hb = take(hw);
    w.Pa = take(2 * hw);
    w.Pb = take(2 * hw);
    w.PH = take((size_t)(T + 1) * 2 * hw);
    w.Useg = take((size_t)(S + 1) * nv);
    w.Dseg = take((size_t)(S + 1) * nv);
    w.Ubar_new = take(nv);
    w.Ubar_old = take(nv);
    w.Wbar = take(nv);
    w.Dbar = take(nv);
    w.Hbar = take(hw);
    w.Pbar_a = take(2 * hw);
    w.Pbar_b = take(2 * hw);
    w.acc = (double *)take(3 * kAccCopies * sizeof(double));
    w.Hall = keep ? take((size_t)S * g.Z * hw) : nullptr;
    w.PHall = keep ? take((size_t)S * g.Z * (T + 1) * 2 * hw) : nullptr;
    return w;
}

struct Prm {
    float rho, lam, gam, tau, eps;
    int K, T, S;
    float theta() const { return lam / (rho + 2.f * gam); }
};

inline dim3 pgrid(const Geo &g) { return dim3((unsigned)((g.HW() + kT - 1) / kT), g.B); }
inline dim3 grid2d(const Geo &g)
{
    const int rows = (g.H + kT / 32 - 1) / (kT / 32);
    return dim3((unsigned)((g.W + 31) / 32), (unsigned)std::min(rows, 65535), g.B);
}

#define LAUNCH(kid, ...)                    \
    do {                                    \
        LaunchScope ls_((kid), s);          \
        __VA_ARGS__;                        \
        CSLSM_LAUNCHED();                   \
    } while (0)

// Neighbour slices of slice n at its Gauss-Seidel update (newest values): the
// previous slice is already new (old u_{Z-1} for n = 0), the next still old
// (new u_0 for n = Z-1).
inline void neighbours(const Geo &g, int n, float *Uold, float *Unew, float *&A, float *&C)
{
    const size_t HW = g.HW();
    A = n >= 1 ? Unew + (size_t)(n - 1) * HW : Uold + (size_t)(g.Z - 1) * HW;
    C = n < g.Z - 1 ? Uold + (size_t)(n + 1) * HW : Unew;
}

// Runs one slice's prox (recording the dual iterates into PH when given).
cslsm_status slice_prox(const Geo &g, const Prm &P, const float *Hb, float *Pa, float *Pb,
                        float *PH, float **pT, cudaStream_t s)
{
    const float theta = P.theta();
    const size_t hw2 = (size_t)g.B * 2 * g.HW();
    const int T = theta > 0.f ? P.T : 0;
    float *cur = PH ? PH : Pa;
    CSLSM_CUDA(cudaMemsetAsync(cur, 0, hw2 * sizeof(float), s));
    for (int t = 0; t < T; ++t) {
        float *nxt = PH ? PH + (size_t)(t + 1) * hw2 : (cur == Pa ? Pb : Pa);
        DualArgs A{cur, nxt, Hb, g, 1.f / theta, P.tau, P.eps / theta};
        LAUNCH(K_DIFF, dual_fwd_kernel<<<grid2d(g), kT, 0, s>>>(A));
        cur = nxt;
    }
    *pT = cur;
    return CSLSM_OK;
}

// One forward iteration on (U, D) in place; writes v when vout != null.  With
// Hrec / PHrec (keep_duals), slice n's prox input goes to Hrec + n [B][H][W]
// and its dual iterates to PHrec + n [T + 1][B][2][H][W].
cslsm_status fwd_iter(const Geo &g, const Prm &P, const float *logits, const float *b, Ws &w,
                      float *vout, cudaStream_t s, float *Hrec = nullptr, float *PHrec = nullptr)
{
    const float gam = g.Z > 1 ? P.gam : 0.f;
    LAUNCH(K_DIFF, ux_fwd_kernel<<<pgrid(g), kT, 0, s>>>(w.U, w.D, logits, b, g, P.rho, w.Wb, vout));
    const float theta = P.lam / (P.rho + 2.f * gam);
    Prm Q = P;
    Q.gam = gam;
    for (int n = 0; n < g.Z; ++n) {
        float *A, *C;
        neighbours(g, n, w.U, w.U, A, C);  // in place: the array holds the newest values
        const size_t off = (size_t)n * g.HW();
        const size_t hwf = (size_t)g.B * g.HW();
        float *Hb = Hrec ? Hrec + (size_t)n * hwf : w.Hb;
        float *PH = PHrec ? PHrec + (size_t)n * (P.T + 1) * 2 * hwf : nullptr;
        LAUNCH(K_DIFF, hform_kernel<<<pgrid(g), kT, 0, s>>>(w.Wb + off, A, C, g, P.rho, gam, Hb));
        float *pT = nullptr;
        cslsm_status e = slice_prox(g, Q, Hb, w.Pa, w.Pb, PH, &pT, s);
        if (e) return e;
        LAUNCH(K_DIFF, prox_out_kernel<<<pgrid(g), kT, 0, s>>>(pT, Hb, g, theta, w.Wb + off,
                                                                 w.U + off, w.D + off));
    }
    return CSLSM_OK;
}

}  // namespace

size_t unrolled_workspace_bytes(int B, int Z, int H, int W, int T, int S, int keep)
{
    return ws_bytes(Geo{B, Z, H, W}, T, S, keep);
}

cslsm_status unrolled_forward(int B, int Z, int H, int W, float rho, float lam, float gam,
                              int K, int T, float tau, float eps, int S, const float *logits,
                              const float *b, float *vout, float *ckpt, void *ws, cudaStream_t s)
{
    const Geo g{B, Z, H, W};
    const Prm P{rho, lam, gam, tau, eps, K, T, S};
    Ws w = carve(ws, g, T, S, 0);  // the kept duals, if any, lie beyond this part
    const size_t nv = (size_t)B * g.NV();
    CSLSM_CUDA(cudaMemsetAsync(w.U, 0, nv * 4, s));
    CSLSM_CUDA(cudaMemsetAsync(w.D, 0, nv * 4, s));
    for (int k = 0; k < K; ++k) {
        if (k % S == 0 && ckpt) {
            float *c = ckpt + (size_t)(k / S) * 2 * nv;
            CSLSM_CUDA(cudaMemcpyAsync(c, w.U, nv * 4, cudaMemcpyDeviceToDevice, s));
            CSLSM_CUDA(cudaMemcpyAsync(c + nv, w.D, nv * 4, cudaMemcpyDeviceToDevice, s));
        }
        cslsm_status e = fwd_iter(g, P, logits, b, w, k == K - 1 ? vout : nullptr, s);
        if (e) return e;
    }
    return CSLSM_OK;
}

cslsm_status unrolled_backward(int B, int Z, int H, int W, float rho, float lam, float gam,
                               int K, int T, float tau, float eps, int S, int keep,
                               const float *logits, const float *b, const float *ckpt,
                               const float *vbar, float *logits_bar, double *scal_bar, void *ws,
                               cudaStream_t s)
{
    const Geo g{B, Z, H, W};
    Prm P{rho, lam, gam, tau, eps, K, T, S};
    const float gz = Z > 1 ? gam : 0.f;
    P.gam = gz;
    Ws w = carve(ws, g, T, S, keep);
    const size_t nv = (size_t)B * g.NV(), HW = g.HW(), hw2 = (size_t)B * 2 * HW;
    const size_t hwf = (size_t)B * HW;
    const float den = rho + 2.f * gz, theta = lam / den;
    CSLSM_CUDA(cudaMemsetAsync(w.acc, 0, 3 * kAccCopies * sizeof(double), s));
    CSLSM_CUDA(cudaMemsetAsync(logits_bar, 0, nv * 4, s));
    // adjoint of the state after the last iteration: only v^K is observed
    CSLSM_CUDA(cudaMemsetAsync(w.Ubar_new, 0, nv * 4, s));
    CSLSM_CUDA(cudaMemsetAsync(w.Dbar, 0, nv * 4, s));
    const int nseg = (K + S - 1) / S;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int k0 = sg * S, k1 = std::min(K, k0 + S);
        // recompute the segment's states u^k, d^k for k = k0 .. k1
        const float *c = ckpt + (size_t)sg * 2 * nv;
        CSLSM_CUDA(cudaMemcpyAsync(w.U, c, nv * 4, cudaMemcpyDeviceToDevice, s));
        CSLSM_CUDA(cudaMemcpyAsync(w.D, c + nv, nv * 4, cudaMemcpyDeviceToDevice, s));
        for (int k = k0; k <= k1; ++k) {
            const int slot = k - k0;
            CSLSM_CUDA(cudaMemcpyAsync(w.Useg + (size_t)slot * nv, w.U, nv * 4,
                                       cudaMemcpyDeviceToDevice, s));
            CSLSM_CUDA(cudaMemcpyAsync(w.Dseg + (size_t)slot * nv, w.D, nv * 4,
                                       cudaMemcpyDeviceToDevice, s));
            if (k < k1) {
                // keep_duals: record every slice's h and dual iterates of iteration k
                cslsm_status e =
                    fwd_iter(g, P, logits, b, w, nullptr, s,
                             keep ? w.Hall + (size_t)slot * Z * hwf : nullptr,
                             keep ? w.PHall + (size_t)slot * Z * (T + 1) * hw2 : nullptr);
                if (e) return e;
            }
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const int slot = k - k0;
            float *Uo = w.Useg + (size_t)slot * nv, *Do = w.Dseg + (size_t)slot * nv;
            float *Un = w.Useg + (size_t)(slot + 1) * nv;
            // w^{k+1} from (u^k, d^k)
            LAUNCH(K_DIFF, ux_fwd_kernel<<<pgrid(g), kT, 0, s>>>(Uo, Do, logits, b, g, rho, w.Wb,
                                                                   nullptr));
            // d^{k+1} = w - u^{k+1}:  wbar = dbar, ubar_new -= dbar
            CSLSM_CUDA(cudaMemcpyAsync(w.Wbar, w.Dbar, nv * 4, cudaMemcpyDeviceToDevice, s));
            LAUNCH(K_DIFF, axpy_kernel<<<4096, kT, 0, s>>>(w.Ubar_new, w.Dbar, -1.f, nv));
            CSLSM_CUDA(cudaMemsetAsync(w.Ubar_old, 0, nv * 4, s));
            // reverse Gauss-Seidel sweep
            for (int n = Z - 1; n >= 0; --n) {
                float *A, *C;
                neighbours(g, n, Uo, Un, A, C);
                float *Ab, *Cb;
                neighbours(g, n, w.Ubar_old, w.Ubar_new, Ab, Cb);
                const size_t off = (size_t)n * HW;
                const int Tn = theta > 0.f ? T : 0;
                // the prox input h and its dual iterates p^0 .. p^T: kept by the
                // segment's recompute, or recomputed here
                float *Hn = w.Hb, *PHn = w.PH, *pT = nullptr;
                if (keep) {
                    Hn = w.Hall + ((size_t)slot * Z + n) * hwf;
                    PHn = w.PHall + ((size_t)slot * Z + n) * (T + 1) * hw2;
                    pT = PHn + (size_t)Tn * hw2;
                } else {
                    LAUNCH(K_DIFF, hform_kernel<<<pgrid(g), kT, 0, s>>>(w.Wb + off, A, C, g, rho,
                                                                        gz, w.Hb));
                    cslsm_status e = slice_prox(g, P, w.Hb, w.Pa, w.Pb, w.PH, &pT, s);
                    if (e) return e;
                }
                LAUNCH(K_DIFF, prox_out_bwd_kernel<<<pgrid(g), kT, 0, s>>>(
                                   pT, g, theta, w.Ubar_new + off, w.Hbar, w.Pbar_a, w.acc));
                float *pb_in = w.Pbar_a, *pb_out = w.Pbar_b;
                const dim3 tgrid((unsigned)(((W + kBT - 1) / kBT) * ((H + kBT - 1) / kBT)), B);
                for (int t = Tn - 1; t >= 0; --t) {
                    DualArgs Ad{PHn + (size_t)t * hw2, nullptr, Hn, g, 1.f / theta, tau,
                                eps / theta};
                    LAUNCH(K_DIFF, dual_bwd_kernel<<<tgrid, kT, 0, s>>>(Ad, pb_in, pb_out, w.Hbar,
                                                                         eps, w.acc));
                    std::swap(pb_in, pb_out);
                }
                LAUNCH(K_DIFF, hform_bwd_kernel<<<pgrid(g), kT, 0, s>>>(
                                   w.Hbar, w.Wb + off, A, C, g, rho, gz, w.Wbar + off, Ab, Cb,
                                   w.acc));
            }
            // x-update reverse: u^k, d^k adjoints
            LAUNCH(K_DIFF, ux_bwd_kernel<<<pgrid(g), kT, 0, s>>>(
                               Uo, Do, logits, b, g, rho, k == K - 1 ? vbar : nullptr, w.Wbar,
                               w.Ubar_old, w.Dbar, logits_bar, w.acc));
            std::swap(w.Ubar_new, w.Ubar_old);  // adjoint of u^k becomes the next "new"
        }
    }
    // scalars: rho_direct, gamma_direct, theta_total -> (rho, lambda, gamma)
    double copies[3 * kAccCopies], acc[3] = {0.0, 0.0, 0.0};
    CSLSM_CUDA(cudaMemcpyAsync(copies, w.acc, sizeof(copies), cudaMemcpyDeviceToHost, s));
    CSLSM_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < 3; ++q)
        for (int c = 0; c < kAccCopies; ++c) acc[q] += copies[q * kAccCopies + c];
    const double dd = (double)den;
    double out[3];
    out[1] = acc[2] / dd;                                   // dtheta/dlambda = 1/den
    out[0] = acc[0] - acc[2] * lam / (dd * dd);             // dtheta/drho = -lambda/den^2
    out[2] = (Z > 1 ? acc[1] - 2.0 * acc[2] * lam / (dd * dd) : 0.0);
    CSLSM_CUDA(cudaMemcpyAsync(scal_bar, out, sizeof(out), cudaMemcpyHostToDevice, s));
    CSLSM_CUDA(cudaStreamSynchronize(s));
    return CSLSM_OK;
}

}  // namespace cslsm
