// BM3D u-step (the non-local denoiser plugged into Eq. u-sub; its lambda is a
// noise level, Sec. IV-C), per 2-D slice:
//   stage 1: block matching on 8-bit codes of g, 3-D transform (8x8 DCT-II of
//            every patch, Haar along the group), hard threshold 2.7 sigma,
//            inverse, Kaiser-weighted aggregation -> basic estimate;
//   stage 2: block matching on the basic estimate, Wiener shrinkage
//            |T(B)|^2 / (|T(B)|^2 + sigma^2) applied to T(g), aggregation.
// Reference patches every 3 pixels plus the last position; 39x39 search
// window; groups of the reference plus up to 15 others by (SSD, y*W + x),
// cut to a power of two; match thresholds 64*2500 (hard) and 64*400 (Wiener)
// on the integer SSD of the 8-bit codes clamp(rint(x*255), 0, 255).
//
// GB300 design.
//  - Matching (integer ALU bound): one warp per reference.  The window's codes
//    are staged in shared memory; lane = candidate column, and each lane walks
//    the image rows once, keeping the partial sums of the 8 candidates that
//    overlap the current row in a rotating register window.  The SSD is
//    sum a^2 + sum b^2 - 2 sum ab with the cross terms from __dp4a on packed
//    bytes (exact int32).  Each lane keeps a sorted top-15 list of 32-bit keys
//    (SSD << 12 | window index, which orders like the global linear index);
//    the warp merges the 32 lists with __reduce_min_sync.  Bit-exact.
//  - Filtering (FP32): one warp per group.  Lane (k, h) holds rows 4h..4h+3 of
//    patch k; the row DCT runs in registers, then the lane pair swaps 4x4
//    blocks (shuffles) so that each lane holds 4 whole columns for the column
//    DCT, and the Haar transform is a butterfly across lanes; every DCT
//    coefficient is a compile-time constant-bank operand.
//    A CTA owns an 8x8 block of references: it stages g (and the basic
//    estimate) of the block's footprint in shared memory and aggregates the
//    block's estimates there with shared atomics before one global atomic
//    flush per footprint pixel.  Numerators and denominators accumulate in
//    FP64, so the order of the atomics changes sums only at the 1e-16 level and
//    repeated calls give the same FP32 result.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "storage.cuh"

namespace cslsm {
namespace {

constexpr int kPS = 8;          // patch size
constexpr int kHalfWin = 19;    // 39 x 39 window
constexpr int kStep = 3;        // reference step
constexpr int kMaxGroup = 16;
constexpr float kLambda3D = 2.7f;
constexpr int kTauHard = 2500, kTauWiener = 400;
constexpr int kWinPx = 2 * kHalfWin + kPS;  // 46 pixel rows / columns of a window
constexpr int kWinWords = 12;               // 48 bytes per staged row
constexpr int kMatchWarps = 8;
constexpr int kRefBlock = 8;                // references per CTA side in the filter
constexpr int kFoot = (kRefBlock - 1) * kStep + 2 * kHalfWin + kPS;  // 67
constexpr int kFootPitch = kFoot + 1;
constexpr int kFilterWarps = 8;

__constant__ float c_dct[kPS * kPS];     // C[k][n], orthonormal DCT-II
__constant__ float c_kaiser[kPS * kPS];  // separable Kaiser window, beta = 2

__host__ __device__ inline int ref_pos(int k, int n) { return min(k * kStep, n - kPS); }
__host__ __device__ inline int n_refs(int n) { return n < kPS ? 0 : (n - kPS + kStep - 1) / kStep + 1; }

// ---- g formation and 8-bit codes -----------------------------------------
// g = (rho w + gamma (u_{n-1} + u_{n+1})) / (rho + 2 gamma) for gamma > 0, else
// g = src; codes = clamp(rint(g * 255), 0, 255).
template <typename S>
__global__ void bm3d_prep_kernel(const S *__restrict__ src, const S *__restrict__ u,
                                 int Z, int n0, int ns, int HW, float rho, float gamma,
                                 float inv_rho2g, float *__restrict__ g,
                                 uint8_t *__restrict__ codes, const int *__restrict__ stop)
{
    if (stop && *stop) return;  // a tolerance-stopped solve: nothing more to do
    const long long N = (long long)ns * HW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int sl = (int)(i / HW), p = (int)(i - (long long)sl * HW);
        const int n = n0 + sl;
        float v = ld<S>(src + (size_t)n * HW + p);
        if (gamma > 0.f) {
            const float um = ld<S>(u + (size_t)((n + Z - 1) % Z) * HW + p);
            const float up = ld<S>(u + (size_t)((n + 1) % Z) * HW + p);
            v = (rho * v + gamma * (um + up)) * inv_rho2g;
        }
        if (g) g[i] = v;
        const float r = rintf(__fmul_rn(v, 255.f));
        codes[i] = (uint8_t)(r < 0.f ? 0.f : (r > 255.f ? 255.f : r));
    }
}

// ---- block matching --------------------------------------------------------
__device__ __forceinline__ void row_bytes(const uint32_t *row, int c, uint32_t &lo, uint32_t &hi)
{
    const int w = c >> 2, sh = (c & 3) * 8;
    const uint32_t a = row[w], b = row[w + 1], d = row[w + 2];
    lo = __funnelshift_r(a, b, sh);
    hi = __funnelshift_r(b, d, sh);
}

__device__ __forceinline__ void insert_key(uint32_t (&keys)[kMaxGroup - 1], uint32_t key)
{
    if (key >= keys[kMaxGroup - 2]) return;
#pragma unroll
    for (int t = 0; t < kMaxGroup - 1; ++t) {
        const uint32_t lo = min(keys[t], key);
        key = max(keys[t], key);
        keys[t] = lo;
    }
}

// Walks candidate rows [ra, rb] of window column cc (local coordinates) and
// inserts every passing candidate into the lane's list.
__device__ __forceinline__ void scan_column(const uint32_t (*win)[kWinWords], int cc, int ra,
                                            int rb, const uint32_t (&rlo)[kPS],
                                            const uint32_t (&rhi)[kPS], int refsq, int thr,
                                            int skip_l, uint32_t (&keys)[kMaxGroup - 1])
{
    uint32_t ab[kPS];
    uint32_t sq[kPS];
    uint32_t sqsum = 0;
#pragma unroll
    for (int t = 0; t < kPS; ++t) ab[t] = sq[t] = 0;
    for (int yb = ra; yb <= rb + kPS - 1; yb += kPS) {
#pragma unroll
        for (int m = 0; m < kPS; ++m) {
            const int y = yb + m;
            if (y > rb + kPS - 1) break;
            uint32_t lo, hi;
            row_bytes(win[y], cc, lo, hi);
            const uint32_t s2 = __dp4a(hi, hi, __dp4a(lo, lo, 0u));
            sqsum += s2 - sq[m];  // running sum of b^2 over the last 8 rows
            sq[m] = s2;
            ab[m] = 0;  // candidate starting at row y
#pragma unroll
            for (int a = 0; a < kPS; ++a) {
                const int k = (m - a + kPS) % kPS;  // candidate row y - a
                ab[k] = __dp4a(hi, rhi[a], __dp4a(lo, rlo[a], ab[k]));
            }
            const int ci = y - (kPS - 1);  // candidate finished at this row
            if (ci >= ra) {
                const int k = (m + 1) % kPS;
                const int ssd = refsq + (int)sqsum - 2 * (int)ab[k];
                const int l = ci * 64 + cc;
                if (ssd <= thr && l != skip_l) insert_key(keys, ((uint32_t)ssd << 12) | (uint32_t)l);
            }
        }
    }
}

__global__ void __launch_bounds__(kMatchWarps * 32)
bm3d_match_kernel(const uint8_t *__restrict__ codes, int H, int W, int ns, int thr,
                  int *__restrict__ lists, int *__restrict__ counts, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    __shared__ uint32_t s_win[kMatchWarps][kWinPx][kWinWords];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t (*win)[kWinWords] = s_win[wid];
    const int nri = n_refs(H), nrj = n_refs(W);
    const long long total = (long long)ns * nri * nrj;
    for (long long t = (long long)blockIdx.x * kMatchWarps + wid; t < total;
         t += (long long)gridDim.x * kMatchWarps) {
        const int sl = (int)(t / ((long long)nri * nrj));
        const int r = (int)(t - (long long)sl * nri * nrj);
        const int ri = ref_pos(r / nrj, H), rj = ref_pos(r % nrj, W);
        const int ci0 = max(0, ri - kHalfWin), ci1 = min(H - kPS, ri + kHalfWin);
        const int cj0 = max(0, rj - kHalfWin), cj1 = min(W - kPS, rj + kHalfWin);
        const int nrow = ci1 - ci0 + kPS, ncol = cj1 - cj0 + kPS;
        const uint8_t *img = codes + (size_t)sl * H * W;
        __syncwarp();
        for (int idx = lane; idx < nrow * kWinWords; idx += 32) {
            const int y = idx / kWinWords, wd = idx - y * kWinWords;
            uint32_t v = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int c = wd * 4 + b;
                if (c < ncol) v |= (uint32_t)img[(size_t)(ci0 + y) * W + cj0 + c] << (8 * b);
            }
            win[y][wd] = v;
        }
        __syncwarp();
        uint32_t rlo[kPS], rhi[kPS];
        int refsq = 0;
#pragma unroll
        for (int a = 0; a < kPS; ++a) {
            row_bytes(win[ri - ci0 + a], rj - cj0, rlo[a], rhi[a]);
            refsq += (int)__dp4a(rhi[a], rhi[a], __dp4a(rlo[a], rlo[a], 0u));
        }
        uint32_t keys[kMaxGroup - 1];
#pragma unroll
        for (int k = 0; k < kMaxGroup - 1; ++k) keys[k] = 0xffffffffu;
        const int ncc = cj1 - cj0 + 1, ncr = ci1 - ci0 + 1;  // candidate columns / rows
        const int skip_l = (ri - ci0) * 64 + (rj - cj0);
        if (lane < ncc) scan_column(win, lane, 0, ncr - 1, rlo, rhi, refsq, thr, skip_l, keys);
        // columns 32..38: 7 columns x 4 row segments of 10 candidate rows
        if (ncc > 32 && lane < 28) {
            const int cc = 32 + lane % 7, seg = lane / 7;
            const int ra = seg * 10, rb = min(ra + 9, ncr - 1);
            if (cc < ncc && ra <= rb) scan_column(win, cc, ra, rb, rlo, rhi, refsq, thr, skip_l, keys);
        }
        int *out = lists + (size_t)t * kMaxGroup;
        int m = 1;
        if (lane == 0) out[0] = ri * W + rj;
        for (; m < kMaxGroup; ++m) {
            const uint32_t best = __reduce_min_sync(0xffffffffu, keys[0]);
            if (best == 0xffffffffu) break;
            if (keys[0] == best) {
#pragma unroll
                for (int k = 0; k < kMaxGroup - 2; ++k) keys[k] = keys[k + 1];
                keys[kMaxGroup - 2] = 0xffffffffu;
            }
            if (lane == 0) {
                const int l = (int)(best & 0xfffu);
                out[m] = (ci0 + l / 64) * W + cj0 + l % 64;
            }
        }
        if (lane == 0) {
            for (int k = m; k < kMaxGroup; ++k) out[k] = -1;
            counts[t] = m;
        }
    }
}

// ---- collaborative filtering ----------------------------------------------
// Lane (k, h) = (lane >> 1, lane & 1) holds x[r][c] = rows 4h + r of patch k.
__device__ __forceinline__ void dct_rows(float (&x)[4][kPS], bool inverse)
{
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float y[kPS];
#pragma unroll
        for (int o = 0; o < kPS; ++o) {
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < kPS; ++c)
                s = fmaf(inverse ? c_dct[c * kPS + o] : c_dct[o * kPS + c], x[r][c], s);
            y[o] = s;
        }
#pragma unroll
        for (int o = 0; o < kPS; ++o) x[r][o] = y[o];
    }
}

// Layout change between the row layout x[r][c] (rows 4h+r, all 8 columns) and
// the column layout y[q][c] (all 8 rows, columns 4h+c) of a lane pair (h = 0,
// 1): each lane keeps its own 4x4 block and swaps the other with its partner.
// Register indices stay compile-time constants (h only drives selects).
__device__ __forceinline__ void rows_to_cols(const float (&x)[4][kPS], float (&y)[kPS][4], int h)
{
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float own = h ? x[r][4 + c] : x[r][c];
            const float give = h ? x[r][c] : x[r][4 + c];
            const float got = __shfl_xor_sync(0xffffffffu, give, 1);
            y[r][c] = h ? got : own;
            y[4 + r][c] = h ? own : got;
        }
}

__device__ __forceinline__ void cols_to_rows(const float (&y)[kPS][4], float (&x)[4][kPS], int h)
{
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float own = h ? y[4 + r][c] : y[r][c];
            const float give = h ? y[r][c] : y[4 + r][c];
            const float got = __shfl_xor_sync(0xffffffffu, give, 1);
            x[r][c] = h ? got : own;
            x[r][4 + c] = h ? own : got;
        }
}

// Column DCT in the column layout: Y[a][c] = sum_q C[a][q] X[q][c] (inverse:
// C^T).  Every coefficient index is a compile-time constant.
__device__ __forceinline__ void dct_cols(float (&y)[kPS][4], bool inverse)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float t[kPS];
#pragma unroll
        for (int a = 0; a < kPS; ++a) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < kPS; ++q)
                s = fmaf(inverse ? c_dct[q * kPS + a] : c_dct[a * kPS + q], y[q][c], s);
            t[a] = s;
        }
#pragma unroll
        for (int a = 0; a < kPS; ++a) y[a][c] = t[a];
    }
}

// Orthonormal Haar along the group (patch index k), as butterflies on pairs
// (k, k + s) with k % 2s == 0: low <- (lo + hi)/sqrt2, high <- (lo - hi)/sqrt2.
// The butterfly matrix is its own inverse; the inverse runs the levels in
// reverse order.
__device__ __forceinline__ void haar(float (&x)[kPS][4], int k, int L, bool inverse)
{
    const float r2 = 0.70710678118654752f;
    for (int lev = 0; (1 << lev) < L; ++lev) {
        const int s = inverse ? (L >> (lev + 1)) : (1 << lev);
        const bool lo = (k % (2 * s)) == 0, hi = (k % (2 * s)) == s;
#pragma unroll
        for (int r = 0; r < kPS; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float o = __shfl_xor_sync(0xffffffffu, x[r][c], 2 * s);
                if (lo) x[r][c] = (x[r][c] + o) * r2;
                else if (hi) x[r][c] = (o - x[r][c]) * r2;
            }
    }
}

struct FilterArgs {
    const float *noisy;   // [ns][H][W] g
    const float *guide;   // [ns][H][W] basic estimate (Wiener) or null
    const int *lists;     // [ns][nref][16]
    const int *counts;    // [ns][nref]
    double *num, *den;    // [ns][H][W] accumulators
    int H, W, ns;
    float sigma;
    const int *stop;      // tolerance-stopped solve: skip (or nullptr)
};

template <bool kWiener>
__global__ void __launch_bounds__(kFilterWarps * 32, 2) bm3d_filter_kernel(const FilterArgs a)
{
    if (a.stop && *a.stop) return;
    __shared__ double s_num[kFoot * kFootPitch], s_den[kFoot * kFootPitch];
    __shared__ float s_n[kFoot * kFootPitch];
    __shared__ float s_b[kWiener ? kFoot * kFootPitch : 1];
    const int H = a.H, W = a.W;
    const int nri = n_refs(H), nrj = n_refs(W);
    const int sl = blockIdx.z;
    const int bi = blockIdx.y * kRefBlock, bj = blockIdx.x * kRefBlock;
    const int ei = min(bi + kRefBlock, nri) - 1, ej = min(bj + kRefBlock, nrj) - 1;
    const int f0 = max(0, ref_pos(bi, H) - kHalfWin), f1 = min(H, ref_pos(ei, H) + kHalfWin + kPS);
    const int g0 = max(0, ref_pos(bj, W) - kHalfWin), g1 = min(W, ref_pos(ej, W) + kHalfWin + kPS);
    const int fh = f1 - f0, fw = g1 - g0;
    const size_t HW = (size_t)H * W;
    const float *noisy = a.noisy + sl * HW;
    const float *guide = kWiener ? a.guide + sl * HW : nullptr;
    for (int idx = threadIdx.x; idx < fh * fw; idx += blockDim.x) {
        const int y = idx / fw, x = idx - y * fw;
        const int l = y * kFootPitch + x;
        const size_t o = (size_t)(f0 + y) * W + g0 + x;
        s_num[l] = 0.0;
        s_den[l] = 0.0;
        s_n[l] = noisy[o];
        if (kWiener) s_b[l] = guide[o];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = lane >> 1, h = lane & 1;
    const float sigma = a.sigma, s2 = sigma * sigma, thr = kLambda3D * sigma;
    const int nblk = (ei - bi + 1) * (ej - bj + 1);
    for (int rr = wid; rr < nblk; rr += kFilterWarps) {
        const int r = (bi + rr / (ej - bj + 1)) * nrj + bj + rr % (ej - bj + 1);
        const size_t gi = (size_t)sl * nri * nrj + r;
        const int m = a.counts[gi];
        int L = 1;
        while (2 * L <= m) L *= 2;
        const bool act = k < L;
        const int lin = act ? a.lists[gi * kMaxGroup + k] : a.lists[gi * kMaxGroup];
        const int py = lin / W - f0, px = lin % W - g0;
        // Wiener: the shrinkage factors come from the guide's spectrum, taken
        // first so that only the factors (not the guide's coefficients) stay live.
        float x[4][kPS], y[kPS][4], wt[kPS][4];
        float wsum = 0.f;
        if (kWiener) {
#pragma unroll
            for (int rw = 0; rw < 4; ++rw)
#pragma unroll
                for (int c = 0; c < kPS; ++c)
                    x[rw][c] = act ? s_b[(py + 4 * h + rw) * kFootPitch + px + c] : 0.f;
            dct_rows(x, false);
            rows_to_cols(x, y, h);
            dct_cols(y, false);
            haar(y, k, L, false);
#pragma unroll
            for (int q = 0; q < kPS; ++q)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float bb = y[q][c] * y[q][c];
                    wt[q][c] = act ? bb / (bb + s2) : 0.f;
                    wsum = fmaf(wt[q][c], wt[q][c], wsum);
                }
        }
#pragma unroll
        for (int rw = 0; rw < 4; ++rw)
#pragma unroll
            for (int c = 0; c < kPS; ++c)
                x[rw][c] = act ? s_n[(py + 4 * h + rw) * kFootPitch + px + c] : 0.f;
        dct_rows(x, false);
        rows_to_cols(x, y, h);
        dct_cols(y, false);
        haar(y, k, L, false);
        if (kWiener) {
#pragma unroll
            for (int q = 0; q < kPS; ++q)
#pragma unroll
                for (int c = 0; c < 4; ++c) y[q][c] *= wt[q][c];
        } else {
#pragma unroll
            for (int q = 0; q < kPS; ++q)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const bool keep = act && fabsf(y[q][c]) > thr;
                    y[q][c] = keep ? y[q][c] : 0.f;
                    wsum += keep ? 1.f : 0.f;
                }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
        const float weight = kWiener ? (wsum > 0.f ? 1.f / (s2 * wsum) : 1.f / s2)
                                     : 1.f / (s2 * fmaxf(wsum, 1.f));
        haar(y, k, L, true);
        dct_cols(y, true);
        cols_to_rows(y, x, h);
        dct_rows(x, true);
        if (act) {
#pragma unroll
            for (int rw = 0; rw < 4; ++rw)
#pragma unroll
                for (int c = 0; c < kPS; ++c) {
                    const int l = (py + 4 * h + rw) * kFootPitch + px + c;
                    const float kw = weight * c_kaiser[(4 * h + rw) * kPS + c];
                    atomicAdd(&s_num[l], (double)(kw * x[rw][c]));
                    atomicAdd(&s_den[l], (double)kw);
                }
        }
    }
    __syncthreads();
    double *num = a.num + sl * HW, *den = a.den + sl * HW;
    for (int idx = threadIdx.x; idx < fh * fw; idx += blockDim.x) {
        const int y = idx / fw, x = idx - y * fw;
        const int l = y * kFootPitch + x;
        const double d = s_den[l];
        if (d != 0.0) {
            const size_t o = (size_t)(f0 + y) * W + g0 + x;
            atomicAdd(&num[o], s_num[l]);
            atomicAdd(&den[o], d);
        }
    }
}

// ---- WNNM (weighted nuclear norm minimisation) on the same groups ------------
//
// One warp per group of m <= 16 patches from the hard-stage block matching: lane
// pair (k, h) holds rows 4h..4h+3 of patch k, i.e. half of column k of the
// 64 x m group matrix Y.  The columns are centred on the mean patch, then
// orthogonalised by one-sided (Hestenes) Jacobi rotations: 15 rounds of 8
// disjoint column pairs per sweep (round-robin pairing), a fixed number of
// sweeps, the same (c, s) computed bit for bit by both members of a pair.
// The rotated columns are B = Yc V with norms s_k (the singular values), so the
// estimate is Xc = B diag(x_k / s_k) V^T with the weighted soft threshold
// x_k = max(s_k - sigma^2 w_k, 0), w_k = c sqrt(m) / (sigma_hat_k + eps),
// sigma_hat_k = sqrt(max(s_k^2 - 64 sigma^2, 0)); Xhat = Xc + mean.  Every
// estimated patch is aggregated with weight 1 (FP64 sums; the counts are exact).
constexpr int kJacobiSweeps = 8;
constexpr float kWnnmC = 2.8284271247461903f;  // 2 sqrt(2)

struct WnnmArgs {
    const float *noisy;  // [ns][H][W] g
    const int *lists;    // [ns][nref][16]
    const int *counts;   // [ns][nref]
    double *num, *den;   // [ns][H][W] accumulators
    int H, W, ns;
    float sigma;
    const int *stop;
};

// Partner of column k in round r of the round robin over 16 columns.
__device__ __forceinline__ int rr_partner(int k, int r)
{
    if (k == 0) return r != 0 ? r : 15;
    int q = (2 * r - k) % 15;
    if (q < 0) q += 15;
    if (q == 0) q = 15;
    return q == k ? 0 : q;
}

__global__ void __launch_bounds__(kFilterWarps * 32, 2) wnnm_filter_kernel(const WnnmArgs a)
{
    if (a.stop && *a.stop) return;
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ double s_num[kFoot * kFootPitch], s_den[kFoot * kFootPitch];
    __shared__ float s_n[kFoot * kFootPitch];
    __shared__ float s_mu[kFilterWarps][kPS * kPS];
    __shared__ float s_v[kFilterWarps][kMaxGroup][kMaxGroup + 1];  // [row l][column k]
    __shared__ float s_f[kFilterWarps][kMaxGroup];
    const int H = a.H, W = a.W;
    const int nri = n_refs(H), nrj = n_refs(W);
    const int sl = blockIdx.z;
    const int bi = blockIdx.y * kRefBlock, bj = blockIdx.x * kRefBlock;
    const int ei = min(bi + kRefBlock, nri) - 1, ej = min(bj + kRefBlock, nrj) - 1;
    const int f0 = max(0, ref_pos(bi, H) - kHalfWin), f1 = min(H, ref_pos(ei, H) + kHalfWin + kPS);
    const int g0 = max(0, ref_pos(bj, W) - kHalfWin), g1 = min(W, ref_pos(ej, W) + kHalfWin + kPS);
    const int fh = f1 - f0, fw = g1 - g0;
    const size_t HW = (size_t)H * W;
    const float *noisy = a.noisy + sl * HW;
    for (int idx = threadIdx.x; idx < fh * fw; idx += blockDim.x) {
        const int y = idx / fw, x = idx - y * fw;
        const int l = y * kFootPitch + x;
        s_num[l] = 0.0;
        s_den[l] = 0.0;
        s_n[l] = noisy[(size_t)(f0 + y) * W + g0 + x];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = lane >> 1, h = lane & 1;
    const float sigma = a.sigma, s2 = sigma * sigma;
    const int nblk = (ei - bi + 1) * (ej - bj + 1);
    for (int rr = wid; rr < nblk; rr += kFilterWarps) {
        const int r = (bi + rr / (ej - bj + 1)) * nrj + bj + rr % (ej - bj + 1);
        const size_t gi = (size_t)sl * nri * nrj + r;
        const int m = a.counts[gi];
        const bool act = k < m;
        const int lin = act ? a.lists[gi * kMaxGroup + k] : a.lists[gi * kMaxGroup];
        const int py = lin / W - f0, px = lin % W - g0;
        float x[4 * kPS];  // [rw * 8 + c]: pixel (py + 4h + rw, px + c)
#pragma unroll
        for (int rw = 0; rw < 4; ++rw)
#pragma unroll
            for (int c = 0; c < kPS; ++c)
                x[rw * kPS + c] = act ? s_n[(py + 4 * h + rw) * kFootPitch + px + c] : 0.f;
        // the mean patch over the m active columns (butterfly over lanes of this half)
        const float inv_m = 1.f / (float)m;
#pragma unroll
        for (int i = 0; i < 4 * kPS; ++i) {
            float t = x[i];
            t += __shfl_xor_sync(FULL, t, 2);
            t += __shfl_xor_sync(FULL, t, 4);
            t += __shfl_xor_sync(FULL, t, 8);
            t += __shfl_xor_sync(FULL, t, 16);
            const float mu = t * inv_m;
            if (k == 0) s_mu[wid][h * 4 * kPS + i] = mu;
            x[i] = act ? x[i] - mu : 0.f;
        }
        // V = I: lane (k, h) holds V[8h + j][k]
        float vc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) vc[j] = (8 * h + j == k) ? 1.f : 0.f;
        for (int sw = 0; sw < kJacobiSweeps; ++sw) {
            for (int rd = 0; rd < 15; ++rd) {
                const int p = rr_partner(k, rd);
                const int src = 2 * p + h;
                float own2 = 0.f, dot = 0.f;
#pragma unroll
                for (int i = 0; i < 4 * kPS; ++i) {
                    const float o = __shfl_sync(FULL, x[i], src);
                    own2 = fmaf(x[i], x[i], own2);
                    dot = fmaf(x[i], o, dot);
                }
                own2 += __shfl_xor_sync(FULL, own2, 1);
                dot += __shfl_xor_sync(FULL, dot, 1);
                const float oth2 = __shfl_sync(FULL, own2, src);
                const bool lo = k < p;
                const float alpha = lo ? own2 : oth2, beta = lo ? oth2 : own2;
                float c = 1.f, sn = 0.f;
                if (fabsf(dot) > 1e-7f * sqrtf(alpha * beta)) {
                    const float zeta = (beta - alpha) / (2.f * dot);
                    const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    c = 1.f / sqrtf(1.f + t * t);
                    sn = c * t;
                }
#pragma unroll
                for (int i = 0; i < 4 * kPS; ++i) {
                    const float o = __shfl_sync(FULL, x[i], src);
                    x[i] = lo ? c * x[i] - sn * o : sn * o + c * x[i];
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float o = __shfl_sync(FULL, vc[j], src);
                    vc[j] = lo ? c * vc[j] - sn * o : sn * o + c * vc[j];
                }
            }
        }
        // singular values and the weighted soft threshold
        float nrm2 = 0.f;
#pragma unroll
        for (int i = 0; i < 4 * kPS; ++i) nrm2 = fmaf(x[i], x[i], nrm2);
        nrm2 += __shfl_xor_sync(FULL, nrm2, 1);
        const float sk = sqrtf(nrm2);
        const float sh = sqrtf(fmaxf(nrm2 - 64.f * s2, 0.f));
        const float wk = kWnnmC * sqrtf((float)m) / (sh + 1e-8f);
        const float xk = fmaxf(sk - s2 * wk, 0.f);
        if (h == 0) s_f[wid][k] = (act && sk > 0.f) ? xk / sk : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) s_v[wid][8 * h + j][k] = vc[j];
        __syncwarp();
        // column k of Xc = sum_kk B[:, kk] f_kk V[k][kk]
        float o[4 * kPS];
#pragma unroll
        for (int i = 0; i < 4 * kPS; ++i) o[i] = 0.f;
        for (int kk = 0; kk < kMaxGroup; ++kk) {
            const float coef = s_f[wid][kk] * s_v[wid][k][kk];
#pragma unroll
            for (int i = 0; i < 4 * kPS; ++i)
                o[i] = fmaf(coef, __shfl_sync(FULL, x[i], 2 * kk + h), o[i]);
        }
        if (act) {
#pragma unroll
            for (int rw = 0; rw < 4; ++rw)
#pragma unroll
                for (int c = 0; c < kPS; ++c) {
                    const int l = (py + 4 * h + rw) * kFootPitch + px + c;
                    const float est = o[rw * kPS + c] + s_mu[wid][h * 4 * kPS + rw * kPS + c];
                    atomicAdd(&s_num[l], (double)est);
                    atomicAdd(&s_den[l], 1.0);
                }
        }
        __syncwarp();
    }
    __syncthreads();
    double *num = a.num + sl * HW, *den = a.den + sl * HW;
    for (int idx = threadIdx.x; idx < fh * fw; idx += blockDim.x) {
        const int y = idx / fw, x = idx - y * fw;
        const int l = y * kFootPitch + x;
        const double d = s_den[l];
        if (d != 0.0) {
            const size_t o = (size_t)(f0 + y) * W + g0 + x;
            atomicAdd(&num[o], s_num[l]);
            atomicAdd(&den[o], d);
        }
    }
}

// out = num / den (or out = num when den is null) and clears the
// accumulators; optionally dual = w - out (the ADMM dual update of the
// slices) and the 8-bit codes of out for the next stage's matching.
template <typename S>
__global__ void bm3d_finish_kernel(double *__restrict__ num, double *__restrict__ den,
                                   S *__restrict__ out, const S *__restrict__ w,
                                   S *__restrict__ dual, uint8_t *__restrict__ codes,
                                   long long N, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        float v;
        if (den) {
            v = (float)(num[i] / den[i]);
            num[i] = 0.0;
            den[i] = 0.0;
        } else {
            v = (float)num[i];
        }
        st<S>(out + i, v);
        if (dual) st<S>(dual + i, ld<S>(w + i) - rnd<S>(v));
        if (codes) {
            const float r = rintf(__fmul_rn(v, 255.f));
            codes[i] = (uint8_t)(r < 0.f ? 0.f : (r > 255.f ? 255.f : r));
        }
    }
}

// out = g where no patch fits (the identity), with the same epilogue.
template <typename S>
__global__ void bm3d_copy_kernel(const float *__restrict__ g, S *__restrict__ out,
                                 const S *__restrict__ w, S *__restrict__ dual, long long N,
                                 const int *__restrict__ stop)
{
    if (stop && *stop) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        st<S>(out + i, g[i]);
        if (dual) st<S>(dual + i, ld<S>(w + i) - rnd<S>(g[i]));
    }
}

std::mutex g_mu;
std::vector<int> g_ready;  // per device: constants uploaded

cslsm_status upload_constants()
{
    int dev = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_ready.size() <= dev) g_ready.resize(dev + 1, 0);
    if (g_ready[dev]) return CSLSM_OK;
    const double pi = 3.14159265358979323846;
    float C[kPS * kPS], K[kPS * kPS];
    double k1[kPS];
    auto i0 = [](double x) {  // modified Bessel I0 by its power series
        double t = 1.0, s = 1.0;
        for (int m = 1; m < 60; ++m) {
            t *= (x / 2.0) / m;
            s += t * t;
        }
        return s;
    };
    for (int k = 0; k < kPS; ++k)
        for (int n = 0; n < kPS; ++n)
            C[k * kPS + n] = (float)((k == 0 ? std::sqrt(1.0 / kPS) : std::sqrt(2.0 / kPS)) *
                                     std::cos(pi * (2 * n + 1) * k / (2.0 * kPS)));
    for (int n = 0; n < kPS; ++n) {
        const double r = 2.0 * n / (kPS - 1) - 1.0;
        k1[n] = i0(2.0 * std::sqrt(1.0 - r * r)) / i0(2.0);
    }
    for (int p = 0; p < kPS; ++p)
        for (int q = 0; q < kPS; ++q) K[p * kPS + q] = (float)(k1[p] * k1[q]);
    CSLSM_CUDA(cudaMemcpyToSymbol(c_dct, C, sizeof(C)));
    CSLSM_CUDA(cudaMemcpyToSymbol(c_kaiser, K, sizeof(K)));
    g_ready[dev] = 1;
    return CSLSM_OK;
}

inline unsigned grid_for(long long n, int threads)
{
    long long b = (n + threads - 1) / threads;
    return (unsigned)std::max(1ll, std::min(b, 16384ll));
}

// Workspace carve-up for ns slices (256-byte aligned pieces).
struct Ws {
    float *g, *basic;
    double *num, *den;
    uint8_t *codes;
    int *lists, *counts;
};

inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

Ws carve(void *base, int ns, int H, int W)
{
    const size_t HW = (size_t)H * W, nref = (size_t)n_refs(H) * n_refs(W);
    char *p = (char *)base;
    Ws w;
    w.g = (float *)p;
    p += al(ns * HW * sizeof(float));
    w.basic = (float *)p;
    p += al(ns * HW * sizeof(float));
    w.num = (double *)p;
    p += al(ns * HW * sizeof(double));
    w.den = (double *)p;
    p += al(ns * HW * sizeof(double));
    w.codes = (uint8_t *)p;
    p += al(ns * HW);
    w.lists = (int *)p;
    p += al(ns * nref * kMaxGroup * sizeof(int));
    w.counts = (int *)p;
    return w;
}

template <typename S>
cslsm_status prep(const S *src, const S *u, int Z, int n0, int ns, int HW, float rho,
                  float gamma, float *g, uint8_t *codes, cudaStream_t s,
                  const int *stop = nullptr)
{
    LaunchScope ls(K_BM3D_PREP, s);
    bm3d_prep_kernel<S><<<grid_for((long long)ns * HW, 256), 256, 0, s>>>(
        src, u, Z, n0, ns, HW, rho, gamma, 1.f / (rho + 2.f * gamma), g, codes, stop);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status match(const uint8_t *codes, int ns, int H, int W, int stage, int *lists,
                   int *counts, cudaStream_t s, const int *stop = nullptr)
{
    const long long total = (long long)ns * n_refs(H) * n_refs(W);
    if (total == 0) return CSLSM_OK;
    const int thr = kPS * kPS * (stage == 1 ? kTauHard : kTauWiener);
    LaunchScope ls(K_BM3D_MATCH, s);
    bm3d_match_kernel<<<grid_for(total, kMatchWarps), kMatchWarps * 32, 0, s>>>(
        codes, H, W, ns, thr, lists, counts, stop);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status filter(int stage, const float *noisy, const float *guide, const Ws &w, int ns,
                    int H, int W, float sigma, cudaStream_t s, const int *stop = nullptr)
{
    FilterArgs a{noisy, guide, w.lists, w.counts, w.num, w.den, H, W, ns, sigma, stop};
    const dim3 grid((n_refs(W) + kRefBlock - 1) / kRefBlock, (n_refs(H) + kRefBlock - 1) / kRefBlock,
                    ns);
    LaunchScope ls(K_BM3D_FILTER, s);
    if (stage == 1) bm3d_filter_kernel<false><<<grid, kFilterWarps * 32, 0, s>>>(a);
    else bm3d_filter_kernel<true><<<grid, kFilterWarps * 32, 0, s>>>(a);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

template <typename S>
cslsm_status finish(double *num, double *den, S *out, const S *w, S *dual, uint8_t *codes,
                    long long N, cudaStream_t s, const int *stop = nullptr)
{
    LaunchScope ls(K_BM3D_FINISH, s);
    bm3d_finish_kernel<S><<<grid_for(N, 256), 256, 0, s>>>(num, den, out, w, dual, codes, N,
                                                            stop);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

cslsm_status wnnm_filter(const float *noisy, const Ws &w, int ns, int H, int W, float sigma,
                         cudaStream_t s, const int *stop)
{
    WnnmArgs a{noisy, w.lists, w.counts, w.num, w.den, H, W, ns, sigma, stop};
    const dim3 grid((n_refs(W) + kRefBlock - 1) / kRefBlock, (n_refs(H) + kRefBlock - 1) / kRefBlock,
                    ns);
    LaunchScope ls(K_WNNM, s);
    wnnm_filter_kernel<<<grid, kFilterWarps * 32, 0, s>>>(a);
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

template <typename S>
cslsm_status wnnm_typed(const Bm3dSlices &b, void *ws, cudaStream_t s)
{
    const int H = b.H, W = b.W, ns = b.nslices;
    const size_t HW = (size_t)H * W;
    const long long N = (long long)ns * HW;
    const Ws w = carve(ws, ns, H, W);
    const float gam = b.Z > 1 ? b.gamma : 0.f;
    S *out = (S *)b.out + (size_t)b.n0 * HW;
    S *dual = b.dual ? (S *)b.dual + (size_t)b.n0 * HW : nullptr;
    const S *src = (const S *)b.src + (size_t)b.n0 * HW;
    const int *stop = b.stop;
    cslsm_status e;
    if ((e = prep<S>((const S *)b.src, (const S *)b.u, b.Z, b.n0, ns, (int)HW, b.rho, gam, w.g,
                     w.codes, s, stop)))
        return e;
    if (H < kPS || W < kPS) {  // no patch fits: the denoiser is the identity
        LaunchScope ls(K_BM3D_FINISH, s);
        bm3d_copy_kernel<S><<<grid_for(N, 256), 256, 0, s>>>(w.g, out, src, dual, N, stop);
        CSLSM_LAUNCHED();
        return CSLSM_OK;
    }
    if ((e = match(w.codes, ns, H, W, 1, w.lists, w.counts, s, stop))) return e;
    if ((e = wnnm_filter(w.g, w, ns, H, W, b.sigma, s, stop))) return e;
    return finish<S>(w.num, w.den, out, src, dual, nullptr, N, s, stop);
}

template <typename S>
cslsm_status slices_typed(const Bm3dSlices &b, void *ws, cudaStream_t s)
{
    const int H = b.H, W = b.W, ns = b.nslices;
    const size_t HW = (size_t)H * W;
    const long long N = (long long)ns * HW;
    const Ws w = carve(ws, ns, H, W);
    const float gam = b.Z > 1 ? b.gamma : 0.f;
    S *out = (S *)b.out + (size_t)b.n0 * HW;
    S *dual = b.dual ? (S *)b.dual + (size_t)b.n0 * HW : nullptr;
    const S *src = (const S *)b.src + (size_t)b.n0 * HW;
    cslsm_status e;
    const int *stop = b.stop;
    if ((e = prep<S>((const S *)b.src, (const S *)b.u, b.Z, b.n0, ns, (int)HW, b.rho, gam, w.g,
                     w.codes, s, stop)))
        return e;
    if (H < kPS || W < kPS) {  // no patch fits: the denoiser is the identity
        LaunchScope ls(K_BM3D_FINISH, s);
        bm3d_copy_kernel<S><<<grid_for(N, 256), 256, 0, s>>>(w.g, out, src, dual, N, stop);
        CSLSM_LAUNCHED();
        return CSLSM_OK;
    }
    if ((e = match(w.codes, ns, H, W, 1, w.lists, w.counts, s, stop))) return e;
    if ((e = filter(1, w.g, nullptr, w, ns, H, W, b.sigma, s, stop))) return e;
    if ((e = finish<float>(w.num, w.den, w.basic, nullptr, nullptr, w.codes, N, s, stop)))
        return e;
    if ((e = match(w.codes, ns, H, W, 2, w.lists, w.counts, s, stop))) return e;
    if ((e = filter(2, w.g, w.basic, w, ns, H, W, b.sigma, s, stop))) return e;
    return finish<S>(w.num, w.den, out, src, dual, nullptr, N, s, stop);
}

}  // namespace

int bm3d_nref(int H, int W) { return n_refs(H) * n_refs(W); }

size_t bm3d_workspace_bytes(int ns, int H, int W)
{
    const size_t HW = (size_t)H * W, nref = (size_t)n_refs(H) * n_refs(W);
    return 2 * al(ns * HW * sizeof(float)) + 2 * al(ns * HW * sizeof(double)) + al(ns * HW) +
           al(ns * nref * kMaxGroup * sizeof(int)) + al(ns * nref * sizeof(int)) + 256;
}

cslsm_status wnnm_slices(const Bm3dSlices &b, void *ws, cudaStream_t s)
{
    cslsm_status e = upload_constants();
    if (e) return e;
    if (b.storage == CSLSM_STORE_BF16) return wnnm_typed<__nv_bfloat16>(b, ws, s);
    if (b.storage == CSLSM_STORE_FP16) return wnnm_typed<__half>(b, ws, s);
    return wnnm_typed<float>(b, ws, s);
}

cslsm_status bm3d_slices(const Bm3dSlices &b, void *ws, cudaStream_t s)
{
    cslsm_status e = upload_constants();
    if (e) return e;
    if (b.storage == CSLSM_STORE_BF16) return slices_typed<__nv_bfloat16>(b, ws, s);
    if (b.storage == CSLSM_STORE_FP16) return slices_typed<__half>(b, ws, s);
    return slices_typed<float>(b, ws, s);
}

cslsm_status bm3d_stage_only(int stage, const float *noisy, const float *guide, float *out,
                             int ns, int H, int W, float sigma, void *ws, cudaStream_t s)
{
    cslsm_status e = upload_constants();
    if (e) return e;
    const Ws w = carve(ws, ns, H, W);
    const long long N = (long long)ns * H * W;
    const float *img = stage == 1 ? noisy : guide;
    if ((e = prep<float>(img, nullptr, ns, 0, ns, H * W, 1.f, 0.f, nullptr, w.codes, s)))
        return e;
    if (H < kPS || W < kPS) {
        // stage output is the noisy input unchanged
        CSLSM_CUDA(cudaMemcpyAsync(out, noisy, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
        return CSLSM_OK;
    }
    if ((e = match(w.codes, ns, H, W, stage, w.lists, w.counts, s))) return e;
    if ((e = filter(stage, noisy, guide, w, ns, H, W, sigma, s))) return e;
    return finish<float>(w.num, w.den, out, nullptr, nullptr, nullptr, N, s);
}

cslsm_status bm3d_match_only(const float *img, int ns, int H, int W, int stage, int *lists,
                             int *counts, void *ws, cudaStream_t s)
{
    const Ws w = carve(ws, ns, H, W);
    cslsm_status e = prep<float>(img, nullptr, ns, 0, ns, H * W, 1.f, 0.f, nullptr, w.codes, s);
    if (e) return e;
    return match(w.codes, ns, H, W, stage, lists, counts, s);
}

}  // namespace cslsm
