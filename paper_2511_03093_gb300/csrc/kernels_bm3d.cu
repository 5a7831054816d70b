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

// ---- collaborative filtering on the tensor cores ------------------------------
// One warp per group of L <= 16 patches (L a power of two).  With G the L x 64
// group matrix (row k = patch k, column p = 8 r + q = pixel (r, q)) and
// T = C (x) C the 64 x 64 matrix of the separable 8 x 8 DCT-II
// (T[8u + v][8r + q] = C[u][r] C[v][q]), the group transform and its inverse
// are four small dense products:
//   forward   Y^T = T G^T                      (64 coefficients x 16 patches)
//             Z^T = Y^T H_un^T, z = Z^T diag(s) (Haar along the group, written
//                   H = diag(s) H_un with H_un in {0, +-1} and s_j = 1/sqrt(support))
//   shrink    hard threshold or Wiener factors, elementwise in FP32 registers
//   inverse   Y'^T = (z' diag(s)) H_un,  G' = Y' T.
// Each product runs as mma.sync m16n8k16 (FP16 operands, FP32 accumulation).
// An FP32 operand x is carried as hi + lo, two FP16 values (22 significant
// bits), and a product as hi*hi + hi*lo + lo*hi (the dropped lo*lo term is
// about 2^-22 relative).  Before the split the group is scaled by a power of
// two (max |x| in [1, 2)) and T by 2^8, so that no FP16 value overflows and
// the lo parts of the constants stay normal; the scalings are exact and are
// undone exactly.
// Fragment layouts (thread (g, t) = (lane / 4, lane % 4)):
//   A 16 x 16: {A[g][2t], A[g][2t+1]}, {A[g+8][2t], ..}, {A[g][2t+8], ..}, {A[g+8][2t+8], ..}
//   B 16 x 8:  {B[2t][g], B[2t+1][g]}, {B[2t+8][g], B[2t+9][g]}
//   C 16 x 8:  C[g][2t], C[g][2t+1], C[g+8][2t], C[g+8][2t+1]
// so the accumulators of two adjacent n-tiles, packed in pairs, are the A
// fragment of the next product (Y^T -> Haar -> inverse Haar); the one
// transpose (Y'^T -> Y') is movmatrix on the packed FP16 halves.
// Aggregation: the numerator goes to FP64 global atomics (reductions in L2,
// no shared-memory compare-and-swap); the denominator is the weight image A
// (group weight added at every patch position, 16 atomics per group) whose
// correlation with the Kaiser window the finish kernel takes.
constexpr int kTcWarps = 8;

struct TcTables {
    uint4 fwd[4 * 4 * 2][32];  // [mt][kt][hi, lo]: A fragments of 2^8 T (M = coefficient, K = pixel)
    uint4 inv[4 * 4 * 2][32];  // [kc][np / 2][hi, lo]: B fragments of 2^8 T (K = coefficient,
                               // N = pixel), two n-tiles per entry
    uint4 haar[5 * 2][32];     // [log2 L][forward, inverse]: B fragments of H_un^T / H_un
    float scale[5][16];        // s_j per log2 L
};
constexpr size_t kTcSmem = sizeof(TcTables);
constexpr size_t kFootBytes = sizeof(float) * kFoot * kFootPitch;

__device__ TcTables g_tc;
__constant__ float c_k1[kPS];  // 1-D Kaiser window (K[a][b] = k1[a] k1[b])

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1)
{
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// x0 + x1 * 2^16-lane packing: hi = fp16 pair of (x0, x1), lo = fp16 pair of
// the remainders (x - hi is exact in FP32).
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

__device__ __forceinline__ uint32_t movm_trans(uint32_t x)
{
    uint32_t y;
    asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

__device__ __forceinline__ void red_add_f64(double *p, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// Power-of-two scale 2^e with max|x| 2^e in [1, 2) (1 for an all-zero group);
// e limited to [-100, 100] so that 2^e and 2^-(e+8) stay normal.
__device__ __forceinline__ int group_exponent(float mx_abs)
{
    const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(mx_abs));
    if (b == 0u) return 0;
    const int E = (int)((b >> 23) & 255u) - 126;  // mx = f 2^E, f in [0.5, 1)
    return max(-100, min(100, 1 - E));
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Loads the 16 x 64 group of patches at the lane's two positions from the
// staged footprint: x[nt][kt][0..3] = pixels (2kt, 2t), (2kt, 2t+1),
// (2kt+1, 2t), (2kt+1, 2t+1) of patch 8 nt + g (zero for inactive patches).
__device__ __forceinline__ void load_group(const float *img, const int (&off)[2],
                                           const bool (&act)[2], int t, float (&x)[2][4][4])
{
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            const float *p = img + off[nt] + 2 * kt * kFootPitch + 2 * t;
            x[nt][kt][0] = act[nt] ? p[0] : 0.f;
            x[nt][kt][1] = act[nt] ? p[1] : 0.f;
            x[nt][kt][2] = act[nt] ? p[kFootPitch] : 0.f;
            x[nt][kt][3] = act[nt] ? p[kFootPitch + 1] : 0.f;
        }
}

// Forward transform of a loaded group: z[mt][nj][c] = 2^e times the 3-D
// transform coefficient (coefficient 16 mt + g (+8 for c >= 2), group index
// 8 nj + 2t + (c & 1)).
__device__ __forceinline__ void forward_3d(const TcTables &tb, float (&x)[2][4][4], int lgL,
                                           int lane, float sc, float (&z)[4][2][4])
{
    float acc[4][2][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[mt][nt][c] = 0.f;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            split2(x[nt][kt][0] * sc, x[nt][kt][1] * sc, bh[nt][0], bl[nt][0]);
            split2(x[nt][kt][2] * sc, x[nt][kt][3] * sc, bh[nt][1], bl[nt][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const uint4 ah = tb.fwd[(mt * 4 + kt) * 2][lane];
            const uint4 al = tb.fwd[(mt * 4 + kt) * 2 + 1][lane];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                mma16816(acc[mt][nt], al.x, al.y, al.z, al.w, bh[nt][0], bh[nt][1]);
                mma16816(acc[mt][nt], ah.x, ah.y, ah.z, ah.w, bl[nt][0], bl[nt][1]);
                mma16816(acc[mt][nt], ah.x, ah.y, ah.z, ah.w, bh[nt][0], bh[nt][1]);
            }
        }
    }
    // Haar along the group: Z^T = Y^T H_un^T, then z = Z^T diag(s)
    const uint4 hf = tb.haar[lgL * 2][lane];
    const float r8 = 1.f / 256.f;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        uint32_t ah[4], al[4];
        split2(acc[mt][0][0] * r8, acc[mt][0][1] * r8, ah[0], al[0]);
        split2(acc[mt][0][2] * r8, acc[mt][0][3] * r8, ah[1], al[1]);
        split2(acc[mt][1][0] * r8, acc[mt][1][1] * r8, ah[2], al[2]);
        split2(acc[mt][1][2] * r8, acc[mt][1][3] * r8, ah[3], al[3]);
#pragma unroll
        for (int nj = 0; nj < 2; ++nj) {
#pragma unroll
            for (int c = 0; c < 4; ++c) z[mt][nj][c] = 0.f;
            const uint32_t b0 = nj ? hf.z : hf.x, b1 = nj ? hf.w : hf.y;
            mma16816(z[mt][nj], al[0], al[1], al[2], al[3], b0, b1);
            mma16816(z[mt][nj], ah[0], ah[1], ah[2], ah[3], b0, b1);
        }
    }
    const int t = lane & 3;
#pragma unroll
    for (int nj = 0; nj < 2; ++nj) {
        const float s0 = tb.scale[lgL][8 * nj + 2 * t], s1 = tb.scale[lgL][8 * nj + 2 * t + 1];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            z[mt][nj][0] *= s0;
            z[mt][nj][1] *= s1;
            z[mt][nj][2] *= s0;
            z[mt][nj][3] *= s1;
        }
    }
}

// Inverse transform of q = z' diag(s) (scaled by 2^e): o[np][c] = 2^(e+8) G'
// at patch g (c < 2) / g + 8 (c >= 2), pixel (np, 2t + (c & 1)).
__device__ __forceinline__ void inverse_3d(const TcTables &tb, const float (&q)[4][2][4],
                                           int lgL, int lane, float (&o)[8][4])
{
    const uint4 hv = tb.haar[lgL * 2 + 1][lane];
    uint32_t a4h[4][4], a4l[4][4];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        uint32_t ah[4], al[4];
        split2(q[mt][0][0], q[mt][0][1], ah[0], al[0]);
        split2(q[mt][0][2], q[mt][0][3], ah[1], al[1]);
        split2(q[mt][1][0], q[mt][1][1], ah[2], al[2]);
        split2(q[mt][1][2], q[mt][1][3], ah[3], al[3]);
        float y[2][4];
#pragma unroll
        for (int nk = 0; nk < 2; ++nk) {
#pragma unroll
            for (int c = 0; c < 4; ++c) y[nk][c] = 0.f;
            const uint32_t b0 = nk ? hv.z : hv.x, b1 = nk ? hv.w : hv.y;
            mma16816(y[nk], al[0], al[1], al[2], al[3], b0, b1);
            mma16816(y[nk], ah[0], ah[1], ah[2], ah[3], b0, b1);
        }
        // Y'^T (coefficients x patches) -> Y' (patches x coefficients): the
        // 8 x 8 block (rows 16 mt + 8 h + .., columns 8 nk + ..) transposed is
        // register 2 h + nk of the A fragment of k-tile mt.
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int nk = 0; nk < 2; ++nk) {
                uint32_t hi, lo;
                split2(y[nk][2 * h], y[nk][2 * h + 1], hi, lo);
                a4h[mt][2 * h + nk] = movm_trans(hi);
                a4l[mt][2 * h + nk] = movm_trans(lo);
            }
    }
#pragma unroll
    for (int np = 0; np < 8; ++np)
#pragma unroll
        for (int c = 0; c < 4; ++c) o[np][c] = 0.f;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
#pragma unroll
        for (int npp = 0; npp < 4; ++npp) {
            const uint4 bh = tb.inv[(kc * 4 + npp) * 2][lane];
            const uint4 bl = tb.inv[(kc * 4 + npp) * 2 + 1][lane];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int np = 2 * npp + u;
                const uint32_t h0 = u ? bh.z : bh.x, h1 = u ? bh.w : bh.y;
                const uint32_t l0 = u ? bl.z : bl.x, l1 = u ? bl.w : bl.y;
                mma16816(o[np], a4l[kc][0], a4l[kc][1], a4l[kc][2], a4l[kc][3], h0, h1);
                mma16816(o[np], a4h[kc][0], a4h[kc][1], a4h[kc][2], a4h[kc][3], l0, l1);
                mma16816(o[np], a4h[kc][0], a4h[kc][1], a4h[kc][2], a4h[kc][3], h0, h1);
            }
        }
}

struct FilterArgs {
    const float *noisy;   // [ns][H][W] g
    const float *guide;   // [ns][H][W] basic estimate (Wiener) or null
    const int *lists;     // [ns][nref][16]
    const int *counts;    // [ns][nref]
    double *num, *wimg;   // [ns][H][W] numerator and weight-image accumulators
    int H, W, ns;
    float sigma;
    const int *stop;      // tolerance-stopped solve: skip (or nullptr)
    float *stat;          // [ns][nref] per-group kept count / sum W^2, or nullptr
};

// Persistent: each CTA takes 8 x 8 blocks of references (one slice each) in
// turn, stages the block's footprint of g (and of the guide) in shared
// memory, and its warps filter the block's groups one per warp.
template <bool kWiener>
__global__ void __launch_bounds__(kTcWarps * 32, 2) bm3d_filter_tc_kernel(const FilterArgs a)
{
    if (a.stop && *a.stop) return;
    extern __shared__ __align__(16) unsigned char smem[];
    TcTables &tb = *reinterpret_cast<TcTables *>(smem);
    float *s_n = reinterpret_cast<float *>(smem + kTcSmem);
    float *s_b = s_n + kFoot * kFootPitch;
    // Wiener factors of the warp's current group, [value][lane] (kept out of
    // registers while the noisy group is transformed)
    float *s_w = s_b + kFoot * kFootPitch + (threadIdx.x >> 5) * 32 * 32 + (threadIdx.x & 31);
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(&g_tc);
        uint4 *dst = reinterpret_cast<uint4 *>(smem);
        for (int i = threadIdx.x; i < (int)(kTcSmem / 16); i += blockDim.x) dst[i] = src[i];
    }
    const int H = a.H, W = a.W;
    const int nri = n_refs(H), nrj = n_refs(W);
    const int tbx = (nrj + kRefBlock - 1) / kRefBlock, tby = (nri + kRefBlock - 1) / kRefBlock;
    const long long ntiles = (long long)tbx * tby * a.ns;
    const size_t HW = (size_t)H * W;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const float sigma = a.sigma, s2 = sigma * sigma, thr = kLambda3D * sigma;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int sl = (int)(tile / ((long long)tbx * tby));
        const int rem = (int)(tile - (long long)sl * tbx * tby);
        const int bi = (rem / tbx) * kRefBlock, bj = (rem % tbx) * kRefBlock;
        const int ei = min(bi + kRefBlock, nri) - 1, ej = min(bj + kRefBlock, nrj) - 1;
        const int f0 = max(0, ref_pos(bi, H) - kHalfWin);
        const int f1 = min(H, ref_pos(ei, H) + kHalfWin + kPS);
        const int g0 = max(0, ref_pos(bj, W) - kHalfWin);
        const int g1 = min(W, ref_pos(ej, W) + kHalfWin + kPS);
        const int fh = f1 - f0, fw = g1 - g0;
        const float *noisy = a.noisy + sl * HW;
        const float *guide = kWiener ? a.guide + sl * HW : nullptr;
        __syncthreads();  // the previous block's readers are done (and the tables are in)
        for (int idx = threadIdx.x; idx < fh * fw; idx += blockDim.x) {
            const int y = idx / fw, x = idx - y * fw;
            const size_t o = (size_t)(f0 + y) * W + g0 + x;
            s_n[y * kFootPitch + x] = noisy[o];
            if (kWiener) s_b[y * kFootPitch + x] = guide[o];
        }
        __syncthreads();
        double *num = a.num + sl * HW, *wimg = a.wimg + sl * HW;
        const int nblk = (ei - bi + 1) * (ej - bj + 1);
        for (int rr = wid; rr < nblk; rr += kTcWarps) {
            const int r = (bi + rr / (ej - bj + 1)) * nrj + bj + rr % (ej - bj + 1);
            const size_t gi = (size_t)sl * nri * nrj + r;
            const int m = a.counts[gi];
            int lgL = 0;
            while ((2 << lgL) <= m) ++lgL;
            const int L = 1 << lgL;
            int off[2], py[2], px[2];
            bool act[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = g + 8 * q;
                act[q] = k < L;
                const int lin = a.lists[gi * kMaxGroup + (act[q] ? k : 0)];
                py[q] = lin / W - f0;
                px[q] = lin % W - g0;
                off[q] = py[q] * kFootPitch + px[q];
            }
            float x[2][4][4], z[4][2][4];
            float wsum = 0.f, mx;
            int e;
            if (kWiener) {  // Wiener factors from the guide's spectrum
                load_group(s_b, off, act, t, x);
                mx = 0.f;
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                        for (int c = 0; c < 4; ++c) mx = fmaxf(mx, fabsf(x[nt][kt][c]));
                e = group_exponent(mx);
                forward_3d(tb, x, lgL, lane, pow2f(e), z);
                const float ie = pow2f(-e);
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                    for (int nj = 0; nj < 2; ++nj)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float bb = z[mt][nj][c] * ie;
                            const float b2 = bb * bb;
                            const float wv = b2 / (b2 + s2);
                            s_w[((mt * 2 + nj) * 4 + c) * 32] = wv;
                            wsum = fmaf(wv, wv, wsum);
                        }
                __syncwarp();  // keeps the two transforms apart (register pressure)
            }
            load_group(s_n, off, act, t, x);
            mx = 0.f;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                    for (int c = 0; c < 4; ++c) mx = fmaxf(mx, fabsf(x[nt][kt][c]));
            e = group_exponent(mx);
            forward_3d(tb, x, lgL, lane, pow2f(e), z);
            // shrink; q = z' diag(s) for the inverse
            const float thr_s = thr * pow2f(e);
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const float s0 = tb.scale[lgL][8 * nj + 2 * t];
                const float s1 = tb.scale[lgL][8 * nj + 2 * t + 1];
#pragma unroll
                for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float v = z[mt][nj][c];
                        if (kWiener) {
                            v *= s_w[((mt * 2 + nj) * 4 + c) * 32];
                        } else {
                            const bool keep = fabsf(v) > thr_s;
                            v = keep ? v : 0.f;
                            wsum += keep ? 1.f : 0.f;
                        }
                        z[mt][nj][c] = v * ((c & 1) ? s1 : s0);
                    }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
            const float weight = kWiener ? (wsum > 0.f ? 1.f / (s2 * wsum) : 1.f / s2)
                                         : 1.f / (s2 * fmaxf(wsum, 1.f));
            if (a.stat && lane == 0) a.stat[gi] = wsum;
            float o[8][4];
            inverse_3d(tb, z, lgL, lane, o);
            const float back = pow2f(-e - 8);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!act[q]) continue;
                double *nrow = num + (size_t)(f0 + py[q]) * W + g0 + px[q] + 2 * t;
#pragma unroll
                for (int np = 0; np < 8; ++np)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float kw = weight * (c_k1[np] * c_k1[2 * t + c]);
                        red_add_f64(nrow + (size_t)np * W + c, (double)(kw * (o[np][2 * q + c] * back)));
                    }
                if (t == 0) red_add_f64(wimg + (size_t)(f0 + py[q]) * W + g0 + px[q], (double)weight);
            }
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

// out = num / den with den = sum_{a, b < 8} A[y - a][x - b] k1[a] k1[b], the
// correlation of the weight image A (the group weights added at the patch
// positions) with the Kaiser window, in a fixed order; clears num (A is
// cleared by the caller after the launch, since neighbouring blocks read it).
// Optionally dual = w - out and the 8-bit codes of out for the next stage.
constexpr int kFinX = 32, kFinY = 8;
template <typename S>
__global__ void __launch_bounds__(kFinX * kFinY)
bm3d_finish_wimg_kernel(double *__restrict__ num, const double *__restrict__ wimg,
                        S *__restrict__ out, const S *__restrict__ w, S *__restrict__ dual,
                        uint8_t *__restrict__ codes, int H, int W, const int *__restrict__ stop)
{
    if (stop && *stop) return;
    __shared__ float s_a[kFinY + kPS - 1][kFinX + kPS];
    const int x0 = blockIdx.x * kFinX, y0 = blockIdx.y * kFinY;
    const size_t base = (size_t)blockIdx.z * H * W;
    for (int i = threadIdx.x; i < (kFinY + kPS - 1) * (kFinX + kPS - 1); i += blockDim.x) {
        const int r = i / (kFinX + kPS - 1), c = i - r * (kFinX + kPS - 1);
        const int y = y0 - (kPS - 1) + r, x = x0 - (kPS - 1) + c;
        s_a[r][c] = (y >= 0 && y < H && x >= 0 && x < W) ? (float)wimg[base + (size_t)y * W + x]
                                                         : 0.f;
    }
    __syncthreads();
    const int tx = threadIdx.x % kFinX, ty = threadIdx.x / kFinX;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= W || y >= H) return;
    float den = 0.f;
#pragma unroll
    for (int a = 0; a < kPS; ++a) {
        float r = 0.f;
#pragma unroll
        for (int b = 0; b < kPS; ++b) r = fmaf(c_k1[b], s_a[ty + kPS - 1 - a][tx + kPS - 1 - b], r);
        den = fmaf(c_k1[a], r, den);
    }
    const size_t i = base + (size_t)y * W + x;
    const float v = (float)(num[i] / (double)den);
    num[i] = 0.0;
    const float ur = keep<S>(v, i, kKeyU);
    st<S>(out + i, ur);
    if (dual) st<S>(dual + i, keep<S>(ld<S>(w + i) - ur, i, kKeyD));
    if (codes) {
        const float rr = rintf(__fmul_rn(v, 255.f));
        codes[i] = (uint8_t)(rr < 0.f ? 0.f : (rr > 255.f ? 255.f : rr));
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
        const float ur = keep<S>(v, (size_t)i, kKeyU);
        st<S>(out + i, ur);
        if (dual) st<S>(dual + i, keep<S>(ld<S>(w + i) - ur, (size_t)i, kKeyD));
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
        const float ur = keep<S>(g[i], (size_t)i, kKeyU);
        st<S>(out + i, ur);
        if (dual) st<S>(dual + i, keep<S>(ld<S>(w + i) - ur, (size_t)i, kKeyD));
    }
}

std::mutex g_mu;
std::vector<int> g_ready;  // per device: constants uploaded

// FP16 bits of a double (round to nearest even, through float).
uint16_t half_bits(double x)
{
    const __half_raw r = __float2half_rn((float)x);
    return r.x;
}

// hi / lo FP16 pair of each of two values, packed as the fragment registers
// want them (first element in the low 16 bits).
void split_pack(double x0, double x1, uint32_t &hi, uint32_t &lo)
{
    const uint16_t h0 = half_bits(x0), h1 = half_bits(x1);
    __half_raw r0, r1;
    r0.x = h0;
    r1.x = h1;
    const double e0 = x0 - (double)__half2float(__half(r0));
    const double e1 = x1 - (double)__half2float(__half(r1));
    hi = (uint32_t)h0 | ((uint32_t)h1 << 16);
    lo = (uint32_t)half_bits(e0) | ((uint32_t)half_bits(e1) << 16);
}

// The tensor-core tables: 2^8 T = 256 (C (x) C) as forward A and inverse B
// fragments (hi / lo), and the group Haar matrices H = diag(s) H_un for
// L = 1, 2, .., 16: the orthonormal Haar basis on L points, rows ordered as
// the mean, then the differences of halves over supports L, L/2, .., 2
// (each a +1 half and a -1 half, scaled by 1/sqrt(support)).
void build_tc_tables(const double *C, TcTables &tb)
{
    auto T = [&](int c, int p) {
        return 256.0 * C[(c / kPS) * kPS + p / kPS] * C[(c % kPS) * kPS + p % kPS];
    };
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t = lane & 3;
        for (int mt = 0; mt < 4; ++mt)
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t h[4], l[4];
                const int r0 = 16 * mt + g, c0 = 16 * kt + 2 * t;
                split_pack(T(r0, c0), T(r0, c0 + 1), h[0], l[0]);
                split_pack(T(r0 + 8, c0), T(r0 + 8, c0 + 1), h[1], l[1]);
                split_pack(T(r0, c0 + 8), T(r0, c0 + 9), h[2], l[2]);
                split_pack(T(r0 + 8, c0 + 8), T(r0 + 8, c0 + 9), h[3], l[3]);
                tb.fwd[(mt * 4 + kt) * 2][lane] = make_uint4(h[0], h[1], h[2], h[3]);
                tb.fwd[(mt * 4 + kt) * 2 + 1][lane] = make_uint4(l[0], l[1], l[2], l[3]);
            }
        for (int kc = 0; kc < 4; ++kc)
            for (int npp = 0; npp < 4; ++npp) {
                uint32_t h[4], l[4];
                for (int u = 0; u < 2; ++u) {
                    const int n = 8 * (2 * npp + u) + g, k0 = 16 * kc + 2 * t;
                    split_pack(T(k0, n), T(k0 + 1, n), h[2 * u], l[2 * u]);
                    split_pack(T(k0 + 8, n), T(k0 + 9, n), h[2 * u + 1], l[2 * u + 1]);
                }
                tb.inv[(kc * 4 + npp) * 2][lane] = make_uint4(h[0], h[1], h[2], h[3]);
                tb.inv[(kc * 4 + npp) * 2 + 1][lane] = make_uint4(l[0], l[1], l[2], l[3]);
            }
    }
    for (int lg = 0; lg < 5; ++lg) {
        const int L = 1 << lg;
        int Hu[kMaxGroup][kMaxGroup] = {};  // H_un[j][k]
        float sc[kMaxGroup] = {};
        for (int k = 0; k < L; ++k) Hu[0][k] = 1;
        sc[0] = (float)(1.0 / std::sqrt((double)L));
        int j = 1;
        for (int S = L; S >= 2; S /= 2)
            for (int b0 = 0; b0 < L; b0 += S, ++j) {
                for (int k = b0; k < b0 + S; ++k) Hu[j][k] = k < b0 + S / 2 ? 1 : -1;
                sc[j] = (float)(1.0 / std::sqrt((double)S));
            }
        for (int q = 0; q < kMaxGroup; ++q) tb.scale[lg][q] = sc[q];
        auto pk = [](int a, int b) {
            return (uint32_t)half_bits(a) | ((uint32_t)half_bits(b) << 16);
        };
        for (int lane = 0; lane < 32; ++lane) {
            const int g = lane >> 2, t = lane & 3;
            uint32_t f[4], v[4];
            for (int n = 0; n < 2; ++n) {
                const int c = 8 * n + g;
                // forward: B[k][j] = H_un[j][k], column j = c
                f[2 * n] = pk(Hu[c][2 * t], Hu[c][2 * t + 1]);
                f[2 * n + 1] = pk(Hu[c][2 * t + 8], Hu[c][2 * t + 9]);
                // inverse: B[j][k] = H_un[j][k], column k = c
                v[2 * n] = pk(Hu[2 * t][c], Hu[2 * t + 1][c]);
                v[2 * n + 1] = pk(Hu[2 * t + 8][c], Hu[2 * t + 9][c]);
            }
            tb.haar[lg * 2][lane] = make_uint4(f[0], f[1], f[2], f[3]);
            tb.haar[lg * 2 + 1][lane] = make_uint4(v[0], v[1], v[2], v[3]);
        }
    }
}

cslsm_status upload_constants()
{
    int dev = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_ready.size() <= dev) g_ready.resize(dev + 1, 0);
    if (g_ready[dev]) return CSLSM_OK;
    const double pi = 3.14159265358979323846;
    double C[kPS * kPS];
    float k1f[kPS];
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
            C[k * kPS + n] = (k == 0 ? std::sqrt(1.0 / kPS) : std::sqrt(2.0 / kPS)) *
                             std::cos(pi * (2 * n + 1) * k / (2.0 * kPS));
    for (int n = 0; n < kPS; ++n) {
        const double r = 2.0 * n / (kPS - 1) - 1.0;
        k1f[n] = (float)(i0(2.0 * std::sqrt(1.0 - r * r)) / i0(2.0));
    }
    static TcTables tb;  // 38 KB: built once, off the stack
    build_tc_tables(C, tb);
    CSLSM_CUDA(cudaMemcpyToSymbol(c_k1, k1f, sizeof(k1f)));
    CSLSM_CUDA(cudaMemcpyToSymbol(g_tc, &tb, sizeof(tb)));
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

template <bool kWiener>
cslsm_status launch_filter_tc(const FilterArgs &a, cudaStream_t s)
{
    const size_t smem =
        kTcSmem + (kWiener ? 2 * kFootBytes + sizeof(float) * kTcWarps * 32 * 32 : kFootBytes);
    static int per_sm[2] = {0, 0};  // resident CTAs per SM (same on every GB300)
    int &ps = per_sm[kWiener ? 1 : 0];
    if (ps == 0) {
        CSLSM_CUDA(cudaFuncSetAttribute(bm3d_filter_tc_kernel<kWiener>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int n = 0;
        CSLSM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, bm3d_filter_tc_kernel<kWiener>, kTcWarps * 32, smem));
        ps = std::max(1, n);
    }
    int dev = 0, sms = 0;
    CSLSM_CUDA(cudaGetDevice(&dev));
    CSLSM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const long long tiles = (long long)((n_refs(a.W) + kRefBlock - 1) / kRefBlock) *
                            ((n_refs(a.H) + kRefBlock - 1) / kRefBlock) * a.ns;
    const unsigned grid = (unsigned)std::max(1ll, std::min(tiles, (long long)ps * sms));
    bm3d_filter_tc_kernel<kWiener><<<grid, kTcWarps * 32, smem, s>>>(a);
    return CSLSM_OK;
}

cslsm_status filter(int stage, const float *noisy, const float *guide, const Ws &w, int ns,
                    int H, int W, float sigma, cudaStream_t s, const int *stop = nullptr,
                    float *stat = nullptr)
{
    FilterArgs a{noisy, guide, w.lists, w.counts, w.num, w.den, H, W, ns, sigma, stop, stat};
    LaunchScope ls(K_BM3D_FILTER, s);
    cslsm_status e = stage == 1 ? launch_filter_tc<false>(a, s) : launch_filter_tc<true>(a, s);
    if (e) return e;
    CSLSM_LAUNCHED();
    return CSLSM_OK;
}

// Stage output out = num / (A * Kaiser), num cleared by the kernel, the weight
// image A cleared after it.
template <typename S>
cslsm_status finish_stage(const Ws &w, S *out, const S *src, S *dual, uint8_t *codes, int ns,
                          int H, int W, cudaStream_t s, const int *stop = nullptr)
{
    {
        LaunchScope ls(K_BM3D_FINISH, s);
        const dim3 grid((W + kFinX - 1) / kFinX, (H + kFinY - 1) / kFinY, ns);
        bm3d_finish_wimg_kernel<S><<<grid, kFinX * kFinY, 0, s>>>(w.num, w.den, out, src, dual,
                                                                  codes, H, W, stop);
        CSLSM_LAUNCHED();
    }
    CSLSM_CUDA(cudaMemsetAsync(w.den, 0, sizeof(double) * (size_t)ns * H * W, s));
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
    if ((e = finish_stage<float>(w, w.basic, nullptr, nullptr, w.codes, ns, H, W, s, stop)))
        return e;
    if ((e = match(w.codes, ns, H, W, 2, w.lists, w.counts, s, stop))) return e;
    if ((e = filter(2, w.g, w.basic, w, ns, H, W, b.sigma, s, stop))) return e;
    return finish_stage<S>(w, out, src, dual, nullptr, ns, H, W, s, stop);
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
                             int ns, int H, int W, float sigma, void *ws, cudaStream_t s,
                             int *lists, int *counts, float *stat)
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
    const size_t nref = (size_t)ns * n_refs(H) * n_refs(W);
    if (lists)
        CSLSM_CUDA(cudaMemcpyAsync(lists, w.lists, sizeof(int) * nref * kMaxGroup,
                                   cudaMemcpyDeviceToDevice, s));
    if (counts)
        CSLSM_CUDA(cudaMemcpyAsync(counts, w.counts, sizeof(int) * nref, cudaMemcpyDeviceToDevice, s));
    if ((e = filter(stage, noisy, guide, w, ns, H, W, sigma, s, nullptr, stat))) return e;
    return finish_stage<float>(w, out, nullptr, nullptr, nullptr, ns, H, W, s);
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
