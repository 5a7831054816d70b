/*
 * BM3D denoiser of the u-step, for the FP64 oracle.  TEST INFRASTRUCTURE ONLY.
 *
 * The paper plugs BM3D (block matching and 3-D collaborative filtering,
 * Dabov et al. 2007) into Eq. (u-sub) and treats its lambda as a noise level
 * (Sec. IV-C); it states none of BM3D's internals.  This file is the plain
 * statement of the variant used here, applied to each 2-D slice on its own:
 *
 *  - patches 8 x 8; reference patches every 3 pixels in each direction plus
 *    the last position (H-8, W-8); images smaller than 8 in either direction
 *    are returned unchanged;
 *  - block matching inside the 39 x 39 window of patch positions centred on
 *    the reference (clipped to the image), on 8-bit codes
 *    q = clamp(rint(x * 255), 0, 255) computed in float32 (round half to
 *    even), by the exact integer sum of squared differences; a candidate
 *    joins the group when its SSD <= 64 * tau (tau = 2500 in the hard stage,
 *    400 in the Wiener stage); the reference comes first, then up to 15 other
 *    positions in increasing (SSD, y * W + x); the group keeps the largest
 *    power of two <= its size;
 *  - 3-D transform: orthonormal 8 x 8 DCT-II of every patch, then the
 *    orthonormal Haar transform along the group;
 *  - hard stage: coefficients with |c| <= 2.7 sigma are zeroed; the group's
 *    weight is 1 / (sigma^2 max(1, kept coefficients));
 *  - Wiener stage (guide = basic estimate): matching on the guide, groups of
 *    the guide (B) and of the noisy input (N) at the same positions,
 *    shrinkage W = T(B)^2 / (T(B)^2 + sigma^2) applied to T(N); weight
 *    1 / (sigma^2 sum W^2) (1 / sigma^2 if every W vanishes);
 *  - aggregation: every estimate patch is added with its group weight times
 *    an 8 x 8 separable Kaiser window (beta = 2) into numerator and
 *    denominator images; the stage output is their ratio.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define PS 8
#define HALF_WIN 19
#define REF_STEP 3
#define MAX_GROUP 16
#define LAMBDA_3D 2.7
#define TAU_HARD 2500
#define TAU_WIENER 400
#define KAISER_BETA 2.0

static const double PI = 3.14159265358979323846;

int or_bm3d_ref_positions(int n, int *out)
{
    int k = 0;
    for (int x = 0; x < n - PS; x += REF_STEP) out[k++] = x;
    out[k++] = n - PS;
    return k;
}

/* 8-bit matching code of one float32 value */
static int code8(double x)
{
    const float s = (float)x * 255.0f;
    const float r = nearbyintf(s);
    if (r < 0.0f) return 0;
    if (r > 255.0f) return 255;
    return (int)r;
}

typedef struct {
    long ssd;
    long lin;
} cand_t;

static int cand_cmp(const void *a, const void *b)
{
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->ssd != y->ssd) return x->ssd < y->ssd ? -1 : 1;
    if (x->lin != y->lin) return x->lin < y->lin ? -1 : 1;
    return 0;
}

/* Group of reference (ri, rj) on the code image q: writes the linear indices
 * of the chosen patch positions (reference first) and returns their count m
 * (1..16, before the power-of-two cut). */
static int match_one(const int *q, int H, int W, int ri, int rj, long thr, cand_t *buf,
                     long *out)
{
    int nc = 0;
    const int i0 = ri - HALF_WIN < 0 ? 0 : ri - HALF_WIN;
    const int i1 = ri + HALF_WIN > H - PS ? H - PS : ri + HALF_WIN;
    const int j0 = rj - HALF_WIN < 0 ? 0 : rj - HALF_WIN;
    const int j1 = rj + HALF_WIN > W - PS ? W - PS : rj + HALF_WIN;
    for (int ci = i0; ci <= i1; ++ci)
        for (int cj = j0; cj <= j1; ++cj) {
            if (ci == ri && cj == rj) continue;
            long ssd = 0;
            for (int a = 0; a < PS; ++a)
                for (int b = 0; b < PS; ++b) {
                    const long t = q[(ri + a) * W + rj + b] - q[(ci + a) * W + cj + b];
                    ssd += t * t;
                }
            if (ssd <= thr) {
                buf[nc].ssd = ssd;
                buf[nc].lin = (long)ci * W + cj;
                ++nc;
            }
        }
    qsort(buf, nc, sizeof(cand_t), cand_cmp);
    out[0] = (long)ri * W + rj;
    int m = 1;
    for (int k = 0; k < nc && m < MAX_GROUP; ++k) out[m++] = buf[k].lin;
    return m;
}

/* Match lists of every reference of one slice (row-major over the reference
 * grid): idx [nref][16] patch-position linear indices, cnt [nref] group sizes
 * m before the power-of-two cut.  stage 1 uses tau = 2500, stage 2 tau = 400.
 * Returns nref, or -1 on allocation failure, 0 if the image is too small. */
int or_bm3d_match(int H, int W, const double *img, int stage, long *idx, int *cnt)
{
    if (H < PS || W < PS) return 0;
    int *q = malloc(sizeof(int) * (size_t)H * W);
    int *ri = malloc(sizeof(int) * (H / REF_STEP + 2));
    int *rj = malloc(sizeof(int) * (W / REF_STEP + 2));
    cand_t *buf = malloc(sizeof(cand_t) * (2 * HALF_WIN + 1) * (2 * HALF_WIN + 1));
    if (!q || !ri || !rj || !buf) {
        free(q); free(ri); free(rj); free(buf);
        return -1;
    }
    for (size_t p = 0; p < (size_t)H * W; ++p) q[p] = code8(img[p]);
    const long thr = (long)PS * PS * (stage == 1 ? TAU_HARD : TAU_WIENER);
    const int ni = or_bm3d_ref_positions(H, ri), nj = or_bm3d_ref_positions(W, rj);
    for (int a = 0; a < ni; ++a)
        for (int b = 0; b < nj; ++b) {
            const int r = a * nj + b;
            long tmp[MAX_GROUP];
            const int m = match_one(q, H, W, ri[a], rj[b], thr, buf, tmp);
            for (int k = 0; k < MAX_GROUP; ++k) idx[(size_t)r * MAX_GROUP + k] = k < m ? tmp[k] : -1;
            cnt[r] = m;
        }
    free(q); free(ri); free(rj); free(buf);
    return ni * nj;
}

/* Orthonormal DCT-II matrix: C[k][n] = a_k cos(pi (2n+1) k / 16). */
void or_bm3d_dct8(double *C)
{
    for (int k = 0; k < PS; ++k)
        for (int n = 0; n < PS; ++n)
            C[k * PS + n] = (k == 0 ? sqrt(1.0 / PS) : sqrt(2.0 / PS)) *
                            cos(PI * (2 * n + 1) * k / (2.0 * PS));
}

/* Orthonormal Haar transform of v[0..L) (L a power of two), stride s: each
 * level replaces the first `len` entries by len/2 scaled sums followed by
 * len/2 scaled differences, then recurses on the sums. */
static void haar_fwd(double *v, int L, int s)
{
    double t[MAX_GROUP];
    for (int len = L; len > 1; len /= 2) {
        for (int i = 0; i < len / 2; ++i) {
            t[i] = (v[(2 * i) * s] + v[(2 * i + 1) * s]) / sqrt(2.0);
            t[len / 2 + i] = (v[(2 * i) * s] - v[(2 * i + 1) * s]) / sqrt(2.0);
        }
        for (int i = 0; i < len; ++i) v[i * s] = t[i];
    }
}

static void haar_inv(double *v, int L, int s)
{
    double t[MAX_GROUP];
    for (int len = 2; len <= L; len *= 2) {
        for (int i = 0; i < len / 2; ++i) {
            t[2 * i] = (v[i * s] + v[(len / 2 + i) * s]) / sqrt(2.0);
            t[2 * i + 1] = (v[i * s] - v[(len / 2 + i) * s]) / sqrt(2.0);
        }
        for (int i = 0; i < len; ++i) v[i * s] = t[i];
    }
}

/* Forward 3-D transform of a group g [L][8][8] in place: per-patch 2-D DCT
 * (rows then columns), then Haar along the group at every (a, b). */
void or_bm3d_transform(int L, double *g, int inverse)
{
    double C[PS * PS], tmp[PS * PS];
    or_bm3d_dct8(C);
    if (inverse)
        for (int ab = 0; ab < PS * PS; ++ab) haar_inv(g + ab, L, PS * PS);
    for (int k = 0; k < L; ++k) {
        double *x = g + (size_t)k * PS * PS;
        /* forward: Y = C X C^T;  inverse: X = C^T Y C */
        for (int a = 0; a < PS; ++a)
            for (int b = 0; b < PS; ++b) {
                double s = 0.0;
                for (int c = 0; c < PS; ++c)
                    s += (inverse ? C[c * PS + a] : C[a * PS + c]) * x[c * PS + b];
                tmp[a * PS + b] = s;
            }
        for (int a = 0; a < PS; ++a)
            for (int b = 0; b < PS; ++b) {
                double s = 0.0;
                for (int c = 0; c < PS; ++c)
                    s += tmp[a * PS + c] * (inverse ? C[c * PS + b] : C[b * PS + c]);
                x[a * PS + b] = s;
            }
    }
    if (!inverse)
        for (int ab = 0; ab < PS * PS; ++ab) haar_fwd(g + ab, L, PS * PS);
}

/* Modified Bessel function I0 by its power series sum_m ((x/2)^m / m!)^2. */
static double bessel_i0(double x)
{
    double term = 1.0, sum = 1.0;
    for (int m = 1; m < 60; ++m) {
        term *= (x / 2.0) / m;
        sum += term * term;
    }
    return sum;
}

/* 8 x 8 separable Kaiser window, K[a][b] = k[a] k[b],
 * k[n] = I0(beta sqrt(1 - (2n/7 - 1)^2)) / I0(beta). */
void or_bm3d_kaiser(double *K)
{
    double k[PS];
    for (int n = 0; n < PS; ++n) {
        const double r = 2.0 * n / (PS - 1) - 1.0;
        k[n] = bessel_i0(KAISER_BETA * sqrt(1.0 - r * r)) / bessel_i0(KAISER_BETA);
    }
    for (int a = 0; a < PS; ++a)
        for (int b = 0; b < PS; ++b) K[a * PS + b] = k[a] * k[b];
}

static int pow2_floor(int m)
{
    int L = 1;
    while (L * 2 <= m) L *= 2;
    return L;
}

/* One BM3D stage on one slice.
 *   guide == NULL: hard-threshold stage on `noisy` (threshold lambda3d * sigma);
 *   guide != NULL: Wiener stage with guide as the basic estimate.
 * out [H][W] receives the aggregated estimate. */
int or_bm3d_stage(int H, int W, const double *noisy, const double *guide, double sigma,
                  double lambda3d, double *out)
{
    const size_t HW = (size_t)H * W;
    if (H < PS || W < PS) {
        memcpy(out, noisy, HW * sizeof(double));
        return 0;
    }
    const int stage = guide ? 2 : 1;
    const int nref = ((H - PS + REF_STEP - 1) / REF_STEP + 1) * ((W - PS + REF_STEP - 1) / REF_STEP + 1);
    long *idx = malloc(sizeof(long) * (size_t)(nref + 4) * MAX_GROUP);
    int *cnt = malloc(sizeof(int) * (size_t)(nref + 4));
    double *num = calloc(HW, sizeof(double)), *den = calloc(HW, sizeof(double));
    if (!idx || !cnt || !num || !den) {
        free(idx); free(cnt); free(num); free(den);
        return -1;
    }
    const int nr = or_bm3d_match(H, W, guide ? guide : noisy, stage, idx, cnt);
    if (nr < 0) {
        free(idx); free(cnt); free(num); free(den);
        return -1;
    }
    double K[PS * PS];
    or_bm3d_kaiser(K);
    const double s2 = sigma * sigma, thr = lambda3d * sigma;
    double gN[MAX_GROUP * PS * PS], gB[MAX_GROUP * PS * PS];
    for (int r = 0; r < nr; ++r) {
        const int L = pow2_floor(cnt[r]);
        for (int k = 0; k < L; ++k) {
            const long lin = idx[(size_t)r * MAX_GROUP + k];
            const int ci = (int)(lin / W), cj = (int)(lin % W);
            for (int a = 0; a < PS; ++a)
                for (int b = 0; b < PS; ++b) {
                    gN[(k * PS + a) * PS + b] = noisy[(size_t)(ci + a) * W + cj + b];
                    if (guide) gB[(k * PS + a) * PS + b] = guide[(size_t)(ci + a) * W + cj + b];
                }
        }
        or_bm3d_transform(L, gN, 0);
        double weight;
        if (!guide) {
            int kept = 0;
            for (int t = 0; t < L * PS * PS; ++t) {
                if (fabs(gN[t]) <= thr) gN[t] = 0.0;
                else ++kept;
            }
            weight = 1.0 / (s2 * (kept > 1 ? kept : 1));
        } else {
            or_bm3d_transform(L, gB, 0);
            double wsum = 0.0;
            for (int t = 0; t < L * PS * PS; ++t) {
                const double wt = gB[t] * gB[t] / (gB[t] * gB[t] + s2);
                gN[t] *= wt;
                wsum += wt * wt;
            }
            weight = wsum > 0.0 ? 1.0 / (s2 * wsum) : 1.0 / s2;
        }
        or_bm3d_transform(L, gN, 1);
        for (int k = 0; k < L; ++k) {
            const long lin = idx[(size_t)r * MAX_GROUP + k];
            const int ci = (int)(lin / W), cj = (int)(lin % W);
            for (int a = 0; a < PS; ++a)
                for (int b = 0; b < PS; ++b) {
                    const size_t p = (size_t)(ci + a) * W + cj + b;
                    num[p] += weight * K[a * PS + b] * gN[(k * PS + a) * PS + b];
                    den[p] += weight * K[a * PS + b];
                }
        }
    }
    for (size_t p = 0; p < HW; ++p) out[p] = num[p] / den[p];
    free(idx); free(cnt); free(num); free(den);
    return 0;
}

/* BM3D of one slice: hard-threshold stage, then Wiener stage guided by it. */
int or_bm3d(int H, int W, const double *g, double sigma, double *u)
{
    const size_t HW = (size_t)H * W;
    double *basic = malloc(HW * sizeof(double));
    if (!basic) return -1;
    int rc = or_bm3d_stage(H, W, g, NULL, sigma, LAMBDA_3D, basic);
    if (!rc) rc = or_bm3d_stage(H, W, g, basic, sigma, LAMBDA_3D, u);
    free(basic);
    return rc;
}
