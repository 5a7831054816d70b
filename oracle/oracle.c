/*
 * FP64 CPU oracle for PnP-ADMM compressive light-sheet reconstruction
 * (Gong, Zhang, Chai, Ding, Lou, "A Plug-and-Play Framework for Volumetric
 * Light-Sheet Image Reconstruction", arXiv 2511.03093).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the reconstruction computes.  Only the test-suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load it; the
 * CUDA library never does, and the two share no code.
 *
 * Every routine works in double precision on row-major arrays with the last
 * index (x, width W) fastest:
 *   volume v, u, d : [Z][H][W], Z = N*R, slice n = j*R + r   (shot j, plane r)
 *   measurement b  : [N][H][W]
 *   masks phi      : [R][H][W] shared by all shots, or [Z][H][W] per slice
 *                    (per_slice != 0).  Entries are the DMD pattern values:
 *                    {0,1} for binary masks, any real for relaxed masks.
 *
 * Readings of points the paper leaves open (each applied below):
 *  - The data term carries 1/2 everywhere, so that the printed closed-form
 *    v-update (Eq. v-update) is the exact minimiser of the v-subproblem.
 *  - "Phi^T b / (rho + Phi Phi^T)" in the final Woodbury update is read as
 *    Phi^T [ b ./ (rho + D) ], D = diag(Phi Phi^T) (what the derivation gives).
 *  - Periodic z boundary: each cyclic neighbour pair is one term, and the
 *    Gauss-Seidel sweep over n = 1..NR reads the newest value of every
 *    neighbour (slice 1 reads u_NR from the previous sweep, slice NR reads the
 *    freshly updated u_1).  Z = 1 has no z term.
 *  - u^0 = d^0 = 0 unless the caller supplies them.
 *  - TV prox: Chambolle's 2004 dual projection, cold start p^0 = 0, isotropic
 *    TV per slice, forward differences with a zero gradient on the last
 *    row / column, div = -grad^T; step tau and inner count T from the caller.
 *  - Stopping: ||v^{k+1} - v^k||_2 / ||v^k||_2 < tol, when tol > 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define IDX2(i, j, W) ((size_t)(i) * (size_t)(W) + (size_t)(j))

static const double *mask_plane(const double *phi, int per_slice, int j, int R, int r,
                                size_t HW)
{
    return phi + (size_t)(per_slice ? j * R + r : r) * HW;
}

/* ---------------------------------------------------------------------------
 * Forward operator, Sec. III-A and Eq. (model-slice):
 *   b_j = sum_{r=1..R} phi_r (Hadamard) v_{(j-1)R + r}
 * ------------------------------------------------------------------------- */
void or_forward(int N, int R, int H, int W, const double *phi, int per_slice,
                const double *v, double *b)
{
    const size_t HW = (size_t)H * W;
    for (int j = 0; j < N; ++j) {
#pragma omp parallel for schedule(static) if (HW >= 16384)
        for (size_t p = 0; p < HW; ++p) {
            double s = 0.0;
            for (int r = 0; r < R; ++r)
                s += mask_plane(phi, per_slice, j, R, r, HW)[p] * v[(size_t)(j * R + r) * HW + p];
            b[(size_t)j * HW + p] = s;
        }
    }
}

/* Adjoint Phi^T (the transpose used in Eq. v-update): v_{(j-1)R+r} = phi_r b_j. */
void or_adjoint(int N, int R, int H, int W, const double *phi, int per_slice,
                const double *b, double *v)
{
    const size_t HW = (size_t)H * W;
    for (int j = 0; j < N; ++j)
        for (int r = 0; r < R; ++r) {
            const double *m = mask_plane(phi, per_slice, j, R, r, HW);
            double *out = v + (size_t)(j * R + r) * HW;
#pragma omp parallel for schedule(static) if (HW >= 16384)
            for (size_t p = 0; p < HW; ++p)
                out[p] = m[p] * b[(size_t)j * HW + p];
        }
}

/* D = diag(Phi Phi^T) per shot, Sec. III-B: Phi Phi^T is diagonal because each
 * phi_r is; its entry at a pixel is sum_r phi_r^2.  Output [N][H][W]. */
void or_phiphit(int N, int R, int H, int W, const double *phi, int per_slice, double *D)
{
    const size_t HW = (size_t)H * W;
    for (int j = 0; j < N; ++j)
        for (size_t p = 0; p < HW; ++p) {
            double s = 0.0;
            for (int r = 0; r < R; ++r) {
                const double m = mask_plane(phi, per_slice, j, R, r, HW)[p];
                s += m * m;
            }
            D[(size_t)j * HW + p] = s;
        }
}

/* ---------------------------------------------------------------------------
 * v-update, Eq. (v-update) simplified by the Woodbury identity (Eq. Woodbury
 * and the derivation that follows it, Sec. III-B):
 *   v = Phi^T [b / (rho + D)] + g - Phi^T [ (Phi g) / (rho + D) ],  g = u - d,
 * per shot j, element-wise per pixel.
 * ------------------------------------------------------------------------- */
void or_vupdate(int N, int R, int H, int W, const double *phi, int per_slice,
                const double *b, const double *u, const double *d, double rho, double *v)
{
    const size_t HW = (size_t)H * W;
    for (int j = 0; j < N; ++j) {
#pragma omp parallel for schedule(static) if (HW >= 16384)
        for (size_t p = 0; p < HW; ++p) {
            double D = 0.0, phig = 0.0;
            for (int r = 0; r < R; ++r) {
                const size_t n = (size_t)(j * R + r) * HW + p;
                const double m = mask_plane(phi, per_slice, j, R, r, HW)[p];
                D += m * m;
                phig += m * (u[n] - d[n]);
            }
            const double bj = b[(size_t)j * HW + p];
            for (int r = 0; r < R; ++r) {
                const size_t n = (size_t)(j * R + r) * HW + p;
                const double m = mask_plane(phi, per_slice, j, R, r, HW)[p];
                const double g = u[n] - d[n];
                v[n] = m * (bj / (rho + D)) + g - m * (phig / (rho + D));
            }
        }
    }
}

/* ---------------------------------------------------------------------------
 * Isotropic TV prox by Chambolle's dual projection (the TV denoiser named in
 * Sec. III-B after Eq. u-sub):
 *   u = argmin_u theta * TV(u) + 1/2 ||u - g||^2 on one H x W slice,
 *   p^0 = 0,
 *   p^{t+1} = (p^t + tau grad(div p^t - g/theta)) / (1 + tau |grad(div p^t - g/theta)|),
 *   u = g - theta div p^T.
 * grad: forward differences, zero on the last row (component 1, along i) and
 * the last column (component 2, along j).  div = -grad^T.
 * ------------------------------------------------------------------------- */
static double tv_div(const double *p1, const double *p2, int H, int W, int i, int j)
{
    const double a = (i < H - 1 ? p1[IDX2(i, j, W)] : 0.0) - (i > 0 ? p1[IDX2(i - 1, j, W)] : 0.0);
    const double c = (j < W - 1 ? p2[IDX2(i, j, W)] : 0.0) - (j > 0 ? p2[IDX2(i, j - 1, W)] : 0.0);
    return a + c;
}

int or_tv_prox(int H, int W, const double *g, double theta, int T, double tau, double *u)
{
    const size_t HW = (size_t)H * W;
    if (!(theta > 0.0)) { /* zero weight: the prox is the identity */
        memcpy(u, g, HW * sizeof(double));
        return 0;
    }
    double *p1 = calloc(HW, sizeof(double));
    double *p2 = calloc(HW, sizeof(double));
    double *q = malloc(HW * sizeof(double));
    if (!p1 || !p2 || !q) {
        free(p1); free(p2); free(q);
        return -1;
    }
    for (int t = 0; t < T; ++t) {
#pragma omp parallel for schedule(static) if (HW >= 16384)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j)
                q[IDX2(i, j, W)] = tv_div(p1, p2, H, W, i, j) - g[IDX2(i, j, W)] / theta;
#pragma omp parallel for schedule(static) if (HW >= 16384)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                const double qc = q[IDX2(i, j, W)];
                const double gx = (i < H - 1) ? q[IDX2(i + 1, j, W)] - qc : 0.0;
                const double gy = (j < W - 1) ? q[IDX2(i, j + 1, W)] - qc : 0.0;
                const double den = 1.0 + tau * sqrt(gx * gx + gy * gy);
                p1[IDX2(i, j, W)] = (p1[IDX2(i, j, W)] + tau * gx) / den;
                p2[IDX2(i, j, W)] = (p2[IDX2(i, j, W)] + tau * gy) / den;
            }
    }
#pragma omp parallel for schedule(static) if (HW >= 16384)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j)
            u[IDX2(i, j, W)] = g[IDX2(i, j, W)] - theta * tv_div(p1, p2, H, W, i, j);
    free(p1); free(p2); free(q);
    return 0;
}

/* ---------------------------------------------------------------------------
 * PSNR over a whole volume, Sec. IV (PSNR definition and its 3D extension):
 * 10 log10( n V^2 / ||x - ref||^2 ), V = max of the reference.
 * ------------------------------------------------------------------------- */
double or_psnr(size_t n, const double *x, const double *ref)
{
    double V = ref[0], e = 0.0;
    for (size_t i = 0; i < n; ++i) {
        if (ref[i] > V) V = ref[i];
        const double t = x[i] - ref[i];
        e += t * t;
    }
    return 10.0 * log10((double)n * V * V / e);
}

/* ---------------------------------------------------------------------------
 * 3-D SSIM (Sec. IV, evaluation metrics): the local ssim of Wang et al. with
 * means, variances and the covariance taken over an 11 x 11 x 11 Gaussian
 * window (standard deviation 1.5) centred on every voxel, c1 = (0.01 L)^2,
 * c2 = (0.03 L)^2 with L = 1, averaged over every voxel of the volume.  The
 * paper does not say how the window meets the volume's faces; here it is
 * clipped to the volume and its weights renormalised to sum to one.  The
 * Gaussian weights and the box clipping are both separable, so the window
 * mean of any field is three 1-D normalised passes (x, then y, then z).
 * Variances and the covariance are the window means of x^2, y^2, x y minus
 * the products of the window means.
 * ------------------------------------------------------------------------- */
#define SSIM_R 5

static void ssim_pass(const double *in, double *out, int Z, int H, int W, int axis,
                      const double *g)
{
    const int n = axis == 0 ? W : (axis == 1 ? H : Z);
    const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)W : (size_t)H * W);
#pragma omp parallel for if ((size_t)Z * H * W >= 16384)
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int c = axis == 0 ? x : (axis == 1 ? y : z);
                const size_t o = ((size_t)z * H + y) * W + x;
                double s = 0.0, ws = 0.0;
                for (int k = -SSIM_R; k <= SSIM_R; ++k) {
                    const int q = c + k;
                    if (q < 0 || q >= n) continue;
                    s += g[k + SSIM_R] * in[(size_t)((long long)o + (long long)k * (long long)stride)];
                    ws += g[k + SSIM_R];
                }
                out[o] = s / ws;
            }
}

static void ssim_mean(const double *f, double *out, double *tmp, int Z, int H, int W,
                      const double *g)
{
    ssim_pass(f, out, Z, H, W, 0, g);
    ssim_pass(out, tmp, Z, H, W, 1, g);
    ssim_pass(tmp, out, Z, H, W, 2, g);
}

double or_ssim3d(int Z, int H, int W, const double *x, const double *y, double *map)
{
    const size_t n = (size_t)Z * H * W;
    double g[2 * SSIM_R + 1];
    for (int k = -SSIM_R; k <= SSIM_R; ++k) g[k + SSIM_R] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
    double *buf = (double *)malloc(sizeof(double) * n * 7);
    if (!buf) return NAN;
    double *f = buf, *tmp = buf + n, *mx = buf + 2 * n, *my = buf + 3 * n, *sxx = buf + 4 * n,
           *syy = buf + 5 * n, *sxy = buf + 6 * n;
    ssim_mean(x, mx, tmp, Z, H, W, g);
    ssim_mean(y, my, tmp, Z, H, W, g);
    for (size_t i = 0; i < n; ++i) f[i] = x[i] * x[i];
    ssim_mean(f, sxx, tmp, Z, H, W, g);
    for (size_t i = 0; i < n; ++i) f[i] = y[i] * y[i];
    ssim_mean(f, syy, tmp, Z, H, W, g);
    for (size_t i = 0; i < n; ++i) f[i] = x[i] * y[i];
    ssim_mean(f, sxy, tmp, Z, H, W, g);
    const double c1 = 0.01 * 0.01, c2 = 0.03 * 0.03;
    double acc = 0.0;
    for (size_t i = 0; i < n; ++i) {
        const double vx = sxx[i] - mx[i] * mx[i], vy = syy[i] - my[i] * my[i];
        const double cxy = sxy[i] - mx[i] * my[i];
        const double s = (2.0 * mx[i] * my[i] + c1) * (2.0 * cxy + c2) /
                         ((mx[i] * mx[i] + my[i] * my[i] + c1) * (vx + vy + c2));
        if (map) map[i] = s;
        acc += s;
    }
    free(buf);
    return acc / (double)n;
}

/* ---------------------------------------------------------------------------
 * Algorithm 1 (CS LSM temporal reconstruction; gamma = 0 is the slice-based
 * method of Sec. III-B).  One iteration k:
 *   1. v^{k+1} by Eq. (v-update) per shot (Woodbury form above);
 *   2. for n = 1..NR in order: g = (rho (v_n + d_n) + gamma (u_{n-1} + u_{n+1}))
 *      / (rho + 2 gamma) and u_n = denoise(g) per Eq. (u-update);
 *   3. d^{k+1} = d^k + v^{k+1} - u^{k+1}.
 * Denoisers (Eq. u-update with psi):
 *   OR_TIKHONOV: psi = ||u||^2, u_n = (rho(v_n+d_n) + gamma(u_{n-1}+u_{n+1}))
 *                / (2 lambda + rho + 2 gamma)  (closed forms of Sec. III-B/C);
 *   OR_TV:       Chambolle prox of g with theta = lambda / (rho + 2 gamma);
 *   OR_BM3D:     BM3D of g with noise level sigma (lambda is a noise level
 *                for this prior, Sec. IV-C), see or_bm3d().
 * Returns v^K (Algorithm 1's output); u, d hold u^K, d^K.
 * ------------------------------------------------------------------------- */
int or_admm(int N, int R, int H, int W, const double *phi, int per_slice, const double *b,
            double rho, double lambda, double gamma, int iters, double tol, int denoiser,
            int tv_inner, double tv_tau, double bm3d_sigma, int init_user,
            double *v, double *u, double *d, int *iters_done)
{
    const int Z = N * R;
    const size_t HW = (size_t)H * W, NV = (size_t)Z * HW;
    if (!init_user) {
        memset(u, 0, NV * sizeof(double));
        memset(d, 0, NV * sizeof(double));
    }
    memset(v, 0, NV * sizeof(double));
    double *vprev = malloc(NV * sizeof(double));
    double *g = malloc(HW * sizeof(double));
    if (!vprev || !g) {
        free(vprev); free(g);
        return -1;
    }
    const double gam = (Z > 1) ? gamma : 0.0;
    int k;
    for (k = 0; k < iters; ++k) {
        memcpy(vprev, v, NV * sizeof(double));
        /* step 1: v-update for every shot */
        or_vupdate(N, R, H, W, phi, per_slice, b, u, d, rho, v);
        /* step 2: Gauss-Seidel sweep over the slices, in place in u */
        for (int n = 0; n < Z; ++n) {
            const double *un1 = u + (size_t)((n + Z - 1) % Z) * HW; /* u_{n-1}: newest value */
            const double *up1 = u + (size_t)((n + 1) % Z) * HW;     /* u_{n+1}: newest value */
            const double *vn = v + (size_t)n * HW, *dn = d + (size_t)n * HW;
            double *un = u + (size_t)n * HW;
            if (denoiser == OR_TIKHONOV) {
                for (size_t p = 0; p < HW; ++p)
                    g[p] = (rho * (vn[p] + dn[p]) + gam * (un1[p] + up1[p])) /
                           (2.0 * lambda + rho + 2.0 * gam);
                memcpy(un, g, HW * sizeof(double));
                continue;
            }
            for (size_t p = 0; p < HW; ++p)
                g[p] = (rho * (vn[p] + dn[p]) + gam * (un1[p] + up1[p])) / (rho + 2.0 * gam);
            int rc;
            if (denoiser == OR_TV)
                rc = or_tv_prox(H, W, g, lambda / (rho + 2.0 * gam), tv_inner, tv_tau, un);
            else if (denoiser == OR_BM3D)
                rc = or_bm3d(H, W, g, bm3d_sigma, un);
            else
                rc = -2;
            if (rc) {
                free(vprev); free(g);
                return rc;
            }
        }
        /* step 3: dual update */
        for (size_t i = 0; i < NV; ++i)
            d[i] = d[i] + v[i] - u[i];
        if (tol > 0.0 && k > 0) {
            double num = 0.0, den = 0.0;
            for (size_t i = 0; i < NV; ++i) {
                num += (v[i] - vprev[i]) * (v[i] - vprev[i]);
                den += vprev[i] * vprev[i];
            }
            if (den > 0.0 && sqrt(num / den) < tol) {
                ++k;
                break;
            }
        }
    }
    if (iters_done) *iters_done = k;
    free(vprev); free(g);
    return 0;
}
