/* FP64 CPU oracle: declarations.  TEST INFRASTRUCTURE ONLY (see oracle.c). */
#ifndef CSLSM_ORACLE_H
#define CSLSM_ORACLE_H
#include <stddef.h>
#include <stdint.h>

enum { OR_TIKHONOV = 0, OR_TV = 1, OR_BM3D = 2 };

void or_forward(int N, int R, int H, int W, const double *phi, int per_slice,
                const double *v, double *b);
void or_adjoint(int N, int R, int H, int W, const double *phi, int per_slice,
                const double *b, double *v);
void or_phiphit(int N, int R, int H, int W, const double *phi, int per_slice, double *D);
void or_vupdate(int N, int R, int H, int W, const double *phi, int per_slice,
                const double *b, const double *u, const double *d, double rho, double *v);
int or_tv_prox(int H, int W, const double *g, double theta, int T, double tau, double *u);
double or_psnr(size_t n, const double *x, const double *ref);
double or_ssim3d(int Z, int H, int W, const double *x, const double *y, double *map);
int or_bm3d(int H, int W, const double *g, double sigma, double *u);
int or_bm3d_stage(int H, int W, const double *noisy, const double *guide, double sigma,
                  double lambda3d, double *out);
int or_bm3d_match(int H, int W, const double *img, int stage, long *idx, int *cnt);
int or_bm3d_ref_positions(int n, int *out);
void or_bm3d_dct8(double *C);
void or_bm3d_transform(int L, double *g, int inverse);
void or_bm3d_kaiser(double *K);
int or_admm(int N, int R, int H, int W, const double *phi, int per_slice, const double *b,
            double rho, double lambda, double gamma, int iters, double tol, int denoiser,
            int tv_inner, double tv_tau, double bm3d_sigma, int init_user,
            double *v, double *u, double *d, int *iters_done);
#endif
