/* FP64 type-3 non-uniform FFT of the CPU oracle (test infrastructure only).
 *
 * Sec. 2.2.3 evaluates the plane-wave matrices F_{Y->s} and F_{s->X} with a non-uniform
 * FFT (the method of Dutt & Rokhlin 1993, improved by Greengard & Lee 2004) instead of
 * assembling them.  This module is that transform for one box:
 *   forward  F_q = sum_j c_j exp(-i s_q . x_j)
 *   adjoint  v_j = sum_q z_q exp(+i s_q . x_j)
 * for points x_j in the cube [-d/2, d/2]^3 (box-centred) and frequencies s_q = k shat_q
 * with |shat_q| = 1.  Nothing here is shared with the CUDA path. */
#pragma once
#include <stdint.h>

typedef struct {
    int w;          /* kernel width in grid points */
    double beta;    /* exponential-of-semicircle shape parameter */
    int M;          /* cells per box edge on the spreading grid */
    double h;       /* spreading-grid spacing, d / M */
    int n1;         /* spreading grid n1^3 (box centred at grid point c0 = n1 / 2) */
    int n2;         /* FFT grid n2^3 */
    int nq;         /* number of frequencies */
    const double *s;  /* nq x 3 frequencies (caller-owned) */
    double *corr;     /* nq: prod_d 2 / (w n2 phihat(w h s_qd / 2)) */
    double *cinv;     /* n1: 1 / c(m - c0), the deconvolution of the FFT-grid kernel */
} orc_nu;

/* Parameters of the reading: w = clamp(ceil(-log10 eps) + 4, 6, 12), beta = 2.30 w,
 * M = ceil(d k / (2 pi - 2 beta / w)), n1 = M + w + 2 rounded up to even, n2 = the
 * smallest integer >= 2 n1 with no prime factor above 7. */
void orc_nu_params(double d, double k, double eps, int *w, double *beta, int *M, int *n1, int *n2);
int orc_nu_init(orc_nu *nu, double d, double k, double eps, const double *s, int nq);
void orc_nu_free(orc_nu *nu);
void orc_nu_forward(const orc_nu *nu, const double *x, int64_t n, const double *cr, const double *ci, double *Fr,
                    double *Fi);
void orc_nu_adjoint(const orc_nu *nu, const double *x, int64_t n, const double *zr, const double *zi, double *vr,
                    double *vi);
/* pieces exposed for the pins */
double orc_es_kernel(double z, double beta);
double orc_es_hat(double xi, double beta);
void orc_dft3(int n, double *re, double *im, int sign);
