/* FP64 type-3 non-uniform FFT of the CPU oracle (test infrastructure only; only tests/,
 * the smoke check and the bench's CPU leg reach it).
 *
 * Sec. 2.2.3 computes the plane-wave matrices F_{Y->s} and F_{s->X} by a non-uniform FFT
 * and refers to Dutt & Rokhlin (1993) and Greengard & Lee (2004) for it.  This is a
 * plain restatement of that method for one box, with the "exponential of semicircle"
 * spreading kernel of Barnett, Magland & af Klinteberg (2019), written step by step:
 *
 *   forward F(s) = sum_j c_j e^{-i s.x_j}, |x_j,d| <= d/2, |s_d| <= k:
 *   1. spread the charges onto a grid of spacing h (x_m = (m - c0) h, m in [0, n1)^3):
 *        b_m = sum_j c_j prod_d phi((m_d - p_jd) / (w/2)),  p_j = c0 + x_j / h;
 *      b(x) = sum_j c_j phi_h(x - x_j) has the Fourier transform phihat_h(s) F(s), and
 *      h^3 sum_m b_m e^{-i s.x_m} samples it without aliasing when 2 pi / h - k is beyond
 *      the kernel's band, i.e. k h <= 2 pi - 2 beta / w;
 *   2. the type-2 sum g(s) = sum_m b_m e^{-i s.x_m} = sum_{m'} b_{m'} e^{-i m'.theta},
 *      theta = s h, m' = m - c0, through an oversampled grid of n2 >= 2 n1 points per axis:
 *      deconvolve b by the Fourier coefficients c(m') of the 2 pi-periodised kernel
 *      psi(theta) = phi(theta / (w pi / n2)) and zero-pad to n2^3;
 *   3. DFT of size n2^3 (sign -1);
 *   4. interpolate at t = theta n2 / (2 pi) with psi and multiply by the correction
 *      prod_d 2 / (w n2 phihat(w h s_d / 2)).
 *   adjoint v(x_j) = sum_q z_q e^{+i s_q.x_j}: the transposed steps in reverse order
 *   (spread the corrected z_q onto the DFT grid, DFT of sign +1, deconvolve and
 *   truncate to n1^3, interpolate at the points with phi).
 *
 * phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1, zero outside; phihat(xi) its
 * Fourier integral over [-1, 1], by Gauss-Legendre quadrature.  A point's window is the
 * w grid nodes floor(p - w/2) + 1, ..., floor(p - w/2) + w. */
#include "nufft_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NU_PI 3.14159265358979323846
#define NU_QUAD 128

void orc_gauss_legendre(int n, double *x, double *w);

double orc_es_kernel(double z, double beta)
{
    if (fabs(z) > 1.0) return 0.0;
    return exp(beta * (sqrt(1.0 - z * z) - 1.0));
}

double orc_es_hat(double xi, double beta)
{
    double t[NU_QUAD], wq[NU_QUAD];
    orc_gauss_legendre(NU_QUAD, t, wq);
    double s = 0.0;
    for (int i = 0; i < NU_QUAD; ++i) s += wq[i] * orc_es_kernel(t[i], beta) * cos(xi * t[i]);
    return s;
}

static int smooth7(int n)
{
    for (int p = 2; p <= 7; ++p)
        while (n % p == 0) n /= p;
    return n == 1;
}

void orc_nu_params(double d, double k, double eps, int *w, double *beta, int *M, int *n1, int *n2)
{
    int ww = (int)ceil(-log10(eps)) + 4;
    if (ww < 6) ww = 6;
    if (ww > 12) ww = 12;
    double b = 2.30 * ww;
    int m = (int)ceil(d * k / (2.0 * NU_PI - 2.0 * b / ww));
    if (m < 1) m = 1;
    int a = m + ww + 2;
    a += a & 1;
    int f = 2 * a;
    while (!smooth7(f)) ++f;
    *w = ww;
    *beta = b;
    *M = m;
    *n1 = a;
    *n2 = f;
}

int orc_nu_init(orc_nu *nu, double d, double k, double eps, const double *s, int nq)
{
    memset(nu, 0, sizeof *nu);
    orc_nu_params(d, k, eps, &nu->w, &nu->beta, &nu->M, &nu->n1, &nu->n2);
    nu->h = d / nu->M;
    nu->nq = nq;
    nu->s = s;
    nu->corr = (double *)malloc(sizeof(double) * (nq > 0 ? nq : 1));
    nu->cinv = (double *)malloc(sizeof(double) * nu->n1);
    if (!nu->corr || !nu->cinv) return 1;
    double a1 = 0.5 * nu->w * nu->h;
    for (int q = 0; q < nq; ++q) {
        double c = 1.0;
        for (int dd = 0; dd < 3; ++dd) c *= 2.0 / (nu->w * nu->n2 * orc_es_hat(a1 * s[3 * q + dd], nu->beta));
        nu->corr[q] = c;
    }
    double a2 = nu->w * NU_PI / nu->n2;
    int c0 = nu->n1 / 2;
    for (int m = 0; m < nu->n1; ++m) nu->cinv[m] = 2.0 * NU_PI / (a2 * orc_es_hat(a2 * (m - c0), nu->beta));
    return 0;
}

void orc_nu_free(orc_nu *nu)
{
    free(nu->corr);
    free(nu->cinv);
    nu->corr = nu->cinv = NULL;
}

/* the w window nodes of position p and their kernel values */
static void window(double p, int w, double beta, int *first, double *val)
{
    int f = (int)floor(p - 0.5 * w) + 1;
    *first = f;
    for (int i = 0; i < w; ++i) val[i] = orc_es_kernel((f + i - p) / (0.5 * w), beta);
}

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* 1-D DFT out[k] = sum_j in[j] e^{sign 2 pi i j k / n}: split by the smallest prime
 * factor p (n = p m), transform the p decimated subsequences, recombine; a prime length
 * is summed directly. */
static void dft1(int n, double complex *a, int sign)
{
    if (n == 1) return;
    int p = 2;
    while (n % p) ++p;
    double complex *t = (double complex *)malloc(sizeof(double complex) * n);
    if (p == n) {
        for (int kk = 0; kk < n; ++kk) {
            double complex s = 0;
            for (int j = 0; j < n; ++j) s += a[j] * cexp(sign * 2.0 * NU_PI * I * (double)(((int64_t)j * kk) % n) / n);
            t[kk] = s;
        }
        memcpy(a, t, sizeof(double complex) * n);
        free(t);
        return;
    }
    int m = n / p;
    for (int r = 0; r < p; ++r)
        for (int j = 0; j < m; ++j) t[r * m + j] = a[j * p + r];
    for (int r = 0; r < p; ++r) dft1(m, t + r * m, sign);
    for (int kk = 0; kk < m; ++kk)
        for (int u = 0; u < p; ++u) {
            int kt = kk + m * u;
            double complex s = 0;
            for (int r = 0; r < p; ++r)
                s += t[r * m + kk] * cexp(sign * 2.0 * NU_PI * I * (double)(((int64_t)r * kt) % n) / n);
            a[kt] = s;
        }
    free(t);
}

/* 3-D DFT of an n^3 array (index (i0 n + i1) n + i2), one axis at a time */
static void dft3c(int n, double complex *a, int sign)
{
    double complex *line = (double complex *)malloc(sizeof(double complex) * n);
    int64_t st[3] = {(int64_t)n * n, n, 1};
    for (int ax = 0; ax < 3; ++ax) {
        int64_t s = st[ax];
        int64_t o1 = st[(ax + 1) % 3], o2 = st[(ax + 2) % 3];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                int64_t base = i * o1 + j * o2;
                for (int e = 0; e < n; ++e) line[e] = a[base + e * s];
                dft1(n, line, sign);
                for (int e = 0; e < n; ++e) a[base + e * s] = line[e];
            }
    }
    free(line);
}

void orc_dft3(int n, double *re, double *im, int sign)
{
    int64_t N = (int64_t)n * n * n;
    double complex *a = (double complex *)malloc(sizeof(double complex) * N);
    for (int64_t i = 0; i < N; ++i) a[i] = re[i] + I * im[i];
    dft3c(n, a, sign);
    for (int64_t i = 0; i < N; ++i) {
        re[i] = creal(a[i]);
        im[i] = cimag(a[i]);
    }
    free(a);
}

void orc_nu_forward(const orc_nu *nu, const double *x, int64_t n, const double *cr, const double *ci, double *Fr,
                    double *Fi)
{
    int w = nu->w, n1 = nu->n1, n2 = nu->n2, c0 = n1 / 2;
    int64_t N1 = (int64_t)n1 * n1 * n1, N2 = (int64_t)n2 * n2 * n2;
    double complex *b = (double complex *)calloc((size_t)N1, sizeof(double complex));
    double complex *f = (double complex *)calloc((size_t)N2, sizeof(double complex));
    double wx[3][16];
    int fx[3];
    /* 1. spread */
    for (int64_t j = 0; j < n; ++j) {
        for (int d = 0; d < 3; ++d) window(c0 + x[3 * j + d] / nu->h, w, nu->beta, &fx[d], wx[d]);
        double complex c = cr[j] + I * ci[j];
        for (int a = 0; a < w; ++a)
            for (int bb = 0; bb < w; ++bb)
                for (int cc = 0; cc < w; ++cc)
                    b[((int64_t)(fx[0] + a) * n1 + (fx[1] + bb)) * n1 + (fx[2] + cc)] +=
                        c * wx[0][a] * wx[1][bb] * wx[2][cc];
    }
    /* 2. deconvolve and zero-pad */
    for (int i0 = 0; i0 < n1; ++i0)
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i2 = 0; i2 < n1; ++i2)
                f[((int64_t)wrap(i0 - c0, n2) * n2 + wrap(i1 - c0, n2)) * n2 + wrap(i2 - c0, n2)] =
                    b[((int64_t)i0 * n1 + i1) * n1 + i2] * nu->cinv[i0] * nu->cinv[i1] * nu->cinv[i2];
    /* 3. DFT */
    dft3c(n2, f, -1);
    /* 4. interpolate and correct */
    double sc = nu->h * n2 / (2.0 * NU_PI);
    for (int q = 0; q < nu->nq; ++q) {
        for (int d = 0; d < 3; ++d) window(nu->s[3 * q + d] * sc, w, nu->beta, &fx[d], wx[d]);
        double complex g = 0;
        for (int a = 0; a < w; ++a)
            for (int bb = 0; bb < w; ++bb)
                for (int cc = 0; cc < w; ++cc)
                    g += f[((int64_t)wrap(fx[0] + a, n2) * n2 + wrap(fx[1] + bb, n2)) * n2 + wrap(fx[2] + cc, n2)] *
                         wx[0][a] * wx[1][bb] * wx[2][cc];
        g *= nu->corr[q];
        Fr[q] = creal(g);
        Fi[q] = cimag(g);
    }
    free(b);
    free(f);
}

void orc_nu_adjoint(const orc_nu *nu, const double *x, int64_t n, const double *zr, const double *zi, double *vr,
                    double *vi)
{
    int w = nu->w, n1 = nu->n1, n2 = nu->n2, c0 = n1 / 2;
    int64_t N2 = (int64_t)n2 * n2 * n2;
    double complex *f = (double complex *)calloc((size_t)N2, sizeof(double complex));
    double wx[3][16];
    int fx[3];
    /* 4'. spread the corrected coefficients onto the DFT grid */
    double sc = nu->h * n2 / (2.0 * NU_PI);
    for (int q = 0; q < nu->nq; ++q) {
        for (int d = 0; d < 3; ++d) window(nu->s[3 * q + d] * sc, w, nu->beta, &fx[d], wx[d]);
        double complex z = (zr[q] + I * zi[q]) * nu->corr[q];
        for (int a = 0; a < w; ++a)
            for (int bb = 0; bb < w; ++bb)
                for (int cc = 0; cc < w; ++cc)
                    f[((int64_t)wrap(fx[0] + a, n2) * n2 + wrap(fx[1] + bb, n2)) * n2 + wrap(fx[2] + cc, n2)] +=
                        z * wx[0][a] * wx[1][bb] * wx[2][cc];
    }
    /* 3'. DFT of the opposite sign */
    dft3c(n2, f, +1);
    /* 2'. truncate to the n1^3 modes and deconvolve; 1'. interpolate at the points */
    for (int64_t j = 0; j < n; ++j) {
        for (int d = 0; d < 3; ++d) window(c0 + x[3 * j + d] / nu->h, w, nu->beta, &fx[d], wx[d]);
        double complex v = 0;
        for (int a = 0; a < w; ++a)
            for (int bb = 0; bb < w; ++bb)
                for (int cc = 0; cc < w; ++cc) {
                    int i0 = fx[0] + a, i1 = fx[1] + bb, i2 = fx[2] + cc;
                    v += f[((int64_t)wrap(i0 - c0, n2) * n2 + wrap(i1 - c0, n2)) * n2 + wrap(i2 - c0, n2)] *
                         nu->cinv[i0] * nu->cinv[i1] * nu->cinv[i2] * wx[0][a] * wx[1][bb] * wx[2][cc];
                }
        vr[j] = creal(v);
        vi[j] = cimag(v);
    }
    free(f);
}
