/*
 * FFM oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of
 *   (O1) the discrete convolution v_i = sum_j w_j G(x_i - y_j) u_j   (Sec. 1, eqs. 3-4)
 *   (O2) the Fast Free Memory method: two cubic octrees of equal edge (Sec. 2.2.1),
 *        descent-only traversal with the admissibility test of Sec. 2.2.2,
 *        Chebyshev-Lagrange far field (Sec. 2.2.2), Gegenbauer plane-wave far field
 *        (Sec. 2.2.3, eqs. 10-14), stopping criterion (Sec. 2.2.4), dense near field.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this
 * library.  It shares no code, header, table or helper with the CUDA path.  Every
 * transfer matrix and every Gegenbauer transfer function is evaluated afresh for each
 * box pair, straight from its definition (no caching by translation), so that the GPU
 * path's translation tables are checked against an independent computation.
 *
 * Readings where the paper is silent or garbled (all plan constants):
 *   - Gegenbauer series summed from p = 0 (eq. 12 prints p = 1).
 *   - Phases taken relative to the box centres, so the transfer carries no r0 phase
 *     (eq. 13/15 print e^{+ik r0.s}, which has the wrong sign).
 *   - L = floor(|k| sqrt(3) d_l - ln(eps)) with the natural logarithm (eq. 13).
 *   - Quadrature of n_Q = 2L(L+1) nodes: (L+1) Gauss-Legendre nodes in cos(theta)
 *     times 2L equispaced azimuths phi_j = j*pi/L (Sec. 3.3, eq. 17).
 *   - Admissible iff the max-norm of the centre offset is >= 2 d_l (Sec. 2.2.2).
 *   - Root cubes centred on each set's tight box, common edge d0*(1+2^-20) (Sec. 2.2.1);
 *     integer box coordinate floor(((x-o)/d0) * 2^l) in FP64, clamped to [0, 2^l-1].
 *   - Stop after level l if no near pair is left, or if the mean number of points per
 *     non-empty box at level l (both trees) is below n_leaf, or at l = 21 (Sec. 2.2.4).
 *   - Pairs at distance 0 contribute nothing for the singular kernels.
 *   - Plane waves at level l iff the kernel is Helmholtz and k d_l >= kappa_switch (2.0);
 *     otherwise Lagrange with r1 from the calibrated error table below.
 *   - ACA of T (eq. 11, optional, Laplace single layer): full pivoting on the explicit
 *     r x r matrix, near-ties of pivot magnitudes (within a factor 1 - 1e-9) to the first
 *     entry in row-major order, stop once |T - A B^T|_F <= aca_eps |T|_F or at min(r, 64)
 *     terms (orc_aca).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (see oracle/build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "nufft_oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 21
#define ORC_PI 3.14159265358979323846

enum { ORC_LAPLACE = 0, ORC_HELMHOLTZ = 1, ORC_POLY = 2, ORC_LAPLACE_DL = 3, ORC_LAPLACE_GRAD = 4 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2 };
enum { ORC_MODE_NONE = 0, ORC_MODE_LAGRANGE = 1, ORC_MODE_PLANEWAVE = 2 };

/* ------------------------------------------------------------------ kernels */

/* Test-only polynomial kernel: degree <= 3 in each coordinate of d = x - y, so a
 * Lagrange interpolation with r1 >= 4 nodes per axis reproduces it exactly. */
static double poly_kernel(double dx, double dy, double dz)
{
    return 1.0 + 0.5 * dx - 0.25 * dy * dz + 0.125 * dx * dx * dy - 0.0625 * dz * dz * dz
           + 0.03125 * dx * dy * dz;
}

/* G(x - y) for the Laplace kernel 1/(4 pi r) (eq. 19), the Helmholtz kernel
 * e^{ikr}/(4 pi r) (eq. 9), or the polynomial test kernel. r = 0 gives 0 for the
 * singular kernels.  The double-layer kind is built on the Laplace G: its transfer
 * operators are those of G, its source step differentiates the interpolant. */
static void orc_kernel(int kind, double k, double dx, double dy, double dz, double *gr, double *gi)
{
    if (kind == ORC_POLY) {
        *gr = poly_kernel(dx, dy, dz);
        *gi = 0.0;
        return;
    }
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r == 0.0) {
        *gr = 0.0;
        *gi = 0.0;
        return;
    }
    double a = 1.0 / (4.0 * ORC_PI * r);
    if (kind == ORC_LAPLACE || kind == ORC_LAPLACE_DL || kind == ORC_LAPLACE_GRAD) {
        *gr = a;
        *gi = 0.0;
    } else {
        *gr = a * cos(k * r);
        *gi = a * sin(k * r);
    }
}

int orc_nthreads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void orc_kernel_eval(int kind, double k, double dx, double dy, double dz, double *gr, double *gi)
{
    orc_kernel(kind, k, dx, dy, dz, gr, gi);
}

/* ------------------------------------------------------------ O1 direct sum */

/* v_i = sum_j w_j G(x_i - y_j) u_j  (eq. 3), every pair, FP64.
 * X: nx*3 row-major, Y: ny*3 row-major, w: ny or NULL (w = 1).
 * u: ny*nrhs column-major (ure, uim; uim NULL means real u).
 * tsel: nsel target indices, or NULL for all nx targets (nsel ignored).
 * v: nsel*nrhs column-major (vre, vim). */
int orc_direct(const double *X, int64_t nx, const double *Y, int64_t ny, const double *w,
               const double *ure, const double *uim, int nrhs, int kind, double k,
               const int64_t *tsel, int64_t nsel, double *vre, double *vim)
{
    if (nx < 0 || ny < 0 || nrhs < 1) return ORC_EINVAL;
    int64_t nt = tsel ? nsel : nx;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nt; ++s) {
        int64_t i = tsel ? tsel[s] : s;
        const double *x = X + 3 * i;
        for (int m = 0; m < nrhs; ++m) {
            double ar = 0.0, ai = 0.0;
            for (int64_t j = 0; j < ny; ++j) {
                double gr, gi;
                orc_kernel(kind, k, x[0] - Y[3 * j], x[1] - Y[3 * j + 1], x[2] - Y[3 * j + 2], &gr, &gi);
                double wj = w ? w[j] : 1.0;
                double qr = wj * ure[j + ny * m];
                double qi = uim ? wj * uim[j + ny * m] : 0.0;
                ar += gr * qr - gi * qi;
                ai += gr * qi + gi * qr;
            }
            vre[s + nt * m] = ar;
            vim[s + nt * m] = ai;
        }
    }
    return ORC_OK;
}

/* Double-layer direct sum: v_i = sum_j w_j u_j dG/dn_y(x_i - y_j) with the Laplace G,
 * dG/dn_y = n_j . (x_i - y_j) / (4 pi |x_i - y_j|^3); pairs at distance 0 contribute 0.
 * nrm: ny*3 row-major source normals (any length: the kernel is linear in n).  Real
 * densities u (ny*nrhs column-major); v: nsel*nrhs (all nx targets if tsel is NULL). */
int orc_direct_dl(const double *X, int64_t nx, const double *Y, int64_t ny, const double *nrm, const double *w,
                  const double *u, int nrhs, const int64_t *tsel, int64_t nsel, double *v)
{
    if (nx < 0 || ny < 0 || nrhs < 1 || !nrm) return ORC_EINVAL;
    int64_t nt = tsel ? nsel : nx;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nt; ++s) {
        int64_t i = tsel ? tsel[s] : s;
        const double *x = X + 3 * i;
        for (int m = 0; m < nrhs; ++m) {
            double acc = 0.0;
            for (int64_t j = 0; j < ny; ++j) {
                double d0 = x[0] - Y[3 * j], d1 = x[1] - Y[3 * j + 1], d2 = x[2] - Y[3 * j + 2];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                if (r2 == 0.0) continue;
                double r = sqrt(r2);
                double nd = nrm[3 * j] * d0 + nrm[3 * j + 1] * d1 + nrm[3 * j + 2] * d2;
                double wj = w ? w[j] : 1.0;
                acc += wj * u[j + ny * m] * nd / (4.0 * ORC_PI * r2 * r);
            }
            v[s + nt * m] = acc;
        }
    }
    return ORC_OK;
}

/* O1 for the gradient of the single layer in the target variable (the MFIE kernel of
 * Sec. 4.2): v_i = sum_j w_j u_j grad_x G(x_i - y_j), grad_x G = -(x - y) / (4 pi |x - y|^3);
 * component d of right-hand side m in column 3 m + d of v (nt x 3 nrhs, column-major). */
int orc_direct_grad(const double *X, int64_t nx, const double *Y, int64_t ny, const double *w, const double *u,
                    int nrhs, const int64_t *tsel, int64_t nsel, double *v)
{
    if (nx < 0 || ny < 0 || nrhs < 1) return ORC_EINVAL;
    int64_t nt = tsel ? nsel : nx;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < nt; ++s) {
        int64_t i = tsel ? tsel[s] : s;
        const double *x = X + 3 * i;
        for (int m = 0; m < nrhs; ++m) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int64_t j = 0; j < ny; ++j) {
                double d[3] = {x[0] - Y[3 * j], x[1] - Y[3 * j + 1], x[2] - Y[3 * j + 2]};
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 == 0.0) continue;
                double f = (w ? w[j] : 1.0) * u[j + ny * m] / (4.0 * ORC_PI * r2 * sqrt(r2));
                for (int c = 0; c < 3; ++c) acc[c] -= f * d[c];
            }
            for (int c = 0; c < 3; ++c) v[s + nt * (3 * m + c)] = acc[c];
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------- octree */

static uint64_t spread_bits(uint64_t g)
{
    uint64_t r = 0;
    for (int b = 0; b < ORC_LMAX; ++b) r |= ((g >> b) & 1ULL) << (3 * b);
    return r;
}

static uint64_t gather_bits(uint64_t key)
{
    uint64_t r = 0;
    for (int b = 0; b < ORC_LMAX; ++b) r |= ((key >> (3 * b)) & 1ULL) << b;
    return r;
}

/* Morton key of integer coordinates (gx, gy, gz), 21 bits each: bit 3b+2 holds bit b
 * of gx, bit 3b+1 of gy, bit 3b of gz. */
uint64_t orc_morton(uint64_t gx, uint64_t gy, uint64_t gz)
{
    return (spread_bits(gx) << 2) | (spread_bits(gy) << 1) | spread_bits(gz);
}

typedef struct {
    int64_t n;
    double o[3];
    int64_t *perm; /* sorted position -> original index */
    uint64_t *key; /* Morton key per sorted position */
    double *p;     /* sorted coordinates, n*3 */
} otree;

typedef struct {
    uint64_t key;
    int64_t idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *u = (const keyidx *)a, *v = (const keyidx *)b;
    if (u->key < v->key) return -1;
    if (u->key > v->key) return 1;
    return (u->idx < v->idx) ? -1 : (u->idx > v->idx);
}

/* Integer coordinate of x on the finest grid (level 21) of a cube with corner o and
 * edge d0: floor(((x - o)/d0) * 2^21) in FP64, clamped to [0, 2^21 - 1]. The box
 * coordinate at level l is this value shifted right by 21 - l, which equals
 * floor(((x - o)/d0) * 2^l) because the scaling by a power of two is exact. */
static uint64_t fine_coord(double x, double o, double d0)
{
    double t = (x - o) / d0;
    double f = floor(ldexp(t, ORC_LMAX));
    if (f < 0.0) f = 0.0;
    double mx = ldexp(1.0, ORC_LMAX) - 1.0;
    if (f > mx) f = mx;
    return (uint64_t)f;
}

static int tree_build(otree *t, const double *P, int64_t n, const double o[3], double d0)
{
    t->n = n;
    memcpy(t->o, o, sizeof(double) * 3);
    t->perm = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    t->p = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * (n > 0 ? n : 1));
    if (!t->perm || !t->key || !t->p || !ki) {
        free(ki);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        uint64_t g0 = fine_coord(P[3 * i], o[0], d0);
        uint64_t g1 = fine_coord(P[3 * i + 1], o[1], d0);
        uint64_t g2 = fine_coord(P[3 * i + 2], o[2], d0);
        ki[i].key = orc_morton(g0, g1, g2);
        ki[i].idx = i;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int64_t s = 0; s < n; ++s) {
        t->perm[s] = ki[s].idx;
        t->key[s] = ki[s].key;
        memcpy(t->p + 3 * s, P + 3 * ki[s].idx, sizeof(double) * 3);
    }
    free(ki);
    return ORC_OK;
}

static void tree_free(otree *t)
{
    free(t->perm);
    free(t->key);
    free(t->p);
}

/* A box at level l: sorted range [s, e), box id = key >> 3(21-l), integer coords g. */
typedef struct {
    int64_t s, e;
    uint64_t id;
    int64_t g[3];
    int64_t c0, c1; /* children range in the next level's box list */
} obox;

static obox *boxes_at(const otree *t, int l, int64_t *nb)
{
    int sh = 3 * (ORC_LMAX - l);
    int64_t cnt = 0;
    for (int64_t s = 0; s < t->n; ++s)
        if (s == 0 || (t->key[s] >> sh) != (t->key[s - 1] >> sh)) ++cnt;
    obox *b = (obox *)calloc((size_t)(cnt > 0 ? cnt : 1), sizeof(obox));
    if (!b) return NULL;
    int64_t c = -1;
    for (int64_t s = 0; s < t->n; ++s) {
        uint64_t id = t->key[s] >> sh;
        if (s == 0 || id != (t->key[s - 1] >> sh)) {
            ++c;
            b[c].s = s;
            b[c].id = id;
            uint64_t full = id << sh;
            b[c].g[0] = (int64_t)(gather_bits(full >> 2) >> (ORC_LMAX - l));
            b[c].g[1] = (int64_t)(gather_bits(full >> 1) >> (ORC_LMAX - l));
            b[c].g[2] = (int64_t)(gather_bits(full) >> (ORC_LMAX - l));
        }
        b[c].e = s + 1;
    }
    *nb = cnt;
    return b;
}

/* Link each parent box to its children range in the child list (ids sorted). */
static void link_children(obox *par, int64_t np, obox *ch, int64_t nc)
{
    int64_t j = 0;
    for (int64_t i = 0; i < np; ++i) {
        while (j < nc && (ch[j].id >> 3) < par[i].id) ++j;
        par[i].c0 = j;
        while (j < nc && (ch[j].id >> 3) == par[i].id) ++j;
        par[i].c1 = j;
    }
}

/* Admissibility (Sec. 2.2.2) on the max-norm, non-strict: with sigma = (oX - oY)/d0 and
 * integer offset m = gX - gY at level l, the centre offset in units of d_l is
 * sigma*2^l + m; the pair is compressible iff some component has |.| >= 2. */
int orc_admissible(const double sigma[3], int l, const int64_t m[3])
{
    for (int d = 0; d < 3; ++d) {
        double t = fabs(ldexp(sigma[d], l) + (double)m[d]);
        if (t >= 2.0) return 1;
    }
    return 0;
}

/* ------------------------------------------------- Lagrange (Sec. 2.2.2) */

/* Calibrated worst-pair errors of the tensor Chebyshev-Lagrange interpolation, per r1,
 * for the Laplace kernel and for the Helmholtz kernel at k d = 2 (the oscillation
 * switch). Index r1 = 2..10. The rule picks the smallest r1 whose error is <= eps. The
 * values come from orc_lagrange_block_err (see oracle/calibrate_r1.py), rounded up. */
static const double ORC_R1_ERR_LAPLACE[11] = {1, 1, 3.2e-2, 4.8e-3, 7.6e-4, 1.1e-4, 1.6e-5, 2.0e-6, 2.4e-7, 8.1e-8, 1.1e-8};
static const double ORC_R1_ERR_HELM[11] = {1, 1, 2.4e-1, 3.4e-2, 3.6e-3, 3.6e-4, 4.0e-5, 3.9e-6, 3.9e-7, 1.3e-7, 1.4e-8};
static const double ORC_R1_ERR_LAPLACE_DL[11] = {1, 1, 1.2e-1, 2.4e-2, 5.1e-3, 1.1e-3, 1.8e-4, 2.6e-5, 3.9e-6, 1.5e-6, 2.0e-7};

static const double *r1_table(int kind)
{
    /* the gradient's component kernels dG/dx_d = -(x - y)_d / (4 pi |x - y|^3) are the double
     * layer's up to sign: same interpolation error, same table */
    return kind == ORC_HELMHOLTZ ? ORC_R1_ERR_HELM
           : (kind == ORC_LAPLACE_DL || kind == ORC_LAPLACE_GRAD) ? ORC_R1_ERR_LAPLACE_DL
                                                                  : ORC_R1_ERR_LAPLACE;
}

int orc_r1_rule(int kind, double eps)
{
    const double *tab = r1_table(kind);
    for (int r1 = 2; r1 <= 10; ++r1)
        if (tab[r1] <= eps) return r1;
    return 10;
}

void orc_r1_table(int kind, double *out11)
{
    memcpy(out11, r1_table(kind), sizeof(double) * 11);
}

/* First-kind Chebyshev nodes t_a = cos((2a+1) pi / (2 r1)). */
static void cheb_nodes(int r1, double *t)
{
    for (int a = 0; a < r1; ++a) t[a] = cos((2.0 * a + 1.0) * ORC_PI / (2.0 * r1));
}

/* 1-D Lagrange polynomials at the nodes t, evaluated at xi (product form). */
static void lagrange_1d(int r1, const double *t, double xi, double *l)
{
    for (int a = 0; a < r1; ++a) {
        double v = 1.0;
        for (int b = 0; b < r1; ++b)
            if (b != a) v *= (xi - t[b]) / (t[a] - t[b]);
        l[a] = v;
    }
}

/* Tensor basis L_{abc}(x) at a point x in the box of centre c and edge d; index
 * (a*r1 + b)*r1 + c over axes x, y, z. */
static void lagrange_3d(int r1, const double *t, const double *x, const double *c, double d, double *L)
{
    double lx[16], ly[16], lz[16];
    lagrange_1d(r1, t, (x[0] - c[0]) / (0.5 * d), lx);
    lagrange_1d(r1, t, (x[1] - c[1]) / (0.5 * d), ly);
    lagrange_1d(r1, t, (x[2] - c[2]) / (0.5 * d), lz);
    for (int a = 0; a < r1; ++a)
        for (int b = 0; b < r1; ++b)
            for (int e = 0; e < r1; ++e) L[(a * r1 + b) * r1 + e] = lx[a] * ly[b] * lz[e];
}

/* Relative Frobenius error of the Lagrange approximation L_X^T T L_Y of the kernel
 * block between two boxes of edge d whose centres differ by (2d, 0, 0) (the closest
 * admissible pair), sampled on a 6x6x6 grid of points in each box. */
double orc_lagrange_block_err(int kind, double k, int r1, double d)
{
    int ng = 6, np = ng * ng * ng, r = r1 * r1 * r1;
    double t[16];
    cheb_nodes(r1, t);
    double cx[3] = {2.0 * d, 0.0, 0.0}, cy[3] = {0.0, 0.0, 0.0};
    /* the double layer n . grad_y G is three interpolated component kernels dG/dy_e,
     * weighted by the source's normal (a fixed unit vector per sample point) */
    int nc = kind == ORC_LAPLACE_DL ? 3 : 1;
    double *px = (double *)malloc(sizeof(double) * 3 * np), *py = (double *)malloc(sizeof(double) * 3 * np);
    double *nj = (double *)malloc(sizeof(double) * 3 * np);
    double *LX = (double *)malloc(sizeof(double) * np * r), *LY = (double *)malloc(sizeof(double) * np * r);
    double *Tr = (double *)malloc(sizeof(double) * r * r), *Ti = (double *)malloc(sizeof(double) * r * r);
    double *Mr = (double *)malloc(sizeof(double) * np * r), *Mi = (double *)malloc(sizeof(double) * np * r);
    double *Ar = (double *)calloc((size_t)np * np, sizeof(double)), *Ai = (double *)calloc((size_t)np * np, sizeof(double));
    int q = 0;
    for (int a = 0; a < ng; ++a)
        for (int b = 0; b < ng; ++b)
            for (int e = 0; e < ng; ++e, ++q) {
                double o[3] = {((a + 0.5) / ng - 0.5) * d, ((b + 0.5) / ng - 0.5) * d, ((e + 0.5) / ng - 0.5) * d};
                for (int dd = 0; dd < 3; ++dd) {
                    px[3 * q + dd] = cx[dd] + o[dd];
                    py[3 * q + dd] = cy[dd] + o[dd] * 0.93;
                }
            }
    for (int jj = 0; jj < np; ++jj) {
        double v[3] = {sin(1.3 * jj + 0.2), cos(2.1 * jj), sin(0.7 * jj + 1.0)};
        double nn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        for (int dd = 0; dd < 3; ++dd) nj[3 * jj + dd] = v[dd] / nn;
    }
    for (int i = 0; i < np; ++i) {
        lagrange_3d(r1, t, px + 3 * i, cx, d, LX + (size_t)i * r);
        lagrange_3d(r1, t, py + 3 * i, cy, d, LY + (size_t)i * r);
    }
    for (int comp = 0; comp < nc; ++comp) {
        for (int a = 0; a < r; ++a) {
            int ax = a / (r1 * r1), ay = (a / r1) % r1, az = a % r1;
            double xc[3] = {cx[0] + t[ax] * 0.5 * d, cx[1] + t[ay] * 0.5 * d, cx[2] + t[az] * 0.5 * d};
            for (int b = 0; b < r; ++b) {
                int bx = b / (r1 * r1), by = (b / r1) % r1, bz = b % r1;
                double yc[3] = {cy[0] + t[bx] * 0.5 * d, cy[1] + t[by] * 0.5 * d, cy[2] + t[bz] * 0.5 * d};
                double dd[3] = {xc[0] - yc[0], xc[1] - yc[1], xc[2] - yc[2]};
                if (kind == ORC_LAPLACE_DL) {
                    double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                    Tr[a * r + b] = dd[comp] / (4.0 * ORC_PI * r2 * sqrt(r2));
                    Ti[a * r + b] = 0.0;
                } else {
                    orc_kernel(kind, k, dd[0], dd[1], dd[2], &Tr[a * r + b], &Ti[a * r + b]);
                }
            }
        }
        /* M = T L_Y^T  (r x np), then approx(i,j) += w_j sum_a LX[i,a] M[a,j] */
        for (int a = 0; a < r; ++a)
            for (int jj = 0; jj < np; ++jj) {
                double sr = 0, si = 0;
                for (int b = 0; b < r; ++b) {
                    sr += Tr[a * r + b] * LY[(size_t)jj * r + b];
                    si += Ti[a * r + b] * LY[(size_t)jj * r + b];
                }
                Mr[(size_t)a * np + jj] = sr;
                Mi[(size_t)a * np + jj] = si;
            }
        for (int i = 0; i < np; ++i)
            for (int jj = 0; jj < np; ++jj) {
                double sr = 0, si = 0;
                for (int a = 0; a < r; ++a) {
                    sr += LX[(size_t)i * r + a] * Mr[(size_t)a * np + jj];
                    si += LX[(size_t)i * r + a] * Mi[(size_t)a * np + jj];
                }
                double wgt = kind == ORC_LAPLACE_DL ? nj[3 * jj + comp] : 1.0;
                Ar[(size_t)i * np + jj] += wgt * sr;
                Ai[(size_t)i * np + jj] += wgt * si;
            }
    }
    double num = 0, den = 0;
    for (int i = 0; i < np; ++i)
        for (int jj = 0; jj < np; ++jj) {
            double gr, gi;
            double dx = px[3 * i] - py[3 * jj], dy = px[3 * i + 1] - py[3 * jj + 1], dz = px[3 * i + 2] - py[3 * jj + 2];
            if (kind == ORC_LAPLACE_DL) {
                double r2 = dx * dx + dy * dy + dz * dz;
                gr = (nj[3 * jj] * dx + nj[3 * jj + 1] * dy + nj[3 * jj + 2] * dz) / (4.0 * ORC_PI * r2 * sqrt(r2));
                gi = 0.0;
            } else {
                orc_kernel(kind, k, dx, dy, dz, &gr, &gi);
            }
            double sr = Ar[(size_t)i * np + jj], si = Ai[(size_t)i * np + jj];
            num += (sr - gr) * (sr - gr) + (si - gi) * (si - gi);
            den += gr * gr + gi * gi;
        }
    free(px);
    free(py);
    free(nj);
    free(LX);
    free(LY);
    free(Tr);
    free(Ti);
    free(Mr);
    free(Mi);
    free(Ar);
    free(Ai);
    return sqrt(num / den);
}

/* ---------------------------------------------- plane waves (Sec. 2.2.3) */

/* Gauss-Legendre nodes (ascending) and weights on [-1, 1], Newton on P_n. */
void orc_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* Rank L of eq. 13 with the natural logarithm; at least 1. */
int orc_pw_rank(double k, double dl, double eps)
{
    int L = (int)floor(fabs(k) * sqrt(3.0) * dl - log(eps));
    return L < 1 ? 1 : L;
}

/* Quadrature of eq. 17: direction q = i*(2L) + j, cos(theta_i) the i-th Gauss-Legendre
 * node of order L+1 (ascending), phi_j = j*pi/L; weight w_i * pi/L. s: nQ*3. */
void orc_sphere_quad(int L, double *s, double *w)
{
    int nt = L + 1, np = 2 * L;
    double *mu = (double *)malloc(sizeof(double) * nt), *wg = (double *)malloc(sizeof(double) * nt);
    orc_gauss_legendre(nt, mu, wg);
    for (int i = 0; i < nt; ++i) {
        double st = sqrt(1.0 - mu[i] * mu[i]);
        for (int j = 0; j < np; ++j) {
            int q = i * np + j;
            double ph = j * ORC_PI / L;
            s[3 * q] = st * cos(ph);
            s[3 * q + 1] = st * sin(ph);
            s[3 * q + 2] = mu[i];
            w[q] = wg[i] * ORC_PI / L;
        }
    }
    free(mu);
    free(wg);
}

/* Spherical Hankel functions h_p^(1)(z), p = 0..L, by upward recurrence from
 * h_0 = -i e^{iz}/z and h_1 = -e^{iz}(z + i)/z^2. */
void orc_hankel(int L, double z, double *hr, double *hi)
{
    double c = cos(z), s = sin(z);
    hr[0] = s / z;
    hi[0] = -c / z;
    if (L >= 1) {
        hr[1] = (-c * z + s) / (z * z);
        hi[1] = (-s * z - c) / (z * z);
    }
    for (int p = 1; p < L; ++p) {
        double f = (2.0 * p + 1.0) / z;
        hr[p + 1] = f * hr[p] - hr[p - 1];
        hi[p + 1] = f * hi[p] - hi[p - 1];
    }
}

/* Gegenbauer transfer function of eq. 12 summed from p = 0:
 * T(s) = sum_{p=0}^{L} (2p+1) i^p h_p(k|r0|) P_p(s . r0/|r0|) / (4 pi). hr/hi precomputed. */
static void gegenbauer_T(int L, const double *hr, const double *hi, double cosg, double *tr, double *ti)
{
    double p0 = 1.0, p1 = cosg;
    double ar = 0.0, ai = 0.0;
    for (int p = 0; p <= L; ++p) {
        double P = (p == 0) ? 1.0 : (p == 1 ? cosg : 0.0);
        if (p >= 2) {
            double p2 = ((2.0 * p - 1.0) * cosg * p1 - (p - 1.0) * p0) / p;
            p0 = p1;
            p1 = p2;
            P = p2;
        }
        /* i^p */
        double ipr = (p % 4 == 0) ? 1.0 : ((p % 4 == 2) ? -1.0 : 0.0);
        double ipi = (p % 4 == 1) ? 1.0 : ((p % 4 == 3) ? -1.0 : 0.0);
        double cr = (2.0 * p + 1.0) * (ipr * hr[p] - ipi * hi[p]);
        double ci = (2.0 * p + 1.0) * (ipr * hi[p] + ipi * hr[p]);
        ar += cr * P;
        ai += ci * P;
    }
    *tr = ar / (4.0 * ORC_PI);
    *ti = ai / (4.0 * ORC_PI);
}

void orc_gegenbauer(double k, const double r0[3], int L, const double s[3], double *tr, double *ti)
{
    double R = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    double *hr = (double *)malloc(sizeof(double) * (L + 1)), *hi = (double *)malloc(sizeof(double) * (L + 1));
    orc_hankel(L, k * R, hr, hi);
    double cg = (s[0] * r0[0] + s[1] * r0[1] + s[2] * r0[2]) / R;
    gegenbauer_T(L, hr, hi, cg, tr, ti);
    free(hr);
    free(hi);
}

/* Single-pair plane-wave approximation of e^{ik|x-y|}/(4 pi |x-y|) (eqs. 10-16):
 * (1/4pi) ik sum_q w_q T(s_q) e^{ik s_q.(x - x0)} e^{-ik s_q.(y - y0)}. */
void orc_pw_pair(double k, int L, const double x[3], const double y[3], const double x0[3], const double y0[3],
                 double *gr, double *gi)
{
    int nq = 2 * L * (L + 1);
    double *s = (double *)malloc(sizeof(double) * 3 * nq), *w = (double *)malloc(sizeof(double) * nq);
    double *hr = (double *)malloc(sizeof(double) * (L + 1)), *hi = (double *)malloc(sizeof(double) * (L + 1));
    orc_sphere_quad(L, s, w);
    double r0[3] = {x0[0] - y0[0], x0[1] - y0[1], x0[2] - y0[2]};
    double R = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    orc_hankel(L, k * R, hr, hi);
    double ar = 0, ai = 0;
    for (int q = 0; q < nq; ++q) {
        const double *sq = s + 3 * q;
        double tr, ti;
        gegenbauer_T(L, hr, hi, (sq[0] * r0[0] + sq[1] * r0[1] + sq[2] * r0[2]) / R, &tr, &ti);
        double ph = k * (sq[0] * (x[0] - x0[0]) + sq[1] * (x[1] - x0[1]) + sq[2] * (x[2] - x0[2]))
                    - k * (sq[0] * (y[0] - y0[0]) + sq[1] * (y[1] - y0[1]) + sq[2] * (y[2] - y0[2]));
        double er = cos(ph), ei = sin(ph);
        /* ik * w * T * e */
        double ar1 = w[q] * (tr * er - ti * ei), ai1 = w[q] * (tr * ei + ti * er);
        ar += -k * ai1;
        ai += k * ar1;
    }
    *gr = ar / (4.0 * ORC_PI);
    *gi = ai / (4.0 * ORC_PI);
    free(s);
    free(w);
    free(hr);
    free(hi);
}

/* ---------------------------------------------------------------- the plan */

typedef struct {
    int n_leaf;
    int l_cap;
    double kappa_switch;
    int r1_override; /* 0: rule */
    int mode_override; /* 0: auto, 1: Lagrange everywhere, 2: plane waves everywhere */
    int pw_transform;  /* plane-wave steps F: 0 direct sums, 1 type-3 NUFFT (nufft_oracle.c) */
    double aca_eps;    /* > 0: Laplace Lagrange transfers as ACA factors A B^T (eq. 11) */
} orc_opts;

typedef struct {
    int l_stop;
    int root_admissible;
    double d0;
    double oX[3], oY[3];
    int64_t nboxX[ORC_LMAX + 1], nboxY[ORC_LMAX + 1];
    int64_t n_adm[ORC_LMAX + 1], n_near[ORC_LMAX + 1];
    int64_t n_trans[ORC_LMAX + 1];
    int mode[ORC_LMAX + 1];
    int r1[ORC_LMAX + 1];
    int L[ORC_LMAX + 1];
    int nQ[ORC_LMAX + 1];
    int aca_rank[ORC_LMAX + 1]; /* with aca_eps: largest ACA rank over the level's translations */
} orc_stats;

typedef struct {
    int64_t a, b;
} opair;

typedef struct {
    otree tx, ty;
    int kind;
    double k, eps;
    orc_opts opt;
    orc_stats st;
    double d0, sigma[3];
    obox *bx[ORC_LMAX + 1], *by[ORC_LMAX + 1];
    int64_t nbx[ORC_LMAX + 1], nby[ORC_LMAX + 1];
    opair *adm[ORC_LMAX + 1];
    opair *nearp; /* near pairs at l_stop */
    int64_t n_nearp;
} orc_plan;

static int cmp_pair(const void *a, const void *b)
{
    const opair *u = (const opair *)a, *v = (const opair *)b;
    if (u->a != v->a) return (u->a < v->a) ? -1 : 1;
    if (u->b != v->b) return (u->b < v->b) ? -1 : 1;
    return 0;
}

static void bbox(const double *P, int64_t n, double lo[3], double hi[3])
{
    for (int d = 0; d < 3; ++d) {
        lo[d] = P[d];
        hi[d] = P[d];
    }
    for (int64_t i = 1; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            if (P[3 * i + d] < lo[d]) lo[d] = P[3 * i + d];
            if (P[3 * i + d] > hi[d]) hi[d] = P[3 * i + d];
        }
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t u = *(const uint64_t *)a, v = *(const uint64_t *)b;
    return (u < v) ? -1 : (u > v);
}

static int64_t count_translations(const opair *pr, int64_t n, const obox *bx, const obox *by)
{
    if (n == 0) return 0;
    uint64_t *code = (uint64_t *)malloc(sizeof(uint64_t) * n);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t c = 0;
        for (int d = 0; d < 3; ++d) c = (c << 21) | (uint64_t)((bx[pr[i].a].g[d] - by[pr[i].b].g[d]) + (1 << 20));
        code[i] = c;
    }
    qsort(code, (size_t)n, sizeof(uint64_t), cmp_u64);
    int64_t u = 1;
    for (int64_t i = 1; i < n; ++i)
        if (code[i] != code[i - 1]) ++u;
    free(code);
    return u;
}

void orc_default_opts(orc_opts *o)
{
    o->n_leaf = 64;
    o->l_cap = ORC_LMAX;
    o->kappa_switch = 2.0;
    o->r1_override = 0;
    o->mode_override = 0;
    o->pw_transform = 0;
    o->aca_eps = 0.0;
}

static int level_mode(const orc_plan *p, int l)
{
    double dl = ldexp(p->d0, -l);
    if (p->opt.mode_override == 1) return ORC_MODE_LAGRANGE;
    if (p->opt.mode_override == 2) return ORC_MODE_PLANEWAVE;
    if (p->kind == ORC_HELMHOLTZ && p->k * dl >= p->opt.kappa_switch) return ORC_MODE_PLANEWAVE;
    return ORC_MODE_LAGRANGE;
}

void orc_plan_destroy(orc_plan *p)
{
    if (!p) return;
    tree_free(&p->tx);
    tree_free(&p->ty);
    for (int l = 0; l <= ORC_LMAX; ++l) {
        free(p->bx[l]);
        free(p->by[l]);
        free(p->adm[l]);
    }
    free(p->nearp);
    free(p);
}

static int level_aca_rank(const orc_plan *p, int l);

/* Build both trees and the per-level pair lists (Sec. 2.2.1, 2.2.2, 2.2.4). */
orc_plan *orc_plan_create(const double *X, int64_t nx, const double *Y, int64_t ny, int kind, double k,
                          double eps, const orc_opts *opts)
{
    if (nx < 1 || ny < 1 || !(eps > 0.0 && eps < 1.0) || k < 0.0) return NULL;
    orc_plan *p = (orc_plan *)calloc(1, sizeof(orc_plan));
    if (!p) return NULL;
    p->kind = kind;
    p->k = k;
    p->eps = eps;
    if (opts)
        p->opt = *opts;
    else
        orc_default_opts(&p->opt);

    /* Root cubes (Sec. 2.2.1): common edge d0 = max over both sets of the largest
     * extent, inflated by 2^-20; each cube centred on its set's tight box. */
    double lx[3], hx[3], ly[3], hy[3];
    bbox(X, nx, lx, hx);
    bbox(Y, ny, ly, hy);
    double ex = 0, ey = 0;
    for (int d = 0; d < 3; ++d) {
        if (hx[d] - lx[d] > ex) ex = hx[d] - lx[d];
        if (hy[d] - ly[d] > ey) ey = hy[d] - ly[d];
    }
    double d0 = (ex > ey ? ex : ey);
    d0 = (d0 > 0.0) ? d0 * (1.0 + ldexp(1.0, -20)) : 1.0;
    double oX[3], oY[3];
    for (int d = 0; d < 3; ++d) {
        oX[d] = 0.5 * (lx[d] + hx[d]) - 0.5 * d0;
        oY[d] = 0.5 * (ly[d] + hy[d]) - 0.5 * d0;
        p->sigma[d] = (oX[d] - oY[d]) / d0;
    }
    p->d0 = d0;
    p->st.d0 = d0;
    memcpy(p->st.oX, oX, sizeof oX);
    memcpy(p->st.oY, oY, sizeof oY);
    if (tree_build(&p->tx, X, nx, oX, d0) || tree_build(&p->ty, Y, ny, oY, d0)) {
        orc_plan_destroy(p);
        return NULL;
    }

    /* Level 0 */
    p->bx[0] = boxes_at(&p->tx, 0, &p->nbx[0]);
    p->by[0] = boxes_at(&p->ty, 0, &p->nby[0]);
    p->st.nboxX[0] = p->nbx[0];
    p->st.nboxY[0] = p->nby[0];
    int64_t m0[3] = {0, 0, 0};
    opair *near = (opair *)malloc(sizeof(opair));
    int64_t nnear = 1;
    near[0].a = 0;
    near[0].b = 0;
    p->st.l_stop = 0;
    if (orc_admissible(p->sigma, 0, m0)) {
        p->adm[0] = near;
        p->st.n_adm[0] = 1;
        p->st.n_trans[0] = 1;
        p->st.mode[0] = level_mode(p, 0);
        p->st.root_admissible = 1;
        p->nearp = NULL;
        p->n_nearp = 0;
        goto annotate;
    }
    p->st.n_near[0] = 1;
    for (int l = 0;; ++l) {
        int stop = (nnear == 0) || ((nx + ny) < (int64_t)p->opt.n_leaf * (p->nbx[l] + p->nby[l])) ||
                   (l >= p->opt.l_cap);
        if (stop) {
            p->st.l_stop = l;
            p->nearp = near;
            p->n_nearp = nnear;
            break;
        }
        int lc = l + 1;
        p->bx[lc] = boxes_at(&p->tx, lc, &p->nbx[lc]);
        p->by[lc] = boxes_at(&p->ty, lc, &p->nby[lc]);
        p->st.nboxX[lc] = p->nbx[lc];
        p->st.nboxY[lc] = p->nby[lc];
        link_children(p->bx[l], p->nbx[l], p->bx[lc], p->nbx[lc]);
        link_children(p->by[l], p->nby[l], p->by[lc], p->nby[lc]);
        int64_t ncand = 0;
        for (int64_t i = 0; i < nnear; ++i) {
            const obox *A = &p->bx[l][near[i].a], *B = &p->by[l][near[i].b];
            ncand += (A->c1 - A->c0) * (B->c1 - B->c0);
        }
        opair *adm = (opair *)malloc(sizeof(opair) * (ncand > 0 ? ncand : 1));
        opair *nn = (opair *)malloc(sizeof(opair) * (ncand > 0 ? ncand : 1));
        int64_t na = 0, nb = 0;
        for (int64_t i = 0; i < nnear; ++i) {
            const obox *A = &p->bx[l][near[i].a], *B = &p->by[l][near[i].b];
            for (int64_t ca = A->c0; ca < A->c1; ++ca)
                for (int64_t cb = B->c0; cb < B->c1; ++cb) {
                    int64_t m[3];
                    for (int d = 0; d < 3; ++d) m[d] = p->bx[lc][ca].g[d] - p->by[lc][cb].g[d];
                    opair q = {ca, cb};
                    if (orc_admissible(p->sigma, lc, m))
                        adm[na++] = q;
                    else
                        nn[nb++] = q;
                }
        }
        free(near);
        near = nn;
        nnear = nb;
        qsort(adm, (size_t)na, sizeof(opair), cmp_pair);
        qsort(near, (size_t)nnear, sizeof(opair), cmp_pair);
        p->adm[lc] = adm;
        p->st.n_adm[lc] = na;
        p->st.n_near[lc] = nnear;
        p->st.n_trans[lc] = count_translations(adm, na, p->bx[lc], p->by[lc]);
        p->st.mode[lc] = na > 0 ? level_mode(p, lc) : ORC_MODE_NONE;
    }
annotate:
    for (int l = 0; l <= ORC_LMAX; ++l) {
        if (p->st.n_adm[l] == 0) continue;
        double dl = ldexp(d0, -l);
        if (p->st.mode[l] == ORC_MODE_LAGRANGE) {
            p->st.r1[l] = p->opt.r1_override > 0 ? p->opt.r1_override : orc_r1_rule(kind, eps);
            if (p->opt.aca_eps > 0.0 && kind == ORC_LAPLACE) p->st.aca_rank[l] = level_aca_rank(p, l);
        } else {
            p->st.L[l] = orc_pw_rank(k, dl, eps);
            p->st.nQ[l] = 2 * p->st.L[l] * (p->st.L[l] + 1);
        }
    }
    return p;
}

void orc_plan_stats(const orc_plan *p, orc_stats *s) { *s = p->st; }

/* Pairs of a level as Morton box ids (level l): which = 0 admissible pairs at level l,
 * 1 near pairs at the stop level (l ignored). Returns the count; fills idX/idY if
 * non-NULL. */
int64_t orc_plan_pairs(const orc_plan *p, int l, int which, uint64_t *idX, uint64_t *idY)
{
    const opair *pr;
    int64_t n;
    int lev;
    if (which == 0) {
        if (l < 0 || l > ORC_LMAX || !p->adm[l]) return 0;
        pr = p->adm[l];
        n = p->st.n_adm[l];
        lev = l;
    } else {
        pr = p->nearp;
        n = p->n_nearp;
        lev = p->st.l_stop;
    }
    if (idX && idY)
        for (int64_t i = 0; i < n; ++i) {
            idX[i] = p->bx[lev][pr[i].a].id;
            idY[i] = p->by[lev][pr[i].b].id;
        }
    return n;
}

/* Sorted permutation of a tree (which = 0 X, 1 Y): position -> original index. */
void orc_plan_perm(const orc_plan *p, int which, int64_t *out)
{
    const otree *t = which ? &p->ty : &p->tx;
    memcpy(out, t->perm, sizeof(int64_t) * t->n);
}

/* ------------------------------------------------------------- the apply */

static void box_centre(const double o[3], const int64_t g[3], double dl, double c[3])
{
    for (int d = 0; d < 3; ++d) c[d] = o[d] + ((double)g[d] + 0.5) * dl;
}

/* ------------------------------------------------ adaptive cross approximation */

#define ORC_ACA_KMAX 64

/* Adaptive cross approximation of a small explicit matrix (Sec. 2.2.2, eq. 11, after
 * Bebendorf), with full pivoting: M (nr x nc, row-major) ~ S_k = sum_{l<k} a_l b_l^T,
 * a_l = A + l nr, b_l = B + l nc.  Step k takes the residual R = M - S_k, its entry of
 * largest magnitude (i, j) (near-ties within a factor 1 - 1e-9 go to the first in
 * row-major order), a = R(:, j), b = R(i, :) / R(i, j), and subtracts a b^T from R.  It
 * stops once |R|_F <= tol |M|_F, at a zero residual, or after kmax terms.  Returns k. */
int orc_aca(const double *M, int nr, int nc, double tol, int kmax, double *A, double *B)
{
    size_t n = (size_t)nr * nc;
    double *R = (double *)malloc(sizeof(double) * n);
    memcpy(R, M, sizeof(double) * n);
    double m2 = 0.0;
    for (size_t e = 0; e < n; ++e) m2 += M[e] * M[e];
    int k = 0;
    while (k < kmax) {
        double mx = 0.0;
        for (size_t e = 0; e < n; ++e)
            if (fabs(R[e]) > mx) mx = fabs(R[e]);
        if (mx == 0.0) break;
        double thr = (1.0 - 1e-9) * mx;
        size_t piv = 0;
        while (fabs(R[piv]) < thr) ++piv;
        int i = (int)(piv / nc), j = (int)(piv % nc);
        double delta = R[piv];
        double *a = A + (size_t)k * nr, *b = B + (size_t)k * nc;
        for (int ii = 0; ii < nr; ++ii) a[ii] = R[(size_t)ii * nc + j];
        for (int jj = 0; jj < nc; ++jj) b[jj] = R[(size_t)i * nc + jj] / delta;
        double r2 = 0.0;
        for (int ii = 0; ii < nr; ++ii)
            for (int jj = 0; jj < nc; ++jj) {
                double v = R[(size_t)ii * nc + jj] - a[ii] * b[jj];
                R[(size_t)ii * nc + jj] = v;
                r2 += v * v;
            }
        ++k;
        if (r2 <= tol * tol * m2) break;
    }
    free(R);
    return k;
}

static double dot(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* T of the Laplace single layer between the control nodes of boxes with centres ca
 * (targets, rows i) and cb (sources, columns j), Sec. 2.2.2. */
static void laplace_T(int r1, const double *t, double dl, const double ca[3], const double cb[3], double *T)
{
    int r = r1 * r1 * r1;
    for (int i = 0; i < r; ++i) {
        int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
        for (int j = 0; j < r; ++j) {
            int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
            double dx = (ca[0] + t[ix] * 0.5 * dl) - (cb[0] + t[jx] * 0.5 * dl);
            double dy = (ca[1] + t[iy] * 0.5 * dl) - (cb[1] + t[jy] * 0.5 * dl);
            double dz = (ca[2] + t[iz] * 0.5 * dl) - (cb[2] + t[jz] * 0.5 * dl);
            double gi;
            orc_kernel(ORC_LAPLACE, 0.0, dx, dy, dz, &T[(size_t)i * r + j], &gi);
        }
    }
}

/* Largest ACA rank over the distinct translations of a Laplace Lagrange level (the first
 * pair of each translation, in sorted pair order). */
static int level_aca_rank(const orc_plan *p, int l)
{
    int64_t na = p->st.n_adm[l];
    int r1 = p->st.r1[l], r = r1 * r1 * r1, kmax = r < ORC_ACA_KMAX ? r : ORC_ACA_KMAX;
    double t[16], dl = ldexp(p->d0, -l);
    cheb_nodes(r1, t);
    keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * (size_t)na);
    for (int64_t e = 0; e < na; ++e) {
        uint64_t c = 0;
        for (int d = 0; d < 3; ++d)
            c = (c << 21) | (uint64_t)((p->bx[l][p->adm[l][e].a].g[d] - p->by[l][p->adm[l][e].b].g[d]) + (1 << 20));
        ki[e].key = c;
        ki[e].idx = e;
    }
    qsort(ki, (size_t)na, sizeof(keyidx), cmp_keyidx);
    int best = 0;
    double *T = (double *)malloc(sizeof(double) * r * r), *A = (double *)malloc(sizeof(double) * r * kmax),
           *B = (double *)malloc(sizeof(double) * r * kmax);
    for (int64_t e = 0; e < na; ++e) {
        if (e > 0 && ki[e].key == ki[e - 1].key) continue;
        const opair *pr = &p->adm[l][ki[e].idx];
        double ca[3], cb[3];
        box_centre(p->tx.o, p->bx[l][pr->a].g, dl, ca);
        box_centre(p->ty.o, p->by[l][pr->b].g, dl, cb);
        laplace_T(r1, t, dl, ca, cb, T);
        int k = orc_aca(T, r, r, p->opt.aca_eps, kmax, A, B);
        if (k > best) best = k;
    }
    free(T);
    free(A);
    free(B);
    free(ki);
    return best;
}

/* Far field of level l (Lagrange, Sec. 2.2.2): u~_b = L_Y(b) (w u)_b for every source
 * box, v~_a = sum_b T_ab u~_b with T_ab computed from its definition for each pair,
 * v_a += L_X(a)^T v~_a. acc: sorted-order accumulators (nx*nrhs). */
/* Far field of a Lagrange level (Sec. 2.2.2, eq. 8): source step L_Y (w u) per source
 * box, transfer T per admissible pair (kernel at the control nodes, evaluated for each
 * pair), target step L_X^T per target box.  With qv (double layer, 3-vector densities
 * w u n per source, qv[3 (j + ny m) + axis]) the kernel n_y . grad_y G is the sum over
 * the axes d of n_d dG/dy_d(x - y): each component kernel is interpolated on its own
 * (source step L_Y (w u n_d), transfer with dG/dy_d at the control nodes) and the three
 * results are added before the target step.  With aca_eps (Laplace single layer) each
 * pair's T is replaced by its ACA factors: v~_a += A (B^T u~_b) (eq. 11). */
static void far_lagrange(const orc_plan *p, int l, const double *qr, const double *qi, const double *qv, int nrhs,
                         double *accr, double *acci)
{
    int r1 = p->st.r1[l], r = r1 * r1 * r1;
    double t[16];
    cheb_nodes(r1, t);
    double dl = ldexp(p->d0, -l);
    int64_t nbY = p->nby[l], nbX = p->nbx[l];
    int64_t ny = p->ty.n, nx = p->tx.n;
    int nc = qv ? 3 : 1; /* kernel components */
    double *utr = (double *)calloc((size_t)nbY * nrhs * nc * r, sizeof(double));
    double *uti = (double *)calloc((size_t)nbY * nrhs * nc * r, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nbY; ++b) {
        const obox *B = &p->by[l][b];
        double c[3], Lb[1000];
        box_centre(p->ty.o, B->g, dl, c);
        for (int64_t j = B->s; j < B->e; ++j) {
            lagrange_3d(r1, t, p->ty.p + 3 * j, c, dl, Lb);
            if (qv) {
                for (int m = 0; m < nrhs; ++m)
                    for (int d = 0; d < 3; ++d)
                        for (int a = 0; a < r; ++a)
                            utr[(((size_t)b * nrhs + m) * 3 + d) * r + a] += Lb[a] * qv[3 * (j + ny * m) + d];
                continue;
            }
            for (int m = 0; m < nrhs; ++m)
                for (int a = 0; a < r; ++a) {
                    utr[((size_t)b * nrhs + m) * r + a] += Lb[a] * qr[j + ny * m];
                    uti[((size_t)b * nrhs + m) * r + a] += Lb[a] * qi[j + ny * m];
                }
        }
    }
    /* group admissible pairs by target box (they are sorted by (a, b)) */
    int64_t na = p->st.n_adm[l];
    const opair *adm = p->adm[l];
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (nbX + 1));
    {
        int64_t i = 0;
        for (int64_t a = 0; a <= nbX; ++a) {
            while (i < na && adm[i].a < a) ++i;
            first[a] = i;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < nbX; ++a) {
        if (first[a] == first[a + 1]) continue;
        const obox *A = &p->bx[l][a];
        double ca[3];
        box_centre(p->tx.o, A->g, dl, ca);
        double *vtr = (double *)calloc((size_t)nrhs * r, sizeof(double));
        double *vti = (double *)calloc((size_t)nrhs * r, sizeof(double));
        double *Tr = (double *)malloc(sizeof(double) * r * r), *Ti = (double *)malloc(sizeof(double) * r * r);
        const int aca = p->opt.aca_eps > 0.0 && p->kind == ORC_LAPLACE && !qv;
        const int kmax = r < ORC_ACA_KMAX ? r : ORC_ACA_KMAX;
        double *Aa = aca ? (double *)malloc(sizeof(double) * r * kmax) : NULL;
        double *Ba = aca ? (double *)malloc(sizeof(double) * r * kmax) : NULL;
        for (int64_t e = first[a]; e < first[a + 1]; ++e)
          for (int d = 0; d < nc; ++d) {
            int64_t b = adm[e].b;
            double cb[3];
            box_centre(p->ty.o, p->by[l][b].g, dl, cb);
            for (int i = 0; i < r; ++i) {
                int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
                double xc[3] = {ca[0] + t[ix] * 0.5 * dl, ca[1] + t[iy] * 0.5 * dl, ca[2] + t[iz] * 0.5 * dl};
                for (int j = 0; j < r; ++j) {
                    int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
                    double yc[3] = {cb[0] + t[jx] * 0.5 * dl, cb[1] + t[jy] * 0.5 * dl, cb[2] + t[jz] * 0.5 * dl};
                    double dd[3] = {xc[0] - yc[0], xc[1] - yc[1], xc[2] - yc[2]};
                    if (qv) {
                        /* dG/dy_d = (x - y)_d / (4 pi |x - y|^3) */
                        double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                        Tr[i * r + j] = dd[d] / (4.0 * ORC_PI * r2 * sqrt(r2));
                        Ti[i * r + j] = 0.0;
                    } else {
                        orc_kernel(p->kind, p->k, dd[0], dd[1], dd[2], &Tr[i * r + j], &Ti[i * r + j]);
                    }
                }
            }
            if (aca) {
                int kk = orc_aca(Tr, r, r, p->opt.aca_eps, kmax, Aa, Ba);
                for (int m = 0; m < nrhs; ++m) {
                    const double *ur = utr + ((size_t)b * nrhs + m) * r;
                    for (int q = 0; q < kk; ++q) {
                        double s = dot(Ba + (size_t)q * r, ur, r); /* B^T u~ */
                        for (int i = 0; i < r; ++i) vtr[m * r + i] += Aa[(size_t)q * r + i] * s;
                    }
                }
                continue;
            }
            for (int m = 0; m < nrhs; ++m) {
                const double *ur = utr + (((size_t)b * nrhs + m) * nc + d) * r, *ui = uti + (((size_t)b * nrhs + m) * nc + d) * r;
                for (int i = 0; i < r; ++i) {
                    double sr = 0, si = 0;
                    for (int j = 0; j < r; ++j) {
                        sr += Tr[i * r + j] * ur[j] - Ti[i * r + j] * ui[j];
                        si += Tr[i * r + j] * ui[j] + Ti[i * r + j] * ur[j];
                    }
                    vtr[m * r + i] += sr;
                    vti[m * r + i] += si;
                }
            }
        }
        double La[1000];
        for (int64_t i = A->s; i < A->e; ++i) {
            lagrange_3d(r1, t, p->tx.p + 3 * i, ca, dl, La);
            for (int m = 0; m < nrhs; ++m) {
                double sr = 0, si = 0;
                for (int q = 0; q < r; ++q) {
                    sr += La[q] * vtr[m * r + q];
                    si += La[q] * vti[m * r + q];
                }
                accr[i + nx * m] += sr;
                acci[i + nx * m] += si;
            }
        }
        free(vtr);
        free(vti);
        free(Tr);
        free(Ti);
        free(Aa);
        free(Ba);
    }
    free(first);
    free(utr);
    free(uti);
}

/* Far field of level l (plane waves, Sec. 2.2.3): forward transform per source box,
 * diagonal Gegenbauer transfer per pair (evaluated from eq. 12 for each pair), backward
 * transform per target box. */
static void far_planewave(const orc_plan *p, int l, const double *qr, const double *qi, int nrhs, double *accr,
                          double *acci)
{
    int L = p->st.L[l], nq = p->st.nQ[l];
    double k = p->k;
    double dl = ldexp(p->d0, -l);
    double *s = (double *)malloc(sizeof(double) * 3 * nq), *w = (double *)malloc(sizeof(double) * nq);
    orc_sphere_quad(L, s, w);
    int64_t nbY = p->nby[l], nbX = p->nbx[l], ny = p->ty.n, nx = p->tx.n;
    double *utr = (double *)calloc((size_t)nbY * nrhs * nq, sizeof(double));
    double *uti = (double *)calloc((size_t)nbY * nrhs * nq, sizeof(double));
    int64_t na = p->st.n_adm[l];
    const opair *adm = p->adm[l];
    char *used = (char *)calloc((size_t)nbY, 1);
    for (int64_t e = 0; e < na; ++e) used[adm[e].b] = 1;
    /* NUFFT mode: the same sums as below, through the type-3 NUFFT of one box at a time
     * (frequencies k s_q, points relative to the box centre) */
    const int nufft = p->opt.pw_transform == 1;
    double *ks = (double *)malloc(sizeof(double) * 3 * nq);
    for (int i = 0; i < 3 * nq; ++i) ks[i] = k * s[i];
    orc_nu nu;
    if (nufft) orc_nu_init(&nu, dl, k, p->eps, ks, nq);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nbY; ++b) {
        if (!used[b]) continue;
        if (nufft) {
            const obox *B = &p->by[l][b];
            double c[3];
            box_centre(p->ty.o, B->g, dl, c);
            int64_t nb = B->e - B->s;
            double *xr = (double *)malloc(sizeof(double) * 3 * (nb > 0 ? nb : 1));
            double *cr = (double *)malloc(sizeof(double) * (nb > 0 ? nb : 1));
            double *ci = (double *)malloc(sizeof(double) * (nb > 0 ? nb : 1));
            for (int64_t j = 0; j < nb; ++j)
                for (int d = 0; d < 3; ++d) xr[3 * j + d] = p->ty.p[3 * (B->s + j) + d] - c[d];
            for (int m = 0; m < nrhs; ++m) {
                for (int64_t j = 0; j < nb; ++j) {
                    cr[j] = qr[B->s + j + ny * m];
                    ci[j] = qi[B->s + j + ny * m];
                }
                orc_nu_forward(&nu, xr, nb, cr, ci, utr + ((size_t)b * nrhs + m) * nq, uti + ((size_t)b * nrhs + m) * nq);
            }
            free(xr);
            free(cr);
            free(ci);
            continue;
        }
        const obox *B = &p->by[l][b];
        double c[3];
        box_centre(p->ty.o, B->g, dl, c);
        for (int64_t j = B->s; j < B->e; ++j) {
            const double *y = p->ty.p + 3 * j;
            double d[3] = {y[0] - c[0], y[1] - c[1], y[2] - c[2]};
            for (int q = 0; q < nq; ++q) {
                double ph = -k * (s[3 * q] * d[0] + s[3 * q + 1] * d[1] + s[3 * q + 2] * d[2]);
                double er = cos(ph), ei = sin(ph);
                for (int m = 0; m < nrhs; ++m) {
                    double ur = qr[j + ny * m], ui = qi[j + ny * m];
                    utr[((size_t)b * nrhs + m) * nq + q] += er * ur - ei * ui;
                    uti[((size_t)b * nrhs + m) * nq + q] += er * ui + ei * ur;
                }
            }
        }
    }
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (nbX + 1));
    {
        int64_t i = 0;
        for (int64_t a = 0; a <= nbX; ++a) {
            while (i < na && adm[i].a < a) ++i;
            first[a] = i;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < nbX; ++a) {
        if (first[a] == first[a + 1]) continue;
        const obox *A = &p->bx[l][a];
        double ca[3];
        box_centre(p->tx.o, A->g, dl, ca);
        double *vtr = (double *)calloc((size_t)nrhs * nq, sizeof(double));
        double *vti = (double *)calloc((size_t)nrhs * nq, sizeof(double));
        double *hr = (double *)malloc(sizeof(double) * (L + 1)), *hi = (double *)malloc(sizeof(double) * (L + 1));
        for (int64_t e = first[a]; e < first[a + 1]; ++e) {
            int64_t b = adm[e].b;
            double cb[3];
            box_centre(p->ty.o, p->by[l][b].g, dl, cb);
            double r0[3] = {ca[0] - cb[0], ca[1] - cb[1], ca[2] - cb[2]};
            double R = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
            orc_hankel(L, k * R, hr, hi);
            for (int q = 0; q < nq; ++q) {
                double tr, ti;
                gegenbauer_T(L, hr, hi, (s[3 * q] * r0[0] + s[3 * q + 1] * r0[1] + s[3 * q + 2] * r0[2]) / R, &tr, &ti);
                /* D = ik w_q T */
                double dr = -k * w[q] * ti, di = k * w[q] * tr;
                for (int m = 0; m < nrhs; ++m) {
                    double ur = utr[((size_t)b * nrhs + m) * nq + q], ui = uti[((size_t)b * nrhs + m) * nq + q];
                    vtr[(size_t)m * nq + q] += dr * ur - di * ui;
                    vti[(size_t)m * nq + q] += dr * ui + di * ur;
                }
            }
        }
        if (nufft) {
            int64_t na_ = A->e - A->s;
            double *xr = (double *)malloc(sizeof(double) * 3 * (na_ > 0 ? na_ : 1));
            double *or_ = (double *)malloc(sizeof(double) * (na_ > 0 ? na_ : 1));
            double *oi = (double *)malloc(sizeof(double) * (na_ > 0 ? na_ : 1));
            for (int64_t i = 0; i < na_; ++i)
                for (int d = 0; d < 3; ++d) xr[3 * i + d] = p->tx.p[3 * (A->s + i) + d] - ca[d];
            for (int m = 0; m < nrhs; ++m) {
                orc_nu_adjoint(&nu, xr, na_, vtr + (size_t)m * nq, vti + (size_t)m * nq, or_, oi);
                for (int64_t i = 0; i < na_; ++i) {
                    accr[A->s + i + nx * m] += or_[i] / (4.0 * ORC_PI);
                    acci[A->s + i + nx * m] += oi[i] / (4.0 * ORC_PI);
                }
            }
            free(xr);
            free(or_);
            free(oi);
        }
        for (int64_t i = A->s; i < A->e && !nufft; ++i) {
            const double *x = p->tx.p + 3 * i;
            double d[3] = {x[0] - ca[0], x[1] - ca[1], x[2] - ca[2]};
            for (int m = 0; m < nrhs; ++m) {
                double sr = 0, si = 0;
                for (int q = 0; q < nq; ++q) {
                    double ph = k * (s[3 * q] * d[0] + s[3 * q + 1] * d[1] + s[3 * q + 2] * d[2]);
                    double er = cos(ph), ei = sin(ph);
                    sr += er * vtr[(size_t)m * nq + q] - ei * vti[(size_t)m * nq + q];
                    si += er * vti[(size_t)m * nq + q] + ei * vtr[(size_t)m * nq + q];
                }
                accr[i + nx * m] += sr / (4.0 * ORC_PI);
                acci[i + nx * m] += si / (4.0 * ORC_PI);
            }
        }
        free(vtr);
        free(vti);
        free(hr);
        free(hi);
    }
    free(first);
    free(used);
    free(utr);
    free(uti);
    free(s);
    free(w);
    free(ks);
    if (nufft) orc_nu_free(&nu);
}

/* Near field at the stop level (Sec. 2.2.4): the dense product over the remaining
 * non-admissible leaf pairs. */
/* Near field at the stop level (Sec. 2.2.4): the direct sum over the near leaf pairs.
 * With qv (double layer): sum_j (w u n)_j . (x - y_j) / (4 pi |x - y_j|^3). */
static void near_field(const orc_plan *p, const double *qr, const double *qi, const double *qv, int nrhs,
                       double *accr, double *acci)
{
    int l = p->st.l_stop;
    int64_t nbX = p->nbx[l], nn = p->n_nearp, nx = p->tx.n, ny = p->ty.n;
    const opair *pr = p->nearp;
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (nbX + 1));
    {
        int64_t i = 0;
        for (int64_t a = 0; a <= nbX; ++a) {
            while (i < nn && pr[i].a < a) ++i;
            first[a] = i;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < nbX; ++a) {
        const obox *A = &p->bx[l][a];
        for (int64_t i = A->s; i < A->e; ++i) {
            const double *x = p->tx.p + 3 * i;
            for (int m = 0; m < nrhs; ++m) {
                double sr = 0, si = 0;
                for (int64_t e = first[a]; e < first[a + 1]; ++e) {
                    const obox *B = &p->by[l][pr[e].b];
                    for (int64_t j = B->s; j < B->e; ++j) {
                        const double *y = p->ty.p + 3 * j;
                        if (qv) {
                            double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
                            double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                            if (r2 == 0.0) continue;
                            const double *q3 = qv + 3 * (j + ny * m);
                            sr += (q3[0] * d0 + q3[1] * d1 + q3[2] * d2) / (4.0 * ORC_PI * r2 * sqrt(r2));
                            continue;
                        }
                        double gr, gi;
                        orc_kernel(p->kind, p->k, x[0] - y[0], x[1] - y[1], x[2] - y[2], &gr, &gi);
                        double ur = qr[j + ny * m], ui = qi[j + ny * m];
                        sr += gr * ur - gi * ui;
                        si += gr * ui + gi * ur;
                    }
                }
                accr[i + nx * m] += sr;
                acci[i + nx * m] += si;
            }
        }
    }
    free(first);
}

/* v = G W u by the FFM: far field of every level with admissible pairs, then the near
 * field; inputs and outputs in the caller's (original) order, column-major per RHS.
 * uim/w may be NULL. v is overwritten. */
int orc_apply(const orc_plan *p, const double *w, const double *ure, const double *uim, int nrhs, double *vre,
              double *vim)
{
    if (!p || nrhs < 1) return ORC_EINVAL;
    int64_t nx = p->tx.n, ny = p->ty.n;
    double *qr = (double *)malloc(sizeof(double) * ny * nrhs), *qi = (double *)malloc(sizeof(double) * ny * nrhs);
    double *accr = (double *)calloc((size_t)nx * nrhs, sizeof(double));
    double *acci = (double *)calloc((size_t)nx * nrhs, sizeof(double));
    if (!qr || !qi || !accr || !acci) {
        free(qr);
        free(qi);
        free(accr);
        free(acci);
        return ORC_ENOMEM;
    }
    /* w u in sorted source order */
    for (int m = 0; m < nrhs; ++m)
        for (int64_t j = 0; j < ny; ++j) {
            int64_t o = p->ty.perm[j];
            double wj = w ? w[o] : 1.0;
            qr[j + ny * m] = wj * ure[o + ny * m];
            qi[j + ny * m] = uim ? wj * uim[o + ny * m] : 0.0;
        }
    for (int l = 0; l <= ORC_LMAX; ++l) {
        if (p->st.n_adm[l] == 0) continue;
        if (p->st.mode[l] == ORC_MODE_LAGRANGE)
            far_lagrange(p, l, qr, qi, NULL, nrhs, accr, acci);
        else
            far_planewave(p, l, qr, qi, nrhs, accr, acci);
    }
    if (p->n_nearp > 0) near_field(p, qr, qi, NULL, nrhs, accr, acci);
    for (int m = 0; m < nrhs; ++m)
        for (int64_t i = 0; i < nx; ++i) {
            int64_t o = p->tx.perm[i];
            vre[o + nx * m] = accr[i + nx * m];
            vim[o + nx * m] = acci[i + nx * m];
        }
    free(qr);
    free(qi);
    free(accr);
    free(acci);
    return ORC_OK;
}

/* Double-layer product by the FFM for a plan built with kind ORC_LAPLACE_DL: the
 * densities w u n (nrm: ny*3 row-major normals in the caller's order) go through the
 * three component kernels dG/dy_d of every Lagrange level and the double-layer near
 * field; real u and v, column-major per RHS, caller's order. */
int orc_apply_dl(const orc_plan *p, const double *nrm, const double *w, const double *u, int nrhs, double *v)
{
    if (!p || !nrm || nrhs < 1 || p->kind != ORC_LAPLACE_DL) return ORC_EINVAL;
    int64_t nx = p->tx.n, ny = p->ty.n;
    double *qv = (double *)malloc(sizeof(double) * 3 * ny * nrhs);
    double *zero = (double *)calloc((size_t)ny * nrhs, sizeof(double));
    double *accr = (double *)calloc((size_t)nx * nrhs, sizeof(double));
    double *acci = (double *)calloc((size_t)nx * nrhs, sizeof(double));
    if (!qv || !zero || !accr || !acci) {
        free(qv);
        free(zero);
        free(accr);
        free(acci);
        return ORC_ENOMEM;
    }
    for (int m = 0; m < nrhs; ++m)
        for (int64_t j = 0; j < ny; ++j) {
            int64_t o = p->ty.perm[j];
            double s = (w ? w[o] : 1.0) * u[o + ny * m];
            for (int ax = 0; ax < 3; ++ax) qv[3 * (j + ny * m) + ax] = s * nrm[3 * o + ax];
        }
    for (int l = 0; l <= ORC_LMAX; ++l)
        if (p->st.n_adm[l] > 0) far_lagrange(p, l, zero, zero, qv, nrhs, accr, acci);
    if (p->n_nearp > 0) near_field(p, zero, zero, qv, nrhs, accr, acci);
    for (int m = 0; m < nrhs; ++m)
        for (int64_t i = 0; i < nx; ++i) v[p->tx.perm[i] + nx * m] = accr[i + nx * m];
    free(qv);
    free(zero);
    free(accr);
    free(acci);
    return ORC_OK;
}

/* Gradient (kind ORC_LAPLACE_GRAD), one Lagrange level: the source step is the plain
 * Laplace one, u~_b = L_Y(b) w u; the three component kernels dG/dx_d are interpolated
 * separately (Sec. 2.2.2 per component), v~^d_a = sum_b T^d_{ab} u~_b with
 * T^d_{ab}[i][j] = -(x_i - y_j)_d / (4 pi |x_i - y_j|^3) at the Chebyshev nodes, and the
 * target step interpolates each component. */
static void far_lagrange_grad(const orc_plan *p, int l, const double *q, int nrhs, double *acc)
{
    int r1 = p->st.r1[l], r = r1 * r1 * r1;
    double t[16];
    cheb_nodes(r1, t);
    double dl = ldexp(p->d0, -l);
    int64_t nbY = p->nby[l], nbX = p->nbx[l];
    int64_t ny = p->ty.n, nx = p->tx.n;
    double *ut = (double *)calloc((size_t)nbY * nrhs * r, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nbY; ++b) {
        const obox *B = &p->by[l][b];
        double c[3], Lb[1000];
        box_centre(p->ty.o, B->g, dl, c);
        for (int64_t j = B->s; j < B->e; ++j) {
            lagrange_3d(r1, t, p->ty.p + 3 * j, c, dl, Lb);
            for (int m = 0; m < nrhs; ++m)
                for (int a = 0; a < r; ++a) ut[((size_t)b * nrhs + m) * r + a] += Lb[a] * q[j + ny * m];
        }
    }
    int64_t na = p->st.n_adm[l];
    const opair *adm = p->adm[l];
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (nbX + 1));
    {
        int64_t i = 0;
        for (int64_t a = 0; a <= nbX; ++a) {
            while (i < na && adm[i].a < a) ++i;
            first[a] = i;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < nbX; ++a) {
        if (first[a] == first[a + 1]) continue;
        const obox *A = &p->bx[l][a];
        double ca[3];
        box_centre(p->tx.o, A->g, dl, ca);
        double *vt = (double *)calloc((size_t)nrhs * 3 * r, sizeof(double));
        double *T = (double *)malloc(sizeof(double) * 3 * r * r);
        for (int64_t e = first[a]; e < first[a + 1]; ++e) {
            int64_t b = adm[e].b;
            double cb[3];
            box_centre(p->ty.o, p->by[l][b].g, dl, cb);
            for (int i = 0; i < r; ++i) {
                int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
                double xc[3] = {ca[0] + t[ix] * 0.5 * dl, ca[1] + t[iy] * 0.5 * dl, ca[2] + t[iz] * 0.5 * dl};
                for (int j = 0; j < r; ++j) {
                    int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
                    double yc[3] = {cb[0] + t[jx] * 0.5 * dl, cb[1] + t[jy] * 0.5 * dl, cb[2] + t[jz] * 0.5 * dl};
                    double dd[3] = {xc[0] - yc[0], xc[1] - yc[1], xc[2] - yc[2]};
                    double r2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
                    for (int d = 0; d < 3; ++d) T[((size_t)d * r + i) * r + j] = -dd[d] / (4.0 * ORC_PI * r2 * sqrt(r2));
                }
            }
            for (int m = 0; m < nrhs; ++m) {
                const double *u = ut + ((size_t)b * nrhs + m) * r;
                for (int d = 0; d < 3; ++d)
                    for (int i = 0; i < r; ++i) {
                        double sum = 0;
                        for (int j = 0; j < r; ++j) sum += T[((size_t)d * r + i) * r + j] * u[j];
                        vt[((size_t)m * 3 + d) * r + i] += sum;
                    }
            }
        }
        double La[1000];
        for (int64_t i = A->s; i < A->e; ++i) {
            lagrange_3d(r1, t, p->tx.p + 3 * i, ca, dl, La);
            for (int m = 0; m < nrhs; ++m)
                for (int d = 0; d < 3; ++d) {
                    double sum = 0;
                    for (int c = 0; c < r; ++c) sum += La[c] * vt[((size_t)m * 3 + d) * r + c];
                    acc[i + nx * (3 * m + d)] += sum;
                }
        }
        free(vt);
        free(T);
    }
    free(first);
    free(ut);
}

/* Gradient near field at the stop level: the direct sum over the near leaf pairs. */
static void near_field_grad(const orc_plan *p, const double *q, int nrhs, double *acc)
{
    int l = p->st.l_stop;
    int64_t nbX = p->nbx[l], nn = p->n_nearp, nx = p->tx.n, ny = p->ty.n;
    const opair *pr = p->nearp;
    int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (nbX + 1));
    {
        int64_t i = 0;
        for (int64_t a = 0; a <= nbX; ++a) {
            while (i < nn && pr[i].a < a) ++i;
            first[a] = i;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < nbX; ++a) {
        const obox *A = &p->bx[l][a];
        for (int64_t i = A->s; i < A->e; ++i) {
            const double *x = p->tx.p + 3 * i;
            for (int m = 0; m < nrhs; ++m) {
                double g[3] = {0, 0, 0};
                for (int64_t e = first[a]; e < first[a + 1]; ++e) {
                    const obox *B = &p->by[l][pr[e].b];
                    for (int64_t j = B->s; j < B->e; ++j) {
                        const double *y = p->ty.p + 3 * j;
                        double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (r2 == 0.0) continue;
                        double f = q[j + ny * m] / (4.0 * ORC_PI * r2 * sqrt(r2));
                        for (int c = 0; c < 3; ++c) g[c] -= f * d[c];
                    }
                }
                for (int c = 0; c < 3; ++c) acc[i + nx * (3 * m + c)] += g[c];
            }
        }
    }
    free(first);
}

/* Gradient product by the FFM for a plan built with kind ORC_LAPLACE_GRAD (Lagrange levels
 * only): v (nx x 3 nrhs, column 3 m + d) = sum_j w_j u_j grad_x G(x_i - y_j). */
int orc_apply_grad(const orc_plan *p, const double *w, const double *u, int nrhs, double *v)
{
    if (!p || nrhs < 1 || p->kind != ORC_LAPLACE_GRAD) return ORC_EINVAL;
    int64_t nx = p->tx.n, ny = p->ty.n;
    double *q = (double *)malloc(sizeof(double) * ny * nrhs);
    double *acc = (double *)calloc((size_t)nx * 3 * nrhs, sizeof(double));
    if (!q || !acc) {
        free(q);
        free(acc);
        return ORC_ENOMEM;
    }
    for (int m = 0; m < nrhs; ++m)
        for (int64_t j = 0; j < ny; ++j) {
            int64_t o = p->ty.perm[j];
            q[j + ny * m] = (w ? w[o] : 1.0) * u[o + ny * m];
        }
    for (int l = 0; l <= ORC_LMAX; ++l)
        if (p->st.n_adm[l] > 0) far_lagrange_grad(p, l, q, nrhs, acc);
    if (p->n_nearp > 0) near_field_grad(p, q, nrhs, acc);
    for (int c = 0; c < 3 * nrhs; ++c)
        for (int64_t i = 0; i < nx; ++i) v[p->tx.perm[i] + nx * c] = acc[i + nx * c];
    free(q);
    free(acc);
    return ORC_OK;
}
