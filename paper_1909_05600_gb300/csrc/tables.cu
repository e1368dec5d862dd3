// Per-level transfer operators, one per distinct integer box translation (Sec. 3.1,
// proof of Prop. 1: the number of distinct transfers per level does not depend on l).
//   Lagrange levels (Sec. 2.2.2): T_t[i][j] = G(x_c,i - y_c,j), Chebyshev control nodes.
//   Plane-wave levels (Sec. 2.2.3): quadrature of eq. 17, diagonal transfer
//     D_t(q) = ik w_q T_{L,r0}(s_q) / (4 pi) with the Gegenbauer series of eq. 12 summed
//     from p = 0 (phases are box-centred, so no r0 phase enters), and octant phase
//     factors e^{-ik s_q . delta} that move a leaf-centred sum to its ancestor's centre.
// Tables are computed in FP64 and stored in FP32.
#include <cmath>
#include <vector>

#include "ffm_internal.cuh"

namespace ffm {

struct alignas(32) Dir4 {
    double x, y, z, w;
};

// Worst-pair relative error of the tensor Chebyshev-Lagrange interpolation per r1 (index
// r1 = 2..10), for the Laplace kernel and for the Helmholtz kernel at k d = 2.  These are
// plan constants: the smallest r1 whose error is <= eps is used.
static const double R1_ERR_LAPLACE[11] = {1, 1, 3.2e-2, 4.8e-3, 7.6e-4, 1.1e-4, 1.6e-5, 2.0e-6, 2.4e-7, 8.1e-8, 1.1e-8};
static const double R1_ERR_HELM[11] = {1, 1, 2.4e-1, 3.4e-2, 3.6e-3, 3.6e-4, 4.0e-5, 3.9e-6, 3.9e-7, 1.3e-7, 1.4e-8};

int r1_rule(int kind, double eps) {
    const double *t = kind == FFM_HELMHOLTZ ? R1_ERR_HELM : R1_ERR_LAPLACE;
    for (int r1 = 2; r1 <= 10; ++r1)
        if (t[r1] <= eps) return r1;
    return 10;
}

struct LagGeo {
    double oxy[3]; // oX - oY
    double dl;
    double k;
    int r1;
    int kind;
};

__device__ __forceinline__ void kernel_fp64(int kind, double k, double dx, double dy, double dz, double &gr,
                                            double &gi) {
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r == 0.0) {
        gr = gi = 0.0;
        return;
    }
    double a = 1.0 / (4.0 * PI * r);
    if (kind == FFM_LAPLACE) {
        gr = a;
        gi = 0.0;
    } else {
        double sn, cs;
        sincos(k * r, &sn, &cs);
        gr = a * cs;
        gi = a * sn;
    }
}

// T stored as [t][j][i] (source node j outer) so the transfer kernel reads it along i.
__global__ void k_lag_table(const int4 *__restrict__ m, int ntrans, LagGeo geo, float *__restrict__ T) {
    int t = blockIdx.x;
    int r1 = geo.r1, r = r1 * r1 * r1;
    int4 mt = m[t];
    double r0x = geo.oxy[0] + mt.x * geo.dl, r0y = geo.oxy[1] + mt.y * geo.dl, r0z = geo.oxy[2] + mt.z * geo.dl;
    double h = 0.5 * geo.dl;
    bool cplx = geo.kind == FFM_HELMHOLTZ;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        int j = e / r, i = e % r;
        int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
        int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
        double c = PI / (2.0 * r1);
        double dx = r0x + h * (cos((2 * ix + 1) * c) - cos((2 * jx + 1) * c));
        double dy = r0y + h * (cos((2 * iy + 1) * c) - cos((2 * jy + 1) * c));
        double dz = r0z + h * (cos((2 * iz + 1) * c) - cos((2 * jz + 1) * c));
        double gr, gi;
        kernel_fp64(geo.kind, geo.k, dx, dy, dz, gr, gi);
        size_t o = (size_t)t * r * r + (size_t)j * r + i;
        if (cplx) {
            T[2 * o] = (float)gr;
            T[2 * o + 1] = (float)gi;
        } else {
            T[o] = (float)gr;
        }
    }
}

// D_t(q) = (i k w_q / (4 pi)) sum_{p=0}^{L} c_t[p] P_p(s_q . rhat_t)
__global__ void k_pw_table(const Dir4 *__restrict__ sw, int nQ, const double2 *__restrict__ coef, int L,
                           const Dir4 *__restrict__ rhat, double k, float2 *__restrict__ D) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int t = blockIdx.y;
    if (q >= nQ) return;
    Dir4 s = sw[q];
    Dir4 rh = rhat[t];
    double x = s.x * rh.x + s.y * rh.y + s.z * rh.z;
    const double2 *c = coef + (size_t)t * (L + 1);
    double p0 = 1.0, p1 = x;
    double ar = c[0].x, ai = c[0].y;
    if (L >= 1) {
        ar += c[1].x * x;
        ai += c[1].y * x;
    }
    for (int p = 1; p < L; ++p) {
        double p2 = ((2.0 * p + 1.0) * x * p1 - p * p0) / (p + 1.0);
        p0 = p1;
        p1 = p2;
        ar += c[p + 1].x * p2;
        ai += c[p + 1].y * p2;
    }
    double f = k * s.w / (4.0 * PI);
    D[(size_t)t * nQ + q] = make_float2((float)(-f * ai), (float)(f * ar));
}

// E[d][oct][q] = e^{-ik s_q . delta}, delta_axis = (bit - 1/2) d_m for depth m = l+1+d.
__global__ void k_pw_octants(const Dir4 *__restrict__ sw, int nQ, double k, double d_first, int ndepth,
                             float2 *__restrict__ E) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int d = blockIdx.y, oct = blockIdx.z;
    if (q >= nQ || d >= ndepth) return;
    double dm = ldexp(d_first, -d);
    Dir4 s = sw[q];
    double bx = ((oct >> 2) & 1) - 0.5, by = ((oct >> 1) & 1) - 0.5, bz = (oct & 1) - 0.5;
    double ph = -k * dm * (s.x * bx + s.y * by + s.z * bz);
    double sn, cs;
    sincos(ph, &sn, &cs);
    E[((size_t)d * 8 + oct) * nQ + q] = make_float2((float)cs, (float)sn);
}

// Gauss-Legendre nodes (ascending) and weights of order n by Newton's method on P_n.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double a = 1.0, b = z;
            for (int j = 2; j <= n; ++j) {
                double c = ((2.0 * j - 1.0) * z * b - (j - 1.0) * a) / j;
                a = b;
                b = c;
            }
            dp = n * (z * b - a) / (z * z - 1.0);
            double step = b / dp;
            z -= step;
            if (std::fabs(step) < 1e-16) break;
        }
        double a = 1.0, b = z;
        for (int j = 2; j <= n; ++j) {
            double c = ((2.0 * j - 1.0) * z * b - (j - 1.0) * a) / j;
            a = b;
            b = c;
        }
        dp = n * (z * b - a) / (z * z - 1.0);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// h_p^(1)(z), p = 0..L, upward recurrence from h_0 = -i e^{iz}/z, h_1 = -e^{iz}(z+i)/z^2.
static void hankel1(int L, double z, std::vector<double> &hr, std::vector<double> &hi) {
    hr.assign(L + 1, 0.0);
    hi.assign(L + 1, 0.0);
    double c = std::cos(z), s = std::sin(z);
    hr[0] = s / z;
    hi[0] = -c / z;
    if (L >= 1) {
        hr[1] = (s - z * c) / (z * z);
        hi[1] = (-c - z * s) / (z * z);
    }
    for (int p = 1; p < L; ++p) {
        double f = (2.0 * p + 1.0) / z;
        hr[p + 1] = f * hr[p] - hr[p - 1];
        hi[p + 1] = f * hi[p] - hi[p - 1];
    }
}

void build_tables(ffm_plan_s *p, int l, Alloc &tmp) {
    FarLevel &F = p->far[l];
    cudaStream_t s = p->stream;
    double dl = std::ldexp(p->d0, -l);
    double oxy[3] = {p->oX[0] - p->oY[0], p->oX[1] - p->oY[1], p->oX[2] - p->oY[2]};
    if (F.mode == 1) {
        if (F.r1 > R1MAX) fail(FFM_EUNSUPPORTED, "eps needs more than 8 Chebyshev nodes per axis");
        int r = F.r1 * F.r1 * F.r1;
        bool cplx = p->kind == FFM_HELMHOLTZ;
        F.T = p->mem.get<float>((size_t)F.n_trans * r * r * (cplx ? 2 : 1));
        LagGeo g{};
        for (int d = 0; d < 3; ++d) g.oxy[d] = oxy[d];
        g.dl = dl;
        g.k = p->k;
        g.r1 = F.r1;
        g.kind = p->kind;
        FFM_LAUNCH(k_lag_table, F.n_trans, 256, 0, s, F.trans_m, F.n_trans, g, F.T);
        return;
    }
    // plane waves: quadrature of eq. 17
    int L = F.L, nQ = F.nQ, np = 2 * L;
    std::vector<double> mu, wg;
    gauss_legendre(L + 1, mu, wg);
    std::vector<Dir4> sw(nQ);
    std::vector<float4> ks(nQ);
    for (int i = 0; i <= L; ++i) {
        double st = std::sqrt(1.0 - mu[i] * mu[i]);
        for (int j = 0; j < np; ++j) {
            double ph = j * PI / L;
            int q = i * np + j;
            sw[q] = Dir4{st * std::cos(ph), st * std::sin(ph), mu[i], wg[i] * PI / L};
            ks[q] = make_float4((float)(p->k * sw[q].x), (float)(p->k * sw[q].y), (float)(p->k * sw[q].z), 0.f);
        }
    }
    // Gegenbauer coefficients c_t[p] = (2p+1) i^p h_p(k |r0_t|) / (4 pi) and r0 directions
    int nt = F.n_trans;
    std::vector<double2> coef((size_t)nt * (L + 1));
    std::vector<Dir4> rhat(nt);
    std::vector<double> hr, hi;
    for (int t = 0; t < nt; ++t) {
        int4 m = F.h_trans_m[t];
        double r0[3] = {oxy[0] + m.x * dl, oxy[1] + m.y * dl, oxy[2] + m.z * dl};
        double R = std::sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
        rhat[t] = Dir4{r0[0] / R, r0[1] / R, r0[2] / R, R};
        hankel1(L, p->k * R, hr, hi);
        for (int q = 0; q <= L; ++q) {
            double ipr = (q % 4 == 0) ? 1.0 : (q % 4 == 2 ? -1.0 : 0.0);
            double ipi = (q % 4 == 1) ? 1.0 : (q % 4 == 3 ? -1.0 : 0.0);
            double f = (2.0 * q + 1.0) / (4.0 * PI);
            coef[(size_t)t * (L + 1) + q] = make_double2(f * (ipr * hr[q] - ipi * hi[q]), f * (ipr * hi[q] + ipi * hr[q]));
        }
    }
    Dir4 *d_sw = tmp.get<Dir4>(nQ);
    double2 *d_coef = tmp.get<double2>(coef.size());
    Dir4 *d_rhat = tmp.get<Dir4>(nt);
    FFM_CUDA(cudaMemcpyAsync(d_sw, sw.data(), sizeof(Dir4) * nQ, cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(d_coef, coef.data(), sizeof(double2) * coef.size(), cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(d_rhat, rhat.data(), sizeof(Dir4) * nt, cudaMemcpyHostToDevice, s));
    F.ks = p->mem.get<float4>(nQ);
    FFM_CUDA(cudaMemcpyAsync(F.ks, ks.data(), sizeof(float4) * nQ, cudaMemcpyHostToDevice, s));
    F.D = p->mem.get<float2>((size_t)nt * nQ);
    dim3 g1(cdiv(nQ, 128), nt);
    FFM_LAUNCH(k_pw_table, g1, 128, 0, s, d_sw, nQ, d_coef, L, d_rhat, p->k, F.D);
    int ndepth = p->l_stop - l;
    if (ndepth > 0) {
        F.E = p->mem.get<float2>((size_t)ndepth * 8 * nQ);
        dim3 g2(cdiv(nQ, 128), ndepth, 8);
        FFM_LAUNCH(k_pw_octants, g2, 128, 0, s, d_sw, nQ, p->k, std::ldexp(p->d0, -(l + 1)), ndepth, F.E);
    }
    // host vectors die here: wait for the copies that read them
    FFM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace ffm
