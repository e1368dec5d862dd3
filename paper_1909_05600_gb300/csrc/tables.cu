// Per-level transfer operators, one per distinct integer box translation (Sec. 3.1,
// proof of Prop. 1: the number of distinct transfers per level does not depend on l).
//   Lagrange levels (Sec. 2.2.2): T_t[i][j] = G(x_c,i - y_c,j), Chebyshev control nodes.
//   Plane-wave levels (Sec. 2.2.3): quadrature of eq. 17, diagonal transfer
//     D_t(q) = ik w_q T_{L,r0}(s_q) / (4 pi) with the Gegenbauer series of eq. 12 summed
//     from p = 0 (phases are box-centred, so no r0 phase enters), and octant phase
//     factors e^{-ik s_q . delta} that move a leaf-centred sum to its ancestor's centre.
// Tables are computed in FP64 and stored in FP32.
#include <cmath>
#include <map>
#include <tuple>
#include <type_traits>
#include <vector>

#include "ffm_internal.cuh"

namespace ffm {

// Worst-pair relative error of the tensor Chebyshev-Lagrange interpolation per r1 (index
// r1 = 2..10), for the Laplace kernel and for the Helmholtz kernel at k d = 2.  These are
// plan constants: the smallest r1 whose error is <= eps is used.
static const double R1_ERR_LAPLACE[11] = {1, 1, 3.2e-2, 4.8e-3, 7.6e-4, 1.1e-4, 1.6e-5, 2.0e-6, 2.4e-7, 8.1e-8, 1.1e-8};
static const double R1_ERR_HELM[11] = {1, 1, 2.4e-1, 3.4e-2, 3.6e-3, 3.6e-4, 4.0e-5, 3.9e-6, 3.9e-7, 1.3e-7, 1.4e-8};
// the double layer: its three component kernels dG/dy_d, weighted by the source normals
static const double R1_ERR_LAPLACE_DL[11] = {1, 1, 1.2e-1, 2.4e-2, 5.1e-3, 1.1e-3, 1.8e-4, 2.6e-5, 3.9e-6, 1.5e-6, 2.0e-7};

int r1_rule(int kind, double eps) {
    // the gradient's component kernels are the double layer's up to sign: same table
    const double *t = kind == FFM_HELMHOLTZ                                  ? R1_ERR_HELM
                      : (kind == FFM_LAPLACE_DL || kind == FFM_LAPLACE_GRAD) ? R1_ERR_LAPLACE_DL
                                                                             : R1_ERR_LAPLACE;
    for (int r1 = 2; r1 <= 10; ++r1)
        if (t[r1] <= eps) return r1;
    return 10;
}

struct LagGeo {
    double oxy[3];  // oX - oY
    double dl;
    float k;
    int r1;
    int kind;
    float hnode[R1MAX];  // (d_l / 2) cos((2a+1) pi / (2 r1))
};

// T stored as [t][i][j] (source node j innermost): rows of T are K-major operands of the
// transfer GEMMs.
// The translation r0 is formed in FP64 and rounded once; node differences, the distance
// and the kernel are FP32 (admissible control nodes are at least d_l apart, so the
// difference loses nothing), and T is stored in FP32.
__global__ void k_lag_table(const int4 *__restrict__ m, int ntrans, LagGeo geo, float *__restrict__ T) {
    int t = blockIdx.x;
    int r1 = geo.r1, r = r1 * r1 * r1;
    int4 mt = m[t];
    float r0x = (float)(geo.oxy[0] + mt.x * geo.dl), r0y = (float)(geo.oxy[1] + mt.y * geo.dl),
          r0z = (float)(geo.oxy[2] + mt.z * geo.dl);
    bool cplx = geo.kind == FFM_HELMHOLTZ;
    const float c4pi = 0.07957747154594767f;  // 1 / (4 pi)
    if (geo.kind == FFM_LAPLACE_GRAD) {
        // the gradient's component kernels dG/dx_d = -(x - y)_d / (4 pi |x - y|^3), one
        // r x r block per component: T[(d * ntrans + t)][i][j]
        for (int e = threadIdx.x; e < 3 * r * r; e += blockDim.x) {
            int d = e / (r * r), ij = e - d * r * r, i = ij / r, j = ij - i * r;
            int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
            int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
            float dv[3] = {r0x + (geo.hnode[ix] - geo.hnode[jx]), r0y + (geo.hnode[iy] - geo.hnode[jy]),
                           r0z + (geo.hnode[iz] - geo.hnode[jz])};
            float r2 = fmaf(dv[0], dv[0], fmaf(dv[1], dv[1], dv[2] * dv[2]));
            float rr = sqrtf(r2);
            T[((size_t)d * ntrans + t) * r * r + ij] = -c4pi * dv[d] / (r2 * rr);
        }
        return;
    }
    if (geo.kind == FFM_LAPLACE_DL) {
        // the double layer's component kernels dG/dy_d = (x - y)_d / (4 pi |x - y|^3),
        // stacked along K: T[t][i][d r + j]
        for (int e = threadIdx.x; e < 3 * r * r; e += blockDim.x) {
            int i = e / (3 * r), jj = e % (3 * r), d = jj / r, j = jj % r;
            int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
            int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
            float dv[3] = {r0x + (geo.hnode[ix] - geo.hnode[jx]), r0y + (geo.hnode[iy] - geo.hnode[jy]),
                           r0z + (geo.hnode[iz] - geo.hnode[jz])};
            float r2 = fmaf(dv[0], dv[0], fmaf(dv[1], dv[1], dv[2] * dv[2]));
            float rr = sqrtf(r2);
            T[(size_t)t * 3 * r * r + e] = c4pi * dv[d] / (r2 * rr);
        }
        return;
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        int i = e / r, j = e % r;
        int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
        int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
        float dx = r0x + (geo.hnode[ix] - geo.hnode[jx]);
        float dy = r0y + (geo.hnode[iy] - geo.hnode[jy]);
        float dz = r0z + (geo.hnode[iz] - geo.hnode[jz]);
        float rr = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        float a = c4pi / rr;
        size_t o = (size_t)t * r * r + (size_t)i * r + j;
        if (cplx) {
            float sn, cs;
            sincosf(geo.k * rr, &sn, &cs);
            T[2 * o] = a * cs;
            T[2 * o + 1] = a * sn;
        } else {
            T[o] = a;
        }
    }
}

// T_t split for the target-stationary tensor-core transfer: per translation a 64 x 64 hi
// block then a 64 x 64 lo block (rows i, K = j; zero beyond r), each in the K-major
// core-matrix order the MMA reads from shared memory.  hi keeps the TF32 bits (low 13
// mantissa bits cleared), lo = T - hi exactly.
// Per translation, the image the target-stationary transfer copies into shared memory for
// each half of K (source nodes 0..31, 32..63): the TF32 hi block, then the lo block, each 64
// rows (target nodes) x 32 in the K-major core-matrix layout; zero padded beyond r.
__global__ void k_lag_table_split(const float *__restrict__ T, int r, float *__restrict__ out) {
    int t = blockIdx.x;
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        int i = e / 64, j = e % 64;
        float v = (i < r && j < r) ? T[(size_t)t * r * r + (size_t)i * r + j] : 0.f;
        float hi = __uint_as_float(__float_as_uint(v) & 0xffffe000u);
        int h = j >> 5;
        uint32_t o = kmajor_index(i, j & 31, 32);
        out[(size_t)t * 8192 + h * 4096 + o] = hi;
        out[(size_t)t * 8192 + h * 4096 + 2048 + o] = v - hi;
    }
}

void launch_table_split(ffm_plan_s *p, int l, cudaStream_t s) {
    FarLevel &F = p->far[l];
    int r = F.r1 * F.r1 * F.r1;
    F.Tsp = p->mem.get<float>((size_t)F.n_trans * 8192);
    FFM_LAUNCH(k_lag_table_split, F.n_trans, 256, 0, s, F.T, r, F.Tsp);
}

// ---- double-float arithmetic (unevaluated sums hi + lo of two floats, FMA-based)

struct dflt {
    float hi, lo;
};

__device__ __forceinline__ dflt df_fast_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dflt df_two_sum(float a, float b) {
    float s = a + b;
    float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
    dflt s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dflt df_split(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}

// D_t(q) = (i k w_q / (4 pi)) sum_{p=0}^{L} c_t[p] P_p(s_q . rhat_t).
// The Legendre recurrence P_{p+1} = x P_p + p/(p+1) (x P_p - P_{p-1}) and the sum run in
// double-float arithmetic on the FP32 pipe (FP64 throughput on this part is a small
// fraction of FP32), giving ~2^-44 relative accuracy before the final rounding.
// coef: per translation L+1 complex coefficients split as (re.hi, re.lo, im.hi, im.lo);
// beta: L entries p/(p+1) split as (hi, lo).
// a double as an unevaluated FP32 pair
__device__ __forceinline__ dd split_dd(double v) {
    float h = (float)v;
    return dd(h, (float)(v - (double)h));
}

// complex value (re, im) stored as the table's element type
template <class OUT>
__device__ __forceinline__ OUT make_out(double re, double im) {
    if constexpr (std::is_same<OUT, float2>::value)
        return make_float2((float)re, (float)im);
    else if constexpr (std::is_same<OUT, double2>::value)
        return make_double2(re, im);
    else
        return dd2{split_dd(re), split_dd(im)};
}

template <class OUT>
__device__ __forceinline__ void put_d(OUT *D, size_t o, double f, dflt r, dflt i) {
    // D = i f (sum_re + i sum_im)
    double tr = (double)r.hi + (double)r.lo, ti = (double)i.hi + (double)i.lo;
    D[o] = make_out<OUT>(-f * ti, f * tr);
}

// FP32 levels (the quadrature sum's cancellation ratio is at most 250): the same recurrence and
// partial sums in FP32, each partial sum compensated (its rounding error carried in a second
// FP32 term, TwoSum).  The forward Legendre recurrence is stable, its error grows about
// linearly with the degree.
__device__ __forceinline__ void comp_add(float &sum, float &cmp, float term) {
    float t = sum + term;
    float bb = t - sum;
    cmp += (sum - (t - bb)) + (term - bb);
    sum = t;
}

__global__ void __launch_bounds__(256) k_pw_table_f32(const D4 *__restrict__ sw, int nH, const float4 *__restrict__ coef,
                                                      const float2 *__restrict__ beta, int L,
                                                      const D4 *__restrict__ rhat, const int2 *__restrict__ pairs,
                                                      double k, float2 *__restrict__ D) {
    extern __shared__ float4 sm[];
    float4 *sc = sm;                                      // L+1 coefficients
    float2 *sb = reinterpret_cast<float2 *>(sm + L + 1);  // L betas
    int2 tp = pairs[blockIdx.y];
    int t = tp.x;
    for (int i = threadIdx.x; i <= L; i += blockDim.x) sc[i] = coef[(size_t)t * (L + 1) + i];
    for (int i = threadIdx.x; i < L; i += blockDim.x) sb[i] = beta[i];
    __syncthreads();
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nH) return;
    D4 sv = sw[q];
    D4 rh = rhat[t];
    float x = (float)(sv.x * rh.x + sv.y * rh.y + sv.z * rh.z);
    float p0 = 1.f, p1 = x;
    float4 c0 = sc[0];
    float er = c0.x + c0.y, ei = c0.z + c0.w, erc = 0.f, eic = 0.f;
    float orr = 0.f, oi = 0.f, orc = 0.f, oic = 0.f;
    if (L >= 1) {
        float4 c1 = sc[1];
        orr = (c1.x + c1.y) * x;
        oi = (c1.z + c1.w) * x;
    }
    // P_{p+1} = x P_p + (p/(p+1)) (x P_p - P_{p-1}); degree p+1 is even for odd p
    auto step = [&](int pp) {
        float xp = x * p1;
        float p2 = fmaf(sb[pp].x, xp - p0, xp);
        p0 = p1;
        p1 = p2;
        return p2;
    };
    int pp = 1;
    for (; pp + 1 < L; pp += 2) {
        float pe = step(pp);
        float4 c = sc[pp + 1];
        comp_add(er, erc, (c.x + c.y) * pe);
        comp_add(ei, eic, (c.z + c.w) * pe);
        float po = step(pp + 1);
        float4 d = sc[pp + 2];
        comp_add(orr, orc, (d.x + d.y) * po);
        comp_add(oi, oic, (d.z + d.w) * po);
    }
    if (pp < L) {
        float pe = step(pp);
        float4 c = sc[pp + 1];
        comp_add(er, erc, (c.x + c.y) * pe);
        comp_add(ei, eic, (c.z + c.w) * pe);
    }
    double f = k * sv.w / (4.0 * PI);
    double Er = (double)er + erc, Ei = (double)ei + eic, Or = (double)orr + orc, Oi = (double)oi + oic;
    size_t nQ = 2 * (size_t)nH;
    // D = i f (sum_re + i sum_im), sum = E + O for direction h and E - O for its antipode
    float2 dp = make_float2((float)(-f * (Ei + Oi)), (float)(f * (Er + Or)));
    float2 dm = make_float2((float)(-f * (Ei - Oi)), (float)(f * (Er - Or)));
    D[(size_t)t * nQ + q] = dp;
    D[(size_t)t * nQ + q + nH] = dm;
    if (tp.y >= 0) {
        D[(size_t)tp.y * nQ + q] = dm;
        D[(size_t)tp.y * nQ + q + nH] = dp;
    }
}

// One Legendre recurrence serves four table entries.  With x = s_h . rhat_t, the sum splits
// into even-degree and odd-degree parts E(x) + O(x); direction h + nQ/2 is -s_h, where the
// sum is E - O.  A translation -m with the same length (the two root boxes share their
// centre) has rhat = -rhat_t, so its entries are the same two values with the directions
// swapped.  pairs[c] = (t, partner of t or -1).
template <class OUT>
__global__ void __launch_bounds__(256) k_pw_table(const D4 *__restrict__ sw, int nH, const float4 *__restrict__ coef,
                                                  const float2 *__restrict__ beta, int L,
                                                  const D4 *__restrict__ rhat, const int2 *__restrict__ pairs,
                                                  double k, OUT *__restrict__ D) {
    extern __shared__ float4 sm[];
    float4 *sc = sm;                                  // L+1 coefficients
    float2 *sb = reinterpret_cast<float2 *>(sm + L + 1);  // L betas
    int2 tp = pairs[blockIdx.y];
    int t = tp.x;
    for (int i = threadIdx.x; i <= L; i += blockDim.x) sc[i] = coef[(size_t)t * (L + 1) + i];
    for (int i = threadIdx.x; i < L; i += blockDim.x) sb[i] = beta[i];
    __syncthreads();
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nH) return;
    D4 s = sw[q];
    D4 rh = rhat[t];
    dflt x = df_split(s.x * rh.x + s.y * rh.y + s.z * rh.z);
    dflt p0 = {1.f, 0.f}, p1 = x;
    float4 c0 = sc[0];
    dflt er = {c0.x, c0.y}, ei = {c0.z, c0.w}, orr = {0.f, 0.f}, oi = {0.f, 0.f};
    if (L >= 1) {
        float4 c1 = sc[1];
        orr = df_mul({c1.x, c1.y}, x);
        oi = df_mul({c1.z, c1.w}, x);
    }
    // P_{p+1} = x P_p + (p/(p+1)) (x P_p - P_{p-1}); degree p+1 is even for odd p
    auto step = [&](int pp) {
        dflt xp = df_mul(x, p1);
        dflt diff = df_add(xp, {-p0.hi, -p0.lo});
        float2 b = sb[pp];
        dflt p2 = df_add(xp, df_mul({b.x, b.y}, diff));
        p0 = p1;
        p1 = p2;
        return p2;
    };
    int pp = 1;
    for (; pp + 1 < L; pp += 2) {
        dflt pe = step(pp);
        float4 c = sc[pp + 1];
        er = df_add(er, df_mul({c.x, c.y}, pe));
        ei = df_add(ei, df_mul({c.z, c.w}, pe));
        dflt po = step(pp + 1);
        float4 d = sc[pp + 2];
        orr = df_add(orr, df_mul({d.x, d.y}, po));
        oi = df_add(oi, df_mul({d.z, d.w}, po));
    }
    if (pp < L) {
        dflt pe = step(pp);
        float4 c = sc[pp + 1];
        er = df_add(er, df_mul({c.x, c.y}, pe));
        ei = df_add(ei, df_mul({c.z, c.w}, pe));
    }
    double f = k * s.w / (4.0 * PI);
    dflt pr = df_add(er, orr), pi = df_add(ei, oi);
    dflt mr = df_add(er, {-orr.hi, -orr.lo}), mi = df_add(ei, {-oi.hi, -oi.lo});
    size_t nQ = 2 * (size_t)nH;
    put_d(D, (size_t)t * nQ + q, f, pr, pi);
    put_d(D, (size_t)t * nQ + q + nH, f, mr, mi);
    if (tp.y >= 0) {
        put_d(D, (size_t)tp.y * nQ + q, f, mr, mi);
        put_d(D, (size_t)tp.y * nQ + q + nH, f, pr, pi);
    }
}

// E[d][oct][q] = e^{-ik s_q . delta}, delta_axis = (bit - 1/2) d_m for depth m = l+1+d.
template <class OUT>
__global__ void k_pw_octants(const D4 *__restrict__ sw, int nQ, double k, double d_first, int ndepth,
                             OUT *__restrict__ E) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int d = blockIdx.y, oct = blockIdx.z;
    if (q >= nQ || d >= ndepth) return;
    double dm = ldexp(d_first, -d);
    D4 s = sw[q];
    double bx = ((oct >> 2) & 1) - 0.5, by = ((oct >> 1) & 1) - 0.5, bz = (oct & 1) - 0.5;
    double ph = -k * dm * (s.x * bx + s.y * by + s.z * bz);
    double sn, cs;
    sincos(ph, &sn, &cs);
    size_t o = ((size_t)d * 8 + oct) * nQ + q;
    E[o] = make_out<OUT>(cs, sn);
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

void gauss_legendre_nodes(int n, std::vector<double> &x, std::vector<double> &w) { gauss_legendre(n, x, w); }

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

TableJob::TableJob(cudaStream_t main) : side(main) { tmp.stream = main; }

TableJob::~TableJob() {
    // host staging buffers may still be read by queued copies
    cudaStreamSynchronize(side);
    tmp.release();
}

// ---- ACA of the transfer matrices (Sec. 2.2.2, eq. 11), after Bebendorf, with full
// pivoting on the explicit r x r matrix (it is small, and full pivoting bounds the
// Frobenius error exactly): step k takes the residual R = T - S_k, its entry of largest
// magnitude (i, j) (near-ties within a factor 1 - 1e-9 go to the first in row-major
// order), a = R(:, j), b = R(i, :) / R(i, j), and subtracts a b^T; it stops once
// |R|_F <= tol |T|_F, at a zero residual, or after kmax terms.  One block per translation,
// FP64 throughout (entries from the FP64 translation and node offsets); the products are
// rounded before the subtraction (no contraction) so that the pivots follow the plain
// FP64 arithmetic of the definition.
constexpr int ACA_T = 512, ACA_KMAX = 64;

struct AcaGeo {
    double oxy[3];
    double dl;
    int r1;
    double hnode[R1MAX];  // (d_l / 2) cos((2a+1) pi / (2 r1))
};

// Magnitudes are compared as the bit patterns of non-negative doubles (their order is the
// unsigned integer order), which keeps the maxima and the pivot search off the FP64 pipe.
__device__ __forceinline__ unsigned long long mag_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// block-wide sum and maximum in one pass (ACA_T threads)
__device__ __forceinline__ void aca_block_sum_max(double &sum, unsigned long long &mx, double *reds,
                                                  unsigned long long *redm) {
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        reds[threadIdx.x >> 5] = sum;
        redm[threadIdx.x >> 5] = mx;
    }
    __syncthreads();
    sum = 0.0;
    mx = 0ull;
    for (int w = 0; w < ACA_T / 32; ++w) {
        sum += reds[w];
        mx = max(mx, redm[w]);
    }
}

__device__ __forceinline__ unsigned aca_block_min(unsigned v, unsigned *red) {
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned s = 0xffffffffu;
    for (int w = 0; w < ACA_T / 32; ++w) s = min(s, red[w]);
    return s;
}

// The residual lives in shared memory when it fits (r <= 125: up to 125 KB), else in the
// global scratch R.
__global__ void __launch_bounds__(ACA_T) k_lag_aca(const int4 *__restrict__ m, AcaGeo g, double tol, int kmax,
                                                   int in_smem, double *__restrict__ R, double *__restrict__ Ad,
                                                   double *__restrict__ Bd, int *__restrict__ rank) {
    extern __shared__ double sR[];
    __shared__ double sa[R1MAX * R1MAX * R1MAX], sb[R1MAX * R1MAX * R1MAX];
    __shared__ double reds[ACA_T / 32];
    __shared__ unsigned long long redm[ACA_T / 32];
    __shared__ unsigned redi[ACA_T / 32];
    const int t = blockIdx.x, r1 = g.r1, r = r1 * r1 * r1, n = r * r;
    double *Rt = in_smem ? sR : R + (size_t)t * n;
    const int4 mt = m[t];
    const double r0x = g.oxy[0] + mt.x * g.dl, r0y = g.oxy[1] + mt.y * g.dl, r0z = g.oxy[2] + mt.z * g.dl;
    double m2 = 0.0;
    unsigned long long mx = 0ull;
    for (int e = threadIdx.x; e < n; e += ACA_T) {
        int i = e / r, j = e - i * r;
        int ix = i / (r1 * r1), iy = (i / r1) % r1, iz = i % r1;
        int jx = j / (r1 * r1), jy = (j / r1) % r1, jz = j % r1;
        double dx = r0x + (g.hnode[ix] - g.hnode[jx]), dy = r0y + (g.hnode[iy] - g.hnode[jy]),
               dz = r0z + (g.hnode[iz] - g.hnode[jz]);
        double v = 1.0 / (4.0 * 3.14159265358979323846 * sqrt(dx * dx + dy * dy + dz * dz));
        Rt[e] = v;
        m2 += v * v;
        mx = max(mx, mag_bits(v));
    }
    aca_block_sum_max(m2, mx, reds, redm);
    int k = 0;
    while (k < kmax && mx != 0ull) {
        const unsigned long long thr = mag_bits((1.0 - 1e-9) * __longlong_as_double((long long)mx));
        unsigned first = 0xffffffffu;
        for (int e = threadIdx.x; e < n; e += ACA_T)
            if (mag_bits(Rt[e]) >= thr) {
                first = (unsigned)e;
                break;
            }
        const unsigned piv = aca_block_min(first, redi);
        const int i = (int)(piv / (unsigned)r), j = (int)(piv % (unsigned)r);
        const double delta = Rt[piv];
        double *a = Ad + ((size_t)t * kmax + k) * r, *b = Bd + ((size_t)t * kmax + k) * r;
        for (int q = threadIdx.x; q < r; q += ACA_T) {
            double av = Rt[(size_t)q * r + j], bv = Rt[(size_t)i * r + q] / delta;
            sa[q] = av;
            sb[q] = bv;
            a[q] = av;
            b[q] = bv;
        }
        __syncthreads();
        double r2 = 0.0;
        mx = 0ull;
        for (int e = threadIdx.x; e < n; e += ACA_T) {
            int ii = e / r, jj = e - ii * r;
            double v = __dsub_rn(Rt[e], __dmul_rn(sa[ii], sb[jj]));
            Rt[e] = v;
            r2 = fma(v, v, r2);
            mx = max(mx, mag_bits(v));
        }
        aca_block_sum_max(r2, mx, reds, redm);
        ++k;
        if (r2 <= tol * tol * m2) break;
    }
    if (threadIdx.x == 0) rank[t] = k;
}

// FP32 operands of the two transfer stages: B^T as [t][rb][cb] (row q = b_q), A as
// [t][ra][ca] (column q = a_q), zero past the rank and past r.
__global__ void k_aca_pack(const double *__restrict__ Ad, const double *__restrict__ Bd, const int *__restrict__ rank,
                           int kmax, int r, int rb, int cb, int ra, int ca, float *__restrict__ Bt,
                           float *__restrict__ At) {
    const int t = blockIdx.x, kt = rank[t];
    for (int e = threadIdx.x; e < rb * cb; e += blockDim.x) {
        int q = e / cb, j = e - q * cb;
        Bt[(size_t)t * rb * cb + e] = (q < kt && j < r) ? (float)Bd[((size_t)t * kmax + q) * r + j] : 0.f;
    }
    for (int e = threadIdx.x; e < ra * ca; e += blockDim.x) {
        int i = e / ca, q = e - i * ca;
        At[(size_t)t * ra * ca + e] = (q < kt && i < r) ? (float)Ad[((size_t)t * kmax + q) * r + i] : 0.f;
    }
}

__global__ void k_aca_pair_id(uint32_t *id, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = (uint32_t)i;
}

static void build_aca(ffm_plan_s *p, int l, const double oxy[3], double dl, TableJob &tj) {
    FarLevel &F = p->far[l];
    cudaStream_t s = tj.side;
    Alloc &tmp = tj.tmp;
    const int r = F.r1 * F.r1 * F.r1, kmax = std::min(r, ACA_KMAX), nt = F.n_trans;
    AcaGeo g{};
    for (int d = 0; d < 3; ++d) g.oxy[d] = oxy[d];
    g.dl = dl;
    g.r1 = F.r1;
    for (int a = 0; a < F.r1; ++a) g.hnode[a] = 0.5 * dl * std::cos((2.0 * a + 1.0) * PI / (2.0 * F.r1));
    const size_t rbytes = sizeof(double) * (size_t)r * r;
    const int in_smem = rbytes <= 125 * 1024;
    double *R = in_smem ? nullptr : tmp.get<double>((size_t)nt * r * r);
    double *Ad = tmp.get<double>((size_t)nt * kmax * r), *Bd = tmp.get<double>((size_t)nt * kmax * r);
    int *rank = tmp.get<int>(nt);
    FFM_CUDA(cudaFuncSetAttribute(k_lag_aca, cudaFuncAttributeMaxDynamicSharedMemorySize, 125 * 1024));
    FFM_LAUNCH(k_lag_aca, nt, ACA_T, in_smem ? rbytes : 0, s, F.trans_m, g, p->aca_eps, kmax, in_smem, R, Ad, Bd,
               rank);
    std::vector<int> hr(nt);
    FFM_CUDA(cudaMemcpyAsync(hr.data(), rank, sizeof(int) * nt, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    if (R) tmp.drop(R);
    int kt = 1;
    for (int v : hr) kt = std::max(kt, v);
    // ACA terms over the translations, and over the pairs (each pair applies its translation's)
    std::vector<uint32_t> hoff(nt + 1);
    FFM_CUDA(cudaMemcpyAsync(hoff.data(), F.bt_off, sizeof(uint32_t) * (nt + 1), cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    int64_t terms = 0, pair_terms = 0;
    for (int t = 0; t < nt; ++t) {
        terms += hr[t];
        pair_terms += (int64_t)hr[t] * (hoff[t + 1] - hoff[t]);
    }
    p->info.aca_terms[l] = terms;
    p->info.aca_pair_terms[l] = pair_terms;
    F.aca = true;
    F.aca_rank = kt;
    p->info.aca_rank[l] = kt;
    const int npad = (r + 15) / 16 * 16, rp16 = (kt + 15) / 16 * 16;
    // tensor cores (the tcgen05 transfer in row blocks of at most 224), unless the CUDA-core
    // transfer is forced
    F.aca_tc = rp16 <= 224 && F.tc_tiles > 0 && F.rkp > 0 && p->lag_transfer != 1;
    F.aca_rp = F.aca_tc ? rp16 : kt;
    const int rb = F.aca_rp, cb = F.aca_tc ? F.rkp : r, ra = F.aca_tc ? npad : r, ca = F.aca_rp;
    F.Bca = p->mem.get<float>((size_t)nt * rb * cb);
    F.Aca = p->mem.get<float>((size_t)nt * ra * ca);
    FFM_LAUNCH(k_aca_pack, nt, 256, 0, s, Ad, Bd, rank, kmax, r, rb, cb, ra, ca, F.Bca, F.Aca);
    F.pair_id = p->mem.get<uint32_t>((size_t)F.n_adm);
    FFM_LAUNCH(k_aca_pair_id, cdiv(F.n_adm, 256), 256, 0, s, F.pair_id, F.n_adm);
}

void build_tables(ffm_plan_s *p, int l, TableJob &tj) {
    FarLevel &F = p->far[l];
    cudaStream_t s = tj.side;
    Alloc &tmp = tj.tmp;
    if (F.mode == 1 && F.r1 > R1MAX) fail(FFM_EUNSUPPORTED, "eps needs more than 8 Chebyshev nodes per axis");
    double dl = std::ldexp(p->d0, -l);
    double oxy[3] = {p->oX[0] - p->oY[0], p->oX[1] - p->oY[1], p->oX[2] - p->oY[2]};
    if (F.mode == 1) {
        int r = F.r1 * F.r1 * F.r1;
        bool cplx = p->kind == FFM_HELMHOLTZ;
        bool three = p->kind == FFM_LAPLACE_DL || p->kind == FFM_LAPLACE_GRAD;
        F.T = p->mem.get<float>((size_t)F.n_trans * r * r * (cplx ? 2 : three ? 3 : 1));
            LagGeo g{};
        for (int d = 0; d < 3; ++d) g.oxy[d] = oxy[d];
        g.dl = dl;
        g.k = (float)p->k;
        g.r1 = F.r1;
        g.kind = p->kind;
        for (int a = 0; a < F.r1; ++a) g.hnode[a] = (float)(0.5 * dl * std::cos((2.0 * a + 1.0) * PI / (2.0 * F.r1)));
        FFM_LAUNCH(k_lag_table, F.n_trans, 256, 0, s, F.trans_m, F.n_trans, g, F.T);
        int rk = p->kind == FFM_LAPLACE_DL ? 3 * r : r, npad = (r + 15) / 16 * 16;
        if (!cplx) {
            // the tensor-core transfer's operand: T_t with npad rows of rkp (a multiple of its
            // 16-node K chunks) floats, padding zero; the gradient's three component blocks one
            // after another
            int nblk = p->kind == FFM_LAPLACE_GRAD ? 3 : 1;
            F.rkp = (rk + 15) / 16 * 16;
            size_t tsz = (size_t)nblk * F.n_trans * npad * F.rkp;
            F.Tsh = p->mem.get<float>(tsz);
            split_pad(F.T, (int64_t)nblk * F.n_trans, r, rk, npad, F.rkp, F.Tsh, nullptr, s);
        }
        if (p->aca_eps > 0.0 && p->kind == FFM_LAPLACE) build_aca(p, l, oxy, dl, tj);
        return;
    }
    // plane waves: quadrature of eq. 17, (L+1) Gauss-Legendre nodes in cos(theta) times 2L
    // azimuths phi_j = j pi / L.  The set is antipodally symmetric (mu_{L-i} = -mu_i,
    // phi_{j+L} = phi_j + pi); it is ordered so that direction h + nQ/2 is exactly -s_h,
    // which lets the transforms derive both phasors of a pair from one sincos.
    int L = F.L, nQ = F.nQ, np = 2 * L, nH = nQ / 2;
    std::vector<double> mu, wg;
    gauss_legendre(L + 1, mu, wg);
    std::vector<D4> sw(nQ);
    {
        // the azimuths' cosines and sines depend on j only: 2L library calls, not 2 nQ
        std::vector<double> cph(np), sph(np);
        for (int j = 0; j < np; ++j) {
            double ph = j * PI / L;
            cph[j] = std::cos(ph);
            sph[j] = std::sin(ph);
        }
        int h = 0;
        auto put = [&](int i, int j) {
            double st = std::sqrt(1.0 - mu[i] * mu[i]);
            sw[h] = D4{st * cph[j], st * sph[j], mu[i], wg[i] * PI / L};
            sw[h + nH] = D4{-sw[h].x, -sw[h].y, -sw[h].z, sw[h].w};
            ++h;
        };
        for (int i = 0; i < (L + 1) / 2; ++i)
            for (int j = 0; j < np; ++j) put(i, j);
        if (L % 2 == 0)
            for (int j = 0; j < L; ++j) put(L / 2, j);  // equator: phi_j and phi_j + pi pair up
    }
    // Gegenbauer coefficients c_t[p] = (2p+1) i^p h_p(k |r0_t|) / (4 pi) and r0 directions
    int nt = F.n_trans;
    std::vector<double> cr((size_t)nt * (L + 1)), ci((size_t)nt * (L + 1));
    std::vector<D4> rhat(nt);
    std::vector<double> hr, hi;
    int tmin = 0;
    for (int t = 0; t < nt; ++t) {
        int4 m = F.h_trans_m[t];
        double r0[3] = {oxy[0] + m.x * dl, oxy[1] + m.y * dl, oxy[2] + m.z * dl};
        double R = std::sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
        rhat[t] = D4{r0[0] / R, r0[1] / R, r0[2] / R, R};
        if (R < rhat[tmin].w) tmin = t;
        hankel1(L, p->k * R, hr, hi);
        for (int q = 0; q <= L; ++q) {
            double ipr = (q % 4 == 0) ? 1.0 : (q % 4 == 2 ? -1.0 : 0.0);
            double ipi = (q % 4 == 1) ? 1.0 : (q % 4 == 3 ? -1.0 : 0.0);
            double f = (2.0 * q + 1.0) / (4.0 * PI);
            cr[(size_t)t * (L + 1) + q] = f * (ipr * hr[q] - ipi * hi[q]);
            ci[(size_t)t * (L + 1) + q] = f * (ipr * hi[q] + ipi * hr[q]);
        }
    }
    // Cancellation of the quadrature sum for the closest translation:
    // C = sum_q |D(q)| / |sum_q D(q)|, large at low k d_l where the Hankel terms with
    // p > k |r0| grow.  Rounding errors of the FP32 kernels are amplified by about C:
    // measured on ill-conditioned cube surfaces, the result moves by up to ~2.3e-9 C with
    // the hardware sincos and ~1.3e-9 C with the compensated kernels.  The level runs
    // FP32 for C <= 250, compensated FP32 for C <= 4e3 (both below 6e-6), FP64 above.
    F.cancel = 0.0;
    if (L > 1.1 * p->k * rhat[tmin].w) {
        double sa = 0.0, ar = 0.0, ai = 0.0;
        const D4 &rh = rhat[tmin];
        for (int q = 0; q < nQ; ++q) {
            double x = sw[q].x * rh.x + sw[q].y * rh.y + sw[q].z * rh.z;
            double p0 = 1.0, p1 = x, tr = cr[(size_t)tmin * (L + 1)], ti = ci[(size_t)tmin * (L + 1)];
            tr += cr[(size_t)tmin * (L + 1) + 1] * x;
            ti += ci[(size_t)tmin * (L + 1) + 1] * x;
            for (int pp = 1; pp < L; ++pp) {
                double p2 = ((2.0 * pp + 1.0) * x * p1 - pp * p0) / (pp + 1.0);
                p0 = p1;
                p1 = p2;
                tr += cr[(size_t)tmin * (L + 1) + pp + 1] * p2;
                ti += ci[(size_t)tmin * (L + 1) + pp + 1] * p2;
            }
            sa += sw[q].w * std::sqrt(tr * tr + ti * ti);
            ar += sw[q].w * tr;
            ai += sw[q].w * ti;
        }
        F.cancel = sa / std::sqrt(ar * ar + ai * ai);
    }
    if (p->precision != FFM_PREC_AUTO)
        F.prec = p->precision;
    else
        F.prec = F.cancel <= 250.0 ? FFM_PREC_F32 : F.cancel <= 4e3 ? FFM_PREC_F32C : FFM_PREC_F32X2;
    p->info.pw_prec[l] = F.prec;
    bool dbl = F.prec == FFM_PREC_F64, dfl = F.prec == FFM_PREC_F32X2;
    p->info.cancel[l] = F.cancel;
    std::vector<float4> coef((size_t)nt * (L + 1));
    for (size_t i = 0; i < coef.size(); ++i) {
        float a = (float)cr[i], b = (float)ci[i];
        coef[i] = make_float4(a, (float)(cr[i] - (double)a), b, (float)(ci[i] - (double)b));
    }
    std::vector<float2> beta(L > 0 ? L : 1);
    for (int q = 0; q < L; ++q) {
        double bq = (double)q / (q + 1.0);
        float h = (float)bq;
        beta[q] = make_float2(h, (float)(bq - (double)h));
    }
    // canonical translations: t with its partner -m (when the root centres coincide the
    // set of translations is symmetric and -m has the same coefficients)
    std::vector<int2> pairs;
    {
        bool same_centre = oxy[0] == 0.0 && oxy[1] == 0.0 && oxy[2] == 0.0;
        std::map<std::tuple<int, int, int>, int> idx;
        if (same_centre)
            for (int t = 0; t < nt; ++t) idx[{F.h_trans_m[t].x, F.h_trans_m[t].y, F.h_trans_m[t].z}] = t;
        for (int t = 0; t < nt; ++t) {
            int partner = -1;
            if (same_centre) {
                auto it = idx.find({-F.h_trans_m[t].x, -F.h_trans_m[t].y, -F.h_trans_m[t].z});
                if (it != idx.end()) partner = it->second;
            }
            if (partner >= 0 && partner < t) continue;  // done with its partner
            pairs.push_back(make_int2(t, partner == t ? -1 : partner));
        }
    }
    int npairs = (int)pairs.size();
    dim3 g1(cdiv(nH, 256), npairs);
    p->info.pw_recurrences[l] = (int64_t)npairs * nH;
    size_t sm1 = sizeof(float4) * (L + 1) + sizeof(float2) * L;
    if (dbl) {
        F.ksd = p->mem.get<D4>(nQ);
        F.Dd = p->mem.get<double2>((size_t)nt * nQ);
    } else if (dfl) {
        F.ksx = p->mem.get<dd4>(nQ);
        F.Dx = p->mem.get<dd2>((size_t)nt * nQ);
        if (!p->sctab) {
            // sin and cos of j/64 for the double-float sincos
            std::vector<float4> tab(2 * DD_SC_J + 1);
            for (int j = -DD_SC_J; j <= DD_SC_J; ++j) {
                double a = j / 64.0, sa = std::sin(a), ca = std::cos(a);
                float sh = (float)sa, ch = (float)ca;
                tab[j + DD_SC_J] = make_float4(sh, (float)(sa - (double)sh), ch, (float)(ca - (double)ch));
            }
            p->sctab = p->mem.get<float4>(tab.size());
            size_t nb = sizeof(float4) * tab.size();
            FFM_CUDA(cudaMemcpyAsync(p->sctab, tj.keep.hold(std::move(tab)), nb, cudaMemcpyHostToDevice, s));
        }
    } else {
        F.ks = p->mem.get<float4>(nQ);
        F.D = p->mem.get<float2>((size_t)nt * nQ);
    }
    D4 *d_sw = tmp.get<D4>(nQ);
    tj.d_sw[l] = d_sw;
    float4 *d_coef = tmp.get<float4>(coef.size());
    float2 *d_beta = tmp.get<float2>(beta.size());
    D4 *d_rhat = tmp.get<D4>(nt);
    int2 *d_pairs = tmp.get<int2>(npairs);
    HostKeep &keep = tj.keep;
    const D4 *h_sw = keep.hold(std::vector<D4>(sw));
    size_t ncoef = coef.size(), nbeta = beta.size();
    FFM_CUDA(cudaMemcpyAsync(d_sw, h_sw, sizeof(D4) * nQ, cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(d_coef, keep.hold(std::move(coef)), sizeof(float4) * ncoef, cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(d_beta, keep.hold(std::move(beta)), sizeof(float2) * nbeta, cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(d_rhat, keep.hold(std::move(rhat)), sizeof(D4) * nt, cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(d_pairs, keep.hold(std::move(pairs)), sizeof(int2) * npairs, cudaMemcpyHostToDevice, s));
    if (dbl) {
        std::vector<D4> ks(nQ);
        for (int q = 0; q < nQ; ++q) ks[q] = D4{p->k * sw[q].x, p->k * sw[q].y, p->k * sw[q].z, 0.0};
        FFM_CUDA(cudaMemcpyAsync(F.ksd, keep.hold(std::move(ks)), sizeof(D4) * nQ, cudaMemcpyHostToDevice, s));
        FFM_LAUNCH(k_pw_table<double2>, g1, 256, sm1, s, d_sw, nH, d_coef, d_beta, L, d_rhat, d_pairs, p->k, F.Dd);
    } else if (dfl) {
        auto sp = [](double v) {
            float h = (float)v;
            return dd(h, (float)(v - (double)h));
        };
        std::vector<dd4> ks(nQ);
        for (int q = 0; q < nQ; ++q)
            ks[q] = dd4{sp(p->k * sw[q].x), sp(p->k * sw[q].y), sp(p->k * sw[q].z), dd(0.f)};
        FFM_CUDA(cudaMemcpyAsync(F.ksx, keep.hold(std::move(ks)), sizeof(dd4) * nQ, cudaMemcpyHostToDevice, s));
        FFM_LAUNCH(k_pw_table<dd2>, g1, 256, sm1, s, d_sw, nH, d_coef, d_beta, L, d_rhat, d_pairs, p->k, F.Dx);
    } else {
        std::vector<float4> ks(nQ);
        for (int q = 0; q < nQ; ++q)
            ks[q] = make_float4((float)(p->k * sw[q].x), (float)(p->k * sw[q].y), (float)(p->k * sw[q].z), 0.f);
        FFM_CUDA(cudaMemcpyAsync(F.ks, keep.hold(std::move(ks)), sizeof(float4) * nQ, cudaMemcpyHostToDevice, s));
        // the FP32 table only where the sum is well conditioned (a forced FP32 level with a large
        // cancellation ratio keeps the double-float table, so only the sum itself is FP32)
        if (F.prec == FFM_PREC_F32 && F.cancel <= 250.0)
            FFM_LAUNCH(k_pw_table_f32, g1, 256, sm1, s, d_sw, nH, d_coef, d_beta, L, d_rhat, d_pairs, p->k, F.D);
        else
            FFM_LAUNCH(k_pw_table<float2>, g1, 256, sm1, s, d_sw, nH, d_coef, d_beta, L, d_rhat, d_pairs, p->k, F.D);
    }
}

void build_octants(ffm_plan_s *p, int l, TableJob &tj) {
    FarLevel &F = p->far[l];
    int ndepth = p->l_stop - l;
    if (F.mode != 2 || ndepth <= 0) return;
    int nQ = F.nQ;
    dim3 g2(cdiv(nQ, 128), ndepth, 8);
    double half = std::ldexp(p->d0, -(l + 1));
    if (F.prec == FFM_PREC_F64) {
        F.Ed = p->mem.get<double2>((size_t)ndepth * 8 * nQ);
        FFM_LAUNCH(k_pw_octants<double2>, g2, 128, 0, tj.side, tj.d_sw[l], nQ, p->k, half, ndepth, F.Ed);
    } else if (F.prec == FFM_PREC_F32X2) {
        F.Ex = p->mem.get<dd2>((size_t)ndepth * 8 * nQ);
        FFM_LAUNCH(k_pw_octants<dd2>, g2, 128, 0, tj.side, tj.d_sw[l], nQ, p->k, half, ndepth, F.Ex);
    } else {
        F.E = p->mem.get<float2>((size_t)ndepth * 8 * nQ);
        FFM_LAUNCH(k_pw_octants<float2>, g2, 128, 0, tj.side, tj.d_sw[l], nQ, p->k, half, ndepth, F.E);
    }
}

}  // namespace ffm
