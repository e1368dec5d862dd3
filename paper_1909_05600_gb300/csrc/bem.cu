// Boundary-element wrapper around the FFM (Sec. 4.2): the Galerkin matrix of the Laplace single
// layer on P1 (nodal, piecewise-linear) functions over a flat-triangle mesh,
//   S = (Lambda*)^T (G W) Lambda + C,
// with 3-point node quadrature per triangle (barycentric (2/3, 1/6, 1/6) and permutations,
// weights area / 3): Lambda carries vertex values to the nodes, G W is one FFM product over
// the nodes (coincident nodes skipped), (Lambda*)^T brings the weighted node values back to
// the vertices, and the sparse C replaces each triangle's node-quadrature self-interaction
// by its exact element matrix (the inner integral in closed form: the in-plane potential of
// a linear density on a flat triangle; the outer by a collapsed 32 x 32 Gauss rule).  The
// system S x = b is solved by restarted GMRES whose vector work runs in this file's kernels
// and whose products are the FFM; the small Hessenberg problem is solved on the host.
#include <cmath>
#include <algorithm>
#include <vector>

#include "ffm_internal.cuh"

namespace ffm {
namespace {

constexpr int BEM_OUTER = 32;  // collapsed Gauss rule of the self-element integrals

struct GlOuter {
    double t[BEM_OUTER], w[BEM_OUTER];
};

__constant__ double c_bary[3][3] = {{2.0 / 3, 1.0 / 6, 1.0 / 6}, {1.0 / 6, 2.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 6, 2.0 / 3}};

__device__ __forceinline__ double3 sub3(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double dot3(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 cross3(double3 a, double3 b) {
    return make_double3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double3 axpy3(double a, double3 x, double3 y) {
    return make_double3(a * x.x + y.x, a * x.y + y.y, a * x.z + y.z);
}
__device__ __forceinline__ double norm3(double3 a) { return sqrt(dot3(a, a)); }

// quadrature nodes (3 per triangle) and weights
__global__ void k_bem_nodes(const double *__restrict__ V, const int *__restrict__ F, int64_t nt,
                            double *__restrict__ X, double *__restrict__ w) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    double3 p[3];
    for (int k = 0; k < 3; ++k) {
        int v = F[3 * t + k];
        p[k] = make_double3(V[3 * v], V[3 * v + 1], V[3 * v + 2]);
    }
    double area = 0.5 * norm3(cross3(sub3(p[1], p[0]), sub3(p[2], p[0])));
    for (int q = 0; q < 3; ++q) {
        double3 x = make_double3(0, 0, 0);
        for (int k = 0; k < 3; ++k) x = axpy3(c_bary[q][k], p[k], x);
        X[3 * (3 * t + q)] = x.x;
        X[3 * (3 * t + q) + 1] = x.y;
        X[3 * (3 * t + q) + 2] = x.z;
        w[3 * t + q] = area / 3.0;
    }
}

// Self-interaction correction of triangle t: exact element matrix minus the node quadrature.
// One block per triangle, threads over the outer Gauss points; the inner integral of phi_b(y)
// / |x - y| over the triangle at an in-plane point x is V0 phi_b(x) + grad phi_b . Vv with
// V0 = sum_e d_e ln((s+ + R+) / (s- + R-)) and Vv = sum_e d_e [n_e (atan(s+/d_e) -
// atan(s-/d_e)) + t_e ln(R+/R-)] (polar coordinates about x, edge by edge).
__global__ void __launch_bounds__(256) k_bem_self(const double *__restrict__ V, const int *__restrict__ F,
                                                  GlOuter g, double *__restrict__ C9) {
    __shared__ double red[256][9];
    int64_t t = blockIdx.x;
    double3 p[3];
    for (int k = 0; k < 3; ++k) {
        int v = F[3 * t + k];
        p[k] = make_double3(V[3 * v], V[3 * v + 1], V[3 * v + 2]);
    }
    double3 nrm = cross3(sub3(p[1], p[0]), sub3(p[2], p[0]));
    double area2 = norm3(nrm);
    double3 grad[3] = {cross3(nrm, sub3(p[2], p[1])), cross3(nrm, sub3(p[0], p[2])), cross3(nrm, sub3(p[1], p[0]))};
    for (int k = 0; k < 3; ++k) {
        double s = 1.0 / (area2 * area2);
        grad[k] = make_double3(grad[k].x * s, grad[k].y * s, grad[k].z * s);
    }
    double acc[9];
    for (int i = 0; i < 9; ++i) acc[i] = 0.0;
    for (int o = threadIdx.x; o < BEM_OUTER * BEM_OUTER; o += blockDim.x) {
        double u = g.t[o / BEM_OUTER], v = g.t[o % BEM_OUTER];
        double wo = g.w[o / BEM_OUTER] * g.w[o % BEM_OUTER] * u * area2;
        double lam[3] = {1.0 - u, u * (1.0 - v), u * v};
        double3 x = make_double3(0, 0, 0);
        for (int k = 0; k < 3; ++k) x = axpy3(lam[k], p[k], x);
        double V0 = 0.0;
        double3 Vv = make_double3(0, 0, 0);
        for (int e = 0; e < 3; ++e) {
            double3 a = p[e], b = p[(e + 1) % 3];
            double3 ab = sub3(b, a);
            double3 te = make_double3(ab.x / norm3(ab), ab.y / norm3(ab), ab.z / norm3(ab));
            double3 foot = axpy3(dot3(sub3(x, a), te), te, a);
            double3 ne = sub3(foot, x);
            double d = norm3(ne);
            ne = make_double3(ne.x / d, ne.y / d, ne.z / d);
            double sa = dot3(sub3(a, foot), te), sb = dot3(sub3(b, foot), te);
            double ra = norm3(sub3(x, a)), rb = norm3(sub3(x, b));
            V0 += d * log((sb + rb) / (sa + ra));
            Vv = axpy3(d * (atan(sb / d) - atan(sa / d)), ne, Vv);
            Vv = axpy3(d * log(rb / ra), te, Vv);
        }
        for (int bb = 0; bb < 3; ++bb) {
            double inner = (lam[bb] * V0 + dot3(grad[bb], Vv)) * (0.25 / PI);
            for (int aa = 0; aa < 3; ++aa) acc[aa * 3 + bb] += wo * lam[aa] * inner;
        }
    }
    for (int i = 0; i < 9; ++i) red[threadIdx.x][i] = acc[i];
    __syncthreads();
    if (threadIdx.x < 9) {
        double s = 0.0;
        for (int j = 0; j < (int)blockDim.x; ++j) s += red[j][threadIdx.x];
        // minus the node quadrature of the same interaction (coincident nodes skipped)
        int aa = threadIdx.x / 3, bb = threadIdx.x % 3;
        double3 xq[3];
        for (int q = 0; q < 3; ++q) {
            xq[q] = make_double3(0, 0, 0);
            for (int k = 0; k < 3; ++k) xq[q] = axpy3(c_bary[q][k], p[k], xq[q]);
        }
        double wq = 0.5 * area2 / 3.0, nodes = 0.0;
        for (int q = 0; q < 3; ++q)
            for (int r = 0; r < 3; ++r)
                if (q != r) nodes += c_bary[q][aa] * wq * (0.25 / PI) / norm3(sub3(xq[q], xq[r])) * wq * c_bary[r][bb];
        C9[9 * t + threadIdx.x] = s - nodes;
    }
}

// u~ = Lambda u: node value from the triangle's three vertex values
__global__ void k_bem_lambda(const int *__restrict__ F, int64_t nt, const double *__restrict__ u,
                             double *__restrict__ ug) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= 3 * nt) return;
    int64_t t = g / 3;
    int q = (int)(g - 3 * t);
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += c_bary[q][k] * u[F[3 * t + k]];
    ug[g] = s;
}

// v = (Lambda*)^T (w g) + C u: per vertex, its triangles' weighted node values (CSR of
// (triangle, corner) pairs) and its row of the correction
__global__ void k_bem_lambda_t(const int64_t *__restrict__ adj_off, const int *__restrict__ adj,
                               const double *__restrict__ w, const double *__restrict__ gv,
                               const int64_t *__restrict__ c_off, const int *__restrict__ c_col,
                               const double *__restrict__ c_val, const double *__restrict__ u, int64_t nv,
                               double *__restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double s = 0.0;
    for (int64_t e = adj_off[i]; e < adj_off[i + 1]; ++e) {
        int tk = adj[e];
        int64_t t = tk / 3;
        int k = tk - 3 * (int)t;
        for (int q = 0; q < 3; ++q) s += c_bary[q][k] * w[3 * t + q] * gv[3 * t + q];
    }
    for (int64_t e = c_off[i]; e < c_off[i + 1]; ++e) s += c_val[e] * u[c_col[e]];
    v[i] = s;
}

// ---- vector kernels of GMRES (n = number of vertices)
// h[j] = sum_i V[j][i] w[i] for j < nb (one block row per j, grid-stride over i)
__global__ void k_bem_dots(const double *__restrict__ Vb, int nb, int64_t n, const double *__restrict__ w,
                           double *__restrict__ h) {
    __shared__ double red[256];
    int j = blockIdx.y;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += Vb[(int64_t)j * n + i] * w[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&h[j], red[0]);
}
// w -= sum_j h[j] V[j]
__global__ void k_bem_orth(const double *__restrict__ Vb, int nb, int64_t n, const double *__restrict__ h,
                           double *__restrict__ w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = w[i];
    for (int j = 0; j < nb; ++j) s -= h[j] * Vb[(int64_t)j * n + i];
    w[i] = s;
}
// y = a x (+ y if acc)
__global__ void k_bem_axpy(double a, const double *__restrict__ x, int64_t n, int acc, double *__restrict__ y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * x[i] + (acc ? y[i] : 0.0);
}

}  // namespace
}  // namespace ffm

using namespace ffm;

struct ffm_bem_s {
    int64_t nv = 0, nt = 0;
    cudaStream_t stream = nullptr;
    Alloc mem;
    int *F = nullptr;
    double *w = nullptr;
    int64_t *adj_off = nullptr;
    int *adj = nullptr;
    int64_t *c_off = nullptr;
    int *c_col = nullptr;
    double *c_val = nullptr;
    ffm_plan_t *plan = nullptr;
    int64_t products = 0;  // FFM products of the last solve
    ~ffm_bem_s() {
        if (plan) ffm_destroy(plan);
    }
};

namespace {

template <class F>
ffm_status bem_guarded(F &&f) {
    try {
        f();
        return FFM_OK;
    } catch (const Error &e) {
        set_last_error(e.msg);
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return FFM_ENOMEM;
    } catch (...) {
        set_last_error("unexpected exception");
        return FFM_ECUDA;
    }
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
std::vector<T> host_copy(const T *p, size_t n, cudaStream_t s) {
    std::vector<T> h(n);
    FFM_CUDA(cudaMemcpyAsync(h.data(), p, sizeof(T) * n, on_device(p) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    return h;
}

void bem_apply(ffm_bem_s *b, const double *u, double *v, Alloc &tmp, cudaStream_t s) {
    int64_t ng = 3 * b->nt;
    double *ug = tmp.get<double>(ng), *gv = tmp.get<double>(ng);
    FFM_LAUNCH(k_bem_lambda, cdiv(ng, 256), 256, 0, s, b->F, b->nt, u, ug);
    ffm_status st = ffm_apply(b->plan, ug, FFM_F64, 1, gv, s);
    if (st != FFM_OK) fail(st, std::string("FFM product in the BEM operator: ") + ffm_last_error());
    FFM_LAUNCH(k_bem_lambda_t, cdiv(b->nv, 256), 256, 0, s, b->adj_off, b->adj, b->w, gv, b->c_off, b->c_col,
               b->c_val, u, b->nv, v);
    tmp.drop(gv);
    tmp.drop(ug);
}

}  // namespace

extern "C" {

ffm_status ffm_bem_create(const double *vertices, int64_t nv, const int *triangles, int64_t nt, ffm_kernel kernel,
                          double k, double eps, const ffm_opts *opts, void *stream, ffm_bem_t **out) {
    ffm_bem_s *b = nullptr;
    ffm_status st = bem_guarded([&] {
        if (!out || !vertices || !triangles) fail(FFM_EINVAL, "NULL argument");
        *out = nullptr;
        if (nv < 3 || nt < 1) fail(FFM_EINVAL, "the mesh needs at least one triangle");
        if (kernel != FFM_LAPLACE) fail(FFM_EUNSUPPORTED, "the boundary-element wrapper implements the Laplace single layer");
        (void)k;
        cudaStream_t s = (cudaStream_t)stream;
        b = new ffm_bem_s();
        b->nv = nv;
        b->nt = nt;
        b->stream = s;
        b->mem.stream = s;
        Alloc tmp;
        tmp.stream = s;
        // mesh on the host: checks and the vertex -> (triangle, corner) lists
        std::vector<int> hF = host_copy(triangles, 3 * (size_t)nt, s);
        std::vector<int64_t> off(nv + 1, 0);
        for (int64_t i = 0; i < 3 * nt; ++i) {
            if (hF[i] < 0 || hF[i] >= nv) fail(FFM_EINVAL, "triangle vertex index out of range");
            ++off[hF[i] + 1];
        }
        for (int64_t i = 0; i < nv; ++i) off[i + 1] += off[i];
        std::vector<int> adj(3 * nt);
        {
            std::vector<int64_t> cur(off.begin(), off.end() - 1);
            for (int64_t i = 0; i < 3 * nt; ++i) adj[cur[hF[i]]++] = (int)i;
        }
        b->F = b->mem.get<int>(3 * nt);
        FFM_CUDA(cudaMemcpyAsync(b->F, hF.data(), sizeof(int) * 3 * nt, cudaMemcpyHostToDevice, s));
        b->adj_off = b->mem.get<int64_t>(nv + 1);
        b->adj = b->mem.get<int>(3 * nt);
        FFM_CUDA(cudaMemcpyAsync(b->adj_off, off.data(), sizeof(int64_t) * (nv + 1), cudaMemcpyHostToDevice, s));
        FFM_CUDA(cudaMemcpyAsync(b->adj, adj.data(), sizeof(int) * 3 * nt, cudaMemcpyHostToDevice, s));
        const double *dV = vertices;
        if (!on_device(vertices)) {
            double *d = tmp.get<double>(3 * nv);
            FFM_CUDA(cudaMemcpyAsync(d, vertices, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, s));
            dV = d;
        }
        // quadrature nodes and weights; the FFM plan over the nodes
        int64_t ng = 3 * nt;
        double *X = tmp.get<double>(3 * ng);
        b->w = b->mem.get<double>(ng);
        FFM_LAUNCH(k_bem_nodes, cdiv(nt, 256), 256, 0, s, dV, b->F, nt, X, b->w);
        ffm_opts o{};
        if (opts) o = *opts;
        o.weights = b->w;
        o.weights_dtype = FFM_F64;
        ffm_status ps = ffm_plan(X, FFM_F64, ng, X, FFM_F64, ng, FFM_LAPLACE, 0.0, eps, &o, s, &b->plan);
        if (ps != FFM_OK) fail(ps, std::string("FFM plan over the quadrature nodes: ") + ffm_last_error());
        // self-interaction correction, assembled into CSR by vertex row
        GlOuter g;
        {
            std::vector<double> gt, gw;
            gauss_legendre_nodes(BEM_OUTER, gt, gw);
            for (int i = 0; i < BEM_OUTER; ++i) {
                g.t[i] = 0.5 * (gt[i] + 1.0);
                g.w[i] = 0.5 * gw[i];
            }
        }
        double *C9 = tmp.get<double>(9 * nt);
        FFM_LAUNCH(k_bem_self, (unsigned)nt, 256, 0, s, dV, b->F, g, C9);
        std::vector<double> hC = host_copy(C9, 9 * (size_t)nt, s);
        std::vector<std::pair<int64_t, double>> ent;
        ent.reserve(9 * nt);
        for (int64_t t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c) ent.push_back({(int64_t)hF[3 * t + a] * nv + hF[3 * t + c], hC[9 * t + 3 * a + c]});
        std::sort(ent.begin(), ent.end(), [](const auto &x, const auto &y) { return x.first < y.first; });
        std::vector<int64_t> coff(nv + 1, 0);
        std::vector<int> ccol;
        std::vector<double> cval;
        for (size_t i = 0; i < ent.size();) {
            size_t j = i;
            double sum = 0.0;
            while (j < ent.size() && ent[j].first == ent[i].first) sum += ent[j++].second;
            ccol.push_back((int)(ent[i].first % nv));
            cval.push_back(sum);
            ++coff[ent[i].first / nv + 1];
            i = j;
        }
        for (int64_t i = 0; i < nv; ++i) coff[i + 1] += coff[i];
        b->c_off = b->mem.get<int64_t>(nv + 1);
        b->c_col = b->mem.get<int>(ccol.size());
        b->c_val = b->mem.get<double>(cval.size());
        FFM_CUDA(cudaMemcpyAsync(b->c_off, coff.data(), sizeof(int64_t) * (nv + 1), cudaMemcpyHostToDevice, s));
        FFM_CUDA(cudaMemcpyAsync(b->c_col, ccol.data(), sizeof(int) * ccol.size(), cudaMemcpyHostToDevice, s));
        FFM_CUDA(cudaMemcpyAsync(b->c_val, cval.data(), sizeof(double) * cval.size(), cudaMemcpyHostToDevice, s));
        FFM_CUDA(cudaStreamSynchronize(s));
        tmp.release();
        *out = b;
    });
    if (st != FFM_OK && b) {
        cudaStreamSynchronize(b->stream);
        cudaGetLastError();
        delete b;
    }
    return st;
}

ffm_status ffm_bem_apply(ffm_bem_t *b, const double *u, double *v, void *stream) {
    return bem_guarded([&] {
        if (!b || !u || !v) fail(FFM_EINVAL, "NULL argument");
        cudaStream_t s = (cudaStream_t)stream;
        Alloc tmp;
        tmp.stream = s;
        const double *du = u;
        if (!on_device(u)) {
            double *d = tmp.get<double>(b->nv);
            FFM_CUDA(cudaMemcpyAsync(d, u, sizeof(double) * b->nv, cudaMemcpyHostToDevice, s));
            du = d;
        }
        bool host_v = !on_device(v);
        double *dv = host_v ? tmp.get<double>(b->nv) : v;
        bem_apply(b, du, dv, tmp, s);
        if (host_v) {
            FFM_CUDA(cudaMemcpyAsync(v, dv, sizeof(double) * b->nv, cudaMemcpyDeviceToHost, s));
            FFM_CUDA(cudaStreamSynchronize(s));
        }
        tmp.release();
    });
}

ffm_status ffm_bem_solve(ffm_bem_t *b, const double *rhs, double *x, double tol, int restart, int maxit, int *iters,
                         double *relres, void *stream) {
    return bem_guarded([&] {
        if (!b || !rhs || !x) fail(FFM_EINVAL, "NULL argument");
        if (!(tol > 0.0) || restart < 1 || maxit < 1) fail(FFM_EINVAL, "tol > 0, restart >= 1 and maxit >= 1 required");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t n = b->nv;
        const int m = restart;
        Alloc tmp;
        tmp.stream = s;
        double *db = tmp.get<double>(n);
        FFM_CUDA(cudaMemcpyAsync(db, rhs, sizeof(double) * n, on_device(rhs) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        double *dx = tmp.get<double>(n), *r = tmp.get<double>(n), *Vb = tmp.get<double>((size_t)(m + 1) * n);
        double *dh = tmp.get<double>(m + 1);
        FFM_CUDA(cudaMemsetAsync(dx, 0, sizeof(double) * n, s));
        const unsigned gb = cdiv(n, 256), gd = (unsigned)std::min<int64_t>(cdiv(n, 256), 152 * 4);
        auto dots = [&](int nb, const double *w, std::vector<double> &h) {
            FFM_CUDA(cudaMemsetAsync(dh, 0, sizeof(double) * nb, s));
            FFM_LAUNCH(k_bem_dots, dim3(gd, nb), 256, 0, s, Vb, nb, n, w, dh);
            h.resize(nb);
            FFM_CUDA(cudaMemcpyAsync(h.data(), dh, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
            FFM_CUDA(cudaStreamSynchronize(s));
        };
        auto norm_of = [&](const double *w) {
            FFM_CUDA(cudaMemsetAsync(dh, 0, sizeof(double), s));
            FFM_LAUNCH(k_bem_dots, dim3(gd, 1), 256, 0, s, w, 1, n, w, dh);
            double v = 0.0;
            FFM_CUDA(cudaMemcpyAsync(&v, dh, sizeof(double), cudaMemcpyDeviceToHost, s));
            FFM_CUDA(cudaStreamSynchronize(s));
            return std::sqrt(v);
        };
        const double bnorm = norm_of(db);
        if (bnorm == 0.0) {
            FFM_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));  // b = 0: x = 0
            if (iters) *iters = 0;
            if (relres) *relres = 0.0;
            return;
        }
        int it = 0;
        double res = 1.0;
        b->products = 0;
        std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gvec(m + 1), h, h2;
        while (it < maxit) {
            // r = b - S x (x = 0 at the start: r = b)
            if (it == 0) {
                FFM_CUDA(cudaMemcpyAsync(r, db, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            } else {
                bem_apply(b, dx, r, tmp, s);
                ++b->products;
                FFM_LAUNCH(k_bem_axpy, gb, 256, 0, s, -1.0, (const double *)r, n, 0, r);
                FFM_LAUNCH(k_bem_axpy, gb, 256, 0, s, 1.0, (const double *)db, n, 1, r);
            }
            double beta = norm_of(r);
            res = beta / bnorm;
            if (res <= tol) break;
            FFM_LAUNCH(k_bem_axpy, gb, 256, 0, s, 1.0 / beta, (const double *)r, n, 0, Vb);
            std::fill(gvec.begin(), gvec.end(), 0.0);
            gvec[0] = beta;
            int j = 0;
            for (; j < m && it < maxit; ++j, ++it) {
                double *wj = Vb + (size_t)(j + 1) * n;
                bem_apply(b, Vb + (size_t)j * n, wj, tmp, s);
                ++b->products;
                // classical Gram-Schmidt, twice
                dots(j + 1, wj, h);
                FFM_CUDA(cudaMemcpyAsync(dh, h.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
                FFM_LAUNCH(k_bem_orth, gb, 256, 0, s, Vb, j + 1, n, (const double *)dh, wj);
                dots(j + 1, wj, h2);
                FFM_CUDA(cudaMemcpyAsync(dh, h2.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
                FFM_LAUNCH(k_bem_orth, gb, 256, 0, s, Vb, j + 1, n, (const double *)dh, wj);
                for (int i = 0; i <= j; ++i) h[i] += h2[i];
                double hn = norm_of(wj);
                if (hn > 0.0) FFM_LAUNCH(k_bem_axpy, gb, 256, 0, s, 1.0 / hn, (const double *)wj, n, 0, wj);
                // Givens rotations of column j
                for (int i = 0; i < j; ++i) {
                    double a = cs[i] * h[i] + sn[i] * h[i + 1];
                    h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
                    h[i] = a;
                }
                double den = std::hypot(h[j], hn);
                cs[j] = den > 0 ? h[j] / den : 1.0;
                sn[j] = den > 0 ? hn / den : 0.0;
                h[j] = den;
                gvec[j + 1] = -sn[j] * gvec[j];
                gvec[j] = cs[j] * gvec[j];
                for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
                res = std::fabs(gvec[j + 1]) / bnorm;
                if (res <= tol || hn == 0.0) {
                    ++j;
                    ++it;
                    break;
                }
            }
            // x += V y with H y = g (upper triangular, j columns)
            std::vector<double> y(j);
            for (int i = j - 1; i >= 0; --i) {
                double sum = gvec[i];
                for (int c = i + 1; c < j; ++c) sum -= H[(size_t)i * m + c] * y[c];
                y[i] = sum / H[(size_t)i * m + i];
            }
            for (int i = 0; i < j; ++i)
                FFM_LAUNCH(k_bem_axpy, gb, 256, 0, s, y[i], (const double *)(Vb + (size_t)i * n), n, 1, dx);
            if (res <= tol) break;
        }
        FFM_CUDA(cudaMemcpyAsync(x, dx, sizeof(double) * n, on_device(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        FFM_CUDA(cudaStreamSynchronize(s));
        if (iters) *iters = it;
        if (relres) *relres = res;
        tmp.release();
    });
}

ffm_status ffm_bem_products(const ffm_bem_t *b, int64_t *products) {
    if (!b || !products) return FFM_EINVAL;
    *products = b->products;
    return FFM_OK;
}

void ffm_bem_destroy(ffm_bem_t *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    delete b;
    cudaGetLastError();
}

}  // extern "C"
