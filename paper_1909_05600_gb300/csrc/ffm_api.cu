// C ABI of libffm_gb300.so (include/ffm.h): argument checks, host/device staging, the
// apply sequence (gather w u in Morton order, far field per level, near field, FP64
// per-target accumulation, scatter to the caller's order) and plan introspection.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "ffm_internal.cuh"
#include <memory>

namespace ffm {

std::atomic<uint64_t> g_launches{0};
static thread_local std::string g_last_error;

// ------------------------------------------------------------- profiling

bool g_profile = false;
thread_local int64_t *g_capture_count = nullptr;
struct ProfRec {
    std::string name;
    cudaEvent_t e0, e1;
};
// Open records, and a pool of event pairs reused after each flush, so that a profiled
// launch costs two event records on the host and no event creation.
static std::vector<ProfRec> g_prof_open;
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_prof_pool;
static std::vector<std::pair<std::string, std::pair<uint64_t, double>>> g_prof_tot;

void profile_begin(const char *name, cudaStream_t s) {
    ProfRec r;
    r.name = name;
    if (!g_prof_pool.empty()) {
        r.e0 = g_prof_pool.back().first;
        r.e1 = g_prof_pool.back().second;
        g_prof_pool.pop_back();
    } else {
        cudaEventCreate(&r.e0);
        cudaEventCreate(&r.e1);
    }
    cudaEventRecord(r.e0, s);
    g_prof_open.push_back(r);
}

void profile_end(cudaStream_t s) { cudaEventRecord(g_prof_open.back().e1, s); }

static void profile_flush() {
    for (ProfRec &r : g_prof_open) {
        cudaEventSynchronize(r.e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        g_prof_pool.push_back({r.e0, r.e1});
        bool found = false;
        for (auto &t : g_prof_tot)
            if (t.first == r.name) {
                t.second.first += 1;
                t.second.second += ms;
                found = true;
                break;
            }
        if (!found) g_prof_tot.push_back({r.name, {1, (double)ms}});
    }
    g_prof_open.clear();
    cudaGetLastError();
}

void fail(ffm_status s, const std::string &msg) { throw Error{s, msg}; }

void set_last_error(const std::string &msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    ffm_status s = (e == cudaErrorMemoryAllocation) ? FFM_ENOMEM : FFM_ECUDA;
    if (s == FFM_ENOMEM) cudaGetLastError();  // clear the sticky-free allocation error
    fail(s, std::string(what) + ": " + cudaGetErrorString(e));
}

void *Alloc::raw(size_t n) {
    void *p = nullptr;
    if (n == 0) n = 16;
    cudaError_t e = cudaMallocAsync(&p, n, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? FFM_ENOMEM : FFM_ECUDA,
             std::string("device allocation of ") + std::to_string(n) + " bytes: " + cudaGetErrorString(e));
    }
    ptrs.push_back(p);
    bytes += n;
    return p;
}

void Alloc::drop(void *p) {
    for (size_t i = 0; i < ptrs.size(); ++i)
        if (ptrs[i] == p) {
            cudaFreeAsync(p, stream);
            ptrs.erase(ptrs.begin() + (long)i);
            return;
        }
}

void Alloc::release() {
    for (void *p : ptrs) cudaFreeAsync(p, stream);
    ptrs.clear();
    bytes = 0;
}

// The default pool of each device keeps freed memory (stream-ordered frees of one product
// are reused by the next); set once per device.
static void keep_pool_memory() {
    static std::atomic<bool> done[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return;
    }
    if (done[dev].load()) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev].store(true);
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------ apply kernels

// q_j = w_j u_{perm_j} for every right-hand side, in Morton order, rounded to FP32.
template <class UT, bool CPLX>
__global__ void k_gather_q(const UT *__restrict__ u, const uint32_t *__restrict__ perm, const double *__restrict__ w,
                           int64_t ny, int nrhs, void *__restrict__ q) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (j >= ny) return;
    int64_t o = (int64_t)perm[j] + (int64_t)m * ny;
    double wj = w ? w[j] : 1.0;
    if constexpr (CPLX) {
        double re = (double)u[2 * o] * wj, im = (double)u[2 * o + 1] * wj;
        reinterpret_cast<float2 *>(q)[(int64_t)m * ny + j] = make_float2((float)re, (float)im);
    } else {
        reinterpret_cast<float *>(q)[(int64_t)m * ny + j] = (float)((double)u[o] * wj);
    }
}

// v = near field and plane-wave levels (FP64 accumulators) + Lagrange levels (FP32), summed
// in FP64 per target, back in the caller's order.
// Double layer: q_j = w_j u_{perm_j} n_j, a 3-vector per source and right-hand side, formed
// in FP64 and stored as an unevaluated FP32 pair: q[2 (m ny + j)] = hi, [+1] = lo.
template <class UT>
__global__ void k_gather_q_dl(const UT *__restrict__ u, const uint32_t *__restrict__ perm,
                              const double *__restrict__ w, const float4 *__restrict__ nh,
                              const float4 *__restrict__ nl, int64_t ny, float4 *__restrict__ q) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int m = blockIdx.y;
    if (j >= ny) return;
    double s = (double)u[(int64_t)perm[j] + (int64_t)m * ny] * (w ? w[j] : 1.0);
    float4 a = nh[j], b = nl[j];
    double qx = s * ((double)a.x + (double)b.x), qy = s * ((double)a.y + (double)b.y), qz = s * ((double)a.z + (double)b.z);
    float hx = (float)qx, hy = (float)qy, hz = (float)qz;
    int64_t o = 2 * ((int64_t)m * ny + j);
    q[o] = make_float4(hx, hy, hz, 0.f);
    q[o + 1] = make_float4((float)(qx - (double)hx), (float)(qy - (double)hy), (float)(qz - (double)hz), 0.f);
}

// accumulator slot sl = d nrhs + m (d < ncomp) -> output column ncomp m + d
template <class VT, bool CPLX>
__global__ void k_scatter_v(const double2 *__restrict__ acc, const float2 *__restrict__ accf,
                            const uint32_t *__restrict__ perm, int64_t nx, int nrhs, int ncomp, VT *__restrict__ v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int sl = blockIdx.y;
    if (i >= nx) return;
    double2 a = acc[(int64_t)sl * nx + i];
    float2 f = accf[(int64_t)sl * nx + i];
    a.x += (double)f.x;
    a.y += (double)f.y;
    int col = ncomp == 1 ? sl : ncomp * (sl % nrhs) + sl / nrhs;
    int64_t o = (int64_t)perm[i] + (int64_t)col * nx;
    if constexpr (CPLX) {
        v[2 * o] = (VT)a.x;
        v[2 * o + 1] = (VT)a.y;
    } else {
        v[o] = (VT)a.x;
    }
}

static size_t dtype_size(ffm_dtype d) {
    switch (d) {
        case FFM_F32: return 4;
        case FFM_F64: return 8;
        case FFM_C64: return 8;
        case FFM_C128: return 16;
    }
    return 0;
}

static void apply_impl(ffm_plan_s *p, const void *u, ffm_dtype udt, int nrhs, void *v, cudaStream_t s) {
    bool helm = p->kind == FFM_HELMHOLTZ;
    if (helm && udt != FFM_C64 && udt != FFM_C128) fail(FFM_EINVAL, "Helmholtz densities must be FFM_C64 or FFM_C128");
    if (!helm && udt != FFM_F32 && udt != FFM_F64) fail(FFM_EINVAL, "Laplace densities must be FFM_F32 or FFM_F64");
    Alloc tmp;
    tmp.stream = s;
    int64_t nx = p->nx, ny = p->ny;
    const int ncomp = p->kind == FFM_LAPLACE_GRAD ? 3 : 1;  // outputs per target and density
    const int nout = ncomp * nrhs;
    if (nout > 65535) fail(FFM_EINVAL, "the gradient takes at most 21845 right-hand sides");
    size_t ub = dtype_size(udt) * (size_t)ny * nrhs, vb = dtype_size(udt) * (size_t)nx * nout;
    const void *du = u;
    if (!is_device_ptr(u)) {
        void *d = tmp.raw(ub);
        FFM_CUDA(cudaMemcpyAsync(d, u, ub, cudaMemcpyHostToDevice, s));
        du = d;
    }
    bool host_v = !is_device_ptr(v);
    void *dv = host_v ? tmp.raw(vb) : v;
    bool dl = p->kind == FFM_LAPLACE_DL;
    void *q = tmp.raw((dl ? 32 : helm ? 8 : 4) * (size_t)ny * nrhs);
    double2 *acc = tmp.get<double2>((size_t)nx * nout);
    FFM_CUDA(cudaMemsetAsync(acc, 0, sizeof(double2) * (size_t)nx * nout, s));
    float2 *accf = tmp.get<float2>((size_t)nx * nout);
    FFM_CUDA(cudaMemsetAsync(accf, 0, sizeof(float2) * (size_t)nx * nout, s));
    dim3 gy(cdiv(ny, 256), nrhs), gx(cdiv(nx, 256), nout);
    if (dl) {
        if (udt == FFM_F64)
            FFM_LAUNCH(k_gather_q_dl<double>, gy, 256, 0, s, (const double *)du, p->permY, p->wY, p->nY, p->nYlo, ny,
                       (float4 *)q);
        else
            FFM_LAUNCH(k_gather_q_dl<float>, gy, 256, 0, s, (const float *)du, p->permY, p->wY, p->nY, p->nYlo, ny,
                       (float4 *)q);
    } else switch (udt) {
        case FFM_F32: FFM_LAUNCH((k_gather_q<float, false>), gy, 256, 0, s, (const float *)du, p->permY, p->wY, ny, nrhs, q); break;
        case FFM_F64: FFM_LAUNCH((k_gather_q<double, false>), gy, 256, 0, s, (const double *)du, p->permY, p->wY, ny, nrhs, q); break;
        case FFM_C64: FFM_LAUNCH((k_gather_q<float, true>), gy, 256, 0, s, (const float *)du, p->permY, p->wY, ny, nrhs, q); break;
        case FFM_C128: FFM_LAUNCH((k_gather_q<double, true>), gy, 256, 0, s, (const double *)du, p->permY, p->wY, ny, nrhs, q); break;
    }
    for (int l = 0; l <= p->l_stop; ++l) {
        const FarLevel &F = p->far[l];
        if (F.n_adm == 0) continue;
        if (F.mode == 1)
            far_lagrange(p, l, q, nrhs, accf, tmp, s);
        else
            far_planewave(p, l, (const float2 *)q, nrhs, acc, tmp, s);
    }
    near_field(p, q, nrhs, acc, s);
    switch (udt) {
        case FFM_F32: FFM_LAUNCH((k_scatter_v<float, false>), gx, 256, 0, s, acc, accf, p->permX, nx, nrhs, ncomp, (float *)dv); break;
        case FFM_F64: FFM_LAUNCH((k_scatter_v<double, false>), gx, 256, 0, s, acc, accf, p->permX, nx, nrhs, ncomp, (double *)dv); break;
        case FFM_C64: FFM_LAUNCH((k_scatter_v<float, true>), gx, 256, 0, s, acc, accf, p->permX, nx, nrhs, ncomp, (float *)dv); break;
        case FFM_C128: FFM_LAUNCH((k_scatter_v<double, true>), gx, 256, 0, s, acc, accf, p->permX, nx, nrhs, ncomp, (double *)dv); break;
    }
    if (host_v) {
        FFM_CUDA(cudaMemcpyAsync(v, dv, vb, cudaMemcpyDeviceToHost, s));
        FFM_CUDA(cudaStreamSynchronize(s));
    }
    tmp.release();
}

static uint64_t spread_host(uint64_t g) {
    uint64_t r = 0;
    for (int b = 0; b < LMAX; ++b) r |= ((g >> b) & 1ull) << (3 * b);
    return r;
}
static uint64_t morton_host(int4 g) {
    return (spread_host((uint64_t)g.x) << 2) | (spread_host((uint64_t)g.y) << 1) | spread_host((uint64_t)g.z);
}

template <class T>
static std::vector<T> to_host(const T *d, size_t n, cudaStream_t s) {
    std::vector<T> h(n);
    if (n) FFM_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
    return h;
}

}  // namespace ffm

using namespace ffm;

template <class F>
static ffm_status guarded(F &&f) {
    try {
        f();
        return FFM_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return FFM_ENOMEM;
    } catch (...) {
        g_last_error = "unexpected exception";
        return FFM_ECUDA;
    }
}

extern "C" {

ffm_status ffm_plan(const void *X, ffm_dtype xdt, int64_t nx, const void *Y, ffm_dtype ydt, int64_t ny,
                    ffm_kernel kernel, double k, double eps, const ffm_opts *opts, void *stream, ffm_plan_t **out) {
    if (out) *out = nullptr;
    ffm_plan_s *p = nullptr;
    ffm_status st = guarded([&] {
        if (!out || !X || !Y) fail(FFM_EINVAL, "NULL argument");
        if (nx < 1 || ny < 1) fail(FFM_EINVAL, "point sets must be non-empty");
        if ((int64_t)nx + ny >= ((int64_t)1 << 31)) fail(FFM_EUNSUPPORTED, "more than 2^31 points in total");
        if (xdt != FFM_F32 && xdt != FFM_F64) fail(FFM_EINVAL, "X dtype must be FFM_F32 or FFM_F64");
        if (ydt != FFM_F32 && ydt != FFM_F64) fail(FFM_EINVAL, "Y dtype must be FFM_F32 or FFM_F64");
        if (kernel != FFM_LAPLACE && kernel != FFM_HELMHOLTZ && kernel != FFM_LAPLACE_DL && kernel != FFM_LAPLACE_GRAD)
            fail(FFM_EINVAL, "unknown kernel");
        if (kernel == FFM_LAPLACE_DL && (!opts || !opts->normals))
            fail(FFM_EINVAL, "the double layer needs source normals (opts.normals)");
        if (!(eps > 0.0 && eps < 1.0)) fail(FFM_EINVAL, "eps must lie in (0, 1)");
        if (kernel == FFM_HELMHOLTZ && !(k >= 0.0 && std::isfinite(k))) fail(FFM_EINVAL, "k must be finite and >= 0");
        const void *w = nullptr;
        ffm_dtype wdt = FFM_F64;
        p = new ffm_plan_s();
        p->nx = nx;
        p->ny = ny;
        p->kind = kernel;
        p->k = kernel == FFM_HELMHOLTZ ? k : 0.0;
        p->eps = eps;
        if (opts) {
            if (opts->n_leaf < 0 || opts->l_cap < 0 || opts->l_cap > LMAX || opts->kappa_switch < 0 ||
                opts->r1_override < 0 || opts->r1_override > R1MAX || opts->r1_override == 1 ||
                opts->precision < FFM_PREC_AUTO || opts->precision > FFM_PREC_F32X2 ||
                opts->lagrange_transfer < 0 || opts->lagrange_transfer > 3 || opts->pw_transform < 0 ||
                opts->pw_transform > 3 || !(opts->aca_eps >= 0.0 && opts->aca_eps < 1.0) || opts->wait_tries < -1)
                fail(FFM_EINVAL, "bad option value");
            if (opts->aca_eps > 0.0 && kernel != FFM_LAPLACE)
                fail(FFM_EUNSUPPORTED, "the ACA transfer is built for the Laplace single layer");
            if (opts->n_leaf > 0) p->n_leaf = opts->n_leaf;
            if (opts->l_cap > 0) p->l_cap = opts->l_cap;
            if (opts->kappa_switch > 0) p->kappa = opts->kappa_switch;
            p->r1_override = opts->r1_override;
            p->precision = opts->precision;
            p->lag_transfer = opts->lagrange_transfer;
            p->pw_transform = opts->pw_transform;
            p->aca_eps = opts->aca_eps;
            if (opts->autotune_cache) p->tune_cache = opts->autotune_cache;
            if (opts->wait_tries != 0) p->wait_tries = opts->wait_tries < 0 ? 0 : opts->wait_tries;
            w = opts->weights;
            wdt = opts->weights_dtype;
            if (w && wdt != FFM_F32 && wdt != FFM_F64) fail(FFM_EINVAL, "weights dtype must be FFM_F32 or FFM_F64");
            if (kernel == FFM_LAPLACE_DL) {
                if (opts->normals_dtype != FFM_F32 && opts->normals_dtype != FFM_F64)
                    fail(FFM_EINVAL, "normals dtype must be FFM_F32 or FFM_F64");
                p->normals_in = opts->normals;
                p->normals_dt = opts->normals_dtype;
            }
        }
        p->stream = (cudaStream_t)stream;
        p->mem.stream = p->stream;
        keep_pool_memory();
        Alloc tmp;
        tmp.stream = p->stream;
        build_plan(p, X, xdt, Y, ydt, w, wdt, tmp);
        tmp.release();
        if (opts && opts->autotune_cache) {
            ffm::apply_cached_picks(p, opts->autotune_cache, p->stream);
            FFM_CUDA(cudaStreamSynchronize(p->stream));
        }
        p->info.nx = nx;
        p->info.ny = ny;
        *out = p;
    });
    if (st != FFM_OK && p) {
        cudaStreamSynchronize(p->stream);
        cudaGetLastError();
        delete p;
    }
    return st;
}

ffm_status ffm_apply(ffm_plan_t *plan, const void *u, ffm_dtype udt, int nrhs, void *v, void *stream) {
    return guarded([&] {
        if (!plan || !u || !v) fail(FFM_EINVAL, "NULL argument");
        if (nrhs < 1 || nrhs > 65535) fail(FFM_EINVAL, "nrhs must lie in [1, 65535]");
        apply_impl(plan, u, udt, nrhs, v, (cudaStream_t)stream);
    });
}

ffm_status ffm_autotune(ffm_plan_t *plan, int nrhs, const char *cache_path, void *stream) {
    return guarded([&] {
        if (!plan) fail(FFM_EINVAL, "NULL plan");
        if (nrhs < 1 || nrhs > 65535) fail(FFM_EINVAL, "nrhs must lie in [1, 65535]");
        ffm::autotune(plan, nrhs, cache_path, (cudaStream_t)stream);
    });
}

struct ffm_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    ~ffm_graph_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

ffm_status ffm_graph_create(ffm_plan_t *plan, const void *u, ffm_dtype udt, int nrhs, void *v, ffm_graph_t **out) {
    return guarded([&] {
        if (!out) fail(FFM_EINVAL, "NULL out");
        *out = nullptr;
        if (!plan || !u || !v) fail(FFM_EINVAL, "NULL argument");
        if (nrhs < 1 || nrhs > 65535) fail(FFM_EINVAL, "nrhs must lie in [1, 65535]");
        if (!is_device_ptr(u) || !is_device_ptr(v)) fail(FFM_EINVAL, "a captured apply needs device buffers u and v");
        std::unique_ptr<ffm_graph_s> g(new ffm_graph_s);
        cudaStream_t cs;
        FFM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        int64_t count = 0;
        g_capture_count = &count;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            g_capture_count = nullptr;
            cudaStreamDestroy(cs);
            check_cuda(e, "cudaStreamBeginCapture");
        }
        try {
            apply_impl(plan, u, udt, nrhs, v, cs);
        } catch (...) {
            cudaGraph_t partial = nullptr;
            cudaStreamEndCapture(cs, &partial);
            if (partial) cudaGraphDestroy(partial);
            cudaGetLastError();
            g_capture_count = nullptr;
            cudaStreamDestroy(cs);
            throw;
        }
        g_capture_count = nullptr;
        e = cudaStreamEndCapture(cs, &g->graph);
        cudaStreamDestroy(cs);
        check_cuda(e, "cudaStreamEndCapture");
        FFM_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
        g->kernels = count;
        *out = g.release();
    });
}

ffm_status ffm_graph_launch(ffm_graph_t *graph, void *stream) {
    return guarded([&] {
        if (!graph) fail(FFM_EINVAL, "NULL graph");
        FFM_CUDA(cudaGraphLaunch(graph->exec, (cudaStream_t)stream));
        g_launches.fetch_add((uint64_t)graph->kernels, std::memory_order_relaxed);
    });
}

int64_t ffm_graph_kernels(const ffm_graph_t *graph) { return graph ? graph->kernels : 0; }

void ffm_graph_destroy(ffm_graph_t *graph) {
    delete graph;
    cudaGetLastError();
}

void ffm_destroy(ffm_plan_t *plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->stream);
    delete plan;  // Alloc destructor frees the device memory on the plan's stream
    cudaGetLastError();
}

ffm_status ffm_plan_bytes(const ffm_plan_t *plan, size_t *bytes) {
    if (!plan || !bytes) return FFM_EINVAL;
    *bytes = plan->mem.bytes;
    return FFM_OK;
}

ffm_status ffm_plan_info(const ffm_plan_t *plan, ffm_info *info) {
    if (!plan || !info) return FFM_EINVAL;
    *info = plan->info;
    info->autotuned = plan->autotuned;
    info->p2p_tchunk = plan->p2p_tchunk;
    info->p2p_smax = (int)plan->p2p_smax;
    for (int l = 0; l <= ffm::LMAX; ++l) {
        const ffm::FarLevel &F = plan->far[l];
        bool act = l <= plan->l_stop && F.n_adm > 0;
        // the variant far_lagrange runs: ACA levels by their own choice, dense levels on tcgen05
        // (row blocks of <= 224) wherever the padded real operator exists
        bool tc = F.aca ? F.aca_tc : (F.tune_tc != 0 && F.tc_tiles > 0 && F.Tsh != nullptr);
        bool ts = F.ts_ok && F.Tsp && F.tune_tc == 2;
        info->tune_tc[l] = act && F.mode == 1 ? (ts ? 2 : tc ? 1 : 0) : 0;
        info->tune_pw[l][0] = act && F.mode == 2 ? F.pw_qpt : 0;
        info->tune_pw[l][1] = act && F.mode == 2 ? F.pw_ppt : 0;
        info->tune_pw[l][2] = act && F.mode == 2 ? (F.pw_tc == 1 ? 0 : F.pw_mc) : 0;
        info->n_src_boxes[l] = F.n_src;
        info->n_tgt_boxes[l] = F.n_tgt;
    }
    int err = 0;
    if (cudaMemcpy(&err, plan->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return FFM_ECUDA;
    }
    info->device_errors = err;
    return err ? FFM_ETIMEOUT : FFM_OK;
}

ffm_status ffm_plan_export(const ffm_plan_t *plan, int what, int level, void *host_out, int64_t *count) {
    return guarded([&] {
        if (!plan || !count) fail(FFM_EINVAL, "NULL argument");
        cudaStream_t s = plan->stream;
        if (what == FFM_EXPORT_PERM_X || what == FFM_EXPORT_PERM_Y) {
            int64_t n = what == FFM_EXPORT_PERM_X ? plan->nx : plan->ny;
            *count = n;
            if (!host_out) return;
            auto h = to_host(what == FFM_EXPORT_PERM_X ? plan->permX : plan->permY, n, s);
            FFM_CUDA(cudaStreamSynchronize(s));
            int64_t *o = (int64_t *)host_out;
            for (int64_t i = 0; i < n; ++i) o[i] = h[i];
            return;
        }
        if (what == FFM_EXPORT_ADM) {
            if (level < 0 || level > plan->l_stop) {
                *count = 0;
                return;
            }
            const FarLevel &F = plan->far[level];
            *count = F.n_adm;
            if (!host_out || F.n_adm == 0) return;
            auto tgt = to_host(F.tgt, F.n_tgt, s);
            auto off = to_host(F.adm_off, F.n_tgt + 1, s);
            auto src = to_host(F.adm_src, F.n_adm, s);
            auto gx = to_host(plan->bx[level].g, plan->bx[level].nb, s);
            auto gy = to_host(plan->by[level].g, plan->by[level].nb, s);
            FFM_CUDA(cudaStreamSynchronize(s));
            uint64_t *o = (uint64_t *)host_out;
            int64_t c = 0;
            for (int64_t x = 0; x < F.n_tgt; ++x)
                for (uint32_t e = off[x]; e < off[x + 1]; ++e) {
                    o[2 * c] = morton_host(gx[tgt[x]]);
                    o[2 * c + 1] = morton_host(gy[src[e]]);
                    ++c;
                }
            return;
        }
        if (what == FFM_EXPORT_NEAR) {
            *count = plan->n_near;
            if (!host_out || plan->n_near == 0) return;
            int ls = plan->l_stop;
            auto off = to_host(plan->near_off, plan->bx[ls].nb + 1, s);
            auto src = to_host(plan->near_src, plan->n_near, s);
            auto gx = to_host(plan->bx[ls].g, plan->bx[ls].nb, s);
            auto gy = to_host(plan->by[ls].g, plan->by[ls].nb, s);
            FFM_CUDA(cudaStreamSynchronize(s));
            uint64_t *o = (uint64_t *)host_out;
            int64_t c = 0;
            for (int64_t a = 0; a < plan->bx[ls].nb; ++a)
                for (uint32_t e = off[a]; e < off[a + 1]; ++e) {
                    o[2 * c] = morton_host(gx[a]);
                    o[2 * c + 1] = morton_host(gy[src[e]]);
                    ++c;
                }
            return;
        }
        fail(FFM_EINVAL, "unknown export");
    });
}

uint64_t ffm_launch_count(void) { return g_launches.load(); }

void ffm_profile_enable(int on) {
    if (!on) profile_flush();
    g_profile = on != 0;
}

void ffm_profile_reset(void) {
    profile_flush();
    g_prof_tot.clear();
}

int ffm_profile_read(char *names, uint64_t *launches, double *ms, int cap) {
    profile_flush();
    int n = 0;
    for (auto &t : g_prof_tot) {
        if (n >= cap) break;
        if (names) {
            std::strncpy(names + 64 * n, t.first.c_str(), 63);
            names[64 * n + 63] = 0;
        }
        if (launches) launches[n] = t.second.first;
        if (ms) ms[n] = t.second.second;
        ++n;
    }
    return n;
}

const char *ffm_status_str(ffm_status s) {
    switch (s) {
        case FFM_OK: return "FFM_OK";
        case FFM_EINVAL: return "FFM_EINVAL";
        case FFM_ENOMEM: return "FFM_ENOMEM";
        case FFM_ECUDA: return "FFM_ECUDA";
        case FFM_ETIMEOUT: return "FFM_ETIMEOUT";
        case FFM_EUNSUPPORTED: return "FFM_EUNSUPPORTED";
    }
    return "unknown status";
}

const char *ffm_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
