// Autotuner: the kernel variants of an apply are picked by timing them on the plan's own
// data.  Near field: the work-item shape (targets and source points per item), which sets
// how clustered, unevenly filled leaves spread over the SMs.  Lagrange levels: the
// transfer GEMM on tcgen05 tiles or on CUDA cores.  Plane-wave levels: work per thread of
// the transforms.  Picks can be kept in a text cache keyed by device and level sizes.
#include <cmath>
#include <cstdio>
#include <fstream>
#include <limits>
#include <map>
#include <sstream>
#include <string>

#include "ffm_internal.cuh"

namespace ffm {

namespace {

class Timer {
  public:
    explicit Timer(cudaStream_t s) : s_(s) {
        FFM_CUDA(cudaEventCreate(&a_));
        FFM_CUDA(cudaEventCreate(&b_));
    }
    ~Timer() {
        cudaEventDestroy(a_);
        cudaEventDestroy(b_);
    }
    // mean device time of one call of f over `reps` calls
    template <class F>
    float time(F &&f, int reps) {
        FFM_CUDA(cudaEventRecord(a_, s_));
        for (int i = 0; i < reps; ++i) f();
        FFM_CUDA(cudaEventRecord(b_, s_));
        FFM_CUDA(cudaEventSynchronize(b_));
        float ms = 0.f;
        FFM_CUDA(cudaEventElapsedTime(&ms, a_, b_));
        return ms / reps;
    }
    // one untimed call, one timed call, and more timed calls while they are short
    template <class F>
    float measure(F &&f) {
        f();
        float ms = time(f, 1);
        if (ms < 5.f) ms = std::min(ms, time(f, ms < 0.5f ? 8 : 3));
        return ms;
    }

  private:
    cudaStream_t s_;
    cudaEvent_t a_, b_;
};

int lg2(double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); }
int rhs_bucket(int nrhs) { return nrhs == 1 ? 1 : nrhs <= 8 ? 8 : 64; }

std::string device_tag() {
    int d = 0;
    cudaGetDevice(&d);
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, d) != cudaSuccess) return "unknown";
    std::string n = pr.name;
    for (char &c : n)
        if (c == ' ') c = '_';
    return n + "_" + std::to_string(pr.multiProcessorCount) + "sm";
}

// "key value..." lines; the last line of a key wins
class Cache {
  public:
    explicit Cache(const char *path) {
        if (!path) return;
        path_ = path;
        std::ifstream f(path_);
        std::string line;
        while (std::getline(f, line)) {
            size_t sp = line.find(" = ");
            if (sp != std::string::npos) kv_[line.substr(0, sp)] = line.substr(sp + 3);
        }
    }
    bool get(const std::string &k, std::string &v) const {
        auto it = kv_.find(k);
        if (it == kv_.end()) return false;
        v = it->second;
        return true;
    }
    void put(const std::string &k, const std::string &v) {
        kv_[k] = v;
        if (path_.empty()) return;
        std::ofstream f(path_, std::ios::app);
        f << k << " = " << v << '\n';
    }

  private:
    std::string path_;
    std::map<std::string, std::string> kv_;
};

std::string near_key(const ffm_plan_s *p, const std::string &dev, int rhsb) {
    char key[320];
    snprintf(key, sizeof key, "near %s kind=%d rhs=%d near=%d pairs=%d", dev.c_str(), p->kind, rhsb,
             lg2((double)p->n_near), lg2((double)p->info.p2p_pairs));
    return key;
}

std::string lag_key(const ffm_plan_s *p, int l, const std::string &dev, int rhsb) {
    const FarLevel &F = p->far[l];
    char key[320];
    snprintf(key, sizeof key, "lag %s r1=%d rhs=%d adm=%d trans=%d", dev.c_str(), F.r1, rhsb, lg2((double)F.n_adm),
             lg2((double)F.n_trans));
    return key;
}

std::string pw_key(const ffm_plan_s *p, int l, const std::string &dev, int rhsb) {
    const FarLevel &F = p->far[l];
    char key[320];
    snprintf(key, sizeof key, "pw %s prec=%d nQ=%d rhs=%d pts=%d depth=%d", dev.c_str(), F.prec, F.nQ, rhsb,
             lg2((double)(p->info.src_points[l] + p->info.tgt_points[l])), p->l_stop - l);
    return key;
}

bool parse_near(const std::string &v, int &tch, unsigned &smax) {
    return sscanf(v.c_str(), "%d %u", &tch, &smax) == 2 && tch >= 1 && tch <= P2P_T && smax >= 1;
}
bool parse_lag(const std::string &v, int &pick) { return sscanf(v.c_str(), "%d", &pick) == 1 && pick >= 0 && pick <= 2; }
// c: right-hand sides per thread of the several-RHS kernels, or 0 for the tensor-core transforms
bool parse_pw(const std::string &v, int &a, int &b, int &c) {
    return sscanf(v.c_str(), "%d %d %d", &a, &b, &c) == 3 && (a == 2 || a == 4) && (b == 2 || b == 4) &&
           (c == 0 || c == 4 || c == 8);
}

void set_pw_multi(FarLevel &F, int c) {
    F.pw_tc = c == 0 ? 1 : 0;
    if (c != 0) F.pw_mc = c;
}

void set_items(ffm_plan_s *p, int tch, unsigned smax, Alloc &tmp, cudaStream_t s) {
    if (tch == p->p2p_tchunk && smax == p->p2p_smax) return;
    p->p2p_tchunk = tch;
    p->p2p_smax = smax;
    if (p->n_near == 0 || !p->items) return;
    int4 *old = p->items;
    p->n_items = build_p2p_items(p, tch, smax, p->mem, &p->items, tmp, s);
    p->mem.drop(old);
}

}  // namespace

int cached_lag_pick(const ffm_plan_s *p, int l) {
    if (p->tune_cache.empty()) return -1;
    Cache cache(p->tune_cache.c_str());
    std::string v;
    int a = -1;
    if (cache.get(lag_key(p, l, device_tag(), 1), v) && parse_lag(v, a)) return a;
    return -1;
}

void apply_cached_picks(ffm_plan_s *p, const char *cache_path, cudaStream_t s) {
    Cache cache(cache_path);
    const std::string dev = device_tag();
    Alloc tmp;
    tmp.stream = s;
    std::string v;
    int tch = 0;
    unsigned smax = 0;
    if (p->n_near > 0 && cache.get(near_key(p, dev, 1), v) && parse_near(v, tch, smax)) set_items(p, tch, smax, tmp, s);
    for (int l = 0; l <= p->l_stop; ++l) {
        FarLevel &F = p->far[l];
        if (F.n_adm == 0) continue;
        int a, b, c;
        if (F.mode == 1) {
            if (cache.get(lag_key(p, l, dev, 1), v) && parse_lag(v, a)) {
                if (a == 2) prepare_target_stationary(p, l, s);
                if (a != 2 || F.ts_ok) F.tune_tc = a;
            }
        } else if (F.prec != FFM_PREC_F64) {
            if (cache.get(pw_key(p, l, dev, 1), v) && parse_pw(v, a, b, c)) {
                F.pw_qpt = a;
                F.pw_ppt = b;
            }
            if ((cache.get(pw_key(p, l, dev, 64), v) || cache.get(pw_key(p, l, dev, 8), v)) && parse_pw(v, a, b, c))
                set_pw_multi(F, c);
        }
    }
    tmp.release();
}

void autotune(ffm_plan_s *p, int nrhs, const char *cache_path, cudaStream_t s) {
    Cache cache(cache_path);
    const std::string dev = device_tag();
    const bool helm = p->kind == FFM_HELMHOLTZ;
    Alloc tmp;
    tmp.stream = s;
    // densities and accumulators of the timing runs (values do not change the timing), sized as
    // in an apply: the double layer's densities are hi / lo float4 pairs, the gradient has three
    // outputs per target and density
    size_t qb = (p->kind == FFM_LAPLACE_DL ? 32 : helm ? 8 : 4) * (size_t)p->ny * nrhs;
    void *q = tmp.raw(qb);
    FFM_CUDA(cudaMemsetAsync(q, 0, qb, s));
    size_t nout = (size_t)nrhs * (p->kind == FFM_LAPLACE_GRAD ? 3 : 1);
    double2 *acc = tmp.get<double2>((size_t)p->nx * nout);
    FFM_CUDA(cudaMemsetAsync(acc, 0, sizeof(double2) * (size_t)p->nx * nout, s));
    float2 *accf = tmp.get<float2>((size_t)p->nx * nout);
    FFM_CUDA(cudaMemsetAsync(accf, 0, sizeof(float2) * (size_t)p->nx * nout, s));
    Timer T(s);

    // ---- near field: work-item shape
    if (p->n_near > 0 && p->n_items > 0) {
        std::string key = near_key(p, dev, rhs_bucket(nrhs)), v;
        int tch = p->p2p_tchunk;
        unsigned smax = p->p2p_smax;
        if (!cache.get(key, v) || !parse_near(v, tch, smax)) {
            static const int cand[][2] = {{128, 4096}, {64, 4096}, {128, 2048}, {128, 8192}, {64, 2048}, {64, 8192}};
            float best = std::numeric_limits<float>::infinity();
            for (const auto &c : cand) {
                Alloc im;
                im.stream = s;
                int4 *items = nullptr;
                int64_t n = build_p2p_items(p, c[0], (uint32_t)c[1], im, &items, tmp, s);
                float ms = T.measure([&] { near_field_items(p, items, n, c[0], q, nrhs, acc, s); });
                if (ms < best) {
                    best = ms;
                    tch = c[0];
                    smax = (unsigned)c[1];
                }
            }
            cache.put(key, std::to_string(tch) + " " + std::to_string(smax));
        }
        set_items(p, tch, smax, tmp, s);
    }

    // ---- far field, level by level
    for (int l = 0; l <= p->l_stop; ++l) {
        FarLevel &F = p->far[l];
        if (F.n_adm == 0) continue;
        auto run_level = [&] {
            Alloc lt;
            lt.stream = s;
            if (F.mode == 1)
                far_lagrange(p, l, q, nrhs, accf, lt, s);
            else
                far_planewave(p, l, (const float2 *)q, nrhs, acc, lt, s);
        };
        std::string v;
        if (F.mode == 1) {
            int r = F.r1 * F.r1 * F.r1;
            if (!helm && !F.aca) build_translation_groups(p, l, s);  // the per-translation candidates
            bool tc_ok = !helm && F.tc_tiles > 0 && !F.aca;
            if (!tc_ok) continue;
            std::string key = lag_key(p, l, dev, rhs_bucket(nrhs));
            int pick = -1;
            bool cached = cache.get(key, v) && parse_lag(v, pick);
            if (!cached || pick == 2) prepare_target_stationary(p, l, s);
            if (!cached || (pick == 2 && !F.ts_ok)) {
                // 0: CUDA-core GEMM per translation, 1: tcgen05 per translation,
                // 2: tcgen05 target-stationary
                float best = std::numeric_limits<float>::infinity();
                for (int c = 0; c <= (F.ts_ok ? 2 : 1); ++c) {
                    F.tune_tc = c;
                    float ms = T.measure(run_level);
                    if (ms < best) {
                        best = ms;
                        pick = c;
                    }
                }
                cache.put(key, std::to_string(pick));
            }
            F.tune_tc = pick;
        } else {
            if (F.prec == FFM_PREC_F64 || F.nufft) continue;  // FP64 and NUFFT levels keep their kernels
            std::string key = pw_key(p, l, dev, rhs_bucket(nrhs));
            int a = 0, b = 0, c = 0;
            if (!cache.get(key, v) || !parse_pw(v, a, b, c)) {
                float best = std::numeric_limits<float>::infinity();
                a = 4, b = 4, c = 8;
                if (nrhs == 1) {
                    static const int cand[][2] = {{4, 4}, {2, 4}, {4, 2}, {2, 2}};
                    for (const auto &cd : cand) {
                        F.pw_qpt = cd[0];
                        F.pw_ppt = cd[1];
                        float ms = T.measure(run_level);
                        if (ms < best) {
                            best = ms;
                            a = cd[0];
                            b = cd[1];
                        }
                    }
                } else {
                    // CUDA-core kernels with 8 or 4 right-hand sides per thread, and the
                    // tensor-core transforms where the level has them (c = 0)
                    const bool tc = F.pw_chunks != nullptr && p->pw_transform == 0;
                    for (int mc : {8, 4, 0}) {
                        if (mc == 0 && !tc) continue;
                        set_pw_multi(F, mc);
                        float ms = T.measure(run_level);
                        if (ms < best) {
                            best = ms;
                            c = mc;
                        }
                    }
                }
                cache.put(key, std::to_string(a) + " " + std::to_string(b) + " " + std::to_string(c));
            }
            F.pw_qpt = a;
            F.pw_ppt = b;
            if (nrhs == 1)
                F.pw_mc = c;
            else
                set_pw_multi(F, c);
        }
    }
    p->autotuned = 1;
    tmp.release();
    FFM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace ffm
