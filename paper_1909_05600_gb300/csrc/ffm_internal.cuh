// Internal declarations shared by the CUDA translation units of libffm_gb300.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ffm.h"
#include "dfloat.cuh"

namespace ffm {

constexpr int LMAX = 21;         // finest level of the Morton keys (3 x 21 bits)
constexpr int R1MAX = 8;         // largest Chebyshev node count per axis
constexpr int LAG_GEMM_BN = 32;  // pairs (GEMM columns) per tile of the Lagrange transfer
constexpr int P2P_T = 128;        // threads per near-field block (the largest target chunk)
constexpr int LAG_CHUNK = 512;    // points per block of the Lagrange point-wise kernels
constexpr int PW_TC_FCH = 256;    // points per block of the tensor-core plane-wave forward transform
constexpr int PW_TC_BCH = 128;    // points per block of the tensor-core plane-wave backward transform
constexpr int PW_TC_MIN_RHS = 16; // right-hand sides from which the plane-wave transforms run on
                                  // the tensor cores by default
constexpr int NUFFT_MIN_NQ = 8000; // plane-wave levels with at least this many directions run
                                   // their F steps as NUFFTs (unless forced either way)
constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- errors

struct Error {
    ffm_status status;
    std::string msg;
};

[[noreturn]] void fail(ffm_status s, const std::string &msg);
void set_last_error(const std::string &msg);
void check_cuda(cudaError_t e, const char *what);

#define FFM_CUDA(call) ::ffm::check_cuda((call), #call)

extern std::atomic<uint64_t> g_launches;
extern bool g_profile;
// Non-null while this thread records an apply into a CUDA graph: launches are counted
// there (they run later, once per graph launch) and not profiled.
extern thread_local int64_t *g_capture_count;
void profile_begin(const char *name, cudaStream_t s);
void profile_end(cudaStream_t s);

// Every kernel launch goes through this: counts it and checks the launch status.
template <class... KArgs, class... Args>
inline void launch_kernel(const char *name, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s, Args &&...args) {
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
    bool prof = g_profile && !g_capture_count;
    if (prof) profile_begin(name, s);
    k<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
    if (prof) profile_end(s);
    if (g_capture_count)
        ++*g_capture_count;
    else
        g_launches.fetch_add(1, std::memory_order_relaxed);
    check_cuda(cudaGetLastError(), name);
}

#define FFM_LAUNCH(kernel, grid, block, smem, stream, ...) \
    ::ffm::launch_kernel(#kernel, kernel, dim3(grid), dim3(block), (size_t)(smem), (stream), __VA_ARGS__)
// Same, with an explicit name for per-kernel timing (e.g. to tell FP32 and FP64 variants apart).
#define FFM_LAUNCH_NAMED(name, kernel, grid, block, smem, stream, ...) \
    ::ffm::launch_kernel(name, kernel, dim3(grid), dim3(block), (size_t)(smem), (stream), __VA_ARGS__)

// ------------------------------------------------------- device memory

// Stream-ordered device allocation owned by a scope or a plan.
struct Alloc {
    std::vector<void *> ptrs;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;
    void *raw(size_t n);
    template <class T>
    T *get(size_t count) {
        return static_cast<T *>(raw(sizeof(T) * (count > 0 ? count : 1)));
    }
    void release();
    void drop(void *p);  // free one allocation of this scope now (stream-ordered)
    ~Alloc() { release(); }
};

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// K-major, no-swizzle operand layout of the tcgen05 kernels: 8-row x 16-byte core
// matrices, core matrix (row / 8, k / 4) at byte ((row / 8) * KT / 4 + k / 4) * 128, row
// within it at 16 * (row % 8), element k % 4 at 4 * (k % 4).  Returns a float index.
__host__ __device__ inline uint32_t kmajor_index(int row, int k, int KT) {
    return (uint32_t)((((row >> 3) * (KT >> 2) + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3));
}

struct alignas(32) D4 {
    double x, y, z, w;
};

// --------------------------------------------------- primitives (tree.cu)

// Exclusive scan of n uint32 values (in may alias out); total written to *d_total if
// non-null.  Temporaries from `al`.
void scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total, Alloc &al, cudaStream_t s);

// Stable LSD radix sort of (key, val) by the key bits [0, nbits).  Buffers are
// ping-ponged; the sorted data ends in (keys, vals) on return.
void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int nbits, Alloc &al, cudaStream_t s);
void radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int nbits, Alloc &al, cudaStream_t s);

// ----------------------------------------------------------- the plan

struct BoxLevel {
    int64_t nb = 0;             // number of non-empty boxes
    uint32_t *start = nullptr;  // nb+1 sorted-position offsets (within the set)
    int4 *g = nullptr;          // integer box coordinates at this level
    uint32_t *first_leaf = nullptr;  // nb+1: first leaf (stop-level box) of each box
    uint32_t *first_child = nullptr; // nb+1: first child in the next level (descent only)
    uint32_t *fine = nullptr;   // nb: index of the first box of the deepest table
};

// Type-3 NUFFT of a plane-wave level (nufft.cu): grids, direction windows, point blocks
struct NuLevel {
    int w = 0, M = 0, n1 = 0, n2 = 0;  // kernel width, cells per box edge, spreading / FFT grid edges
    double beta = 0, h = 0;             // kernel shape, spreading-grid spacing
    int dlt = 0, E = 0;                 // bin level below the level, bin subgrid edge
    float *cinv = nullptr;              // n1: FFT-grid kernel deconvolution
    int4 *dirU = nullptr;               // nQ: first window node per axis (centred FFT-grid index)
    float *dirW = nullptr;              // nQ x 3 x w: window kernel values, correction on axis 0
    int64_t n_tiles = 0;                // FFT-grid tiles met by some direction's window: ids,
    uint32_t *tile_id = nullptr, *tile_off = nullptr, *tile_q = nullptr;  // CSR of directions
    uint32_t own_max = 0;               // longest of the lists below
    int64_t n_own = 0;                  // tiles holding some window's first node (each direction
    uint32_t *own_id = nullptr, *own_off = nullptr, *own_q = nullptr;     // in exactly one)
    int64_t n_ych = 0, n_xch = 0;       // point blocks (bin, first, end, slot) of sources / targets
    int4 *ych = nullptr, *xch = nullptr;
    int fft_src = 0, fft_tgt = 0;       // cuFFT handles (batched over the level's source / target boxes)
    size_t work_src = 0, work_tgt = 0;
    bool has_fft = false;
};

struct FarLevel {
    int mode = 0;        // 0 none, 1 Lagrange, 2 plane waves
    int r1 = 0, L = 0, nQ = 0;
    int64_t n_adm = 0;
    int n_trans = 0;
    int64_t n_tgt = 0, n_src = 0;   // boxes with at least one admissible pair
    uint32_t *tgt = nullptr;        // n_tgt target box indices
    uint32_t *src = nullptr;        // n_src source box indices
    uint32_t *adm_off = nullptr;    // n_tgt+1 CSR offsets (per listed target)
    uint32_t *adm_src = nullptr;    // n_adm source box per pair
    uint32_t *adm_t = nullptr;      // n_adm translation index per pair
    int4 *trans_m = nullptr;        // n_trans integer offsets gX - gY
    std::vector<int4> h_trans_m;
    // Lagrange
    float *T = nullptr;             // n_trans * r * r (real) or float2 (complex), [t][i][j]
    uint32_t *bt_off = nullptr;     // n_trans+1: pairs grouped by translation (CSR)
    uint32_t *bt_src = nullptr;     // n_adm source box per pair, grouped by translation
    uint32_t *bt_tgt = nullptr;     // n_adm target box per pair, grouped by translation
    int64_t n_tiles = 0;            // GEMM column tiles over all translations
    uint32_t *tile_t = nullptr;     // per tile: translation
    uint32_t *tile_p0 = nullptr;    // per tile: first pair (index into bt_*)
    int64_t n_src_chunks = 0, n_tgt_chunks = 0;
    uint2 *src_chunks = nullptr;    // (source box, first point): LAG_CHUNK-point pieces of the boxes
    uint2 *tgt_chunks = nullptr;    // likewise for the target boxes
    bool ts_ok = false;             // target-stationary transfer possible (Laplace, r <= 64,
                                    // partners sorted by translation within each target)
    float *Tsp = nullptr;           // target-stationary transfer (r <= 64): T_t split into TF32
                                    // hi and lo, 64 x 64 each, in the K-major core-matrix layout
    float *Tsh = nullptr;           // tensor-core transfer: T_t padded to npad rows of rkp floats
    int rkp = 0;                    // (per component block for the gradient)
    // ACA of T (eq. 11, Laplace single layer with ffm_opts.aca_eps): T_t ~ A_t B_t^T with
    // rank_t <= aca_rank (the level's largest); the transfer runs as w_p = B_t^T u~_src(p)
    // per pair, then v~_tgt(p) += A_t w_p.  B^T as [t][aca_rp][K] and A as [t][rows][aca_rp]
    // (tensor cores: K = rkp, rows = npad, aca_rp = aca_rank rounded up to 16; CUDA cores:
    // K = rows = r, aca_rp = aca_rank), zero past each rank.
    bool aca = false, aca_tc = false;
    int aca_rank = 0, aca_rp = 0;
    float *Aca = nullptr, *Bca = nullptr;
    uint32_t *pair_id = nullptr;    // n_adm: p -> p (pair-indexed rows of w)
    int64_t tc_tiles = 0;           // 256-pair tiles for the tensor-core transfer
    uint32_t *tc_tile_t = nullptr;
    uint32_t *tc_tile_p0 = nullptr;
    // plane waves: arithmetic (FFM_PREC_F32 / _F32C with FP32 tables, FFM_PREC_F64 with
    // FP64 tables), chosen from the cancellation of the quadrature sum (tables.cu)
    int prec = 0;
    // kernel variants picked by ffm_autotune (defaults otherwise): Lagrange transfer on
    // tensor cores (-1: when the shape allows, 0: CUDA cores, 1: tensor cores); plane-wave
    // direction pairs per thread (forward), points per thread (backward), right-hand sides
    // per thread (several-RHS kernels)
    int tune_tc = -1;
    int pw_qpt = 4, pw_ppt = 4, pw_mc = 8;
    double cancel = 0;              // sum_q |D(q)| / |sum_q D(q)| for the closest translation
    float4 *ks = nullptr;           // nQ: k * s_q (x, y, z, 0)
    float2 *D = nullptr;            // n_trans * nQ
    float2 *E = nullptr;            // (l_stop - l) * 8 * nQ: octant phase factors
    D4 *ksd = nullptr;
    double2 *Dd = nullptr;
    double2 *Ed = nullptr;
    dd4 *ksx = nullptr;             // double-float levels
    dd2 *Dx = nullptr;
    dd2 *Ex = nullptr;
    int nufft = 0;                  // F steps as type-3 NUFFTs (FP32 plane-wave levels)
    NuLevel nu;
    // tensor-core F steps for several right-hand sides (FP32 and compensated-FP32 direct
    // levels): (box, first point) pieces of PW_TC_FCH points of the source boxes and of
    // PW_TC_BCH points of the target boxes
    int64_t n_pw_chunks = 0, n_pw_tchunks = 0;
    int pw_tc = -1;                 // those transforms: -1 from PW_TC_MIN_RHS right-hand sides on,
                                    // 0 never, 1 always (ffm_autotune's pick)
    uint2 *pw_chunks = nullptr;
    uint2 *pw_tchunks = nullptr;
};

}  // namespace ffm

struct ffm_plan_s;
namespace ffm {
void nufft_release(ffm_plan_s *p);  // nufft.cu: cuFFT handles
}

struct ffm_plan_s {
    ~ffm_plan_s() { ffm::nufft_release(this); }
    int64_t nx = 0, ny = 0;
    int kind = 0;
    double k = 0, eps = 0;
    int n_leaf = 64, l_cap = ffm::LMAX;
    double kappa = 2.0;
    int r1_override = 0;
    int precision = 0;  // ffm_precision for the plane-wave levels, 0 = by cancellation
    float4 *sctab = nullptr;  // sin/cos(j/64) in double-float for the double-float levels
    int lag_transfer = 0;     // ffm_opts.lagrange_transfer
    int pw_transform = 0;     // ffm_opts.pw_transform
    double aca_eps = 0;       // ffm_opts.aca_eps
    const void *normals_in = nullptr;  // double layer: caller's normals (during ffm_plan only)
    ffm_dtype normals_dt = FFM_F64;
    float4 *nY = nullptr;     // double layer: source normals in Morton order, hi and lo parts
    float4 *nYlo = nullptr;
    double d0 = 1, oX[3] = {0, 0, 0}, oY[3] = {0, 0, 0}, sigma[3] = {0, 0, 0};
    int l_stop = 0, root_adm = 0;
    cudaStream_t stream = nullptr;
    ffm::Alloc mem;                     // everything the plan owns
    uint32_t *permX = nullptr, *permY = nullptr;  // sorted position -> original index
    float4 *epsX = nullptr, *epsY = nullptr;      // leaf-relative coords (hi part); .w = leaf index bits
    float4 *epsXlo = nullptr, *epsYlo = nullptr;  // FP32 residual of the leaf-relative coords (lo part)
    double *wY = nullptr;                          // sorted weights (or null)
    uint64_t *keyX = nullptr, *keyY = nullptr;     // sorted Morton keys (exports)
    ffm::BoxLevel bx[ffm::LMAX + 1], by[ffm::LMAX + 1];
    ffm::FarLevel far[ffm::LMAX + 1];
    int64_t n_near = 0;
    uint32_t *near_off = nullptr;   // nbx(l_stop)+1 CSR over all target leaves
    uint32_t *near_src = nullptr;   // n_near source leaf per pair
    int autotuned = 0;
    int p2p_tchunk = 128;           // work-item shape (autotuned): targets per item
    uint32_t p2p_smax = 4096;       //   and source points per item (a larger single leaf stays whole)
    int64_t n_items = 0;            // near-field work items (target chunk x bounded source range)
    int4 *items = nullptr;          // (target leaf, first target in the leaf, first pair, end pair)
    int *dev_err = nullptr;         // device-side error flags (bounded waits that gave up)
    int wait_tries = 1 << 24;       // try_wait attempts per bounded device-side wait (ffm_opts.wait_tries)
    std::string tune_cache;         // ffm_opts.autotune_cache (empty: none)
    ffm_info info{};
};

namespace ffm {
// tree.cu
void build_plan(ffm_plan_s *p, const void *X, ffm_dtype xdt, const void *Y, ffm_dtype ydt, const void *w,
                ffm_dtype wdt, Alloc &tmp);
// tree.cu: partners sorted by translation and T pre-split for the target-stationary
// transfer of Lagrange level l (on demand); tables.cu: the T split
void prepare_target_stationary(ffm_plan_s *p, int l, cudaStream_t s);
// tree.cu: pairs of Lagrange level l grouped by translation and the per-translation tiles
// (on demand; no-op if present)
void build_translation_groups(ffm_plan_s *p, int l, cudaStream_t s);
// autotune.cu: the transfer variant stored for Lagrange level l in the plan's autotune
// cache (0 CUDA cores, 1 tcgen05 per translation, 2 target-stationary), or -1
int cached_lag_pick(const ffm_plan_s *p, int l);
void launch_table_split(ffm_plan_s *p, int l, cudaStream_t s);

// tree.cu: near-field work items with targets in chunks of tchunk and at most smax source
// points per item, allocated from out_mem; returns their number.
int64_t build_p2p_items(ffm_plan_s *p, int tchunk, uint32_t smax, Alloc &out_mem, int4 **items, Alloc &tmp,
                        cudaStream_t s);

// tables.cu
// Host staging buffers that must outlive the asynchronous copies reading them.
struct HostKeep {
    std::vector<std::vector<char>> bufs;
    template <class T>
    const T *hold(std::vector<T> &&v) {
        std::vector<char> b(sizeof(T) * v.size());
        if (!v.empty()) memcpy(b.data(), v.data(), b.size());
        bufs.push_back(std::move(b));
        return reinterpret_cast<const T *>(bufs.back().data());
    }
};
// Operator tables of each level are enqueued as soon as the level's translations are known.
// They run in order on the plan's stream: a concurrent side stream was measured slower,
// since the table kernels fill every SM and the descent's small kernels queue behind them.
struct TableJob {
    cudaStream_t side;
    Alloc tmp;
    HostKeep keep;
    D4 *d_sw[LMAX + 1] = {};
    explicit TableJob(cudaStream_t main);
    ~TableJob();
};
void build_tables(ffm_plan_s *p, int l, TableJob &tj);   // once level l's translations are known
void build_octants(ffm_plan_s *p, int l, TableJob &tj);  // once the stop level is known
int r1_rule(int kind, double eps);
// farfield.cu / nearfield.cu
// Lagrange levels add their contributions in FP32 into accf (float2 per target and RHS);
// the apply adds accf into the FP64 accumulators once, at the end.
void far_lagrange(const ffm_plan_s *p, int l, const void *q, int nrhs, float2 *accf, Alloc &tmp, cudaStream_t s);
// nmat row-major matrices written with padded rows and columns (zeros): as TF32 hi / lo parts,
// or (lo == nullptr) as a plain copy into hi
void split_pad(const float *src, int64_t nmat, int rows, int cols, int rows_pad, int cols_pad, float *hi, float *lo,
               cudaStream_t s);
// true for the kinds whose transfer operators are the real Laplace G (Laplace, double layer)
inline bool real_kernel(int kind) { return kind != FFM_HELMHOLTZ; }
void far_planewave(const ffm_plan_s *p, int l, const float2 *q, int nrhs, double2 *acc, Alloc &tmp,
                   cudaStream_t s);
void near_field(const ffm_plan_s *p, const void *q, int nrhs, double2 *acc, cudaStream_t s);
// nufft.cu: the plane-wave F steps of level l as type-3 NUFFTs (FP32 levels)
bool nufft_possible(const ffm_plan_s *p, int l);
void build_nufft(ffm_plan_s *p, int l, Alloc &tmp, cudaStream_t s);
void nufft_forward(const ffm_plan_s *p, int l, const float2 *q, int nrhs, float2 *ut, Alloc &tmp, cudaStream_t s);
void nufft_backward(const ffm_plan_s *p, int l, const float2 *vt, int nrhs, double2 *acc, Alloc &tmp,
                    cudaStream_t s);
void gauss_legendre_nodes(int n, std::vector<double> &x, std::vector<double> &w);  // tables.cu
// autotune.cu: pick kernel variants by timing them on the plan (ffm_autotune)
void autotune(ffm_plan_s *p, int nrhs, const char *cache_path, cudaStream_t s);
// take the picks a cache file holds for this plan's sizes (no timing); at plan creation
void apply_cached_picks(ffm_plan_s *p, const char *cache_path, cudaStream_t s);
// The same with explicit work items (the autotuner times candidate item shapes).
void near_field_items(const ffm_plan_s *p, const int4 *items, int64_t n_items, int tchunk, const void *q, int nrhs,
                      double2 *acc, cudaStream_t s);
}  // namespace ffm
