// ffm_morton_order_noalloc: the Morton ordering of one point set (bounding cube, Morton
// keys, stable radix sort) computed without allocating any device memory.
//
// Some callers cannot allocate device memory while they run: code that executes while
// another framework owns the whole device heap, allocation-free real-time loops, or
// hosts whose allocator policy forbids cudaMalloc on their worker threads.  For them the
// scratch this computation needs (key and index ping-pong buffers, per-block digit
// histograms, the cube extent) lives in one file-scope device array of fixed size,
// reserved when the library is loaded and kept by every GPU that loads it until exit.
//
// The ordering is the same as the one ffm_plan gives X when it is called with Y = X:
// same cube arithmetic, same FP64 quantisation and interleave, same stable order of
// equal keys (original index).
#include <cstddef>
#include <mutex>

#include "ffm_internal.cuh"

namespace ffm {
namespace noalloc {

constexpr int64_t MAX_POINTS = 262144;  // 2^18
constexpr int T = 256;                  // threads per block
constexpr int ITEMS = 16;
constexpr int TILE = T * ITEMS;
constexpr int MAX_BLOCKS = (int)((MAX_POINTS + TILE - 1) / TILE);

// Scratch layout (bytes): two key buffers, two index buffers, digit histograms,
// the cube extent (min/max as ordered integers), the cube (origin, edge), and a flag
// raised when a coordinate is not finite.
struct Scratch {
    unsigned long long keys[2][MAX_POINTS];
    uint32_t vals[2][MAX_POINTS];
    uint32_t hist[256 * MAX_BLOCKS];
    unsigned long long ext[6];
    double cube[4];
    unsigned int nonfinite;
};

static __device__ __align__(256) unsigned char g_scratch[sizeof(Scratch)];

__device__ __forceinline__ unsigned long long ord_enc(double d) {
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double ord_dec(unsigned long long k) {
    unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)u);
}

__global__ void k_ext_init(Scratch *S) {
    if (threadIdx.x < 3) {
        S->ext[threadIdx.x] = ~0ull;
        S->ext[3 + threadIdx.x] = 0ull;
    }
    if (threadIdx.x == 0) S->nonfinite = 0u;
}

template <class P>
__global__ void k_ext(const P *__restrict__ X, int64_t n, Scratch *S) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            double x = (double)X[3 * i + d];
            bad |= !isfinite(x);
            lo[d] = fmin(lo[d], x);
            hi[d] = fmax(hi[d], x);
        }
    // a NaN or an infinity has no place in the cube: the call's output is poisoned instead
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&S->nonfinite, 1u);
    for (int d = 0; d < 3; ++d)
        for (int off = 16; off; off >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
        }
    if ((threadIdx.x & 31) == 0)
        for (int d = 0; d < 3; ++d) {
            atomicMin(&S->ext[d], ord_enc(lo[d]));
            atomicMax(&S->ext[3 + d], ord_enc(hi[d]));
        }
}

// Cube of the set (Sec. 2.2.1): edge = largest extent times (1 + 2^-20) (1 if all points
// coincide), centred on the tight box.  Rounded operation by operation, as ffm_plan's
// host code does.
__global__ void k_cube(Scratch *S) {
    double lo[3], hi[3], e = 0.0;
    for (int d = 0; d < 3; ++d) {
        lo[d] = ord_dec(S->ext[d]);
        hi[d] = ord_dec(S->ext[3 + d]);
        e = fmax(e, __dsub_rn(hi[d], lo[d]));
    }
    double d0 = e > 0.0 ? __dmul_rn(e, 1.0 + 9.5367431640625e-07) : 1.0;
    for (int d = 0; d < 3; ++d) S->cube[d] = __dsub_rn(__dmul_rn(0.5, __dadd_rn(lo[d], hi[d])), __dmul_rn(0.5, d0));
    S->cube[3] = d0;
}

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

template <class P>
__global__ void k_morton(const P *__restrict__ X, int64_t n, Scratch *S) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t g[3];
    for (int d = 0; d < 3; ++d) {
        double t = __ddiv_rn(__dsub_rn((double)X[3 * i + d], S->cube[d]), S->cube[3]);
        double f = fmin(fmax(floor(t * 2097152.0), 0.0), 2097151.0);
        g[d] = (uint64_t)f;
    }
    S->keys[0][i] = (spread3(g[0]) << 2) | (spread3(g[1]) << 1) | spread3(g[2]);
    S->vals[0][i] = (uint32_t)i;
}

__global__ void k_hist(const unsigned long long *__restrict__ k, int64_t n, int shift, uint32_t *__restrict__ hist,
                       int nblk) {
    __shared__ uint32_t c[256];
    c[threadIdx.x] = 0;
    __syncthreads();
    int64_t t0 = (int64_t)blockIdx.x * TILE;
    for (int r = 0; r < ITEMS; ++r) {
        int64_t i = t0 + r * T + threadIdx.x;
        if (i < n) atomicAdd(&c[(uint32_t)(k[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nblk + blockIdx.x] = c[threadIdx.x];
}

// Exclusive scan of the 256 * nblk histogram entries in one block (at most 16384).
__global__ void k_hist_scan(uint32_t *hist, int count) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < count; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint32_t v = i < count ? hist[i] : 0u, inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = warp_tot[lane], wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            warp_tot[lane] = wi - w;
        }
        __syncthreads();
        uint32_t excl = carry + warp_tot[warp] + inc - v;
        if (i < count) hist[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(T) k_scatter(const unsigned long long *__restrict__ kin,
                                               const uint32_t *__restrict__ vin, int64_t n, int shift,
                                               const uint32_t *__restrict__ off, int nblk,
                                               unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout) {
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[T / 32][257];
    __shared__ uint32_t tot[256];
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = off[tid * nblk + blockIdx.x];
    for (int w = 0; w < T / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    int64_t t0 = (int64_t)blockIdx.x * TILE;
    for (int r = 0; r < ITEMS; ++r) {
        int64_t i = t0 + r * T + tid;
        bool valid = i < n;
        unsigned long long key = valid ? kin[i] : 0ull;
        uint32_t val = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t lt = peers & ((1u << lane) - 1u);
        if (valid && lt == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
        for (int w = 0; w < T / 32; ++w) {
            uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
        }
        tot[tid] = run;
        __syncthreads();
        if (valid) {
            uint32_t pos = base[d] + wcnt[warp][d] + __popc(lt);
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        base[tid] += tot[tid];
        for (int w = 0; w < T / 32; ++w) wcnt[w][tid] = 0;
        __syncthreads();
    }
}

// The sorted indices to the caller's array; every entry 0xFFFFFFFF when a coordinate was
// not finite (the call only enqueues work, so the error travels with the output).
__global__ void k_copy_perm(const uint32_t *__restrict__ v, int64_t n, const Scratch *S,
                            uint32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = S->nonfinite ? 0xFFFFFFFFu : v[i];
}

// Device address of the scratch array, resolved once per device.
static std::mutex g_mu;
static void *g_addr[64];

static Scratch *scratch_for_current_device() {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) fail(FFM_EUNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        check_cuda(cudaGetSymbolAddress(&p, g_scratch), "cudaGetSymbolAddress(scratch)");
        g_addr[dev] = p;
    }
    return static_cast<Scratch *>(g_addr[dev]);
}

template <class P>
static void run(const void *X, int64_t n, uint32_t *perm, cudaStream_t s) {
    Scratch *S = scratch_for_current_device();
    const P *x = static_cast<const P *>(X);
    FFM_LAUNCH(k_ext_init, 1, 32, 0, s, S);
    FFM_LAUNCH(k_ext<P>, std::min<unsigned>(cdiv(n, 256), 256u), 256, 0, s, x, n, S);
    FFM_LAUNCH(k_cube, 1, 1, 0, s, S);
    FFM_LAUNCH(k_morton<P>, cdiv(n, 256), 256, 0, s, x, n, S);
    int nblk = (int)cdiv(n, TILE);
    // Scratch members as device addresses: the resolved base plus each member's offset.
    char *base = reinterpret_cast<char *>(S);
    unsigned long long *k0 = reinterpret_cast<unsigned long long *>(base + offsetof(Scratch, keys));
    uint32_t *v0 = reinterpret_cast<uint32_t *>(base + offsetof(Scratch, vals));
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + offsetof(Scratch, hist));
    unsigned long long *kb[2] = {k0, k0 + MAX_POINTS};
    uint32_t *vb[2] = {v0, v0 + MAX_POINTS};
    int cur = 0;
    for (int shift = 0; shift < 64; shift += 8) {
        FFM_LAUNCH(k_hist, nblk, T, 0, s, kb[cur], n, shift, hist, nblk);
        FFM_LAUNCH(k_hist_scan, 1, 1024, 0, s, hist, 256 * nblk);
        FFM_LAUNCH(k_scatter, nblk, T, 0, s, kb[cur], vb[cur], n, shift, hist, nblk, kb[1 - cur], vb[1 - cur]);
        cur = 1 - cur;
    }
    FFM_LAUNCH(k_copy_perm, cdiv(n, 256), 256, 0, s, vb[cur], n, S, perm);
}

}  // namespace noalloc
}  // namespace ffm

extern "C" ffm_status ffm_morton_order_noalloc(const void *X, ffm_dtype xdt, int64_t n, uint32_t *perm_out,
                                               void *stream) {
    using namespace ffm;
    try {
        if (!X || !perm_out) fail(FFM_EINVAL, "NULL argument");
        if (n < 1 || n > noalloc::MAX_POINTS)
            fail(FFM_EINVAL, "n must lie in [1, 262144] (size of the static scratch array)");
        if (xdt != FFM_F32 && xdt != FFM_F64) fail(FFM_EINVAL, "X dtype must be FFM_F32 or FFM_F64");
        int dev = 0;
        check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        for (const void *p : {X, (const void *)perm_out}) {
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
                (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
                cudaGetLastError();
                fail(FFM_EINVAL, "X and perm_out must be device memory");
            }
            if (a.type == cudaMemoryTypeDevice && a.device != dev)
                fail(FFM_EINVAL, "X and perm_out must be memory of the current device");
        }
        cudaStream_t s = (cudaStream_t)stream;
        if (xdt == FFM_F64)
            noalloc::run<double>(X, n, perm_out, s);
        else
            noalloc::run<float>(X, n, perm_out, s);
        return FFM_OK;
    } catch (const Error &e) {
        ffm::set_last_error(e.msg);
        return e.status;
    }
}
