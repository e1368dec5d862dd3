// Plan construction on the device (Sec. 2.2.1, 2.2.2, 2.2.4 and Sec. 3.1):
//   bounding cubes of equal edge, Morton keys, stable radix sort, per-level box tables,
//   and the descent-only pair lists (children of near pairs split into admissible and
//   near pairs), grouped by target box and keyed by integer box translation.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ffm_internal.cuh"

namespace ffm {

// ==================================================================== scan

constexpr int SCAN_T = 512;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_T * SCAN_IPT;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total in *tot.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sm_warp, uint32_t *tot) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) sm_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? sm_warp[lane] : 0;
        uint32_t wi = warp_incl_scan(w);
        if (lane < nw) sm_warp[lane] = wi - w;
        if (lane == nw - 1) *tot = wi;
    }
    __syncthreads();
    return inc - v + sm_warp[warp];
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, int64_t n, uint32_t *__restrict__ bsum) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
        int64_t g = base + i;
        if (g < n) s += in[g];
    }
    __shared__ uint32_t sw[32];
    __shared__ uint32_t tot;
    block_excl_scan(s, sw, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_bsums(uint32_t *bsum, int64_t nb, uint32_t *d_total) {
    __shared__ uint32_t sw[32];
    __shared__ uint32_t tot;
    uint32_t carry = 0;
    for (int64_t c = 0; c < nb; c += blockDim.x) {
        int64_t i = c + threadIdx.x;
        uint32_t v = i < nb ? bsum[i] : 0;
        uint32_t e = block_excl_scan(v, sw, &tot);
        if (i < nb) bsum[i] = e + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void k_scan_down(const uint32_t *in, uint32_t *out, int64_t n, const uint32_t *__restrict__ bsum) {
    __shared__ uint32_t tile[SCAN_TILE];
    __shared__ uint32_t sw[32];
    __shared__ uint32_t tot;
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
        int64_t g = base + i;
        tile[i] = g < n ? in[g] : 0;
    }
    __syncthreads();
    uint32_t loc[SCAN_IPT];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_IPT; ++j) {
        loc[j] = s;
        s += tile[threadIdx.x * SCAN_IPT + j];
    }
    uint32_t e = block_excl_scan(s, sw, &tot) + bsum[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_IPT; ++j) tile[threadIdx.x * SCAN_IPT + j] = loc[j] + e;
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
        int64_t g = base + i;
        if (g < n) out[g] = tile[i];
    }
}

// The whole scan in one block, tile after tile with a running carry: one launch instead
// of three for the many small scans of a plan.
constexpr int64_t SCAN_SMALL = 16 * SCAN_TILE;
__global__ void __launch_bounds__(SCAN_T) k_scan_small(const uint32_t *in, uint32_t *out, int64_t n,
                                                       uint32_t *d_total) {
    __shared__ uint32_t tile[SCAN_TILE];
    __shared__ uint32_t sw[32];
    __shared__ uint32_t tot;
    uint32_t carry = 0;
    for (int64_t base = 0; base < n; base += SCAN_TILE) {
        for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
            int64_t g = base + i;
            tile[i] = g < n ? in[g] : 0;
        }
        __syncthreads();
        uint32_t loc[SCAN_IPT];
        uint32_t sum = 0;
#pragma unroll
        for (int j = 0; j < SCAN_IPT; ++j) {
            loc[j] = sum;
            sum += tile[threadIdx.x * SCAN_IPT + j];
        }
        uint32_t e = block_excl_scan(sum, sw, &tot) + carry;
#pragma unroll
        for (int j = 0; j < SCAN_IPT; ++j) tile[threadIdx.x * SCAN_IPT + j] = loc[j] + e;
        __syncthreads();
        for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
            int64_t g = base + i;
            if (g < n) out[g] = tile[i];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && d_total) *d_total = carry;
}

void scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total, Alloc &al, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) FFM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
        return;
    }
    if (n <= SCAN_SMALL) {
        FFM_LAUNCH(k_scan_small, 1, SCAN_T, 0, s, in, out, n, d_total);
        return;
    }
    int64_t nb = cdiv(n, SCAN_TILE);
    uint32_t *bsum = al.get<uint32_t>(nb);
    FFM_LAUNCH(k_scan_reduce, (unsigned)nb, SCAN_T, 0, s, in, n, bsum);
    FFM_LAUNCH(k_scan_bsums, 1, 1024, 0, s, bsum, nb, d_total);
    FFM_LAUNCH(k_scan_down, (unsigned)nb, SCAN_T, 0, s, in, out, n, bsum);
}

// ============================================================== radix sort

constexpr int RS_T = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_T * RS_ITEMS;

template <class K>
__global__ void k_rs_bits(const K *__restrict__ k, int64_t n, unsigned long long *orand) {
    unsigned long long o = 0, a = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long v = (unsigned long long)k[i];
        o |= v;
        a &= v;
    }
    for (int off = 16; off; off >>= 1) {
        o |= __shfl_xor_sync(0xffffffffu, o, off);
        a &= __shfl_xor_sync(0xffffffffu, a, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&orand[0], o);
        atomicAnd(&orand[1], a);
    }
}

template <class K>
__global__ void k_rs_hist(const K *__restrict__ kin, int64_t n, int shift, uint32_t *__restrict__ hist, int nblk) {
    __shared__ uint32_t c[256];
    c[threadIdx.x] = 0;
    __syncthreads();
    int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        int64_t i = t0 + r * RS_T + threadIdx.x;
        if (i < n) atomicAdd(&c[(uint32_t)(kin[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = c[threadIdx.x];
}

__device__ __forceinline__ unsigned long long ld_stream(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Stable scatter staged in shared memory.  A block owns a tile of RS_TILE elements; warp w
// takes the tile's elements w RS_ITEMS 32 .. in order, 32 per round.  Each element's rank
// within its warp's digit run comes from a warp match mask and a warp-private count per
// digit (no block barrier per round); the warps' counts are then turned into offsets within
// the tile's digit runs (in element order: warps in turn), and each element is placed in a
// shared-memory copy of the tile, which ends up sorted by digit.  The block then writes that
// copy in order: consecutive threads write consecutive slots of one digit's run in the
// output (its start from the scanned digit-major histogram), so the stores are coalesced.
// The tile's own digit counts are differences of consecutive entries of the scanned
// histogram.
template <class K>
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                     int64_t n, int shift, const uint32_t *__restrict__ off,
                                                     int nblk, K *__restrict__ kout, uint32_t *__restrict__ vout) {
    extern __shared__ __align__(16) unsigned char rs_smem[];
    K *skey = reinterpret_cast<K *>(rs_smem);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + RS_TILE);
    __shared__ uint32_t base[256], start[256];
    __shared__ uint32_t wc[RS_T / 32][256];  // per warp and digit: counts, then offsets in the tile
    __shared__ uint32_t wtot[RS_T / 32];
    int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    const int tile_n = (int)min((int64_t)RS_TILE, n - t0);
#pragma unroll
    for (int d = 0; d < 256; d += 32) wc[warp][d + lane] = 0u;
    {
        const int64_t flat = (int64_t)tid * nblk + blockIdx.x;
        const uint32_t b = off[flat];
        const uint32_t c = flat + 1 < 256LL * nblk ? off[flat + 1] - b : (uint32_t)(n - b);
        base[tid] = b;
        // exclusive prefix of the tile's digit counts (digit = thread)
        uint32_t inc = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wtot[warp] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wtot[w];
        start[tid] = before + inc - c;
    }
    // warp-local stable ranks, RS_ITEMS rounds of 32 consecutive elements; every load of the
    // warp is issued first (volatile, so the compiler keeps them here, all in flight)
    K keys[RS_ITEMS];
    uint32_t vals[RS_ITEMS], rk[RS_ITEMS], dg[RS_ITEMS];
    const int64_t w0 = t0 + (int64_t)warp * RS_ITEMS * 32;
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = w0 + r * 32 + lane;
        keys[r] = (K)0;
        vals[r] = 0u;
        if (i < n) {
            keys[r] = ld_stream(kin + i);
            vals[r] = ld_stream(vin + i);
        }
    }
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = w0 + r * 32 + lane;
        const bool valid = i < n;
        const uint32_t d = valid ? ((uint32_t)(keys[r] >> shift) & 255u) : 256u;
        dg[r] = d;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t lt = peers & ((1u << lane) - 1u);
        rk[r] = valid ? wc[warp][d] + __popc(lt) : 0u;
        __syncwarp();
        if (valid && lt == 0) wc[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        // digit tid: the warps' runs in turn, after the runs of the smaller digits
        uint32_t o = start[tid];
#pragma unroll
        for (int w = 0; w < RS_T / 32; ++w) {
            const uint32_t c = wc[w][tid];
            wc[w][tid] = o;
            o += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ITEMS; ++r)
        if (dg[r] < 256u) {
            const uint32_t pos = wc[warp][dg[r]] + rk[r];
            skey[pos] = keys[r];
            sval[pos] = vals[r];
        }
    __syncthreads();
    for (int i = tid; i < tile_n; i += RS_T) {
        K key = skey[i];
        uint32_t d = (uint32_t)(key >> shift) & 255u;
        uint32_t gp = base[d] + (uint32_t)i - start[d];
        kout[gp] = key;
        vout[gp] = sval[i];
    }
}

template <class K>
static void radix_sort(K *keys, uint32_t *vals, int64_t n, int nbits, Alloc &al, cudaStream_t s) {
    if (n <= 1) return;
    unsigned long long *orand = al.get<unsigned long long>(2);
    unsigned long long init[2] = {0ull, ~0ull};
    FFM_CUDA(cudaMemcpyAsync(orand, init, sizeof init, cudaMemcpyHostToDevice, s));
    FFM_LAUNCH(k_rs_bits<K>, std::min<unsigned>(cdiv(n, 256), 1024u), 256, 0, s, keys, n, orand);
    unsigned long long h[2];
    FFM_CUDA(cudaMemcpyAsync(h, orand, sizeof h, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    unsigned long long vary = h[0] ^ h[1];
    int nblk = (int)cdiv(n, RS_TILE);
    uint32_t *hist = al.get<uint32_t>((size_t)256 * nblk);
    K *k2 = al.get<K>(n);
    uint32_t *v2 = al.get<uint32_t>(n);
    K *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    const size_t scatter_smem = (size_t)RS_TILE * (sizeof(K) + sizeof(uint32_t));
    FFM_CUDA(cudaFuncSetAttribute(k_rs_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem));
    for (int shift = 0; shift < nbits; shift += 8) {
        if (((vary >> shift) & 255ull) == 0) continue;
        FFM_LAUNCH(k_rs_hist<K>, nblk, RS_T, 0, s, ka, n, shift, hist, nblk);
        scan_u32(hist, hist, (int64_t)256 * nblk, nullptr, al, s);
        FFM_LAUNCH(k_rs_scatter<K>, nblk, RS_T, scatter_smem, s, ka, va, n, shift, hist, nblk, kb, vb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        FFM_CUDA(cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, s));
        FFM_CUDA(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
}

void radix_sort_u64(uint64_t *keys, uint32_t *vals, int64_t n, int nbits, Alloc &al, cudaStream_t s) {
    radix_sort<unsigned long long>((unsigned long long *)keys, vals, n, nbits, al, s);
}
void radix_sort_u32(uint32_t *keys, uint32_t *vals, int64_t n, int nbits, Alloc &al, cudaStream_t s) {
    radix_sort<uint32_t>(keys, vals, n, nbits, al, s);
}

// ========================================================== bounding cubes

__device__ __forceinline__ unsigned long long ord_enc(double d) {
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
static double ord_dec(unsigned long long k) {
    unsigned long long u = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double d;
    memcpy(&d, &u, sizeof d);
    return d;
}

// out[0..2] = encoded min, out[3..5] = encoded max, out[6] = non-finite flag.
template <class T>
__global__ void k_bbox(const T *__restrict__ P, int64_t n, unsigned long long *out) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    unsigned long long bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = (double)P[3 * i + d];
            if (!isfinite(x)) bad = 1;
            lo[d] = fmin(lo[d], x);
            hi[d] = fmax(hi[d], x);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        for (int off = 16; off; off >>= 1) {
            lo[d] = fmin(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], off));
            hi[d] = fmax(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], off));
        }
    bad = __any_sync(0xffffffffu, bad != 0);
    if ((threadIdx.x & 31) == 0) {
        for (int d = 0; d < 3; ++d) {
            atomicMin(&out[d], ord_enc(lo[d]));
            atomicMax(&out[3 + d], ord_enc(hi[d]));
        }
        if (bad) atomicOr(&out[6], 1ull);
    }
}

// =================================================================== keys

__device__ __forceinline__ uint64_t spread3(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ __forceinline__ uint64_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return x;
}

// Finest-grid coordinate floor(((x - o)/d0) * 2^21), clamped to [0, 2^21 - 1]; the
// subtraction and the division are IEEE FP64 operations, the scaling is exact.
__device__ __forceinline__ uint64_t fine_coord(double x, double o, double d0) {
    double t = __ddiv_rn(__dsub_rn(x, o), d0);
    double f = floor(t * 2097152.0);
    f = fmax(f, 0.0);
    f = fmin(f, 2097151.0);
    return (uint64_t)f;
}

struct D3 {
    double v[3];
};

template <class T>
__global__ void k_keys(const T *__restrict__ P, int64_t n, D3 o, double d0, uint64_t setbit, uint32_t idx0,
                       uint64_t *__restrict__ keys, uint32_t *__restrict__ idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t g0 = fine_coord((double)P[3 * i], o.v[0], d0);
    uint64_t g1 = fine_coord((double)P[3 * i + 1], o.v[1], d0);
    uint64_t g2 = fine_coord((double)P[3 * i + 2], o.v[2], d0);
    keys[i] = setbit | (spread3(g0) << 2) | (spread3(g1) << 1) | spread3(g2);
    idx[i] = idx0 + (uint32_t)i;
}

// After the joint sort: split (keys, vals) into the X part [0, nx) and the Y part.
__global__ void k_split_sorted(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t nx,
                               int64_t n, uint64_t *__restrict__ kx, uint64_t *__restrict__ ky,
                               uint32_t *__restrict__ px, uint32_t *__restrict__ py) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = keys[i] & 0x7fffffffffffffffull;
    if (i < nx) {
        kx[i] = k;
        px[i] = vals[i];
    } else {
        ky[i - nx] = k;
        py[i - nx] = vals[i] - (uint32_t)nx;
    }
}

// First level at which point i and point i-1 lie in different boxes; counts per level.
__global__ void k_levels(const uint64_t *__restrict__ key, int64_t n, uint8_t *__restrict__ f,
                         unsigned long long *__restrict__ counts) {
    __shared__ unsigned int c[LMAX + 1];
    if (threadIdx.x <= LMAX) c[threadIdx.x] = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int lev = 0;
        if (i > 0) {
            uint64_t d = key[i] ^ key[i - 1];
            lev = d ? LMAX - (63 - __clzll((long long)d)) / 3 : LMAX + 1;
        }
        f[i] = (uint8_t)lev;
        if (i > 0 && lev <= LMAX) atomicAdd(&c[lev], 1u);
    }
    __syncthreads();
    if (threadIdx.x <= LMAX && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)c[threadIdx.x]);
}

__global__ void k_flag_le(const uint8_t *__restrict__ f, int64_t n, int l, uint32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (f[i] <= l) ? 1u : 0u;
}

// Deepest box table: starts of boxes (points with f <= l) and each box's f value.
__global__ void k_compact_pts(const uint8_t *__restrict__ f, const uint32_t *__restrict__ pos, int64_t n, int l,
                              uint32_t *__restrict__ start, uint8_t *__restrict__ bf, int64_t nb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && f[i] <= l) {
        start[pos[i]] = (uint32_t)i;
        bf[pos[i]] = f[i];
    }
    if (i == 0) start[nb] = (uint32_t)n;
}

// Coarser table from the deepest one: boxes of the deep table with f <= l.
__global__ void k_compact_boxes(const uint8_t *__restrict__ bf, const uint32_t *__restrict__ dstart,
                                const uint32_t *__restrict__ pos, int64_t nd, int l, int64_t n,
                                uint32_t *__restrict__ start, uint32_t *__restrict__ fine, int64_t nb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nd && bf[i] <= l) {
        start[pos[i]] = dstart[i];
        fine[pos[i]] = (uint32_t)i;
    }
    if (i == 0) start[nb] = (uint32_t)n;
}

__global__ void k_iota(uint32_t *a, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = (uint32_t)i;
}

__global__ void k_box_coords(const uint64_t *__restrict__ key, const uint32_t *__restrict__ start, int64_t nb,
                             int l, int4 *__restrict__ g) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    uint64_t k = key[start[b]];
    int sh = LMAX - l;
    g[b] = make_int4((int)(compact3(k >> 2) >> sh), (int)(compact3(k >> 1) >> sh), (int)(compact3(k) >> sh), 0);
}

// out[b] = first index j in sorted `hay` (length nh) with hay[j] >= needle[b]; out[nb] = nh.
__global__ void k_lower_bound(const uint32_t *__restrict__ needle, int64_t nb, const uint32_t *__restrict__ hay,
                              int64_t nh, uint32_t *__restrict__ out) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nb) return;
    if (b == nb) {
        out[nb] = (uint32_t)nh;
        return;
    }
    uint32_t x = needle[b];
    int64_t lo = 0, hi = nh;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (hay[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    out[b] = (uint32_t)lo;
}

// ================================================================== descent

// Two-pass expansion without candidate arrays: pass 1 counts the admissible children of
// each near pair, pass 2 writes admissible and near child pairs at their scanned offsets.
// Children of (a, b) are visited in the same order in both passes.

// Admissibility of a child pair as integer comparisons.  The offset test |sigma + k| >= 2
// (k = g_X - g_Y per axis, sigma the trees' shift in box units, FP64) depends on k through
// the rounded sum fl(sigma + k), which is non-decreasing in k: it holds exactly for k >= klo
// or k <= khi, the two integer thresholds found on the host by evaluating that same FP64
// sum (adm_thresholds).  The decision is therefore the FP64 one, bit for bit.
struct AdmK {
    int lo[3], hi[3];
};

__device__ __forceinline__ bool child_adm_k(int4 p, int4 q, const AdmK &K) {
    int kx = p.x - q.x, ky = p.y - q.y, kz = p.z - q.z;
    return kx >= K.lo[0] || kx <= K.hi[0] || ky >= K.lo[1] || ky <= K.hi[1] || kz >= K.lo[2] || kz <= K.hi[2];
}

static AdmK adm_thresholds(const D3 &sig) {
    AdmK K;
    for (int d = 0; d < 3; ++d) {
        const volatile double sv = sig.v[d];
        // smallest k with fl(sigma + k) >= 2, largest k with fl(sigma + k) <= -2
        int lo = (int)std::floor(2.0 - sv) - 2;
        while (!(sv + (double)lo >= 2.0)) ++lo;
        while (sv + (double)(lo - 1) >= 2.0) --lo;
        int hi = (int)std::ceil(-2.0 - sv) + 2;
        while (!(sv + (double)hi <= -2.0)) --hi;
        while (sv + (double)(hi + 1) <= -2.0) ++hi;
        K.lo[d] = lo;
        K.hi[d] = hi;
    }
    return K;
}

// One warp per near pair (a, b) of level l: lane c takes child pair c and c + 32 of the at
// most 8 x 8 children (a2 = first child of a + c / nb, b2 = first child of b + c % nb);
// ballots count and place the admissible ones and the near ones, so a warp writes its
// pairs contiguously.
constexpr int EXP_W = 8;  // warps (near pairs) per block

__global__ void __launch_bounds__(32 * EXP_W) k_expand_count(const uint32_t *__restrict__ na,
                                                            const uint32_t *__restrict__ nbb, int64_t nnear,
                                                            const uint32_t *__restrict__ fcx,
                                                            const uint32_t *__restrict__ fcy,
                                                            const int4 *__restrict__ gx, const int4 *__restrict__ gy,
                                                            AdmK K, uint32_t *__restrict__ nadm,
                                                            uint32_t *__restrict__ nnr) {
    const int lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * EXP_W + (threadIdx.x >> 5);
    if (e >= nnear) return;
    const uint32_t a = na[e], b = nbb[e];
    const uint32_t a0 = fcx[a], b0 = fcy[b];
    const int nax = (int)(fcx[a + 1] - a0), nby = (int)(fcy[b + 1] - b0), tot = nax * nby;
    uint32_t c = 0;
    for (int c0 = 0; c0 < tot; c0 += 32) {
        const int ci = c0 + lane;
        bool adm = false;
        if (ci < tot) adm = child_adm_k(gx[a0 + ci / nby], gy[b0 + ci % nby], K);
        c += __popc(__ballot_sync(0xffffffffu, adm));
    }
    if (lane == 0) {
        nadm[e] = c;
        nnr[e] = (uint32_t)tot - c;
    }
}

__global__ void __launch_bounds__(32 * EXP_W) k_expand_emit(const uint32_t *__restrict__ na,
                                                           const uint32_t *__restrict__ nbb, int64_t nnear,
                                                           const uint32_t *__restrict__ fcx,
                                                           const uint32_t *__restrict__ fcy,
                                                           const int4 *__restrict__ gx, const int4 *__restrict__ gy,
                                                           AdmK K, const uint32_t *__restrict__ oadm,
                                                           const uint32_t *__restrict__ onr, uint32_t *__restrict__ aa,
                                                           uint32_t *__restrict__ ab, uint32_t *__restrict__ ea,
                                                           uint32_t *__restrict__ eb) {
    const int lane = threadIdx.x & 31;
    const int64_t e = (int64_t)blockIdx.x * EXP_W + (threadIdx.x >> 5);
    if (e >= nnear) return;
    const uint32_t a = na[e], b = nbb[e];
    const uint32_t a0 = fcx[a], b0 = fcy[b];
    const int nax = (int)(fcx[a + 1] - a0), nby = (int)(fcy[b + 1] - b0), tot = nax * nby;
    uint32_t ia = oadm[e], in = onr[e];
    const uint32_t below = (1u << lane) - 1u;
    for (int c0 = 0; c0 < tot; c0 += 32) {
        const int ci = c0 + lane;
        const bool valid = ci < tot;
        uint32_t a2 = 0, b2 = 0;
        bool adm = false;
        if (valid) {
            a2 = a0 + (uint32_t)(ci / nby);
            b2 = b0 + (uint32_t)(ci % nby);
            adm = child_adm_k(gx[a2], gy[b2], K);
        }
        const uint32_t ma = __ballot_sync(0xffffffffu, valid && adm), mn = __ballot_sync(0xffffffffu, valid && !adm);
        if (valid) {
            if (adm) {
                uint32_t o = ia + __popc(ma & below);
                aa[o] = a2;
                ab[o] = b2;
            } else {
                uint32_t o = in + __popc(mn & below);
                ea[o] = a2;
                eb[o] = b2;
            }
        }
        ia += __popc(ma);
        in += __popc(mn);
    }
}


__global__ void k_gather_u32(const uint32_t *__restrict__ src, const uint32_t *__restrict__ idx, int64_t n,
                             uint32_t *__restrict__ dst) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// Translation code of a pair: integer offset m = gX - gY relative to c = round(-sigma 2^l),
// 4 bits per axis (the descent bounds |sigma 2^l + m| < 5).
// Translation code of every pair; the codes in use are collected in a 4096-bit map per block
// (shared atomics) and written once per block and code, not once per pair.
__global__ void k_trans_code(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b, int64_t n,
                             const int4 *__restrict__ gx, const int4 *__restrict__ gy, int4 c,
                             uint32_t *__restrict__ code, uint32_t *__restrict__ used, int *__restrict__ err) {
    __shared__ uint32_t bits[128];
    if (threadIdx.x < 128) bits[threadIdx.x] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int4 p = gx[a[i]], q = gy[b[i]];
        int mx = p.x - q.x - c.x + 8, my = p.y - q.y - c.y + 8, mz = p.z - q.z - c.z + 8;
        if (mx < 0 || mx > 15 || my < 0 || my > 15 || mz < 0 || mz > 15) {
            atomicOr(err, 1);
            mx = my = mz = 0;
        }
        uint32_t k = (uint32_t)(mx | (my << 4) | (mz << 8));
        code[i] = k;
        atomicOr(&bits[k >> 5], 1u << (k & 31));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 4096; k += blockDim.x)
        if (bits[k >> 5] & (1u << (k & 31))) used[k] = 1u;
}

__global__ void k_trans_list(const uint32_t *__restrict__ used, const uint32_t *__restrict__ pos, int4 c,
                             int4 *__restrict__ m) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 4096 && used[k]) m[pos[k]] = make_int4((k & 15) - 8 + c.x, ((k >> 4) & 15) - 8 + c.y, (k >> 8) - 8 + c.z, 0);
}

__global__ void k_map(const uint32_t *__restrict__ code, const uint32_t *__restrict__ pos, int64_t n,
                      uint32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = pos[code[i]];
}

__global__ void k_run_starts(const uint32_t *__restrict__ a, int64_t n, uint32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (i == 0 || a[i] != a[i - 1]) ? 1u : 0u;
}

__global__ void k_run_list(const uint32_t *__restrict__ a, const uint32_t *__restrict__ flag,
                           const uint32_t *__restrict__ pos, int64_t n, int64_t nruns, uint32_t *__restrict__ ids,
                           uint32_t *__restrict__ off) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) {
        ids[pos[i]] = a[i];
        off[pos[i]] = (uint32_t)i;
    }
    if (i == 0) off[nruns] = (uint32_t)n;
}

__global__ void k_mark(const uint32_t *__restrict__ b, int64_t n, uint32_t *__restrict__ used) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) used[b[i]] = 1u;
}

__global__ void k_list_marked(const uint32_t *__restrict__ used, const uint32_t *__restrict__ pos, int64_t n,
                              uint32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && used[i]) out[pos[i]] = (uint32_t)i;
}

// sum over listed boxes of their point counts
__global__ void k_sum_sizes(const uint32_t *__restrict__ list, int64_t n, const uint32_t *__restrict__ start,
                            unsigned long long *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) v = start[list[i] + 1] - start[list[i]];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// sum over pairs (a, b) of n_a * n_b
__global__ void k_sum_pair_sizes(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b, int64_t n,
                                 const uint32_t *__restrict__ sa, const uint32_t *__restrict__ sb,
                                 unsigned long long *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long v = 0;
    if (i < n) v = (unsigned long long)(sa[a[i] + 1] - sa[a[i]]) * (sb[b[i] + 1] - sb[b[i]]);
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

static int64_t read_u64(const unsigned long long *d, cudaStream_t s) {
    unsigned long long h;
    FFM_CUDA(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    return (int64_t)h;
}

__global__ void k_hist_u32(const uint32_t *__restrict__ a, int64_t n, uint32_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[a[i]], 1u);
}

// CSR offsets of a sorted key array: off[b] = first i with key[i] >= b, b = 0..nkeys.
__global__ void k_csr_offsets(const uint32_t *__restrict__ key, int64_t n, int64_t nkeys, uint32_t *__restrict__ off) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nkeys) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (key[mid] < (uint32_t)b)
            lo = mid + 1;
        else
            hi = mid;
    }
    off[b] = (uint32_t)lo;
}

static uint32_t read_u32(const uint32_t *d, cudaStream_t s) {
    uint32_t h;
    FFM_CUDA(cudaMemcpyAsync(&h, d, sizeof h, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    return h;
}

// Near-field work items of one target leaf: its targets in chunks of tchunk times its
// near pairs split into consecutive ranges of at most smax source points.
__device__ __forceinline__ int p2p_ranges(const uint32_t *off, const uint32_t *src, const uint32_t *ystart, int64_t a,
                                          int4 *out, int base, int tc, int tchunk, uint32_t smax) {
    int nr = 0;
    uint32_t e0 = off[a], acc = 0;
    for (uint32_t e = off[a]; e < off[a + 1]; ++e) {
        uint32_t nb = ystart[src[e] + 1] - ystart[src[e]];
        if (acc > 0 && acc + nb > smax) {
            if (out)
                for (int c = 0; c < tc; ++c) out[base + nr * tc + c] = make_int4((int)a, c * tchunk, (int)e0, (int)e);
            ++nr;
            e0 = e;
            acc = 0;
        }
        acc += nb;
    }
    if (off[a + 1] > off[a]) {
        if (out)
            for (int c = 0; c < tc; ++c)
                out[base + nr * tc + c] = make_int4((int)a, c * tchunk, (int)e0, (int)off[a + 1]);
        ++nr;
    }
    return nr;
}

__global__ void k_p2p_items(const uint32_t *__restrict__ off, const uint32_t *__restrict__ src,
                            const uint32_t *__restrict__ xstart, const uint32_t *__restrict__ ystart, int64_t nleaf,
                            int tchunk, uint32_t smax, const uint32_t *__restrict__ pos, uint32_t *__restrict__ cnt,
                            int4 *__restrict__ out) {
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nleaf) return;
    int np = (int)(xstart[a + 1] - xstart[a]);
    int tc = (np + tchunk - 1) / tchunk;
    if (!out) {
        cnt[a] = (uint32_t)(p2p_ranges(off, src, ystart, a, nullptr, 0, tc, tchunk, smax) * tc);
    } else {
        p2p_ranges(off, src, ystart, a, out, (int)pos[a], tc, tchunk, smax);
    }
}

// Work items for the near field with targets in chunks of tchunk (<= P2P_T) and at most
// smax source points per item (a larger single leaf stays whole); returns the count.
int64_t build_p2p_items(ffm_plan_s *p, int tchunk, uint32_t smax, Alloc &out_mem, int4 **items, Alloc &tmp,
                        cudaStream_t s) {
    int ls = p->l_stop;
    int64_t nleafX = p->bx[ls].nb;
    uint32_t *icnt = tmp.get<uint32_t>(nleafX + 1), *ipos = tmp.get<uint32_t>(nleafX + 1);
    FFM_CUDA(cudaMemsetAsync(icnt, 0, sizeof(uint32_t) * (nleafX + 1), s));
    FFM_LAUNCH(k_p2p_items, cdiv(nleafX, 128), 128, 0, s, p->near_off, p->near_src, p->bx[ls].start, p->by[ls].start,
               nleafX, tchunk, smax, (const uint32_t *)nullptr, icnt, (int4 *)nullptr);
    uint32_t *itot = tmp.get<uint32_t>(1);
    scan_u32(icnt, ipos, nleafX + 1, itot, tmp, s);
    int64_t n = read_u32(itot, s);
    *items = out_mem.get<int4>(n);
    FFM_LAUNCH(k_p2p_items, cdiv(nleafX, 128), 128, 0, s, p->near_off, p->near_src, p->bx[ls].start, p->by[ls].start,
               nleafX, tchunk, smax, ipos, icnt, *items);
    return n;
}

// Target box of every pair of a CSR list (pairs of listed target x: [off[x], off[x+1])).
__global__ void k_expand_csr_targets(const uint32_t *__restrict__ tgt, const uint32_t *__restrict__ off, int64_t nt,
                                     uint32_t *__restrict__ out) {
    int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nt) return;
    for (uint32_t e = off[x]; e < off[x + 1]; ++e) out[e] = tgt[x];
}

// ======================================================== leaf coordinates

template <class T>
__global__ void k_leaf_eps(const T *__restrict__ P, const uint32_t *__restrict__ perm,
                           const uint64_t *__restrict__ key, const uint32_t *__restrict__ lstart, int64_t nleaf,
                           int64_t n, D3 o, double dls, int ls, float4 *__restrict__ eps, float4 *__restrict__ lo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = key[i];
    int sh = LMAX - ls;
    double g0 = (double)(compact3(k >> 2) >> sh), g1 = (double)(compact3(k >> 1) >> sh), g2 = (double)(compact3(k) >> sh);
    uint32_t j = perm[i];
    // leaf-relative coordinates as an unevaluated FP32 pair hi + lo
    double d0 = (double)P[3 * (int64_t)j] - (o.v[0] + (g0 + 0.5) * dls);
    double d1 = (double)P[3 * (int64_t)j + 1] - (o.v[1] + (g1 + 0.5) * dls);
    double d2 = (double)P[3 * (int64_t)j + 2] - (o.v[2] + (g2 + 0.5) * dls);
    float e0 = (float)d0, e1 = (float)d1, e2 = (float)d2;
    int64_t lo_ = 0, hi_ = nleaf - 1;  // last leaf with start <= i
    while (lo_ < hi_) {
        int64_t mid = (lo_ + hi_ + 1) >> 1;
        if (lstart[mid] <= (uint32_t)i)
            lo_ = mid;
        else
            hi_ = mid - 1;
    }
    eps[i] = make_float4(e0, e1, e2, __uint_as_float((uint32_t)lo_));
    lo[i] = make_float4((float)(d0 - (double)e0), (float)(d1 - (double)e1), (float)(d2 - (double)e2), 0.f);
}

template <class T>
__global__ void k_sorted_weights(const T *__restrict__ w, const uint32_t *__restrict__ perm, int64_t n,
                                 double *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)w[perm[i]];
}

// Source normals in Morton order as unevaluated FP32 pairs (hi, lo): the double layer's
// n . (x - y) cancels to second order in |x - y| for points of one surface.
template <class T>
__global__ void k_sorted_normals(const T *__restrict__ nrm, const uint32_t *__restrict__ perm, int64_t n,
                                 float4 *__restrict__ hi, float4 *__restrict__ lo) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T *v = nrm + 3 * (int64_t)perm[i];
    double a = (double)v[0], b = (double)v[1], c = (double)v[2];
    float ah = (float)a, bh = (float)b, ch = (float)c;
    hi[i] = make_float4(ah, bh, ch, 0.f);
    lo[i] = make_float4((float)(a - (double)ah), (float)(b - (double)bh), (float)(c - (double)ch), 0.f);
}

// ================================================================ host side

static int bits_for(int64_t n) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) < n) ++b;
    return b;
}

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device copy of a caller array (host or device) of `bytes` bytes.
static const void *to_device(const void *p, size_t bytes, Alloc &tmp, cudaStream_t s) {
    if (is_device_ptr(p)) return p;
    void *d = tmp.raw(bytes);
    FFM_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s));
    return d;
}

template <class T>
static void launch_keys(const void *P, int64_t n, const double o[3], double d0, uint64_t setbit, uint32_t idx0,
                        uint64_t *keys, uint32_t *idx, cudaStream_t s) {
    D3 oo{{o[0], o[1], o[2]}};
    FFM_LAUNCH(k_keys<T>, cdiv(n, 256), 256, 0, s, (const T *)P, n, oo, d0, setbit, idx0, keys, idx);
}

template <class T>
static void launch_bbox(const void *P, int64_t n, unsigned long long *out, cudaStream_t s) {
    FFM_LAUNCH(k_bbox<T>, std::min<unsigned>(cdiv(n, 256), 2048u), 256, 0, s, (const T *)P, n, out);
}

template <class T>
static void launch_leaf_eps(const void *P, const uint32_t *perm, const uint64_t *key, const uint32_t *lstart,
                            int64_t nleaf, int64_t n, const double o[3], double dls, int ls, float4 *eps,
                            float4 *lo, cudaStream_t s) {
    D3 oo{{o[0], o[1], o[2]}};
    FFM_LAUNCH(k_leaf_eps<T>, cdiv(n, 256), 256, 0, s, (const T *)P, perm, key, lstart, nleaf, n, oo, dls, ls, eps,
               lo);
}


// Box tables of one set for levels 0..ldeep (boxes at level l = runs of key >> 3(21-l)).
static void build_boxes(ffm_plan_s *p, BoxLevel *bl, const uint64_t *key, int64_t n, const uint8_t *f,
                        const int64_t *nb, int ldeep, Alloc &tmp, cudaStream_t s) {
    Alloc &m = p->mem;
    uint32_t *flag = tmp.get<uint32_t>(n), *pos = tmp.get<uint32_t>(n);
    FFM_LAUNCH(k_flag_le, cdiv(n, 256), 256, 0, s, f, n, ldeep, flag);
    scan_u32(flag, pos, n, nullptr, tmp, s);
    int64_t nd = nb[ldeep];
    BoxLevel &D = bl[ldeep];
    D.nb = nd;
    D.start = m.get<uint32_t>(nd + 1);
    uint8_t *bf = tmp.get<uint8_t>(nd);
    FFM_LAUNCH(k_compact_pts, cdiv(n, 256), 256, 0, s, f, pos, n, ldeep, D.start, bf, nd);
    D.fine = m.get<uint32_t>(nd);
    FFM_LAUNCH(k_iota, cdiv(nd, 256), 256, 0, s, D.fine, nd);
    uint32_t *bflag = tmp.get<uint32_t>(nd), *bpos = tmp.get<uint32_t>(nd);
    for (int l = 0; l < ldeep; ++l) {
        BoxLevel &B = bl[l];
        B.nb = nb[l];
        B.start = m.get<uint32_t>(B.nb + 1);
        B.fine = m.get<uint32_t>(B.nb);
        FFM_LAUNCH(k_flag_le, cdiv(nd, 256), 256, 0, s, bf, nd, l, bflag);
        scan_u32(bflag, bpos, nd, nullptr, tmp, s);
        FFM_LAUNCH(k_compact_boxes, cdiv(nd, 256), 256, 0, s, bf, D.start, bpos, nd, l, n, B.start, B.fine, B.nb);
    }
    for (int l = 0; l <= ldeep; ++l) {
        BoxLevel &B = bl[l];
        B.g = m.get<int4>(B.nb);
        FFM_LAUNCH(k_box_coords, cdiv(B.nb, 256), 256, 0, s, key, B.start, B.nb, l, B.g);
        if (l < ldeep) {
            B.first_child = m.get<uint32_t>(B.nb + 1);
            FFM_LAUNCH(k_lower_bound, cdiv(B.nb + 1, 256), 256, 0, s, B.fine, B.nb, bl[l + 1].fine, bl[l + 1].nb,
                       B.first_child);
        }
    }
}

// Sort pairs (a, b) by a (stable), then CSR: list of distinct a (ids), offsets per id.
struct Csr {
    int64_t n = 0, nruns = 0;
    uint32_t *a = nullptr, *b = nullptr, *ids = nullptr, *off = nullptr, *perm = nullptr;
};

static Csr group_by_target(uint32_t *a, uint32_t *b, int64_t n, int64_t nbx, Alloc &dst, Alloc &tmp,
                           cudaStream_t s) {
    Csr c;
    c.n = n;
    c.perm = tmp.get<uint32_t>(n);
    FFM_LAUNCH(k_iota, cdiv(n, 256), 256, 0, s, c.perm, n);
    radix_sort_u32(a, c.perm, n, bits_for(nbx), tmp, s);
    c.a = a;
    c.b = dst.get<uint32_t>(n);
    FFM_LAUNCH(k_gather_u32, cdiv(n, 256), 256, 0, s, b, c.perm, n, c.b);
    uint32_t *flag = tmp.get<uint32_t>(n), *pos = tmp.get<uint32_t>(n), *tot = tmp.get<uint32_t>(1);
    FFM_LAUNCH(k_run_starts, cdiv(n, 256), 256, 0, s, a, n, flag);
    scan_u32(flag, pos, n, tot, tmp, s);
    c.nruns = read_u32(tot, s);
    c.ids = dst.get<uint32_t>(c.nruns);
    c.off = dst.get<uint32_t>(c.nruns + 1);
    FFM_LAUNCH(k_run_list, cdiv(n, 256), 256, 0, s, a, flag, pos, n, c.nruns, c.ids, c.off);
    return c;
}

static int oscillatory(const ffm_plan_s *p, int l) {
    double dl = std::ldexp(p->d0, -l);
    return p->kind == FFM_HELMHOLTZ && p->k * dl >= p->kappa;
}

static int pw_rank(double k, double dl, double eps) {
    int L = (int)std::floor(std::fabs(k) * std::sqrt(3.0) * dl - std::log(eps));
    return L < 1 ? 1 : L;
}

// Record the admissible pairs of level l: CSR by target box, source list, translations.
// Chunks of at most ch points of the listed boxes: (box, first point), so that the
// point-wise kernels of a level spread large boxes over many blocks.
__global__ void k_chunk_count(const uint32_t *__restrict__ list, int64_t n, const uint32_t *__restrict__ start,
                              uint32_t ch, uint32_t *__restrict__ cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t b = list[i];
    cnt[i] = (start[b + 1] - start[b] + ch - 1) / ch;
}
__global__ void k_chunk_emit(const uint32_t *__restrict__ list, int64_t n, const uint32_t *__restrict__ start,
                             uint32_t ch, const uint32_t *__restrict__ pos, uint2 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t b = list[i], k = pos[i];
    for (uint32_t q = start[b]; q < start[b + 1]; q += ch) out[k++] = make_uint2(b, q);
}

static uint2 *build_chunks(ffm_plan_s *p, const uint32_t *list, int64_t n, const uint32_t *start, int64_t *count,
                           Alloc &tmp, cudaStream_t s, uint32_t ch = LAG_CHUNK) {
    uint32_t *cnt = tmp.get<uint32_t>(n), *pos = tmp.get<uint32_t>(n), *tot = tmp.get<uint32_t>(1);
    FFM_LAUNCH(k_chunk_count, cdiv(n, 256), 256, 0, s, list, n, start, ch, cnt);
    scan_u32(cnt, pos, n, tot, tmp, s);
    *count = read_u32(tot, s);
    uint2 *out = p->mem.get<uint2>(*count);
    FFM_LAUNCH(k_chunk_emit, cdiv(n, 256), 256, 0, s, list, n, start, ch, pos, out);
    return out;
}

// Admissible partners of each target box sorted by translation index, one warp per target.
// Translations are distinct within a target and below 4096, so the sort is a rank by
// counting: the warp sets one bit per partner's translation in a 4096-bit map in shared
// memory, prefix-counts the map's words, and each partner's rank is the number of set bits
// below its own.  Targets with more than 512 partners are left as they are and flagged.
constexpr int SP_MAX = 512;
__global__ void __launch_bounds__(128) k_sort_partners(const uint32_t *__restrict__ off, int64_t n_tgt,
                                                       uint32_t *__restrict__ src, uint32_t *__restrict__ tr,
                                                       int *__restrict__ too_long) {
    __shared__ uint32_t bm[4][128], pre[4][128];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t x = (int64_t)blockIdx.x * 4 + w;
    if (x >= n_tgt) return;  // warp-level work only: no block barrier below
    uint32_t e0 = off[x];
    int n = (int)(off[x + 1] - e0);
    if (n > SP_MAX) {
        if (lane == 0) atomicOr(too_long, 1);
        return;
    }
    uint32_t *b = bm[w], *pr = pre[w];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[lane * 4 + j] = 0u;
    __syncwarp();
    uint32_t t[SP_MAX / 32], sv[SP_MAX / 32];
#pragma unroll
    for (int k = 0; k < SP_MAX / 32; ++k) {
        int i = lane + 32 * k;
        if (i < n) {
            t[k] = tr[e0 + i];
            sv[k] = src[e0 + i];
            atomicOr(&b[t[k] >> 5], 1u << (t[k] & 31));
        }
    }
    __syncwarp();
    uint32_t c[4], tot = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c[j] = __popc(b[lane * 4 + j]);
        tot += c[j];
    }
    uint32_t inc = tot;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
    }
    uint32_t run = inc - tot;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        pr[lane * 4 + j] = run;
        run += c[j];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < SP_MAX / 32; ++k) {
        int i = lane + 32 * k;
        if (i < n) {
            uint32_t q = t[k];
            uint32_t rank = pr[q >> 5] + __popc(b[q >> 5] & ((1u << (q & 31)) - 1u));
            tr[e0 + rank] = q;
            src[e0 + rank] = sv[k];
        }
    }
}

// Data of the target-stationary transfer for Lagrange level l, made on demand (it is used
// when forced or picked by the autotuner): partners sorted by translation within each
// target (the sort keeps every other consumer of the CSR lists valid) and T_t pre-split.
// Sets ts_ok if every target has at most 512 partners.
void prepare_target_stationary(ffm_plan_s *p, int l, cudaStream_t s) {
    FarLevel &F = p->far[l];
    if (F.mode != 1 || F.n_adm == 0 || F.Tsp || p->kind != FFM_LAPLACE || F.r1 > 4) return;
    Alloc tmp;
    tmp.stream = s;
    int *flag = tmp.get<int>(1);
    FFM_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    FFM_LAUNCH(k_sort_partners, cdiv(F.n_tgt, 4), 128, 0, s, F.adm_off, F.n_tgt, F.adm_src, F.adm_t, flag);
    launch_table_split(p, l, s);
    int hflag = 1;
    FFM_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    F.ts_ok = hflag == 0;
    // a level the target-stationary kernel cannot take runs the per-translation transfer
    if (!F.ts_ok) build_translation_groups(p, l, s);
}

// Column tiles of the per-translation transfer: tile i of translation t covers pairs
// off[t] + i bn .. (count per translation, then one block per translation emits its tiles).
__global__ void k_tile_count(const uint32_t *__restrict__ off, int n_trans, uint32_t bn, uint32_t *__restrict__ cnt) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n_trans) cnt[t] = (off[t + 1] - off[t] + bn - 1) / bn;
}
__global__ void k_tile_emit(const uint32_t *__restrict__ off, uint32_t bn, const uint32_t *__restrict__ pos,
                            uint32_t *__restrict__ tt, uint32_t *__restrict__ tp) {
    int t = blockIdx.x;
    uint32_t p0 = off[t], n = (off[t + 1] - p0 + bn - 1) / bn, o = pos[t];
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        tt[o + i] = (uint32_t)t;
        tp[o + i] = p0 + i * bn;
    }
}

static int64_t build_tiles(ffm_plan_s *p, const FarLevel &F, uint32_t bn, uint32_t **tt, uint32_t **tp, Alloc &tmp,
                           cudaStream_t s) {
    uint32_t *cnt = tmp.get<uint32_t>(F.n_trans), *pos = tmp.get<uint32_t>(F.n_trans), *tot = tmp.get<uint32_t>(1);
    FFM_LAUNCH(k_tile_count, cdiv(F.n_trans, 256), 256, 0, s, F.bt_off, F.n_trans, bn, cnt);
    scan_u32(cnt, pos, F.n_trans, tot, tmp, s);
    int64_t n = read_u32(tot, s);
    *tt = p->mem.get<uint32_t>(n);
    *tp = p->mem.get<uint32_t>(n);
    if (n > 0) FFM_LAUNCH(k_tile_emit, F.n_trans, 128, 0, s, F.bt_off, bn, pos, *tt, *tp);
    return n;
}

// Pairs of Lagrange level l grouped by translation (CSR bt_off over translations, with each
// pair's source and target box) and the column tiles of the per-translation transfer
// kernels (32 pairs for the CUDA-core GEMM, 256 for tcgen05).  Made while the plan is built,
// or later by the autotuner or when the target-stationary transfer cannot take the level;
// a level that runs the target-stationary transfer does without them.
void build_translation_groups(ffm_plan_s *p, int l, cudaStream_t s) {
    FarLevel &F = p->far[l];
    if (F.mode != 1 || F.n_adm == 0 || F.bt_off) return;
    const int64_t na = F.n_adm;
    Alloc tmp;
    tmp.stream = s;
    uint32_t *tk = tmp.get<uint32_t>(na), *pidx = tmp.get<uint32_t>(na);
    FFM_CUDA(cudaMemcpyAsync(tk, F.adm_t, sizeof(uint32_t) * na, cudaMemcpyDeviceToDevice, s));
    FFM_LAUNCH(k_iota, cdiv(na, 256), 256, 0, s, pidx, na);
    radix_sort_u32(tk, pidx, na, bits_for(F.n_trans), tmp, s);
    // target of every pair in CSR order
    uint32_t *ptgt = tmp.get<uint32_t>(na);
    FFM_LAUNCH(k_expand_csr_targets, cdiv(F.n_tgt, 128), 128, 0, s, F.tgt, F.adm_off, F.n_tgt, ptgt);
    F.bt_src = p->mem.get<uint32_t>(na);
    F.bt_tgt = p->mem.get<uint32_t>(na);
    FFM_LAUNCH(k_gather_u32, cdiv(na, 256), 256, 0, s, F.adm_src, pidx, na, F.bt_src);
    FFM_LAUNCH(k_gather_u32, cdiv(na, 256), 256, 0, s, ptgt, pidx, na, F.bt_tgt);
    F.bt_off = p->mem.get<uint32_t>(F.n_trans + 1);
    FFM_LAUNCH(k_csr_offsets, cdiv(F.n_trans + 1, 256), 256, 0, s, tk, na, F.n_trans, F.bt_off);
    F.n_tiles = build_tiles(p, F, LAG_GEMM_BN, &F.tile_t, &F.tile_p0, tmp, s);
    F.tc_tiles = build_tiles(p, F, 256, &F.tc_tile_t, &F.tc_tile_p0, tmp, s);
    tmp.release();
}

static void finish_far_level(ffm_plan_s *p, int l, uint32_t *aa, uint32_t *ab, int64_t na, Alloc &tmp,
                             cudaStream_t s) {
    FarLevel &F = p->far[l];
    F.n_adm = na;
    p->info.n_adm[l] = na;
    if (na == 0) return;
    F.mode = oscillatory(p, l) ? 2 : 1;
    Csr c = group_by_target(aa, ab, na, p->bx[l].nb, p->mem, tmp, s);
    F.n_tgt = c.nruns;
    F.tgt = c.ids;
    F.adm_off = c.off;
    F.adm_src = c.b;
    // translations
    int4 cc;
    cc.x = (int)std::floor(-std::ldexp(p->sigma[0], l) + 0.5);
    cc.y = (int)std::floor(-std::ldexp(p->sigma[1], l) + 0.5);
    cc.z = (int)std::floor(-std::ldexp(p->sigma[2], l) + 0.5);
    cc.w = 0;
    if (l == 0) cc = make_int4(0, 0, 0, 0);  // the single root pair has m = 0
    uint32_t *code = tmp.get<uint32_t>(na), *used = tmp.get<uint32_t>(4096), *upos = tmp.get<uint32_t>(4096);
    uint32_t *tot = tmp.get<uint32_t>(1);
    int *err = tmp.get<int>(1);
    FFM_CUDA(cudaMemsetAsync(used, 0, 4096 * sizeof(uint32_t), s));
    FFM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    FFM_LAUNCH(k_trans_code, std::min<unsigned>(cdiv(na, 256), 152u * 8u), 256, 0, s, c.a, c.b, na, p->bx[l].g,
               p->by[l].g, cc, code, used, err);
    scan_u32(used, upos, 4096, tot, tmp, s);
    F.adm_t = p->mem.get<uint32_t>(na);
    FFM_LAUNCH(k_map, cdiv(na, 256), 256, 0, s, code, upos, na, F.adm_t);
    int herr = 0;
    FFM_CUDA(cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, s));
    F.n_trans = (int)read_u32(tot, s);
    if (herr) fail(FFM_ECUDA, "box translation outside the expected range");
    F.trans_m = p->mem.get<int4>(F.n_trans);
    FFM_LAUNCH(k_trans_list, 16, 256, 0, s, used, upos, cc, F.trans_m);
    F.h_trans_m.resize(F.n_trans);
    FFM_CUDA(cudaMemcpyAsync(F.h_trans_m.data(), F.trans_m, sizeof(int4) * F.n_trans, cudaMemcpyDeviceToHost, s));
    p->info.n_trans[l] = F.n_trans;
    // source boxes in use
    int64_t nby = p->by[l].nb;
    uint32_t *su = tmp.get<uint32_t>(nby), *spos = tmp.get<uint32_t>(nby);
    FFM_CUDA(cudaMemsetAsync(su, 0, sizeof(uint32_t) * nby, s));
    FFM_LAUNCH(k_mark, cdiv(na, 256), 256, 0, s, F.adm_src, na, su);
    scan_u32(su, spos, nby, tot, tmp, s);
    F.n_src = read_u32(tot, s);
    F.src = p->mem.get<uint32_t>(F.n_src);
    FFM_LAUNCH(k_list_marked, cdiv(nby, 256), 256, 0, s, su, spos, nby, F.src);
    unsigned long long *sums = tmp.get<unsigned long long>(2);
    FFM_CUDA(cudaMemsetAsync(sums, 0, 2 * sizeof(unsigned long long), s));
    FFM_LAUNCH(k_sum_sizes, cdiv(F.n_src, 256), 256, 0, s, F.src, F.n_src, p->by[l].start, sums);
    FFM_LAUNCH(k_sum_sizes, cdiv(F.n_tgt, 256), 256, 0, s, F.tgt, F.n_tgt, p->bx[l].start, sums + 1);
    p->info.src_points[l] = read_u64(sums, s);
    p->info.tgt_points[l] = read_u64(sums + 1, s);
    if (F.mode == 1) {
        F.r1 = p->r1_override > 0 ? p->r1_override : r1_rule(p->kind, p->eps);
        if (p->lag_transfer > 0) F.tune_tc = p->lag_transfer - 1;  // forced variant
        // pairs grouped by translation for the per-translation transfer kernels, unless the
        // level is to run the target-stationary transfer, which reads the per-target lists
        // (forced, or the pick stored in the plan's autotune cache); ACA levels need them
        const int pick = p->lag_transfer == 0 ? cached_lag_pick(p, l) : -1;
        const bool ts_first = (p->lag_transfer == 3 || pick == 2) && p->kind == FFM_LAPLACE && F.r1 <= 4 &&
                              !(p->aca_eps > 0.0);
        if (!ts_first) build_translation_groups(p, l, s);
        F.src_chunks = build_chunks(p, F.src, F.n_src, p->by[l].start, &F.n_src_chunks, tmp, s);
        F.tgt_chunks = build_chunks(p, F.tgt, F.n_tgt, p->bx[l].start, &F.n_tgt_chunks, tmp, s);
    }
    p->info.mode[l] = F.mode;
    if (F.mode == 1) {
        F.r1 = p->r1_override > 0 ? p->r1_override : r1_rule(p->kind, p->eps);
        p->info.r1[l] = F.r1;
    } else {
        F.L = pw_rank(p->k, std::ldexp(p->d0, -l), p->eps);
        F.nQ = 2 * F.L * (F.L + 1);
        p->info.L[l] = F.L;
        p->info.nQ[l] = F.nQ;
    }
}

void build_plan(ffm_plan_s *p, const void *X, ffm_dtype xdt, const void *Y, ffm_dtype ydt, const void *w,
                ffm_dtype wdt, Alloc &tmp) {
    cudaStream_t s = p->stream;
    int64_t nx = p->nx, ny = p->ny, n = nx + ny;
    size_t xb = (xdt == FFM_F64 ? 8 : 4) * 3 * (size_t)nx, yb = (ydt == FFM_F64 ? 8 : 4) * 3 * (size_t)ny;
    const void *dX = to_device(X, xb, tmp, s), *dY = to_device(Y, yb, tmp, s);

    p->dev_err = p->mem.get<int>(4);
    FFM_CUDA(cudaMemsetAsync(p->dev_err, 0, 4 * sizeof(int), s));

    // ---- root cubes (Sec. 2.2.1)
    unsigned long long *bb = tmp.get<unsigned long long>(14);
    unsigned long long init[14];
    for (int i = 0; i < 2; ++i) {
        for (int d = 0; d < 3; ++d) {
            init[7 * i + d] = ~0ull;
            init[7 * i + 3 + d] = 0ull;
        }
        init[7 * i + 6] = 0ull;
    }
    FFM_CUDA(cudaMemcpyAsync(bb, init, sizeof init, cudaMemcpyHostToDevice, s));
    if (xdt == FFM_F64)
        launch_bbox<double>(dX, nx, bb, s);
    else
        launch_bbox<float>(dX, nx, bb, s);
    if (ydt == FFM_F64)
        launch_bbox<double>(dY, ny, bb + 7, s);
    else
        launch_bbox<float>(dY, ny, bb + 7, s);
    unsigned long long hb[14];
    FFM_CUDA(cudaMemcpyAsync(hb, bb, sizeof hb, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    if (hb[6] || hb[13]) fail(FFM_EINVAL, "non-finite coordinate in X or Y");
    double lx[3], hx[3], ly[3], hy[3];
    for (int d = 0; d < 3; ++d) {
        lx[d] = ord_dec(hb[d]);
        hx[d] = ord_dec(hb[3 + d]);
        ly[d] = ord_dec(hb[7 + d]);
        hy[d] = ord_dec(hb[10 + d]);
    }
    double ex = 0, ey = 0;
    for (int d = 0; d < 3; ++d) {
        ex = std::max(ex, hx[d] - lx[d]);
        ey = std::max(ey, hy[d] - ly[d]);
    }
    double d0 = std::max(ex, ey);
    double infl = 1.0 + std::ldexp(1.0, -20);
    d0 = d0 > 0.0 ? d0 * infl : 1.0;
    for (int d = 0; d < 3; ++d) {
        double cx = 0.5 * (lx[d] + hx[d]), cy = 0.5 * (ly[d] + hy[d]);
        double hd = 0.5 * d0;
        p->oX[d] = cx - hd;
        p->oY[d] = cy - hd;
        p->sigma[d] = (p->oX[d] - p->oY[d]) / d0;
    }
    p->d0 = d0;
    p->info.d0 = d0;
    for (int d = 0; d < 3; ++d) {
        p->info.oX[d] = p->oX[d];
        p->info.oY[d] = p->oY[d];
    }

    // ---- Morton keys and the joint stable sort (X first: set bit 0; Y: set bit 1)
    Alloc sortmem;  // keys, indices and the sort's ping-pong buffers: released after the split
    sortmem.stream = s;
    uint64_t *keys = sortmem.get<uint64_t>(n);
    uint32_t *vals = sortmem.get<uint32_t>(n);
    if (xdt == FFM_F64)
        launch_keys<double>(dX, nx, p->oX, d0, 0ull, 0u, keys, vals, s);
    else
        launch_keys<float>(dX, nx, p->oX, d0, 0ull, 0u, keys, vals, s);
    if (ydt == FFM_F64)
        launch_keys<double>(dY, ny, p->oY, d0, 1ull << 63, (uint32_t)nx, keys + nx, vals + nx, s);
    else
        launch_keys<float>(dY, ny, p->oY, d0, 1ull << 63, (uint32_t)nx, keys + nx, vals + nx, s);
    radix_sort_u64(keys, vals, n, 64, sortmem, s);
    p->keyX = p->mem.get<uint64_t>(nx);
    p->keyY = p->mem.get<uint64_t>(ny);
    p->permX = p->mem.get<uint32_t>(nx);
    p->permY = p->mem.get<uint32_t>(ny);
    FFM_LAUNCH(k_split_sorted, cdiv(n, 256), 256, 0, s, keys, vals, nx, n, p->keyX, p->keyY, p->permX, p->permY);
    sortmem.release();

    // ---- boxes per level
    uint8_t *fX = tmp.get<uint8_t>(nx), *fY = tmp.get<uint8_t>(ny);
    unsigned long long *cnt = tmp.get<unsigned long long>(2 * (LMAX + 1));
    FFM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * (LMAX + 1), s));
    FFM_LAUNCH(k_levels, cdiv(nx, 256), 256, 0, s, p->keyX, nx, fX, cnt);
    FFM_LAUNCH(k_levels, cdiv(ny, 256), 256, 0, s, p->keyY, ny, fY, cnt + LMAX + 1);
    unsigned long long hc[2 * (LMAX + 1)];
    FFM_CUDA(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    int64_t nbx[LMAX + 1], nby[LMAX + 1];
    nbx[0] = nby[0] = 1;
    for (int l = 1; l <= LMAX; ++l) {
        nbx[l] = nbx[l - 1] + (int64_t)hc[l];
        nby[l] = nby[l - 1] + (int64_t)hc[LMAX + 1 + l];
    }
    // deepest level the occupancy rule can reach
    int ldeep = 0;
    while (ldeep < p->l_cap && !(n < (int64_t)p->n_leaf * (nbx[ldeep] + nby[ldeep]))) ++ldeep;
    build_boxes(p, p->bx, p->keyX, nx, fX, nbx, ldeep, tmp, s);
    build_boxes(p, p->by, p->keyY, ny, fY, nby, ldeep, tmp, s);
    for (int l = 0; l <= ldeep; ++l) {
        p->info.nboxX[l] = nbx[l];
        p->info.nboxY[l] = nby[l];
    }

    // ---- descent (Sec. 2.2.2, 2.2.4)
    bool root_adm = false;
    for (int d = 0; d < 3; ++d)
        if (std::fabs(p->sigma[d]) >= 2.0) root_adm = true;
    Alloc levels[LMAX + 2];  // per-level temporaries of the descent, released level by level
    TableJob tj(s);
    uint32_t *nearA = tmp.get<uint32_t>(1), *nearB = tmp.get<uint32_t>(1);
    FFM_CUDA(cudaMemsetAsync(nearA, 0, sizeof(uint32_t), s));
    FFM_CUDA(cudaMemsetAsync(nearB, 0, sizeof(uint32_t), s));
    int64_t nnear = 1;
    p->l_stop = 0;
    if (root_adm) {
        p->root_adm = 1;
        p->info.root_admissible = 1;
        finish_far_level(p, 0, nearA, nearB, 1, tmp, s);
        if (p->far[0].n_adm > 0) build_tables(p, 0, tj);
        nnear = 0;
    } else {
        p->info.n_near[0] = 1;
        for (int l = 0;; ++l) {
            bool stop = nnear == 0 || n < (int64_t)p->n_leaf * (nbx[l] + nby[l]) || l >= p->l_cap;
            if (stop) {
                p->l_stop = l;
                break;
            }
            int lc = l + 1;
            D3 sg{{std::ldexp(p->sigma[0], lc), std::ldexp(p->sigma[1], lc), std::ldexp(p->sigma[2], lc)}};
            Alloc &lvl = levels[lc];
            lvl.stream = s;
            uint32_t *nadm = lvl.get<uint32_t>(nnear), *nnr = lvl.get<uint32_t>(nnear);
            uint32_t *oadm = lvl.get<uint32_t>(nnear), *onr = lvl.get<uint32_t>(nnear);
            uint32_t *tot = lvl.get<uint32_t>(2);
            const AdmK K = adm_thresholds(sg);
            FFM_LAUNCH(k_expand_count, cdiv(nnear, EXP_W), 32 * EXP_W, 0, s, nearA, nearB, nnear,
                       p->bx[l].first_child, p->by[l].first_child, p->bx[lc].g, p->by[lc].g, K, nadm, nnr);
            scan_u32(nadm, oadm, nnear, tot, lvl, s);
            scan_u32(nnr, onr, nnear, tot + 1, lvl, s);
            uint32_t htot[2];
            FFM_CUDA(cudaMemcpyAsync(htot, tot, sizeof htot, cudaMemcpyDeviceToHost, s));
            FFM_CUDA(cudaStreamSynchronize(s));
            int64_t na = htot[0], nn = htot[1];
            uint32_t *aa = lvl.get<uint32_t>(na), *ab = lvl.get<uint32_t>(na);
            uint32_t *ea = lvl.get<uint32_t>(nn), *eb = lvl.get<uint32_t>(nn);
            FFM_LAUNCH(k_expand_emit, cdiv(nnear, EXP_W), 32 * EXP_W, 0, s, nearA, nearB, nnear,
                       p->bx[l].first_child, p->by[l].first_child, p->bx[lc].g, p->by[lc].g, K, oadm, onr, aa, ab,
                       ea, eb);
            // the previous level's near list is no longer needed
            if (l >= 1) levels[l].release();
            finish_far_level(p, lc, aa, ab, na, lvl, s);
            if (p->far[lc].n_adm > 0) build_tables(p, lc, tj);
            nearA = ea;
            nearB = eb;
            nnear = nn;
            p->info.n_near[lc] = nn;
        }
    }
    int ls = p->l_stop;
    p->info.l_stop = ls;

    // ---- near pairs at the stop level: CSR over all target leaves
    p->n_near = nnear;
    int64_t nleafX = p->bx[ls].nb;
    p->near_off = p->mem.get<uint32_t>(nleafX + 1);
    if (nnear > 0) {
        Csr c = group_by_target(nearA, nearB, nnear, nleafX, p->mem, tmp, s);
        p->near_src = c.b;
        FFM_LAUNCH(k_csr_offsets, cdiv(nleafX + 1, 256), 256, 0, s, c.a, nnear, nleafX, p->near_off);
        // work items: target chunks x bounded source ranges
        p->n_items = build_p2p_items(p, p->p2p_tchunk, p->p2p_smax, p->mem, &p->items, tmp, s);
        unsigned long long *pp = tmp.get<unsigned long long>(1);
        FFM_CUDA(cudaMemsetAsync(pp, 0, sizeof(unsigned long long), s));
        FFM_LAUNCH(k_sum_pair_sizes, cdiv(nnear, 256), 256, 0, s, c.a, c.b, nnear, p->bx[ls].start, p->by[ls].start,
                   pp);
        p->info.p2p_pairs = read_u64(pp, s);
    } else {
        FFM_CUDA(cudaMemsetAsync(p->near_off, 0, sizeof(uint32_t) * (nleafX + 1), s));
    }

    // ---- leaf links and leaf-relative coordinates
    for (int l = 0; l <= ls; ++l) {
        for (BoxLevel *B : {&p->bx[l], &p->by[l]}) {
            BoxLevel &Lf = (B == &p->bx[l]) ? p->bx[ls] : p->by[ls];
            B->first_leaf = p->mem.get<uint32_t>(B->nb + 1);
            FFM_LAUNCH(k_lower_bound, cdiv(B->nb + 1, 256), 256, 0, s, B->fine, B->nb, Lf.fine, Lf.nb, B->first_leaf);
        }
    }
    double dls = std::ldexp(d0, -ls);
    p->epsX = p->mem.get<float4>(nx);
    p->epsY = p->mem.get<float4>(ny);
    p->epsXlo = p->mem.get<float4>(nx);
    p->epsYlo = p->mem.get<float4>(ny);
    if (xdt == FFM_F64)
        launch_leaf_eps<double>(dX, p->permX, p->keyX, p->bx[ls].start, p->bx[ls].nb, nx, p->oX, dls, ls, p->epsX, p->epsXlo, s);
    else
        launch_leaf_eps<float>(dX, p->permX, p->keyX, p->bx[ls].start, p->bx[ls].nb, nx, p->oX, dls, ls, p->epsX, p->epsXlo, s);
    if (ydt == FFM_F64)
        launch_leaf_eps<double>(dY, p->permY, p->keyY, p->by[ls].start, p->by[ls].nb, ny, p->oY, dls, ls, p->epsY, p->epsYlo, s);
    else
        launch_leaf_eps<float>(dY, p->permY, p->keyY, p->by[ls].start, p->by[ls].nb, ny, p->oY, dls, ls, p->epsY, p->epsYlo, s);
    if (w) {
        const void *dw = to_device(w, (wdt == FFM_F64 ? 8 : 4) * (size_t)ny, tmp, s);
        p->wY = p->mem.get<double>(ny);
        if (wdt == FFM_F64)
            FFM_LAUNCH(k_sorted_weights<double>, cdiv(ny, 256), 256, 0, s, (const double *)dw, p->permY, ny, p->wY);
        else
            FFM_LAUNCH(k_sorted_weights<float>, cdiv(ny, 256), 256, 0, s, (const float *)dw, p->permY, ny, p->wY);
    }
    if (p->kind == FFM_LAPLACE_DL) {
        size_t esz = p->normals_dt == FFM_F64 ? 8 : 4;
        const void *dn = to_device(p->normals_in, 3 * esz * (size_t)ny, tmp, s);
        p->nY = p->mem.get<float4>(ny);
        p->nYlo = p->mem.get<float4>(ny);
        if (p->normals_dt == FFM_F64)
            FFM_LAUNCH(k_sorted_normals<double>, cdiv(ny, 256), 256, 0, s, (const double *)dn, p->permY, ny, p->nY,
                       p->nYlo);
        else
            FFM_LAUNCH(k_sorted_normals<float>, cdiv(ny, 256), 256, 0, s, (const float *)dn, p->permY, ny, p->nY,
                       p->nYlo);
    }
    for (int l = 0; l <= ls; ++l)
        if (p->far[l].n_adm > 0) build_octants(p, l, tj);
    if (p->lag_transfer == 3)
        for (int l = 0; l <= ls; ++l) prepare_target_stationary(p, l, s);
    // plane-wave levels whose F steps run as type-3 NUFFTs: FP32 levels with many directions
    // (the NUFFT's cost per box barely depends on nQ, the direct sums' grows with it), all
    // FP32 and compensated-FP32 levels when forced, none when direct sums are forced
    for (int l = 0; l <= ls; ++l) {
        const FarLevel &F = p->far[l];
        if (F.mode != 2 || F.n_adm == 0) continue;
        bool want = p->pw_transform == 2   ? (F.prec == FFM_PREC_F32 || F.prec == FFM_PREC_F32C)
                    : p->pw_transform == 1 ? false
                                           : (F.prec == FFM_PREC_F32 && F.nQ >= NUFFT_MIN_NQ);
        if (want && nufft_possible(p, l)) build_nufft(p, l, tmp, s);
    }
    // the remaining FP32 and compensated-FP32 direct levels: point pieces of their boxes for
    // the tensor-core transforms of several right-hand sides (not with direct sums forced
    // onto the CUDA cores, nor for the NUFFT)
    if (p->pw_transform == 0 || p->pw_transform == 3)
        for (int l = 0; l <= ls; ++l) {
            FarLevel &F = p->far[l];
            if (F.mode != 2 || F.n_adm == 0 || F.nufft || (F.prec != FFM_PREC_F32 && F.prec != FFM_PREC_F32C))
                continue;
            F.pw_chunks = build_chunks(p, F.src, F.n_src, p->by[l].start, &F.n_pw_chunks, tmp, s, PW_TC_FCH);
            F.pw_tchunks = build_chunks(p, F.tgt, F.n_tgt, p->bx[l].start, &F.n_pw_tchunks, tmp, s, PW_TC_BCH);
        }
    FFM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace ffm
