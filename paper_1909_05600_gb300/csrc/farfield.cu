// Far field of one level, computed on the fly from the plan's per-translation tables.
//
// Lagrange levels (Sec. 2.2.2):      u~_b = L_Y(b) (w u)_b ;  v~_a = sum_b T_t(a,b) u~_b ;
//                                    v_a += L_X(a)^T v~_a
// Plane-wave levels (Sec. 2.2.3):    u~_b(q) = sum_{j in b} e^{-ik s_q.(y_j - y0_b)} (w u)_j
//                                    v~_a(q) = sum_b D_t(a,b)(q) u~_b(q)
//                                    v_i    += sum_q e^{ik s_q.(x_i - x0_a)} v~_a(q)
//
// Plane-wave phases are split at the leaf: y - y0_b = (y - c_leaf) + (c_leaf - y0_b).
// The first factor has a small argument (|k s.(y - c_leaf)| <= k sqrt(3) d_leaf / 2) and
// is evaluated per (point, direction) with the FP32 special-function unit; the second
// is a product of tabulated octant factors, one per level between the box and the leaf,
// so that no large phase is ever rounded to FP32.  This only re-associates the sums of
// Sec. 2.2.3 (e^{a+b} = e^a e^b); the F matrices are still applied exactly, without
// NUFFT.
#include <type_traits>

#include "ffm_internal.cuh"
#include "dfloat.cuh"

namespace ffm {

// ----------------------------------------------------------- helpers

struct Cheb {
    float t[R1MAX];  // Chebyshev nodes cos((2a+1) pi / (2 r1))
    float w[R1MAX];  // 1 / prod_{b != a} (t_a - t_b)
    int r1;
};

static Cheb make_cheb(int r1) {
    Cheb c{};
    c.r1 = r1;
    double t[R1MAX];
    for (int a = 0; a < r1; ++a) t[a] = std::cos((2.0 * a + 1.0) * PI / (2.0 * r1));
    for (int a = 0; a < r1; ++a) {
        double d = 1.0;
        for (int b = 0; b < r1; ++b)
            if (b != a) d *= t[a] - t[b];
        c.t[a] = (float)t[a];
        c.w[a] = (float)(1.0 / d);
    }
    return c;
}

// 1-D Lagrange basis at xi via prefix / suffix products.
__device__ __forceinline__ void lag1d(const Cheb &c, float xi, float *out) {
    float pre[R1MAX], suf[R1MAX];
    float acc = 1.f;
#pragma unroll
    for (int a = 0; a < R1MAX; ++a) {
        if (a < c.r1) {
            pre[a] = acc;
            acc *= xi - c.t[a];
        }
    }
    acc = 1.f;
#pragma unroll
    for (int a = R1MAX - 1; a >= 0; --a) {
        if (a < c.r1) {
            suf[a] = acc;
            acc *= xi - c.t[a];
        }
    }
#pragma unroll
    for (int a = 0; a < R1MAX; ++a)
        if (a < c.r1) out[a] = c.w[a] * pre[a] * suf[a];
}

// Offset of a leaf centre from the centre of its ancestor at level l, per axis:
// d_ls * ((g_leaf + 1/2) - (g_box + 1/2) 2^(ls-l)).
__device__ __forceinline__ float3 leaf_offset(int4 gl, int4 gb, int shift, float dls) {
    float half = 0.5f * (float)(1 << shift);
    return make_float3(dls * ((float)(gl.x - (gb.x << shift)) + 0.5f - half),
                       dls * ((float)(gl.y - (gb.y << shift)) + 0.5f - half),
                       dls * ((float)(gl.z - (gb.z << shift)) + 0.5f - half));
}

template <bool CPLX>
struct QT;
template <>
struct QT<false> {
    typedef float T;
};
template <>
struct QT<true> {
    typedef float2 T;
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

struct LevelArgs {
    // boxes of the level and the leaves
    const uint32_t *box_start;
    const int4 *box_g;
    const uint32_t *box_leaf;   // first leaf of each box (nb + 1)
    const uint32_t *leaf_start;
    const int4 *leaf_g;
    const float4 *eps;
    int shift;  // l_stop - l
    float dls;  // leaf edge
    float inv_half_dl;  // 2 / d_l
};

// ========================================================= Lagrange kernels

constexpr int LAG_T = 256;

// Source step of a Lagrange level (L_Y u of eq. 8): u~_b(abc) = sum_{j in b} L_a(x_j) L_b(y_j) L_c(z_j) q_j.
// One block per chunk of at most LAG_CHUNK points of a box; each thread owns up to two
// control nodes.  A box split into several chunks adds its partial sums with atomics
// (u~ is zeroed first); a single-chunk box stores them.
template <bool CPLX, int R1>
__global__ void __launch_bounds__(LAG_T) k_lag_anterp(LevelArgs A, const uint2 *__restrict__ chunks, Cheb cb,
                                                      const typename QT<CPLX>::T *__restrict__ q, int64_t ny,
                                                      int nrhs, typename QT<CPLX>::T *__restrict__ ut) {
    typedef typename QT<CPLX>::T Q;
    constexpr int r = R1 * R1 * R1;
    // per staged point: x weights (times q for real densities), y and z weights
    __shared__ float sl[LAG_T][3 * R1 + 1];
    __shared__ Q sq[CPLX ? LAG_T : 1];
    uint2 ck = chunks[blockIdx.x];
    int b = (int)ck.x, m = blockIdx.y;
    uint32_t s0 = ck.y, bend = A.box_start[b + 1];
    uint32_t s1 = min(bend, s0 + (uint32_t)LAG_CHUNK);
    bool sole = s0 == A.box_start[b] && s1 == bend;
    int4 gb = A.box_g[b];
    float accr[2] = {0.f, 0.f}, acci[2] = {0.f, 0.f};
    for (uint32_t base = s0; base < s1; base += LAG_T) {
        uint32_t j = base + threadIdx.x;
        if (j < s1) {
            float4 e = A.eps[j];
            int4 gl = A.leaf_g[__float_as_uint(e.w)];
            float3 o = leaf_offset(gl, gb, A.shift, A.dls);
            float lx[R1MAX], ly[R1MAX], lz[R1MAX];
            lag1d(cb, (o.x + e.x) * A.inv_half_dl, lx);
            lag1d(cb, (o.y + e.y) * A.inv_half_dl, ly);
            lag1d(cb, (o.z + e.z) * A.inv_half_dl, lz);
            Q w = q[(int64_t)m * ny + j];
#pragma unroll
            for (int a = 0; a < R1; ++a) {
                if constexpr (CPLX)
                    sl[threadIdx.x][a] = lx[a];
                else
                    sl[threadIdx.x][a] = lx[a] * w;
                sl[threadIdx.x][R1 + a] = ly[a];
                sl[threadIdx.x][2 * R1 + a] = lz[a];
            }
            if constexpr (CPLX) sq[threadIdx.x] = w;
        }
        __syncthreads();
        int cnt = (int)min((uint32_t)LAG_T, s1 - base);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int a = threadIdx.x + h * LAG_T;
            if (a < r) {
                int ia = a / (R1 * R1), ib = (a / R1) % R1, ic = a % R1;
                for (int jj = 0; jj < cnt; ++jj) {
                    float L = sl[jj][ia] * sl[jj][R1 + ib];
                    if constexpr (CPLX) {
                        L *= sl[jj][2 * R1 + ic];
                        accr[h] = fmaf(L, sq[jj].x, accr[h]);
                        acci[h] = fmaf(L, sq[jj].y, acci[h]);
                    } else {
                        accr[h] = fmaf(L, sl[jj][2 * R1 + ic], accr[h]);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int a = threadIdx.x + h * LAG_T;
        if (a < r) {
            size_t o = ((size_t)b * nrhs + m) * r + a;
            if constexpr (CPLX) {
                if (sole) {
                    ut[o] = make_float2(accr[h], acci[h]);
                } else {
                    atomicAdd(&ut[o].x, accr[h]);
                    atomicAdd(&ut[o].y, acci[h]);
                }
            } else {
                if (sole)
                    ut[o] = accr[h];
                else
                    atomicAdd(&ut[o], accr[h]);
            }
        }
    }
}

// Source step of a double-layer Lagrange level.  The kernel n_y . grad_y G is the sum over
// the axes d of n_d dG/dy_d(x - y); each component kernel is interpolated on its own, so
// the source step gives three coefficient blocks u~_b[d r + abc] = sum_j q_{j,d} L_abc(y_j)
// with q_j = w_j u_j n_j, and the transfer multiplies them by the stacked operator
// [T^1 T^2 T^3] (K = 3 r).  Chunked like k_lag_anterp.
template <int R1>
__global__ void __launch_bounds__(LAG_T) k_lag_anterp_dl(LevelArgs A, const uint2 *__restrict__ chunks, Cheb cb,
                                                         const float4 *__restrict__ q, int64_t ny, int nrhs,
                                                         float *__restrict__ ut) {
    constexpr int r = R1 * R1 * R1;
    __shared__ float sl[LAG_T][3 * R1 + 4];  // x, y, z basis values, then q
    uint2 ck = chunks[blockIdx.x];
    int b = (int)ck.x, m = blockIdx.y;
    uint32_t s0 = ck.y, bend = A.box_start[b + 1];
    uint32_t s1 = min(bend, s0 + (uint32_t)LAG_CHUNK);
    bool sole = s0 == A.box_start[b] && s1 == bend;
    int4 gb = A.box_g[b];
    float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    for (uint32_t base = s0; base < s1; base += LAG_T) {
        uint32_t j = base + threadIdx.x;
        if (j < s1) {
            float4 e = A.eps[j];
            int4 gl = A.leaf_g[__float_as_uint(e.w)];
            float3 o = leaf_offset(gl, gb, A.shift, A.dls);
            lag1d(cb, (o.x + e.x) * A.inv_half_dl, &sl[threadIdx.x][0]);
            lag1d(cb, (o.y + e.y) * A.inv_half_dl, &sl[threadIdx.x][R1]);
            lag1d(cb, (o.z + e.z) * A.inv_half_dl, &sl[threadIdx.x][2 * R1]);
            float4 qj = q[2 * ((int64_t)m * ny + j)];  // hi part (the far field is smooth)
            sl[threadIdx.x][3 * R1] = qj.x;
            sl[threadIdx.x][3 * R1 + 1] = qj.y;
            sl[threadIdx.x][3 * R1 + 2] = qj.z;
        }
        __syncthreads();
        int cnt = (int)min((uint32_t)LAG_T, s1 - base);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int a = threadIdx.x + h * LAG_T;
            if (a < r) {
                int ia = a / (R1 * R1), ib = (a / R1) % R1, ic = a % R1;
                for (int jj = 0; jj < cnt; ++jj) {
                    const float *v = sl[jj];
                    float L = v[ia] * v[R1 + ib] * v[2 * R1 + ic];
                    acc[h][0] = fmaf(L, v[3 * R1], acc[h][0]);
                    acc[h][1] = fmaf(L, v[3 * R1 + 1], acc[h][1]);
                    acc[h][2] = fmaf(L, v[3 * R1 + 2], acc[h][2]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int a = threadIdx.x + h * LAG_T;
        if (a < r) {
            size_t o = ((size_t)b * nrhs + m) * 3 * r + a;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (sole)
                    ut[o + (size_t)d * r] = acc[h][d];
                else
                    atomicAdd(&ut[o + (size_t)d * r], acc[h][d]);
            }
        }
    }
}

// Transfer as one GEMM per translation (Sec. 2.2.2, T depends only on the box offset):
// C(i, p) = sum_j T_t(i, j) u~_{src(p)}(j) for the pairs p of a column tile of translation t,
// then v~_{tgt(p)}(i) += C(i, p).  A tile is BM control nodes x BN pairs; K runs over the r
// source nodes in steps of BK.  Source columns are gathered from u~ by pair; the result is
// scatter-added with FP32 atomics (a target box receives from up to 316-665 translations).
constexpr int LG_BM = 64, LG_BK = 16, LG_T = 256;
template <bool CPLX>
__global__ void __launch_bounds__(LG_T) k_lag_gemm(const uint32_t *__restrict__ tile_t,
                                                   const uint32_t *__restrict__ tile_p0,
                                                   const uint32_t *__restrict__ bt_off,
                                                   const uint32_t *__restrict__ bt_src,
                                                   const uint32_t *__restrict__ bt_tgt, const float *__restrict__ T,
                                                   int r, int rk, int nrhs, const typename QT<CPLX>::T *__restrict__ ut,
                                                   typename QT<CPLX>::T *__restrict__ vt) {
    // rk: K extent (rk = r, or 3 r for the double layer's stacked component kernels)
    typedef typename QT<CPLX>::T Q;
    constexpr int BN = LAG_GEMM_BN;
    __shared__ Q As[LG_BK][LG_BM];
    __shared__ Q Bs[LG_BK][BN];
    __shared__ uint32_t s_src[BN], s_tgt[BN];
    int t = tile_t[blockIdx.x];
    uint32_t p0 = tile_p0[blockIdx.x];
    int np = (int)min((uint32_t)BN, bt_off[t + 1] - p0);
    int i0 = blockIdx.y * LG_BM, m = blockIdx.z;
    int tid = threadIdx.x;
    if (tid < BN) {
        s_src[tid] = tid < np ? bt_src[p0 + tid] : 0u;
        s_tgt[tid] = tid < np ? bt_tgt[p0 + tid] : 0u;
    }
    int ti = tid % 16, tp = tid / 16;  // 4 rows x 2 columns per thread
    float cr[4][2], ci[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) cr[a][b] = ci[a][b] = 0.f;
    const Q *Tt = reinterpret_cast<const Q *>(T) + (size_t)t * r * rk;
    __syncthreads();
    for (int j0 = 0; j0 < rk; j0 += LG_BK) {
        for (int e = tid; e < LG_BK * LG_BM; e += LG_T) {
            int jj = e / LG_BM, ii = e % LG_BM;
            int j = j0 + jj, i = i0 + ii;
            Q v;
            if constexpr (CPLX)
                v = (j < rk && i < r) ? Tt[(size_t)i * rk + j] : make_float2(0.f, 0.f);
            else
                v = (j < rk && i < r) ? Tt[(size_t)i * rk + j] : 0.f;
            As[jj][ii] = v;
        }
        for (int e = tid; e < LG_BK * BN; e += LG_T) {
            int jj = e % LG_BK, pp = e / LG_BK;
            int j = j0 + jj;
            Q v;
            if constexpr (CPLX)
                v = (j < rk && pp < np) ? ut[((size_t)s_src[pp] * nrhs + m) * rk + j] : make_float2(0.f, 0.f);
            else
                v = (j < rk && pp < np) ? ut[((size_t)s_src[pp] * nrhs + m) * rk + j] : 0.f;
            Bs[jj][pp] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < LG_BK; ++kk) {
            Q a[4], b[2];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = As[kk][ti * 4 + x];
#pragma unroll
            for (int y = 0; y < 2; ++y) b[y] = Bs[kk][tp * 2 + y];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 2; ++y) {
                    if constexpr (CPLX) {
                        cr[x][y] = fmaf(a[x].x, b[y].x, fmaf(-a[x].y, b[y].y, cr[x][y]));
                        ci[x][y] = fmaf(a[x].x, b[y].y, fmaf(a[x].y, b[y].x, ci[x][y]));
                    } else {
                        cr[x][y] = fmaf(a[x], b[y], cr[x][y]);
                    }
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int y = 0; y < 2; ++y) {
        int pp = tp * 2 + y;
        if (pp >= np) continue;
        Q *dst = vt + ((size_t)s_tgt[pp] * nrhs + m) * r;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            int i = i0 + ti * 4 + x;
            if (i >= r) continue;
            if constexpr (CPLX) {
                atomicAdd(&dst[i].x, cr[x][y]);
                atomicAdd(&dst[i].y, ci[x][y]);
            } else {
                atomicAdd(&dst[i], cr[x][y]);
            }
        }
    }
}

// ---- tensor-core transfer (5th-generation tensor cores, tcgen05, TF32 with hi/lo split)
//
// D(p, i) = sum_j u~_{src(p)}(j) T_t(i, j) for 128 pairs p of translation t (one MMA
// half-tile): A = gathered u~ columns (M = 128 pairs, K = r, K-major), B = rows of T_t (N
// = a row block of at most 224, a multiple of 16, K-major), accumulator in TMEM (lane = pair,
// column = i).  Each operand is
// split into hi + lo TF32 parts (hi: low 13 mantissa bits cleared, lo = x - hi exactly), and
// D += A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32, about 2^-21 relative per product.
// Operands use the no-swizzle K-major layout of 8-row x 16-byte core matrices: core matrix
// (g, c) at byte (g * KT/4 + c) * 128, leading-dimension (K) stride 128 B, 8-row-group stride
// KT/4 * 128 B.  One thread issues the MMAs; completion is tracked by an mbarrier with a
// bounded wait that raises a device error flag instead of hanging.
constexpr int TC_M = 128;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int KT) {
    return (uint32_t)((((row >> 3) * (KT >> 2) + (k >> 2)) << 7) + ((row & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// bulk copy global -> shared, completion counted in bytes on an mbarrier
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// Bounded wait for the completion of phase `parity` of an mbarrier: at most `tries`
// try_wait attempts (none for tries <= 0); false if it gave up.
// With `abort` (the launch's device error flag), the wait also gives up once another CTA has
// raised the flag (checked every 1024 attempts), so one failure does not make every later
// CTA spend its whole limit.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int tries, const int *abort = nullptr) {
    uint32_t done = 0;
    for (int it = 0; it < tries && !done; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(smem_addr(bar)), "r"(parity));
        if (!done && abort && (it & 1023) == 1023 && *reinterpret_cast<const volatile int *>(abort)) break;
    }
    return done != 0;
}

// After a wait has given up, a kernel still waits for the tensor-core operations it has
// already committed before it releases TMEM and exits (they read its shared memory and
// write its TMEM columns); that wait is bounded too, by this larger count.
constexpr int DRAIN_TRIES = 1 << 28;

__device__ __forceinline__ void store_split(float *hi, float *lo, uint32_t o, float4 x) {
    float4 h, l;
    tf32_split(x.x, h.x, l.x);
    tf32_split(x.y, h.y, l.y);
    tf32_split(x.z, h.z, l.z);
    tf32_split(x.w, h.w, l.w);
    *reinterpret_cast<float4 *>(hi + o) = h;
    *reinterpret_cast<float4 *>(lo + o) = l;
}

// Tiles of up to 256 pairs of one translation: two 128-pair halves, each with its own TMEM
// accumulator, share every chunk of T_t.  The K loop runs over chunks of KT source nodes.
// Warps 1-7 copy each chunk's rows (u~ of the pairs' source boxes, and T_t) as raw FP32
// into an NR-deep ring with cp.async, each thread always the same 16-byte segments; once its
// own segments have landed a thread splits them into TF32 hi and lo parts and stores them
// into the NO-deep ring of MMA operands (K-major core matrices), then arrives on that
// stage's "full" mbarrier.  One thread of warp 0 waits on "full", issues the MMAs
// (hi*hi + hi*lo + lo*hi for each half) and commits them to the stage's "empty" mbarrier,
// which the copying threads wait on before they overwrite the stage.  Operands are padded
// (rows of rkp floats, T_t with npad rows), so every copy is a whole, aligned segment.
constexpr int TC_P = 256;  // pairs per tensor-core tile

template <int KT, int NR, int NO>
__global__ void __launch_bounds__(256) k_lag_gemm_tc(const uint32_t *__restrict__ tile_t,
                                                     const uint32_t *__restrict__ tile_p0,
                                                     const uint32_t *__restrict__ bt_off,
                                                     const uint32_t *__restrict__ bt_src,
                                                     const uint32_t *__restrict__ bt_tgt, const float *__restrict__ Tp,
                                                     int64_t tstride, int ostride, int nout, int rkp, int npad,
                                                     int tcols, int nrhs,
                                                     const float *__restrict__ up, float *__restrict__ vt,
                                                     int *__restrict__ err, int tries) {
    constexpr int C4 = KT / 4;  // 16-byte segments per row and chunk
    constexpr int NP = 224;     // copying threads (warps 1-7)
    extern __shared__ __align__(1024) unsigned char smem[];
    const int op_f = 2 * TC_P * KT + 2 * npad * KT;  // floats per operand stage: A hi, A lo, B hi, B lo
    const int raw_f = (TC_P + npad) * KT;            // floats per raw stage: A rows, then B rows
    float *op0 = reinterpret_cast<float *>(smem);
    float *raw0 = op0 + (size_t)NO * op_f;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_full[NO], s_empty[NO];
    __shared__ uint32_t s_src[TC_P], s_tgt[TC_P];
    __shared__ int s_bad;
    int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int t = tile_t[blockIdx.x], m = blockIdx.y;
    uint32_t p0 = tile_p0[blockIdx.x];
    int np = (int)min((uint32_t)TC_P, bt_off[t + 1] - p0);
    const int nh = np > 128 ? 2 : 1;  // halves with pairs
    {
        // rows past the tile's pairs repeat its first pair; their TMEM lanes are not read
        s_src[tid] = bt_src[p0 + (tid < np ? tid : 0)];
        s_tgt[tid] = tid < np ? bt_tgt[p0 + tid] : 0u;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(2 * tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_bad = 0;
        for (int i = 0; i < NO; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&s_full[i])), "r"(NP));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_empty[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t tmem = s_tmem;
    const float *Tt = Tp + (size_t)t * tstride;
    const uint32_t lbo = 128, sbo = (KT / 4) * 128;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const int nk = rkp / KT;
    const int nseg = (TC_P + npad) * C4;
    bool ok = true;
    if (warp >= 1) {
        // ---- copying warps: segments e = pt, pt + NP, ... of every chunk
        const int pt = tid - 32;
        auto copy_chunk = [&](int kc) {
            float *raw = raw0 + (size_t)(kc % NR) * raw_f;
            const int k0 = kc * KT;
            for (int e = pt; e < nseg; e += NP) {
                int row = e / C4, c = e - row * C4;
                const float *g = row < TC_P ? up + ((size_t)s_src[row] * nrhs + m) * rkp + k0 + 4 * c
                                            : Tt + (size_t)(row - TC_P) * rkp + k0 + 4 * c;
                cp_async16(raw + row * KT + 4 * c, g);
            }
        };
        for (int kc = 0; kc < NR - 1; ++kc) {
            if (kc < nk) copy_chunk(kc);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        for (int kn = 0; kn < nk; ++kn) {
            if (kn + NR - 1 < nk) copy_chunk(kn + NR - 1);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group %0;" ::"n"(NR - 1) : "memory");  // chunk kn's segments landed
            const int b = kn % NO;
            // MMAs of kn - NO done; a thread that gives up stops copying (its copies in
            // flight are awaited below)
            if (kn >= NO && !mbar_wait(&s_empty[b], (uint32_t)((kn / NO - 1) & 1), tries, err)) {
                ok = false;
                break;
            }
            const float *raw = raw0 + (size_t)(kn % NR) * raw_f;
            float *sAh = op0 + (size_t)b * op_f, *sAl = sAh + TC_P * KT, *sBh = sAl + TC_P * KT,
                  *sBl = sBh + npad * KT;
            for (int e = pt; e < nseg; e += NP) {
                int row = e / C4, c = e - row * C4;
                float4 x = *reinterpret_cast<const float4 *>(raw + row * KT + 4 * c);
                if (row < TC_P)
                    store_split(sAh, sAl, kmajor_off(row, 4 * c, KT) >> 2, x);
                else
                    store_split(sBh, sBl, kmajor_off(row - TC_P, 4 * c, KT) >> 2, x);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&s_full[b])) : "memory");
        }
    } else if (lane == 0) {
        // ---- MMA thread
        int issued = 0;  // chunks whose MMAs were committed
        for (int kc = 0; kc < nk; ++kc) {
            const int b = kc % NO;
            if (!mbar_wait(&s_full[b], (uint32_t)((kc / NO) & 1), tries, err)) {
                ok = false;  // operands not ready: issue nothing more
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float *sAh = op0 + (size_t)b * op_f, *sAl = sAh + TC_P * KT, *sBh = sAl + TC_P * KT,
                  *sBl = sBh + npad * KT;
            for (int h = 0; h < nh; ++h) {
                uint32_t d = tmem + (uint32_t)(h * tcols);
                uint32_t ao = smem_addr(sAh + h * 128 * KT), alo = smem_addr(sAl + h * 128 * KT);
#pragma unroll
                for (int ks = 0; ks < KT / 8; ++ks) {
                    uint64_t ah = umma_desc(ao + ks * 256, lbo, sbo);
                    uint64_t al = umma_desc(alo + ks * 256, lbo, sbo);
                    uint64_t bh = umma_desc(smem_addr(sBh) + ks * 256, lbo, sbo);
                    uint64_t bl = umma_desc(smem_addr(sBl) + ks * 256, lbo, sbo);
                    uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                        "l"(ah), "l"(bh), "r"(idesc), "r"(acc0));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(d), "l"(ah),
                                 "l"(bl), "r"(idesc));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(d), "l"(al),
                                 "l"(bh), "r"(idesc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&s_empty[b]))
                         : "memory");
            issued = kc + 1;
        }
        // the last committed chunk's MMAs complete after all earlier ones; after a give-up
        // this wait (bounded by DRAIN_TRIES) keeps TMEM and the operand ring owned until
        // every committed MMA has finished
        if (issued > 0) {
            uint64_t *last = &s_empty[(issued - 1) % NO];
            const uint32_t par = (uint32_t)(((issued - 1) / NO) & 1);
            if (!ok || !mbar_wait(last, par, tries, err)) {
                ok = false;
                mbar_wait(last, par, DRAIN_TRIES);
            }
        }
    }
    if (warp >= 1) asm volatile("cp.async.wait_all;" ::: "memory");
    if (!ok) s_bad = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    ok = s_bad == 0;
    if (!ok && tid == 0) atomicOr(err, 1);
    // epilogue (skipped after a give-up: the accumulators are incomplete): warp w reads TMEM
    // lanes 32 (w % 4) .. + 31 of half w / 4; columns = target nodes
    const int h = warp >> 2, quarter = warp & 3;
    const int p = h * 128 + quarter * 32 + lane;
    if (ok && h < nh) {
        float *dst = vt + ((size_t)s_tgt[p] * nrhs + m) * ostride;
        for (int c0 = 0; c0 < npad; c0 += 8) {
            uint32_t v[8];
            uint32_t addr = tmem + (uint32_t)(h * tcols) + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                         : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (p < np) {
                if ((ostride & 3) == 0 && c0 + 8 <= nout) {
                    atomicAdd(reinterpret_cast<float4 *>(dst + c0),
                              make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]),
                                          __uint_as_float(v[3])));
                    atomicAdd(reinterpret_cast<float4 *>(dst + c0 + 4),
                              make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]), __uint_as_float(v[6]),
                                          __uint_as_float(v[7])));
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (c0 + q < nout) atomicAdd(dst + c0 + q, __uint_as_float(v[q]));
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * tcols));
}

// nmat row-major matrices (rows x cols) copied with rows_pad rows of cols_pad floats each
// (padding zero); with lo != nullptr the TF32 hi part goes to out and the lo part to lo.
__global__ void k_split_pad(const float *__restrict__ src, int64_t nmat, int rows, int cols, int rows_pad,
                            int cols_pad, float *__restrict__ out, float *__restrict__ lo) {
    int64_t n = nmat * rows_pad * (int64_t)cols_pad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t mat = i / ((int64_t)rows_pad * cols_pad);
        int rem = (int)(i - mat * rows_pad * (int64_t)cols_pad);
        int row = rem / cols_pad, col = rem - row * cols_pad;
        float x = row < rows && col < cols ? src[(mat * rows + row) * (int64_t)cols + col] : 0.f;
        if (lo) {
            float h, l;
            tf32_split(x, h, l);
            out[i] = h;
            lo[i] = l;
        } else {
            out[i] = x;
        }
    }
}

// ---- target-stationary tensor-core transfer (r <= 64)
//
// A CTA owns TS_M = 128 consecutive target boxes of the level (TMEM lane = box) and runs
// over every translation t present among their admissible pairs, in increasing order
// (partners are sorted by translation within each target, so a per-row cursor finds the
// row's source box for t, or none).  For each t it multiplies the source rows u~_b (zero
// rows for boxes without a partner at t) by T_t (N = 64 target nodes, K = 64 source nodes,
// zero padded beyond r) and accumulates D(a, i) = sum_t sum_j u~_{b(a,t)}(j) T_t(i, j) in
// TMEM; each target's v~ is written once, with no atomics.  TF32 hi/lo split with three
// MMAs per K step (hi hi + hi lo + lo hi), FP32 accumulation.
//
// Operands.  The A operand (the gathered source rows) lives in tensor memory: the MMAs read
// it from TMEM, so shared memory only carries T_t (the B operand), and the operand reads of
// the tensor cores from shared memory drop to a third.  A step is one translation (K = 64
// source nodes, 24 MMAs).  Warps 1-8 produce; the two producers of a target row each own 32
// of the row's 64 values.  A producer loads its values of the row's source (zero where the
// row has no partner) from global memory into registers TS_P steps ahead, splits them into
// TF32 hi and lo parts and writes them into one of TS_NA TMEM operand stages (tcgen05.st),
// then arrives on that stage's "A full" mbarrier.  The first producer also starts a bulk copy
// of T_t's pre-split image (32 KB) into one of TS_NB shared stages, TS_DB steps ahead,
// counted in bytes on that stage's "B full" mbarrier.  One thread of
// warp 0 waits on both, issues the step's 24 MMAs and commits them to the B stage's "empty"
// mbarrier; the producers wait on it (TS_NA steps later) before they reuse the A and B
// stages.  Each barrier round trip thus serves 24 MMAs.
//
// Accumulation.  One long tcgen05 accumulation loses accuracy, so the tile alternates
// between two TMEM accumulators (64 columns each) every TS_DRAIN translations; the producers
// add each finished accumulator into FP32 registers (tcgen05.ld) while the tensor cores fill
// the other one, and the MMA thread waits for that drain before it reuses the accumulator.
// Every wait is bounded; a give-up raises the device error flag, the CTA then waits for its
// copies and committed MMAs, skips its results and frees TMEM.
constexpr int TS_M = 128;
constexpr int TS_K = 64;              // source nodes (K) per step: one translation
constexpr int TS_BH = 64 * 32;        // floats per B hi or lo block of one half of K
constexpr int TS_BST = 4 * TS_BH;     // floats per B stage: T_t's whole image (32 KB)
constexpr int TS_NA = 3;              // A stages (tensor memory); producers run TS_NA steps ahead
constexpr int TS_DB = 2;              // steps the copies of T_t's image run ahead
constexpr int TS_NB = TS_NA + TS_DB;  // B stages (shared memory)
constexpr int TS_P = 2;               // steps the source loads run ahead (registers)
constexpr int TS_MAXT = 4096;         // translation codes lie in a 16^3 range
constexpr int TS_DRAIN = 8;           // translations per TMEM accumulator fill
constexpr int TS_NP = 2 * TS_M;       // producer threads (warps 1-8)
constexpr int TS_TCOLS = 512;         // TMEM: 2 accumulators x 64 columns, TS_NA A stages x 128 (hi, lo)
constexpr size_t TS_SMEM = sizeof(float) * (size_t)TS_NB * TS_BST;

// 16 values of one lane into consecutive TMEM columns of the warp's lanes
__device__ __forceinline__ void tmem_st16(uint32_t ta, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(ta),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

// eight floats from a 32-byte aligned global address, one 256-bit load through the read-only path
__device__ __forceinline__ void ldg8(const float *p, float4 &a, float4 &b) {
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

// 8 values of one lane into consecutive TMEM columns of the warp's lanes
__device__ __forceinline__ void tmem_st8(uint32_t ta, const uint32_t (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(ta), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}

// u holds rows of 64 floats (r <= 64, zero padded): row (b, m) at ((b nrhs + m) 64).
__global__ void __launch_bounds__(TS_NP + 32, 1) k_lag_gemm_ts(const uint32_t *__restrict__ tgt, int64_t n_tgt,
                                                              const uint32_t *__restrict__ adm_off,
                                                              const uint32_t *__restrict__ adm_src,
                                                              const uint32_t *__restrict__ adm_t, int n_trans,
                                                              const float *__restrict__ Tsp, int r, int nrhs,
                                                              const float *__restrict__ u, float *__restrict__ vt,
                                                              int *__restrict__ err, int tries) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float *bring = reinterpret_cast<float *>(smem);
    __shared__ uint32_t s_bits[TS_MAXT / 32];
    __shared__ uint16_t s_tl[TS_MAXT];  // the translations present, in increasing order
    __shared__ uint32_t s_wpre[TS_MAXT / 32 + 1];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bfull[TS_NB], s_empty[TS_NB], s_afull[TS_NA], s_drained;
    __shared__ int s_bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = blockIdx.y;
    const int64_t x0 = (int64_t)blockIdx.x * TS_M;
    const int nw = (n_trans + 31) / 32;
    for (int w = tid; w < TS_MAXT / 32; w += blockDim.x) s_bits[w] = 0u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(TS_TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_bad = 0;
        for (int i = 0; i < TS_NB; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_empty[i])));
        }
        for (int i = 0; i < TS_NA; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&s_afull[i])), "r"(TS_NP));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&s_drained)), "r"(TS_NP));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    // producers: warp w (1-8) holds TMEM lanes 32 (w % 4) .. + 31, one target row per lane,
    // and values 32 qh .. 32 qh + 31 of each step
    const bool prod = warp >= 1;
    const int dq = warp & 3, qh = (warp - 1) >> 2, row = dq * 32 + lane;
    const int64_t x = x0 + row;
    const bool has = prod && x < n_tgt;
    uint32_t cur = has ? adm_off[x] : 0u, end = has ? adm_off[x + 1] : 0u;
    if (has && qh == 0)
        for (uint32_t e = cur; e < end; ++e) {
            uint32_t t = adm_t[e];
            atomicOr(&s_bits[t >> 5], 1u << (t & 31));
        }
    __syncthreads();
    // list of the translations present: word counts, their prefix, then the set bits in order
    if (tid < TS_MAXT / 32) s_wpre[tid + 1] = __popc(s_bits[tid]);
    if (tid == 0) s_wpre[0] = 0u;
    __syncthreads();
    if (tid == 0)
        for (int w = 1; w <= TS_MAXT / 32; ++w) s_wpre[w] += s_wpre[w - 1];
    __syncthreads();
    if (tid < nw) {
        uint32_t bits = s_bits[tid], o = s_wpre[tid];
        while (bits) {
            s_tl[o++] = (uint16_t)(tid * 32 + __ffs(bits) - 1);
            bits &= bits - 1;
        }
    }
    __syncthreads();
    const int nsteps = (int)s_wpre[TS_MAXT / 32];
    bool ok = true;
    if (prod) {
        const int p = tid - 32;
        float sum[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) sum[c] = 0.f;
        int drained = 0;  // accumulator fills added into sum (columns 32 qh .. + 31)
        auto drain = [&](int k) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = tmem + (uint32_t)((k & 1) * 64 + qh * 32) + ((uint32_t)(dq * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 8) {
                uint32_t v[8];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                               "=r"(v[7])
                             : "r"(base + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 8; ++q) sum[c0 + q] += __uint_as_float(v[q]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&s_drained)) : "memory");
        };
        // T_t's image of step sp into B stage sp % TS_NB: one bulk copy (32 KB) by the first
        // producer, counted in bytes on the stage's "B full" barrier
        int last_b = -1;
        auto copy_b = [&](int sp) {
            if (p != 0 || sp >= nsteps) return;
            uint64_t *bar = &s_bfull[sp % TS_NB];
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                         "r"((uint32_t)(TS_BST * sizeof(float)))
                         : "memory");
            bulk_g2s(bring + (size_t)(sp % TS_NB) * TS_BST, Tsp + (size_t)s_tl[sp] * TS_BST,
                     (uint32_t)(TS_BST * sizeof(float)), bar);
            last_b = sp;
        };
        // this row's source values of step sp (zero without a partner), into registers.  The
        // row's next two partners (translation, source) are held in registers and the one after
        // is loaded as one is used, so the source row's address never waits on a list load.
        uint32_t t0 = 0xffffffffu, b0 = 0u, t1 = 0xffffffffu, b1 = 0u;
        if (cur < end) {
            t0 = adm_t[cur];
            b0 = adm_src[cur];
        }
        if (cur + 1 < end) {
            t1 = adm_t[cur + 1];
            b1 = adm_src[cur + 1];
        }
        float4 ring[TS_P][8];
        auto load_a = [&](int sp, float4 *dst) {
            bool use = false;
            uint32_t src = 0u;
            if (sp < nsteps && t0 == (uint32_t)s_tl[sp]) {
                use = true;
                src = b0;
                t0 = t1;
                b0 = b1;
                ++cur;
                t1 = 0xffffffffu;
                if (cur + 1 < end) {
                    t1 = adm_t[cur + 1];
                    b1 = adm_src[cur + 1];
                }
            }
            // 256-bit loads: half the load instructions (and L1 wavefronts) of 128-bit ones
            const float *g = u + ((size_t)src * nrhs + m) * 64 + qh * 32;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (use) {
                    ldg8(g + 8 * c, dst[2 * c], dst[2 * c + 1]);
                } else {
                    dst[2 * c] = make_float4(0.f, 0.f, 0.f, 0.f);
                    dst[2 * c + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        };
#pragma unroll
        for (int k = 0; k < TS_P; ++k) load_a(k, ring[k]);
        for (int sp = 0; sp < TS_DB; ++sp) copy_b(sp);
        for (int s0 = 0; s0 < nsteps && ok; s0 += TS_P) {
#pragma unroll
            for (int k = 0; k < TS_P; ++k) {
                const int s = s0 + k;
                // (no break in this loop: it is unrolled so that the ring slot k is static)
                if (s >= nsteps || !ok) continue;
                if (s >= TS_NA) {
                    // the MMAs of step s - TS_NA are done: its A and B stages are free.  A fill k
                    // is drained once the first step of fill k + 1 is done: then the fill is
                    // final, and the MMA thread has passed its wait for the drain of fill k - 1,
                    // so the drain barrier is never two phases ahead of that wait (a give-up
                    // is made warp-uniform: the drains are warp-wide TMEM loads)
                    const int sb = s - TS_NA;
                    bool w_ok = mbar_wait(&s_empty[sb % TS_NB], (uint32_t)((sb / TS_NB) & 1), tries, err);
                    if (!__all_sync(0xffffffffu, w_ok)) {
                        ok = false;
                        continue;
                    }
                    const int done = sb / TS_DRAIN;
                    while (drained < done) drain(drained++);
                }
                // split into TF32 hi and lo and write A stage s % TS_NA: columns 128 + 128 (s % TS_NA)
                // + 32 qh (hi) and + 64 (lo), lane = row
                const uint32_t ta =
                    tmem + (uint32_t)(128 + (s % TS_NA) * 128 + qh * 32) + ((uint32_t)(dq * 32) << 16);
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {  // 16 values at a time: fewer live registers
                    uint32_t hv[16], lv[16];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float4 f4 = ring[k][4 * hh + c];
                        const float v4[4] = {f4.x, f4.y, f4.z, f4.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            float h, l;
                            tf32_split(v4[q], h, l);
                            hv[4 * c + q] = __float_as_uint(h);
                            lv[4 * c + q] = __float_as_uint(l);
                        }
                    }
                    tmem_st16(ta + 16u * hh, hv);
                    tmem_st16(ta + 64u + 16u * hh, lv);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&s_afull[s % TS_NA])) : "memory");
                copy_b(s + TS_DB);          // its stage held step s - TS_NA's image
                load_a(s + TS_P, ring[k]);  // this ring slot's next step
            }
        }
        if (ok && nsteps > 0) {
            // the last step's MMAs complete after all others: then the last fills
            const int l = nsteps - 1;
            bool w_ok = mbar_wait(&s_empty[l % TS_NB], (uint32_t)((l / TS_NB) & 1), tries, err);
            if (!__all_sync(0xffffffffu, w_ok)) ok = false;
            const int fills = (nsteps + TS_DRAIN - 1) / TS_DRAIN;
            while (ok && drained < fills) drain(drained++);
        }
        if (!ok) {
            s_bad = 1;
            for (int sp = max(0, last_b - TS_NB + 1); sp <= last_b; ++sp)  // copies still in flight
                mbar_wait(&s_bfull[sp % TS_NB], (uint32_t)((sp / TS_NB) & 1), DRAIN_TRIES);
        }
        if (ok && x < n_tgt) {
            float *dst = vt + ((size_t)tgt[x] * nrhs + m) * r + qh * 32;
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (qh * 32 + c < r) dst[c] = sum[c];
        }
    } else if (lane == 0) {
        // ---- MMA thread
        const uint32_t lbo = 128, sbo = 8 * 128;  // B image: per half of K, 64 rows x 32 in core matrices
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) |
                               ((uint32_t)(TS_M >> 4) << 24);
        int issued = 0;
        for (int s = 0; s < nsteps; ++s) {
            const int fill = s / TS_DRAIN;
            // the accumulator of fill - 2 must have been added into the producers' sums
            if (s % TS_DRAIN == 0 && fill >= 2 && !mbar_wait(&s_drained, (uint32_t)((fill - 2) & 1), tries, err)) {
                ok = false;
                break;
            }
            const int b = s % TS_NB;
            if (!mbar_wait(&s_bfull[b], (uint32_t)((s / TS_NB) & 1), tries, err) ||
                !mbar_wait(&s_afull[s % TS_NA], (uint32_t)((s / TS_NA) & 1), tries, err)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + (uint32_t)((fill & 1) * 64);
            const uint32_t a0 = tmem + (uint32_t)(128 + (s % TS_NA) * 128);
            const uint32_t bst = smem_addr(bring + (size_t)b * TS_BST);
#pragma unroll
            for (int ks = 0; ks < TS_K / 8; ++ks) {
                // K step ks: A columns 8 ks (hi) and 64 + 8 ks (lo); B in half ks / 4 of the image
                // (hi block, then lo block), core matrices 2 (ks % 4) and 2 (ks % 4) + 1
                const uint32_t ah = a0 + (uint32_t)(ks * 8), al = a0 + 64u + (uint32_t)(ks * 8);
                const uint32_t bh0 = bst + (uint32_t)((ks >> 2) * 2 * TS_BH * 4 + (ks & 3) * 256);
                const uint64_t bh = umma_desc(bh0, lbo, sbo), bl = umma_desc(bh0 + TS_BH * 4, lbo, sbo);
                const uint32_t acc0 = (s % TS_DRAIN != 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
                    "r"(ah), "l"(bh), "r"(idesc), "r"(acc0));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(d), "r"(ah), "l"(bl),
                             "r"(idesc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(d), "r"(al), "l"(bh),
                             "r"(idesc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&s_empty[b]))
                         : "memory");
            issued = s + 1;
        }
        // after a give-up: keep TMEM and the stages owned until the committed MMAs are done
        if (!ok) {
            s_bad = 1;
            if (issued > 0)
                mbar_wait(&s_empty[(issued - 1) % TS_NB], (uint32_t)(((issued - 1) / TS_NB) & 1), DRAIN_TRIES);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TS_TCOLS));
}

// u~ rows of r < 64 floats copied into rows of 64 (zero padded), the row layout the
// target-stationary transfer reads.
__global__ void k_pad_rows64(const float *__restrict__ u, int64_t nrow, int r, float *__restrict__ out) {
    int64_t n = nrow * 64;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t row = i >> 6;
        int k = (int)(i & 63);
        out[i] = k < r ? u[row * r + k] : 0.f;
    }
}

// Target step of a Lagrange level (L_X^T v~ of eq. 8): v_i += sum_abc L_a(x_i) L_b(y_i) L_c(z_i) v~_a(abc),
// one block per chunk of at most LAG_CHUNK points of a target box, added in FP32 into accf.
template <bool CPLX, int R1>
__global__ void __launch_bounds__(128) k_lag_interp(LevelArgs A, const uint2 *__restrict__ chunks, Cheb cb,
                                                    const typename QT<CPLX>::T *__restrict__ vt, int nrhs,
                                                    int64_t nx, float2 *__restrict__ accf) {
    typedef typename QT<CPLX>::T Q;
    constexpr int r = R1 * R1 * R1;
    __shared__ Q sv[r];
    uint2 ck = chunks[blockIdx.x];
    int a = (int)ck.x, m = blockIdx.y;
    for (int i = threadIdx.x; i < r; i += blockDim.x) sv[i] = vt[((size_t)a * nrhs + m) * r + i];
    __syncthreads();
    uint32_t s0 = ck.y, s1 = min(A.box_start[a + 1], s0 + (uint32_t)LAG_CHUNK);
    int4 gb = A.box_g[a];
    for (uint32_t i = s0 + threadIdx.x; i < s1; i += blockDim.x) {
        float4 e = A.eps[i];
        int4 gl = A.leaf_g[__float_as_uint(e.w)];
        float3 o = leaf_offset(gl, gb, A.shift, A.dls);
        float lx[R1MAX], ly[R1MAX], lz[R1MAX];
        lag1d(cb, (o.x + e.x) * A.inv_half_dl, lx);
        lag1d(cb, (o.y + e.y) * A.inv_half_dl, ly);
        lag1d(cb, (o.z + e.z) * A.inv_half_dl, lz);
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int ia = 0; ia < R1; ++ia)
#pragma unroll
            for (int ib = 0; ib < R1; ++ib) {
                float lab = lx[ia] * ly[ib];
                const Q *row = sv + (ia * R1 + ib) * R1;
                float pr = 0.f, pi = 0.f;
#pragma unroll
                for (int ic = 0; ic < R1; ++ic) {
                    if constexpr (CPLX) {
                        pr = fmaf(lz[ic], row[ic].x, pr);
                        pi = fmaf(lz[ic], row[ic].y, pi);
                    } else {
                        pr = fmaf(lz[ic], row[ic], pr);
                    }
                }
                sr = fmaf(lab, pr, sr);
                if constexpr (CPLX) si = fmaf(lab, pi, si);
            }
        float2 &dst = accf[(int64_t)m * nx + i];
        dst.x += sr;
        if constexpr (CPLX) dst.y += si;
    }
}

static LevelArgs level_args(const ffm_plan_s *p, const BoxLevel &B, const BoxLevel &Lf, const float4 *eps, int l) {
    LevelArgs A;
    A.box_start = B.start;
    A.box_g = B.g;
    A.box_leaf = B.first_leaf;
    A.leaf_start = Lf.start;
    A.leaf_g = Lf.g;
    A.eps = eps;
    A.shift = p->l_stop - l;
    A.dls = (float)std::ldexp(p->d0, -p->l_stop);
    A.inv_half_dl = (float)(2.0 / std::ldexp(p->d0, -l));
    return A;
}

// ---- warp-per-chunk forms of the two point-wise Lagrange steps
//
// Fine levels of clustered inputs have millions of boxes holding a few points each; a block
// per chunk then leaves most of its threads idle.  Here a warp takes one chunk (at most
// LAG_CHUNK points of a box) and a block holds eight of them.  Source step: the lanes form
// the 1-D Lagrange weights of 32 points at a time into the warp's shared rows, then each
// lane adds those points into its own control nodes (lane, lane + 32, ...).  Target step:
// the warp stages the box's r coefficients once and each lane interpolates its own points.
constexpr int LAG_WC = 8;  // chunks (warps) per block

template <bool CPLX, int R1>
__global__ void __launch_bounds__(32 * LAG_WC) k_lag_anterp_w(LevelArgs A, const uint2 *__restrict__ chunks,
                                                             int64_t nchunks, Cheb cb,
                                                             const typename QT<CPLX>::T *__restrict__ q, int64_t ny,
                                                             int nrhs, typename QT<CPLX>::T *__restrict__ ut) {
    typedef typename QT<CPLX>::T Q;
    constexpr int r = R1 * R1 * R1, NA = (r + 31) / 32, W = 3 * R1;
    __shared__ float sl[LAG_WC][32][W + 1];
    __shared__ Q sq[LAG_WC][CPLX ? 32 : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ci = (int64_t)blockIdx.x * LAG_WC + warp;
    if (ci >= nchunks) return;  // warp-level work only: no block barrier below
    const int m = blockIdx.y;
    const uint2 ck = chunks[ci];
    const int b = (int)ck.x;
    const uint32_t s0 = ck.y, bend = A.box_start[b + 1], s1 = min(bend, s0 + (uint32_t)LAG_CHUNK);
    const bool sole = s0 == A.box_start[b] && s1 == bend;
    const int4 gb = A.box_g[b];
    float accr[NA], acci[NA];
#pragma unroll
    for (int k = 0; k < NA; ++k) accr[k] = acci[k] = 0.f;
    float(*row)[W + 1] = sl[warp];
    for (uint32_t base = s0; base < s1; base += 32) {
        const uint32_t j = base + lane;
        if (j < s1) {
            float4 e = A.eps[j];
            int4 gl = A.leaf_g[__float_as_uint(e.w)];
            float3 o = leaf_offset(gl, gb, A.shift, A.dls);
            float lx[R1MAX], ly[R1MAX], lz[R1MAX];
            lag1d(cb, (o.x + e.x) * A.inv_half_dl, lx);
            lag1d(cb, (o.y + e.y) * A.inv_half_dl, ly);
            lag1d(cb, (o.z + e.z) * A.inv_half_dl, lz);
            Q w = q[(int64_t)m * ny + j];
#pragma unroll
            for (int a = 0; a < R1; ++a) {
                if constexpr (CPLX)
                    row[lane][a] = lx[a];
                else
                    row[lane][a] = lx[a] * w;
                row[lane][R1 + a] = ly[a];
                row[lane][2 * R1 + a] = lz[a];
            }
            if constexpr (CPLX) sq[warp][lane] = w;
        }
        __syncwarp();
        const int cnt = (int)min((uint32_t)32, s1 - base);
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const int a = lane + 32 * k;
            if (a < r) {
                const int ia = a / (R1 * R1), ib = (a / R1) % R1, ic = a % R1;
                for (int jj = 0; jj < cnt; ++jj) {
                    float L = row[jj][ia] * row[jj][R1 + ib];
                    if constexpr (CPLX) {
                        L *= row[jj][2 * R1 + ic];
                        accr[k] = fmaf(L, sq[warp][jj].x, accr[k]);
                        acci[k] = fmaf(L, sq[warp][jj].y, acci[k]);
                    } else {
                        accr[k] = fmaf(L, row[jj][2 * R1 + ic], accr[k]);
                    }
                }
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < NA; ++k) {
        const int a = lane + 32 * k;
        if (a < r) {
            size_t o = ((size_t)b * nrhs + m) * r + a;
            if constexpr (CPLX) {
                if (sole) {
                    ut[o] = make_float2(accr[k], acci[k]);
                } else {
                    atomicAdd(&ut[o].x, accr[k]);
                    atomicAdd(&ut[o].y, acci[k]);
                }
            } else {
                if (sole)
                    ut[o] = accr[k];
                else
                    atomicAdd(&ut[o], accr[k]);
            }
        }
    }
}

template <bool CPLX, int R1>
__global__ void __launch_bounds__(32 * LAG_WC) k_lag_interp_w(LevelArgs A, const uint2 *__restrict__ chunks,
                                                             int64_t nchunks, Cheb cb,
                                                             const typename QT<CPLX>::T *__restrict__ vt, int nrhs,
                                                             int64_t nx, float2 *__restrict__ accf) {
    typedef typename QT<CPLX>::T Q;
    constexpr int r = R1 * R1 * R1;
    __shared__ Q sv[LAG_WC][r];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ci = (int64_t)blockIdx.x * LAG_WC + warp;
    if (ci >= nchunks) return;  // warp-level work only: no block barrier below
    const int m = blockIdx.y;
    const uint2 ck = chunks[ci];
    const int a = (int)ck.x;
    Q *v = sv[warp];
    for (int i = lane; i < r; i += 32) v[i] = vt[((size_t)a * nrhs + m) * r + i];
    __syncwarp();
    const uint32_t s0 = ck.y, s1 = min(A.box_start[a + 1], s0 + (uint32_t)LAG_CHUNK);
    const int4 gb = A.box_g[a];
    for (uint32_t i = s0 + lane; i < s1; i += 32) {
        float4 e = A.eps[i];
        int4 gl = A.leaf_g[__float_as_uint(e.w)];
        float3 o = leaf_offset(gl, gb, A.shift, A.dls);
        float lx[R1MAX], ly[R1MAX], lz[R1MAX];
        lag1d(cb, (o.x + e.x) * A.inv_half_dl, lx);
        lag1d(cb, (o.y + e.y) * A.inv_half_dl, ly);
        lag1d(cb, (o.z + e.z) * A.inv_half_dl, lz);
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int ia = 0; ia < R1; ++ia)
#pragma unroll
            for (int ib = 0; ib < R1; ++ib) {
                float lab = lx[ia] * ly[ib];
                const Q *rw = v + (ia * R1 + ib) * R1;
                float pr = 0.f, pi = 0.f;
#pragma unroll
                for (int ic = 0; ic < R1; ++ic) {
                    if constexpr (CPLX) {
                        pr = fmaf(lz[ic], rw[ic].x, pr);
                        pi = fmaf(lz[ic], rw[ic].y, pi);
                    } else {
                        pr = fmaf(lz[ic], rw[ic], pr);
                    }
                }
                sr = fmaf(lab, pr, sr);
                if constexpr (CPLX) si = fmaf(lab, pi, si);
            }
        float2 &dst = accf[(int64_t)m * nx + i];
        dst.x += sr;
        if constexpr (CPLX) dst.y += si;
    }
}

template <bool CPLX, int R1>
static void lagrange_points(const ffm_plan_s *p, const FarLevel &F, const LevelArgs &A, const Cheb &cb, bool anterp,
                            const void *in, int nrhs, void *out, cudaStream_t s) {
    typedef typename QT<CPLX>::T Q;
    // warp per chunk up to r = 64 (the ranks of eps >= 1e-4 for the single layer); the block
    // forms keep the larger bases, whose per-point sums need more registers per thread
    if constexpr (R1 <= 4) {
        if (anterp) {
            dim3 g(cdiv(F.n_src_chunks, LAG_WC), nrhs);
            FFM_LAUNCH((k_lag_anterp_w<CPLX, R1>), g, 32 * LAG_WC, 0, s, A, F.src_chunks, F.n_src_chunks, cb,
                       (const Q *)in, p->ny, nrhs, (Q *)out);
        } else {
            dim3 g(cdiv(F.n_tgt_chunks, LAG_WC), nrhs);
            FFM_LAUNCH((k_lag_interp_w<CPLX, R1>), g, 32 * LAG_WC, 0, s, A, F.tgt_chunks, F.n_tgt_chunks, cb,
                       (const Q *)in, nrhs, p->nx, (float2 *)out);
        }
        return;
    }
    if (anterp) {
        dim3 g((unsigned)F.n_src_chunks, nrhs);
        FFM_LAUNCH((k_lag_anterp<CPLX, R1>), g, LAG_T, 0, s, A, F.src_chunks, cb, (const Q *)in, p->ny, nrhs,
                   (Q *)out);
    } else {
        dim3 g((unsigned)F.n_tgt_chunks, nrhs);
        FFM_LAUNCH((k_lag_interp<CPLX, R1>), g, 128, 0, s, A, F.tgt_chunks, cb, (const Q *)in, nrhs, p->nx,
                   (float2 *)out);
    }
}

template <int R1>
static void lagrange_anterp_dl(const ffm_plan_s *p, const FarLevel &F, const LevelArgs &A, const Cheb &cb,
                               const void *q, int nrhs, void *ut, cudaStream_t s) {
    dim3 g((unsigned)F.n_src_chunks, nrhs);
    FFM_LAUNCH((k_lag_anterp_dl<R1>), g, LAG_T, 0, s, A, F.src_chunks, cb, (const float4 *)q, p->ny, nrhs, (float *)ut);
}

static void lagrange_anterp_dl_r1(const ffm_plan_s *p, const FarLevel &F, const LevelArgs &A, const Cheb &cb,
                                  const void *q, int nrhs, void *ut, cudaStream_t s) {
    switch (F.r1) {
        case 2: lagrange_anterp_dl<2>(p, F, A, cb, q, nrhs, ut, s); break;
        case 3: lagrange_anterp_dl<3>(p, F, A, cb, q, nrhs, ut, s); break;
        case 4: lagrange_anterp_dl<4>(p, F, A, cb, q, nrhs, ut, s); break;
        case 5: lagrange_anterp_dl<5>(p, F, A, cb, q, nrhs, ut, s); break;
        case 6: lagrange_anterp_dl<6>(p, F, A, cb, q, nrhs, ut, s); break;
        case 7: lagrange_anterp_dl<7>(p, F, A, cb, q, nrhs, ut, s); break;
        case 8: lagrange_anterp_dl<8>(p, F, A, cb, q, nrhs, ut, s); break;
        default: fail(FFM_EUNSUPPORTED, "Chebyshev nodes per axis outside 2..8");
    }
}

template <bool CPLX>
static void lagrange_points_r1(const ffm_plan_s *p, const FarLevel &F, const LevelArgs &A, const Cheb &cb,
                               bool anterp, const void *in, int nrhs, void *out, cudaStream_t s) {
    switch (F.r1) {
        case 2: lagrange_points<CPLX, 2>(p, F, A, cb, anterp, in, nrhs, out, s); break;
        case 3: lagrange_points<CPLX, 3>(p, F, A, cb, anterp, in, nrhs, out, s); break;
        case 4: lagrange_points<CPLX, 4>(p, F, A, cb, anterp, in, nrhs, out, s); break;
        case 5: lagrange_points<CPLX, 5>(p, F, A, cb, anterp, in, nrhs, out, s); break;
        case 6: lagrange_points<CPLX, 6>(p, F, A, cb, anterp, in, nrhs, out, s); break;
        case 7: lagrange_points<CPLX, 7>(p, F, A, cb, anterp, in, nrhs, out, s); break;
        case 8: lagrange_points<CPLX, 8>(p, F, A, cb, anterp, in, nrhs, out, s); break;
        default: fail(FFM_EUNSUPPORTED, "Chebyshev nodes per axis outside 2..8");
    }
}

void split_pad(const float *src, int64_t nmat, int rows, int cols, int rows_pad, int cols_pad, float *hi, float *lo,
               cudaStream_t s) {  // lo == nullptr: padded copy into hi
    int64_t n = nmat * rows_pad * (int64_t)cols_pad;
    unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16);
    FFM_LAUNCH(k_split_pad, g, 256, 0, s, src, nmat, rows, cols, rows_pad, cols_pad, hi, lo);
}

// The tcgen05 transfer over row blocks of the operator: every launch takes rows [row0, row0 +
// nb) of each T_t (nb <= 224, a multiple of 16, the blocks as even as possible) with the
// whole K, and adds output columns row0 .. of v~.  T_t starts every tstride floats with rows
// of rkp floats (zero past `rows`); v~ rows are ostride floats apart.
static void tc_transfer(const FarLevel &F, const uint32_t *src, const uint32_t *tgt, const float *Tp, int64_t tstride,
                        int rows, int rkp, int ostride, int nrhs, const float *up, float *vt, int *err,
                        int tries, cudaStream_t s) {
    constexpr int KT = 16, NR = 3, NO = 2;
    auto smem_of = [](int np_) {
        return (size_t)NO * (2 * TC_P * KT + 2 * np_ * KT) * sizeof(float) + (size_t)NR * (TC_P + np_) * KT * sizeof(float);
    };
    // per device and cheap: set before every launch (plans may live on several devices)
    FFM_CUDA(cudaFuncSetAttribute(k_lag_gemm_tc<KT, NR, NO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_of(224)));
    const int npad = (rows + 15) / 16 * 16, parts = cdiv(npad, 224);
    const int nb = (cdiv(npad, parts) + 15) / 16 * 16;
    for (int row0 = 0; row0 < npad; row0 += nb) {
        const int nbk = std::min(nb, npad - row0), nout = std::min(nbk, rows - row0);
        int tcols = 32;
        while (tcols < nbk) tcols <<= 1;
        FFM_LAUNCH((k_lag_gemm_tc<KT, NR, NO>), dim3((unsigned)F.tc_tiles, nrhs), 256, smem_of(nbk), s, F.tc_tile_t,
                   F.tc_tile_p0, F.bt_off, src, tgt, Tp + (size_t)row0 * rkp, tstride, ostride, nout, rkp, nbk, tcols,
                   nrhs, up, vt + row0, err, tries);
    }
}

void far_lagrange(const ffm_plan_s *p, int l, const void *q, int nrhs, float2 *accf, Alloc &tmp, cudaStream_t s) {
    const FarLevel &F = p->far[l];
    int ls = p->l_stop;
    int r = F.r1 * F.r1 * F.r1;
    Cheb cb = make_cheb(F.r1);
    LevelArgs AY = level_args(p, p->by[l], p->by[ls], p->epsY, l);
    LevelArgs AX = level_args(p, p->bx[l], p->bx[ls], p->epsX, l);
    bool cplx = p->kind == FFM_HELMHOLTZ;
    int rk = p->kind == FFM_LAPLACE_DL ? 3 * r : r;  // K extent of the transfer
    size_t esz = cplx ? sizeof(float2) : sizeof(float);
    size_t ub = esz * rk * nrhs * (size_t)p->by[l].nb,
           vb = esz * r * nrhs * (size_t)p->bx[l].nb * (p->kind == FFM_LAPLACE_GRAD ? 3 : 1);
    void *ut = tmp.raw(ub);
    void *vt = tmp.raw(vb);
    dim3 gg((unsigned)F.n_tiles, cdiv(r, LG_BM), nrhs);
    FFM_CUDA(cudaMemsetAsync(ut, 0, ub, s));
    FFM_CUDA(cudaMemsetAsync(vt, 0, vb, s));
    if (cplx) {
        lagrange_points_r1<true>(p, F, AY, cb, true, q, nrhs, ut, s);
        FFM_LAUNCH(k_lag_gemm<true>, gg, LG_T, 0, s, F.tile_t, F.tile_p0, F.bt_off, F.bt_src, F.bt_tgt, F.T, r, rk,
                   nrhs, (const float2 *)ut, (float2 *)vt);
        lagrange_points_r1<true>(p, F, AX, cb, false, vt, nrhs, accf, s);
    } else {
        if (p->kind == FFM_LAPLACE_DL)
            lagrange_anterp_dl_r1(p, F, AY, cb, q, nrhs, ut, s);
        else
            lagrange_points_r1<false>(p, F, AY, cb, true, q, nrhs, ut, s);
        int npad = (r + 15) / 16 * 16;
        if (F.aca) {
            // ACA factors (eq. 11): w_p = B_t^T u~_src(p) for every pair p of translation t
            // (rows of w indexed by pair), then v~_tgt(p) += A_t w_p
            const int rp = F.aca_rp;
            float *w = tmp.get<float>((size_t)F.n_adm * nrhs * rp);
            FFM_CUDA(cudaMemsetAsync(w, 0, sizeof(float) * (size_t)F.n_adm * nrhs * rp, s));
            if (F.aca_tc) {
                int64_t nrow = (int64_t)p->by[l].nb * nrhs;
                float *upad = tmp.get<float>((size_t)nrow * F.rkp);
                split_pad((const float *)ut, 1, (int)nrow, r, (int)nrow, F.rkp, upad, nullptr, s);
                tc_transfer(F, F.bt_src, F.pair_id, F.Bca, (int64_t)rp * F.rkp, rp, F.rkp, rp, nrhs, upad, w,
                            p->dev_err, p->wait_tries, s);
                tc_transfer(F, F.pair_id, F.bt_tgt, F.Aca, (int64_t)npad * rp, r, rp, r, nrhs, w, (float *)vt,
                            p->dev_err, p->wait_tries, s);
                tmp.drop(upad);
            } else {
                dim3 g1((unsigned)F.n_tiles, cdiv(rp, LG_BM), nrhs);
                FFM_LAUNCH(k_lag_gemm<false>, g1, LG_T, 0, s, F.tile_t, F.tile_p0, F.bt_off, F.bt_src, F.pair_id,
                           F.Bca, rp, r, nrhs, (const float *)ut, w);
                FFM_LAUNCH(k_lag_gemm<false>, gg, LG_T, 0, s, F.tile_t, F.tile_p0, F.bt_off, F.pair_id, F.bt_tgt,
                           F.Aca, r, rp, nrhs, (const float *)w, (float *)vt);
            }
            tmp.drop(w);
            lagrange_points_r1<false>(p, F, AX, cb, false, vt, nrhs, accf, s);
            return;
        }
        // the gradient has three operator blocks (component-major) and three outputs per
        // target; v~ and the FP32 accumulators are component-major too
        const int ncomp = p->kind == FFM_LAPLACE_GRAD ? 3 : 1;
        const size_t tblk = (size_t)F.n_trans * r * rk;
        const size_t vblk = (size_t)r * nrhs * p->bx[l].nb;
        float *upad = nullptr, *uts = nullptr;
        const bool use_tc = !(F.ts_ok && F.Tsp && F.tune_tc == 2) && F.tc_tiles > 0 && F.tune_tc != 0 && F.Tsh;
        if (use_tc) {
            // u~ with rows padded to rkp floats (whole, aligned 16-byte segments for cp.async)
            int64_t nrow = (int64_t)p->by[l].nb * nrhs;
            upad = tmp.get<float>((size_t)nrow * F.rkp);
            split_pad((const float *)ut, 1, (int)nrow, rk, (int)nrow, F.rkp, upad, nullptr, s);
        }
        for (int d = 0; d < ncomp; ++d) {
            const float *Td = F.T + d * tblk;
            float *vtd = (float *)vt + d * vblk;
        if (F.ts_ok && F.Tsp && F.tune_tc == 2) {
            FFM_CUDA(cudaFuncSetAttribute(k_lag_gemm_ts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS_SMEM));
            const float *u64 = (const float *)ut;
            if (r < 64) {  // rows of 64 floats, once for all components
                const int64_t nrow = (int64_t)p->by[l].nb * nrhs;
                if (!uts) {
                    uts = tmp.get<float>((size_t)nrow * 64);
                    unsigned gs = (unsigned)std::min<int64_t>(cdiv(nrow * 64, 256), 152 * 16);
                    FFM_LAUNCH(k_pad_rows64, gs, 256, 0, s, (const float *)ut, nrow, r, uts);
                }
                u64 = uts;
            }
            dim3 gts(cdiv(F.n_tgt, TS_M), nrhs);
            FFM_LAUNCH(k_lag_gemm_ts, gts, TS_NP + 32, TS_SMEM, s, F.tgt, F.n_tgt, F.adm_off, F.adm_src, F.adm_t,
                       F.n_trans, F.Tsp, r, nrhs, u64, vtd, p->dev_err, p->wait_tries);
        } else if (use_tc) {
            // tensor cores: 256-pair tiles, K chunks of 16 source nodes, row blocks of <= 224
            const int rkp = F.rkp;
            const size_t dsz = (size_t)F.n_trans * npad * rkp;
            tc_transfer(F, F.bt_src, F.bt_tgt, F.Tsh + d * dsz, (int64_t)npad * rkp, r, rkp, r, nrhs, upad, vtd,
                        p->dev_err, p->wait_tries, s);
        } else {
            FFM_LAUNCH(k_lag_gemm<false>, gg, LG_T, 0, s, F.tile_t, F.tile_p0, F.bt_off, F.bt_src, F.bt_tgt, Td, r,
                       rk, nrhs, (const float *)ut, vtd);
        }
            lagrange_points_r1<false>(p, F, AX, cb, false, vtd, nrhs, accf + (size_t)d * nrhs * p->nx, s);
        }
        if (upad) tmp.drop(upad);
        if (uts) tmp.drop(uts);
    }
}

// ======================================================= plane-wave kernels

constexpr int PW_CHUNK = 256; // staged points per block iteration
constexpr int PW_MAXD = 16;   // deepest supported level gap between box and leaf
constexpr int PW_QC = 512;    // directions staged per block iteration in the backward transform

// Scalar-type traits: FP32 levels use float tables and MUFU sincos; FP64 levels (large
// cancellation in the quadrature sum) use double tables, leaf coordinates hi + lo and
// FP64 sincos.
template <class R>
struct PwT;
template <>
struct PwT<float> {
    typedef float2 C;
    typedef float4 K;
};
template <>
struct PwT<double> {
    typedef double2 C;
    typedef D4 K;
};
// double-float levels: tables and sums as unevaluated FP32 pairs (dfloat.cuh)
template <>
struct PwT<dd> {
    typedef dd2 C;
    typedef dd4 K;
};

__device__ __forceinline__ dd2 cmul(dd2 a, dd2 b) { return dd2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ dd2 cmulc(dd2 a, dd2 b) { return dd2{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y}; }
__device__ __forceinline__ dd2 czero(dd) { return dd2{dd(0.f), dd(0.f)}; }
__device__ __forceinline__ dd2 cone(dd) { return dd2{dd(1.f), dd(0.f)}; }

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 czero(float) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double2 czero(double) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 cone(float) { return make_float2(1.f, 0.f); }
__device__ __forceinline__ double2 cone(double) { return make_double2(1.0, 0.0); }

// Phasor modes of the FP32 levels: the hardware sincos approximation on the phase as is
// (PH_MUFU) or after Cody-Waite reduction to [-pi, pi] (PH_MUFU_RED), or the accurate
// sincos below (PH_ACC, compensated levels).  FP64 levels ignore the mode.
constexpr int PH_MUFU = 0, PH_MUFU_RED = 1, PH_ACC = 2;

// sin and cos to about one FP32 ulp: x = n pi/2 + r with |r| <= pi/4 (Cody and Waite's
// reduction, pi/2 split in two FP32 terms), then the Taylor series of sin r to r^9 and of
// cos r to r^10, whose first omitted terms are below 3e-9, and the quadrant's symmetry.
__device__ __forceinline__ void sincos_acc(float x, float &s, float &c) {
    constexpr double PIO2 = 1.5707963267948966;
    constexpr float PIO2_HI = (float)PIO2;
    constexpr float PIO2_LO = (float)(PIO2 - (double)PIO2_HI);
    constexpr float TWO_OVER_PI = (float)(2.0 / 3.14159265358979323846);
    // n = nearest integer of x 2/pi by the 1.5 2^23 shifter; its low bits give the quadrant
    float t = fmaf(x, TWO_OVER_PI, 12582912.f);
    float n = t - 12582912.f;
    float r = fmaf(-n, PIO2_HI, x);
    r = fmaf(-n, PIO2_LO, r);
    float r2 = r * r;
    // coefficients (-1)^j / (2j+1)! and (-1)^j / (2j)!
    float ps = fmaf(r2, (float)(1.0 / 362880.0), (float)(-1.0 / 5040.0));
    ps = fmaf(r2, ps, (float)(1.0 / 120.0));
    ps = fmaf(r2, ps, (float)(-1.0 / 6.0));
    float sr = fmaf(r * r2, ps, r);
    float pc = fmaf(r2, (float)(-1.0 / 3628800.0), (float)(1.0 / 40320.0));
    pc = fmaf(r2, pc, (float)(-1.0 / 720.0));
    pc = fmaf(r2, pc, (float)(1.0 / 24.0));
    pc = fmaf(r2, pc, -0.5f);
    float cr = fmaf(r2, pc, 1.0f);
    int q = __float_as_int(t) & 3;
    float a = (q & 1) ? cr : sr, b = (q & 1) ? sr : cr;
    s = (q & 2) ? -a : a;
    c = ((q + 1) & 2) ? -b : b;
}

template <int PH>
__device__ __forceinline__ void phase_sincos(float ph, float &s, float &c, const float4 *) {
    if constexpr (PH == PH_ACC) {
        sincos_acc(ph, s, c);
    } else {
        if constexpr (PH == PH_MUFU_RED) {
            float n = rintf(ph * 0.15915494309189535f);
            ph = fmaf(-n, 6.28318548202514648f, ph);
            ph = fmaf(-n, -1.7484555314695172e-07f, ph);
        }
        __sincosf(ph, &s, &c);
    }
}
template <int PH>
__device__ __forceinline__ void phase_sincos(double ph, double &s, double &c, const float4 *) {
    sincos(ph, &s, &c);
}
template <int PH>
__device__ __forceinline__ void phase_sincos(dd ph, dd &s, dd &c, const float4 *tab) {
    dd_sincos(ph, s, c, tab);
}

// hi + t with the rounding error carried into lo (Knuth's TwoSum; no ordering assumption)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float t) {
    float sum = hi + t;
    float bb = sum - hi;
    lo += (hi - (sum - bb)) + (t - bb);
    hi = sum;
}
__device__ __forceinline__ void two_sum_acc(double &hi, double &, double t) { hi += t; }
__device__ __forceinline__ void two_sum_acc(dd &hi, dd &, dd t) { hi = hi + t; }

// Leaf-relative coordinates of a point in the level's scalar type (hi part only in FP32,
// hi + lo in FP64).
template <class R>
struct Coord;
template <>
struct Coord<float> {
    static __device__ __forceinline__ float3 get(const float4 &hi, const float4 *, uint32_t) {
        return make_float3(hi.x, hi.y, hi.z);
    }
};
template <>
struct Coord<dd> {
    static __device__ __forceinline__ dd3 get(const float4 &hi, const float4 *lo, uint32_t i) {
        float4 l = lo[i];
        return dd3{dd(hi.x, l.x), dd(hi.y, l.y), dd(hi.z, l.z)};
    }
};
template <>
struct Coord<double> {
    static __device__ __forceinline__ double3 get(const float4 &hi, const float4 *lo, uint32_t i) {
        float4 l = lo[i];
        return make_double3((double)hi.x + (double)l.x, (double)hi.y + (double)l.y, (double)hi.z + (double)l.z);
    }
};

template <class R>
struct PwArgs {
    LevelArgs A;
    const float4 *eps_lo;  // lo parts of the leaf-relative coordinates (FP64 levels)
    const typename PwT<R>::K *ks;
    const typename PwT<R>::C *E;  // [depth][oct][q]
    int nQ;
    const float4 *sctab;          // double-float sin/cos table (double-float levels)
};

// Octant path of a leaf: oct[d] = octant of its ancestor at depth l+1+d within its parent.
__device__ __forceinline__ int leaf_octant(int4 gl, int shift, int d) {
    int sh = shift - 1 - d;  // depth l+1+d sits sh levels above the leaf
    return (((gl.x >> sh) & 1) << 2) | (((gl.y >> sh) & 1) << 1) | ((gl.z >> sh) & 1);
}

// Leaf factor prod_d E[d][oct[d]][q] (conjugated when CONJ), octant path from shared memory.
template <bool CONJ, class R>
__device__ __forceinline__ typename PwT<R>::C leaf_factor(const PwArgs<R> &P, const int *oct, int q) {
    typename PwT<R>::C f = cone(R(0));
    for (int d = 0; d < P.A.shift; ++d) {
        typename PwT<R>::C e = P.E[((size_t)d * 8 + oct[d]) * P.nQ + q];
        f = CONJ ? cmulc(f, e) : cmul(f, e);
    }
    return f;
}

// Forward transform: u~_b(q) for a chunk of direction pairs of one source box.  The
// leaves of the box are visited in order; each leaf's points are staged in shared memory
// and summed with leaf-centred phases in a tight loop, then the leaf sum is moved to the
// box centre by its octant factor.  Directions h and h + nQ/2 are antipodal, so one
// sincos of k s_h . e serves both: with P = sum cos(ph) w and Q = sum sin(ph) w, the leaf
// sums are P - iQ (direction h, phasor e^{-i ph}) and P + iQ (its antipode).  Each thread
// owns QPT pairs.
template <class R, int PH, int QPT>
__global__ void __launch_bounds__(128) k_pw_forward(PwArgs<R> P, const uint32_t *__restrict__ src,
                                                    const float2 *__restrict__ q, int64_t ny, int nrhs,
                                                    typename PwT<R>::C *__restrict__ ut) {
    typedef typename PwT<R>::C C2;
    __shared__ float4 se[PW_CHUNK];
    __shared__ float4 sl[sizeof(R) == 8 ? PW_CHUNK : 1];
    __shared__ float2 sq[PW_CHUNK];
    __shared__ int soct[PW_MAXD];
    int b = src[blockIdx.x], m = blockIdx.z;
    int nH = P.nQ / 2;
    int h0 = blockIdx.y * blockDim.x * QPT + threadIdx.x;  // pairs h0 + t * blockDim.x
    R kx[QPT], ky[QPT], kz[QPT];
    bool on[QPT];
#pragma unroll
    for (int t = 0; t < QPT; ++t) {
        int hh = h0 + t * blockDim.x;
        on[t] = hh < nH;
        int hc = on[t] ? hh : 0;
        kx[t] = P.ks[hc].x;
        ky[t] = P.ks[hc].y;
        kz[t] = P.ks[hc].z;
    }
    C2 acc[QPT], acb[QPT];
#pragma unroll
    for (int t = 0; t < QPT; ++t) acc[t] = acb[t] = czero(R(0));
    const float2 *qm = q + (int64_t)m * ny;
    uint32_t lf0 = P.A.box_leaf[b], lf1 = P.A.box_leaf[b + 1];
    for (uint32_t leaf = lf0; leaf < lf1; ++leaf) {
        uint32_t p0 = P.A.leaf_start[leaf], p1 = P.A.leaf_start[leaf + 1];
        C2 Pc[QPT], Qs[QPT];
#pragma unroll
        for (int t = 0; t < QPT; ++t) Pc[t] = Qs[t] = czero(R(0));
        for (uint32_t base = p0; base < p1; base += PW_CHUNK) {
            int cnt = (int)min((uint32_t)PW_CHUNK, p1 - base);
            __syncthreads();
            for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
                se[j] = P.A.eps[base + j];
                if constexpr (sizeof(R) == 8) sl[j] = P.eps_lo[base + j];
                sq[j] = qm[base + j];
            }
            if (base == p0 && threadIdx.x < P.A.shift) soct[threadIdx.x] = leaf_octant(P.A.leaf_g[leaf], P.A.shift, threadIdx.x);
            __syncthreads();
#pragma unroll 2
            for (int j = 0; j < cnt; ++j) {
                auto e = Coord<R>::get(se[j], sl, (uint32_t)j);
                float2 w = sq[j];
#pragma unroll
                for (int t = 0; t < QPT; ++t) {
                    R ph = fma(kx[t], e.x, fma(ky[t], e.y, kz[t] * e.z));
                    R sn, cs;
                    phase_sincos<PH>(ph, sn, cs, P.sctab);
                    Pc[t].x = fma(cs, (R)w.x, Pc[t].x);
                    Pc[t].y = fma(cs, (R)w.y, Pc[t].y);
                    Qs[t].x = fma(sn, (R)w.x, Qs[t].x);
                    Qs[t].y = fma(sn, (R)w.y, Qs[t].y);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < QPT; ++t) {
            if (!on[t]) continue;
            int hh = h0 + t * blockDim.x;
            C2 S, Sb;
            S.x = Pc[t].x + Qs[t].y;
            S.y = Pc[t].y - Qs[t].x;
            Sb.x = Pc[t].x - Qs[t].y;
            Sb.y = Pc[t].y + Qs[t].x;
            // the antipode's octant factor is the conjugate of direction h's
            C2 f = leaf_factor<false>(P, soct, hh);
            C2 v = cmul(f, S), vb = cmulc(Sb, f);
            acc[t].x += v.x;
            acc[t].y += v.y;
            acb[t].x += vb.x;
            acb[t].y += vb.y;
        }
    }
#pragma unroll
    for (int t = 0; t < QPT; ++t)
        if (on[t]) {
            int hh = h0 + t * blockDim.x;
            C2 *o = ut + ((size_t)b * nrhs + m) * P.nQ;
            o[hh] = acc[t];
            o[hh + nH] = acb[t];
        }
}

// Diagonal transfer: v~_a(q) = sum_{b adm a} D_t(q) u~_b(q), all right-hand sides of a
// direction in one thread so that D_t(q) is read once per pair.  COMP: the sum over the
// admissible sources is compensated (TwoSum).
template <class C2, int MR, bool COMP>
__global__ void k_pw_transfer(const uint32_t *__restrict__ tgt, const uint32_t *__restrict__ off,
                              const uint32_t *__restrict__ asrc, const uint32_t *__restrict__ at,
                              const C2 *__restrict__ D, int nQ, int nrhs, const C2 *__restrict__ ut,
                              C2 *__restrict__ vt) {
    int x = blockIdx.x;
    int q = blockIdx.y * blockDim.x + threadIdx.x;
    if (q >= nQ) return;
    for (int m0 = 0; m0 < nrhs; m0 += MR) {
        C2 a[MR], al[MR];
#pragma unroll
        for (int m = 0; m < MR; ++m) a[m].x = a[m].y = al[m].x = al[m].y = 0;
        for (uint32_t e = off[x]; e < off[x + 1]; ++e) {
            uint32_t b = asrc[e], t = at[e];
            C2 d = D[(size_t)t * nQ + q];
            const C2 *ub = ut + ((size_t)b * nrhs + m0) * nQ + q;
#pragma unroll
            for (int m = 0; m < MR; ++m)
                if (m0 + m < nrhs) {
                    C2 u = ub[(size_t)m * nQ];
                    if constexpr (COMP) {
                        two_sum_acc(a[m].x, al[m].x, fma(d.x, u.x, -d.y * u.y));
                        two_sum_acc(a[m].y, al[m].y, fma(d.x, u.y, d.y * u.x));
                    } else {
                        a[m].x = fma(d.x, u.x, fma(-d.y, u.y, a[m].x));
                        a[m].y = fma(d.x, u.y, fma(d.y, u.x, a[m].y));
                    }
                }
        }
#pragma unroll
        for (int m = 0; m < MR; ++m)
            if (m0 + m < nrhs) {
                C2 r = a[m];
                if constexpr (COMP) {
                    r.x += al[m].x;
                    r.y += al[m].y;
                }
                vt[((size_t)tgt[x] * nrhs + m0 + m) * nQ + q] = r;
            }
    }
}

// Staged backward weights of direction pair h: with W_h = v~_a(h) conj(F_leaf(h)) and
// W_b = v~_a(h + nQ/2) F_leaf(h), the pair contributes
// e^{+i ph} W_h + e^{-i ph} W_b = cos(ph) A + sin(ph) B, A = W_h + W_b, B = i (W_h - W_b).
template <class C2>
__device__ __forceinline__ void backward_weights(C2 vh, C2 vb, C2 f, C2 &A, C2 &B) {
    C2 wh = cmulc(vh, f), wb = cmul(vb, f);
    A.x = wh.x + wb.x;
    A.y = wh.y + wb.y;
    B.x = wb.y - wh.y;
    B.y = wh.x - wb.x;
}

// Backward transform for one target leaf: v_i += sum_q e^{ik s_q.(x_i - c_leaf)} W(q),
// W(q) = v~_a(q) prod conj(E) (the leaf's octant path up to its level-l ancestor a).
// Each thread owns PPT points of the leaf (one shared-memory read of a direction serves
// PPT phasors); thread groups split the directions when the leaf is small.  In the
// compensated mode the sum over directions carries its rounding error (TwoSum).
template <class R, int PH, int PPT>
__global__ void __launch_bounds__(128) k_pw_backward(PwArgs<R> P, const uint32_t *__restrict__ box_fine,
                                                     int64_t nbox, const uint32_t *__restrict__ leaf_fine,
                                                     const int *__restrict__ slot,
                                                     const typename PwT<R>::C *__restrict__ vt, int nrhs, int64_t nx,
                                                     double2 *__restrict__ acc) {
    typedef typename PwT<R>::C C2;
    typedef typename PwT<R>::K K4;
    constexpr bool COMP = PH == PH_ACC && sizeof(R) == 4;
    constexpr int QC = sizeof(R) == 8 ? PW_QC / 4 : PW_QC;  // direction pairs per chunk
    __shared__ K4 sk[QC];
    __shared__ C2 sA[QC];
    __shared__ C2 sB[QC];
    __shared__ C2 red[128 * PPT];
    __shared__ C2 redl[COMP ? 128 * PPT : 1];
    int leaf = blockIdx.x, m = blockIdx.z;
    // ancestor at level l: last box whose first deep box index <= the leaf's
    uint32_t lf = leaf_fine[leaf];
    int64_t lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (box_fine[mid] <= lf)
            lo = mid;
        else
            hi = mid - 1;
    }
    int a = (int)lo;
    if (slot[a] < 0) return;
    uint32_t p0 = P.A.leaf_start[leaf], p1 = P.A.leaf_start[leaf + 1];
    int np = (int)(p1 - p0);
    int slots = (np + PPT - 1) / PPT;        // thread slots needed for the whole leaf
    int pr = slots < 128 ? slots : 128;      // threads per group
    int G = 128 / pr;                        // groups splitting the directions
    int grp = threadIdx.x / pr, pi = threadIdx.x % pr;
    bool active = grp < G;
    __shared__ int soct[PW_MAXD];
    if (threadIdx.x < P.A.shift) soct[threadIdx.x] = leaf_octant(P.A.leaf_g[leaf], P.A.shift, threadIdx.x);
    const C2 *va = vt + ((size_t)a * nrhs + m) * P.nQ;
    for (int pb = 0; pb < np; pb += pr * PPT) {
        decltype(Coord<R>::get(float4(), nullptr, 0u)) e[PPT];
        bool valid[PPT];
        R sr[PPT], si[PPT], lr[PPT], li[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            int idx = pb + pi + u * pr;
            valid[u] = active && idx < np;
            float4 eh = valid[u] ? P.A.eps[p0 + idx] : make_float4(0.f, 0.f, 0.f, 0.f);
            e[u] = Coord<R>::get(eh, P.eps_lo, valid[u] ? p0 + idx : 0u);
            sr[u] = si[u] = lr[u] = li[u] = 0;
        }
        int nH = P.nQ / 2;
        for (int qb = 0; qb < nH; qb += QC) {
            int qc = min(QC, nH - qb);
            __syncthreads();
            for (int j = threadIdx.x; j < qc; j += blockDim.x) {
                sk[j] = P.ks[qb + j];
                backward_weights(va[qb + j], va[qb + j + nH], leaf_factor<false>(P, soct, qb + j), sA[j], sB[j]);
            }
            __syncthreads();
            if (active) {
                int j0 = grp * qc / G, j1 = (grp + 1) * qc / G;  // this group's slice
#pragma unroll 2
                for (int j = j0; j < j1; ++j) {
                    K4 k4 = sk[j];
                    C2 A = sA[j], B = sB[j];
#pragma unroll
                    for (int u = 0; u < PPT; ++u) {
                        R ph = fma(k4.x, e[u].x, fma(k4.y, e[u].y, k4.z * e[u].z));
                        R sn, cs;
                        phase_sincos<PH>(ph, sn, cs, P.sctab);
                        if constexpr (COMP) {
                            two_sum_acc(sr[u], lr[u], fma(cs, A.x, sn * B.x));
                            two_sum_acc(si[u], li[u], fma(cs, A.y, sn * B.y));
                        } else {
                            sr[u] = fma(cs, A.x, fma(sn, B.x, sr[u]));
                            si[u] = fma(cs, A.y, fma(sn, B.y, si[u]));
                        }
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            red[threadIdx.x * PPT + u].x = sr[u];
            red[threadIdx.x * PPT + u].y = si[u];
            if constexpr (COMP) {
                redl[threadIdx.x * PPT + u].x = lr[u];
                redl[threadIdx.x * PPT + u].y = li[u];
            }
        }
        __syncthreads();
        if (active && grp == 0) {
#pragma unroll
            for (int u = 0; u < PPT; ++u) {
                if (!valid[u]) continue;
                double tr = 0, ti = 0;
                for (int g = 0; g < G; ++g) {
                    tr += (double)red[(g * pr + pi) * PPT + u].x;
                    ti += (double)red[(g * pr + pi) * PPT + u].y;
                    if constexpr (COMP) {
                        tr += (double)redl[(g * pr + pi) * PPT + u].x;
                        ti += (double)redl[(g * pr + pi) * PPT + u].y;
                    }
                }
                double2 &dst = acc[(int64_t)m * nx + p0 + pb + pi + u * pr];
                dst.x += tr;
                dst.y += ti;
            }
        }
    }
}

// ---- several right-hand sides: each phasor is computed once and applied to MC densities

// Forward transform for MC right-hand sides m0..m0+MC-1.  Thread owns one direction pair
// (h, h + nQ/2).  The leaf factor is folded into the phasor, e = F_leaf(h) e^{-i k s_h.e},
// and the antipode's phasor is conj(e) (the whole of F is conjugate-symmetric under
// s -> -s): with P = sum Re(e) w and Q = sum Im(e) w the two sums are P + iQ and P - iQ.
template <class R, int PH, int MC>
__global__ void __launch_bounds__(128) k_pw_forward_mr(PwArgs<R> P, const uint32_t *__restrict__ src,
                                                       const float2 *__restrict__ q, int64_t ny, int nrhs,
                                                       typename PwT<R>::C *__restrict__ ut) {
    typedef typename PwT<R>::C C2;
    constexpr int CH = 128;
    __shared__ float4 se[CH];
    __shared__ float4 sl[sizeof(R) == 8 ? CH : 1];
    __shared__ __align__(16) float2 sq[CH][MC];
    __shared__ int soct[PW_MAXD];
    static_assert(MC % 2 == 0, "right-hand sides are read in pairs");
    int b = src[blockIdx.x], m0 = blockIdx.z * MC;
    int nH = P.nQ / 2;
    int h = blockIdx.y * blockDim.x + threadIdx.x;
    bool on = h < nH;
    int hc = on ? h : 0;
    R kx = P.ks[hc].x, ky = P.ks[hc].y, kz = P.ks[hc].z;
    C2 Pc[MC], Qs[MC];
#pragma unroll
    for (int m = 0; m < MC; ++m) Pc[m] = Qs[m] = czero(R(0));
    uint32_t lf0 = P.A.box_leaf[b], lf1 = P.A.box_leaf[b + 1];
    for (uint32_t leaf = lf0; leaf < lf1; ++leaf) {
        uint32_t p0 = P.A.leaf_start[leaf], p1 = P.A.leaf_start[leaf + 1];
        C2 f = cone(R(0));
        for (uint32_t base = p0; base < p1; base += CH) {
            int cnt = (int)min((uint32_t)CH, p1 - base);
            __syncthreads();
            for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
                se[j] = P.A.eps[base + j];
                if constexpr (sizeof(R) == 8) sl[j] = P.eps_lo[base + j];
            }
            for (int e = threadIdx.x; e < cnt * MC; e += blockDim.x) {
                int j = e % cnt, m = e / cnt;
                sq[j][m] = (m0 + m < nrhs) ? q[(int64_t)(m0 + m) * ny + base + j] : make_float2(0.f, 0.f);
            }
            if (base == p0 && threadIdx.x < P.A.shift) soct[threadIdx.x] = leaf_octant(P.A.leaf_g[leaf], P.A.shift, threadIdx.x);
            __syncthreads();
            if (base == p0) f = leaf_factor<false>(P, soct, hc);
            for (int j = 0; j < cnt; ++j) {
                auto e3 = Coord<R>::get(se[j], sl, (uint32_t)j);
                R ph = fma(kx, e3.x, fma(ky, e3.y, kz * e3.z));
                R sn, cs;
                phase_sincos<PH>(ph, sn, cs, P.sctab);
                // e = f e^{-i ph}
                R er = fma(f.x, cs, f.y * sn), ei = fma(f.y, cs, -f.x * sn);
                // densities of two right-hand sides per 16-byte read
                const float4 *sq4 = reinterpret_cast<const float4 *>(&sq[j][0]);
#pragma unroll
                for (int m2 = 0; m2 < MC / 2; ++m2) {
                    float4 w2 = sq4[m2];
                    int m = 2 * m2;
                    Pc[m].x = fma(er, (R)w2.x, Pc[m].x);
                    Pc[m].y = fma(er, (R)w2.y, Pc[m].y);
                    Qs[m].x = fma(ei, (R)w2.x, Qs[m].x);
                    Qs[m].y = fma(ei, (R)w2.y, Qs[m].y);
                    Pc[m + 1].x = fma(er, (R)w2.z, Pc[m + 1].x);
                    Pc[m + 1].y = fma(er, (R)w2.w, Pc[m + 1].y);
                    Qs[m + 1].x = fma(ei, (R)w2.z, Qs[m + 1].x);
                    Qs[m + 1].y = fma(ei, (R)w2.w, Qs[m + 1].y);
                }
            }
        }
    }
    if (on)
#pragma unroll
        for (int m = 0; m < MC; ++m)
            if (m0 + m < nrhs) {
                C2 *o = ut + ((size_t)b * nrhs + m0 + m) * P.nQ;
                C2 v, vb;
                v.x = Pc[m].x - Qs[m].y;
                v.y = Pc[m].y + Qs[m].x;
                vb.x = Pc[m].x + Qs[m].y;
                vb.y = Pc[m].y - Qs[m].x;
                o[h] = v;
                o[h + nH] = vb;
            }
}

// Backward transform for MC right-hand sides: one block per target leaf, one thread per
// target point (looping over the leaf), direction pairs staged in shared memory as the
// (A, B) weights of backward_weights.  Compensated mode: TwoSum over the directions.
template <class R, int PH, int MC>
__global__ void __launch_bounds__(128) k_pw_backward_mr(PwArgs<R> P, const uint32_t *__restrict__ box_fine,
                                                        int64_t nbox, const uint32_t *__restrict__ leaf_fine,
                                                        const int *__restrict__ slot,
                                                        const typename PwT<R>::C *__restrict__ vt, int nrhs,
                                                        int64_t nx, double2 *__restrict__ acc) {
    typedef typename PwT<R>::C C2;
    typedef typename PwT<R>::K K4;
    constexpr bool COMP = PH == PH_ACC && sizeof(R) == 4;
    constexpr int QC = 64;
    __shared__ K4 sk[QC];
    // (A, B) of a direction pair and right-hand side side by side: one 16-byte read (FP32)
    struct __align__(16) AB {
        C2 A, B;
    };
    __shared__ AB sw[QC][MC];
    __shared__ int soct[PW_MAXD];
    int leaf = blockIdx.x, m0 = blockIdx.z * MC;
    uint32_t lf = leaf_fine[leaf];
    int64_t lo = 0, hi = nbox - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (box_fine[mid] <= lf)
            lo = mid;
        else
            hi = mid - 1;
    }
    int a = (int)lo;
    if (slot[a] < 0) return;
    if (threadIdx.x < P.A.shift) soct[threadIdx.x] = leaf_octant(P.A.leaf_g[leaf], P.A.shift, threadIdx.x);
    uint32_t p0 = P.A.leaf_start[leaf], p1 = P.A.leaf_start[leaf + 1];
    int np = (int)(p1 - p0);
    int nH = P.nQ / 2;
    for (int pb = 0; pb < np; pb += blockDim.x) {
        bool valid = pb + (int)threadIdx.x < np;
        float4 eh = valid ? P.A.eps[p0 + pb + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
        auto e3 = Coord<R>::get(eh, P.eps_lo, valid ? p0 + pb + threadIdx.x : 0u);
        C2 o[MC], ol[MC];
#pragma unroll
        for (int m = 0; m < MC; ++m) o[m] = ol[m] = czero(R(0));
        for (int qb = 0; qb < nH; qb += QC) {
            int qc = min(QC, nH - qb);
            __syncthreads();
            for (int e = threadIdx.x; e < qc * MC; e += blockDim.x) {
                int j = e % qc, m = e / qc;
                if (m0 + m < nrhs) {
                    const C2 *va = vt + ((size_t)a * nrhs + m0 + m) * P.nQ;
                    backward_weights(va[qb + j], va[qb + j + nH], leaf_factor<false>(P, soct, qb + j), sw[j][m].A,
                                     sw[j][m].B);
                } else {
                    sw[j][m].A = czero(R(0));
                    sw[j][m].B = czero(R(0));
                }
                if (m == 0) sk[j] = P.ks[qb + j];
            }
            __syncthreads();
            if (valid) {
                for (int j = 0; j < qc; ++j) {
                    K4 k4 = sk[j];
                    R ph = fma(k4.x, e3.x, fma(k4.y, e3.y, k4.z * e3.z));
                    R sn, cs;
                    phase_sincos<PH>(ph, sn, cs, P.sctab);
#pragma unroll
                    for (int m = 0; m < MC; ++m) {
                        AB w = sw[j][m];
                        C2 A = w.A, B = w.B;
                        if constexpr (COMP) {
                            two_sum_acc(o[m].x, ol[m].x, fma(cs, A.x, sn * B.x));
                            two_sum_acc(o[m].y, ol[m].y, fma(cs, A.y, sn * B.y));
                        } else {
                            o[m].x = fma(cs, A.x, fma(sn, B.x, o[m].x));
                            o[m].y = fma(cs, A.y, fma(sn, B.y, o[m].y));
                        }
                    }
                }
            }
        }
        if (valid)
#pragma unroll
            for (int m = 0; m < MC; ++m)
                if (m0 + m < nrhs) {
                    double2 &dst = acc[(int64_t)(m0 + m) * nx + p0 + pb + threadIdx.x];
                    dst.x += (double)o[m].x + (COMP ? (double)ol[m].x : 0.0);
                    dst.y += (double)o[m].y + (COMP ? (double)ol[m].y : 0.0);
                }
    }
}

__global__ void k_slot_init(int *slot, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot[i] = -1;
}
__global__ void k_slot_set(const uint32_t *__restrict__ tgt, int64_t n, int *slot) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot[tgt[i]] = (int)i;
}

// ---- several right-hand sides on the tensor cores (FP32 and compensated-FP32 plane-wave levels)
//
// The forward transform of a source box b is a product of a generated matrix and the
// densities: for direction pairs h (antipodes h, h + nQ/2) and right-hand sides m,
//   P(h, m) = sum_j Re(e_hj) w_jm,   Q(h, m) = sum_j Im(e_hj) w_jm,
//   e_hj = F_leaf(j)(h) e^{-i k s_h . e_j}   (leaf-centred phase times the leaf's octant factor),
// and u~(h) = P + iQ, u~(h + nQ/2) = P - iQ per right-hand side (the antipode's phasor is the
// conjugate).  With the complex densities written as 2 real columns per right-hand side,
// both are real GEMMs of M = direction pairs, N = 2 x right-hand sides, K = points.
//
// k_pw_forward_tc: a CTA takes 128 direction pairs (TMEM lanes), 64 right-hand sides (N =
// 128) and one chunk of at most PWT_CH points of a box, in steps of 32 points aligned to the
// density image's 32-point blocks (points outside the chunk get phasor 0).  Warps 1-16
// produce, four threads per direction pair h (8 points of the step each): a thread forms
// its 8 phasors (one sincos each, the leaf factor kept while the leaf does not change),
// splits Re and Im into TF32 hi and lo and writes them into one of two TMEM operand stages
// (tcgen05.st); one producer also starts a bulk copy of the step's density block (hi and
// lo, K-major, 32 KB) two steps ahead into one of four shared stages.  One thread of warp 0
// issues per 8 points hi hi + hi lo + lo hi for P and for Q (6 MMAs, M = 128, N = 128, K =
// 8, A from TMEM) and commits to the stage's "empty" barrier.  The epilogue reads P and Q
// from TMEM and adds u~ into the output (atomics: a box may be split over several chunks;
// the output is zeroed first).  The TF32 x3 products are off by at most about 2^-21 of each
// term, 2^-25 typically (the dropped lo lo product and the rounding of the lo parts).
constexpr int PWT_M = 128;                 // direction pairs per CTA
constexpr int PWT_KC = 32;                 // points per step
constexpr int PWT_MC = 64;                 // right-hand sides per CTA
constexpr int PWT_N = 2 * PWT_MC;          // GEMM columns (re, im of each right-hand side)
constexpr int PWT_CH = PW_TC_FCH;          // points per chunk of a box
constexpr int PWT_NA = 2;                  // A stages (tensor memory)
constexpr int PWT_DB = 2;                  // steps the density copies run ahead
constexpr int PWT_QS = 4;                  // producer threads per direction pair
constexpr int PWT_PP = PWT_KC / PWT_QS;    // points per producer thread and step
constexpr int PWT_NP = PWT_QS * PWT_M;     // producer threads (warps 1-16)
constexpr int PWT_NB = PWT_NA + PWT_DB;    // density stages (shared memory)
constexpr int PWT_BH = PWT_N * PWT_KC;     // floats per density hi or lo block
constexpr int PWT_BST = 2 * PWT_BH;        // floats per density stage (32 KB)
constexpr int PWT_TCOLS = 512;             // TMEM: P 128 + Q 128 columns, 2 A stages x 128
constexpr size_t PWT_SMEM = sizeof(float) * (size_t)PWT_NB * PWT_BST;  // 128 KB: one CTA per SM

// Density image: for every block of 32 consecutive points (Morton order) and every group of
// 64 right-hand sides, the TF32 hi block then the lo block of the K-major operand (rows n =
// 2 m + part, part 0 = real, 1 = imaginary; columns = the block's points), zero beyond ny
// and nrhs.  Its layout does not depend on the level; each tensor-core level builds it.
__global__ void k_pw_density_image(const float2 *__restrict__ q, int64_t ny, int nrhs, int nblk_m,
                                   float *__restrict__ img) {
    const int64_t nimg = (int64_t)((ny + PWT_KC - 1) / PWT_KC) * nblk_m * PWT_BH;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nimg; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = i / PWT_BH;  // (point block, right-hand-side group)
        const int e = (int)(i - blk * PWT_BH);
        const int n = e / PWT_KC, k = e % PWT_KC;
        const int64_t c = blk / nblk_m;
        const int mb = (int)(blk - c * nblk_m);
        const int64_t j = c * PWT_KC + k;
        const int mm = mb * PWT_MC + (n >> 1);
        float v = 0.f;
        if (j < ny && mm < nrhs) {
            float2 w = q[(int64_t)mm * ny + j];
            v = (n & 1) ? w.y : w.x;
        }
        float h, l;
        tf32_split(v, h, l);
        const uint32_t o = kmajor_index(n, k, PWT_KC);
        img[blk * 2 * PWT_BH + o] = h;
        img[blk * 2 * PWT_BH + PWT_BH + o] = l;
    }
}


// Leaf factor F_leaf(h) = prod_d E[d][oct_d][h] of one direction (octant path from the
// leaf's integer coordinates), in the order of leaf_factor.
__device__ __forceinline__ float2 leaf_factor_dir(const PwArgs<float> &P, uint32_t leaf, int h) {
    const int4 gl = P.A.leaf_g[leaf];
    float2 f = make_float2(1.f, 0.f);
    for (int d = 0; d < P.A.shift; ++d) f = cmul(f, P.E[((size_t)d * 8 + leaf_octant(gl, P.A.shift, d)) * P.nQ + h]);
    return f;
}

template <int PH>
__global__ void __launch_bounds__(PWT_NP + 32, 1) k_pw_forward_tc(PwArgs<float> P, const uint2 *__restrict__ chunks,
                                                         const float *__restrict__ img, int nblk_m, int nrhs,
                                                         float2 *__restrict__ ut, int *__restrict__ err, int tries) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float *bring = reinterpret_cast<float *>(smem);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bfull[PWT_NB], s_empty[PWT_NB], s_afull[PWT_NA];
    __shared__ int s_bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // blocks run the direction tiles of a chunk side by side: they share its density blocks
    // in L2, and their atomic additions go to distinct directions
    const int ntile = (P.nQ / 2 + PWT_M - 1) / PWT_M;
    const int tile = (int)(blockIdx.x % (unsigned)ntile);
    const uint2 ck = chunks[blockIdx.x / (unsigned)ntile];
    const int b = (int)ck.x;
    const uint32_t p0 = ck.y, p1 = min(P.A.box_start[b + 1], p0 + (uint32_t)PWT_CH);
    const bool sole = p0 == P.A.box_start[b] && p1 == P.A.box_start[b + 1];
    const int mb = blockIdx.z, nH = P.nQ / 2;
    const uint32_t c0 = p0 / PWT_KC;
    const int nsteps = (int)((p1 + PWT_KC - 1) / PWT_KC - c0);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(PWT_TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_bad = 0;
        for (int i = 0; i < PWT_NB; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_empty[i])));
        }
        for (int i = 0; i < PWT_NA; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&s_afull[i])), "r"(PWT_NP));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    bool ok = true;
    if (warp >= 1) {
        // producer of direction pair h (TMEM lane row), points PWT_PP qq .. PWT_PP (qq + 1) - 1
        // of each step
        const int dq = warp & 3, qq = (warp - 1) >> 2, row = dq * 32 + lane, h = tile * PWT_M + row;
        const bool on = h < nH;
        const float4 kv = P.ks[on ? h : 0];
        int last_b = -1;  // last density copy issued (producer 0)
        auto copy_b = [&](int sp) {
            if (tid != 32 || sp >= nsteps) return;
            uint64_t *bar = &s_bfull[sp % PWT_NB];
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                         "r"((uint32_t)(PWT_BST * sizeof(float)))
                         : "memory");
            bulk_g2s(bring + (size_t)(sp % PWT_NB) * PWT_BST, img + ((size_t)(c0 + sp) * nblk_m + mb) * PWT_BST,
                     (uint32_t)(PWT_BST * sizeof(float)), bar);
            last_b = sp;
        };
        for (int sp = 0; sp < PWT_DB; ++sp) copy_b(sp);
        uint32_t cur_leaf = 0xffffffffu;
        float2 f = make_float2(1.f, 0.f);
        for (int s = 0; s < nsteps && ok; ++s) {
            if (s >= PWT_NA) {
                // the MMAs of step s - PWT_NA are done: its A stage and density stage are free
                const int sb = s - PWT_NA;
                bool w_ok = mbar_wait(&s_empty[sb % PWT_NB], (uint32_t)((sb / PWT_NB) & 1), tries, err);
                if (!__all_sync(0xffffffffu, w_ok)) {
                    ok = false;
                    break;
                }
            }
            copy_b(s + PWT_DB);
            const uint32_t jb = (c0 + (uint32_t)s) * PWT_KC + (uint32_t)(PWT_PP * qq);
            const uint32_t ta =
                tmem + (uint32_t)(256 + (s % PWT_NA) * 128 + PWT_PP * qq) + ((uint32_t)(dq * 32) << 16);
            {
                // the points' coordinates first (one latency for all), then the phasors
                float4 ev[PWT_PP];
#pragma unroll
                for (int i = 0; i < PWT_PP; ++i)
                    ev[i] = (jb + i >= p0 && jb + i < p1) ? P.A.eps[jb + i] : make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t rh[PWT_PP], rl[PWT_PP], ih[PWT_PP], il[PWT_PP];
#pragma unroll
                for (int i = 0; i < PWT_PP; ++i) {
                    const uint32_t j = jb + i;
                    float er = 0.f, ei = 0.f;
                    if (on && j >= p0 && j < p1) {
                        const float4 e = ev[i];
                        const uint32_t leaf = __float_as_uint(e.w);
                        if (leaf != cur_leaf) {
                            f = leaf_factor_dir(P, leaf, h);
                            cur_leaf = leaf;
                        }
                        const float ph = fmaf(kv.x, e.x, fmaf(kv.y, e.y, kv.z * e.z));
                        float sn, cs;
                        phase_sincos<PH>(ph, sn, cs, nullptr);
                        er = fmaf(f.x, cs, f.y * sn);  // e = f e^{-i ph}
                        ei = fmaf(f.y, cs, -f.x * sn);
                    }
                    float a, c;
                    tf32_split(er, a, c);
                    rh[i] = __float_as_uint(a);
                    rl[i] = __float_as_uint(c);
                    tf32_split(ei, a, c);
                    ih[i] = __float_as_uint(a);
                    il[i] = __float_as_uint(c);
                }
                tmem_st8(ta, rh);
                tmem_st8(ta + 32u, rl);
                tmem_st8(ta + 64u, ih);
                tmem_st8(ta + 96u, il);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&s_afull[s % PWT_NA])) : "memory");
        }
        if (ok) {
            // every MMA done (the last commit completes after the others): u~ from P and Q
            const int l = nsteps - 1;
            bool w_ok = mbar_wait(&s_empty[l % PWT_NB], (uint32_t)((l / PWT_NB) & 1), tries, err);
            if (!__all_sync(0xffffffffu, w_ok)) ok = false;
        }
        if (ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t lanes = (uint32_t)(dq * 32) << 16;
#pragma unroll 1
            for (int c8 = qq * PWT_MC / (8 * PWT_QS); c8 < (qq + 1) * PWT_MC / (8 * PWT_QS); ++c8) {
                uint32_t pv[16], qv[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(pv[0]), "=r"(pv[1]), "=r"(pv[2]), "=r"(pv[3]), "=r"(pv[4]), "=r"(pv[5]), "=r"(pv[6]),
                      "=r"(pv[7]), "=r"(pv[8]), "=r"(pv[9]), "=r"(pv[10]), "=r"(pv[11]), "=r"(pv[12]), "=r"(pv[13]),
                      "=r"(pv[14]), "=r"(pv[15])
                    : "r"(tmem + lanes + (uint32_t)(16 * c8)));
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(qv[0]), "=r"(qv[1]), "=r"(qv[2]), "=r"(qv[3]), "=r"(qv[4]), "=r"(qv[5]), "=r"(qv[6]),
                      "=r"(qv[7]), "=r"(qv[8]), "=r"(qv[9]), "=r"(qv[10]), "=r"(qv[11]), "=r"(qv[12]), "=r"(qv[13]),
                      "=r"(qv[14]), "=r"(qv[15])
                    : "r"(tmem + lanes + 128u + (uint32_t)(16 * c8)));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int mm = 0; mm < 8; ++mm) {
                    const int m = mb * PWT_MC + c8 * 8 + mm;
                    if (!on || m >= nrhs) continue;
                    const float pr = __uint_as_float(pv[2 * mm]), pi = __uint_as_float(pv[2 * mm + 1]);
                    const float qr = __uint_as_float(qv[2 * mm]), qi = __uint_as_float(qv[2 * mm + 1]);
                    float2 *o = ut + ((size_t)b * nrhs + m) * P.nQ;
                    if (sole) {
                        o[h] = make_float2(pr - qi, pi + qr);
                        o[h + nH] = make_float2(pr + qi, pi - qr);
                    } else {
                        atomicAdd(&o[h].x, pr - qi);
                        atomicAdd(&o[h].y, pi + qr);
                        atomicAdd(&o[h + nH].x, pr + qi);
                        atomicAdd(&o[h + nH].y, pi - qr);
                    }
                }
            }
        } else {
            s_bad = 1;
            // density copies in flight complete on their own: wait for the last one issued
            // into each stage
            for (int sp = max(0, last_b - PWT_NB + 1); sp <= last_b; ++sp)
                mbar_wait(&s_bfull[sp % PWT_NB], (uint32_t)((sp / PWT_NB) & 1), DRAIN_TRIES);
        }
    } else if (lane == 0) {
        // ---- MMA thread: per 8 points, P += Re hi B hi + Re hi B lo + Re lo B hi, and Q likewise
        const uint32_t lbo = 128, sbo = (PWT_KC / 4) * 128;
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(PWT_N >> 3) << 17) |
                               ((uint32_t)(PWT_M >> 4) << 24);
        int issued = 0;
        for (int s = 0; s < nsteps; ++s) {
            if (!mbar_wait(&s_bfull[s % PWT_NB], (uint32_t)((s / PWT_NB) & 1), tries, err) ||
                !mbar_wait(&s_afull[s % PWT_NA], (uint32_t)((s / PWT_NA) & 1), tries, err)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = tmem + (uint32_t)(256 + (s % PWT_NA) * 128);
            const uint32_t bst = smem_addr(bring + (size_t)(s % PWT_NB) * PWT_BST);
#pragma unroll
            for (int ks = 0; ks < PWT_KC / 8; ++ks) {
                const uint64_t bh = umma_desc(bst + ks * 256, lbo, sbo);
                const uint64_t bl = umma_desc(bst + PWT_BH * 4 + ks * 256, lbo, sbo);
                const uint32_t acc0 = (s > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
                for (int pq = 0; pq < 2; ++pq) {  // P from Re (columns 0..63 of the stage), Q from Im (64..127)
                    const uint32_t d = tmem + (uint32_t)(128 * pq);
                    const uint32_t ah = a0 + (uint32_t)(64 * pq + ks * 8), al = ah + 32u;
                    asm volatile(
                        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
                        "r"(ah), "l"(bh), "r"(idesc), "r"(acc0));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(d), "r"(ah),
                                 "l"(bl), "r"(idesc));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(d), "r"(al),
                                 "l"(bh), "r"(idesc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&s_empty[s % PWT_NB]))
                         : "memory");
            issued = s + 1;
        }
        if (!ok) {
            s_bad = 1;
            if (issued > 0)
                mbar_wait(&s_empty[(issued - 1) % PWT_NB], (uint32_t)(((issued - 1) / PWT_NB) & 1), DRAIN_TRIES);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PWT_TCOLS));
}

// The backward transform of a target box a is the transposed product: for a point x of the
// box (leaf-relative coordinate e_x) and right-hand side m,
//   v(x, m) = sum_h g_xh a_hm + conj(g_xh) b_hm,   g_xh = e^{i k s_h . e_x} conj(F_leaf(x)(h)),
// with a = v~_a(h), b = v~_a(h + nQ/2).  With S = a + b and D = a - b,
//   Re v = sum_h Re(g) Re(S) - Im(g) Im(D),   Im v = sum_h Re(g) Im(S) + Im(g) Re(D):
// a real GEMM of M = points, K = 2 x direction pairs (Re g, Im g of each), N = 2 x
// right-hand sides, whose B operand (S and D of the box) is shared by all its points.
// k_pw_vt_image writes that operand per target box, per step of 16 direction pairs and per
// group of 64 right-hand sides, split into TF32 hi and lo blocks in the K-major layout.
//
// k_pw_backward_tc: a CTA takes 128 points of one target box (TMEM lanes) and 64 right-hand
// sides.  Warps 1-16 produce, four threads per point (4 direction pairs of each step each):
// a thread forms Re g and Im g (its leaf's octant factors from the E table, one sincos),
// splits them and writes them into one of three TMEM operand stages; one producer copies the
// box's B block of the step (32 KB, bulk copy) into one of five shared stages two steps
// ahead.  One thread of warp 0 issues hi hi + hi lo + lo hi per 8 K values (12 MMAs of M =
// 128, N = 128, K = 8 per step).  The sum over directions alternates between two TMEM
// accumulators every PWB_DRAIN steps; the producers add each finished one into FP32
// registers while the other fills (the same protocol as the target-stationary transfer),
// and add their sums into the point's FP64 accumulator at the end.
constexpr int PWB_M = PW_TC_BCH;         // points per CTA
constexpr int PWB_KC = 32;               // K values per step (16 direction pairs)
constexpr int PWB_N = 128;               // GEMM columns: re, im of 64 right-hand sides
constexpr int PWB_MC = PWB_N / 2;
constexpr int PWB_NA = 3;                // A stages (tensor memory)
constexpr int PWB_DB = 2;                // steps the B copies run ahead
constexpr int PWB_NB = PWB_NA + PWB_DB;  // B stages (shared memory)
constexpr int PWB_DRAIN = 8;             // steps per TMEM accumulator fill
constexpr int PWB_QS = 4;                // producer threads per point
constexpr int PWB_HP = PWB_KC / 2 / PWB_QS;  // direction pairs per producer thread and step
constexpr int PWB_SC = PWB_N / PWB_QS;   // accumulator columns per producer thread
constexpr int PWB_NP = PWB_QS * PWB_M;   // producer threads (warps 1-16)
static_assert(PWB_HP == 4, "a producer reads its octant factors as two float4");
constexpr int PWB_BH = PWB_N * PWB_KC;   // floats per B hi or lo block
constexpr int PWB_BST = 2 * PWB_BH;      // floats per B stage (32 KB)
constexpr int PWB_TCOLS = 512;           // TMEM: 2 accumulators x 128, 3 A stages x 64
constexpr size_t PWB_SMEM = sizeof(float) * (size_t)PWB_NB * PWB_BST;  // 160 KB

// B operand of the backward GEMM: block (target t, step st, group mb) at
// ((t nsteps + st) nblk_m + mb) 2 PWB_BH, hi then lo; row n = 2 m + (0: Re, 1: Im), column
// k = 2 (h - 16 st) + (0: Re g, 1: Im g); zero past nH and nrhs.
__global__ void k_pw_vt_image(const float2 *__restrict__ vt, const uint32_t *__restrict__ tgt, int64_t n_tgt,
                              int nrhs, int nQ, int nsteps, int nblk_m, float *__restrict__ img) {
    const int nH = nQ / 2;
    const int64_t nimg = n_tgt * nsteps * nblk_m * (int64_t)PWB_BH;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nimg; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = i / PWB_BH;
        const int e = (int)(i - blk * PWB_BH);
        const int n = e / PWB_KC, k = e % PWB_KC;
        const int64_t tb = blk / nblk_m;
        const int mb = (int)(blk - tb * nblk_m);
        const int64_t t = tb / nsteps;
        const int st = (int)(tb - t * nsteps);
        const int h = st * (PWB_KC / 2) + (k >> 1), m = mb * PWB_MC + (n >> 1);
        float v = 0.f;
        if (h < nH && m < nrhs) {
            const float2 *va = vt + ((size_t)tgt[t] * nrhs + m) * nQ;
            const float2 a = va[h], b = va[h + nH];
            if ((k & 1) == 0)
                v = (n & 1) ? a.y + b.y : a.x + b.x;  // Re g row: S
            else
                v = (n & 1) ? a.x - b.x : b.y - a.y;  // Im g row: (-Im D, Re D)
        }
        float hi, lo;
        tf32_split(v, hi, lo);
        const uint32_t o = kmajor_index(n, k, PWB_KC);
        img[blk * 2 * PWB_BH + o] = hi;
        img[blk * 2 * PWB_BH + PWB_BH + o] = lo;
    }
}

template <int PH>
__global__ void __launch_bounds__(PWB_NP + 32, 1) k_pw_backward_tc(PwArgs<float> P, const uint2 *__restrict__ chunks,
                                                                  const int *__restrict__ slot,
                                                                  const float *__restrict__ img, int nblk_m,
                                                                  int nrhs, int64_t nx, double2 *__restrict__ acc,
                                                                  int *__restrict__ err, int tries) {
    extern __shared__ __align__(1024) unsigned char smem[];
    float *bring = reinterpret_cast<float *>(smem);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bfull[PWB_NB], s_empty[PWB_NB], s_afull[PWB_NA], s_drained;
    __shared__ int s_bad;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint2 ck = chunks[blockIdx.x];
    const int a = (int)ck.x, mb = blockIdx.y;
    const uint32_t x0 = ck.y, x1 = min(P.A.box_start[a + 1], x0 + (uint32_t)PWB_M);
    const int nH = P.nQ / 2;
    const int nsteps = (nH + PWB_KC / 2 - 1) / (PWB_KC / 2);
    const float *bimg = img + (size_t)slot[a] * nsteps * nblk_m * PWB_BST;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(PWB_TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_bad = 0;
        for (int i = 0; i < PWB_NB; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bfull[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_empty[i])));
        }
        for (int i = 0; i < PWB_NA; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&s_afull[i])), "r"(PWB_NP));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&s_drained)), "r"(PWB_NP));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    bool ok = true;
    if (warp >= 1) {
        // producer of point x (TMEM lane row), direction pairs PWB_HP qq .. PWB_HP (qq + 1) - 1
        // of each step, accumulator columns PWB_SC qq .. PWB_SC (qq + 1) - 1
        const int dq = warp & 3, qq = (warp - 1) >> 2, row = dq * 32 + lane;
        const uint32_t x = x0 + (uint32_t)row;
        const bool on = x < x1;
        const float4 e = P.A.eps[on ? x : x0];
        uint64_t oct = 0;  // octant path of the point's leaf, 3 bits per level
        {
            const int4 gl = P.A.leaf_g[__float_as_uint(e.w)];
            for (int d = 0; d < P.A.shift; ++d) oct |= (uint64_t)leaf_octant(gl, P.A.shift, d) << (3 * d);
        }
        float sum[PWB_SC];
#pragma unroll
        for (int c = 0; c < PWB_SC; ++c) sum[c] = 0.f;
        int drained = 0;
        auto drain = [&](int k) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base =
                tmem + (uint32_t)((k & 1) * 128 + qq * PWB_SC) + ((uint32_t)(dq * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < PWB_SC; c0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(base + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 16; ++q) sum[c0 + q] += __uint_as_float(v[q]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&s_drained)) : "memory");
        };
        int last_b = -1;
        auto copy_b = [&](int sp) {
            if (tid != 32 || sp >= nsteps) return;
            uint64_t *bar = &s_bfull[sp % PWB_NB];
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                         "r"((uint32_t)(PWB_BST * sizeof(float)))
                         : "memory");
            bulk_g2s(bring + (size_t)(sp % PWB_NB) * PWB_BST, bimg + ((size_t)sp * nblk_m + mb) * PWB_BST,
                     (uint32_t)(PWB_BST * sizeof(float)), bar);
            last_b = sp;
        };
        for (int sp = 0; sp < PWB_DB; ++sp) copy_b(sp);
        for (int s = 0; s < nsteps && ok; ++s) {
            if (s >= PWB_NA) {
                // the MMAs of step s - PWB_NA are done: its A and B stages are free; fill k is
                // drained once the first step of fill k + 1 is done (see k_lag_gemm_ts)
                const int sb = s - PWB_NA;
                bool w_ok = mbar_wait(&s_empty[sb % PWB_NB], (uint32_t)((sb / PWB_NB) & 1), tries, err);
                if (!__all_sync(0xffffffffu, w_ok)) {
                    ok = false;
                    break;
                }
                const int done = sb / PWB_DRAIN;
                while (drained < done) drain(drained++);
            }
            copy_b(s + PWB_DB);
            // leaf factors of this thread's PWB_HP directions (one row of the octant factors per
            // level, consecutive directions), then the phasors
            const int h0 = s * (PWB_KC / 2) + PWB_HP * qq;
            const bool full = h0 + PWB_HP <= nH;
            float2 f[PWB_HP];
#pragma unroll
            for (int i = 0; i < PWB_HP; ++i) f[i] = make_float2(1.f, 0.f);
            if (on && full) {
#pragma unroll 2
                for (int d = 0; d < P.A.shift; ++d) {
                    const float4 *er = reinterpret_cast<const float4 *>(
                        P.E + (uint32_t)(d * 8 + (int)((oct >> (3 * d)) & 7)) * (uint32_t)P.nQ + (uint32_t)h0);
                    const float4 e01 = __ldg(er), e23 = __ldg(er + 1);
                    f[0] = cmul(f[0], make_float2(e01.x, e01.y));
                    f[1] = cmul(f[1], make_float2(e01.z, e01.w));
                    f[2] = cmul(f[2], make_float2(e23.x, e23.y));
                    f[3] = cmul(f[3], make_float2(e23.z, e23.w));
                }
            } else if (on) {
                for (int i = 0; i < PWB_HP && h0 + i < nH; ++i)
                    for (int d = 0; d < P.A.shift; ++d)
                        f[i] = cmul(f[i], P.E[(uint32_t)(d * 8 + (int)((oct >> (3 * d)) & 7)) * (uint32_t)P.nQ +
                                             (uint32_t)(h0 + i)]);
            }
            uint32_t hv[2 * PWB_HP], lv[2 * PWB_HP];
#pragma unroll
            for (int i = 0; i < PWB_HP; ++i) {
                const int h = h0 + i;
                float gr = 0.f, gi = 0.f;
                if (on && h < nH) {
                    const float4 kv = P.ks[h];
                    const float ph = fmaf(kv.x, e.x, fmaf(kv.y, e.y, kv.z * e.z));
                    float sn, cs;
                    phase_sincos<PH>(ph, sn, cs, nullptr);
                    gr = fmaf(cs, f[i].x, sn * f[i].y);  // g = e^{i ph} conj(f)
                    gi = fmaf(sn, f[i].x, -cs * f[i].y);
                }
                float hi, lo;
                tf32_split(gr, hi, lo);
                hv[2 * i] = __float_as_uint(hi);
                lv[2 * i] = __float_as_uint(lo);
                tf32_split(gi, hi, lo);
                hv[2 * i + 1] = __float_as_uint(hi);
                lv[2 * i + 1] = __float_as_uint(lo);
            }
            const uint32_t ta =
                tmem + (uint32_t)(256 + (s % PWB_NA) * 64 + 2 * PWB_HP * qq) + ((uint32_t)(dq * 32) << 16);
            tmem_st8(ta, hv);
            tmem_st8(ta + 32u, lv);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&s_afull[s % PWB_NA])) : "memory");
        }
        if (ok) {
            const int l = nsteps - 1;
            bool w_ok = mbar_wait(&s_empty[l % PWB_NB], (uint32_t)((l / PWB_NB) & 1), tries, err);
            if (!__all_sync(0xffffffffu, w_ok)) ok = false;
            const int fills = (nsteps + PWB_DRAIN - 1) / PWB_DRAIN;
            while (ok && drained < fills) drain(drained++);
        }
        if (!ok) {
            s_bad = 1;
            for (int sp = max(0, last_b - PWB_NB + 1); sp <= last_b; ++sp)  // copies still in flight
                mbar_wait(&s_bfull[sp % PWB_NB], (uint32_t)((sp / PWB_NB) & 1), DRAIN_TRIES);
        } else if (on) {
#pragma unroll
            for (int j = 0; j < PWB_SC / 2; ++j) {
                const int m = mb * PWB_MC + (PWB_SC / 2) * qq + j;
                if (m < nrhs) {
                    double2 &dst = acc[(int64_t)m * nx + x];
                    dst.x += (double)sum[2 * j];
                    dst.y += (double)sum[2 * j + 1];
                }
            }
        }
    } else if (lane == 0) {
        // ---- MMA thread
        const uint32_t lbo = 128, sbo = (PWB_KC / 4) * 128;
        const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(PWB_N >> 3) << 17) |
                               ((uint32_t)(PWB_M >> 4) << 24);
        int issued = 0;
        for (int s = 0; s < nsteps; ++s) {
            const int fill = s / PWB_DRAIN;
            if (s % PWB_DRAIN == 0 && fill >= 2 && !mbar_wait(&s_drained, (uint32_t)((fill - 2) & 1), tries, err)) {
                ok = false;
                break;
            }
            if (!mbar_wait(&s_bfull[s % PWB_NB], (uint32_t)((s / PWB_NB) & 1), tries, err) ||
                !mbar_wait(&s_afull[s % PWB_NA], (uint32_t)((s / PWB_NA) & 1), tries, err)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + (uint32_t)((fill & 1) * 128);
            const uint32_t a0 = tmem + (uint32_t)(256 + (s % PWB_NA) * 64);
            const uint32_t bst = smem_addr(bring + (size_t)(s % PWB_NB) * PWB_BST);
#pragma unroll
            for (int ks = 0; ks < PWB_KC / 8; ++ks) {
                const uint32_t ah = a0 + (uint32_t)(ks * 8), al = ah + 32u;
                const uint64_t bh = umma_desc(bst + ks * 256, lbo, sbo);
                const uint64_t bl = umma_desc(bst + PWB_BH * 4 + ks * 256, lbo, sbo);
                const uint32_t acc0 = (s % PWB_DRAIN != 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
                    "r"(ah), "l"(bh), "r"(idesc), "r"(acc0));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(d), "r"(ah), "l"(bl),
                             "r"(idesc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, 1;\n" ::"r"(d), "r"(al), "l"(bh),
                             "r"(idesc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&s_empty[s % PWB_NB]))
                         : "memory");
            issued = s + 1;
        }
        if (!ok) {
            s_bad = 1;
            if (issued > 0)
                mbar_wait(&s_empty[(issued - 1) % PWB_NB], (uint32_t)(((issued - 1) / PWB_NB) & 1), DRAIN_TRIES);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && s_bad) atomicOr(err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PWB_TCOLS));
}

template <class R, int PH>
static void planewave_level(const ffm_plan_s *p, int l, const float2 *q, int nrhs, double2 *acc, Alloc &tmp,
                            cudaStream_t s, const typename PwT<R>::K *ks, const typename PwT<R>::C *D,
                            const typename PwT<R>::C *E) {
    typedef typename PwT<R>::C C2;
    constexpr bool COMP = PH == PH_ACC;
    const char *tag = std::is_same<R, double>::value ? "f64" : std::is_same<R, dd>::value ? "f32x2" : COMP ? "f32c" : "f32";
    auto name = [&](const char *k) {
        static thread_local char buf[64];
        snprintf(buf, sizeof buf, "%s<%s>", k, tag);
        return (const char *)buf;
    };
    const FarLevel &F = p->far[l];
    int ls = p->l_stop;
    PwArgs<R> PY{level_args(p, p->by[l], p->by[ls], p->epsY, l), p->epsYlo, ks, E, F.nQ, p->sctab};
    PwArgs<R> PX{level_args(p, p->bx[l], p->bx[ls], p->epsX, l), p->epsXlo, ks, E, F.nQ, p->sctab};
    C2 *ut = tmp.get<C2>((size_t)p->by[l].nb * nrhs * F.nQ);
    C2 *vt = tmp.get<C2>((size_t)p->bx[l].nb * nrhs * F.nQ);
    // kernel variants (autotuned; FP64 levels keep the defaults)
    constexpr bool dbl = sizeof(R) == 8;
    const int qpt = dbl ? 4 : F.pw_qpt, ppt = dbl ? 4 : F.pw_ppt, mc = dbl ? 8 : F.pw_mc;
    // threads per forward block: 128 unless the ragged tail of the direction range wastes
    // more than 10% of the lanes
    int tb = 128;
    int nH = F.nQ / 2;
    for (int cand : {64, 32})
        if ((double)cdiv(nH, tb * qpt) * tb * qpt > 1.1 * nH) tb = cand;
    bool multi = nrhs > 1;
    constexpr bool f32 = std::is_same<R, float>::value;
    // several right-hand sides on the tensor cores (TF32 x3): the forward transform on FP32
    // and compensated-FP32 levels, the backward transform on FP32 levels (the compensated
    // one carries its rounding error through the direction sum, which the tensor cores do not)
    const bool tc_fwd = f32 && multi && F.pw_chunks != nullptr &&
                        (p->pw_transform == 3 ||
                         (p->pw_transform == 0 && (F.pw_tc > 0 || (F.pw_tc < 0 && nrhs >= PW_TC_MIN_RHS))));
    const bool tc_bwd = tc_fwd && !COMP;
    if (f32 && F.nufft) {
        if constexpr (f32) nufft_forward(p, l, q, nrhs, ut, tmp, s);
    } else if (tc_fwd) {
        if constexpr (f32) {
            const int nblk_m = (int)cdiv(nrhs, PWT_MC);
            float *img = tmp.get<float>((size_t)cdiv(p->ny, PWT_KC) * nblk_m * PWT_BST);
            const int64_t nimg = (int64_t)cdiv(p->ny, PWT_KC) * nblk_m * PWT_BH;
            FFM_LAUNCH(k_pw_density_image, std::min<int64_t>(cdiv(nimg, 256), 152 * 16), 256, 0, s, q, p->ny, nrhs,
                       nblk_m, img);
            FFM_CUDA(cudaMemsetAsync(ut, 0, sizeof(C2) * (size_t)p->by[l].nb * nrhs * F.nQ, s));
            FFM_CUDA(cudaFuncSetAttribute(k_pw_forward_tc<PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)PWT_SMEM));
            dim3 g((unsigned)(F.n_pw_chunks * cdiv(nH, PWT_M)), 1, (unsigned)nblk_m);
            FFM_LAUNCH_NAMED(name("k_pw_forward_tc"), k_pw_forward_tc<PH>, g, PWT_NP + 32, PWT_SMEM, s, PY,
                             F.pw_chunks, img, nblk_m, nrhs, ut, p->dev_err, p->wait_tries);
            tmp.drop(img);
        }
    } else if (multi) {
        if (!dbl && mc == 4) {
            dim3 gm((unsigned)F.n_src, cdiv(nH, 128), cdiv(nrhs, 4));
            FFM_LAUNCH_NAMED(name("k_pw_forward_mr"), (k_pw_forward_mr<R, PH, dbl ? 8 : 4>), gm, 128, 0, s, PY, F.src,
                             q, p->ny, nrhs, ut);
        } else {
            dim3 gm((unsigned)F.n_src, cdiv(nH, 128), cdiv(nrhs, 8));
            FFM_LAUNCH_NAMED(name("k_pw_forward_mr"), (k_pw_forward_mr<R, PH, 8>), gm, 128, 0, s, PY, F.src, q,
                             p->ny, nrhs, ut);
        }
    } else {
        dim3 gf((unsigned)F.n_src, cdiv(nH, tb * qpt), 1);
        if (!dbl && qpt == 2)
            FFM_LAUNCH_NAMED(name("k_pw_forward"), (k_pw_forward<R, PH, dbl ? 4 : 2>), gf, tb, 0, s, PY, F.src, q,
                             p->ny, nrhs, ut);
        else
            FFM_LAUNCH_NAMED(name("k_pw_forward"), (k_pw_forward<R, PH, 4>), gf, tb, 0, s, PY, F.src, q, p->ny, nrhs,
                             ut);
    }
    dim3 gt((unsigned)F.n_tgt, cdiv(F.nQ, 128), 1);
    if (nrhs == 1)
        FFM_LAUNCH_NAMED(name("k_pw_transfer"), (k_pw_transfer<C2, 1, COMP>), gt, 128, 0, s, F.tgt, F.adm_off,
                         F.adm_src, F.adm_t, D, F.nQ, nrhs, (const C2 *)ut, vt);
    else
        FFM_LAUNCH_NAMED(name("k_pw_transfer"), (k_pw_transfer<C2, 8, COMP>), gt, 128, 0, s, F.tgt, F.adm_off,
                         F.adm_src, F.adm_t, D, F.nQ, nrhs, (const C2 *)ut, vt);
    if constexpr (f32) {
        if (F.nufft) {
            nufft_backward(p, l, vt, nrhs, acc, tmp, s);
            return;
        }
    }
    int64_t nbx = p->bx[l].nb;
    int *slot = tmp.get<int>(nbx);
    FFM_LAUNCH(k_slot_init, cdiv(nbx, 256), 256, 0, s, slot, nbx);
    FFM_LAUNCH(k_slot_set, cdiv(F.n_tgt, 256), 256, 0, s, F.tgt, F.n_tgt, slot);
    if (tc_bwd) {
        if constexpr (f32) {
            const int nblk_m = (int)cdiv(nrhs, PWB_MC), nst = (int)cdiv(nH, PWB_KC / 2);
            float *bimg = tmp.get<float>((size_t)F.n_tgt * nst * nblk_m * PWB_BST);
            const int64_t nimg = F.n_tgt * nst * nblk_m * (int64_t)PWB_BH;
            FFM_LAUNCH(k_pw_vt_image, std::min<int64_t>(cdiv(nimg, 256), 152 * 16), 256, 0, s, (const float2 *)vt,
                       F.tgt, F.n_tgt, nrhs, F.nQ, nst, nblk_m, bimg);
            FFM_CUDA(cudaFuncSetAttribute(k_pw_backward_tc<PH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)PWB_SMEM));
            dim3 g((unsigned)F.n_pw_tchunks, (unsigned)nblk_m, 1);
            FFM_LAUNCH_NAMED(name("k_pw_backward_tc"), k_pw_backward_tc<PH>, g, PWB_NP + 32, PWB_SMEM, s, PX,
                             F.pw_tchunks, slot, bimg, nblk_m, nrhs, p->nx, acc, p->dev_err, p->wait_tries);
            tmp.drop(bimg);
        }
        return;
    }
    if (multi) {
        if (!dbl && mc == 4) {
            dim3 gm((unsigned)p->bx[ls].nb, 1, cdiv(nrhs, 4));
            FFM_LAUNCH_NAMED(name("k_pw_backward_mr"), (k_pw_backward_mr<R, PH, dbl ? 8 : 4>), gm, 128, 0, s, PX,
                             p->bx[l].fine, nbx, p->bx[ls].fine, slot, (const C2 *)vt, nrhs, p->nx, acc);
        } else {
            dim3 gm((unsigned)p->bx[ls].nb, 1, cdiv(nrhs, 8));
            FFM_LAUNCH_NAMED(name("k_pw_backward_mr"), (k_pw_backward_mr<R, PH, 8>), gm, 128, 0, s, PX,
                             p->bx[l].fine, nbx, p->bx[ls].fine, slot, (const C2 *)vt, nrhs, p->nx, acc);
        }
        return;
    }
    dim3 gb((unsigned)p->bx[ls].nb, 1, 1);
    if (!dbl && ppt == 2)
        FFM_LAUNCH_NAMED(name("k_pw_backward"), (k_pw_backward<R, PH, dbl ? 4 : 2>), gb, 128, 0, s, PX,
                         p->bx[l].fine, nbx, p->bx[ls].fine, slot, (const C2 *)vt, nrhs, p->nx, acc);
    else
        FFM_LAUNCH_NAMED(name("k_pw_backward"), (k_pw_backward<R, PH, 4>), gb, 128, 0, s, PX, p->bx[l].fine, nbx,
                         p->bx[ls].fine, slot, (const C2 *)vt, nrhs, p->nx, acc);
}

void far_planewave(const ffm_plan_s *p, int l, const float2 *q, int nrhs, double2 *acc, Alloc &tmp,
                   cudaStream_t s) {
    const FarLevel &F = p->far[l];
    if (p->l_stop - l > PW_MAXD) fail(FFM_EUNSUPPORTED, "more than 16 levels between a plane-wave level and the leaves");
    // largest leaf-local phase k sqrt(3) d_leaf / 2: the hardware sincos gets the phase
    // reduced to [-pi, pi] only beyond 2 pi
    bool reduce = p->k * std::sqrt(3.0) * std::ldexp(p->d0, -p->l_stop) * 0.5 > 2.0 * PI;
    if (F.prec == FFM_PREC_F64)
        planewave_level<double, PH_MUFU>(p, l, q, nrhs, acc, tmp, s, F.ksd, F.Dd, F.Ed);
    else if (F.prec == FFM_PREC_F32X2)
        planewave_level<dd, PH_MUFU>(p, l, q, nrhs, acc, tmp, s, F.ksx, F.Dx, F.Ex);
    else if (F.prec == FFM_PREC_F32C)
        planewave_level<float, PH_ACC>(p, l, q, nrhs, acc, tmp, s, F.ks, F.D, F.E);
    else if (reduce)
        planewave_level<float, PH_MUFU_RED>(p, l, q, nrhs, acc, tmp, s, F.ks, F.D, F.E);
    else
        planewave_level<float, PH_MUFU>(p, l, q, nrhs, acc, tmp, s, F.ks, F.D, F.E);
}

}  // namespace ffm
