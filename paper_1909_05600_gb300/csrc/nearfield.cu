// Near field at the stop level (Sec. 2.2.4): the dense product over the non-admissible
// leaf pairs left by the descent, v_i += sum_{j in near leaves} G(x_i - y_j) (w u)_j,
// with pairs at distance 0 skipped.
//
// Work is split into items of at most tchunk targets of one leaf times a range of its
// near pairs holding at most smax source points (both autotuned), so that clustered inputs with very
// uneven leaves still spread over the whole GPU; items add into the FP64 accumulators with
// atomics.  Coordinates are leaf-relative unevaluated FP32 pairs (hi + lo).  Source points
// are staged in shared memory relative to the target leaf centre: the offset between the
// two leaf centres is formed in FP64 once per source leaf, split into hi + lo, and added to
// each point with an FP32 TwoSum.  A difference is then (x_hi - y_hi) + (x_lo - y_lo), whose
// hi part is exact for nearby points (Sterbenz), so |x - y| keeps about 2^-44 relative
// accuracy exactly where the 1/|x - y| terms are largest.  Small chunks are served by
// several thread groups that split the staged sources and are reduced in shared memory.
#include "ffm_internal.cuh"

namespace ffm {

constexpr int P2P_SB = 512;

struct NearArgs {
    const uint32_t *xl_start, *yl_start;  // leaf starts (X, Y)
    const int4 *xl_g, *yl_g;              // leaf integer coords
    const float4 *epsX, *epsY;            // hi parts (.w: leaf index bits)
    const float4 *epsXlo, *epsYlo;        // lo parts
    const uint32_t *off, *src;            // CSR over target leaves
    const int4 *items;                    // (target leaf, first target, first pair, end pair)
    int tchunk;                           // targets per item (<= P2P_T)
    float dls_h, dls_l;                   // leaf edge as an unevaluated FP32 pair
    float oyx_h[3], oyx_l[3];             // oY - oX, likewise
    float k;
};

// y (hi + lo, own leaf frame) plus the leaf-centre offset (oh + ol): an FP32 TwoSum of the
// hi parts, the lo parts added to the rounding error.
__device__ __forceinline__ void stage_coord(float yh, float yl, float oh, float ol, float &hi, float &lo) {
    float s = yh + oh;
    float bb = s - yh;
    float err = (yh - (s - bb)) + (oh - bb);
    hi = s;
    lo = err + (yl + ol);
}

struct Off3 {
    float h[3], l[3];
};

// Offset of source leaf b's centre from target leaf a's, oY - oX + d_ls (g_b - g_a), as
// hi + lo in FP32 only (this part has a small fraction of the FP32 rate in FP64): the
// product by the small integer offset is split exactly (TwoProd by FMA), then added to
// oY - oX with a TwoSum.  Relative accuracy about 2^-44, as for the coordinates.
__device__ __forceinline__ Off3 leaf_offset3(const NearArgs &N, int4 ga, int4 gb) {
    float g[3] = {(float)(gb.x - ga.x), (float)(gb.y - ga.y), (float)(gb.z - ga.z)};
    Off3 r;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float ph = __fmul_rn(N.dls_h, g[d]);
        float pl = fmaf(N.dls_h, g[d], -ph) + N.dls_l * g[d];
        float a = N.oyx_h[d];
        float sum = __fadd_rn(a, ph);
        float bb = __fsub_rn(sum, a);
        float err = __fadd_rn(__fsub_rn(a, __fsub_rn(sum, bb)), __fsub_rn(ph, bb));
        r.h[d] = sum;
        r.l[d] = err + (N.oyx_l[d] + pl);
    }
    return r;
}

// 1/sqrt(x) by the hardware approximation (relative error about 2^-23), subnormal inputs
// flushed to zero; a single special-function instruction.
__device__ __forceinline__ float rsqrt_hw(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Accumulate the staged sources [j0, j1) into (sr, si) for the PT targets x = xh + xl of
// this thread.  Staged source j: sA[j] = (hi.x, hi.y, hi.z, w.re), sB[j] = (lo.x, lo.y,
// lo.z, w.im): two 16-byte loads serve PT pairs.
constexpr int NF_LAPLACE = 0, NF_HELMHOLTZ = 1, NF_DOUBLE_LAYER = 2, NF_GRADIENT = 3;

// a + b with its rounding error (Knuth's TwoSum, no ordering assumption)
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// q . (x - y) with x = xh + xl, y = yh + yl (leaf-frame FP32 pairs, .w of yh/yl unused) and
// q = qh + ql: each component of x - y as a pair (TwoSum), each leading product split
// exactly by FMA, the three leading terms added with TwoSum, all residuals collected in
// FP32.  About 2^-44 relative to |q| |x - y| instead of 2^-24.
__device__ __forceinline__ float dot_pair(float4 xh, float4 xl, float4 yh, float4 yl, float3 qh, float3 ql) {
    float dh0, de0, dh1, de1, dh2, de2;
    two_sum_f(xh.x, -yh.x, dh0, de0);
    two_sum_f(xh.y, -yh.y, dh1, de1);
    two_sum_f(xh.z, -yh.z, dh2, de2);
    float dl0 = de0 + (xl.x - yl.x), dl1 = de1 + (xl.y - yl.y), dl2 = de2 + (xl.z - yl.z);
    float p0 = __fmul_rn(qh.x, dh0), p1 = __fmul_rn(qh.y, dh1), p2 = __fmul_rn(qh.z, dh2);
    float r = fmaf(qh.x, dh0, -p0) + fmaf(qh.y, dh1, -p1) + fmaf(qh.z, dh2, -p2);
    r = fmaf(qh.x, dl0, fmaf(qh.y, dl1, fmaf(qh.z, dl2, r)));
    r = fmaf(ql.x, dh0, fmaf(ql.y, dh1, fmaf(ql.z, dh2, r)));
    float s1, e1, s2, e2;
    two_sum_f(p0, p1, s1, e1);
    two_sum_f(s1, p2, s2, e2);
    return s2 + ((e1 + e2) + r);
}

template <int KIND, int PT>
__device__ __forceinline__ void interact(const float4 *sA, const float4 *sB, const float4 *sC, int j0, int j1,
                                         const float4 *xh, const float4 *xl, float k, float *sr, float *si,
                                         float *sz) {
#pragma unroll 2
    for (int j = j0; j < j1; ++j) {
        float4 y = sA[j];
        float4 yl = sB[j];
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            float dx = (xh[t].x - y.x) + (xl[t].x - yl.x);
            float dy = (xh[t].y - y.y) + (xl[t].y - yl.y);
            float dz = (xh[t].z - y.z) + (xl[t].z - yl.z);
            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            float inv = r2 > 0.f ? rsqrt_hw(r2) : 0.f;  // coincident points contribute nothing
            if constexpr (KIND == NF_DOUBLE_LAYER) {
                // (w u n) . (x - y) / |x - y|^3; for points of one surface the dot product
                // is second order in |x - y|, so it is formed from x - y and q as FP32 pairs
                float4 c = sC[j];  // (q_hi.z, q_lo.x, q_lo.y, q_lo.z)
                float qd = dot_pair(xh[t], xl[t], y, yl, make_float3(y.w, yl.w, c.x), make_float3(c.y, c.z, c.w));
                sr[t] = fmaf(qd, inv * inv * inv, sr[t]);
            } else if constexpr (KIND == NF_GRADIENT) {
                // grad_x of w u / |x - y|: -(x - y) w u / |x - y|^3
                float f = y.w * (inv * inv * inv);
                sr[t] = fmaf(-f, dx, sr[t]);
                si[t] = fmaf(-f, dy, si[t]);
                sz[t] = fmaf(-f, dz, sz[t]);
            } else if constexpr (KIND == NF_HELMHOLTZ) {
                // phase k r reduced to [-pi, pi] (Cody-Waite, two-term 2 pi) before sincos
                float ph = k * (r2 * inv);
                float n = rintf(ph * 0.15915494309189535f);
                ph = fmaf(-n, 6.28318548202514648f, ph);
                ph = fmaf(-n, -1.7484555314695172e-07f, ph);
                float sn, cs;
                __sincosf(ph, &sn, &cs);
                cs *= inv;
                sn *= inv;
                sr[t] = fmaf(cs, y.w, fmaf(-sn, yl.w, sr[t]));
                si[t] = fmaf(cs, yl.w, fmaf(sn, y.w, si[t]));
            } else {
                sr[t] = fmaf(y.w, inv, sr[t]);
            }
        }
    }
}

// One work item: up to tchunk targets of a leaf (PT per thread) against a range of its near
// source leaves, staged P2P_SB points at a time.  When the targets need fewer than P2P_T
// threads, G groups of threads split each staged batch and are reduced in shared memory.
template <int KIND>
__global__ void __launch_bounds__(P2P_T) k_p2p(NearArgs N, const void *__restrict__ qv, int64_t ny, int nrhs,
                                               int64_t nx, double2 *__restrict__ acc) {
    constexpr int PT = 2;
    constexpr bool HELM = KIND == NF_HELMHOLTZ;
    __shared__ float4 sA[P2P_SB];
    __shared__ float4 sB[P2P_SB];
    __shared__ float4 sC[KIND == NF_DOUBLE_LAYER ? P2P_SB : 1];  // double layer: (q_hi.z, q_lo)
    __shared__ float4 red[P2P_T * PT];
    int4 it = N.items[blockIdx.x];
    int a = it.x, m = blockIdx.y;
    uint32_t e0 = (uint32_t)it.z, e1 = (uint32_t)it.w;
    uint32_t p0 = N.xl_start[a] + (uint32_t)it.y;
    int np = min(N.tchunk, (int)(N.xl_start[a + 1] - p0));
    int pr = min((np + PT - 1) / PT, P2P_T);  // threads per group
    int G = P2P_T / pr;
    int grp = threadIdx.x / pr, pi = threadIdx.x % pr;
    bool active = grp < G;
    int4 ga = N.xl_g[a];
    const float *qr = reinterpret_cast<const float *>(qv) + (int64_t)m * ny;
    const float2 *qc = reinterpret_cast<const float2 *>(qv) + (int64_t)m * ny;
    const float4 *q3 = reinterpret_cast<const float4 *>(qv) + 2 * (int64_t)m * ny;
    float4 xh[PT], xl[PT];
    float sr[PT], si[PT], sz[PT];
#pragma unroll
    for (int t = 0; t < PT; ++t) {
        int i = pi + t * pr;
        bool ok = active && i < np;
        xh[t] = ok ? N.epsX[p0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        xl[t] = ok ? N.epsXlo[p0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        sr[t] = si[t] = sz[t] = 0.f;
    }
    int fill = 0;
    for (uint32_t e = e0; e < e1; ++e) {
        uint32_t b = N.src[e];
        uint32_t s0 = N.yl_start[b];
        int cnt = (int)(N.yl_start[b + 1] - s0);
        for (int c0 = 0; c0 < cnt;) {
            int take = min(cnt - c0, P2P_SB - fill);
            // the leaf-centre offset is formed only by the threads that stage points (most
            // near leaves hold fewer points than the block has threads)
            for (int j = threadIdx.x; j < take; j += P2P_T) {
                Off3 oc = leaf_offset3(N, ga, N.yl_g[b]);
                float4 y = N.epsY[s0 + c0 + j];
                float4 yl = N.epsYlo[s0 + c0 + j];
                float hx, lx, hy, ly, hz, lz;
                stage_coord(y.x, yl.x, oc.h[0], oc.l[0], hx, lx);
                stage_coord(y.y, yl.y, oc.h[1], oc.l[1], hy, ly);
                stage_coord(y.z, yl.z, oc.h[2], oc.l[2], hz, lz);
                if constexpr (KIND == NF_DOUBLE_LAYER) {
                    float4 wh = q3[2 * (s0 + c0 + j)], wl = q3[2 * (s0 + c0 + j) + 1];
                    sA[fill + j] = make_float4(hx, hy, hz, wh.x);
                    sB[fill + j] = make_float4(lx, ly, lz, wh.y);
                    sC[fill + j] = make_float4(wh.z, wl.x, wl.y, wl.z);
                } else {
                    float2 w = HELM ? qc[s0 + c0 + j] : make_float2(qr[s0 + c0 + j], 0.f);
                    sA[fill + j] = make_float4(hx, hy, hz, w.x);
                    sB[fill + j] = make_float4(lx, ly, lz, w.y);
                }
            }
            fill += take;
            c0 += take;
            if (fill == P2P_SB) {
                __syncthreads();
                if (active)
                    interact<KIND, PT>(sA, sB, sC, grp * fill / G, (grp + 1) * fill / G, xh, xl, N.k, sr, si, sz);
                __syncthreads();
                fill = 0;
            }
        }
    }
    __syncthreads();
    if (active) interact<KIND, PT>(sA, sB, sC, grp * fill / G, (grp + 1) * fill / G, xh, xl, N.k, sr, si, sz);
#pragma unroll
    for (int t = 0; t < PT; ++t) red[threadIdx.x * PT + t] = make_float4(sr[t], si[t], sz[t], 0.f);
    __syncthreads();
    if (active && grp == 0) {
        const double c = 0.079577471545947667884;  // 1 / (4 pi)
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            int i = pi + t * pr;
            if (i >= np) continue;
            float tr = 0.f, ti = 0.f, tz = 0.f;
            for (int g = 0; g < G; ++g) {
                tr += red[(g * pr + pi) * PT + t].x;
                ti += red[(g * pr + pi) * PT + t].y;
                tz += red[(g * pr + pi) * PT + t].z;
            }
            if constexpr (KIND == NF_GRADIENT) {
                // component d of right-hand side m in accumulator slot d nrhs + m
                atomicAdd(&acc[(int64_t)m * nx + p0 + i].x, (double)tr * c);
                atomicAdd(&acc[((int64_t)nrhs + m) * nx + p0 + i].x, (double)ti * c);
                atomicAdd(&acc[(2 * (int64_t)nrhs + m) * nx + p0 + i].x, (double)tz * c);
                continue;
            }
            double2 *dst = &acc[(int64_t)m * nx + p0 + i];
            atomicAdd(&dst->x, (double)tr * c);
            if (HELM) atomicAdd(&dst->y, (double)ti * c);
        }
    }
}

// ---- Laplace single layer, one right-hand side: packed FP32 pairs
//
// Sources are staged per batch as FP32 structure-of-arrays in the target leaf's frame (hi
// and lo parts of x, y, z, and w u).  A thread holds PT targets, each coordinate part
// duplicated into both halves of a 64-bit register, and takes its sources four at a time
// (one 16-byte shared load per array), so every arithmetic instruction is a packed f32x2
// operation on two pairs: per coordinate the hi difference, the lo difference and their sum
// ((x_hi - y_hi) + (x_lo - y_lo), exact in its hi part for nearby points), a multiply and two
// fused multiply-adds for |x - y|^2, two hardware rsqrt, and one packed multiply-add into the
// target's accumulator pair: 6.5 issue slots of FP32 arithmetic (13 FP32 operations) and one
// special-function result per pair, against about 17 issue slots in the generic kernel.
//
// Coincident points: rsqrt of 0 is +inf, which makes the target's accumulator non-finite.
// Each thread checks its accumulators after every batch and recomputes that batch for the
// affected target with the pair test (pairs with |x - y|^2 below the smallest normal FP32
// number contribute nothing, as in the generic kernel), starting again from the value it
// had before the batch.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

constexpr int LAP_SB = 512;         // staged sources per batch (a multiple of 4)
constexpr float LAP_FAR = 1.0e15f;  // coordinate of the padding sources (weight 0)

// a target: hi and lo parts of each coordinate, duplicated in both halves
struct Tgt2 {
    uint64_t h[3], l[3];
};
// staged sources, structure of arrays: hi x, y, z, lo x, y, z, w u
struct LapStage {
    float4 a[7][LAP_SB / 4];
};

// Two pairs (sources a, b of one quad half) for one target: acc += w / |x - y| in both halves.
template <bool GUARD>
__device__ __forceinline__ uint64_t lap_two(const Tgt2 &x, const uint64_t *yh, const uint64_t *yl, uint64_t w,
                                            uint64_t acc) {
    uint64_t d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] = f2_add(f2_sub(x.h[c], yh[c]), f2_sub(x.l[c], yl[c]));
    uint64_t r2 = f2_fma(d[2], d[2], f2_fma(d[1], d[1], f2_mul(d[0], d[0])));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    float ia = rsqrt_hw(ra), ib = rsqrt_hw(rb);
    if constexpr (GUARD) {
        ia = ra >= 1.17549435e-38f ? ia : 0.f;
        ib = rb >= 1.17549435e-38f ? ib : 0.f;
    }
    return f2_fma(w, f2_pack(ia, ib), acc);
}

template <bool GUARD, int PT>
__device__ __forceinline__ void lap_quads(const LapStage &S, int q0, int q1, int qstep, const Tgt2 *X,
                                          uint64_t *acc) {
#pragma unroll 1
    for (int q = q0; q < q1; q += qstep) {
        float4 v[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) v[c] = S.a[c][q];
        uint64_t ha[3], hb[3], la[3], lb[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ha[c] = f2_pack(v[c].x, v[c].y);
            hb[c] = f2_pack(v[c].z, v[c].w);
            la[c] = f2_pack(v[3 + c].x, v[3 + c].y);
            lb[c] = f2_pack(v[3 + c].z, v[3 + c].w);
        }
        uint64_t wa = f2_pack(v[6].x, v[6].y), wb = f2_pack(v[6].z, v[6].w);
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            acc[t] = lap_two<GUARD>(X[t], ha, la, wa, acc[t]);
            acc[t] = lap_two<GUARD>(X[t], hb, lb, wb, acc[t]);
        }
    }
}

template <int PT>
__global__ void __launch_bounds__(P2P_T) k_p2p_lap(NearArgs N, const float *__restrict__ qv, int64_t nx,
                                                   double2 *__restrict__ acc) {
    __shared__ LapStage S;
    __shared__ float red[P2P_T * PT];
    int4 it = N.items[blockIdx.x];
    int a = it.x;
    uint32_t e0 = (uint32_t)it.z, e1 = (uint32_t)it.w;
    uint32_t p0 = N.xl_start[a] + (uint32_t)it.y;
    int np = min(N.tchunk, (int)(N.xl_start[a + 1] - p0));
    int pr = min((np + PT - 1) / PT, P2P_T);  // threads per group
    int G = P2P_T / pr;
    int grp = threadIdx.x / pr, pi = threadIdx.x % pr;
    bool active = grp < G;
    int4 ga = N.xl_g[a];
    Tgt2 X[PT];
    uint64_t A[PT];
#pragma unroll
    for (int t = 0; t < PT; ++t) {
        int i = pi + t * pr;
        bool ok = active && i < np;
        float4 xh = ok ? N.epsX[p0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 xl = ok ? N.epsXlo[p0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        X[t].h[0] = f2_pack(xh.x, xh.x);
        X[t].h[1] = f2_pack(xh.y, xh.y);
        X[t].h[2] = f2_pack(xh.z, xh.z);
        X[t].l[0] = f2_pack(xl.x, xl.x);
        X[t].l[1] = f2_pack(xl.y, xl.y);
        X[t].l[2] = f2_pack(xl.z, xl.z);
        A[t] = 0ull;  // +0.0f in both halves
    }
    float *f[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) f[c] = reinterpret_cast<float *>(S.a[c]);
    auto run_batch = [&](int fill) {
        // pad to whole quads with far, weightless sources
        for (int j = fill + threadIdx.x; j < ((fill + 3) & ~3); j += P2P_T) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                f[c][j] = LAP_FAR;
                f[3 + c][j] = 0.f;
            }
            f[6][j] = 0.f;
        }
        __syncthreads();
        if (active) {
            const int nq = (fill + 3) >> 2;
            uint64_t save[PT];
#pragma unroll
            for (int t = 0; t < PT; ++t) save[t] = A[t];
            lap_quads<false, PT>(S, grp, nq, G, X, A);
#pragma unroll
            for (int t = 0; t < PT; ++t) {
                float u0, u1;
                f2_unpack(A[t], u0, u1);
                if (!isfinite(u0 + u1)) {  // a coincident pair: this batch again with the pair test
                    uint64_t one[1] = {save[t]};
                    lap_quads<true, 1>(S, grp, nq, G, &X[t], one);
                    A[t] = one[0];
                }
            }
        }
        __syncthreads();
    };
    // Source leaves are taken P2P_T at a time: their start, size and centre offset are read
    // and formed in parallel into a shared table (one thread per leaf), then every thread
    // stages whichever sources of the batch fall to it, finding its leaf by a binary search
    // of the table's prefix sums.  Near leaves of a few points each (fine levels of clustered
    // inputs) are thus staged with all loads in flight at once, not one leaf after another.
    __shared__ uint32_t lb_s0[P2P_T], lb_pre[P2P_T + 1];
    __shared__ float lb_off[6][P2P_T];
    int fill = 0;
    for (uint32_t eg = e0; eg < e1; eg += P2P_T) {
        const int ne = (int)min((uint32_t)P2P_T, e1 - eg);
        uint32_t cnt = 0;
        if ((int)threadIdx.x < ne) {
            uint32_t b = N.src[eg + threadIdx.x];
            uint32_t s0 = N.yl_start[b];
            cnt = N.yl_start[b + 1] - s0;
            Off3 oc = leaf_offset3(N, ga, N.yl_g[b]);
            lb_s0[threadIdx.x] = s0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                lb_off[c][threadIdx.x] = oc.h[c];
                lb_off[3 + c][threadIdx.x] = oc.l[c];
            }
        }
        // inclusive prefix of the leaf sizes (warp scans, then the warp totals)
        {
            __shared__ uint32_t wsum[P2P_T / 32];
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            uint32_t inc = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            if (lane == 31) wsum[warp] = inc;
            __syncthreads();
            for (int w = 0; w < warp; ++w) inc += wsum[w];
            lb_pre[threadIdx.x + 1] = inc;
            if (threadIdx.x == 0) lb_pre[0] = 0;
            __syncthreads();
        }
        const int total = (int)lb_pre[ne];
        for (int base = 0; base < total;) {
            const int take = min(total - base, LAP_SB - fill);
            for (int j = threadIdx.x; j < take; j += P2P_T) {
                const int flat = base + j;
                int lo = 0, hi = ne;  // leaf: last index with lb_pre[leaf] <= flat
                while (hi - lo > 1) {
                    int mid = (lo + hi) >> 1;
                    if ((int)lb_pre[mid] <= flat) lo = mid; else hi = mid;
                }
                const uint32_t i = lb_s0[lo] + (uint32_t)(flat - (int)lb_pre[lo]);
                float4 y = N.epsY[i];
                float4 yl = N.epsYlo[i];
                float hx, lx, hy, ly, hz, lz;
                stage_coord(y.x, yl.x, lb_off[0][lo], lb_off[3][lo], hx, lx);
                stage_coord(y.y, yl.y, lb_off[1][lo], lb_off[4][lo], hy, ly);
                stage_coord(y.z, yl.z, lb_off[2][lo], lb_off[5][lo], hz, lz);
                f[0][fill + j] = hx;
                f[1][fill + j] = hy;
                f[2][fill + j] = hz;
                f[3][fill + j] = lx;
                f[4][fill + j] = ly;
                f[5][fill + j] = lz;
                f[6][fill + j] = qv[i];
            }
            fill += take;
            base += take;
            if (fill == LAP_SB) {
                run_batch(fill);
                fill = 0;
            }
        }
        __syncthreads();  // the table is rewritten for the next leaves
    }
    if (fill > 0) run_batch(fill);
#pragma unroll
    for (int t = 0; t < PT; ++t) {
        float u0, u1;
        f2_unpack(A[t], u0, u1);
        red[threadIdx.x * PT + t] = u0 + u1;
    }
    __syncthreads();
    if (active && grp == 0) {
        const double c = 0.079577471545947667884;  // 1 / (4 pi)
#pragma unroll
        for (int t = 0; t < PT; ++t) {
            int i = pi + t * pr;
            if (i >= np) continue;
            float tr = 0.f;
            for (int g = 0; g < G; ++g) tr += red[(g * pr + pi) * PT + t];
            atomicAdd(&acc[p0 + i].x, (double)tr * c);
        }
    }
}

// Several right-hand sides: each kernel value G(x_i - y_j) is computed once and applied
// to MC densities.  One thread per target point of the leaf.
template <bool HELM, int MC>
__global__ void __launch_bounds__(P2P_T) k_p2p_mr(NearArgs N, const void *__restrict__ qv, int64_t ny, int nrhs,
                                                  int64_t nx, double2 *__restrict__ acc) {
    constexpr int SB = 128;
    __shared__ float4 sy[SB];
    __shared__ float2 syl[SB];
    __shared__ float2 sq[SB][MC];
    int4 it = N.items[blockIdx.x];
    int a = it.x, m0 = blockIdx.y * MC;
    uint32_t e0 = (uint32_t)it.z, e1 = (uint32_t)it.w;
    uint32_t p0 = N.xl_start[a] + (uint32_t)it.y;
    int np = min(N.tchunk, (int)(N.xl_start[a + 1] - p0));
    int4 ga = N.xl_g[a];
    const float *qr = reinterpret_cast<const float *>(qv);
    const float2 *qc = reinterpret_cast<const float2 *>(qv);
    for (int pb = 0; pb < np; pb += P2P_T) {
        bool valid = pb + (int)threadIdx.x < np;
        float4 x = valid ? N.epsX[p0 + pb + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 xl = valid ? N.epsXlo[p0 + pb + threadIdx.x] : make_float4(0.f, 0.f, 0.f, 0.f);
        float2 o[MC];
#pragma unroll
        for (int m = 0; m < MC; ++m) o[m] = make_float2(0.f, 0.f);
        for (uint32_t e = e0; e < e1; ++e) {
            uint32_t b = N.src[e];
            uint32_t s0 = N.yl_start[b];
            int cnt = (int)(N.yl_start[b + 1] - s0);
            Off3 oc = leaf_offset3(N, ga, N.yl_g[b]);
            for (int c0 = 0; c0 < cnt; c0 += SB) {
                int take = min(cnt - c0, SB);
                __syncthreads();
                for (int j = threadIdx.x; j < take; j += P2P_T) {
                    float4 y = N.epsY[s0 + c0 + j];
                    float4 yl = N.epsYlo[s0 + c0 + j];
                    float hx, lx, hy, ly, hz, lz;
                    stage_coord(y.x, yl.x, oc.h[0], oc.l[0], hx, lx);
                    stage_coord(y.y, yl.y, oc.h[1], oc.l[1], hy, ly);
                    stage_coord(y.z, yl.z, oc.h[2], oc.l[2], hz, lz);
                    sy[j] = make_float4(hx, hy, hz, lx);
                    syl[j] = make_float2(ly, lz);
                }
                for (int t = threadIdx.x; t < take * MC; t += P2P_T) {
                    int j = t % take, m = t / take;
                    int64_t idx = (int64_t)(m0 + m) * ny + s0 + c0 + j;
                    float2 w = make_float2(0.f, 0.f);
                    if (m0 + m < nrhs) w = HELM ? qc[idx] : make_float2(qr[idx], 0.f);
                    sq[j][m] = w;
                }
                __syncthreads();
                if (valid) {
                    for (int j = 0; j < take; ++j) {
                        float4 y = sy[j];
                        float2 yl2 = syl[j];
                        float dx = (x.x - y.x) + (xl.x - y.w);
                        float dy = (x.y - y.y) + (xl.y - yl2.x);
                        float dz = (x.z - y.z) + (xl.z - yl2.y);
                        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        float inv = r2 > 0.f ? rsqrt_hw(r2) : 0.f;
                        float gr = inv, gi = 0.f;
                        if constexpr (HELM) {
                            float ph = N.k * (r2 * inv);
                            float n = rintf(ph * 0.15915494309189535f);
                            ph = fmaf(-n, 6.28318548202514648f, ph);
                            ph = fmaf(-n, -1.7484555314695172e-07f, ph);
                            float sn, cs;
                            __sincosf(ph, &sn, &cs);
                            gr = cs * inv;
                            gi = sn * inv;
                        }
#pragma unroll
                        for (int m = 0; m < MC; ++m) {
                            float2 w = sq[j][m];
                            if constexpr (HELM) {
                                o[m].x = fmaf(gr, w.x, fmaf(-gi, w.y, o[m].x));
                                o[m].y = fmaf(gr, w.y, fmaf(gi, w.x, o[m].y));
                            } else {
                                o[m].x = fmaf(gr, w.x, o[m].x);
                            }
                        }
                    }
                }
            }
        }
        if (valid) {
            const double c = 0.079577471545947667884;  // 1 / (4 pi)
#pragma unroll
            for (int m = 0; m < MC; ++m)
                if (m0 + m < nrhs) {
                    double2 *dst = &acc[(int64_t)(m0 + m) * nx + p0 + pb + threadIdx.x];
                    atomicAdd(&dst->x, (double)o[m].x * c);
                    atomicAdd(&dst->y, (double)o[m].y * c);
                }
        }
    }
}

void near_field(const ffm_plan_s *p, const void *q, int nrhs, double2 *acc, cudaStream_t s) {
    near_field_items(p, p->items, p->n_items, p->p2p_tchunk, q, nrhs, acc, s);
}

void near_field_items(const ffm_plan_s *p, const int4 *items, int64_t n_items, int tchunk, const void *q, int nrhs,
                      double2 *acc, cudaStream_t s) {
    if (p->n_near == 0 || n_items == 0) return;
    int ls = p->l_stop;
    NearArgs N;
    N.xl_start = p->bx[ls].start;
    N.yl_start = p->by[ls].start;
    N.xl_g = p->bx[ls].g;
    N.yl_g = p->by[ls].g;
    N.epsX = p->epsX;
    N.epsY = p->epsY;
    N.epsXlo = p->epsXlo;
    N.epsYlo = p->epsYlo;
    N.off = p->near_off;
    N.src = p->near_src;
    N.items = items;
    N.tchunk = tchunk;
    double dls = std::ldexp(p->d0, -ls);
    N.dls_h = (float)dls;
    N.dls_l = (float)(dls - (double)N.dls_h);
    for (int d = 0; d < 3; ++d) {
        double o = p->oY[d] - p->oX[d];
        N.oyx_h[d] = (float)o;
        N.oyx_l[d] = (float)(o - (double)N.oyx_h[d]);
    }
    N.k = (float)p->k;
    if (p->kind == FFM_LAPLACE_DL) {
        dim3 g((unsigned)n_items, nrhs);
        FFM_LAUNCH(k_p2p<NF_DOUBLE_LAYER>, g, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
        return;
    }
    if (p->kind == FFM_LAPLACE_GRAD) {
        dim3 g((unsigned)n_items, nrhs);
        FFM_LAUNCH(k_p2p<NF_GRADIENT>, g, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
        return;
    }
    if (nrhs > 1) {
        constexpr int MC = 8;
        dim3 gm((unsigned)n_items, cdiv(nrhs, MC));
        if (p->kind == FFM_HELMHOLTZ)
            FFM_LAUNCH((k_p2p_mr<true, MC>), gm, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
        else
            FFM_LAUNCH((k_p2p_mr<false, MC>), gm, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
        return;
    }
    dim3 g((unsigned)n_items, nrhs);
    if (p->kind == FFM_HELMHOLTZ)
        FFM_LAUNCH(k_p2p<NF_HELMHOLTZ>, g, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
    else
        FFM_LAUNCH(k_p2p_lap<4>, (unsigned)n_items, P2P_T, 0, s, N, (const float *)q, p->nx, acc);
}

}  // namespace ffm
