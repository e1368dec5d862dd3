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
        FFM_LAUNCH(k_p2p<NF_LAPLACE>, g, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
}

}  // namespace ffm
