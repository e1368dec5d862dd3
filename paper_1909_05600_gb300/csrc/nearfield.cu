// Near field at the stop level (Sec. 2.2.4): the dense product over the non-admissible
// leaf pairs left by the descent, v_i += sum_{j in near leaves} G(x_i - y_j) (w u)_j,
// with pairs at distance 0 skipped.
//
// One block per target leaf.  Coordinates are leaf-relative unevaluated FP32 pairs
// (hi + lo).  Source points of the near leaves are staged in shared memory relative to
// the target leaf centre (re-split in FP64 from their own leaf frame), and a difference is
// formed as (x_hi - y_hi) + (x_lo - y_lo): the hi difference is exact for nearby points
// (Sterbenz), so |x - y| keeps ~2^-48 relative accuracy exactly where the 1/|x - y|
// terms are largest.  Small target leaves are served by several thread groups that split
// the staged sources and are reduced in shared memory.
#include "ffm_internal.cuh"

namespace ffm {

constexpr int P2P_T = 128;
constexpr int P2P_SB = 256;

struct NearArgs {
    const uint32_t *xl_start, *yl_start;  // leaf starts (X, Y)
    const int4 *xl_g, *yl_g;              // leaf integer coords
    const float4 *epsX, *epsY;            // hi parts (.w: leaf index bits)
    const float4 *epsXlo, *epsYlo;        // lo parts
    const uint32_t *off, *src;            // CSR over target leaves
    double dls;                           // leaf edge
    double oyx[3];                        // oY - oX
    float k;
};

// Accumulate the staged sources [grp, fill) step G into (sr, si) for target x = xh + xl.
// Staged source j: sy[j] = (hi.x, hi.y, hi.z, lo.x), syl[j] = (lo.y, lo.z).
template <bool HELM>
__device__ __forceinline__ void interact(const float4 *sy, const float2 *syl, const float2 *sq, int fill, int grp,
                                         int G, float4 xh, float4 xl, float k, float &sr, float &si) {
    for (int j = grp; j < fill; j += G) {
        float4 y = sy[j];
        float2 yl = syl[j];
        float dx = (xh.x - y.x) + (xl.x - y.w);
        float dy = (xh.y - y.y) + (xl.y - yl.x);
        float dz = (xh.z - y.z) + (xl.z - yl.y);
        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        float inv = r2 > 0.f ? rsqrtf(r2) : 0.f;
        float2 w = sq[j];
        if constexpr (HELM) {
            // phase k r reduced to [-pi, pi] (Cody-Waite, two-term 2 pi) before sincos
            float ph = k * (r2 * inv);
            float n = rintf(ph * 0.15915494309189535f);
            ph = fmaf(-n, 6.28318548202514648f, ph);
            ph = fmaf(-n, -1.7484555314695172e-07f, ph);
            float sn, cs;
            __sincosf(ph, &sn, &cs);
            cs *= inv;
            sn *= inv;
            sr = fmaf(cs, w.x, fmaf(-sn, w.y, sr));
            si = fmaf(cs, w.y, fmaf(sn, w.x, si));
        } else {
            sr = fmaf(w.x, inv, sr);
        }
    }
}

template <bool HELM>
__global__ void __launch_bounds__(P2P_T) k_p2p(NearArgs N, const void *__restrict__ qv, int64_t ny, int nrhs,
                                               int64_t nx, double2 *__restrict__ acc) {
    __shared__ float4 sy[P2P_SB];
    __shared__ float2 syl[P2P_SB];
    __shared__ float2 sq[P2P_SB];
    __shared__ float2 red[P2P_T];
    int a = blockIdx.x, m = blockIdx.y;
    uint32_t e0 = N.off[a], e1 = N.off[a + 1];
    if (e0 == e1) return;
    uint32_t p0 = N.xl_start[a], p1 = N.xl_start[a + 1];
    int np = (int)(p1 - p0);
    int pr = np < P2P_T ? np : P2P_T;
    int G = P2P_T / pr;
    int grp = threadIdx.x / pr, pi = threadIdx.x % pr;
    bool active = grp < G;
    int4 ga = N.xl_g[a];
    const float *qr = reinterpret_cast<const float *>(qv) + (int64_t)m * ny;
    const float2 *qc = reinterpret_cast<const float2 *>(qv) + (int64_t)m * ny;
    for (int pb = 0; pb < np; pb += pr) {
        bool valid = active && pb + pi < np;
        float4 x = valid ? N.epsX[p0 + pb + pi] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 xl = valid ? N.epsXlo[p0 + pb + pi] : make_float4(0.f, 0.f, 0.f, 0.f);
        float sr = 0.f, si = 0.f;
        int fill = 0;
        for (uint32_t e = e0; e < e1; ++e) {
            uint32_t b = N.src[e];
            uint32_t s0 = N.yl_start[b];
            int cnt = (int)(N.yl_start[b + 1] - s0);
            int4 gb = N.yl_g[b];
            double ox = N.oyx[0] + N.dls * (double)(gb.x - ga.x);
            double oy = N.oyx[1] + N.dls * (double)(gb.y - ga.y);
            double oz = N.oyx[2] + N.dls * (double)(gb.z - ga.z);
            for (int c0 = 0; c0 < cnt;) {
                int take = min(cnt - c0, P2P_SB - fill);
                for (int j = threadIdx.x; j < take; j += P2P_T) {
                    float4 y = N.epsY[s0 + c0 + j];
                    float4 yl = N.epsYlo[s0 + c0 + j];
                    double rx = ((double)y.x + (double)yl.x) + ox;
                    double ry = ((double)y.y + (double)yl.y) + oy;
                    double rz = ((double)y.z + (double)yl.z) + oz;
                    float hx = (float)rx, hy = (float)ry, hz = (float)rz;
                    sy[fill + j] = make_float4(hx, hy, hz, (float)(rx - (double)hx));
                    syl[fill + j] = make_float2((float)(ry - (double)hy), (float)(rz - (double)hz));
                    if constexpr (HELM)
                        sq[fill + j] = qc[s0 + c0 + j];
                    else
                        sq[fill + j] = make_float2(qr[s0 + c0 + j], 0.f);
                }
                fill += take;
                c0 += take;
                if (fill == P2P_SB) {
                    __syncthreads();
                    if (valid) interact<HELM>(sy, syl, sq, fill, grp, G, x, xl, N.k, sr, si);
                    __syncthreads();
                    fill = 0;
                }
            }
        }
        __syncthreads();
        if (valid) interact<HELM>(sy, syl, sq, fill, grp, G, x, xl, N.k, sr, si);
        red[threadIdx.x] = make_float2(sr, si);
        __syncthreads();
        if (valid && grp == 0) {
            float tr = 0.f, ti = 0.f;
            for (int g = 0; g < G; ++g) {
                tr += red[g * pr + pi].x;
                ti += red[g * pr + pi].y;
            }
            const double c = 0.079577471545947667884;  // 1 / (4 pi)
            double2 &dst = acc[(int64_t)m * nx + p0 + pb + pi];
            dst.x += (double)tr * c;
            dst.y += (double)ti * c;
        }
        __syncthreads();
    }
}

void near_field(const ffm_plan_s *p, const void *q, int nrhs, double2 *acc, cudaStream_t s) {
    if (p->n_near == 0) return;
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
    N.dls = std::ldexp(p->d0, -ls);
    for (int d = 0; d < 3; ++d) N.oyx[d] = p->oY[d] - p->oX[d];
    N.k = (float)p->k;
    dim3 g((unsigned)p->bx[ls].nb, nrhs);
    if (p->kind == FFM_HELMHOLTZ)
        FFM_LAUNCH(k_p2p<true>, g, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
    else
        FFM_LAUNCH(k_p2p<false>, g, P2P_T, 0, s, N, q, p->ny, nrhs, p->nx, acc);
}

}  // namespace ffm
