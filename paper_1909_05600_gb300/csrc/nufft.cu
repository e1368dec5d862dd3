// Type-3 non-uniform FFT for the plane-wave levels (Sec. 2.2.3: "the Fourier transforms are
// computed using the NUFFT" of Dutt & Rokhlin and Greengard).  For every box b of a level
//   forward   u~_b(q) = sum_{j in b} q_j e^{-i k s_q.(y_j - c_b)}
//   backward  v_i    += sum_q v~_a(q) e^{+i k s_q.(x_i - c_a)}        (x_i in box a)
// computed through grids instead of the (points x directions) exponentials:
//   forward:  spread the box's points onto an n1^3 grid of spacing h with the exponential-
//             of-semicircle kernel phi (width w), deconvolve by the Fourier coefficients of
//             the FFT-grid kernel and zero-pad to n2^3, FFT (cuFFT, sign -1), interpolate at
//             t_q = k s_q h n2 / (2 pi) with phi and apply the correction
//             prod_d 2 / (w n2 phihat(w h k s_qd / 2));
//   backward: the transposed steps in reverse order (spread the corrected v~ onto the FFT
//             grid, inverse FFT, deconvolve, interpolate at the points).
// The grid sizes follow from k, d_l and eps by one rule (w from eps, k h <= 2 pi - 2 beta / w,
// n2 >= 2 n1, 7-smooth).  GB300 layout:
//   - points are spread bin by bin (a bin is a tree box a few levels below the NUFFT level,
//     at most ~17 cells wide) into a shared-memory subgrid, then added to the box grid with
//     vector atomics; the backward interpolation stages the same subgrid and gathers;
//   - directions are the same for every box of a level, so their windows (first grid node
//     and kernel values, the correction folded in) are tabulated once per level, and the
//     backward spread runs tile by tile over the FFT grid (per-tile direction lists), each
//     tile written once: no global atomics;
//   - every box's FFT is one batch of a cuFFT plan made at plan time (the work area comes
//     from the apply's stream-ordered temporaries).
#include <cufft.h>

#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "ffm_internal.cuh"

namespace ffm {

namespace {

constexpr int NU_T = 256;       // threads of the point and tile kernels
constexpr int NU_CHUNK_S = 256;  // points per spreading block (source side)
constexpr int NU_CHUNK_T = 1024; // points per interpolation block (target side)
constexpr int NU_TILE = 8;      // FFT-grid tile edge of the backward spread
constexpr int NU_EMAX = 24;     // largest bin subgrid edge (E^3 float2 in shared memory)
constexpr int NU_PB = 64;       // points staged per round of the spreading kernel
constexpr int NU_GL = 32;       // Gauss-Legendre nodes of the kernel's Fourier transform
constexpr int NU_IB = 1;        // boxes per forward-interpolation block
constexpr int NU_BB = 64;       // directions staged per batch of the backward spread

std::mutex g_fft_mu;  // a cuFFT handle's stream and work area are set and used under one lock

void check_fft(cufftResult r, const char *what) {
    if (r != CUFFT_SUCCESS) fail(FFM_ECUDA, std::string(what) + " failed, cuFFT status " + std::to_string((int)r));
}

__device__ __forceinline__ float es_w(float z, float beta) {
    return fabsf(z) <= 1.f ? expf(beta * (sqrtf(fmaxf(0.f, 1.f - z * z)) - 1.f)) : 0.f;
}

struct NuGeo {
    int w, n1, n2, c0, E, H;  // width, grids, grid centre, bin subgrid edge, FFT-grid half
    float beta, inv_h, hs;    // kernel shape, 1 / h, h n2 / (2 pi)
};

struct NuPts {                      // one point set (sources or targets) of a NUFFT level
    const uint32_t *bin_start;      // boxes of the bin level (l + dlt): point ranges
    const int4 *bin_g;              //   and integer coordinates
    const int4 *box_g;              // boxes of the level
    const int4 *leaf_g;             // leaves
    const float4 *eps, *epslo;      // leaf-relative coordinates (hi, lo), leaf index in eps.w
    const uint32_t *slot_box;       // box of each slot (the level's source / target list)
    int dlt, dlf;                   // bin level - level, leaf level - bin level
    float bcell, lcell, corner0;    // bin and leaf edges in cells, c0 - M / 2
};

// Subgrid origin of a point block: the bin's lower corner in grid cells and the first grid
// node any of its points can reach.
__device__ __forceinline__ void bin_origin(const NuGeo &G, const NuPts &P, int4 gbin, int4 gbox, float corner[3],
                                           int lo[3]) {
    corner[0] = P.corner0 + (float)(gbin.x - (gbox.x << P.dlt)) * P.bcell;
    corner[1] = P.corner0 + (float)(gbin.y - (gbox.y << P.dlt)) * P.bcell;
    corner[2] = P.corner0 + (float)(gbin.z - (gbox.z << P.dlt)) * P.bcell;
#pragma unroll
    for (int d = 0; d < 3; ++d) lo[d] = (int)floorf(corner[d] - 0.5f * (float)G.w) + 1;
}

// Position of point pt relative to the subgrid origin, in cells, along axis d: the bin
// corner and the leaf centre are exact in FP32 (small dyadic multiples of the cell), the
// leaf-relative offset (hi + lo) is scaled by 1 / h.
__device__ __forceinline__ float point_cell(const NuPts &P, const NuGeo &G, int4 gbin, const float corner[3],
                                            const int lo[3], int pt, int d) {
    float4 e = P.eps[pt], el = P.epslo[pt];
    int4 gl = P.leaf_g[__float_as_uint(e.w)];
    int glv = d == 0 ? gl.x : d == 1 ? gl.y : gl.z;
    int gbv = d == 0 ? gbin.x : d == 1 ? gbin.y : gbin.z;
    float ev = d == 0 ? e.x : d == 1 ? e.y : e.z;
    float evl = d == 0 ? el.x : d == 1 ? el.y : el.z;
    return (corner[d] - (float)lo[d]) + ((float)(glv - (gbv << P.dlf)) + 0.5f) * P.lcell +
           fmaf(ev, G.inv_h, evl * G.inv_h);
}

// ---- forward: spread one point block into its bin subgrid, add the subgrid to the box grid.
// Each thread owns whole (i0, i1) columns of the subgrid and adds the staged points whose
// window covers its columns: no two threads write one cell, so no shared-memory atomics.
template <int W>
__global__ void __launch_bounds__(NU_T) k_nu_spread(NuGeo G, NuPts P, const int4 *__restrict__ ch,
                                                   const float2 *__restrict__ q, int64_t ny, int64_t nslot,
                                                   float2 *__restrict__ grid) {
    extern __shared__ float2 sg[];  // E^3
    __shared__ float sw[NU_PB][3][W];
    __shared__ int sf[NU_PB][3];
    __shared__ float2 sc[NU_PB];
    const int E = G.E, E3 = E * E * E;
    int4 c = ch[blockIdx.x];
    int m = blockIdx.y;
    int4 gbin = P.bin_g[c.x], gbox = P.box_g[P.slot_box[c.w]];
    float corner[3];
    int lo[3];
    bin_origin(G, P, gbin, gbox, corner, lo);
    for (int i = threadIdx.x; i < E3; i += NU_T) sg[i] = make_float2(0.f, 0.f);
    for (int base = c.y; base < c.z; base += NU_PB) {
        int cnt = min(NU_PB, c.z - base);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * 3; t += NU_T) {
            int j = t / 3, d = t % 3;
            float r = point_cell(P, G, gbin, corner, lo, base + j, d);
            int f = (int)floorf(r - 0.5f * W) + 1;
            f = min(max(f, 0), E - W);  // rounding at a bin face: the clamped node has weight ~e^-beta
            sf[j][d] = f;
#pragma unroll
            for (int a = 0; a < W; ++a) sw[j][d][a] = es_w(((float)(f + a) - r) * (2.f / W), G.beta);
        }
        for (int j = threadIdx.x; j < cnt; j += NU_T) sc[j] = q[(int64_t)m * ny + base + j];
        __syncthreads();
        for (int col = threadIdx.x; col < E * E; col += NU_T) {
            int i0 = col / E, i1 = col - i0 * E;
            float2 *colp = sg + col * E;
            for (int j = 0; j < cnt; ++j) {
                int a = i0 - sf[j][0], b = i1 - sf[j][1];
                if ((unsigned)a >= (unsigned)W || (unsigned)b >= (unsigned)W) continue;
                float wab = sw[j][0][a] * sw[j][1][b];
                float2 cj = sc[j];
                float2 *row = colp + sf[j][2];
#pragma unroll
                for (int cc = 0; cc < W; ++cc) {
                    float wt = wab * sw[j][2][cc];
                    row[cc].x = fmaf(cj.x, wt, row[cc].x);
                    row[cc].y = fmaf(cj.y, wt, row[cc].y);
                }
            }
        }
    }
    __syncthreads();
    const int n1 = G.n1;
    float2 *gb = grid + ((int64_t)m * nslot + c.w) * (int64_t)n1 * n1 * n1;
    for (int i = threadIdx.x; i < E3; i += NU_T) {
        float2 v = sg[i];
        if (v.x == 0.f && v.y == 0.f) continue;
        int a0 = lo[0] + i / (E * E), a1 = lo[1] + (i / E) % E, a2 = lo[2] + i % E;
        if (a0 < 0 || a0 >= n1 || a1 < 0 || a1 >= n1 || a2 < 0 || a2 >= n1) continue;  // outside by construction
        atomicAdd(&gb[((int64_t)a0 * n1 + a1) * n1 + a2], v);
    }
}

// ---- forward: deconvolve and zero-pad the n1^3 grids into the n2^3 FFT grids.  FFT index f
// holds the mode f (f < n2 - c0) or f - n2, i.e. grid node f + c0 or f - n2 + c0.  One block
// per (batch, f0); planes without a grid node are written as zeros.
__global__ void __launch_bounds__(256) k_nu_pad(const float2 *__restrict__ grid, const float *__restrict__ cinv,
                                                int n1, int c0, int n2, float2 *__restrict__ fine) {
    int64_t b = blockIdx.x;
    int f0 = blockIdx.y;
    int nn = n2 * n2;
    float2 *out = fine + (b * n2 + f0) * (int64_t)nn;
    int a0 = f0 < n2 - c0 ? f0 + c0 : f0 - n2 + c0;
    if (a0 >= n1) {
        for (int i = threadIdx.x; i < nn; i += blockDim.x) out[i] = make_float2(0.f, 0.f);
        return;
    }
    const float2 *in = grid + (b * n1 + a0) * (int64_t)n1 * n1;
    float s0 = cinv[a0];
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        int f1 = i / n2, f2 = i - f1 * n2;
        int a1 = f1 < n2 - c0 ? f1 + c0 : f1 - n2 + c0;
        int a2 = f2 < n2 - c0 ? f2 + c0 : f2 - n2 + c0;
        float2 v = make_float2(0.f, 0.f);
        if (a1 < n1 && a2 < n1) {
            v = in[a1 * n1 + a2];
            float sc = s0 * cinv[a1] * cinv[a2];
            v.x *= sc;
            v.y *= sc;
        }
        out[i] = v;
    }
}

// FFT-grid index of centred node u (u - H in (-n2/2, n2/2))
__device__ __forceinline__ int fft_index(int u, int H, int n2) {
    int f = u - H;
    return f < 0 ? f + n2 : f;
}

// ---- forward: interpolate the transformed grids at the directions.  A block stages one
// FFT-grid tile with its halo (the windows of the directions that start in the tile) for
// each box of its group in turn, once per box, and its threads then interpolate all the
// tile's directions from it.
constexpr int NU_IT = 128;  // threads of the interpolation block

template <int W>
__global__ void __launch_bounds__(NU_IT) k_nu_interp(NuGeo G, const float2 *__restrict__ fine,
                                                     const uint32_t *__restrict__ own_id,
                                                     const uint32_t *__restrict__ own_off,
                                                     const uint32_t *__restrict__ own_q,
                                                     const int4 *__restrict__ dirU, const float *__restrict__ dirW,
                                                     int nQ, const uint32_t *__restrict__ slot_box, int64_t nslot,
                                                     int nrhs, float2 *__restrict__ ut) {
    // the staged tile holds real and imaginary parts in separate planes with odd row and
    // plane strides: the directions of a warp start their windows at offsets (ox, oy) that
    // differ by small integers, and odd strides spread those reads over the banks
    constexpr int X = NU_TILE + W - 1, X3 = X * X * X;
    constexpr int XP = X | 1, PS = (X * XP) | 1;
    constexpr int NS = (X3 + NU_IT - 1) / NU_IT;  // staged nodes per thread
    extern __shared__ float sxs[];  // 2 planes of X * PS floats
    float *sre = sxs, *sim = sxs + X * PS;
    const int n2 = G.n2, nt = (n2 + NU_TILE - 1) / NU_TILE;
    uint32_t id = own_id[blockIdx.x];
    int u0 = (int)(id / (nt * nt)) * NU_TILE, v0 = (int)((id / nt) % nt) * NU_TILE, w0 = (int)(id % nt) * NU_TILE;
    int m = blockIdx.z;
    uint32_t e0 = own_off[blockIdx.x], e1 = own_off[blockIdx.x + 1];
    for (int bi = 0; bi < NU_IB; ++bi) {
        int64_t slot = (int64_t)blockIdx.y * NU_IB + bi;
        if (slot >= nslot) break;
        const float2 *F = fine + ((int64_t)m * nslot + slot) * (int64_t)n2 * n2 * n2;
        __syncthreads();
        // compile-time trip count: the loads of several nodes are in flight together
#pragma unroll 4
        for (int sI = 0; sI < NS; ++sI) {
            int i = sI * NU_IT + (int)threadIdx.x;
            if (i < X3) {
                int a = i / (X * X), b = (i / X) % X, cc = i % X;
                int u = u0 + a, v = v0 + b, w = w0 + cc;
                float2 g = make_float2(0.f, 0.f);
                if (u < n2 && v < n2 && w < n2)
                    g = F[((int64_t)fft_index(u, G.H, n2) * n2 + fft_index(v, G.H, n2)) * n2 +
                          fft_index(w, G.H, n2)];
                sre[a * PS + b * XP + cc] = g.x;
                sim[a * PS + b * XP + cc] = g.y;
            }
        }
        __syncthreads();
        for (uint32_t e = e0 + threadIdx.x; e < e1; e += NU_IT) {
            const int q = (int)own_q[e];
            const int4 U = dirU[q];
            const float *wq = dirW + (size_t)q * 3 * W;
            float w0v[W], w1v[W], w2v[W];
#pragma unroll
            for (int a = 0; a < W; ++a) {
                w0v[a] = wq[a];
                w1v[a] = wq[W + a];
                w2v[a] = wq[2 * W + a];
            }
            const int ox = U.x - u0, oy = U.y - v0, oz = U.z - w0;  // in [0, NU_TILE) for an owned direction
            float ax = 0.f, ay = 0.f;
#pragma unroll
            for (int a = 0; a < W; ++a) {
                float bx = 0.f, by = 0.f;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    const int r0 = (ox + a) * PS + (oy + b) * XP + oz;
                    float cx = 0.f, cy = 0.f;
#pragma unroll
                    for (int c = 0; c < W; ++c) {
                        cx = fmaf(sre[r0 + c], w2v[c], cx);
                        cy = fmaf(sim[r0 + c], w2v[c], cy);
                    }
                    bx = fmaf(cx, w1v[b], bx);
                    by = fmaf(cy, w1v[b], by);
                }
                ax = fmaf(bx, w0v[a], ax);
                ay = fmaf(by, w0v[a], ay);
            }
            ut[((int64_t)slot_box[slot] * nrhs + m) * nQ + q] = make_float2(ax, ay);
        }
    }
}

// ---- backward: spread the corrected v~ onto one FFT-grid tile.  A warp owns one tile
// column (NU_TILE cells along z, in registers) for 32 boxes, one box per lane; the tile's
// directions (those whose window meets the tile) are staged in shared memory in batches,
// with the 32 boxes' v~ side by side and each direction's z weights shifted onto the
// tile's cells (zero outside the window).  Per batch a warp finds the directions whose
// window covers its column with one ballot per 32 directions and visits only those.  Each
// tile of each box is written once, no atomics.  Block: 16 warps = 16 of the tile's 64
// columns.
template <int W>
__global__ void __launch_bounds__(512) k_nu_bspread(NuGeo G, const uint32_t *__restrict__ tile_id,
                                                    const uint32_t *__restrict__ tile_off,
                                                    const uint32_t *__restrict__ tile_q,
                                                    const int4 *__restrict__ dirU, const float *__restrict__ dirW,
                                                    int nQ, const uint32_t *__restrict__ slot_box, int64_t nslot,
                                                    int nrhs, const float2 *__restrict__ vt,
                                                    float2 *__restrict__ fine) {
    constexpr int T = NU_TILE;
    static_assert(NU_BB == 64 && T == 8, "two ballots per batch, two float4 of z weights");
    __shared__ int4 sU[NU_BB];
    __shared__ float sW[NU_BB][2 * W];
    __shared__ __align__(16) float sWz[NU_BB][T];
    __shared__ float2 sz[NU_BB][32];
    const int n2 = G.n2, nt = (n2 + T - 1) / T;
    int m = blockIdx.z >> 2, cq = blockIdx.z & 3;
    uint32_t id = tile_id[blockIdx.x];
    int u0 = (int)(id / (nt * nt)) * T, v0 = (int)((id / nt) % nt) * T, w0 = (int)(id % nt) * T;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int col = cq * 16 + warp;
    int i0 = col >> 3, i1 = col & 7;
    int64_t slot = (int64_t)blockIdx.y * 32 + lane;
    float ax[T], ay[T];
#pragma unroll
    for (int cc = 0; cc < T; ++cc) ax[cc] = ay[cc] = 0.f;
    for (int t = threadIdx.x; t < NU_BB * T; t += blockDim.x) sWz[t / T][t % T] = 0.f;
    uint32_t e0 = tile_off[blockIdx.x], e1 = tile_off[blockIdx.x + 1];
    for (uint32_t eb = e0; eb < e1; eb += NU_BB) {
        int cnt = (int)min((uint32_t)NU_BB, e1 - eb);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt * 3 * W; t += blockDim.x) {
            int j = t / (3 * W), k = t - j * (3 * W);
            float wv = dirW[(size_t)tile_q[eb + j] * 3 * W + k];
            if (k < 2 * W)
                sW[j][k] = wv;
            else {
                // z weight of window node k - 2W: cell w0 + cc of the tile with
                // cc = U.z + (k - 2W) - w0
                int cc = dirU[tile_q[eb + j]].z + (k - 2 * W) - w0;
                if ((unsigned)cc < (unsigned)T) sWz[j][cc] = wv;
            }
        }
        for (int t = threadIdx.x; t < cnt; t += blockDim.x) sU[t] = dirU[tile_q[eb + t]];
        for (int t = threadIdx.x; t < cnt * 32; t += blockDim.x) {
            int j = t >> 5, b = t & 31;
            int64_t sl = (int64_t)blockIdx.y * 32 + b;
            sz[j][b] = sl < nslot ? vt[((int64_t)slot_box[sl] * nrhs + m) * nQ + tile_q[eb + j]] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        // which directions of the batch cover this warp's column (u0 + i0, v0 + i1): bit j of
        // the 64-bit mask
        uint64_t mk = 0;
        {
            int4 U0 = lane < cnt ? sU[lane] : make_int4(-(1 << 20), 0, 0, 0);
            int4 U1 = lane + 32 < cnt ? sU[lane + 32] : make_int4(-(1 << 20), 0, 0, 0);
            bool c0 = (unsigned)(u0 + i0 - U0.x) < (unsigned)W && (unsigned)(v0 + i1 - U0.y) < (unsigned)W;
            bool c1 = (unsigned)(u0 + i0 - U1.x) < (unsigned)W && (unsigned)(v0 + i1 - U1.y) < (unsigned)W;
            mk = (uint64_t)__ballot_sync(0xffffffffu, c0) | ((uint64_t)__ballot_sync(0xffffffffu, c1) << 32);
        }
        while (mk) {
            int j = __ffsll((long long)mk) - 1;
            mk &= mk - 1;
            int4 U = sU[j];
            float wab = sW[j][u0 + i0 - U.x] * sW[j][W + (v0 + i1 - U.y)];
            float2 z = sz[j][lane];
            float zx = z.x * wab, zy = z.y * wab;
            float4 wa = *reinterpret_cast<const float4 *>(&sWz[j][0]);
            float4 wb = *reinterpret_cast<const float4 *>(&sWz[j][4]);
            ax[0] = fmaf(zx, wa.x, ax[0]);
            ay[0] = fmaf(zy, wa.x, ay[0]);
            ax[1] = fmaf(zx, wa.y, ax[1]);
            ay[1] = fmaf(zy, wa.y, ay[1]);
            ax[2] = fmaf(zx, wa.z, ax[2]);
            ay[2] = fmaf(zy, wa.z, ay[2]);
            ax[3] = fmaf(zx, wa.w, ax[3]);
            ay[3] = fmaf(zy, wa.w, ay[3]);
            ax[4] = fmaf(zx, wb.x, ax[4]);
            ay[4] = fmaf(zy, wb.x, ay[4]);
            ax[5] = fmaf(zx, wb.y, ax[5]);
            ay[5] = fmaf(zy, wb.y, ay[5]);
            ax[6] = fmaf(zx, wb.z, ax[6]);
            ay[6] = fmaf(zy, wb.z, ay[6]);
            ax[7] = fmaf(zx, wb.w, ax[7]);
            ay[7] = fmaf(zy, wb.w, ay[7]);
        }
        __syncthreads();
        // the next batch's z weights start from zero
        for (int t = threadIdx.x; t < NU_BB * T; t += blockDim.x) sWz[t / T][t % T] = 0.f;
    }
    if (slot >= nslot) return;
    int u = u0 + i0, v = v0 + i1;
    if (u >= n2 || v >= n2) return;
    float2 *F = fine + ((int64_t)m * nslot + slot) * (int64_t)n2 * n2 * n2 +
                ((int64_t)fft_index(u, G.H, n2) * n2 + fft_index(v, G.H, n2)) * n2;
#pragma unroll
    for (int cc = 0; cc < T; ++cc) {
        int w = w0 + cc;
        if (w < n2) F[fft_index(w, G.H, n2)] = make_float2(ax[cc], ay[cc]);
    }
}

// ---- backward: deconvolve the box grid into a bin subgrid and interpolate at its points
template <int W>
__global__ void __launch_bounds__(NU_T) k_nu_binterp(NuGeo G, NuPts P, const int4 *__restrict__ ch,
                                                    const float2 *__restrict__ fine, const float *__restrict__ cinv,
                                                    int64_t nslot, int64_t nx, double2 *__restrict__ acc) {
    extern __shared__ float2 sg[];  // E^3
    const int E = G.E, E3 = E * E * E, n1 = G.n1, n2 = G.n2, c0 = G.c0;
    int4 c = ch[blockIdx.x];
    int m = blockIdx.y;
    int4 gbin = P.bin_g[c.x], gbox = P.box_g[P.slot_box[c.w]];
    float corner[3];
    int lo[3];
    bin_origin(G, P, gbin, gbox, corner, lo);
    const float2 *F = fine + ((int64_t)m * nslot + c.w) * (int64_t)n2 * n2 * n2;
    for (int i = threadIdx.x; i < E3; i += NU_T) {
        int a0 = lo[0] + i / (E * E), a1 = lo[1] + (i / E) % E, a2 = lo[2] + i % E;
        float2 v = make_float2(0.f, 0.f);
        if (a0 >= 0 && a0 < n1 && a1 >= 0 && a1 < n1 && a2 >= 0 && a2 < n1) {
            int f0 = a0 - c0, f1 = a1 - c0, f2 = a2 - c0;
            f0 += f0 < 0 ? n2 : 0;
            f1 += f1 < 0 ? n2 : 0;
            f2 += f2 < 0 ? n2 : 0;
            v = F[((int64_t)f0 * n2 + f1) * n2 + f2];
            float sc = cinv[a0] * cinv[a1] * cinv[a2];
            v.x *= sc;
            v.y *= sc;
        }
        sg[i] = v;
    }
    __syncthreads();
    for (int pt = c.y + threadIdx.x; pt < c.z; pt += NU_T) {
        float w[3][W];
        int f[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            float r = point_cell(P, G, gbin, corner, lo, pt, d);
            f[d] = min(max((int)floorf(r - 0.5f * W) + 1, 0), E - W);
#pragma unroll
            for (int a = 0; a < W; ++a) w[d][a] = es_w(((float)(f[d] + a) - r) * (2.f / W), G.beta);
        }
        float sx = 0.f, sy = 0.f;
#pragma unroll
        for (int a = 0; a < W; ++a) {
            float bx = 0.f, by = 0.f;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float2 *row = sg + ((f[0] + a) * E + (f[1] + b)) * E + f[2];
                float cx = 0.f, cy = 0.f;
#pragma unroll
                for (int cc = 0; cc < W; ++cc) {
                    float2 g = row[cc];
                    cx = fmaf(g.x, w[2][cc], cx);
                    cy = fmaf(g.y, w[2][cc], cy);
                }
                bx = fmaf(cx, w[1][b], bx);
                by = fmaf(cy, w[1][b], by);
            }
            sx = fmaf(bx, w[0][a], sx);
            sy = fmaf(by, w[0][a], sy);
        }
        double2 &dst = acc[(int64_t)m * nx + pt];
        dst.x += (double)sx;
        dst.y += (double)sy;
    }
}

// ---- plan time: direction windows, kernel values and corrections
struct GlTab {
    float t[NU_GL], wphi[NU_GL];  // Gauss-Legendre nodes and weight * phi(node)
};

__device__ __forceinline__ float es_hat(float xi, const GlTab &g) {
    float s = 0.f;
#pragma unroll 8
    for (int i = 0; i < NU_GL; ++i) s = fmaf(g.wphi[i], cosf(xi * g.t[i]), s);
    return s;
}

template <int W>
__global__ void k_nu_dirs(NuGeo G, GlTab gl, float a1, const float4 *__restrict__ ks, int nQ,
                          int4 *__restrict__ dirU, float *__restrict__ dirW) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nQ) return;
    float4 k4 = ks[q];
    float kv[3] = {k4.x, k4.y, k4.z};
    int U[3];
    float corr = 1.f;
    float *wq = dirW + (size_t)q * 3 * W;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float t = kv[d] * G.hs;
        int f = (int)floorf(t - 0.5f * W) + 1;
        U[d] = f + G.H;
        for (int a = 0; a < W; ++a) wq[d * W + a] = es_w(((float)(f + a) - t) * (2.f / W), G.beta);
        corr *= 2.f / ((float)W * (float)G.n2 * es_hat(a1 * kv[d], gl));
    }
    for (int a = 0; a < W; ++a) wq[a] *= corr;  // the correction rides on the first axis
    dirU[q] = make_int4(U[0], U[1], U[2], 0);
}

// Per-tile direction lists: with own = 0 every tile a direction's window meets (backward
// spread), with own = 1 only the tile holding the window's first node (forward
// interpolation).  Counted first (pos == nullptr), then emitted at the cursors pos.
__global__ void k_nu_tile_count(const int4 *__restrict__ dirU, int nQ, int W, int nt, int own,
                                uint32_t *__restrict__ cnt, uint32_t *__restrict__ pos, uint32_t *__restrict__ tile_q) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nQ) return;
    int4 U = dirU[q];
    int ext = own ? 0 : W - 1;
    for (int a = U.x / NU_TILE; a <= (U.x + ext) / NU_TILE; ++a)
        for (int b = U.y / NU_TILE; b <= (U.y + ext) / NU_TILE; ++b)
            for (int c = U.z / NU_TILE; c <= (U.z + ext) / NU_TILE; ++c) {
                uint32_t t = ((uint32_t)a * nt + b) * nt + c;
                if (pos)
                    tile_q[atomicAdd(&pos[t], 1u)] = (uint32_t)q;
                else
                    atomicAdd(&cnt[t], 1u);
            }
}

// ---- plan time: point blocks (bin, first point, end point, slot) of the bins under the
// level's listed boxes
__global__ void k_nu_slot_of(const uint32_t *__restrict__ list, int64_t n, int *__restrict__ slot_of) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot_of[list[i]] = (int)i;
}

__global__ void k_nu_bins(const uint32_t *__restrict__ bin_start, int64_t nbin, const uint32_t *__restrict__ box_start,
                          int64_t nbox, const int *__restrict__ slot_of, uint32_t chunk, uint32_t *__restrict__ cnt,
                          const uint32_t *__restrict__ pos, int4 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbin) return;
    uint32_t s0 = bin_start[i], s1 = bin_start[i + 1];
    // the level box holding the bin: the last box starting at or before s0
    int64_t lo = 0, hi = nbox;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (box_start[mid] <= s0)
            lo = mid;
        else
            hi = mid;
    }
    int slot = slot_of[lo];
    uint32_t n = slot < 0 ? 0u : (s1 - s0 + chunk - 1) / chunk;
    if (!out) {
        cnt[i] = n;
        return;
    }
    uint32_t k = pos[i];
    for (uint32_t a = s0; n > 0 && a < s1; a += chunk) out[k++] = make_int4((int)i, (int)a, (int)min(s1, a + chunk), slot);
}

struct Params {
    int w, M, n1, n2;
    double beta;
};

bool smooth7(int n) {
    for (int p = 2; p <= 7; ++p)
        while (n % p == 0) n /= p;
    return n == 1;
}

// The NUFFT parameters of a level: width from eps, spreading grid fine enough that the
// kernel's band clears the aliased copies (k h <= 2 pi - 2 beta / w), FFT grid at least twice
// the spreading grid with no prime factor above 7.
Params nu_params(double dl, double k, double eps) {
    Params P;
    P.w = std::min(12, std::max(6, (int)std::ceil(-std::log10(eps)) + 4));
    P.beta = 2.30 * P.w;
    P.M = std::max(1, (int)std::ceil(dl * k / (2.0 * PI - 2.0 * P.beta / P.w)));
    P.n1 = P.M + P.w + 2;
    P.n1 += P.n1 & 1;
    P.n2 = 2 * P.n1;
    while (!smooth7(P.n2)) ++P.n2;
    return P;
}

double es_hat_host(double xi, double beta, const std::vector<double> &t, const std::vector<double> &wq) {
    double s = 0.0;
    for (size_t i = 0; i < t.size(); ++i) {
        double z = t[i];
        s += wq[i] * std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0)) * std::cos(xi * z);
    }
    return s;
}

int4 *build_point_blocks(ffm_plan_s *p, const BoxLevel &bins, const BoxLevel &boxes, const uint32_t *list,
                         int64_t nlist, uint32_t chunk, int64_t *count, Alloc &tmp, cudaStream_t s) {
    int *slot_of = tmp.get<int>(boxes.nb);
    FFM_CUDA(cudaMemsetAsync(slot_of, 0xff, sizeof(int) * boxes.nb, s));
    FFM_LAUNCH(k_nu_slot_of, cdiv(nlist, 256), 256, 0, s, list, nlist, slot_of);
    uint32_t *cnt = tmp.get<uint32_t>(bins.nb), *pos = tmp.get<uint32_t>(bins.nb), *tot = tmp.get<uint32_t>(1);
    FFM_LAUNCH(k_nu_bins, cdiv(bins.nb, 256), 256, 0, s, bins.start, bins.nb, boxes.start, boxes.nb, slot_of, chunk,
               cnt, (const uint32_t *)nullptr, (int4 *)nullptr);
    scan_u32(cnt, pos, bins.nb, tot, tmp, s);
    uint32_t n = 0;
    FFM_CUDA(cudaMemcpyAsync(&n, tot, sizeof n, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    *count = n;
    int4 *out = p->mem.get<int4>(n);
    FFM_LAUNCH(k_nu_bins, cdiv(bins.nb, 256), 256, 0, s, bins.start, bins.nb, boxes.start, boxes.nb, slot_of, chunk,
               cnt, pos, out);
    return out;
}

void tile_lists(ffm_plan_s *p, int l, int own, int64_t *n_tiles, uint32_t **ids_out, uint32_t **off_out,
                uint32_t **q_out, uint32_t *max_len, Alloc &tmp, cudaStream_t s) {
    FarLevel &F = p->far[l];
    NuLevel &N = F.nu;
    int nt = (N.n2 + NU_TILE - 1) / NU_TILE;
    int64_t ntt = (int64_t)nt * nt * nt;
    uint32_t *cnt = tmp.get<uint32_t>(ntt);
    FFM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * ntt, s));
    FFM_LAUNCH(k_nu_tile_count, cdiv(F.nQ, 128), 128, 0, s, (const int4 *)N.dirU, F.nQ, N.w, nt, own, cnt,
               (uint32_t *)nullptr, (uint32_t *)nullptr);
    std::vector<uint32_t> hc(ntt);
    FFM_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(uint32_t) * ntt, cudaMemcpyDeviceToHost, s));
    FFM_CUDA(cudaStreamSynchronize(s));
    std::vector<uint32_t> pos(ntt), ids, off;
    uint32_t run = 0;
    *max_len = 0;
    for (int64_t t = 0; t < ntt; ++t) {
        pos[t] = run;
        *max_len = std::max(*max_len, hc[t]);
        if (hc[t]) {
            ids.push_back((uint32_t)t);
            off.push_back(run);
        }
        run += hc[t];
    }
    off.push_back(run);
    *n_tiles = (int64_t)ids.size();
    *ids_out = p->mem.get<uint32_t>(ids.size());
    *off_out = p->mem.get<uint32_t>(off.size());
    *q_out = p->mem.get<uint32_t>(run);
    uint32_t *dpos = tmp.get<uint32_t>(ntt);
    FFM_CUDA(cudaMemcpyAsync(*ids_out, ids.data(), sizeof(uint32_t) * ids.size(), cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(*off_out, off.data(), sizeof(uint32_t) * off.size(), cudaMemcpyHostToDevice, s));
    FFM_CUDA(cudaMemcpyAsync(dpos, pos.data(), sizeof(uint32_t) * ntt, cudaMemcpyHostToDevice, s));
    FFM_LAUNCH(k_nu_tile_count, cdiv(F.nQ, 128), 128, 0, s, (const int4 *)N.dirU, F.nQ, N.w, nt, own, cnt, dpos,
               *q_out);
    FFM_CUDA(cudaStreamSynchronize(s));  // the host vectors feed the copies above
}

// cuFFT plans depend only on (n2, batch) and the device; they are made once per process and
// shared by every FFM plan (use is serialised by g_fft_mu, each call sets its own stream and
// work area).  They live until the process exits.
struct FftKey {
    int dev, n2;
    int64_t batch;
    bool operator<(const FftKey &o) const {
        return dev != o.dev ? dev < o.dev : n2 != o.n2 ? n2 < o.n2 : batch < o.batch;
    }
};
struct FftPlan {
    cufftHandle h;
    size_t work;
};
std::map<FftKey, FftPlan> g_fft_cache;

cufftHandle make_fft_uncached(int n2, int64_t batch, size_t *work) {
    cufftHandle h;
    check_fft(cufftCreate(&h), "cufftCreate");
    check_fft(cufftSetAutoAllocation(h, 0), "cufftSetAutoAllocation");
    long long n[3] = {n2, n2, n2};
    long long dist = (long long)n2 * n2 * n2;
    check_fft(cufftMakePlanMany64(h, 3, n, nullptr, 1, dist, nullptr, 1, dist, CUFFT_C2C, (long long)batch, work),
              "cufftMakePlanMany64");
    return h;
}

cufftHandle make_fft(int n2, int64_t batch, size_t *work) {
    int dev = 0;
    FFM_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_fft_mu);
    FftKey key{dev, n2, batch};
    auto it = g_fft_cache.find(key);
    if (it == g_fft_cache.end()) {
        FftPlan fp;
        fp.h = make_fft_uncached(n2, batch, &fp.work);
        it = g_fft_cache.emplace(key, fp).first;
    }
    *work = it->second.work;
    return it->second.h;
}

// one transform per right-hand side, each over all boxes of the level, in place
void exec_fft(cufftHandle h, size_t work, float2 *data, int64_t per_rhs, int nrhs, int dir, Alloc &tmp,
              cudaStream_t s) {
    void *wa = tmp.raw(work > 0 ? work : 16);
    std::lock_guard<std::mutex> lk(g_fft_mu);
    check_fft(cufftSetStream(h, s), "cufftSetStream");
    check_fft(cufftSetWorkArea(h, wa), "cufftSetWorkArea");
    // the library's kernels are timed as one entry by the profile hooks (not counted as ours)
    bool prof = g_profile && !g_capture_count;
    if (prof) profile_begin("cufftExecC2C (library)", s);
    for (int m = 0; m < nrhs; ++m) {
        cufftComplex *d = reinterpret_cast<cufftComplex *>(data + (int64_t)m * per_rhs);
        check_fft(cufftExecC2C(h, d, d, dir), "cufftExecC2C");
    }
    if (prof) profile_end(s);
}

NuGeo geo_of(const NuLevel &N) {
    NuGeo G;
    G.w = N.w;
    G.n1 = N.n1;
    G.n2 = N.n2;
    G.c0 = N.n1 / 2;
    G.E = N.E;
    G.H = N.n2 / 2;
    G.beta = (float)N.beta;
    G.inv_h = (float)(1.0 / N.h);
    G.hs = (float)(N.h * N.n2 / (2.0 * PI));
    return G;
}

NuPts pts_of(const ffm_plan_s *p, int l, bool src) {
    const NuLevel &N = p->far[l].nu;
    const BoxLevel *B = src ? p->by : p->bx;
    int ls = p->l_stop, lb = l + N.dlt;
    NuPts P;
    P.bin_start = B[lb].start;
    P.bin_g = B[lb].g;
    P.box_g = B[l].g;
    P.leaf_g = B[ls].g;
    P.eps = src ? p->epsY : p->epsX;
    P.epslo = src ? p->epsYlo : p->epsXlo;
    P.slot_box = src ? p->far[l].src : p->far[l].tgt;
    P.dlt = N.dlt;
    P.dlf = ls - lb;
    P.bcell = (float)std::ldexp((double)N.M, -N.dlt);
    P.lcell = (float)std::ldexp((double)N.M, -(ls - l));
    P.corner0 = (float)(N.n1 / 2) - 0.5f * (float)N.M;
    return P;
}

template <int W>
void launch_forward(const ffm_plan_s *p, int l, const float2 *q, int nrhs, float2 *ut, Alloc &tmp, cudaStream_t s) {
    const FarLevel &F = p->far[l];
    const NuLevel &N = F.nu;
    NuGeo G = geo_of(N);
    NuPts P = pts_of(p, l, true);
    int64_t ns = F.n_src;
    int64_t N1 = (int64_t)N.n1 * N.n1 * N.n1, N2 = (int64_t)N.n2 * N.n2 * N.n2;
    float2 *grid = tmp.get<float2>(ns * nrhs * N1);
    FFM_CUDA(cudaMemsetAsync(grid, 0, sizeof(float2) * ns * nrhs * N1, s));
    size_t smem = sizeof(float2) * N.E * N.E * N.E;
    FFM_CUDA(cudaFuncSetAttribute(k_nu_spread<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FFM_LAUNCH(k_nu_spread<W>, dim3((unsigned)N.n_ych, nrhs), NU_T, smem, s, G, P, N.ych, q, p->ny, ns, grid);
    float2 *fine = tmp.get<float2>(ns * nrhs * N2);
    FFM_LAUNCH(k_nu_pad, dim3((unsigned)(ns * nrhs), N.n2), 256, 0, s, (const float2 *)grid, N.cinv, N.n1,
               N.n1 / 2, N.n2, fine);
    tmp.drop(grid);
    exec_fft(N.fft_src, N.work_src, fine, ns * N2, nrhs, CUFFT_FORWARD, tmp, s);
    constexpr int X = NU_TILE + W - 1;
    size_t xs = 2 * sizeof(float) * X * ((X * (X | 1)) | 1);
    FFM_CUDA(cudaFuncSetAttribute(k_nu_interp<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)xs));
    FFM_LAUNCH(k_nu_interp<W>, dim3((unsigned)N.n_own, cdiv(ns, NU_IB), nrhs), NU_IT, xs, s, G, (const float2 *)fine,
               N.own_id, N.own_off, N.own_q, N.dirU, N.dirW, F.nQ, F.src, ns, nrhs, ut);
    tmp.drop(fine);
}

template <int W>
void launch_backward(const ffm_plan_s *p, int l, const float2 *vt, int nrhs, double2 *acc, Alloc &tmp,
                     cudaStream_t s) {
    const FarLevel &F = p->far[l];
    const NuLevel &N = F.nu;
    NuGeo G = geo_of(N);
    NuPts P = pts_of(p, l, false);
    int64_t nt = F.n_tgt;
    int64_t N2 = (int64_t)N.n2 * N.n2 * N.n2;
    float2 *fine = tmp.get<float2>(nt * nrhs * N2);
    FFM_CUDA(cudaMemsetAsync(fine, 0, sizeof(float2) * nt * nrhs * N2, s));
    FFM_LAUNCH(k_nu_bspread<W>, dim3((unsigned)N.n_tiles, cdiv(nt, 32), 4 * nrhs), 512, 0, s, G, N.tile_id, N.tile_off,
               N.tile_q, N.dirU, N.dirW, F.nQ, F.tgt, nt, nrhs, vt, fine);
    exec_fft(N.fft_tgt, N.work_tgt, fine, nt * N2, nrhs, CUFFT_INVERSE, tmp, s);
    size_t smem = sizeof(float2) * N.E * N.E * N.E;
    FFM_CUDA(cudaFuncSetAttribute(k_nu_binterp<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FFM_LAUNCH(k_nu_binterp<W>, dim3((unsigned)N.n_xch, nrhs), NU_T, smem, s, G, P, N.xch, (const float2 *)fine,
               N.cinv, nt, p->nx, acc);
    tmp.drop(fine);
}

template <int W>
void launch_dirs(ffm_plan_s *p, int l, const GlTab &gl, float a1, cudaStream_t s) {
    FarLevel &F = p->far[l];
    NuLevel &N = F.nu;
    FFM_LAUNCH(k_nu_dirs<W>, cdiv(F.nQ, 128), 128, 0, s, geo_of(N), gl, a1, (const float4 *)F.ks, F.nQ, N.dirU,
               N.dirW);
}

#define NU_DISPATCH(w, fn, ...)                                            \
    switch (w) {                                                          \
        case 6: fn<6>(__VA_ARGS__); break;                                \
        case 7: fn<7>(__VA_ARGS__); break;                                \
        case 8: fn<8>(__VA_ARGS__); break;                                \
        case 9: fn<9>(__VA_ARGS__); break;                                \
        case 10: fn<10>(__VA_ARGS__); break;                              \
        case 11: fn<11>(__VA_ARGS__); break;                              \
        case 12: fn<12>(__VA_ARGS__); break;                              \
        default: fail(FFM_EUNSUPPORTED, "NUFFT width outside 6..12");     \
    }

}  // namespace

bool nufft_possible(const ffm_plan_s *p, int l) {
    const FarLevel &F = p->far[l];
    if (F.mode != 2 || F.n_adm == 0 || !F.ks) return false;
    Params P = nu_params(std::ldexp(p->d0, -l), p->k, p->eps);
    int dlt = 0;
    while (std::ldexp((double)P.M, -dlt) + P.w + 1 > NU_EMAX) ++dlt;
    // boxes index grid.y of the per-box kernels
    return l + dlt <= p->l_stop && F.n_src <= 65535 && F.n_tgt <= 65535;
}

void build_nufft(ffm_plan_s *p, int l, Alloc &tmp, cudaStream_t s) {
    FarLevel &F = p->far[l];
    NuLevel &N = F.nu;
    double dl = std::ldexp(p->d0, -l);
    Params P = nu_params(dl, p->k, p->eps);
    N.w = P.w;
    N.beta = P.beta;
    N.M = P.M;
    N.n1 = P.n1;
    N.n2 = P.n2;
    N.h = dl / P.M;
    N.dlt = 0;
    while (std::ldexp((double)P.M, -N.dlt) + P.w + 1 > NU_EMAX) ++N.dlt;
    N.E = (int)std::floor(std::ldexp((double)P.M, -N.dlt)) + P.w + 1;
    // deconvolution of the FFT-grid kernel: 1 / c(m'), c(m') = (a2 / 2 pi) phihat(a2 m'),
    // a2 = w pi / n2 (host FP64, 64-node Gauss-Legendre)
    std::vector<double> gt, gw;
    gauss_legendre_nodes(64, gt, gw);
    std::vector<float> cinv(N.n1);
    double a2 = N.w * PI / N.n2;
    for (int m = 0; m < N.n1; ++m) cinv[m] = (float)(2.0 * PI / (a2 * es_hat_host(a2 * (m - N.n1 / 2), N.beta, gt, gw)));
    N.cinv = p->mem.get<float>(N.n1);
    FFM_CUDA(cudaMemcpyAsync(N.cinv, cinv.data(), sizeof(float) * N.n1, cudaMemcpyHostToDevice, s));
    // direction windows, kernel values and corrections
    std::vector<double> t32, w32;
    gauss_legendre_nodes(NU_GL, t32, w32);
    GlTab gl;
    for (int i = 0; i < NU_GL; ++i) {
        gl.t[i] = (float)t32[i];
        gl.wphi[i] = (float)(w32[i] * std::exp(N.beta * (std::sqrt(1.0 - t32[i] * t32[i]) - 1.0)));
    }
    N.dirU = p->mem.get<int4>(F.nQ);
    N.dirW = p->mem.get<float>((size_t)F.nQ * 3 * N.w);
    float a1 = (float)(0.5 * N.w * N.h);
    NU_DISPATCH(N.w, launch_dirs, p, l, gl, a1, s);
    // per-tile direction lists: every tile a window meets (backward spread), and the tile
    // holding each window's first node (forward interpolation)
    uint32_t tmax = 0;
    tile_lists(p, l, 0, &N.n_tiles, &N.tile_id, &N.tile_off, &N.tile_q, &tmax, tmp, s);
    tile_lists(p, l, 1, &N.n_own, &N.own_id, &N.own_off, &N.own_q, &N.own_max, tmp, s);
    // point blocks of the source and target bins
    int lb = l + N.dlt;
    N.ych = build_point_blocks(p, p->by[lb], p->by[l], F.src, F.n_src, NU_CHUNK_S, &N.n_ych, tmp, s);
    N.xch = build_point_blocks(p, p->bx[lb], p->bx[l], F.tgt, F.n_tgt, NU_CHUNK_T, &N.n_xch, tmp, s);
    // one cuFFT plan per side, batched over the level's boxes
    N.fft_src = make_fft(N.n2, F.n_src, &N.work_src);
    N.fft_tgt = make_fft(N.n2, F.n_tgt, &N.work_tgt);
    N.has_fft = true;
    F.nufft = 1;
    FFM_CUDA(cudaStreamSynchronize(s));  // the host vectors above feed asynchronous copies
    p->info.nufft[l] = 1;
    p->info.nufft_w[l] = N.w;
    p->info.nufft_n2[l] = N.n2;
}

void nufft_forward(const ffm_plan_s *p, int l, const float2 *q, int nrhs, float2 *ut, Alloc &tmp, cudaStream_t s) {
    NU_DISPATCH(p->far[l].nu.w, launch_forward, p, l, q, nrhs, ut, tmp, s);
}

void nufft_backward(const ffm_plan_s *p, int l, const float2 *vt, int nrhs, double2 *acc, Alloc &tmp,
                    cudaStream_t s) {
    NU_DISPATCH(p->far[l].nu.w, launch_backward, p, l, vt, nrhs, acc, tmp, s);
}

void nufft_release(ffm_plan_s *p) {
    for (int l = 0; l <= LMAX; ++l) {
        NuLevel &N = p->far[l].nu;
        if (N.has_fft) {  // the cuFFT plans belong to the process-wide cache
            N.has_fft = false;
        }
    }
}

}  // namespace ffm
