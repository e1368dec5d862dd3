/*
 * ffm.h -- C ABI of the GB300 (sm_103a) Fast Free Memory library, libffm_gb300.so.
 *
 * The library evaluates the discrete convolution of Sec. 1, eqs. 3-4 of Aussal & Bakry,
 * "The Fast and Free Memory Method for the efficient computation of convolution
 * kernels" (arXiv:1909.05600):
 *
 *     v_i = sum_j  w_j G(x_i - y_j) u_j ,      i.e.  v = G W u ,
 *
 * for the Laplace kernel G = 1/(4 pi |x-y|) (Sec. 4.1, eq. 19) and the Helmholtz kernel
 * G = e^{ik|x-y|}/(4 pi |x-y|) (Sec. 2.2.3, eq. 9), by the FFM of Sec. 2: two cubic
 * octrees of equal edge (Sec. 2.2.1), a descent-only traversal with the admissibility
 * test of Sec. 2.2.2, far fields by Chebyshev-Lagrange interpolation (Sec. 2.2.2) or by
 * the Gegenbauer plane-wave expansion (Sec. 2.2.3), and a dense near field at the level
 * where the stopping criterion of Sec. 2.2.4 holds.  Pairs of coincident points
 * (|x-y| = 0) contribute nothing.
 *
 * Every step runs in CUDA kernels on the current device; no CPU fallback exists.
 *
 * Conventions
 *   - Point sets are N x 3 row-major arrays (x0,y0,z0,x1,...) of float or double.
 *   - Densities u (length N_Y per right-hand side) and results v (length N_X per
 *     right-hand side) are column-major with nrhs columns: u[j + N_Y*m].  Complex values
 *     are interleaved (re, im).
 *   - Any array argument may live in device memory or in host memory (pageable or
 *     pinned); host arrays are staged through device memory on the given stream.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls return after
 *     enqueueing their work except where noted; ffm_plan synchronises its stream a
 *     few times (pair counts decide allocation sizes).
 *   - Functions return an ffm_status; no exception crosses the ABI.  On failure, output
 *     handles are set to NULL and ffm_last_error() describes the cause.
 */
#ifndef FFM_GB300_H
#define FFM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ffm_plan_s ffm_plan_t;

typedef enum {
    FFM_OK = 0,
    FFM_EINVAL = 1,      /* bad argument: N <= 0, eps outside (0,1), k < 0, NaN input, bad dtype */
    FFM_ENOMEM = 2,      /* device allocation failed; nothing is leaked, no plan is returned */
    FFM_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    FFM_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
    FFM_EUNSUPPORTED = 5 /* valid request outside what this library implements */
} ffm_status;

/* FFM_LAPLACE_DL is the double layer of the Laplace kernel, dG/dn_y(x - y) =
 * n_y . (x - y) / (4 pi |x - y|^3) with G = 1/(4 pi |x - y|) and n_y the source normals
 * (ffm_opts.normals, required).  FFM_LAPLACE_GRAD is the gradient of the single layer in
 * the target variable, grad_x G(x - y) = -(x - y) / (4 pi |x - y|^3) (the MFIE kernel of
 * Sec. 4.2): three outputs per target and right-hand side.  Both run through the
 * kernel-independent Lagrange path (Sec. 2.2.2) with their three component kernels
 * (x - y)_d / (4 pi |x - y|^3) interpolated separately. */
typedef enum { FFM_LAPLACE = 0, FFM_HELMHOLTZ = 1, FFM_LAPLACE_DL = 2, FFM_LAPLACE_GRAD = 3 } ffm_kernel;

typedef enum {
    FFM_F32 = 0,  /* float */
    FFM_F64 = 1,  /* double */
    FFM_C64 = 2,  /* interleaved complex float */
    FFM_C128 = 3  /* interleaved complex double */
} ffm_dtype;

/* Arithmetic of the plane-wave levels (forward transform, transfer, backward transform).
 * The quadrature sum of a level cancels by the ratio C = sum_q |D(q)| / |sum_q D(q)|
 * (closest translation), which amplifies rounding errors by up to C; it is large at low
 * k d_l and small eps.  FFM_PREC_AUTO picks FP32 for C <= 250, compensated FP32 (own
 * accurate sincos, TwoSum accumulation of the direction and translation sums) for
 * C <= 4e3, double-float above, which keeps the rounding error below ~6e-6 relative.
 * FFM_PREC_F64 is the same arithmetic in FP64 (this part's FP64 rate is a small fraction
 * of its FP32 rate). */
typedef enum {
    FFM_PREC_AUTO = 0,
    FFM_PREC_F32 = 1,   /* FP32, hardware sincos approximation */
    FFM_PREC_F32C = 2,  /* FP32 with accurate sincos and compensated sums */
    FFM_PREC_F64 = 3,   /* FP64 */
    FFM_PREC_F32X2 = 4  /* double-float: unevaluated pairs of FP32 numbers (about 2^-44
                           relative) on the FP32 pipe, with their own sincos */
} ffm_precision;

/* Plan options.  Zero-initialise and set what you need; a NULL opts pointer means all
 * defaults.  The defaults are the plan constants of the method (readings of the paper
 * where it is silent): n_leaf = 64, l_cap = 21, kappa_switch = 2.0, r1 from the
 * calibrated Lagrange error table. */
typedef struct {
    int n_leaf;           /* stop refining once the mean number of points per non-empty
                             box (both trees) drops below n_leaf (Sec. 2.2.4); 0 -> 64 */
    int l_cap;            /* deepest level (<= 21); 0 -> 21 */
    double kappa_switch;  /* Helmholtz: plane waves at level l iff k d_l >= kappa_switch,
                             Lagrange otherwise (Sec. 2.2.3); 0 -> 2.0 */
    int r1_override;      /* Chebyshev nodes per axis for Lagrange levels (2..8); 0 -> rule */
    int precision;        /* plane-wave level arithmetic, one of ffm_precision; 0 -> chosen
                             per level from the quadrature's cancellation ratio */
    const void *weights;  /* quadrature weights w_j (N_Y entries), host or device; NULL -> 1 */
    ffm_dtype weights_dtype; /* FFM_F32 or FFM_F64 */
    const char *autotune_cache; /* NULL, or a file written by ffm_autotune: the plan takes the
                                   picks stored for its sizes (single right-hand side picks;
                                   several-RHS picks from 64, else 8 RHS), timing nothing */
    int lagrange_transfer;      /* Laplace Lagrange levels' transfer: 0 default (tcgen05 per
                                   translation, or ffm_autotune's pick), 1 CUDA-core GEMM per
                                   translation, 2 tcgen05 per translation, 3 tcgen05
                                   target-stationary (r <= 64) */
    const void *normals;        /* FFM_LAPLACE_DL: N_Y x 3 row-major source normals (any
                                   length; the kernel is linear in n), host or device; copied */
    ffm_dtype normals_dtype;    /* FFM_F32 or FFM_F64 */
    int pw_transform;           /* plane-wave source and target steps F_{Y->s}, F_{s->X} (Sec.
                                   2.2.3): 0 chosen per level (the type-3 NUFFT on FP32 levels
                                   with many directions, direct sums elsewhere, or
                                   ffm_autotune's pick; with 16 or more right-hand sides the
                                   direct sums of FP32 and compensated-FP32 levels run as
                                   TF32 x3 tensor-core products), 1 direct sums on the CUDA
                                   cores everywhere, 2 the NUFFT on every FP32 and
                                   compensated-FP32 plane-wave level, 3 as 0 without the NUFFT
                                   and with the tensor-core products from 2 right-hand sides
                                   (the forward transform on FP32 and compensated-FP32 levels,
                                   the backward transform on FP32 levels) */
    double aca_eps;             /* FFM_LAPLACE: 0 -> dense transfer matrices T; > 0 -> each T_t
                                   replaced by its adaptive cross approximation A_t B_t^T (Sec.
                                   2.2.2, eq. 11; full pivoting, FP64, at plan time) with
                                   |T_t - A_t B_t^T|_F <= aca_eps |T_t|_F or rank 64, and the
                                   transfer applied as A_t (B_t^T u~) (two GEMMs per translation);
                                   must be < 1; FFM_EUNSUPPORTED for the other kernels */
    int wait_tries;             /* attempts of each bounded device-side wait (the mbarrier waits
                                   of the tensor-core transfer kernels) before it gives up and
                                   the plan reports FFM_ETIMEOUT: 0 -> 2^24; > 0 -> that many;
                                   -1 -> none, every such wait gives up at once (a host-side way
                                   to exercise the failure path; results are then discarded).
                                   A kernel that gave up still waits for the tensor-core work
                                   it had committed before it frees TMEM, so a timed-out plan
                                   leaves the device usable; its results are unspecified and the
                                   plan should be destroyed */
} ffm_opts;

/* Build a plan for targets X (nx points) and sources Y (ny points) (Sec. 2.2.1-2.2.4):
 * bounding cubes, Morton sort of both sets, per-level box tables, the descent-only
 * admissible / near pair lists, and the per-level transfer operators (one per distinct
 * box translation, Sec. 3.1 proof of Prop. 1).
 *   X, Y      : N x 3 row-major, dtype xdt / ydt in {FFM_F32, FFM_F64}; copied, so the
 *               caller may free them when the call returns.
 *   kernel, k : FFM_LAPLACE (k ignored) or FFM_HELMHOLTZ with wavenumber k >= 0.
 *   eps       : requested accuracy, 0 < eps < 1 (sets the Lagrange rank and the
 *               plane-wave rank L of eq. 13).
 *   opts      : NULL or options (the weights are copied).
 *   stream    : cudaStream_t for all work.
 *   out       : receives the plan (NULL on failure).
 * Errors: FFM_EINVAL on bad arguments or non-finite coordinates, FFM_ENOMEM, FFM_ECUDA,
 * FFM_EUNSUPPORTED (eps needs r1 > 8). */
ffm_status ffm_plan(const void *X, ffm_dtype xdt, int64_t nx, const void *Y, ffm_dtype ydt, int64_t ny,
                    ffm_kernel kernel, double k, double eps, const ffm_opts *opts, void *stream,
                    ffm_plan_t **out);

/* v = G W u through the plan (Sec. 2.2, Fig. of the descent): far field of every level
 * with admissible pairs, near field at the stop level, FP64 accumulation per target.
 *   u   : N_Y x nrhs column-major; Laplace kinds: FFM_F32 or FFM_F64; Helmholtz: FFM_C64
 *         or FFM_C128.
 *   v   : N_X x nrhs column-major, same dtype as u; overwritten (not accumulated).
 *         FFM_LAPLACE_GRAD: N_X x 3 nrhs, component d of right-hand side m in column
 *         3 m + d.
 *   nrhs: number of right-hand sides, >= 1.
 * Works on `stream`; returns once the work is enqueued (device u, v) or after the
 * result has been copied back (host v).  The plan is read-only here, so concurrent
 * applies on different streams are allowed.
 * Errors: FFM_EINVAL (NULL plan, bad dtype, nrhs < 1), FFM_ENOMEM, FFM_ECUDA. */
ffm_status ffm_apply(ffm_plan_t *plan, const void *u, ffm_dtype udt, int nrhs, void *v, void *stream);

/* Release a plan and all its device memory.  NULL-safe.  Synchronises the plan's
 * stream first. */
void ffm_destroy(ffm_plan_t *plan);

/* Device bytes held by the plan (for admission by memory footprint). */
ffm_status ffm_plan_bytes(const ffm_plan_t *plan, size_t *bytes);

/* Per-level description of a plan, for tests and reports.  Arrays are indexed by the
 * level l = 0..21. mode: 0 no far field, 1 Lagrange, 2 plane waves. */
typedef struct {
    int l_stop;                /* level of the near field (leaf level) */
    int root_admissible;       /* 1 if the two roots are already far apart (level-0 far field) */
    double d0;                 /* common edge of the two root cubes */
    double oX[3], oY[3];       /* lower corners of the root cubes */
    int64_t nboxX[22], nboxY[22]; /* non-empty boxes per level (0 beyond the levels built) */
    int64_t n_adm[22];         /* admissible pairs handled at each level */
    int64_t n_near[22];        /* near pairs left after each level */
    int64_t n_trans[22];       /* distinct box translations among the admissible pairs */
    int mode[22];
    int r1[22];                /* Chebyshev nodes per axis (Lagrange levels) */
    int L[22];                 /* Gegenbauer rank (plane-wave levels) */
    int nQ[22];                /* quadrature directions 2L(L+1) (plane-wave levels) */
    int64_t nx, ny;
    int64_t src_points[22];    /* source points in boxes with admissible pairs (per level) */
    int64_t tgt_points[22];    /* target points in boxes with admissible pairs (per level) */
    int64_t p2p_pairs;         /* point pairs of the near field, sum over near leaf pairs of n_a n_b */
    int pw_prec[22];           /* plane-wave levels: the ffm_precision they run in (0 otherwise) */
    double cancel[22];         /* cancellation ratio of the level's quadrature sum (closest pair) */
    int device_errors;         /* nonzero if a bounded device-side wait gave up (results invalid) */
    /* kernel variants in use (ffm_autotune's picks, else the defaults) */
    int autotuned;             /* 1 after ffm_autotune */
    int p2p_tchunk, p2p_smax;  /* near-field work items: targets, source points per item */
    int tune_tc[22];           /* Lagrange levels' transfer: 0 CUDA-core GEMM per translation,
                                  1 tcgen05 GEMM per translation (atomic scatter), 2 tcgen05
                                  target-stationary (one write per target box) */
    int tune_pw[22][3];        /* plane-wave levels: direction pairs per thread (forward), points
                                  per thread (backward), right-hand sides per thread (several; 0:
                                  ffm_autotune picked the tensor-core transforms) */
    int nufft[22];             /* plane-wave levels whose F steps run as type-3 NUFFTs (1) */
    int nufft_w[22];           /* their spreading-kernel width */
    int nufft_n2[22];          /* their FFT grid edge (n2^3 per box) */
    int64_t n_src_boxes[22];   /* source boxes with admissible pairs (per level) */
    int64_t n_tgt_boxes[22];   /* target boxes with admissible pairs (per level) */
    int64_t pw_recurrences[22]; /* plane-wave levels: Legendre recurrences of the transfer table
                                   (one per translation pair and direction pair, L degrees each) */
    int aca_rank[22];          /* Lagrange levels with aca_eps: largest ACA rank over the level's
                                  translations (0 otherwise) */
    int64_t aca_terms[22];     /* sum of the ACA ranks over the level's translations */
    int64_t aca_pair_terms[22]; /* sum over the admissible pairs of their translation's rank */
} ffm_info;

ffm_status ffm_plan_info(const ffm_plan_t *plan, ffm_info *info);

/* Copy plan contents to host memory, for tests.
 *   what = FFM_EXPORT_PERM_X / _PERM_Y: sorted position -> original index (int64, N).
 *   what = FFM_EXPORT_ADM: admissible pairs of `level` as (X box id, Y box id) Morton ids
 *          at that level (uint64 pairs, 2*count values).
 *   what = FFM_EXPORT_NEAR: near pairs at the stop level, same format.
 * With host_out NULL only *count is set.  Blocks until the copy is done. */
enum { FFM_EXPORT_PERM_X = 0, FFM_EXPORT_PERM_Y = 1, FFM_EXPORT_ADM = 2, FFM_EXPORT_NEAR = 3 };
ffm_status ffm_plan_export(const ffm_plan_t *plan, int what, int level, void *host_out, int64_t *count);

/* Pick kernel variants for this plan by timing them on its own data, for products with
 * `nrhs` right-hand sides: the near-field work-item shape (targets and source points per
 * item, which balance clustered leaves), the Lagrange transfer (tcgen05 target-stationary
 * tiles of 128 target boxes, tcgen05 tiles of 256 box pairs of one translation, or
 * CUDA-core tiles of 32 pairs), and per plane-wave level the direction pairs and
 * points per thread of the transforms (or right-hand sides per thread).  Costs a few
 * applies of GPU time; results change only by rounding.
 *   cache_path : NULL, or a text file of earlier picks keyed by device, kernel, level
 *                sizes and nrhs; keys found there are not timed again, new picks are
 *                appended (the file is created if missing).
 *   stream     : cudaStream_t for the timing runs; the call returns when they are done.
 * Errors: FFM_EINVAL, FFM_ENOMEM, FFM_ECUDA. */
ffm_status ffm_autotune(ffm_plan_t *plan, int nrhs, const char *cache_path, void *stream);

/* A captured apply, for iterative solvers that multiply by the same matrix many times
 * with the same buffers (Sec. 4.3's BEM solves: about ten products per GMRES iteration).
 * ffm_graph_create records one ffm_apply(plan, u, udt, nrhs, v) into a CUDA graph and
 * instantiates it; nothing runs.  Each ffm_graph_launch then recomputes v from the current
 * contents of u with one graph launch instead of one launch per kernel (a few hundred for
 * a million-point Helmholtz product), its temporaries being graph-owned allocations.
 *   u, v : DEVICE buffers as for ffm_apply; the graph keeps their addresses, so they must
 *          stay allocated (and the plan alive) until ffm_graph_destroy.
 *   stream (launch): cudaStream_t; the call only enqueues work.
 * Errors: FFM_EINVAL (NULL or host buffers, bad dtype or nrhs), FFM_ENOMEM, FFM_ECUDA. */
typedef struct ffm_graph_s ffm_graph_t;
ffm_status ffm_graph_create(ffm_plan_t *plan, const void *u, ffm_dtype udt, int nrhs, void *v, ffm_graph_t **out);
ffm_status ffm_graph_launch(ffm_graph_t *graph, void *stream);
/* Kernels one launch of the graph runs (they count towards ffm_launch_count). */
int64_t ffm_graph_kernels(const ffm_graph_t *graph);
void ffm_graph_destroy(ffm_graph_t *graph);

/* Number of kernels this library has launched in this process (all threads); a graph
 * launch adds the kernels it contains. */
uint64_t ffm_launch_count(void);

/* Per-kernel device timing, for measurement.  While enabled, each kernel launch of this
 * library is bracketed by two CUDA events on its stream; ffm_profile_read synchronises on
 * those events and returns, per kernel name, the number of launches and the summed
 * device time in milliseconds since the last reset.
 *   names: buffer for up to `cap` NUL-terminated names, 64 bytes each (cap*64 bytes);
 *   launches, ms: arrays of `cap` entries.  Returns the number of entries written.
 * Not thread-safe with respect to concurrent launches from other threads. */
void ffm_profile_enable(int on);
void ffm_profile_reset(void);
int ffm_profile_read(char *names, uint64_t *launches, double *ms, int cap);

/* Morton (Z-order) ordering of one point set, computed without allocating any device
 * memory.  The paper has no counterpart: this entry point serves callers that cannot
 * allocate device memory while they run (code executing while another framework owns
 * the whole device heap, allocation-free real-time loops, hosts whose allocator policy
 * forbids cudaMalloc on their worker threads).
 *   X        : n x 3 row-major DEVICE array, FFM_F32 or FFM_F64.
 *   n        : 1 <= n <= 262144; larger n returns FFM_EINVAL (the scratch is fixed).
 *   perm_out : n uint32 DEVICE entries; receives sorted position -> original index, the
 *              same order ffm_plan gives X when called with Y = X (bounding cube, FP64
 *              quantisation, 63-bit Morton key, ties by original index).  If any
 *              coordinate is NaN or infinite (which ffm_plan refuses with FFM_EINVAL),
 *              every entry is set to 0xFFFFFFFF instead: the call does not synchronise,
 *              so that error is reported in the output, once the stream has run.
 *   stream   : cudaStream_t of the current device; the call only enqueues work.
 * Scratch: one file-scope device array of about 6.3 MB (keys, indices, histograms, cube),
 * reserved on every GPU that loads the library until the process exits; no cudaMalloc,
 * cudaFree or allocating library call is made.  The first call on each device resolves
 * the array's device address (cudaGetSymbolAddress), so make that first call before any
 * stream capture.  All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be serialised by the caller.
 * Errors: FFM_EINVAL (NULL or host pointers, memory of another device, bad dtype, n out
 * of range), FFM_ECUDA. */
ffm_status ffm_morton_order_noalloc(const void *X, ffm_dtype xdt, int64_t n, uint32_t *perm_out, void *stream);

/* ---- Boundary-element wrapper (Sec. 4.2): the Galerkin matrix of a boundary integral operator
 * written as S = (Lambda*)^T (G W) Lambda + C, where Lambda carries the basis functions to the
 * quadrature nodes, G W is one FFM product between the nodes, (Lambda*)^T brings the weighted
 * node values back to the test functions, and C is the sparse matrix that replaces the
 * singular integrals the node quadrature misses.  This version: the Laplace single layer
 * G = 1/(4 pi |x - y|) with P1 (nodal, piecewise-linear) functions on a flat-triangle mesh,
 * 3 quadrature nodes per triangle (barycentric (2/3, 1/6, 1/6) and permutations, weights
 * area / 3), and C holding each triangle's exact self-interaction (closed-form in-plane
 * potential of a linear density, collapsed 32 x 32 Gauss outer rule) minus its node
 * quadrature.  Interactions between distinct triangles use the node quadrature. */
typedef struct ffm_bem_s ffm_bem_t;

/* Build the operator for a mesh.
 *   vertices : nv x 3 row-major FP64, host or device; copied.
 *   triangles: nt x 3 int32 vertex indices (0-based), host or device; copied.
 *   kernel   : FFM_LAPLACE (others return FFM_EUNSUPPORTED); k ignored.
 *   eps      : accuracy of the FFM products; opts as for ffm_plan (its weights are replaced
 *              by the quadrature weights).
 * Errors: FFM_EINVAL (NULL, empty mesh, index out of range), FFM_ENOMEM, FFM_ECUDA. */
ffm_status ffm_bem_create(const double *vertices, int64_t nv, const int *triangles, int64_t nt, ffm_kernel kernel,
                          double k, double eps, const ffm_opts *opts, void *stream, ffm_bem_t **out);
/* v = S u for nv vertex values (FP64, host or device; v overwritten). */
ffm_status ffm_bem_apply(ffm_bem_t *bem, const double *u, double *v, void *stream);
/* Solve S x = rhs by restarted GMRES (restart vectors, at most maxit products, stop at
 * ||rhs - S x|| <= tol ||rhs|| by the GMRES residual estimate); x (FP64, host or device)
 * receives the solution, *iters the products used, *relres the final relative residual.
 * x starts from 0. */
ffm_status ffm_bem_solve(ffm_bem_t *bem, const double *rhs, double *x, double tol, int restart, int maxit,
                         int *iters, double *relres, void *stream);
/* FFM products of the last solve (Arnoldi steps plus restarts). */
ffm_status ffm_bem_products(const ffm_bem_t *bem, int64_t *products);
/* NULL-safe; synchronises the operator's stream first. */
void ffm_bem_destroy(ffm_bem_t *bem);

/* Human-readable status name, and the message of the last failure in this thread. */
const char *ffm_status_str(ffm_status s);
const char *ffm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FFM_GB300_H */
