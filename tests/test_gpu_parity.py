"""GPU path (through the C ABI) against the FP64 CPU oracle.

Integer/index work (sorted permutations, box counts, pair lists, translation counts) must
match the oracle bit for bit; floating-point results must match the plain CPU FFM to
rel-L2 <= 1e-5 at the same eps and plan constants, and the FP64 direct sum to <= eps."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu

TOL_FFM = 1e-5   # vs the plain CPU FFM at the same eps (FP32 arithmetic on the GPU)


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1909_05600_gb300 import build
    build.build()
    ffm.lib()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def gpu_plan(prob, **opts):
    return ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, prob.k, prob.eps, weights=_t(prob.w), **opts)


def gpu_apply(plan, u):
    v = plan.apply(_t(u))
    torch.cuda.synchronize()
    return v.cpu().numpy()


def as_c128(u):
    return np.asarray(u).astype(np.complex128)


def _rows(a):
    a = np.asarray(a, dtype=np.uint64)
    if a.size == 0:
        return a.reshape(0, 2)
    return a[np.lexsort((a[:, 1], a[:, 0]))]


def compare_plans(gp, op):
    gi, oi = gp.info(), op.stats()
    assert gi["l_stop"] == oi["l_stop"]
    assert gi["root_admissible"] == oi["root_admissible"]
    assert gi["d0"] == oi["d0"]
    assert gi["oX"] == oi["oX"] and gi["oY"] == oi["oY"]
    ls = oi["l_stop"]
    for key in ("n_adm", "n_trans", "mode", "r1", "L", "nQ"):
        assert gi[key] == oi[key], key
    for l in range(ls + 1):
        assert gi["nboxX"][l] == oi["nboxX"][l] and gi["nboxY"][l] == oi["nboxY"][l], l
        assert gi["n_near"][l] == oi["n_near"][l], l
    assert np.array_equal(gp.perm("X"), op.perm("X"))
    assert np.array_equal(gp.perm("Y"), op.perm("Y"))
    for l in range(ls + 1):
        if oi["n_adm"][l]:
            assert np.array_equal(_rows(gp.pairs(l, "adm")), _rows(op.pairs(l, "adm"))), l
    assert np.array_equal(_rows(gp.pairs(0, "near")), _rows(op.pairs(0, "near")))


PLAN_CASES = {
    "laplace_sphere_20k": lambda: W.laplace_sphere(20000),
    "helmholtz_sphere_30k": lambda: W.helmholtz_sphere(30000),
    "laplace_cube_volume_xeqy": lambda: (lambda P: W.Problem("cv", P, P.copy(), np.ones(len(P)), np.ones(len(P)),
                                                            W.LAPLACE, 0.0, 1e-3))(W.cube_volume(30000, 4)),
    "laplace_clustered_60k": lambda: W.laplace_clustered(60000),
    "helmholtz_cube_multirhs_20k": lambda: W.helmholtz_cube_multirhs(20000, nrhs=2, eps=1e-4),
}


@pytest.mark.parametrize("case", sorted(PLAN_CASES))
def test_plan_matches_oracle_exactly(case):
    prob = PLAN_CASES[case]()
    op = O.Plan(prob.X, prob.Y, prob.kind, prob.k, prob.eps)
    with gpu_plan(prob) as gp:
        compare_plans(gp, op)


def test_laplace_sphere_20k_full_config():
    prob = W.laplace_sphere(20000)
    with gpu_plan(prob) as gp:
        v = gpu_apply(gp, prob.u)
    ref_ffm = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w)[:, 0]
    ref_dir = O.direct(prob.X, prob.Y, prob.u, O.LAPLACE, w=prob.w)[:, 0]
    assert O.rel_l2(v, ref_ffm) < TOL_FFM
    assert O.rel_l2(v, ref_dir) < prob.eps


@pytest.mark.parametrize("n", [20000, 60000])
def test_helmholtz_sphere_plane_waves(n):
    prob = W.helmholtz_sphere(n)
    with gpu_plan(prob) as gp:
        info = gp.info()
        v = gpu_apply(gp, prob.u)
    assert all(m in (0, 2) for m in info["mode"]) and 2 in info["mode"]
    u = as_c128(prob.u)
    ref_ffm = O.ffm(prob.X, prob.Y, u, O.HELMHOLTZ, prob.k, prob.eps, w=prob.w)[:, 0]
    t = W.sample_targets(n, 1500)
    ref_dir = O.direct(prob.X, prob.Y, u, O.HELMHOLTZ, prob.k, w=prob.w, targets=t)[:, 0]
    assert O.rel_l2(v, ref_ffm) < TOL_FFM
    assert O.rel_l2(v[t], ref_dir) < prob.eps


def test_helmholtz_low_frequency_lagrange():
    prob = W.helmholtz_sphere(15000)
    prob.k = 1.5
    with gpu_plan(prob) as gp:
        info = gp.info()
        v = gpu_apply(gp, prob.u)
    assert 1 in info["mode"] and 2 not in info["mode"]
    ref = O.ffm(prob.X, prob.Y, as_c128(prob.u), O.HELMHOLTZ, 1.5, prob.eps, w=prob.w)[:, 0]
    assert O.rel_l2(v, ref) < TOL_FFM


def test_mixed_levels_coincident_sets_eps_1e4():
    n = 20000
    X = W.cube_surface(n, 31)
    k = 12.0
    u = np.exp(1j * k * X @ np.array([0.0, 0.6, 0.8])).astype(np.complex64)
    prob = W.Problem("mixed", X, X.copy(), u, np.full(n, 6.0 / n), W.HELMHOLTZ, k, 1e-4)
    with gpu_plan(prob) as gp:
        info = gp.info()
        v = gpu_apply(gp, prob.u)
    assert 1 in info["mode"] and 2 in info["mode"]
    ref = O.ffm(X, X, as_c128(u), O.HELMHOLTZ, k, 1e-4, w=prob.w)[:, 0]
    assert O.rel_l2(v, ref) < TOL_FFM


@pytest.mark.parametrize("variant", [ffm.LAG_CUDA_CORES, ffm.LAG_TC_TRANSLATION, ffm.LAG_TC_TARGET])
def test_lagrange_transfer_variants_match_the_oracle(variant):
    """The three Lagrange transfer kernels (CUDA-core GEMM per translation, tcgen05 per
    translation with atomic scatter, tcgen05 target-stationary accumulating every
    translation of 128 target boxes) against the oracle FFM, on uneven clustered boxes."""
    prob, ref = _clustered_reference()
    with gpu_plan(prob, lagrange_transfer=variant) as gp:
        info = gp.info()
        v = gpu_apply(gp, prob.u)
    lag = [l for l in range(info["l_stop"] + 1) if info["mode"][l] == 1 and info["n_adm"][l] > 0]
    assert lag and all(info["tune_tc"][l] == variant - 1 for l in lag)
    assert O.rel_l2(v, ref) < TOL_FFM


@functools.lru_cache(maxsize=1)
def _clustered_reference():
    prob = W.laplace_clustered(40000, seed=4)
    return prob, O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w)[:, 0]


def test_precision_modes_error_tracks_cancellation():
    """Forced plane-wave arithmetic on an ill-conditioned level (cube surface, k d = 3,
    eps = 1e-4, cancellation ratio C ~ 3e4): FP64 and double-float match the oracle FFM to
    1e-6; FP32 and compensated FP32 move the result by at most ~2.3e-9 C and ~1.3e-9 C;
    the automatic choice (double-float here) stays within the 1e-5 parity bar."""
    n = 20000
    X = W.cube_surface(n, 31)
    k = 12.0
    u = np.exp(1j * k * X @ np.array([0.0, 0.6, 0.8])).astype(np.complex64)
    prob = W.Problem("mixed", X, X.copy(), u, np.full(n, 6.0 / n), W.HELMHOLTZ, k, 1e-4)
    ref = O.ffm(X, X, as_c128(u), O.HELMHOLTZ, k, 1e-4, w=prob.w)[:, 0]
    err = {}
    for mode in (ffm.PREC_AUTO, ffm.PREC_F32, ffm.PREC_F32C, ffm.PREC_F64, ffm.PREC_F32X2):
        with gpu_plan(prob, precision=mode) as gp:
            info = gp.info()
            v = gpu_apply(gp, prob.u)
        pw = [l for l in range(info["l_stop"] + 1) if info["mode"][l] == 2]
        assert pw, "the case must have plane-wave levels"
        if mode != ffm.PREC_AUTO:
            assert all(info["pw_prec"][l] == mode for l in pw)
        cmax = max(info["cancel"][l] for l in pw)
        err[mode] = O.rel_l2(v, ref)
    assert cmax > 4e3  # auto picks double-float for this level
    assert err[ffm.PREC_F64] < 1e-6
    assert err[ffm.PREC_F32X2] < 1e-6
    assert err[ffm.PREC_F32C] < 1.5e-9 * cmax
    assert err[ffm.PREC_F32] < 3e-9 * cmax
    assert err[ffm.PREC_AUTO] < TOL_FFM


@pytest.mark.parametrize("kind,k", [(W.LAPLACE, 0.0), (W.HELMHOLTZ, 10.0)])
def test_far_separated_roots(kind, k):
    rng = np.random.default_rng(8)
    X = rng.random((3000, 3))
    Y = rng.random((2500, 3)) + np.array([5.0, 0.5, -0.2])
    u = rng.standard_normal(2500)
    u = u.astype(np.complex64) if kind == W.HELMHOLTZ else u
    prob = W.Problem("far", X, Y, u, np.ones(2500), kind, k, 1e-3)
    with gpu_plan(prob) as gp:
        assert gp.info()["root_admissible"] == 1
        v = gpu_apply(gp, prob.u)
    ref = O.ffm(X, Y, as_c128(u) if kind == W.HELMHOLTZ else u, kind, k, 1e-3)[:, 0]
    assert O.rel_l2(v, ref) < TOL_FFM


def test_small_sets_are_the_direct_sum():
    rng = np.random.default_rng(3)
    X = rng.random((40, 3))
    Y = rng.random((50, 3))
    u = (rng.standard_normal(50) + 1j * rng.standard_normal(50)).astype(np.complex64)
    prob = W.Problem("small", X, Y, u, np.ones(50), W.HELMHOLTZ, 9.0, 1e-3)
    with gpu_plan(prob) as gp:
        assert gp.info()["l_stop"] == 0
        v = gpu_apply(gp, prob.u)
    ref = O.direct(X, Y, as_c128(u), O.HELMHOLTZ, 9.0)[:, 0]
    assert O.rel_l2(v, ref) < 1e-6


def test_single_points_and_coincidence():
    one = np.array([[0.3, 0.3, 0.3]])
    prob = W.Problem("one", one, one.copy(), np.ones(1), np.ones(1), W.LAPLACE, 0.0, 1e-3)
    with gpu_plan(prob) as gp:
        assert gp.info()["d0"] == 1.0
        v = gpu_apply(gp, prob.u)
    assert v[0] == 0.0


@pytest.mark.parametrize("nrhs", [3, 11])
def test_multirhs_columns_match_single_applies_and_are_deterministic(nrhs):
    prob = W.helmholtz_cube_multirhs(30000, nrhs=nrhs, eps=1e-4)
    U = np.ascontiguousarray(prob.u.T)  # (nrhs, n)
    with gpu_plan(prob) as gp:
        V = gpu_apply(gp, U)
        V2 = gpu_apply(gp, U)
        singles = [gpu_apply(gp, np.ascontiguousarray(U[m])) for m in range(3)]
    ref_ffm = O.ffm(prob.X, prob.Y, as_c128(prob.u[:, :3]), O.HELMHOLTZ, prob.k, prob.eps, w=prob.w)
    for m in range(3):
        assert O.rel_l2(V[m], ref_ffm[:, m]) < TOL_FFM
    assert O.rel_l2(V, V2) < 1e-9  # repeatable up to the order of FP64 atomic additions in the near field
    # batched kernels (phasors shared by the RHS) agree with single applies to rounding; the
    # two sum in different orders, and a compensated-FP32 level amplifies rounding by its
    # cancellation ratio (up to 4e3 here)
    for m in range(3):
        assert O.rel_l2(V[m], singles[m]) < 5e-6
    t = W.sample_targets(30000, 800)
    ref = O.direct(prob.X, prob.Y, as_c128(prob.u[:, 1]), O.HELMHOLTZ, prob.k, w=prob.w, targets=t)[:, 0]
    assert O.rel_l2(V[1][t], ref) < 1e-4


def test_host_buffers_match_device_buffers():
    prob = W.laplace_sphere(8000)
    with gpu_plan(prob) as gp:
        vd = gpu_apply(gp, prob.u)
    with ffm.Plan(prob.X, prob.Y, ffm.LAPLACE, 0.0, prob.eps, weights=prob.w) as hp:
        vh = hp.apply(prob.u)
    # same plan and kernels; Lagrange transfers scatter with FP32 atomics, so the order of
    # additions (not the arithmetic) may differ between the two runs
    assert O.rel_l2(vd, vh) < 1e-6


def test_float32_inputs():
    prob = W.laplace_sphere(10000)
    X32, Y32 = prob.X.astype(np.float32), prob.Y.astype(np.float32)
    u32, w32 = prob.u.astype(np.float32), prob.w.astype(np.float32)
    with ffm.Plan(_t(X32), _t(Y32), ffm.LAPLACE, 0.0, 1e-3, weights=_t(w32)) as gp:
        v = gp.apply(_t(u32)).cpu().numpy()
    ref = O.ffm(X32, Y32, u32.astype(np.float64), O.LAPLACE, 0.0, 1e-3, w=w32.astype(np.float64))[:, 0]
    assert O.rel_l2(v, ref) < TOL_FFM


def test_invalid_arguments_raise():
    X = _t(np.random.default_rng(0).random((100, 3)))
    for kw in ({"eps": 0.0}, {"eps": 1.5}):
        with pytest.raises(ffm.FFMError) as e:
            ffm.Plan(X, X, ffm.LAPLACE, 0.0, **kw)
        assert e.value.status == 1
    with pytest.raises(ffm.FFMError):
        ffm.Plan(X, X, ffm.HELMHOLTZ, -1.0, 1e-3)
    bad = np.random.default_rng(0).random((100, 3))
    bad[7, 1] = np.nan
    with pytest.raises(ffm.FFMError) as e:
        ffm.Plan(_t(bad), X, ffm.LAPLACE, 0.0, 1e-3)
    assert e.value.status == 1
    with ffm.Plan(X, X, ffm.HELMHOLTZ, 3.0, 1e-3) as p:
        with pytest.raises(ffm.FFMError):
            p.apply(_t(np.ones(100)))  # Helmholtz needs complex densities
    for prec in (-1, 5):
        with pytest.raises(ffm.FFMError) as e:
            ffm.Plan(X, X, ffm.HELMHOLTZ, 3.0, 1e-3, precision=prec)
        assert e.value.status == 1


def test_full_size_helmholtz_sphere_1M_sampled_targets():
    """The 1,000,000-point Helmholtz workload (k at 10 points per wavelength) in the launch
    configuration the benchmark times, checked on sampled targets against the FP64 direct
    sum."""
    prob = W.helmholtz_sphere(1_000_000)
    with gpu_plan(prob) as gp:
        info = gp.info()
        v = gpu_apply(gp, prob.u)
    assert info["l_stop"] == 6 and info["mode"][2:7] == [2] * 5
    t = W.sample_targets(prob.X.shape[0], 256)
    ref = O.direct(prob.X, prob.Y, as_c128(prob.u), O.HELMHOLTZ, prob.k, w=prob.w, targets=t)[:, 0]
    assert O.rel_l2(v[t], ref) < prob.eps


def test_clustered_laplace_10M_sampled_targets():
    """The clustered Laplace workload (8 Gaussians, sigma 0.05, float32 points and densities)
    at 10,000,000 + 10,000,000 points, in the default launch configuration: uneven leaves of
    up to tens of thousands of near sources per target, checked on 512 seeded targets
    against the FP64 direct sum."""
    prob = W.laplace_clustered(10_000_000)
    with gpu_plan(prob) as gp:
        info = gp.info()
        v = gpu_apply(gp, prob.u)
    assert info["device_errors"] == 0 and info["p2p_pairs"] > 1e11
    t = W.sample_targets(prob.X.shape[0], 512)
    ref = O.direct(prob.X, prob.Y, prob.u.astype(np.float64), O.LAPLACE, 0.0, w=prob.w, targets=t)[:, 0].real
    assert O.rel_l2(v[t], ref) < prob.eps


def test_laplace_volume_eps_1e4_transfer_gemm():
    """Volume points with X = Y at eps = 1e-4: r1 = 6 (216 control nodes), transfers by the
    per-translation GEMM with 189 admissible partners per interior box."""
    P = W.cube_volume(40000, 12)
    u = np.random.default_rng(13).standard_normal(40000)
    prob = W.Problem("vol", P, P.copy(), u, np.full(40000, 1.0 / 40000), W.LAPLACE, 0.0, 1e-4)
    with gpu_plan(prob, n_leaf=32) as gp:
        info = gp.info()
        v = gpu_apply(gp, prob.u)
    assert max(info["r1"]) == 6
    ref = O.ffm(P, P, u, O.LAPLACE, 0.0, 1e-4, w=prob.w, n_leaf=32)[:, 0]
    assert O.rel_l2(v, ref) < TOL_FFM
