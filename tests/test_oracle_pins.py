"""Pins of the FP64 CPU oracle against facts that do not come from the oracle itself:
closed-form potentials, library special functions, invariants of the convolution, exact
reproduction of a polynomial kernel, and the transfer counts printed in the paper.
All CPU-only."""
import math

import numpy as np
import pytest
from scipy.special import spherical_jn, spherical_yn, eval_legendre, gamma

from oracle import oracle as O
from paper_1909_05600_gb300 import workloads as W


def _unit_dirs(n, seed):
    return W.sphere_surface(n, seed)


# ----------------------------------------------------------- O1 closed forms

def test_direct_laplace_charged_sphere():
    """int_{S^2} dS_y / (4 pi |x - y|) = 1 inside the unit sphere and 1/|x| outside
    (potential of a uniformly charged sphere); Y is the oracle's own sphere quadrature."""
    s, w = O.sphere_quad(40)
    radii = np.array([0.0, 0.3, 0.55, 0.8, 1.25, 2.0, 5.0])
    dirs = _unit_dirs(len(radii), 3)
    X = dirs * radii[:, None]
    v = O.direct(X, s, np.ones(len(w)), O.LAPLACE, w=w)[:, 0]
    exact = np.where(radii < 1, 1.0, 1.0 / np.maximum(radii, 1e-300))
    assert np.max(np.abs(v.real - exact)) < 1e-8
    assert np.max(np.abs(v.imag)) == 0.0


@pytest.mark.parametrize("k", [0.7, 5.0, 12.0])
def test_direct_helmholtz_sphere_single_layer(k):
    """int_{S^2} e^{ik|x-y|}/(4 pi |x-y|) dS_y = e^{ik} sin(k|x|)/(k|x|) for |x| < 1 and
    sin(k) e^{ik|x|}/(k|x|) for |x| > 1 (addition theorem: only n = 0 survives)."""
    s, w = O.sphere_quad(48)
    radii = np.array([0.2, 0.5, 0.8, 1.25, 1.7, 3.0])
    X = _unit_dirs(len(radii), 4) * radii[:, None]
    v = O.direct(X, s, np.ones(len(w)), O.HELMHOLTZ, k, w=w)[:, 0]
    inside = np.exp(1j * k) * np.sin(k * radii) / (k * radii)
    outside = np.sin(k) * np.exp(1j * k * radii) / (k * radii)
    exact = np.where(radii < 1, inside, outside)
    assert np.max(np.abs(v - exact)) < 1e-8


def test_direct_helmholtz_plane_wave_density():
    """Funk-Hecke: for u(y) = e^{ik d.y} on the unit sphere and |x| < 1,
    v(x) = sum_n i^n (2n+1) ik j_n(k) h_n(k) j_n(k|x|) P_n(x.d/|x|)."""
    k = 4.0
    s, w = O.sphere_quad(48)
    d = np.array([0.36, -0.48, 0.8])
    u = np.exp(1j * k * (s @ d))
    radii = np.array([0.25, 0.6, 0.8])
    X = _unit_dirs(3, 9) * radii[:, None]
    v = O.direct(X, s, u, O.HELMHOLTZ, k, w=w)[:, 0]
    n = np.arange(60)
    jk = spherical_jn(n, k)
    hk = jk + 1j * spherical_yn(n, k)
    for i in range(3):
        r = radii[i]
        c = X[i] @ d / r
        ex = np.sum((1j ** n) * (2 * n + 1) * 1j * k * jk * hk * spherical_jn(n, k * r) * eval_legendre(n, c))
        assert abs(v[i] - ex) < 1e-8 * max(1.0, abs(ex))


def test_direct_reciprocity_and_linearity():
    """G(x, y) = G(y, x) with no conjugation: a^T (G_XY b) = b^T (G_YX a); the sum is
    linear in u."""
    rng = np.random.default_rng(0)
    X = rng.random((150, 3))
    Y = rng.random((170, 3)) + 0.3
    a = rng.standard_normal(150) + 1j * rng.standard_normal(150)
    b = rng.standard_normal(170) + 1j * rng.standard_normal(170)
    k = 7.5
    lhs = a @ O.direct(X, Y, b, O.HELMHOLTZ, k)[:, 0]
    rhs = b @ O.direct(Y, X, a, O.HELMHOLTZ, k)[:, 0]
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    c = rng.standard_normal(170)
    v1 = O.direct(X, Y, 2.0 * b - 3.0 * c, O.HELMHOLTZ, k)
    v2 = 2.0 * O.direct(X, Y, b, O.HELMHOLTZ, k) - 3.0 * O.direct(X, Y, c, O.HELMHOLTZ, k)
    assert O.rel_l2(v1, v2) < 1e-13


def test_direct_coincident_points_contribute_zero():
    X = np.array([[0.1, 0.2, 0.3]])
    v = O.direct(X, X, np.ones(1), O.LAPLACE)
    assert v[0, 0] == 0.0
    v = O.direct(X, X, np.ones(1), O.HELMHOLTZ, 3.0)
    assert v[0, 0] == 0.0


# ------------------------------------------------- O2 components, textbook pins

@pytest.mark.parametrize("n", [1, 2, 5, 17, 64, 161])
def test_gauss_legendre_matches_numpy(n):
    x, w = O.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    assert np.max(np.abs(x - xr)) < 1e-13
    assert np.max(np.abs(w - wr)) < 1e-13


@pytest.mark.parametrize("L", [1, 4, 11, 30])
def test_sphere_quadrature_integrates_monomials(L):
    """Quadrature of eq. 17: weights sum to 4 pi and monomials x^a y^b z^c of total
    degree < 2L integrate exactly: int = 2 G((a+1)/2) G((b+1)/2) G((c+1)/2) / G((a+b+c+3)/2)
    for even a, b, c, zero otherwise."""
    s, w = O.sphere_quad(L)
    assert len(w) == 2 * L * (L + 1)
    assert abs(w.sum() - 4 * math.pi) < 1e-12
    for (a, b, c) in [(2, 0, 0), (0, 2, 2), (1, 1, 0), (4, 2, 0), (0, 0, 6), (2, 2, 2), (3, 0, 1)]:
        if a + b + c >= 2 * L:
            continue
        num = np.sum(w * s[:, 0] ** a * s[:, 1] ** b * s[:, 2] ** c)
        if a % 2 or b % 2 or c % 2:
            ex = 0.0
        else:
            ex = 2 * gamma((a + 1) / 2) * gamma((b + 1) / 2) * gamma((c + 1) / 2) / gamma((a + b + c + 3) / 2)
        assert abs(num - ex) < 1e-12


@pytest.mark.parametrize("z", [0.5, 3.0, 17.0, 250.0])
def test_hankel_matches_scipy(z):
    L = 60
    h = O.hankel(L, z)
    p = np.arange(L + 1)
    ref = spherical_jn(p, z) + 1j * spherical_yn(p, z)
    rel = np.abs(h - ref) / np.abs(ref)
    assert np.max(rel) < 1e-10


@pytest.mark.parametrize("kd,offset,eps", [
    (2.0, (2, 0, 0), 1e-3), (5.0, (2, 1, 0), 1e-3), (20.0, (2, 2, 2), 1e-3),
    (60.0, (3, -2, 1), 1e-3), (8.0, (-2, 0, 1), 1e-4), (30.0, (0, 2, -3), 1e-4)])
def test_plane_wave_single_pair(kd, offset, eps):
    """Eqs. 10-16 with the readings p from 0, box-centred phases (no r0 phase), natural-log
    rank and the (L+1) x 2L quadrature reproduce e^{ik|x-y|}/(4 pi |x-y|) to eps for a
    box pair at the admissibility distance."""
    d = 1.0
    k = kd / d
    L = O.pw_rank(k, d, eps)
    rng = np.random.default_rng(int(kd * 10))
    y0 = np.zeros(3)
    x0 = np.array(offset, dtype=float) * d
    worst = 0.0
    for _ in range(6):
        x = x0 + (rng.random(3) - 0.5) * d
        y = y0 + (rng.random(3) - 0.5) * d
        r = np.linalg.norm(x - y)
        exact = np.exp(1j * k * r) / (4 * math.pi * r)
        worst = max(worst, abs(O.pw_pair(k, L, x, y, x0, y0) - exact) / abs(exact))
    assert worst < eps


def test_plane_wave_series_from_p1_misses_eps():
    """Eq. 12 as printed sums from p = 1. Dropping the p = 0 term removes
    ik h_0(k r0) j_0(k |r_xy|) / (4 pi) from the single-pair approximation (the quadrature
    integrates e^{ik s.r_xy} to 4 pi j_0 exactly), and the result misses eps by far."""
    k, d, eps = 10.0, 1.0, 1e-3
    L = O.pw_rank(k, d, eps)
    x0 = np.array([2.0, 0.0, 0.0])
    y0 = np.zeros(3)
    x = x0 + np.array([0.2, -0.1, 0.3])
    y = y0 + np.array([-0.25, 0.1, 0.05])
    r = np.linalg.norm(x - y)
    exact = np.exp(1j * k * r) / (4 * math.pi * r)
    good = O.pw_pair(k, L, x, y, x0, y0)
    assert abs(good - exact) < eps * abs(exact)
    rxy = np.linalg.norm((x - x0) - (y - y0))
    h0 = O.hankel(0, k * np.linalg.norm(x0 - y0))[0]
    monopole = 1j * k * h0 * spherical_jn(0, k * rxy) / (4 * math.pi)
    assert abs(good - monopole - exact) > 10 * eps * abs(exact)


def test_r1_table_matches_calibration():
    from oracle.calibrate_r1 import calibrate, round_up
    cal = calibrate()
    for name, kind in (("laplace", O.LAPLACE), ("helmholtz_kd2", O.HELMHOLTZ),
                       ("laplace_double_layer", O.LAPLACE_DL)):
        tab = O.r1_table(kind)
        for r1, e in zip(range(2, 11), cal[name]):
            assert tab[r1] == pytest.approx(round_up(e), rel=1e-12)
    assert O.r1_rule(O.LAPLACE, 1e-3) == 4
    assert O.r1_rule(O.LAPLACE, 1e-4) == 6
    assert O.r1_rule(O.LAPLACE_DL, 1e-3) == 6
    assert O.r1_rule(O.LAPLACE_DL, 1e-4) == 7


# ---- double layer: dG/dn_y with the Laplace G through the Lagrange path, as the three
# component kernels dG/dy_d interpolated on their own and weighted by w u n_d

def _sphere_grid(L):
    n = 2 * L * (L + 1)
    s = np.zeros((n, 3))
    w = np.zeros(n)
    O.lib().orc_sphere_quad(L, s.ctypes.data_as(O._dp), w.ctypes.data_as(O._dp))
    return s, w


def test_double_layer_gauss_law():
    """Gauss: the double-layer potential of the unit density on the unit sphere (outward
    normals) is -1 inside and 0 outside, to quadrature accuracy away from the sphere."""
    s, w = _sphere_grid(40)
    inside = np.array([[0.1, 0.2, -0.3], [0.0, 0.0, 0.0], [-0.4, 0.3, 0.35]])
    outside = np.array([[1.5, 0.3, 0.2], [0.0, -2.0, 0.5], [3.0, 3.0, -3.0]])
    v_in = O.direct_dl(inside, s, s, np.ones(len(w)), w=w)[:, 0]
    v_out = O.direct_dl(outside, s, s, np.ones(len(w)), w=w)[:, 0]
    assert np.max(np.abs(v_in + 1.0)) < 1e-9
    assert np.max(np.abs(v_out)) < 1e-9


def test_double_layer_is_the_normal_derivative_of_the_laplace_kernel():
    """Central differences of the Laplace direct sum in the source position along n."""
    rng = np.random.default_rng(21)
    for _ in range(5):
        x = rng.standard_normal((1, 3))
        y = rng.standard_normal((1, 3))
        n = rng.standard_normal((1, 3))
        h = 1e-5
        g = lambda yy: O.direct(x, yy, np.ones(1), O.LAPLACE)[0, 0].real
        fd = (g(y + h * n) - g(y - h * n)) / (2 * h)
        assert O.direct_dl(x, y, n, np.ones(1))[0, 0] == pytest.approx(fd, rel=1e-7)


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_double_layer_ffm_within_eps(eps):
    """O2 for the double layer against O1 on a sphere with outward normals."""
    n = 12000
    X = W.sphere_surface(n, 1)
    Y = W.sphere_surface(n, 1001)
    u = np.random.default_rng(3).standard_normal(n)
    w = np.full(n, 4 * np.pi / n)
    v = O.ffm_dl(X, Y, Y, u, eps, w=w)[:, 0]
    ref = O.direct_dl(X, Y, Y, u, w=w)[:, 0]
    assert O.rel_l2(v, ref) < eps


def test_morton_interleave():
    assert O.morton(1, 0, 0) == 4
    assert O.morton(0, 1, 0) == 2
    assert O.morton(0, 0, 1) == 1
    # bit b of gx -> 3b+2, of gy -> 3b+1, of gz -> 3b
    gx, gy, gz = 0b1011, 0b0110, 0b1101
    ref = 0
    for b in range(4):
        ref |= ((gx >> b) & 1) << (3 * b + 2) | ((gy >> b) & 1) << (3 * b + 1) | ((gz >> b) & 1) << (3 * b)
    assert O.morton(gx, gy, gz) == ref


# --------------------------------------------------- O2 descent / transfer counts

def test_admissibility_is_non_strict_max_norm():
    z = np.zeros(3)
    assert O.admissible(z, 3, [2, 0, 0])
    assert O.admissible(z, 3, [-2, 1, 1])
    assert not O.admissible(z, 3, [1, 1, 1])
    assert O.admissible(z, 3, [2, 2, 2])
    # shifted trees: the offset is sigma*2^l + m
    sig = np.array([0.25 / 8, 0.0, 0.0])
    assert not O.admissible(sig, 3, [1, 0, 0])   # 1.25
    assert O.admissible(sig, 3, [-3, 0, 0])      # -2.75
    assert not O.admissible(sig, 3, [-2, 0, 0])  # -1.75


def _pairs_per_target(pairs):
    _, c = np.unique(pairs[:, 0], return_counts=True)
    return c


def test_quadtree_transfer_counts_match_paper():
    """Planar points with X = Y (aligned quadtrees, Sec. 3.1 proof of Prop. 1): an interior
    box has 27 admissible partners and a level holds at most 7^2 - 3^2 = 40 distinct
    transfers."""
    rng = np.random.default_rng(11)
    P = np.zeros((20000, 3))
    P[:, :2] = rng.random((20000, 2))
    plan = O.Plan(P, P, O.LAPLACE, 0.0, 1e-3)
    st = plan.stats()
    assert st["l_stop"] >= 4
    for l in range(2, st["l_stop"] + 1):
        assert st["n_trans"][l] == 40
        if l >= 3:
            assert _pairs_per_target(plan.pairs(l, "adm")).max() == 27


def test_octree_transfer_counts():
    """Volume points with X = Y: at most 7^3 - 3^3 = 316 distinct transfers per level and
    6^3 - 3^3 = 189 admissible partners for an interior box."""
    P = W.cube_volume(60000, 5)
    plan = O.Plan(P, P, O.LAPLACE, 0.0, 1e-3, n_leaf=16)
    st = plan.stats()
    for l in range(3, st["l_stop"] + 1):
        assert st["n_trans"][l] == 316
        assert _pairs_per_target(plan.pairs(l, "adm")).max() == 189


def test_stop_rule_mean_occupancy():
    prob = W.laplace_sphere(20000)
    plan = O.Plan(prob.X, prob.Y, O.LAPLACE, 0.0, 1e-3)
    st = plan.stats()
    ls = st["l_stop"]
    tot = prob.X.shape[0] + prob.Y.shape[0]
    assert tot < 64 * (st["nboxX"][ls] + st["nboxY"][ls])
    assert tot >= 64 * (st["nboxX"][ls - 1] + st["nboxY"][ls - 1])


# ------------------------------------------------------------ O2 versus O1

def test_ffm_small_n_is_the_direct_sum():
    """With no more points than one leaf holds the descent stops at the roots and the FFM
    is the dense product."""
    rng = np.random.default_rng(3)
    X = rng.random((40, 3))
    Y = rng.random((50, 3))
    u = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    plan = O.Plan(X, Y, O.HELMHOLTZ, 9.0, 1e-3)
    assert plan.stats()["l_stop"] == 0
    v = plan.apply(u)
    ref = O.direct(X, Y, u, O.HELMHOLTZ, 9.0)
    assert O.rel_l2(v, ref) < 1e-14


def test_ffm_lagrange_reproduces_polynomial_kernel():
    """Tensor Lagrange interpolation with r1 = 4 is exact for a kernel of degree <= 3 per
    coordinate: anterpolation, transfer and interpolation then make no error at all."""
    P = W.cube_volume(6000, 21)
    Q = W.cube_volume(5000, 22) * 0.9 + 0.07
    u = np.random.default_rng(23).standard_normal(5000)
    plan = O.Plan(P, Q, O.POLY, 0.0, 1e-3, r1_override=4, n_leaf=16)
    st = plan.stats()
    assert sum(st["n_adm"]) > 1000
    v = plan.apply(u)
    ref = O.direct(P, Q, u, O.POLY)
    assert O.rel_l2(v, ref) < 1e-11


def test_ffm_laplace_sphere_meets_eps():
    prob = W.laplace_sphere(20000)
    v = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w)
    ref = O.direct(prob.X, prob.Y, prob.u, O.LAPLACE, w=prob.w)
    err = O.rel_l2(v, ref)
    # within eps, and in the band of Table 1 (8e-5 .. 3.5e-4 at eps = 1e-3) to a factor 10
    assert 1e-6 < err < prob.eps


@pytest.mark.parametrize("n", [8000, 30000])
def test_ffm_helmholtz_sphere_meets_eps(n):
    prob = W.helmholtz_sphere(n)
    plan = O.Plan(prob.X, prob.Y, O.HELMHOLTZ, prob.k, prob.eps)
    st = plan.stats()
    assert any(m == O.MODE_PLANEWAVE for m in st["mode"])
    v = plan.apply(prob.u.astype(np.complex128), prob.w)
    t = W.sample_targets(n, 1500)
    ref = O.direct(prob.X, prob.Y, prob.u.astype(np.complex128), O.HELMHOLTZ, prob.k, w=prob.w, targets=t)
    assert O.rel_l2(v[t], ref) < prob.eps


def test_ffm_helmholtz_low_frequency_lagrange_levels():
    """Helmholtz with k d_l below the switch at every level: Lagrange interpolation of the
    oscillatory kernel (complex transfer)."""
    prob = W.helmholtz_sphere(12000, ppw=60.0)
    plan = O.Plan(prob.X, prob.Y, O.HELMHOLTZ, 1.5, 1e-3)
    st = plan.stats()
    assert all(m != O.MODE_PLANEWAVE for m in st["mode"]) and any(m == O.MODE_LAGRANGE for m in st["mode"])
    u = prob.u.astype(np.complex128)
    v = plan.apply(u, prob.w)
    t = W.sample_targets(12000, 1500)
    ref = O.direct(prob.X, prob.Y, u, O.HELMHOLTZ, 1.5, w=prob.w, targets=t)
    assert O.rel_l2(v[t], ref) < 1e-3


def test_ffm_mixed_levels_and_coincident_sets():
    """X = Y on the cube surface (pairs at distance 0 skipped) with plane-wave levels above
    Lagrange levels, eps = 1e-4."""
    n = 15000
    X = W.cube_surface(n, 31)
    k = 12.0
    u = np.exp(1j * k * X @ np.array([0.0, 0.6, 0.8]))
    plan = O.Plan(X, X, O.HELMHOLTZ, k, 1e-4)
    st = plan.stats()
    modes = [m for m in st["mode"] if m]
    assert O.MODE_PLANEWAVE in modes and O.MODE_LAGRANGE in modes
    v = plan.apply(u, np.full(n, 6.0 / n))
    t = W.sample_targets(n, 1500)
    ref = O.direct(X, X, u, O.HELMHOLTZ, k, w=np.full(n, 6.0 / n), targets=t)
    assert O.rel_l2(v[t], ref) < 1e-4


@pytest.mark.parametrize("kind,k", [(O.LAPLACE, 0.0), (O.HELMHOLTZ, 10.0)])
def test_ffm_far_separated_roots(kind, k):
    """Roots already admissible (centres 5 d0 apart): one far-field interaction at level 0."""
    rng = np.random.default_rng(8)
    X = rng.random((3000, 3))
    Y = rng.random((2500, 3)) + np.array([5.0, 0.5, -0.2])
    u = rng.standard_normal(2500)
    plan = O.Plan(X, Y, kind, k, 1e-3)
    st = plan.stats()
    assert st["root_admissible"] == 1 and st["n_adm"][0] == 1 and st["l_stop"] == 0
    v = plan.apply(u)
    ref = O.direct(X, Y, u, kind, k)
    assert O.rel_l2(v, ref) < 1e-3


def test_ffm_linearity_multirhs_and_reciprocity():
    prob = W.helmholtz_sphere(6000, eps=1e-4)
    u = prob.u.astype(np.complex128)
    rng = np.random.default_rng(44)
    u2 = rng.standard_normal(6000) + 0j
    U = np.stack([u, u2, 2 * u - 3j * u2], 1)
    plan = O.Plan(prob.X, prob.Y, O.HELMHOLTZ, prob.k, 1e-4)
    V = plan.apply(U)
    assert O.rel_l2(V[:, 2], 2 * V[:, 0] - 3j * V[:, 1]) < 1e-12
    assert O.rel_l2(V[:, :1], plan.apply(u)) < 1e-14
    # reciprocity a^T G_XY b = b^T G_YX a holds to eps through the FFM
    plan_t = O.Plan(prob.Y, prob.X, O.HELMHOLTZ, prob.k, 1e-4)
    a = rng.standard_normal(6000)
    lhs = a @ V[:, 1]
    rhs = u2 @ plan_t.apply(a)[:, 0]
    assert abs(lhs - rhs) < 1e-4 * abs(lhs)


def test_ffm_translation_and_scaling_invariance():
    prob = W.laplace_sphere(8000)
    v = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, 1e-3)
    s = np.array([0.5, -0.25, 0.125])
    vt = O.ffm(prob.X + s, prob.Y + s, prob.u, O.LAPLACE, 0.0, 1e-3)
    assert O.rel_l2(vt, v) < 1e-10
    vs = O.ffm(2.0 * prob.X, 2.0 * prob.Y, prob.u, O.LAPLACE, 0.0, 1e-3)
    assert O.rel_l2(2.0 * vs, v) < 1e-13
    hp = W.helmholtz_sphere(8000)
    u = hp.u.astype(np.complex128)
    vh = O.ffm(hp.X, hp.Y, u, O.HELMHOLTZ, hp.k, 1e-3)
    vhs = O.ffm(2.0 * hp.X, 2.0 * hp.Y, u, O.HELMHOLTZ, hp.k / 2.0, 1e-3)
    assert O.rel_l2(2.0 * vhs, vh) < 1e-13


def test_ffm_degenerate_inputs():
    one = np.array([[0.3, 0.3, 0.3]])
    plan = O.Plan(one, one, O.LAPLACE, 0.0, 1e-3)
    assert plan.stats()["d0"] == 1.0
    assert plan.apply(np.ones(1))[0, 0] == 0.0
    with pytest.raises(ValueError):
        O.Plan(one, one, O.LAPLACE, 0.0, 0.0)
    with pytest.raises(ValueError):
        O.Plan(one, one, O.HELMHOLTZ, -1.0, 1e-3)


# ------------------------------------------- type-3 NUFFT of the plane-wave steps (Sec. 2.2.3)

def _box_problem(seed, n=1500, nq=600, d=0.5, k=60.0):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-d / 2, d / 2, (n, 3))
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    s = k * _unit_dirs(nq, seed + 7)
    return d, k, x, c, s


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_nufft_forward_and_adjoint_match_the_exponential_sums(eps):
    """Against the plain sums F_q = sum_j c_j e^{-i s_q.x_j} and v_j = sum_q z_q e^{+i s_q.x_j}
    (brute force), within eps / 100: the kernel width makes the NUFFT error that small."""
    d, k, x, c, s = _box_problem(5)
    nu = O.Nufft(d, k, eps, s)
    F = nu.forward(x, c)
    ex = np.exp(-1j * (s @ x.T)) @ c
    assert O.rel_l2(F, ex) < eps / 100
    z = np.random.default_rng(6).standard_normal(len(s)) * (1 + 0.5j)
    v = nu.adjoint(x, z)
    exv = np.exp(1j * (x @ s.T)) @ z
    assert O.rel_l2(v, exv) < eps / 100


def test_nufft_single_point_is_a_plane_wave_and_the_adjoint_is_the_transpose():
    d, k, x, c, s = _box_problem(8, n=1, nq=300)
    x[0] = [0.249, -0.25, 0.1]  # on the box faces
    nu = O.Nufft(d, k, 1e-4, s)
    F = nu.forward(x, np.ones(1))
    assert np.max(np.abs(F - np.exp(-1j * (s @ x[0])))) < 1e-5  # eps / 10 in the max norm
    d, k, x, c, s = _box_problem(9, n=700, nq=400)
    nu = O.Nufft(d, k, 1e-3, s)
    z = np.random.default_rng(10).standard_normal(len(s)) + 1j
    lhs = np.vdot(z, nu.forward(x, c))
    rhs = np.vdot(nu.adjoint(x, z), c)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("n", [7, 12, 30, 35])
def test_oracle_dft_matches_numpy_fft(n):
    """The oracle's mixed-radix DFT (prime lengths summed directly) against numpy.fft."""
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    assert np.max(np.abs(O.dft3(a, -1) - np.fft.fftn(a))) < 1e-10 * n ** 3
    assert np.max(np.abs(O.dft3(a, +1) - np.fft.ifftn(a) * n ** 3)) < 1e-10 * n ** 3


def test_es_kernel_transform_matches_adaptive_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    for w in (6, 8, 10):
        beta = 2.30 * w
        assert O.es_kernel(0.0, beta) == 1.0 and O.es_kernel(1.5, beta) == 0.0
        assert abs(O.es_kernel(1.0, beta) - math.exp(-beta)) < 1e-15
        for xi in (0.0, 1.3, 0.84 * w):
            ref = integrate.quad(lambda z: O.es_kernel(z, beta) * math.cos(xi * z), -1, 1, epsabs=1e-14,
                                 limit=200)[0]
            assert abs(O.es_hat(xi, beta) - ref) < 1e-9 * abs(ref)


def test_nufft_parameter_rule():
    """Width from eps, the spreading grid fine enough that 2 pi / h - k clears the kernel's
    band (k h <= 2 pi - 2 beta / w), the FFT grid twice the spreading grid and 7-smooth."""
    for d, k, eps in [(0.5, 177.2, 1e-3), (0.25, 177.2, 1e-4), (1.0, 3.0, 1e-2), (0.1, 900.0, 1e-6)]:
        w, beta, M, n1, n2 = O.nufft_params(d, k, eps)
        assert w == min(12, max(6, math.ceil(-math.log10(eps)) + 4))
        assert k * d / M <= 2 * math.pi - 2 * beta / w < k * d / (M - 1) if M > 1 else True
        assert n1 >= M + w + 2 and n1 % 2 == 0
        assert n2 >= 2 * n1
        m = n2
        for p in (2, 3, 5, 7):
            while m % p == 0:
                m //= p
        assert m == 1


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_ffm_with_nufft_within_eps(eps):
    """O2 with the NUFFT plane-wave steps against O1 (eps) and against O2 with direct
    sums (within eps / 10: the transform error, ~eps / 200, is amplified by the
    cancellation of the quadrature sums at the small-kd levels) on the Helmholtz sphere."""
    prob = W.helmholtz_sphere(8000, seed=2, eps=eps)
    vn = O.ffm_nufft(prob.X, prob.Y, prob.u, prob.kind, prob.k, eps, w=prob.w)[:, 0]
    vd = O.ffm(prob.X, prob.Y, prob.u, prob.kind, prob.k, eps, w=prob.w)[:, 0]
    ref = O.direct(prob.X, prob.Y, prob.u, prob.kind, prob.k, w=prob.w)[:, 0]
    assert O.rel_l2(vn, ref) < eps
    assert O.rel_l2(vn, vd) < eps / 10
    assert O.Plan(prob.X, prob.Y, prob.kind, prob.k, eps).stats()["mode"][2] == O.MODE_PLANEWAVE


# ------------------------------------------------- gradient of the single layer (Sec. 4.2)

def test_gradient_of_the_charged_sphere_potential():
    """The potential of the uniformly charged unit sphere is 1 inside and 1/|x| outside, so
    its gradient is 0 inside and -x/|x|^3 outside (to quadrature accuracy)."""
    s, w = _sphere_grid(40)
    inside = np.array([[0.1, 0.2, -0.3], [0.0, 0.0, 0.0], [-0.4, 0.3, 0.35]])
    outside = np.array([[1.5, 0.3, 0.2], [0.0, -2.0, 0.5], [3.0, 3.0, -3.0]])
    g_in = O.direct_grad(inside, s, np.ones(len(w)), w=w)[:, 0, :]
    g_out = O.direct_grad(outside, s, np.ones(len(w)), w=w)[:, 0, :]
    assert np.max(np.abs(g_in)) < 1e-9
    exact = -outside / np.linalg.norm(outside, axis=1)[:, None] ** 3
    assert np.max(np.abs(g_out - exact)) < 1e-9


def test_gradient_is_the_derivative_of_the_laplace_potential():
    """Central differences of the Laplace direct sum in the target position."""
    rng = np.random.default_rng(31)
    Y = rng.standard_normal((50, 3))
    u = rng.standard_normal(50)
    x = np.array([[0.3, -2.5, 1.7]])
    h = 1e-5
    g = O.direct_grad(x, Y, u)[0, 0, :]
    for d in range(3):
        e = np.zeros((1, 3))
        e[0, d] = h
        fd = (O.direct(x + e, Y, u, O.LAPLACE)[0, 0].real - O.direct(x - e, Y, u, O.LAPLACE)[0, 0].real) / (2 * h)
        assert abs(fd - g[d]) < 1e-7 * max(1.0, abs(g[d]))


@pytest.mark.parametrize("eps,rad", [(1e-3, 0.6), (1e-4, 1.25)])
def test_gradient_ffm_within_eps(eps, rad):
    """O2 for the gradient against O1, targets on a sphere of radius rad inside / outside
    the source sphere (the far field carries most of the result there)."""
    n = 15000
    Y = W.sphere_surface(n, 1001)
    X = W.sphere_surface(n, 1) * rad
    u = np.random.default_rng(3).standard_normal(n)
    w = np.full(n, 4 * np.pi / n)
    v = O.ffm_grad(X, Y, u, eps, w=w)[:, 0, :]
    ref = O.direct_grad(X, Y, u, w=w)[:, 0, :]
    assert O.rel_l2(v, ref) < eps
    assert O.r1_rule(O.LAPLACE_GRAD, eps) == O.r1_rule(O.LAPLACE_DL, eps)


# ------------------------------------------ boundary-element wrapper (Sec. 4.2, S = L*^T G L)

def _polar_integrals(P, x, n=400):
    """V0 = int_T dA / |y - x| and Vv = int_T (y - x) / |y - x| dA by quadrature over the polar
    angle about x: along direction theta the triangle ends at rho(theta), so V0 = int rho dtheta
    and Vv = int rho dir(theta) dtheta."""
    nrm = np.cross(P[1] - P[0], P[2] - P[0])
    nrm /= np.linalg.norm(nrm)
    e1 = (P[0] - x) / np.linalg.norm(P[0] - x)
    e2 = np.cross(nrm, e1)
    ang = [np.arctan2(np.dot(p - x, e2), np.dot(p - x, e1)) for p in P]
    V0, Vv = 0.0, np.zeros(3)
    t, w = np.polynomial.legendre.leggauss(n)
    for i in range(3):
        a, b = P[i], P[(i + 1) % 3]
        th0, th1 = ang[i], ang[(i + 1) % 3]
        dth = (th1 - th0 + np.pi) % (2 * np.pi) - np.pi
        for tk, wk in zip(t, w):
            th = th0 + 0.5 * (tk + 1) * dth
            d = np.cos(th) * e1 + np.sin(th) * e2
            # the ray x + r d meets the edge line a + s (b - a)
            M = np.stack([d, a - b], 1)
            r = np.linalg.lstsq(M, a - x, rcond=None)[0][0]
            V0 += 0.5 * wk * abs(dth) * r
            Vv += 0.5 * wk * abs(dth) * r * d
    return V0, Vv


def test_bem_plane_integrals_match_polar_quadrature():
    """Closed-form in-plane potential of a constant and of a linear density on a flat
    triangle against quadrature over the polar angle (a separate route)."""
    from oracle import bem as B
    rng = np.random.default_rng(41)
    for _ in range(4):
        P = rng.standard_normal((3, 3))
        lam = rng.dirichlet([2, 2, 2])
        x = lam @ P
        V0, Vv = B.plane_integrals(P, x)
        R0, Rv = _polar_integrals(P, x)
        assert abs(V0 - R0) < 1e-9 * abs(R0)
        assert np.max(np.abs(Vv - Rv)) < 1e-9 * np.linalg.norm(Rv)


def test_bem_self_element_is_symmetric_and_converged():
    from oracle import bem as B
    P = np.random.default_rng(43).standard_normal((2, 3, 3))
    A = B.self_element(P, 32)
    A2 = B.self_element(P, 48)
    assert np.max(np.abs(A - np.swapaxes(A, 1, 2))) < 1e-7 * np.max(np.abs(A))
    assert np.max(np.abs(A - A2)) < 2e-6 * np.max(np.abs(A))


def test_bem_quadrature_integrates_piecewise_linear_functions():
    from oracle import bem as B
    V, F = W.icosphere(2)
    X, w, L = B.quadrature(V, F)
    u = np.random.default_rng(2).standard_normal(len(V))
    P = V[F]
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    exact = np.sum(area * u[F].mean(axis=1))  # integral of a linear function = area x vertex mean
    assert abs(np.dot(w, L @ u) - exact) < 1e-12 * np.sum(area * np.abs(u[F]).mean(axis=1))
    assert np.allclose(L.sum(axis=1), 1.0)


def test_bem_single_layer_of_the_sphere_has_unit_density():
    """The unit sphere's single layer maps the constant 1 to 1 (charged-sphere potential), so
    S sigma = (L*)^T 1 has sigma = 1 up to the discretisation error, which shrinks with h."""
    from oracle import bem as B
    errs = []
    for lev in (2, 3):
        V, F = W.icosphere(lev)
        X, w, L = B.quadrature(V, F)
        sig = np.linalg.solve(B.dense_matrix(V, F), L.T @ w)
        errs.append((abs(sig.mean() - 1), np.max(np.abs(sig - 1))))
    assert errs[1][0] < errs[0][0] and errs[1][0] < 5e-3 and errs[1][1] < 4e-2


def test_bem_ffm_product_matches_the_dense_matrix():
    from oracle import bem as B
    V, F = W.icosphere(2)
    u = np.random.default_rng(4).standard_normal(len(V))
    S = B.dense_matrix(V, F)
    assert O.rel_l2(B.apply_ffm(V, F, u, 1e-4), S @ u) < 1e-4


# ------------------------------------------------- ACA of the transfer (eq. 11)

def _cheb_grid(r1):
    t = np.cos((2 * np.arange(r1) + 1) * np.pi / (2 * r1)) * 0.5
    return np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)


def _laplace_T(r1, offset):
    """The Laplace transfer between the control nodes of two unit boxes whose centres are
    `offset` apart (Sec. 2.2.2), written out from the kernel."""
    g = _cheb_grid(r1)
    d = (g[:, None, :] + np.asarray(offset, float)) - g[None, :, :]
    return 1.0 / (4 * np.pi * np.linalg.norm(d, axis=-1))


def test_aca_recovers_a_low_rank_matrix_exactly():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((50, 3)) @ rng.standard_normal((3, 40))
    A, B = O.aca(M, 1e-12)
    assert A.shape == (50, 3) and B.shape == (40, 3)
    assert np.abs(A @ B.T - M).max() < 1e-13 * np.abs(M).max()


def test_aca_is_gaussian_elimination_with_full_pivoting():
    """After k steps the residual vanishes on k rows and k columns (the pivots), its
    first pivot is the largest entry, and n steps reproduce a full-rank n x n matrix."""
    rng = np.random.default_rng(1)
    M = rng.standard_normal((9, 9))
    A, B = O.aca(M, 0.0)
    assert A.shape[1] == 9 and np.abs(A @ B.T - M).max() < 1e-12
    i, j = np.unravel_index(np.argmax(np.abs(M)), M.shape)
    assert np.allclose(A[:, 0], M[:, j]) and np.allclose(B[:, 0], M[i, :] / M[i, j])
    for k in (2, 5):
        A, B = O.aca(M, 0.0, kmax=k)
        R = M - A @ B.T
        assert np.sum(np.abs(R).max(axis=1) < 1e-12) == k
        assert np.sum(np.abs(R).max(axis=0) < 1e-12) == k


@pytest.mark.parametrize("r1", [4, 5])
@pytest.mark.parametrize("offset", [(2, 0, 0), (2, 2, 2), (3, 1, 0)])
def test_aca_of_the_laplace_transfer_meets_its_tolerance_near_the_optimal_rank(r1, offset):
    """Frobenius error <= tol (the stopping rule is exact), and the rank is at least the
    Eckart-Young minimum for that error (from the singular values) and within a small
    factor of it."""
    T = _laplace_T(r1, offset)
    s = np.linalg.svd(T, compute_uv=False)
    tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]  # tail[k] = error of the best rank-k
    prev = 0
    for tol in (1e-3, 1e-4, 1e-5, 1e-7):
        A, B = O.aca(T, tol)
        k = A.shape[1]
        assert np.linalg.norm(T - A @ B.T) <= tol * np.linalg.norm(T) * (1 + 1e-9)
        kmin = int(np.sum(tail > tol * np.linalg.norm(T)))
        assert kmin <= k <= 1.5 * kmin + 6
        assert k >= prev
        prev = k


def test_ffm_with_aca_within_eps_and_within_aca_eps_of_the_dense_transfer():
    prob = W.laplace_sphere(20000)
    ref = O.direct(prob.X, prob.Y, prob.u, O.LAPLACE, w=prob.w)
    dense = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w)
    ranks = []
    for ae in (1e-4, 1e-5):
        p = O.Plan(prob.X, prob.Y, O.LAPLACE, 0.0, prob.eps, aca_eps=ae)
        st = p.stats()
        v = p.apply(prob.u, prob.w)
        p.close()
        lag = [l for l in range(st["l_stop"] + 1) if st["n_adm"][l] > 0]
        r = st["r1"][lag[0]] ** 3
        assert all(0 < st["aca_rank"][l] < r for l in lag)
        ranks.append(max(st["aca_rank"]))
        assert O.rel_l2(v, ref) < prob.eps
        assert O.rel_l2(v, dense) < ae
    assert ranks[1] > ranks[0]


def test_ffm_with_a_vanishing_aca_tolerance_is_the_dense_ffm():
    prob = W.laplace_sphere(6000)
    dense = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w)
    v = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w, aca_eps=1e-15)
    assert O.rel_l2(v, dense) < 1e-12
