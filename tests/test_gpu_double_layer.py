"""The Laplace double layer (dG/dn_y) through the GPU path: parity with the oracle FFM
and the FP64 direct sum, Gauss's law on the unit sphere, several right-hand sides, and
the argument checks of the normals."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu
TOL_FFM = 1e-5


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _plan(X, Y, nrm, eps, w=None, **kw):
    return ffm.Plan(_t(X), _t(Y), ffm.LAPLACE_DL, 0.0, eps, weights=None if w is None else _t(w), normals=_t(nrm),
                    **kw)


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_double_layer_matches_oracle_ffm_and_direct(eps):
    assert torch.cuda.is_available()
    prob = W.laplace_double_layer_sphere(20000, eps=eps)
    nrm = prob.meta["normals"]
    with _plan(prob.X, prob.Y, nrm, eps, prob.w) as p:
        info = p.info()
        v = p.apply(_t(prob.u)).cpu().numpy()
    lag = [l for l in range(info["l_stop"] + 1) if info["n_adm"][l] > 0]
    assert lag and all(info["mode"][l] == 1 for l in lag)
    assert all(info["r1"][l] == O.r1_rule(O.LAPLACE_DL, eps) for l in lag)
    ref_ffm = O.ffm_dl(prob.X, prob.Y, nrm, prob.u, eps, w=prob.w)[:, 0]
    assert O.rel_l2(v, ref_ffm) < TOL_FFM
    t = W.sample_targets(20000, 2000)
    ref = O.direct_dl(prob.X, prob.Y, nrm, prob.u, w=prob.w, targets=t)[:, 0]
    assert O.rel_l2(v[t], ref) < eps


def test_double_layer_gauss_law_on_gpu():
    """Unit density on a fine random sphere (outward normals, weights 4 pi / n): -1 inside,
    0 outside, to the FFM accuracy plus the Monte Carlo quadrature error."""
    n = 200000
    Y = W.sphere_surface(n, 77)
    w = np.full(n, 4.0 * math.pi / n)
    X = np.array([[0.1, 0.2, -0.3], [0.0, 0.0, 0.05], [-0.4, 0.3, 0.35], [1.5, 0.3, 0.2], [0.0, -2.0, 0.5]])
    with _plan(X, Y, Y, 1e-4, w) as p:
        v = p.apply(_t(np.ones(n))).cpu().numpy()
    direct = O.direct_dl(X, Y, Y, np.ones(n), w=w)[:, 0]
    assert np.max(np.abs(v - direct)) < 3e-4  # GPU vs FP64 sum over the same points (eps = 1e-4)
    assert np.max(np.abs(v[:3] + 1.0)) < 2e-2  # Gauss (Monte Carlo quadrature)
    assert np.max(np.abs(v[3:])) < 2e-2


def test_double_layer_several_rhs_and_float32_normals():
    prob = W.laplace_double_layer_sphere(15000, seed=3)
    nrm = prob.meta["normals"]
    U = np.stack([prob.u, np.random.default_rng(9).standard_normal(15000)], 0)
    with _plan(prob.X, prob.Y, nrm.astype(np.float32), prob.eps, prob.w) as p:
        V = p.apply(_t(U)).cpu().numpy()
    for m in range(2):
        ref = O.ffm_dl(prob.X, prob.Y, nrm.astype(np.float32).astype(np.float64), U[m], prob.eps, w=prob.w)[:, 0]
        assert O.rel_l2(V[m], ref) < TOL_FFM


def test_double_layer_needs_normals():
    X = _t(np.random.default_rng(0).random((100, 3)))
    with pytest.raises(ffm.FFMError) as e:
        ffm.Plan(X, X, ffm.LAPLACE_DL, 0.0, 1e-3)
    assert e.value.status == 1
