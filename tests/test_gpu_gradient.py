"""The gradient of the Laplace single layer in the target variable (FFM_LAPLACE_GRAD, the MFIE
kernel of Sec. 4.2) through the GPU path: parity with the oracle FFM and the FP64 direct sum,
the field of a uniformly charged sphere, several right-hand sides, and the transfer variants."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu
TOL_FFM = 1e-5


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _plan(X, Y, eps, w, **kw):
    return ffm.Plan(_t(X), _t(Y), ffm.LAPLACE_GRAD, 0.0, eps, weights=_t(w), **kw)


def _grad_gpu(p, u):
    v = p.apply(_t(u))
    torch.cuda.synchronize()
    v = v.cpu().numpy()
    return np.moveaxis(v, -2, -1)  # (nx, 3) or (nrhs, nx, 3)


@pytest.mark.parametrize("eps,rad", [(1e-3, 0.6), (1e-4, 1.25)])
def test_gradient_matches_oracle_ffm_and_direct(eps, rad):
    assert torch.cuda.is_available()
    n = 20000
    Y = W.sphere_surface(n, 1001)
    X = W.sphere_surface(n, 1) * rad
    u = np.random.default_rng(3).standard_normal(n)
    w = np.full(n, 4 * np.pi / n)
    with _plan(X, Y, eps, w) as p:
        info = p.info()
        g = _grad_gpu(p, u)
    lag = [l for l in range(info["l_stop"] + 1) if info["n_adm"][l] > 0]
    assert lag and all(info["mode"][l] == 1 and info["r1"][l] == O.r1_rule(O.LAPLACE_GRAD, eps) for l in lag)
    ref_ffm = O.ffm_grad(X, Y, u, eps, w=w)[:, 0, :]
    assert O.rel_l2(g, ref_ffm) < TOL_FFM
    t = W.sample_targets(n, 3000)
    ref = O.direct_grad(X, Y, u, w=w, targets=t)[:, 0, :]
    assert O.rel_l2(g[t], ref) < eps


def test_gradient_of_a_charged_sphere_on_gpu():
    """Unit density on a fine random sphere: field 0 inside, -x/|x|^3 outside, to the FFM
    accuracy against the FP64 sum over the same points plus the quadrature error."""
    n = 200000
    Y = W.sphere_surface(n, 77)
    w = np.full(n, 4 * np.pi / n)
    X = np.array([[0.1, 0.2, -0.3], [0.0, 0.0, 0.05], [1.5, 0.3, 0.2], [0.0, -2.0, 0.5], [2.0, 2.0, -2.0]])
    with _plan(X, Y, 1e-4, w) as p:
        g = _grad_gpu(p, np.ones(n))
    direct = O.direct_grad(X, Y, np.ones(n), w=w)[:, 0, :]
    assert np.max(np.abs(g - direct)) < 1e-4 * max(1.0, np.max(np.abs(direct)))
    assert np.max(np.abs(g[:2])) < 2e-2
    exact = -X[2:] / np.linalg.norm(X[2:], axis=1)[:, None] ** 3
    assert np.max(np.abs(g[2:] - exact)) < 2e-2


def test_gradient_several_rhs_and_transfer_variants():
    n = 15000
    Y = W.sphere_surface(n, 11)
    X = W.sphere_surface(n, 12) * 0.7
    rng = np.random.default_rng(5)
    U = rng.standard_normal((3, n))
    w = np.full(n, 4 * np.pi / n)
    with _plan(X, Y, 1e-3, w) as p:
        G = _grad_gpu(p, U)
        for m in range(3):
            assert O.rel_l2(G[m], _grad_gpu(p, U[m])) < 1e-6
    with _plan(X, Y, 1e-3, w, lagrange_transfer=ffm.LAG_CUDA_CORES) as p:
        Gc = _grad_gpu(p, U)
    assert O.rel_l2(Gc, G) < 5e-6
    ref = O.ffm_grad(X, Y, U.T, 1e-3, w=w)  # (nx, nrhs, 3)
    assert O.rel_l2(G, np.moveaxis(ref, 1, 0)) < TOL_FFM
