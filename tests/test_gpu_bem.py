"""The boundary-element wrapper (Sec. 4.2) on the GPU, through the C ABI: the operator
S = (Lambda*)^T (G W) Lambda + C against the oracle (FFM and dense), GMRES against the dense
solve, and the unit density of the sphere's single layer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import bem as B
from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_bem_operator_matches_the_oracle():
    assert torch.cuda.is_available()
    V, F = W.icosphere(3)
    u = np.random.default_rng(7).standard_normal(len(V))
    with ffm.Bem(_t(V), _t(F), eps=1e-4) as bem:
        v = bem.apply(_t(u)).cpu().numpy()
    C = B.correction(V, F)
    assert O.rel_l2(v, B.apply_ffm(V, F, u, 1e-4, C=C)) < 1e-5
    assert O.rel_l2(v, B.dense_matrix(V, F) @ u) < 1e-4


def test_bem_gmres_matches_the_dense_solve_and_gives_unit_density():
    V, F = W.icosphere(3)
    X, w, L = B.quadrature(V, F)
    rhs = L.T @ w  # Galerkin right-hand side of the constant 1
    with ffm.Bem(_t(V), _t(F), eps=1e-6) as bem:
        # the FFM product's rounding varies from one application to the next (FP32 atomics) at
        # about 1e-7 of its value, which bounds the attainable residual
        x, iters, rr = bem.solve(_t(rhs), tol=1e-7, restart=40, maxit=400)
        assert rr <= 1e-7 and 0 < iters < 400 and bem.products() >= iters
        # the true residual through the operator itself
        res = bem.apply(x).cpu().numpy() - rhs
        assert np.linalg.norm(res) < 1e-6 * np.linalg.norm(rhs)
    x = x.cpu().numpy()
    ref = np.linalg.solve(B.dense_matrix(V, F), rhs)
    assert O.rel_l2(x, ref) < 1e-3
    assert abs(x.mean() - 1.0) < 5e-3 and np.max(np.abs(x - 1.0)) < 4e-2


def test_bem_host_vectors_and_errors():
    V, F = W.icosphere(1)
    with ffm.Bem(V, F, eps=1e-3) as bem:
        u = np.ones(len(V))
        v = bem.apply(u)
        assert v.shape == u.shape and np.all(np.isfinite(v))
        x, it, rr = bem.solve(np.zeros(len(V)))
        assert it == 0 and rr == 0.0 and np.all(x == 0)
    bad = F.copy()
    bad[0, 0] = len(V)
    with pytest.raises(ffm.FFMError) as e:
        ffm.Bem(V, bad)
    assert e.value.status == 1
