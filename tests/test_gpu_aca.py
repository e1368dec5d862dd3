"""ACA of the Lagrange transfer matrices (Sec. 2.2.2, eq. 11) on the GPU through the C ABI:
the per-level ranks equal the oracle's, the products match the oracle's ACA FFM and the
FP64 direct sum, both transfer variants and several right-hand sides agree, and the
options are checked."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu
TOL_FFM = 1e-5


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _plan(prob, eps, **kw):
    return ffm.Plan(_t(prob.X), _t(prob.Y), ffm.LAPLACE, 0.0, eps, weights=_t(prob.w), **kw)


def _apply(p, u):
    v = p.apply(_t(u))
    torch.cuda.synchronize()
    return v.cpu().numpy()


# r = 64 and r = 125 keep the residual in shared memory (125 KB at r = 125), r = 216 in global memory
@pytest.mark.parametrize("n,eps,aca_eps", [(20000, 1e-3, 1e-4), (12000, 5e-4, 5e-5), (8000, 1e-4, 1e-5)])
def test_aca_ranks_and_products_match_the_oracle(n, eps, aca_eps):
    assert torch.cuda.is_available()
    prob = W.laplace_sphere(n)
    with _plan(prob, eps, aca_eps=aca_eps) as p:
        info = p.info()
        v = _apply(p, prob.u)
    op = O.Plan(prob.X, prob.Y, O.LAPLACE, 0.0, eps, aca_eps=aca_eps)
    st = op.stats()
    ref = op.apply(prob.u, prob.w)[:, 0].real
    op.close()
    lag = [l for l in range(info["l_stop"] + 1) if info["n_adm"][l] > 0]
    assert lag and all(info["mode"][l] == 1 for l in lag)
    assert [info["aca_rank"][l] for l in lag] == [st["aca_rank"][l] for l in lag]
    assert O.rel_l2(v, ref) < TOL_FFM
    t = W.sample_targets(n, 2000)
    direct = O.direct(prob.X, prob.Y, prob.u, O.LAPLACE, w=prob.w, targets=t)[:, 0].real
    assert O.rel_l2(v[t], direct) < eps


def test_aca_transfer_variants_and_several_rhs():
    prob = W.laplace_sphere(15000)
    U = np.random.default_rng(5).standard_normal((3, 15000))
    with _plan(prob, 1e-3, aca_eps=1e-4) as p:
        V = _apply(p, U)
        for m in range(3):
            assert O.rel_l2(V[m], _apply(p, U[m])) < 1e-6
    with _plan(prob, 1e-3, aca_eps=1e-4, lagrange_transfer=ffm.LAG_CUDA_CORES) as p:
        Vc = _apply(p, U)
    assert O.rel_l2(Vc, V) < 5e-6
    with _plan(prob, 1e-3) as p:
        Vd = _apply(p, U)
    assert O.rel_l2(V, Vd) < 1e-4  # within aca_eps of the dense transfer


def test_aca_options_are_checked():
    prob = W.laplace_sphere(2000)
    with pytest.raises(ffm.FFMError) as e:
        _plan(prob, 1e-3, aca_eps=-1.0)
    assert e.value.status == 1
    with pytest.raises(ffm.FFMError) as e:
        _plan(prob, 1e-3, aca_eps=1.5)
    assert e.value.status == 1
    X = _t(prob.X)
    with pytest.raises(ffm.FFMError) as e:
        ffm.Plan(X, X, ffm.HELMHOLTZ, 5.0, 1e-3, aca_eps=1e-4)
    assert e.value.status == 5
