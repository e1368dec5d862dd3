"""The tcgen05 Lagrange transfer in row blocks: at eps 1e-6 the Laplace operator has r = 512
rows (r1 = 8), three blocks of at most 224, and must match the oracle FFM and the CUDA-core
transfer."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _apply(prob, **kw):
    with ffm.Plan(_t(prob.X), _t(prob.Y), ffm.LAPLACE, 0.0, prob.eps, weights=_t(prob.w), **kw) as p:
        info = p.info()
        v = p.apply(_t(prob.u))
        torch.cuda.synchronize()
    return info, v.cpu().numpy()


def test_row_blocked_tensor_core_transfer_at_r512():
    assert torch.cuda.is_available()
    prob = W.laplace_sphere(6000, eps=1e-6)
    info, v = _apply(prob)
    lag = [l for l in range(info["l_stop"] + 1) if info["n_adm"][l] > 0]
    assert lag and all(info["r1"][l] == 8 and info["tune_tc"][l] == 1 for l in lag)
    ref = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w)[:, 0].real
    assert O.rel_l2(v, ref) < 1e-5
    info_c, vc = _apply(prob, lagrange_transfer=ffm.LAG_CUDA_CORES)
    assert all(info_c["tune_tc"][l] == 0 for l in lag)
    assert O.rel_l2(vc, v) < 5e-6


def test_aca_second_stage_in_row_blocks_at_r512():
    """ACA at eps 1e-6: stage 2 (A_t, r = 512 rows) runs in three row blocks.  The ranks equal
    the oracle plan's, and the product stays within a few aca_eps of the dense transfer (which
    the test above pins to the oracle)."""
    prob = W.laplace_sphere(6000, eps=1e-6)
    info, v_aca = _apply(prob, aca_eps=1e-6)
    _, v = _apply(prob)
    lag = [l for l in range(info["l_stop"] + 1) if info["n_adm"][l] > 0]
    op = O.Plan(prob.X, prob.Y, O.LAPLACE, 0.0, prob.eps, aca_eps=1e-6)
    ranks = op.stats()["aca_rank"]
    op.close()
    assert [info["aca_rank"][l] for l in lag] == [ranks[l] for l in lag]
    assert all(info["tune_tc"][l] == 1 for l in lag)
    assert O.rel_l2(v_aca, v) < 1e-5
