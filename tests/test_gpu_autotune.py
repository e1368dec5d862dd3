"""ffm_autotune: the picks are valid kernel variants, a tuned plan gives the untuned
plan's result up to rounding, and a cache file replays the same picks on a new plan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _plan(prob):
    return ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, prob.k, prob.eps, weights=_t(prob.w))


def _picks(info):
    return (info["p2p_tchunk"], info["p2p_smax"], tuple(info["tune_tc"]), tuple(map(tuple, info["tune_pw"])))


@pytest.mark.parametrize("case", ["helmholtz", "laplace_clustered", "helmholtz_multirhs"])
def test_autotune_keeps_results_and_replays_from_cache(case, tmp_path):
    assert torch.cuda.is_available()
    if case == "helmholtz":
        prob = W.helmholtz_sphere(100000)
        U, nrhs = prob.u, 1
    elif case == "laplace_clustered":
        prob = W.laplace_clustered(200000)
        U, nrhs = prob.u, 1
    else:
        prob = W.helmholtz_cube_multirhs(30000, nrhs=8, eps=1e-3)
        U, nrhs = prob.u.T, 8
    Ud = _t(U)
    cache = str(tmp_path / "tune.txt")
    with _plan(prob) as p:
        before = p.info()
        assert before["autotuned"] == 0
        v0 = p.apply(Ud).cpu().numpy()
        after = p.autotune(nrhs=nrhs, cache_path=cache)
        v1 = p.apply(Ud).cpu().numpy()
    assert after["autotuned"] == 1
    assert after["p2p_tchunk"] in (64, 128) and after["p2p_smax"] in (2048, 4096, 8192)
    for l in range(after["l_stop"] + 1):
        if after["mode"][l] == 2 and after["n_adm"][l] > 0:
            q, pp, mc = after["tune_pw"][l]
            assert q in (2, 4) and pp in (2, 4) and mc in ((0, 4, 8) if nrhs > 1 else (4, 8))
    # same algorithm and operators: the near-field sums are split differently, and the Lagrange
    # transfer or the several-RHS plane-wave transforms may move between TF32x3 tensor-core and
    # FP32 CUDA-core products, so the results differ by rounding only
    tol = 1e-5 if nrhs > 1 else 5e-6
    assert O.rel_l2(v1, v0) < tol
    lines = open(cache).read().splitlines()
    assert lines and all(" = " in ln for ln in lines)
    with _plan(prob) as p2:
        again = p2.autotune(nrhs=nrhs, cache_path=cache)
    assert _picks(again) == _picks(after)
    assert open(cache).read().splitlines() == lines  # all keys were found: nothing re-timed or appended
    # a plan created with the cache takes the stored picks without timing anything
    with ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, prob.k, prob.eps, weights=_t(prob.w),
                  autotune_cache=cache) as p3:
        made = p3.info()
        v3 = p3.apply(Ud).cpu().numpy()
    if nrhs == 1:
        assert _picks(made) == _picks(after)
    assert O.rel_l2(v3, v0) < tol
