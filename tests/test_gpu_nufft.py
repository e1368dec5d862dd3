"""The plane-wave F steps as type-3 NUFFTs (Sec. 2.2.3) on the GPU, through the C ABI.

Forced NUFFT levels against the oracle's FFM with the same NUFFT (rel-L2 <= 1e-5: the same
approximation, FP32 against FP64 arithmetic) and with direct plane-wave sums (<= eps / 10);
several right-hand sides against one at a time; the automatic choice against the GPU's
own direct sums; a captured apply against the eager one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu

TOL_FFM = 1e-5
KAPPA = 8.0  # plane waves only at k d_l >= 8 on both sides: well-conditioned (FP32) levels


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1909_05600_gb300 import build
    build.build()
    ffm.lib()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _plan(prob, **kw):
    return ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, prob.k, prob.eps, weights=_t(prob.w), **kw)


def _apply(p, u):
    v = p.apply(_t(u))
    torch.cuda.synchronize()
    return v.cpu().numpy()


def _pw_levels(info):
    return [l for l in range(info["l_stop"] + 1) if info["mode"][l] == 2 and info["n_adm"][l] > 0]


@pytest.mark.parametrize("eps,ppw", [(1e-3, 5.0), (1e-4, 6.0)])
def test_forced_nufft_matches_oracle_nufft_and_direct(eps, ppw):
    prob = W.helmholtz_sphere(20000, seed=4, eps=eps, ppw=ppw)
    with _plan(prob, kappa_switch=KAPPA, pw_transform=ffm.PW_NUFFT) as p:
        info = p.info()
        v = _apply(p, prob.u)
    pw = _pw_levels(info)
    assert pw, "the workload must have plane-wave levels"
    assert all(info["nufft"][l] == 1 for l in pw), (info["nufft"], info["pw_prec"])
    u = prob.u.astype(np.complex128)
    ref_nu = O.ffm_nufft(prob.X, prob.Y, u, prob.kind, prob.k, eps, w=prob.w, kappa_switch=KAPPA)[:, 0]
    assert O.rel_l2(v, ref_nu) < TOL_FFM
    # against the same FFM with direct plane-wave sums: the NUFFT's own error, about eps / 200
    # per transform (the Lagrange levels below kappa = 8 are not the NUFFT's concern here)
    ref_d = O.ffm(prob.X, prob.Y, u, prob.kind, prob.k, eps, w=prob.w, kappa_switch=KAPPA)[:, 0]
    assert O.rel_l2(v, ref_d) < eps / 10


def test_forced_nufft_several_rhs_match_one_at_a_time():
    prob = W.helmholtz_sphere(15000, seed=5, eps=1e-3, ppw=5.0)
    rng = np.random.default_rng(11)
    U = np.stack([prob.u, (rng.standard_normal(15000) + 1j * rng.standard_normal(15000)).astype(np.complex64),
                  prob.u * (0.5 - 2j)], 0)
    with _plan(prob, kappa_switch=KAPPA, pw_transform=ffm.PW_NUFFT) as p:
        assert any(p.info()["nufft"])
        V = _apply(p, U)
        for m in range(3):
            assert O.rel_l2(V[m], _apply(p, U[m])) < 1e-6


def test_auto_choice_uses_nufft_on_wide_levels_and_agrees_with_direct_sums():
    prob = W.helmholtz_sphere(200000, seed=6, eps=1e-3)
    with _plan(prob) as p:
        info = p.info()
        v = _apply(p, prob.u)
    with _plan(prob, pw_transform=ffm.PW_DIRECT) as p:
        assert not any(p.info()["nufft"])
        vd = _apply(p, prob.u)
    wide = [l for l in _pw_levels(info) if info["nQ"][l] >= 8000 and info["pw_prec"][l] == ffm.PREC_F32]
    assert wide and all(info["nufft"][l] == 1 for l in wide)
    assert all(info["nufft"][l] == 0 for l in _pw_levels(info) if info["nQ"][l] < 8000)
    # the NUFFT error is about eps / 200 per transform
    assert O.rel_l2(v, vd) < prob.eps / 20
    t = W.sample_targets(prob.X.shape[0], 2000)
    ref = O.direct(prob.X, prob.Y, prob.u.astype(np.complex128), prob.kind, prob.k, w=prob.w, targets=t)[:, 0]
    assert O.rel_l2(v[t], ref) < prob.eps


def test_nufft_apply_in_a_graph_matches_eager():
    prob = W.helmholtz_sphere(15000, seed=7, eps=1e-3, ppw=5.0)
    with _plan(prob, kappa_switch=KAPPA, pw_transform=ffm.PW_NUFFT) as p:
        u = _t(prob.u)
        out = torch.empty_like(u)
        eager = p.apply(u).cpu().numpy()
        with p.graph(u, out) as g:
            for _ in range(2):
                out.zero_()
                g.launch()
                torch.cuda.synchronize()
                assert O.rel_l2(out.cpu().numpy(), eager) < 1e-6


def test_pw_transform_option_is_checked():
    prob = W.helmholtz_sphere(2000, seed=8)
    with pytest.raises(ffm.FFMError) as e:
        _plan(prob, pw_transform=4)
    assert e.value.status == 1
