"""Plane-wave transforms of several right-hand sides on the tensor cores (k_pw_forward_tc,
k_pw_backward_tc: TF32 x3 products, FP32 accumulation in tensor memory) against the plain CPU
FFM, the FP64 direct sum and the CUDA-core kernels of the same plan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu

TOL_FFM = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _device():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1909_05600_gb300 import build
    build.build()
    ffm.lib()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _run(prob, U, pw, **opts):
    """Product of the (nrhs, n) densities U, the kernels that ran, and the plan's info."""
    with ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, prob.k, prob.eps, weights=_t(prob.w), pw_transform=pw,
                  **opts) as gp:
        ffm.profile_enable(True)
        ffm.profile_reset()
        try:
            v = gp.apply(_t(U))
            torch.cuda.synchronize()
            prof = ffm.profile_read()
        finally:
            ffm.profile_enable(False)
        info = gp.info()
    return v.cpu().numpy(), prof, info


def _ran(prof, stem):
    return any(k.startswith(stem + "<") for k in prof)


@pytest.mark.parametrize("nrhs", [3, 70])
def test_tensor_core_transforms_match_the_oracle(nrhs):
    # 70 right-hand sides: two groups of 64 columns, the second ragged
    prob = W.helmholtz_cube_multirhs(30000, nrhs=nrhs, eps=1e-4)
    U = np.ascontiguousarray(prob.u.T)
    V, prof, info = _run(prob, U, ffm.PW_DIRECT_TC)
    assert info["device_errors"] == 0
    assert _ran(prof, "k_pw_forward_tc") and _ran(prof, "k_pw_backward_tc"), sorted(prof)
    Vc, prof_c, _ = _run(prob, U, ffm.PW_DIRECT)
    assert not any(k.startswith("k_pw") and "_tc<" in k for k in prof_c)
    cols = [0, 1, nrhs - 1] if nrhs < 64 else [0, 63, 64, nrhs - 1]
    ref = O.ffm(prob.X, prob.Y, prob.u[:, cols].astype(np.complex128), O.HELMHOLTZ, prob.k, prob.eps, w=prob.w)
    for i, m in enumerate(cols):
        assert O.rel_l2(V[m], ref[:, i]) < TOL_FFM, m
    # against the CUDA-core kernels of the same plan: rounding only
    assert O.rel_l2(V, Vc) < 5e-6
    t = W.sample_targets(30000, 500)
    m = cols[-1]
    direct = O.direct(prob.X, prob.Y, prob.u[:, m].astype(np.complex128), O.HELMHOLTZ, prob.k, w=prob.w,
                      targets=t)[:, 0]
    assert O.rel_l2(V[m][t], direct) < prob.eps


def test_columns_are_independent_and_repeatable():
    # column m of a 66-column product equals the same column in a 2-column product (its group
    # of 64 and its position in the group change), and a second apply gives the same result
    prob = W.helmholtz_cube_multirhs(20000, nrhs=66, eps=1e-4)
    U = np.ascontiguousarray(prob.u.T)
    V, _, _ = _run(prob, U, ffm.PW_DIRECT_TC)
    V2, _, _ = _run(prob, np.ascontiguousarray(U[[65, 3]]), ffm.PW_DIRECT_TC)
    assert O.rel_l2(V2[0], V[65]) < 1e-6
    assert O.rel_l2(V2[1], V[3]) < 1e-6


def test_auto_uses_the_tensor_cores_from_16_right_hand_sides():
    prob = W.helmholtz_cube_multirhs(20000, nrhs=16, eps=1e-4)
    U = np.ascontiguousarray(prob.u.T)
    _, prof16, _ = _run(prob, U, ffm.PW_AUTO)
    _, prof8, _ = _run(prob, np.ascontiguousarray(U[:8]), ffm.PW_AUTO)
    assert _ran(prof16, "k_pw_forward_tc")
    assert not _ran(prof8, "k_pw_forward_tc") and not _ran(prof8, "k_pw_backward_tc")


def test_wait_give_up_reports_timeout_and_leaves_the_device_usable():
    prob = W.helmholtz_cube_multirhs(30000, nrhs=4, eps=1e-4)  # an FP32 and a compensated level
    U = np.ascontiguousarray(prob.u.T)
    with ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, prob.k, prob.eps, weights=_t(prob.w),
                  pw_transform=ffm.PW_DIRECT_TC, wait_tries=-1) as p:
        p.apply(_t(U))
        torch.cuda.synchronize()
        with pytest.raises(ffm.FFMError) as e:
            p.info()
        assert e.value.status == 4  # FFM_ETIMEOUT
    V, prof, info = _run(prob, U, ffm.PW_DIRECT_TC)
    assert info["device_errors"] == 0 and _ran(prof, "k_pw_backward_tc")
    ref = O.ffm(prob.X, prob.Y, prob.u[:, :1].astype(np.complex128), O.HELMHOLTZ, prob.k, prob.eps, w=prob.w)
    assert O.rel_l2(V[0], ref[:, 0]) < TOL_FFM
