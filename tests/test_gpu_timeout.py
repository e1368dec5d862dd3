"""The FFM_ETIMEOUT path of the tensor-core transfer kernels, exercised from the host and
without a fault: with ffm_opts.wait_tries = -1 every bounded mbarrier wait gives up at once.
The kernels then skip their results, still wait for the tensor-core work they had committed
before they free TMEM, and raise the plan's device error flag, which ffm_plan_info reports as
FFM_ETIMEOUT.  Afterwards the device must still compute a correct product."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("variant", [ffm.LAG_TC_TRANSLATION, ffm.LAG_TC_TARGET])
def test_wait_give_up_reports_timeout_and_leaves_the_device_usable(variant):
    assert torch.cuda.is_available()
    prob = W.laplace_sphere(20000, seed=4)
    X, Y, w, u = _t(prob.X), _t(prob.Y), _t(prob.w), _t(prob.u)
    with ffm.Plan(X, Y, ffm.LAPLACE, 0.0, prob.eps, weights=w, lagrange_transfer=variant, wait_tries=-1) as p:
        p.apply(u)
        torch.cuda.synchronize()
        with pytest.raises(ffm.FFMError) as e:
            p.info()
        assert e.value.status == 4  # FFM_ETIMEOUT
    # same device, same variant, default waits: a correct product
    with ffm.Plan(X, Y, ffm.LAPLACE, 0.0, prob.eps, weights=w, lagrange_transfer=variant) as p:
        v = p.apply(u)
        torch.cuda.synchronize()
        info = p.info()
    assert info["device_errors"] == 0
    lag = [l for l in range(info["l_stop"] + 1) if info["n_adm"][l] > 0 and info["mode"][l] == 1]
    assert lag and all(info["tune_tc"][l] == (2 if variant == ffm.LAG_TC_TARGET else 1) for l in lag)
    ref = O.ffm(prob.X, prob.Y, prob.u, O.LAPLACE, 0.0, prob.eps, w=prob.w)[:, 0].real
    assert O.rel_l2(v.cpu().numpy(), ref) < 1e-5


def test_wait_tries_option_is_checked_on_the_host():
    prob = W.laplace_sphere(2000, seed=4)
    with pytest.raises(ffm.FFMError) as e:
        ffm.Plan(_t(prob.X), _t(prob.Y), ffm.LAPLACE, 0.0, prob.eps, wait_tries=-2)
    assert e.value.status == 1
