"""Captured applies (ffm_graph_*): one CUDA graph launch per product gives the result of
ffm_apply on the current contents of u, for repeated products with changing densities
as in an iterative solve, and counts its kernels."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("case", ["helmholtz_multirhs", "laplace"])
def test_graph_replay_equals_apply_on_changing_densities(case):
    assert torch.cuda.is_available()
    rng = np.random.default_rng(5)
    if case == "laplace":
        prob = W.laplace_sphere(20000)
        U = _t(prob.u)
        new = lambda: rng.standard_normal(20000)
    else:
        prob = W.helmholtz_cube_multirhs(20000, nrhs=3, eps=1e-3)
        U = _t(prob.u.T)
        new = lambda: (rng.standard_normal((3, 20000)) + 1j * rng.standard_normal((3, 20000))).astype(np.complex64)
    V = torch.empty_like(U)
    with ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, prob.k, prob.eps, weights=_t(prob.w)) as p:
        n0 = ffm.launch_count()
        with p.graph(U, V) as g:
            assert ffm.launch_count() == n0  # capturing runs nothing
            assert g.kernels > 4
            for trial in range(3):
                U.copy_(_t(new()))
                n1 = ffm.launch_count()
                g.launch()
                torch.cuda.synchronize()
                assert ffm.launch_count() - n1 == g.kernels
                ref = p.apply(U)
                torch.cuda.synchronize()
                # the two runs differ only in the order of atomic additions
                assert O.rel_l2(V.cpu().numpy(), ref.cpu().numpy()) < 1e-6


def test_graph_needs_device_buffers():
    prob = W.laplace_sphere(2000)
    with ffm.Plan(_t(prob.X), _t(prob.Y), prob.kind, 0.0, 1e-3) as p:
        u = np.ones(2000)
        with pytest.raises(ffm.FFMError) as e:
            p.graph(u, np.empty(2000))
        assert e.value.status == 1
