"""Continuous-batching server on the GPU: a request gives the same result alone and in a
mix of concurrent requests (including being merged into a multi-RHS apply with another
request on the same plan), and latency statistics are recorded."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_1909_05600_gb300 import ffm, workloads as W
from paper_1909_05600_gb300.serving import Request, Server, latency_stats

pytestmark = pytest.mark.gpu


def _req(rid, prob, key, u=None):
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return Request(rid=rid, key=key, nx=prob.X.shape[0], ny=prob.Y.shape[0], kind=prob.kind, k=prob.k,
                   eps=prob.eps, X=t(prob.X), Y=t(prob.Y), w=t(prob.w), u=t(prob.u if u is None else u))


def _alone(r):
    with ffm.Plan(r.X, r.Y, r.kind, r.k, r.eps, weights=r.w) as p:
        v = p.apply(r.u)
        torch.cuda.synchronize()
    return v.cpu().numpy()


def test_same_result_alone_and_in_a_mix():
    assert torch.cuda.is_available()
    a = W.helmholtz_sphere(30000, seed=2)
    b = W.laplace_sphere(25000, seed=3)
    c = W.helmholtz_cube_multirhs(20000, nrhs=1, seed=4, eps=1e-4)
    c.u = np.ascontiguousarray(c.u[:, 0])
    d_u = (np.random.default_rng(9).standard_normal(30000) + 0j).astype(np.complex64)
    reqs = [_req(0, a, ("a",)), _req(1, b, ("b",)), _req(2, c, ("c",)), _req(3, a, ("a",), d_u)]
    alone = [_alone(r) for r in reqs]
    srv = Server(workers=3)
    try:
        for r in reqs:
            srv.submit(r)
        srv.drain(len(reqs), timeout=300)
    finally:
        srv.close()
    for r, v0 in zip(reqs, alone):
        assert r.error is None, r.error
        v = r.result.cpu().numpy()
        assert O.rel_l2(v, v0) < 1e-6, (r.rid, O.rel_l2(v, v0))
    st = latency_stats(reqs)
    assert st["completed"] == 4 and st["p99_ms"] >= st["p50_ms"] > 0
    assert srv.batches >= 1 and srv.device_ms > 0


def test_oversize_request_is_rejected_others_complete():
    a = W.laplace_sphere(20000, seed=5)
    srv = Server(workers=2, budget_bytes=400 << 20)
    try:
        big = Request(rid=9, key=("big",), nx=5_000_000, ny=5_000_000, kind=1, k=1.0, eps=1e-3)
        srv.submit(big)
        r = _req(1, a, ("a",))
        srv.submit(r)
        srv.drain(2, timeout=120)
    finally:
        srv.close()
    assert big.error and "budget" in big.error
    assert r.error is None and r.result is not None
