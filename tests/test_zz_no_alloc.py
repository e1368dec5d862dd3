"""ffm_morton_order_noalloc: the Morton ordering computed with no device allocation inside
the library.  It exists for callers that cannot allocate device memory while they run;
its scratch is one fixed static device array.  This checks, through the C ABI, that it
gives exactly the ordering ffm_plan gives X (with Y = X), on consecutive calls that reuse
the shared scratch array, and that sizes beyond the array are refused.  Collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1909_05600_gb300 import ffm, workloads as W

pytestmark = pytest.mark.gpu


def _plan_order(X):
    with ffm.Plan(X, X, ffm.LAPLACE, 0.0, 1e-3) as p:
        return p.perm("X")


def _noalloc_order(X):
    out = torch.empty(X.shape[0], dtype=torch.int32, device=X.device)
    ffm.morton_order_noalloc(X, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).astype(np.int64)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_order_equals_plan_order_on_consecutive_calls(dtype):
    assert torch.cuda.is_available(), "GPU test needs a CUDA device"
    from paper_1909_05600_gb300 import build
    build.build()
    A = torch.as_tensor(W.sphere_surface(200000, 5), device="cuda").to(dtype)
    B = torch.as_tensor(W.gaussian_mixture(70001, 6), device="cuda").to(dtype)
    ref_a, ref_b = _plan_order(A), _plan_order(B)
    # two calls in a row on different inputs, then the first input again: the shared
    # scratch array must not carry anything over
    assert np.array_equal(_noalloc_order(A), ref_a)
    assert np.array_equal(_noalloc_order(B), ref_b)
    assert np.array_equal(_noalloc_order(A), ref_a)


def test_noalloc_refuses_sizes_beyond_its_scratch():
    X = torch.zeros((ffm.NOALLOC_MAX_POINTS + 1, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    with pytest.raises(ffm.FFMError) as e:
        ffm.morton_order_noalloc(X, out)
    assert e.value.status == 1
    one = torch.zeros((1, 3), dtype=torch.float64, device="cuda")
    o1 = torch.empty(1, dtype=torch.int32, device="cuda")
    ffm.morton_order_noalloc(one, o1)
    torch.cuda.synchronize()
    assert int(o1.item()) == 0
