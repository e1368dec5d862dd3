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


def test_noalloc_warm_call_allocates_nothing():
    """Once the first call on the device has resolved the scratch address, a call must leave
    the device's free memory exactly as it found it (no cudaMalloc, no allocating library
    call, no lazily created buffer)."""
    X = torch.as_tensor(W.gaussian_mixture(100000, 9), device="cuda")
    out = torch.empty(X.shape[0], dtype=torch.int32, device="cuda")
    ffm.morton_order_noalloc(X, out)  # warm: address resolution and module loading
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for _ in range(3):
        ffm.morton_order_noalloc(X, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    assert stats1.get("allocation.all.allocated", 0) == stats0.get("allocation.all.allocated", 0)


def test_noalloc_non_finite_coordinates_poison_the_output():
    """A NaN or an infinite coordinate (refused by ffm_plan) sets every entry to 0xFFFFFFFF;
    the next call on finite input, which reuses the shared scratch, is unaffected."""
    Xn = W.sphere_surface(5000, 11)
    good = torch.as_tensor(Xn, device="cuda")
    for bad_value in (float("nan"), float("inf")):
        Xb = Xn.copy()
        Xb[1234, 1] = bad_value
        bad = torch.as_tensor(Xb, device="cuda")
        assert np.all(_noalloc_order(bad) == 0xFFFFFFFF)
        assert np.array_equal(_noalloc_order(good), _plan_order(good))


def test_noalloc_wrapper_checks_its_arguments():
    X = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ffm.morton_order_noalloc(X, torch.empty(10, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        ffm.morton_order_noalloc(X, torch.empty(9, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        ffm.morton_order_noalloc(X[:, :2].contiguous(), torch.empty(10, dtype=torch.int32, device="cuda"))
