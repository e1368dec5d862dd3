"""Host-side logic of the continuous-batching server (no GPU): admission by memory
footprint and free workers, FIFO order, batching of requests that share a plan, rejection
of requests larger than the whole budget, and the reference-counted plan cache."""
from paper_1909_05600_gb300.serving import PlanCache, Request, Scheduler, footprint_bytes


def req(i, key, n=10000, kind=0):
    return Request(rid=i, key=key, nx=n, ny=n, kind=kind, k=0.0, eps=1e-3)


def test_fifo_admission_and_batching_by_plan_key():
    s = Scheduler(budget_bytes=10 << 30, workers=2, max_batch=3)
    for i, key in enumerate(["a", "b", "a", "a", "a", "c"]):
        assert s.submit(req(i, key))
    b1, n1 = s.next_batch()
    assert [r.rid for r in b1] == [0, 2, 3]          # head plus queued requests with the same key, max 3
    b2, n2 = s.next_batch()
    assert [r.rid for r in b2] == [1]
    assert s.next_batch() == (None, 0)                # both workers busy
    s.release(n1)
    b3, _ = s.next_batch()
    assert [r.rid for r in b3] == [4]
    assert n1 == footprint_bytes(10000, 10000, 0, 3)


def test_admission_waits_for_memory_and_rejects_oversize():
    one = footprint_bytes(100000, 100000, 1)
    s = Scheduler(budget_bytes=int(1.5 * one), workers=4)
    assert s.submit(req(0, "x", 100000, 1))
    assert s.submit(req(1, "y", 100000, 1))
    assert not s.submit(req(2, "z", 10_000_000, 1))   # larger than the whole budget
    assert s.rejected[0].error
    b, n = s.next_batch()
    assert b is not None
    assert s.next_batch() == (None, 0)                 # second request waits for memory
    s.release(n)
    b, _ = s.next_batch()
    assert [r.rid for r in b] == [1]


class FakePlan:
    def __init__(self, nbytes):
        self.nbytes = nbytes
        self.closed = False

    def bytes(self):
        return self.nbytes

    def close(self):
        self.closed = True


def test_plan_cache_lru_and_deferred_close():
    c = PlanCache(capacity_bytes=250)
    p1 = c.acquire("a", lambda: FakePlan(100))
    p2 = c.acquire("b", lambda: FakePlan(100))
    c.release(p2)
    assert c.acquire("a", lambda: FakePlan(100)) is p1 and c.hits == 1
    c.release(p1)
    c.release(p1)
    p3 = c.acquire("c", lambda: FakePlan(100))         # evicts the LRU plan "b" (unused): closed now
    assert p2.closed and not p1.closed
    c.acquire("a", lambda: FakePlan(100))              # a in use again
    p4 = c.acquire("d", lambda: FakePlan(100))         # evicts "c" (in use): closed only on release
    assert not p3.closed
    c.release(p3)
    assert p3.closed
    c.release(p4)
    c.clear()
    assert p1.closed and p4.closed


def test_merged_batch_too_large_still_admits_the_head():
    """A budget that fits one right-hand side but not the merged batch: the head (and as
    many same-key requests as fit) must be admitted, not held back forever."""
    one = footprint_bytes(1_000_000, 1_000_000, 1, 1)
    two = footprint_bytes(1_000_000, 1_000_000, 1, 2)
    s = Scheduler(budget_bytes=(one + two) // 2, workers=4, max_batch=16)
    for i in range(6):
        assert s.submit(req(i, "same", 1_000_000, 1))
    b, n = s.next_batch()
    assert b is not None and [r.rid for r in b] == [0] and n == one
    s.release(n)
    s2 = Scheduler(budget_bytes=footprint_bytes(1_000_000, 1_000_000, 1, 3), workers=4, max_batch=16)
    for i in range(6):
        s2.submit(req(i, "same", 1_000_000, 1))
    b, n = s2.next_batch()
    assert [r.rid for r in b] == [0, 1, 2]           # the largest prefix that fits


def test_resident_plans_cost_only_their_apply_and_reservations_follow_real_plan_bytes():
    from paper_1909_05600_gb300.serving import apply_bytes
    resident = {"hot"}
    fp = lambda r, nrhs: (apply_bytes(r.nx, r.ny, r.kind, nrhs) if r.key in resident
                          else footprint_bytes(r.nx, r.ny, r.kind, nrhs))
    budget = footprint_bytes(500_000, 500_000, 0, 1) + apply_bytes(500_000, 500_000, 0, 1)
    s = Scheduler(budget_bytes=budget, workers=4, footprint=fp)
    s.submit(req(0, "cold", 500_000))
    s.submit(req(1, "hot", 500_000))
    b0, n0 = s.next_batch()
    b1, n1 = s.next_batch()                           # fits beside the cold plan: apply only
    assert [r.rid for r in b0] == [0] and [r.rid for r in b1] == [1]
    assert n1 == apply_bytes(500_000, 500_000, 0, 1)
    real = s.adjust(n0, 12345)                        # the cold plan's real size once built
    assert s.in_use == real + n1
    s.release(real)
    s.release(n1)
    assert s.in_use == 0 and s.busy == 0
