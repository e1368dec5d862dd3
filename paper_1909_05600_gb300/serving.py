"""Continuous-batching server for FFM products on one GPU.

Requests (point sets, kernel, k, eps, densities) arrive over time.  The scheduler admits
them while their estimated device footprint fits the HBM budget and a worker is free;
requests that arrive while others run are admitted as slots and memory free up.  Each
worker owns a CUDA stream, so the plans and applies of different requests overlap on the
device.  Plans are kept resident in an LRU cache keyed by (geometry, kernel, k, eps), and
queued requests that share a plan are merged into one multi-right-hand-side apply.

The scheduling logic (`Scheduler`) is pure Python and testable without a GPU; `Server`
drives it with the C ABI (`ffm.Plan`).
"""
import collections
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    key: tuple              # plan key: (geometry id, kernel, k, eps)
    nx: int
    ny: int
    kind: int
    k: float
    eps: float
    X: object = None
    Y: object = None
    w: object = None
    u: object = None        # (ny,) density
    t_arrival: float = 0.0
    t_admit: float = 0.0
    t_done: float = 0.0
    result: object = None
    error: str = None
    batch: int = 1


def apply_bytes(nx, ny, kind, nrhs=1):
    """Device-memory estimate of the temporaries of one apply: w u in Morton order, the FP64
    accumulators and the per-level coefficient arrays (~96 B per point per right-hand side
    for Helmholtz, ~24 B for Laplace), plus a fixed allowance."""
    n = nx + ny
    return (16 << 20) + (96 if kind == 1 else 24) * n * nrhs


def footprint_bytes(nx, ny, kind, nrhs=1):
    """Conservative device-memory estimate of one plan plus one apply, for a plan that does
    not exist yet.  The plan holds ~160 B per point (keys, permutation, hi/lo coordinates,
    box tables, pair lists, operators); once it is built, ffm_plan_bytes gives the real
    figure (Server corrects its reservation with it)."""
    return 160 * (nx + ny) + (48 << 20) + apply_bytes(nx, ny, kind, nrhs)


class Scheduler:
    """FIFO admission by memory footprint and free workers, with batching of queued
    requests that share a plan key (up to max_batch right-hand sides).

    footprint(req, nrhs) gives the bytes a batch of nrhs requests like req needs; by default
    the plan-plus-apply estimate.  A server that keeps plans resident passes one that counts
    only the apply for a resident plan, and corrects reservations with adjust() once a new
    plan's real size is known."""

    def __init__(self, budget_bytes, workers, max_batch=16, footprint=None):
        self.budget = budget_bytes
        self.workers = workers
        self.max_batch = max_batch
        self.footprint = footprint or (lambda req, nrhs: footprint_bytes(req.nx, req.ny, req.kind, nrhs))
        self.queue = collections.deque()
        self.in_use = 0
        self.busy = 0
        self.lock = threading.Lock()
        self.rejected = []

    def submit(self, req):
        with self.lock:
            need = footprint_bytes(req.nx, req.ny, req.kind)
            if need > self.budget:
                req.error = "request needs %d bytes, above the whole budget of %d" % (need, self.budget)
                self.rejected.append(req)
                return False
            self.queue.append(req)
            return True

    def next_batch(self):
        """Pop the head request and queued requests with the same plan key, if a worker is
        free and their footprint fits; returns (batch, reserved bytes) or (None, 0)."""
        with self.lock:
            if not self.queue or self.busy >= self.workers:
                return None, 0
            head = self.queue[0]
            batch = [head]
            for r in list(self.queue)[1:]:
                if len(batch) >= self.max_batch:
                    break
                if r.key == head.key:
                    batch.append(r)
            # the largest prefix of the batch that fits (at least the head, which submit()
            # checked against the whole budget): a merged batch too large for the free
            # memory must not hold back a head that fits alone
            while True:
                need = self.footprint(head, len(batch))
                if self.in_use + need <= self.budget or len(batch) == 1:
                    break
                batch.pop()
            if self.in_use + need > self.budget:
                return None, 0
            for r in batch:
                self.queue.remove(r)
            self.in_use += need
            self.busy += 1
            return batch, need

    def adjust(self, old, new):
        """Replace a running batch's reservation of `old` bytes by `new` (the real size of
        its plan is known once built); returns new."""
        with self.lock:
            self.in_use += new - old
            return new

    def release(self, need):
        with self.lock:
            self.in_use -= need
            self.busy -= 1


class PlanCache:
    """LRU cache of resident plans, bounded in device bytes.  Plans are reference counted:
    an evicted plan is closed only once no worker is still applying it (its buffers may be
    in use on another stream until that worker has synchronised)."""

    def __init__(self, capacity_bytes):
        self.capacity = capacity_bytes
        self.plans = collections.OrderedDict()  # key -> [plan, bytes, refs]
        self.retired = []                       # evicted, still referenced: [plan, bytes, refs]
        self.bytes = 0
        self.lock = threading.Lock()
        self.hits = 0
        self.misses = 0

    def resident(self, key):
        """True if a plan for key is cached (its bytes are already on the device)."""
        with self.lock:
            return key in self.plans

    def acquire(self, key, build):
        with self.lock:
            if key in self.plans:
                self.plans.move_to_end(key)
                self.plans[key][2] += 1
                self.hits += 1
                return self.plans[key][0]
            self.misses += 1
        plan = build()
        nb = plan.bytes()
        with self.lock:
            if key in self.plans:  # built concurrently by another worker
                self.plans[key][2] += 1
                keep = self.plans[key][0]
                plan.close()
                return keep
            self.plans[key] = [plan, nb, 1]
            self.bytes += nb
            self._evict()
        return plan

    def release(self, plan):
        close = []
        with self.lock:
            for ent in self.plans.values():
                if ent[0] is plan:
                    ent[2] -= 1
                    break
            else:
                for ent in self.retired:
                    if ent[0] is plan:
                        ent[2] -= 1
                        if ent[2] == 0:
                            close.append(ent)
                for ent in close:
                    self.retired.remove(ent)
            self._evict()
        for ent in close:
            ent[0].close()

    def _evict(self):
        # caller holds the lock
        while self.bytes > self.capacity and len(self.plans) > 1:
            key = next(iter(self.plans))
            ent = self.plans.pop(key)
            self.bytes -= ent[1]
            if ent[2] == 0:
                ent[0].close()
            else:
                self.retired.append(ent)

    def clear(self):
        with self.lock:
            for ent in list(self.plans.values()) + self.retired:
                ent[0].close()
            self.plans.clear()
            self.retired.clear()
            self.bytes = 0


class Server:
    """Workers with one CUDA stream each pull admitted batches from the scheduler."""

    def __init__(self, device=0, workers=4, budget_bytes=None, max_batch=16, plan_cache_bytes=None):
        import torch
        from . import ffm
        self.torch = torch
        self.ffm = ffm
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        free, _ = torch.cuda.mem_get_info(self.device)
        self.budget = budget_bytes if budget_bytes is not None else int(0.5 * free)
        self.cache = PlanCache(plan_cache_bytes if plan_cache_bytes is not None else int(0.25 * free))
        self.sched = Scheduler(self.budget, workers, max_batch, footprint=self._footprint)
        self.device_ms = 0.0  # summed device time of the batches (CUDA events on each worker stream)
        self.batches = 0
        self.streams = [torch.cuda.Stream(self.device) for _ in range(workers)]
        self.done = []
        self.done_lock = threading.Lock()
        self.stop = False
        self.threads = [threading.Thread(target=self._worker, args=(i,), daemon=True) for i in range(workers)]
        self.wake = threading.Condition()
        for t in self.threads:
            t.start()

    def submit(self, req):
        req.t_arrival = req.t_arrival or time.perf_counter()
        ok = self.sched.submit(req)
        if not ok:
            with self.done_lock:
                self.done.append(req)
        with self.wake:
            self.wake.notify_all()

    def _footprint(self, req, nrhs):
        # a resident plan costs only its apply; a new one the estimate until it is built
        if self.cache.resident(req.key):
            return apply_bytes(req.nx, req.ny, req.kind, nrhs)
        return footprint_bytes(req.nx, req.ny, req.kind, nrhs)

    def _run_batch(self, batch, stream, res):
        """Plan (or cached plan) and one apply of the batch on the worker's stream.  res[0] is
        the batch's reservation; it is corrected to the plan's ffm_plan_bytes (plus the apply)
        if the plan was built here."""
        torch, ffm = self.torch, self.ffm
        head = batch[0]
        built = []
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            def build():
                built.append(1)
                return ffm.Plan(head.X, head.Y, head.kind, head.k, head.eps, weights=head.w, stream=stream)
            ev0.record(stream)
            plan = self.cache.acquire(head.key, build)
            try:
                if built:
                    res[0] = self.sched.adjust(res[0], plan.bytes() + apply_bytes(head.nx, head.ny, head.kind,
                                                                                  len(batch)))
                if len(batch) == 1:
                    U = head.u
                else:
                    U = torch.stack([r.u for r in batch], 0)
                V = plan.apply(U, stream=stream)
                ev1.record(stream)
                stream.synchronize()
            finally:
                self.cache.release(plan)
        t = time.perf_counter()
        ms = ev0.elapsed_time(ev1)
        with self.done_lock:
            self.device_ms += ms
            self.batches += 1
        for i, r in enumerate(batch):
            r.result = V if len(batch) == 1 else V[i]
            r.t_done = t
            r.batch = len(batch)

    def _worker(self, i):
        stream = self.streams[i]
        torch = self.torch
        torch.cuda.set_device(self.device)
        while True:
            with self.wake:
                batch, need = self.sched.next_batch()
                while batch is None and not self.stop:
                    self.wake.wait(0.002)
                    batch, need = self.sched.next_batch()
                if batch is None and self.stop:
                    return
            t0 = time.perf_counter()
            for r in batch:
                r.t_admit = t0
            res = [need]
            try:
                self._run_batch(batch, stream, res)
            except Exception as e:  # report, keep serving
                for r in batch:
                    r.error = str(e)
                    r.t_done = time.perf_counter()
            finally:
                self.sched.release(res[0])
                with self.done_lock:
                    self.done.extend(batch)
                with self.wake:
                    self.wake.notify_all()

    def drain(self, n_expected, timeout=600.0):
        t_end = time.perf_counter() + timeout
        while True:
            with self.done_lock:
                if len(self.done) >= n_expected:
                    return
            if time.perf_counter() > t_end:
                raise TimeoutError("serving did not finish within %.0f s" % timeout)
            time.sleep(0.002)

    def close(self):
        self.stop = True
        with self.wake:
            self.wake.notify_all()
        for t in self.threads:
            t.join(timeout=30)
        self.cache.clear()


def latency_stats(reqs):
    ok = [r for r in reqs if r.error is None]
    lat = np.array([1e3 * (r.t_done - r.t_arrival) for r in ok])
    if not len(lat):
        return {"completed": 0}
    t0 = min(r.t_arrival for r in ok)
    t1 = max(r.t_done for r in ok)
    return {"completed": len(ok), "failed": len(reqs) - len(ok), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "throughput_rps": len(ok) / (t1 - t0), "wall_s": t1 - t0,
            "mean_batch": float(np.mean([r.batch for r in ok]))}
