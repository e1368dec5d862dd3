"""CPU model of the synchronisation of the pipelined tcgen05 kernels (the target-stationary
transfer k_lag_gemm_ts and the plane-wave backward transform k_pw_backward_tc, which share
their constants, and k_pw_forward_tc, two A stages and no accumulator drains): producers, the MMA thread, and the
asynchronous completions of the copies and of the committed MMAs, over random interleavings.  mbarrier waits follow the hardware's parity
rule: a wait for phase k succeeds iff the barrier's completed-phase count has a parity other
than k's, so a barrier two phases ahead of a wait looks incomplete.  The model checks that no
schedule deadlocks and that no wait ever sees its barrier two phases ahead."""
import random

import pytest

NA, DB, DRAIN = 3, 2, 8  # A stages, B copies ahead, steps (translations) per accumulator fill, as in the kernel
NB = NA + DB             # B stages


class Bar:
    def __init__(self, name):
        self.name, self.phase = name, 0

    def arrive(self):  # all arrivals of one phase modelled as one
        self.phase += 1

    def test(self, k):
        ok = (self.phase & 1) != (k & 1)
        assert not ok or self.phase == k + 1, "%s: phase %d seen while waiting for %d" % (self.name, self.phase, k)
        return ok


def run(nsteps, seed, drain_rule, NA=NA, DB=DB, DRAIN=DRAIN):
    NB = NA + DB
    rnd = random.Random(seed)
    bfull = [Bar("bfull%d" % i) for i in range(NB)]
    empty = [Bar("empty%d" % i) for i in range(NB)]
    afull = [Bar("afull%d" % i) for i in range(NA)]
    drained = Bar("drained")
    copies, commits = [], []  # pending completions, each queue in issue order

    def producers():
        n_drained = 0

        def copy_b(sp):
            if sp < nsteps:
                copies.append(bfull[sp % NB])
        for sp in range(DB):
            copy_b(sp)
        for s in range(nsteps):
            if s >= NA:
                sb = s - NA
                while not empty[sb % NB].test(sb // NB):
                    yield
                done = drain_rule(s)
                while n_drained < done:
                    drained.arrive()
                    n_drained += 1
            afull[s % NA].arrive()
            copy_b(s + DB)
            yield
        if nsteps:
            last = nsteps - 1
            while not empty[last % NB].test(last // NB):
                yield
            fills = (nsteps + DRAIN - 1) // DRAIN
            while n_drained < fills:
                drained.arrive()
                n_drained += 1

    def mma():
        for s in range(nsteps):
            fill = s // DRAIN
            if s % DRAIN == 0 and fill >= 2:
                while not drained.test(fill - 2):
                    yield
            while not bfull[s % NB].test(s // NB):
                yield
            while not afull[s % NA].test(s // NA):
                yield
            commits.append(empty[s % NB])
            yield

    live = {"p": producers(), "m": mma()}
    for _ in range(400000):
        if not (live or copies or commits):
            return
        c = rnd.choice(list(live) + (["c"] if copies else []) + (["t"] if commits else []))
        if c == "c":
            copies.pop(0).arrive()
        elif c == "t":
            commits.pop(0).arrive()
        else:
            try:
                next(live[c])
            except StopIteration:
                del live[c]
    raise AssertionError("no progress: deadlock")


KERNEL_RULE = lambda s: (s - NA) // DRAIN  # drain a fill once the next fill's first step is done


@pytest.mark.parametrize("nsteps", [2, 3, 16, 17, 32, 33, 40, 64, 100, 631])
def test_transfer_protocol_never_deadlocks_or_aliases(nsteps):
    for seed in range(10):
        run(nsteps, seed, KERNEL_RULE)


@pytest.mark.parametrize("nsteps", [2, 3, 16, 17, 33, 64, 214])
def test_backward_transform_protocol_never_deadlocks_or_aliases(nsteps):
    for seed in range(10):
        run(nsteps, seed, KERNEL_RULE, NA=3, DB=2)


@pytest.mark.parametrize("nsteps", [1, 2, 3, 5, 8, 9, 31, 214])
def test_forward_transform_protocol_never_deadlocks_or_aliases(nsteps):
    # k_pw_forward_tc: two TMEM operand stages, density copies two steps ahead, one
    # accumulator that is never drained mid-way
    for seed in range(10):
        run(nsteps, seed, lambda s: 0, NA=2, DB=2, DRAIN=1 << 30)


def test_model_catches_a_drain_two_phases_ahead():
    early = lambda s: (s - NA + 1) // DRAIN  # drains as soon as a fill is complete
    with pytest.raises(AssertionError):
        for seed in range(20):
            run(100, seed, early)
