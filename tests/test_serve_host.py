"""Host logic of the serving loop (no GPU): admission by free slots,
continuous batching, completion accounting, FIFO order per lattice size."""
import numpy as np
import pytest

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
        self.log.append(("free", slot))


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


def test_admission_is_refused_when_the_queue_is_full():
    srv = Server([PoolSpec(L=6, slots=1)], pool_factory=FakePool, max_queue=2)
    ok = [srv.submit(Request(rid=i, L=6, seed=i, budget_emcs=2)) for i in range(4)]
    assert ok == [True, True, False, False]
    assert [r.rid for r in srv.refused] == [2, 3]
    done = srv.run([], realtime=False)
    assert sorted(r.rid for r in done) == [0, 1]
    assert srv.stats()["refused"] == 2


def test_cancel_a_waiting_and_a_running_request():
    srv = Server([PoolSpec(L=6, slots=1)], pool_factory=FakePool, max_chunk=4)
    srv.t0 = srv.clock()
    for i, budget in enumerate((10, 3, 3)):
        srv.submit(Request(rid=i, L=6, seed=i, budget_emcs=budget))
    assert srv.cancel(2)                     # still waiting: leaves the queue
    assert [r.rid for r in srv.queue[6]] == [0, 1]
    srv._service(6)                          # admits rid 0, enqueues a chunk of 4
    assert srv.slot_req[6][0].rid == 0
    assert srv.cancel(0)                     # running: freed at the next service point
    srv._service(6)                          # frees slot 0, admits rid 1
    assert srv.slot_req[6][0].rid == 1
    done = srv.run([], realtime=False)
    assert [r.rid for r in done] == [1] and done[0].obs[0][1] == 3
    assert sorted(r.rid for r in srv.cancelled) == [0, 2] and all(r.cancelled for r in srv.cancelled)
    assert not srv.cancel(1) and not srv.cancel(7)
    assert srv.stats()["cancelled"] == 2


def test_cancel_requested_from_outside_the_loop():
    srv = Server([PoolSpec(L=6, slots=2)], pool_factory=FakePool)
    reqs = [Request(rid=i, L=6, seed=i, budget_emcs=5) for i in range(3)]
    srv.request_cancel(1)
    done = srv.run(reqs, realtime=False)
    assert sorted(r.rid for r in done) == [0, 2]
    assert [r.rid for r in srv.cancelled] == [1]


@pytest.mark.parametrize("seed", range(6))
def test_random_streams_keep_the_serving_invariants(seed):
    """Random arrivals, budgets, queue bounds and cancellations against the fake
    pool: a finished request ran exactly its budget on its own slot state, no
    slot ever holds two requests, cancelled and refused requests never finish,
    and every request ends in exactly one of done / cancelled / refused."""
    import numpy as np
    rng = np.random.default_rng(seed)
    specs = [PoolSpec(L=6, slots=int(rng.integers(1, 4))), PoolSpec(L=8, slots=int(rng.integers(1, 3)))]
    srv = Server(specs, pool_factory=FakePool, max_chunk=int(rng.integers(1, 9)),
                 max_queue=int(rng.integers(2, 8)))
    reqs = [Request(rid=i, L=int(rng.choice([6, 8])), seed=1000 + i, budget_emcs=int(rng.integers(1, 20)))
            for i in range(40)]
    for rid in rng.choice(40, size=8, replace=False):
        srv.request_cancel(int(rid))
    done = srv.run(reqs, realtime=False)
    ids_done = {r.rid for r in done}
    ids_cancel = {r.rid for r in srv.cancelled}
    ids_refused = {r.rid for r in srv.refused}
    assert ids_done | ids_cancel | ids_refused == set(range(40))
    assert not (ids_done & ids_cancel) and not (ids_done & ids_refused) and not (ids_cancel & ids_refused)
    for r in done:
        seed_v, emcs = r.obs[0]
        assert seed_v == r.seed and emcs == r.budget_emcs and not r.cancelled
    for L, pool in srv.pools.items():
        live = set()
        for ev in pool.log:
            if ev[0] == "reset":
                assert ev[1] not in live
                live.add(ev[1])
            elif ev[0] == "free":
                live.discard(ev[1])
    st = srv.stats()
    assert st["requests"] == len(done) and st["cancelled"] == len(ids_cancel) and st["refused"] == len(ids_refused)
