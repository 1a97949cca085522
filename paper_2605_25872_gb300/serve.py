"""Continuous-batching request loop for PTHR samples of mixed lattice size.

A request is one disorder sample (couplings, seed, lattice size L) that needs
a fixed budget of EMCS.  The server keeps one resident batch ("pool") per
lattice size, each on its own CUDA stream.  It admits waiting requests into
free slots whenever a slot frees up (by device memory: the pools are sized
from a memory budget).  It advances every pool that has work in chunks of
EMCS that end exactly when the next request of that pool finishes, so pools
overlap on the device and the host meets a pool once per chunk.  It reads a
request's observables back when its budget is done, then frees the slot.

Because every random number is keyed by the request's own seed and
EMCS counter, a request's result is the same whether it runs alone or in a
busy pool; the tests check this bit for bit.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    L: int
    seed: int
    budget_emcs: int
    arrival: float = 0.0                  # seconds since the start of the run
    couplings: np.ndarray | None = None   # FP32 [3, V]; None: drawn on the device from seed
    # filled by the server
    admitted: float | None = None
    finished: float | None = None
    obs: np.ndarray | None = None         # accumulators [n_temps, 8]
    round_trips: np.ndarray | None = None
    cancelled: bool = False               # withdrawn before its budget was done

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


@dataclass
class PoolSpec:
    L: int
    slots: int
    n_temps: int = 24
    t_min: float = 0.2
    t_max: float = 1.6
    n_replicas: int = 4
    n_res: int = 4
    sweeps_per_emcs: int = 10
    res_sweeps_per_emcs: int = 240
    pretherm_sweeps: int = 960
    spin_layout: str = "bytes"      # "bits": 8x less spin memory per slot
    tuning: dict | None = None      # kernel shape (Batch.set_tuning), e.g. the autotuner's

    def updates_per_emcs_per_sample(self):
        V = self.L ** 3
        return self.n_replicas * (self.n_temps * self.sweeps_per_emcs
                                  + self.n_res * self.res_sweeps_per_emcs) * V


class GpuPool:
    """One resident batch of `spec.slots` samples of one lattice size."""

    def __init__(self, spec: PoolSpec, device="cuda", graph=True):
        import torch
        from .batch import Batch
        self.spec = spec
        self.stream = torch.cuda.Stream(device)
        self.cfg = self.config_of(spec)
        self.batch = Batch(self.cfg, device=device, stream=self.stream)
        if spec.tuning:
            self.batch.set_tuning(**spec.tuning)
        self.batch.set_active(0, spec.slots, False)
        self.graph = graph
        self.event = torch.cuda.Event()

    @staticmethod
    def config_of(spec: PoolSpec):
        """The batch configuration of a pool."""
        from .batch import BatchConfig
        return BatchConfig(L=spec.L, n_samples=spec.slots, n_temps=spec.n_temps,
                           t_min=spec.t_min, t_max=spec.t_max, n_replicas=spec.n_replicas,
                           n_res=spec.n_res, sweeps_per_emcs=spec.sweeps_per_emcs,
                           res_sweeps_per_emcs=spec.res_sweeps_per_emcs,
                           er_on=spec.n_res > 0, cluster="acu", spin_layout=spec.spin_layout)

    def reset(self, slot, req: Request):
        self.reset_many([slot], [req])

    def reset_many(self, slots, reqs):
        """Admit requests into slots; consecutive slots whose couplings are all
        given (or all drawn from seeds) share one call, so their reservoir
        pre-thermalisation runs as one launch."""
        order = sorted(range(len(slots)), key=lambda i: slots[i])
        run = []

        def flush():
            if not run:
                return
            first = slots[run[0]]
            seeds = [reqs[i].seed for i in run]
            cpl = None
            if reqs[run[0]].couplings is not None:
                cpl = np.ascontiguousarray(np.stack([reqs[i].couplings for i in run]), np.float32)
            self.batch.reset_samples(first, len(run), seeds=seeds, couplings=cpl,
                                     pretherm_sweeps=self.spec.pretherm_sweeps)
            run.clear()

        for i in order:
            if run and (slots[i] != slots[run[-1]] + 1
                        or (reqs[i].couplings is None) != (reqs[run[0]].couplings is None)):
                flush()
            run.append(i)
        flush()

    def step(self, n=1):
        """Enqueue n EMCS of every active slot; returns at once."""
        self.batch.emcs(n, graph=self.graph)
        self.event.record(self.stream)

    def ready(self):
        return self.event.query()

    def wait(self):
        self.stream.synchronize()

    def read(self, slot):
        with torch_stream(self.stream):
            obs = self.batch.obs[slot].cpu().numpy().copy()
            trips = self.batch.round_trips[slot].cpu().numpy().copy()
        return obs, trips

    def free(self, slot):
        self.batch.set_active(slot, 1, False)


def torch_stream(stream):
    import torch
    return torch.cuda.stream(stream)


class Server:
    """Admission queue -> slots -> chunks of EMCS -> completion -> readback.

    Each pool advances in chunks: k EMCS enqueued at once on its stream, k
    the smallest remaining budget among its busy slots (at most max_chunk),
    so no request runs past its budget and the host meets the device once
    per chunk rather than once per EMCS.  While a chunk runs the host admits
    arrivals into free slots (stream-ordered after the chunk) and services
    the pools whose chunk has finished; pools on different streams overlap
    on the device."""

    def __init__(self, specs, pool_factory=None, clock=None, max_chunk=64, max_queue=None):
        self.specs = {s.L: s for s in specs}
        self.max_queue = max_queue          # waiting requests per lattice size; None: unbounded
        self.refused = []
        self.cancelled = []
        self.cancel_requests = deque()      # rids to withdraw, applied by the run loop
        self.pool_factory = pool_factory or (lambda spec: GpuPool(spec))
        self.max_chunk = max(1, int(max_chunk))
        self.pools = {L: self.pool_factory(s) for L, s in self.specs.items()}
        self.slot_req = {L: [None] * s.slots for L, s in self.specs.items()}
        self.remaining = {L: np.zeros(s.slots, dtype=np.int64) for L, s in self.specs.items()}
        self.in_flight = {L: False for L in self.specs}
        self.queue = {L: deque() for L in self.specs}
        self.done = []
        self.clock = clock or time.perf_counter
        self.t0 = None
        self.emcs_steps = {L: 0 for L in self.specs}
        self.chunks = {L: 0 for L in self.specs}

    def now(self):
        return self.clock() - self.t0

    def submit(self, req: Request) -> bool:
        """Queue a request; False (refused, nothing queued) when its size's
        queue already holds max_queue requests."""
        if req.L not in self.specs:
            raise ValueError(f"no pool for L={req.L}")
        if self.max_queue is not None and len(self.queue[req.L]) >= self.max_queue:
            self.refused.append(req)
            return False
        self.queue[req.L].append(req)
        return True

    def cancel(self, rid: int) -> bool:
        """Withdraw request rid.  A waiting request leaves its queue at once;
        a running one is marked and its slot is freed the next time its pool
        has no chunk in flight (the chunk already queued still advances it;
        its result is discarded).  False if rid is neither waiting nor
        running."""
        for L, q in self.queue.items():
            for req in q:
                if req.rid == rid:
                    q.remove(req)
                    req.cancelled = True
                    req.finished = self.now() if self.t0 is not None else None
                    self.cancelled.append(req)
                    return True
        for slots in self.slot_req.values():
            for req in slots:
                if req is not None and req.rid == rid and not req.cancelled:
                    req.cancelled = True
                    return True
        return False

    def request_cancel(self, rid: int):
        """cancel(rid) from another thread: applied by the run loop."""
        self.cancel_requests.append(rid)

    def _admit(self, L):
        q = self.queue[L]
        slots = self.slot_req[L]
        free = [i for i, r in enumerate(slots) if r is None]
        take = []
        while q and free:
            take.append((free.pop(0), q.popleft()))
        if not take:
            return
        pool = self.pools[L]
        if hasattr(pool, "reset_many"):
            pool.reset_many([s for s, _ in take], [r for _, r in take])
        else:
            for s, r in take:
                pool.reset(s, r)
        t = self.now()
        for slot, req in take:
            req.admitted = t
            slots[slot] = req
            self.remaining[L][slot] = req.budget_emcs

    def _complete(self, L):
        """Read back and free the slots whose budget is done, and free the
        cancelled ones (pool L idle)."""
        pool, rem = self.pools[L], self.remaining[L]
        for slot, req in enumerate(self.slot_req[L]):
            if req is not None and req.cancelled:
                req.finished = self.now()
                pool.free(slot)
                self.slot_req[L][slot] = None
                rem[slot] = 0
                self.cancelled.append(req)
            elif req is not None and rem[slot] == 0:
                req.obs, req.round_trips = pool.read(slot)
                req.finished = self.now()
                pool.free(slot)
                self.slot_req[L][slot] = None
                self.done.append(req)

    def _enqueue_chunk(self, L):
        rem = self.remaining[L]
        busy = [slot for slot, r in enumerate(self.slot_req[L]) if r is not None]
        if not busy:
            self.in_flight[L] = False
            return
        k = int(min(self.max_chunk, min(rem[s] for s in busy)))
        self.pools[L].step(k)
        for s in busy:
            rem[s] -= k
        self.in_flight[L] = True
        self.emcs_steps[L] += k
        self.chunks[L] += 1

    def _service(self, L):
        """Pool L has no chunk in flight: complete, admit, enqueue the next."""
        self._complete(L)
        self._admit(L)
        self._enqueue_chunk(L)

    def fill_and_time(self, requests, n_emcs):
        """Capacity probe: admit `requests` (filling the pools), then time
        n_emcs EMCS of every busy pool, all pools in flight together
        (admission excluded).  Returns seconds per full-pool EMCS."""
        self.t0 = self.clock()
        for r in requests:
            self.submit(r)
        for L in self.pools:
            self._admit(L)
        for p in self.pools.values():
            p.wait()
        t0 = self.clock()
        for L, p in self.pools.items():
            if any(r is not None for r in self.slot_req[L]):
                p.step(n_emcs)
        for p in self.pools.values():
            p.wait()
        return (self.clock() - t0) / n_emcs

    def busy(self):
        return any(self.in_flight.values()) or any(
            r is not None for sl in self.slot_req.values() for r in sl)

    def run(self, requests, realtime=True):
        """Serve `requests` (sorted by arrival).  With realtime=True arrivals
        follow the wall clock; otherwise every request is queued at once."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        self.t0 = self.clock()
        while pending or self.busy() or any(self.queue.values()):
            now = self.now()
            while pending and (not realtime or pending[0].arrival <= now):
                self.submit(pending.popleft())
            while self.cancel_requests:
                self.cancel(self.cancel_requests.popleft())
            progressed = False
            for L, pool in self.pools.items():
                if self.in_flight[L]:
                    if not pool.ready():
                        self._admit(L)          # into free slots, after the chunk
                        continue
                    self._service(L)
                    progressed = True
                elif self.queue[L] or any(r is not None for r in self.slot_req[L]):
                    self._service(L)
                    progressed = True
            if not progressed:
                nxt = pending[0].arrival - self.now() if (pending and realtime) else 0.0
                time.sleep(max(0.0002, min(0.001, nxt)))
        return self.done

    def stats(self):
        lat = np.array([r.latency for r in self.done])
        upd = sum(self.specs[r.L].updates_per_emcs_per_sample() * r.budget_emcs for r in self.done)
        span = max(r.finished for r in self.done) if self.done else 0.0
        return {"requests": len(self.done),
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "makespan_s": span,
                "updates_per_ns": upd / (span * 1e9) if span > 0 else None,
                "emcs_steps": dict(self.emcs_steps), "chunks": dict(self.chunks),
                "refused": len(self.refused), "cancelled": len(self.cancelled)}
