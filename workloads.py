"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds no arithmetic of the method: it only describes the five
workloads (lattice size, samples, temperatures, replicas, schedule) and draws
seeded Gaussian couplings and arrival streams.  Both the CUDA path and the
CPU oracle receive the arrays it produces.

Couplings stand in for the paper's ~2000 disorder samples per L (App. A.2,
Table A1): i.i.d. N(0,1), drawn in FP64 with numpy's PCG64 and rounded to the
nearest multiple of 2^-18 (clipped to |J| <= 8), which makes every coupling
and every partial sum of six couplings exact in FP32.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict

import numpy as np

GRID = 2.0 ** -18
SEED_BASE = 0x5054485200000000  # "PTHR" << 32


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    n_samples: int
    n_temps: int
    t_min: float = 0.2
    t_max: float = 1.6
    n_replicas: int = 4
    n_res: int = 4
    sweeps_per_emcs: int = 10
    res_sweeps_per_emcs: int = 240
    er_on: bool = True
    cluster: str = "acu"
    acu_interval: int = 1
    res_pretherm_sweeps: int = 0
    budget_emcs: int = 0
    index: int = 0

    @property
    def V(self):
        return self.L ** 3

    @property
    def lattices_per_sample(self):
        return self.n_replicas * (self.n_temps + (self.n_res if self.er_on else 0))

    def updates_per_emcs(self):
        """(PT updates, reservoir updates) per EMCS for the whole batch."""
        pt = self.n_samples * self.n_replicas * self.n_temps * self.sweeps_per_emcs * self.V
        res = (self.n_samples * self.n_replicas * self.n_res * self.res_sweeps_per_emcs * self.V
               if self.er_on else 0)
        return pt, res

    def asdict(self):
        return asdict(self)


# The five workloads.  c1: plain PTHR on one L=4 sample, one local sweep per
# EMCS; c2/c3: batched PT + ACU without the reservoir; c4: the full paper EMCS
# at L=16 (10 sweeps + ACU + PT + ER with 240 reservoir sweeps); c5: serving
# requests of mixed L.
WORKLOADS = {
    "c1": Workload("plain L=4 1x12x4", L=4, n_samples=1, n_temps=12, sweeps_per_emcs=1,
                   budget_emcs=20000, index=1),
    "c2": Workload("batched L=8 256x16x4", L=8, n_samples=256, n_temps=16, sweeps_per_emcs=1,
                   er_on=False, budget_emcs=100000, index=2),
    "c3": Workload("batched L=12 1024x24x4", L=12, n_samples=1024, n_temps=24, sweeps_per_emcs=1,
                   er_on=False, budget_emcs=100000, index=3),
    "c4": Workload("PTHR L=16 512x32x4 +res", L=16, n_samples=512, n_temps=32,
                   sweeps_per_emcs=10, res_sweeps_per_emcs=240, er_on=True,
                   res_pretherm_sweeps=960, budget_emcs=100000, index=4),
    "c5": Workload("serving L in {6,8,10,12,16} 1x24x4 +res", L=16, n_samples=1, n_temps=24,
                   sweeps_per_emcs=10, res_sweeps_per_emcs=240, er_on=True,
                   res_pretherm_sweeps=960, budget_emcs=10000, index=5),
}
SERVE_SIZES = (6, 8, 10, 12, 16)


def batch_seed(index: int) -> int:
    return SEED_BASE + index


def sample_seeds(base: int, n: int) -> np.ndarray:
    """Per-sample Philox keys: base + s."""
    return (np.uint64(base) + np.arange(n, dtype=np.uint64)).astype(np.uint64)


def gaussian_couplings(L: int, n_samples: int, seed: int, on_grid: bool = True) -> np.ndarray:
    """FP32 couplings [S, 3, V]: J[s, mu, i] is the bond (i, i + e_mu)."""
    rng = np.random.Generator(np.random.PCG64(seed & 0xFFFFFFFFFFFFFFFF))
    z = rng.standard_normal((n_samples, 3, L ** 3))
    if on_grid:
        z = np.clip(np.rint(z / GRID) * GRID, -8.0, 8.0)
    return z.astype(np.float32)


def random_spins(shape, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.where(rng.random(shape) < 0.5, 1, -1).astype(np.int8)


def poisson_arrivals(n: int, rate_per_s: float, seed: int, sizes=SERVE_SIZES):
    """Seeded Poisson request stream: (arrival times in s, L of each request)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
    Ls = rng.choice(np.asarray(sizes), size=n)
    return t, Ls.astype(int)
