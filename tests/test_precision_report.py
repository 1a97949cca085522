"""Precision report: FP32 local fields / acceptance vs the FP64 oracle.

Prints one line "PRECISION_REPORT {json}" (run with -s) and asserts the
bounds the design states:
  * couplings on the 2^-18 grid: per-observable accumulators (e, e^2, q,
    q^2, q_l, S, q^4) equal the oracle's bit for bit between near ties; the
    fraction of decisions within 1e-6 of their threshold (near ties) and the
    fraction that actually changed the trajectory are reported per
    decision; both stay below 1e-5;
  * energies (double-FP32 exact pairs + FP64 combination on the GPU) vs FP64:
    exactly equal on the grid, relative error < 1e-12 off the grid.
"""
import json

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from mirror import Mirror

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


FIELDS = ("n", "e", "e2", "q", "q2", "ql", "S", "q4")


def trajectory_stats(cfg, n_emcs, seed):
    J = W.gaussian_couplings(cfg.L, cfg.n_samples, seed)
    seeds = W.sample_seeds(W.SEED_BASE + seed, cfg.n_samples)
    gpu = Batch(cfg, couplings=J, seeds=seeds)
    mir = Mirror(cfg, J, seeds)
    near_ties = 0
    diverged = 0
    max_abs = {f: 0.0 for f in FIELDS}
    for _ in range(n_emcs):
        gpu.emcs(1)
        ties, pt_ties = mir.emcs()
        near_ties += sum(len(v) for v in ties.values()) + sum(pt_ties.values())
        g = gpu.export_spins().cpu().numpy()
        if not (np.array_equal(g, mir.spins()) and np.array_equal(gpu.perm.cpu().numpy(), mir.perms())):
            diverged += 1
            gpu.perm.copy_(torch.from_numpy(mir.perms().astype(np.int32)))
            if cfg.n_res:
                gpu.age.copy_(torch.from_numpy(mir.ages().astype(np.int32)))
            gpu.rt_state.copy_(torch.from_numpy(np.stack([s.rt_state for s in mir.samples])))
            gpu.import_spins(torch.from_numpy(mir.spins()))
            gpu.obs.copy_(torch.from_numpy(np.stack([s.obs for s in mir.samples])))
            continue
        d = np.abs(gpu.obs.cpu().numpy() - np.stack([s.obs for s in mir.samples]))
        for i, f in enumerate(FIELDS):
            max_abs[f] = max(max_abs[f], float(d[..., i].max()))
    return mir.decisions, near_ties, diverged, max_abs


def energy_errors(on_grid):
    cfg = BatchConfig(L=12, n_samples=4, n_temps=4, n_replicas=2, n_res=1)
    J = W.gaussian_couplings(cfg.L, cfg.n_samples, 77, on_grid=on_grid)
    gpu = Batch(cfg, couplings=J, seeds=W.sample_seeds(5, cfg.n_samples))
    spins = W.random_spins((cfg.n_samples, cfg.n_lat, cfg.V), 12)
    gpu.import_spins(torch.from_numpy(spins))
    Eg = gpu.energies.cpu().numpy()
    Eo = np.array([[O.energy(cfg.L, J[s].astype(np.float64), spins[s, l]) for l in range(cfg.n_lat)]
                   for s in range(cfg.n_samples)])
    return float(np.max(np.abs(Eg - Eo) / np.maximum(np.abs(Eo), 1.0)))


def test_precision_report():
    cfg = BatchConfig(L=8, n_samples=8, n_temps=16, n_replicas=4, n_res=4, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=8)
    decisions, near, div, max_abs = trajectory_stats(cfg, 60, seed=31)
    rel_grid = energy_errors(True)
    rel_off = energy_errors(False)
    report = {"decisions": decisions, "near_ties": near, "near_tie_rate": near / decisions,
              "diverged_emcs": div, "diverged_rate_per_decision": div / decisions,
              "observable_max_abs_diff": max_abs,
              "energy_rel_err_grid": rel_grid, "energy_rel_err_offgrid": rel_off}
    print("PRECISION_REPORT " + json.dumps(report))
    assert near / decisions < 1e-5
    assert div / decisions < 1e-5
    assert all(v == 0.0 for v in max_abs.values())
    assert rel_grid == 0.0
    assert rel_off < 1e-12
