"""Scenarios run under both builds of the CUDA library (release and the
range-checked PTHR_DEBUG build): every step of the EMCS at several lattice
sizes, both cluster moves, heat bath, MicSA, both spin layouts,
pre-thermalisation and labels.

Run as a script (python tests/debug_build_scenarios.py OUT.npz) it executes
the scenarios in this process with whatever library PTHR_LIBRARY names and
saves every result plus each batch's poll status."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

SCENARIOS = [
    dict(L=4, n_samples=2, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2, res_sweeps_per_emcs=4),
    dict(L=6, n_samples=3, n_temps=8, n_replicas=4, n_res=3, sweeps_per_emcs=1, res_sweeps_per_emcs=3,
         cluster="single"),
    dict(L=8, n_samples=2, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2, res_sweeps_per_emcs=2,
         rule="heatbath"),
    dict(L=12, n_samples=2, n_temps=6, n_replicas=4, n_res=0, er_on=False, sweeps_per_emcs=1),
    dict(L=16, n_samples=2, n_temps=4, n_replicas=4, n_res=2, sweeps_per_emcs=2, res_sweeps_per_emcs=4),
    # bit spin storage, padded rows (L = 12) and full rows (L = 8)
    dict(L=12, n_samples=2, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=1, res_sweeps_per_emcs=3,
         spin_layout="bits"),
    dict(L=8, n_samples=2, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2, res_sweeps_per_emcs=2,
         rule="micsa", spin_layout="bits"),
]


def run_all():
    import torch
    from paper_2605_25872_gb300 import Batch, BatchConfig
    out = {}
    for i, sc in enumerate(SCENARIOS):
        cfg = BatchConfig(**sc)
        J = W.gaussian_couplings(cfg.L, cfg.n_samples, 300 + i)
        b = Batch(cfg, couplings=J, seeds=W.sample_seeds(W.SEED_BASE + 300 + i, cfg.n_samples))
        if cfg.n_res:
            b.prethermalize(5)
        b.emcs(4)
        b.measure(chaos=True)
        out[f"spins{i}"] = b.export_spins().cpu().numpy()
        out[f"obs{i}"] = b.obs.cpu().numpy()
        out[f"chaos{i}"] = b.chaos.cpu().numpy()
        out[f"E{i}"] = b.energies.cpu().numpy()
        out[f"perm{i}"] = b.perm.cpu().numpy()
        out[f"labels{i}"] = b.cluster_labels().cpu().numpy()
        out[f"poll{i}"] = np.array([b.poll(60000), b.check_canaries()])
        torch.cuda.synchronize()
    return out


if __name__ == "__main__":
    np.savez(sys.argv[1], **run_all())
