"""Scenarios run under both builds of the CUDA library (release and the
range-checked PTHR_DEBUG build): every step of the EMCS at several lattice
sizes, both cluster moves, heat bath, MicSA, both spin layouts,
pre-thermalisation and labels.

Run as a script (python tests/debug_build_scenarios.py OUT.npz) it executes
the scenarios in this process with whatever library PTHR_LIBRARY names and
saves every result plus each batch's poll status; with OUT.json --scale it
runs the full-size scenarios and saves their status and result digests."""
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


# the full-size workloads (every kernel at its production grid size): only a
# digest of each result is kept
SCALE_SCENARIOS = [
    (dict(L=16, n_samples=512, n_temps=32, n_res=4, sweeps_per_emcs=10, res_sweeps_per_emcs=240), 960, 2),
    (dict(L=16, n_samples=512, n_temps=32, n_res=4, sweeps_per_emcs=10, res_sweeps_per_emcs=240,
          spin_layout="bits"), 960, 2),
    (dict(L=12, n_samples=1024, n_temps=24, n_res=0, er_on=False, sweeps_per_emcs=1), 0, 10),
    (dict(L=8, n_samples=256, n_temps=16, n_res=0, er_on=False, sweeps_per_emcs=1, cluster="single"), 0, 20),
    (dict(L=24, n_samples=16, n_temps=16, n_res=2, sweeps_per_emcs=4, res_sweeps_per_emcs=16,
          rule="heatbath"), 32, 3),
    (dict(L=20, n_samples=32, n_temps=16, n_res=2, sweeps_per_emcs=4, res_sweeps_per_emcs=16,
          rule="micsa"), 32, 3),
]


def _digest(b):
    import hashlib
    import torch
    torch.cuda.synchronize()
    h = hashlib.sha1()
    for n in ("energies", "perm", "age", "obs", "flips", "cluster_stats", "round_trips", "chaos"):
        h.update(getattr(b, n).cpu().numpy().tobytes())
    h.update(b.export_spins().cpu().numpy().tobytes())
    torch.cuda.synchronize()
    return h.hexdigest()


def run_scale():
    """The full-size scenarios plus the five-size group (mixed spin layouts);
    per case: poll status, first bad guard block, digest of every result."""
    import torch
    from paper_2605_25872_gb300 import Batch, BatchConfig
    from paper_2605_25872_gb300.batch import Group
    out = {}
    for i, (kw, pre, n) in enumerate(SCALE_SCENARIOS):
        cfg = BatchConfig(n_replicas=4, **kw)
        b = Batch(cfg, couplings=W.gaussian_couplings(cfg.L, cfg.n_samples, 9),
                  seeds=W.sample_seeds(W.SEED_BASE + 9, cfg.n_samples), stream=torch.cuda.Stream())
        if pre:
            b.prethermalize(pre)
        b.emcs(n)
        b.measure(chaos=True)
        out[f"scale{i}"] = (b.poll(600000), b.check_canaries(), _digest(b))
        b.close()
    bs = []
    for i, L in enumerate((6, 8, 10, 12, 16)):
        cfg = BatchConfig(L=L, n_samples=128, n_temps=24, n_replicas=4, n_res=4, sweeps_per_emcs=10,
                          res_sweeps_per_emcs=240, spin_layout="bits" if L in (8, 12) else "bytes")
        bs.append(Batch(cfg, couplings=W.gaussian_couplings(L, 128, 20 + i),
                        seeds=W.sample_seeds(W.SEED_BASE + 20 + i, 128), stream=torch.cuda.Stream()))
        bs[-1].prethermalize(240)
    g = Group(bs)
    g.emcs(3)
    for b in bs:
        out[f"group{b.cfg.L}"] = (b.poll(600000), b.check_canaries(), _digest(b))
    return out


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
    if len(sys.argv) > 2 and sys.argv[2] == "--scale":
        import json
        with open(sys.argv[1], "w") as f:
            json.dump(run_scale(), f)
    else:
        np.savez(sys.argv[1], **run_all())
