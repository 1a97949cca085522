"""Command-line run of PTHR on one GPU: a batch of disorder samples advanced
EMCS by EMCS (Sec. 3), measured after every EMCS and averaged in the log2
bins of Sec. 4 (bin 0 = the second half of the run, bin 1 the second quarter,
...), written as JSON lines: one record per (bin, sample, temperature) with
the thermal averages, PT acceptance and the last cluster move's statistics,
then one summary record (tau_TRW of Sec. 5 over the run, throughput).

    python -m paper_2605_25872_gb300.run --L 12 --samples 64 --temps 24 \\
        --emcs 4096 --bins 6 --out run.jsonl
    python -m paper_2605_25872_gb300.run --preset paper-L16 --samples 64 \\
        --emcs 65536 --out l16.jsonl       # Table A1's L = 16 run, shortened

Couplings are drawn on the device from each sample's seed (seed + s) unless
--couplings names a .npy file of FP32 [S, 3, L^3] bonds.  Every step runs in
the CUDA library; this module only schedules the calls.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np


def temperatures(t_min: float, t_max: float, n: int) -> np.ndarray:
    """T_k = t_min + k (t_max - t_min) / (n - 1) (App. A.2)."""
    k = np.arange(n, dtype=np.float64)
    return t_min + (k * (t_max - t_min)) / (n - 1)


# The paper's production runs (App. A.2, Table A1): N_T temperatures uniform in
# [T_min, T_max], 4 replica groups, the EMCS of Sec. 3 (10 sweeps, ACU below
# T = 1, PT, ER with 4 reservoir clones at 240 sweeps).  L = 12 and 14 used
# Metropolis (PTHR); L = 16 switched to MicSA (PTHR*) for bins 0 and 1; L = 18
# used MicSA throughout.
PRESETS = {
    "paper-L12": dict(L=12, t_min=0.42, t_max=1.8, temps=24, samples=2048, emcs=2 ** 17, rule="metropolis",
                      micsa_bins=0),
    "paper-L14": dict(L=14, t_min=0.2, t_max=2.0, temps=48, samples=2000, emcs=6_400_000, rule="metropolis",
                      micsa_bins=0),
    "paper-L16": dict(L=16, t_min=0.2, t_max=2.0, temps=60, samples=2081, emcs=38_400_000, rule="metropolis",
                      micsa_bins=2),
    "paper-L18": dict(L=18, t_min=0.2, t_max=2.0, temps=72, samples=2028, emcs=34_800_000, rule="micsa",
                      micsa_bins=0),
}
DEFAULTS = dict(samples=16, temps=24, t_min=0.2, t_max=1.6, rule="metropolis", micsa_bins=0)


def parse_args(argv=None):
    """Arguments given explicitly override the preset's, which override the
    defaults."""
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--preset", choices=sorted(PRESETS), default=None,
                    help="a run of the paper's Table A1 (explicit arguments override it)")
    ap.add_argument("--L", type=int, default=None)
    ap.add_argument("--samples", type=int, default=None)
    ap.add_argument("--temps", type=int, default=None)
    ap.add_argument("--t-min", type=float, default=None)
    ap.add_argument("--t-max", type=float, default=None)
    ap.add_argument("--replicas", type=int, default=4)
    ap.add_argument("--res", type=int, default=4, help="reservoir clones per replica group (0: no ER)")
    ap.add_argument("--sweeps", type=int, default=10, help="local sweeps per EMCS")
    ap.add_argument("--res-sweeps", type=int, default=240, help="reservoir sweeps per EMCS")
    ap.add_argument("--pretherm", type=int, default=960, help="reservoir pre-thermalisation sweeps")
    ap.add_argument("--rule", default=None, choices=["metropolis", "heatbath", "micsa"])
    ap.add_argument("--cluster", default="acu", choices=["acu", "single", "off"])
    ap.add_argument("--acu-interval", type=int, default=1)
    ap.add_argument("--spin-layout", default="bytes", choices=["bytes", "bits"])
    ap.add_argument("--emcs", type=int, default=None, help="EMCS of the run (t_max)")
    ap.add_argument("--bins", type=int, default=4)
    ap.add_argument("--chaos", action="store_true", help="also accumulate the chaos overlaps (Sec. 5)")
    ap.add_argument("--micsa-bins", type=int, default=None,
                    help="PTHR*: the last N bins run with the MicSA walker (App. A.1)")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--couplings", default=None, help=".npy file of FP32 couplings [S, 3, L^3]")
    ap.add_argument("--out", required=True, help="JSON-lines output file (appended)")
    args = ap.parse_args(argv)
    preset = PRESETS.get(args.preset, {})
    for key in ("L", "samples", "temps", "t_min", "t_max", "emcs", "rule", "micsa_bins"):
        if getattr(args, key) is None:
            setattr(args, key, preset.get(key, DEFAULTS.get(key)))
    if args.L is None or args.emcs is None:
        ap.error("--L and --emcs are required without a preset")
    return args


def run(args) -> dict:
    """Run the batch described by args; append the records to args.out and
    return the summary record."""
    import torch
    from .analysis import (append_jsonl, chaos_from_accumulators, log2_bins, observable_records,
                           tau_trw)
    from .batch import Batch, BatchConfig
    cfg = BatchConfig(L=args.L, n_samples=args.samples, n_temps=args.temps, t_min=args.t_min,
                      t_max=args.t_max, n_replicas=args.replicas, n_res=args.res,
                      sweeps_per_emcs=args.sweeps, res_sweeps_per_emcs=args.res_sweeps if args.res else 0,
                      acu_interval=args.acu_interval, rule=args.rule, cluster=args.cluster,
                      er_on=args.res > 0, seed=args.seed, spin_layout=args.spin_layout)
    J = np.ascontiguousarray(np.load(args.couplings), dtype=np.float32) if args.couplings else None
    stream = torch.cuda.Stream()
    b = Batch(cfg, couplings=J, stream=stream)
    T = temperatures(cfg.t_min, cfg.t_max, cfg.n_temps)
    t0 = time.perf_counter()
    if cfg.er_on and args.pretherm:
        b.prethermalize(args.pretherm)

    def advance(n):
        if n <= 0:
            return
        if args.chaos:                   # the chaos overlaps need their own measurement call
            for _ in range(n):
                b.sweep(cfg.sweeps_per_emcs, cfg.res_sweeps_per_emcs if cfg.er_on else 0)
                if cfg.cluster != "off":
                    b.houdayer()
                b.swap(True, cfg.er_on)
                b.measure(chaos=True)
        else:
            b.emcs(n, graph=True)        # one captured EMCS (measurement included), replayed

    bins = log2_bins(args.emcs, args.bins)
    order = sorted(range(len(bins)), key=lambda i: bins[i][0])      # in time order
    done = 0
    n_records = 0
    for i in order:
        lo, hi = bins[i]
        advance(lo - 1 - done)
        if i < args.micsa_bins and b.cfg.rule != "micsa":
            b.set_rule("micsa")           # PTHR*: the late bins with the walker
        b.synchronize()
        pt_prev = b.pt_accepted.cpu().numpy().copy()
        b.reset_observables()
        advance(hi - lo + 1)
        done = hi
        b.synchronize()
        obs = b.obs.cpu().numpy().copy()
        pt = b.pt_accepted.cpu().numpy().copy()
        recs = observable_records(obs, T, cfg.n_replicas, emcs=hi, pt_accepted=pt - pt_prev,
                                  cluster_stats=b.cluster_stats.cpu().numpy())
        X = chaos_from_accumulators(b.chaos.cpu().numpy(), obs, cfg.n_replicas) if args.chaos else None
        for r in recs:
            r["bin"] = i
            r["rule"] = b.cfg.rule
            if X is not None:
                v = X[r["sample"], r["k"]]
                r["chaos_X"] = float(v) if np.isfinite(v) else None
        n_records += append_jsonl(args.out, recs)
    advance(args.emcs - done)
    b.synchronize()
    dt = time.perf_counter() - t0
    trips = b.round_trips.cpu().numpy().sum(axis=1)
    tau = tau_trw(cfg.n_replicas, cfg.n_temps, args.emcs, trips)
    finite = tau[np.isfinite(tau)]
    V = cfg.L ** 3
    upd = (args.emcs * cfg.n_samples * cfg.n_replicas * V
           * (cfg.n_temps * cfg.sweeps_per_emcs + (cfg.n_res * cfg.res_sweeps_per_emcs if cfg.er_on else 0))
           + (cfg.n_samples * cfg.n_replicas * cfg.n_res * args.pretherm * V if cfg.er_on else 0))
    summary = {"summary": True, "L": cfg.L, "samples": cfg.n_samples, "temps": cfg.n_temps,
               "emcs": args.emcs, "bins": [list(x) for x in bins], "records": n_records,
               "round_trips_median": float(np.median(trips)),
               "tau_trw_median": float(np.median(finite)) if finite.size else None,
               "seconds": dt, "spin_updates_per_ns": upd / (dt * 1e9), "status": b.poll(-1)}
    append_jsonl(args.out, [summary])
    b.close()
    return summary


def main(argv=None) -> int:
    summary = run(parse_args(argv))
    print(json.dumps(summary))
    return 0 if summary["status"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
