"""Throughput of the PTHR hot path on GB300.

Workload (one "step" = one EMCS of the whole batch): PTHR at L=16 with 512
disorder samples x 32 temperatures 0.2..1.6 x 4 replica groups, plus 4
reservoir clones per group at T_max; per EMCS 10 Metropolis sweeps of every
PT clone and 240 of every reservoir clone, the all-cluster Houdayer update at
every T < 1, one PT round and one ER exchange, then the measurement.  The
reservoir is pre-thermalised with 960 sweeps before the warm-up.

Metric: spin updates per ns (PT and reservoir updates summed) for the whole
job, with EMCS/s ("PTHR sweeps/s"), Houdayer pair moves/s and the plain
one-sample-per-launch form reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own 512 samples (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "spin updates/ns and PTHR sweeps/s at L=16 (FP32 batched vs plain)"
METRIC_OTHER = "spin updates/ns and PTHR sweeps/s at L={L} (FP32 batched vs plain)"
UNIT = "spin-updates/ns"
WL = W.WORKLOADS["c4"]      # the headline workload; --workload selects another for reports
# Algorithmic ALU work of one Metropolis spin update: a
# quarter of a Philox4x32-10 call (10 rounds x (4 multiply halves + 2
# three-input XORs) / 4 = 15), the 24-bit uniform (2), the local field
# (6 FMA), -beta dE (2 FMUL), the exponential (1), the two comparisons (2)
# and the conditional flip (1).
OPS_PER_UPDATE = 29
# shared-memory bytes of one update in the packed colour-row layout: the
# 4-site word of the site and its 6 neighbours are read and the site word is
# written once per 4 updates (8 x 4 B / 4).
SMEM_BYTES_PER_UPDATE = 8
# instruction counts of the sweep kernel measured by ncu (per spin update) and
# its DRAM traffic, valid for the kernel source they were taken on
COUNTERS = os.path.join(ROOT, "profiles", "sweep_kernel_L16_counters.json")
PEAK_NAMES = ("smem_read_Bps", "l2_read_Bps", "alu_inst_per_s", "fma_inst_per_s", "fma2_inst_per_s",
              "fp64_inst_per_s")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measure_peaks(dev):
    """On-device microbenchmarks (libpthr.so, pthr_measure_peak): shared-memory
    and L2 load bandwidth and the issue rates of the ALU, FMA, f32x2 and FP64
    pipes, each one timed launch over every SM."""
    import ctypes
    import torch
    from paper_2605_25872_gb300 import _lib
    lib = _lib.load()
    scratch = torch.empty((4096 + (16 << 20),), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    out = {}
    for kind, name in enumerate(PEAK_NAMES):
        rate, sec = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _lib.check(lib.pthr_measure_peak(kind, ctypes.c_void_p(scratch.data_ptr()), scratch.numel(),
                                         ctypes.c_void_p(stream.cuda_stream), ctypes.byref(rate),
                                         ctypes.byref(sec)))
        out[name] = rate.value
    del scratch
    return out


def kernel_counters():
    """ncu counters of the sweep kernel, if they were taken on this source."""
    if not os.path.exists(COUNTERS) or WL is not W.WORKLOADS["c4"]:
        return None
    with open(COUNTERS) as f:
        c = json.load(f)
    return c if c.get("kernel_version") == kernel_version() else None


def sweep_roofline(n_sm, mhz, upd_per_s, measured):
    """Roofline of the sweep kernel, the dominant kernel of the EMCS.

    It is bound by the ALU pipe (integer logic: spin decodes, Philox XORs,
    mask assembly): the ncu count of ALU-pipe thread-instructions per update
    times the updates/s of the live sweep launch, over 64 ALU lanes/clk/SM at
    the median SM clock of the timed region (the lane count is confirmed by
    the lop3 microbenchmark).  Beside it: the issue fraction (all
    thread-instructions over 128/clk/SM), the algorithmic 29 ops/update, and
    the shared-memory fraction against the measured load bandwidth."""
    cnt = kernel_counters()
    alu_peak = n_sm * 64 * mhz * 1e6
    issue_peak = n_sm * 128 * mhz * 1e6
    alg = OPS_PER_UPDATE * upd_per_s
    roof = {"kernel": f"sweep_kernel<{WL.L}, Metropolis>", "bound": "alu"}
    if cnt:
        alu = cnt["alu_inst_per_update"] * upd_per_s
        roof.update({"achieved": alu / 1e12, "peak": alu_peak / 1e12, "unit": "T thread-instr/s (ALU pipe)",
                     "frac": alu / alu_peak, "traffic": cnt.get("dram_bytes_per_launch"),
                     "basis": (f"ncu: {cnt['alu_inst_per_update']:.2f} ALU-pipe thread-instructions per "
                               f"spin update x updates/s of the sweep launch (CUDA events), over {n_sm} SMs "
                               f"x 64 ALU lanes/clk x {mhz:.0f} MHz (median SM clock of the timed region)"),
                     "issue": {"achieved": cnt["inst_per_update"] * upd_per_s / 1e12, "peak": issue_peak / 1e12,
                               "frac": cnt["inst_per_update"] * upd_per_s / issue_peak,
                               "inst_per_update": cnt["inst_per_update"],
                               "basis": "all thread-instructions over 128/clk/SM"}})
    else:
        roof.update({"achieved": alg / 1e12, "peak": issue_peak / 1e12, "unit": "T lane-ops/s",
                     "frac": alg / issue_peak, "traffic": None,
                     "basis": (f"no ncu counters for this kernel source: algorithmic {OPS_PER_UPDATE} ops "
                               f"per update over {n_sm} SMs x 128 lanes x {mhz:.0f} MHz")})
    roof["algorithmic"] = {"ops_per_update": OPS_PER_UPDATE, "achieved": alg / 1e12,
                           "frac_of_issue_peak": alg / issue_peak}
    if measured:
        smem = SMEM_BYTES_PER_UPDATE * upd_per_s
        roof["alu_peak_measured"] = measured["alu_inst_per_s"] / 1e12
        roof["smem"] = {"achieved_TBps": smem / 1e12, "peak_TBps": measured["smem_read_Bps"] / 1e12,
                        "frac": smem / measured["smem_read_Bps"], "bytes_per_update": SMEM_BYTES_PER_UPDATE,
                        "peak_basis": "measured 16-byte shared loads (pthr_measure_peak)",
                        "half_of_smem_roofline_reached": smem >= 0.5 * measured["smem_read_Bps"]}
        roof["l2_peak_TBps"] = measured["l2_read_Bps"] / 1e12
    return roof


RULE = "metropolis"        # local update rule of the timed batch (--rule; profiling cases)
SPINS = "bytes"            # spin storage of the timed batches (--spin-layout)


def batch_config(n_samples=None):
    from paper_2605_25872_gb300 import BatchConfig
    return BatchConfig(L=WL.L, n_samples=n_samples or WL.n_samples, n_temps=WL.n_temps,
                       t_min=WL.t_min, t_max=WL.t_max, n_replicas=WL.n_replicas,
                       n_res=WL.n_res if WL.er_on else 0, sweeps_per_emcs=WL.sweeps_per_emcs,
                       res_sweeps_per_emcs=WL.res_sweeps_per_emcs, er_on=WL.er_on, cluster="acu",
                       rule=RULE, spin_layout=SPINS)


def updates_per_emcs(n_samples):
    V = WL.V
    pt = n_samples * WL.n_replicas * WL.n_temps * WL.sweeps_per_emcs * V
    res = n_samples * WL.n_replicas * WL.n_res * WL.res_sweeps_per_emcs * V if WL.er_on else 0
    return pt, res


def n_acu_temps():
    T = [WL.t_min + k * (WL.t_max - WL.t_min) / (WL.n_temps - 1) for k in range(WL.n_temps)]
    return sum(1 for t in T if t < 1.0)


# ----------------------------------------------------------------------------- CPU legs

def oracle_sample_run(n_threads, n_emcs=1, seed_offset=0):
    """The FP64 oracle, as it stands, on `n_threads` samples of the workload,
    one EMCS each, in parallel host threads.  Returns (updates, seconds)."""
    import oracle as O
    J = W.gaussian_couplings(WL.L, n_threads, W.batch_seed(WL.index) + 17 + seed_offset)
    smps = [O.OracleSample(WL.L, WL.n_temps, WL.t_min, WL.t_max, W.batch_seed(WL.index) + s,
                           J=J[s].astype(np.float64), n_groups=WL.n_replicas,
                           n_res=WL.n_res if WL.er_on else 0, er_on=WL.er_on,
                           sweeps_per_emcs=WL.sweeps_per_emcs,
                           res_sweeps_per_emcs=WL.res_sweeps_per_emcs)
            for s in range(n_threads)]
    t0 = time.perf_counter()
    used = O.run_samples_threaded(smps, n_emcs, n_threads)
    dt = time.perf_counter() - t0
    pt, res = updates_per_emcs(used)
    return (pt + res) * n_emcs, dt, used


def cpu_baseline(target_s=12.0):
    """The oracle on every host core, one sample per thread, sized to about
    target_s seconds of CPU work (a one-EMCS probe sets the EMCS count)."""
    cores = os.cpu_count() or 1
    _, dt1, _ = oracle_sample_run(cores)
    n = max(1, min(5000, int(round(target_s / max(dt1, 1e-4)))))
    upd, dt, used = oracle_sample_run(cores, n_emcs=n, seed_offset=1)
    return {"value": upd / (dt * 1e9), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{used} samples x {n} EMCS of the L={WL.L} workload (one sample per host "
                      f"thread), {upd:.3g} spin updates in {dt:.3g} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample_run(min(cores, 2))
    times, upd_total = [], 0
    for k in range(args.steps):
        upd, dt, used = oracle_sample_run(cores, seed_offset=k)
        times.append(dt)
        upd_total += upd
    value = upd_total / (sum(times) * 1e9)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {cores} samples x 1 EMCS of the workload, one per host thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_dict():
    res = (f" + {WL.n_res} reservoir clones/group" if WL.er_on else "")
    emcs = (f"{WL.sweeps_per_emcs} sweep{'s' if WL.sweeps_per_emcs > 1 else ''} + ACU(T<1) + PT"
            + (f" + ER ({WL.res_sweeps_per_emcs} reservoir sweeps)" if WL.er_on else ""))
    lat = WL.n_samples * WL.lattices_per_sample
    lat_bytes = 2 * WL.L * WL.L * ((WL.L // 2 + 3) // 4) * 4 // (8 if SPINS == "bits" else 1)
    state_mb = (lat * lat_bytes + WL.n_samples * 3 * WL.V * 4) / 1e6
    return {"workload": f"{WL.name} (L={WL.L}, {WL.n_samples} samples x {WL.n_temps} T "
                        f"[{WL.t_min},{WL.t_max}] x {WL.n_replicas} replicas{res}; EMCS = {emcs})",
            "L": WL.L, "n_samples": WL.n_samples, "n_temps": WL.n_temps, "n_replicas": WL.n_replicas,
            "n_res": WL.n_res if WL.er_on else 0, "sweeps_per_emcs": WL.sweeps_per_emcs,
            "res_sweeps_per_emcs": WL.res_sweeps_per_emcs if WL.er_on else 0,
            "update_rule": RULE, "spin_layout": SPINS, "couplings": "N(0,1) on the 2^-18 grid (seeded)",
            "l2": (f"inputs larger than L2: {state_mb:.0f} MB of spins and couplings resident per GPU"
                   if state_mb > 129 else
                   f"{state_mb:.0f} MB of spins and couplings resident per GPU (fits in the 129 MB L2)")}


# ----------------------------------------------------------------------------- GPU arm

def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2605_25872_gb300 import Batch
    from paper_2605_25872_gb300.build import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
        build()

    cfg = batch_config(args.samples)
    S = cfg.n_samples
    schedule = None
    if args.tuned_schedule:
        # the schedule autotuner's cluster-move interval (the smallest whose
        # cluster step is at most 10% of the EMCS on this GPU); it changes the
        # Markov chain, so only this explicitly labelled line uses it
        import dataclasses
        from paper_2605_25872_gb300.autotune import autotune_schedule
        k, schedule = autotune_schedule(cfg, device=dev)
        cfg = dataclasses.replace(cfg, acu_interval=int(k))
    from paper_2605_25872_gb300.shard import shard_seeds
    seeds = shard_seeds(W.batch_seed(WL.index), rank, world, world * S)   # global sample ids
    J = W.gaussian_couplings(WL.L, S, W.batch_seed(WL.index) + rank)
    stream = torch.cuda.Stream(dev)
    b = Batch(cfg, couplings=J, seeds=seeds, device=dev, stream=stream)
    tuned_shape = None
    if args.tuned:
        # the autotuner's shape for this configuration (measured on this GPU
        # on a scratch batch; shapes never change results)
        from paper_2605_25872_gb300.autotune import autotune
        tuned_shape = autotune(cfg, device=dev)
        if tuned_shape:
            b.set_tuning(**tuned_shape)
    if WL.er_on and WL.res_pretherm_sweeps:
        b.prethermalize(WL.res_pretherm_sweeps)
    pt_upd, res_upd = updates_per_emcs(S)
    upd = pt_upd + res_upd

    # ---- on-chip peaks of this GPU (rank 0), then warm-up
    measured = measure_peaks(dev) if (rank == 0 and not args.no_extras) else None
    for _ in range(args.warmup):
        b.emcs(1)
    stream.synchronize()

    # ---- timed region: the EMCS as its four C-ABI calls, CUDA events between
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t_start.record(stream)
        for k in range(args.steps):
            e = ev[k]
            e[0].record(stream)
            b.sweep(WL.sweeps_per_emcs, WL.res_sweeps_per_emcs if WL.er_on else 0)
            e[1].record(stream)
            b.houdayer()
            e[2].record(stream)
            b.swap(True, WL.er_on)
            e[3].record(stream)
            b.measure()
            e[4].record(stream)
        t_end.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ms_total = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
        dist.barrier()
    phase = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(4)] for e in ev])
    ms_sweep = float(phase[:, 0].mean())
    ms_step = ms_total / args.steps
    value = world * upd * args.steps / (ms_total * 1e6)
    assert b.poll(60000) == 0

    if args.no_extras:
        # the same EMCS replayed from one captured CUDA graph
        b.emcs(1, graph=True)
        stream.synchronize()
        gr0, gr1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            gr0.record(stream)
            b.emcs(max(2, args.steps), graph=True)
            gr1.record(stream)
        stream.synchronize()
        ms_gr = gr0.elapsed_time(gr1) / max(2, args.steps)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "updates_per_ns_graph": world * upd / (ms_gr * 1e6),
                              "shape": tuned_shape or "default", "acu_interval": cfg.acu_interval,
                              **({"schedule": schedule} if schedule else {}),
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                              "samples": S, "phase_ms_sweep": ms_sweep,
                              "phase_ms": {n: float(phase[:, i].mean()) for i, n in
                                           enumerate(("sweep", "houdayer", "swap", "measure"))},
                              "clocks": clocks,
                              "note": "profiling case, not a headline line"}))
        if world > 1:
            dist.destroy_process_group()
        return 0

    # ---- graph replay of whole EMCS (same kernels, one launch per EMCS)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.emcs(1, graph=True)
    stream.synchronize()
    n_graph = max(2, min(args.steps, 10))
    with torch.cuda.stream(stream):
        g0.record(stream)
        b.emcs(n_graph, graph=True)
        g1.record(stream)
    stream.synchronize()
    ms_graph = g0.elapsed_time(g1) / n_graph

    # ---- end to end through the public API, on every rank at once: the
    # whole job's updates over the slowest rank's wall time
    if world > 1:
        dist.barrier()
    e2e, e2e_upd, e2e_s = end_to_end(dev, cfg, J, seeds, args.steps)
    if world > 1:
        tu = torch.tensor([e2e_upd], dtype=torch.float64, device=dev)
        ts = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(tu, op=dist.ReduceOp.SUM)
        dist.all_reduce(ts, op=dist.ReduceOp.MAX)
        e2e["value"] = float(tu.item()) / (float(ts.item()) * 1e9)
        e2e["h2d_bytes_per_step"] *= world
        e2e["d2h_bytes_per_step"] *= world

    result = None
    if rank == 0:
        pk, pk_kind = peaks()
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks.get("sm_mhz") or float(pk.get("sm_max_mhz", 2070.0))
        upd_per_s = upd / (ms_sweep * 1e-3)
        roof = sweep_roofline(n_sm, mhz, upd_per_s, measured)
        pairs = S * (WL.n_replicas // 2) * n_acu_temps()
        ms_cluster = float(phase[:, 1].mean())
        plain = plain_form(dev, upd / S, seeds, J)
        autocorr = None
        if WL.er_on and world == 1:
            # reservoir residence calibration (Sec. 3, ER): C(tau) at T_max for
            # tau = 240, 480, 720, 960 sweeps over every reservoir clone
            from paper_2605_25872_gb300.analysis import spin_autocorrelation
            sums = b.reservoir_autocorrelation(4, WL.res_sweeps_per_emcs).cpu().numpy()
            _, cmean, cerr = spin_autocorrelation(sums, WL.n_replicas, WL.n_res, WL.V)
            autocorr = {"tau_sweeps": [WL.res_sweeps_per_emcs * (p + 1) for p in range(4)],
                        "C": [float(x) for x in cmean], "C_err": [float(x) for x in cerr],
                        "t_max": WL.t_max, "samples": S, "clones_per_sample": WL.n_replicas * WL.n_res,
                        "paper": "C(960) < 1e-3 at the paper's T_max = 2 (Sec. 3, ER; App. A.2)"}
            autocorr["t_max_2"] = autocorr_at(dev, 2.0)
        serving = mixed = micsa = None
        if WL is W.WORKLOADS["c4"] and world == 1:
            serving = serve_measure(args.serve_budget, args.serve_requests, args.serve_mem_gb,
                                    args.serve_max_slots, args.serve_chunk, not args.serve_default_shapes)
            mixed = mixed_group_measure(dev)
            micsa = micsa_measure(dev, J, seeds)
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(),
            "emcs_per_s": world * 1e3 / ms_step,
            "emcs_per_s_graph": world * 1e3 / ms_graph,
            "updates_per_ns_graph": world * upd / (ms_graph * 1e6),
            "pt_updates_per_emcs": pt_upd, "res_updates_per_emcs": res_upd,
            "houdayer_pair_moves_per_s": world * pairs * 1e3 / ms_step,
            "sites_labelled_per_ns": pairs * WL.V / (ms_cluster * 1e6) if ms_cluster > 0 else None,
            "phase_ms": {"sweep": ms_sweep, "houdayer": ms_cluster,
                         "swap": float(phase[:, 2].mean()), "measure": float(phase[:, 3].mean())},
            "plain": plain,
            "roofline": roof,
            "measured_peaks": {k: v for k, v in measured.items()} if measured else None,
            "gpu_launches": 4 * args.steps,
            "serving": serving,
            "mixed_sizes": mixed,
            "reservoir_autocorrelation": autocorr,
            "micsa": micsa,
            "cpu_baseline": cpu_baseline() if world == 1 else None,
            "e2e": e2e,
            "clocks": clocks,
        }
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def kernel_version():
    """Hash of the sweep kernel source: a stored DRAM-traffic figure is only
    valid for the kernel it was measured on."""
    import hashlib
    h = hashlib.sha1()
    for f in ("sweep_kernel.cuh", "geometry.cuh", "sweep.cu", "sweep_table.h", "pthr_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2605_25872_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def plain_form(dev, upd_per_sample, seeds, J, n=32):
    """The same kernels with one sample per launch sequence and no graph,
    looped over samples (a bounded sample of n of the 512, scaled)."""
    import torch
    from paper_2605_25872_gb300 import Batch
    cfg = batch_config(1)
    stream = torch.cuda.Stream(dev)
    bs = [Batch(cfg, couplings=J[s:s + 1], seeds=seeds[s:s + 1], device=dev, stream=stream)
          for s in range(n)]
    for x in bs:
        if WL.er_on and WL.res_pretherm_sweeps:
            x.prethermalize(WL.res_pretherm_sweeps)
        x.emcs(1)
    stream.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        t0.record(stream)
        for x in bs:
            x.emcs(1, graph=False)
        t1.record(stream)
    stream.synchronize()
    ms = t0.elapsed_time(t1)
    ms_512 = ms * WL.n_samples / n
    for x in bs:
        x.close()
    return {"updates_per_ns": upd_per_sample * n / (ms * 1e6),
            "emcs_per_s_512_samples": 1e3 / ms_512,
            "sample": f"{n} of {WL.n_samples} samples x 1 EMCS, one sample per launch sequence"}


def end_to_end(dev, cfg, J, seeds, steps):
    """The user's path through the public API with host buffers: pinned host
    couplings copied to the device at creation, reservoir pre-thermalisation,
    `steps` EMCS each followed by a device-to-host read of the observables."""
    import torch
    from paper_2605_25872_gb300 import Batch
    Jp = torch.from_numpy(J).pin_memory()
    out = torch.empty((cfg.n_samples, cfg.n_temps, 8), dtype=torch.float64).pin_memory()
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    b = Batch(cfg, couplings=Jp, seeds=seeds, device=dev, stream=stream)
    if WL.er_on and WL.res_pretherm_sweeps:
        b.prethermalize(WL.res_pretherm_sweeps)
    host = out.numpy()
    for _ in range(steps):
        b.emcs(1, graph=True)
        b.read_observables(out=host)
    stream.synchronize()
    dt = time.perf_counter() - t0
    pt, res = updates_per_emcs(cfg.n_samples)
    pre = cfg.n_samples * WL.n_replicas * WL.n_res * WL.res_pretherm_sweeps * WL.V if WL.er_on else 0
    b.close()
    n_upd = steps * (pt + res) + pre
    return ({"value": n_upd / (dt * 1e9), "unit": UNIT,
             "h2d_bytes_per_step": int((J.nbytes + seeds.nbytes) / steps),
             "d2h_bytes_per_step": int(out.numel() * 8),
             "includes": "H2D couplings+seeds, init, 960-sweep reservoir pre-thermalisation, "
                         f"{steps} EMCS, D2H observables after every EMCS"}, n_upd, dt)


def serve_measure(budget, n_req, mem_gb, max_slots, max_chunk, tuned=True):
    """Serving: Poisson stream of single-sample requests with L uniform in
    {6, 8, 10, 12, 16} (24 temperatures 0.2..1.6, 4 replicas + 4 reservoir
    clones, paper EMCS), admitted into per-L resident pools sized from a
    device-memory budget; rate = 0.8 x the measured capacity.  Returns the
    p50/p99 time from arrival to a finished budget and the aggregate spin
    updates/ns over the run."""
    import torch
    from paper_2605_25872_gb300 import required_bytes, BatchConfig
    from paper_2605_25872_gb300.serve import PoolSpec, Request, Server
    mem = mem_gb * 1e9
    specs = []
    for L in W.SERVE_SIZES:
        one = required_bytes(BatchConfig(L=L, n_samples=1, n_temps=24, spin_layout=SPINS))
        slots = int(min(max_slots, (mem / len(W.SERVE_SIZES)) // one))
        specs.append(PoolSpec(L=L, slots=slots, n_temps=24, spin_layout=SPINS))
    if tuned:
        # each pool's autotuned kernel shape (measured on this GPU for that
        # pool's configuration; shapes never change results)
        from paper_2605_25872_gb300.autotune import autotune
        from paper_2605_25872_gb300.serve import GpuPool
        for sp in specs:
            sp.tuning = autotune(GpuPool.config_of(sp)) or None
    # capacity probe: every pool full, EMCS timed with all pools in flight
    srv = Server(specs, max_chunk=max_chunk)
    probe = [Request(rid=-1 - i * 100000 - k, L=sp.L, seed=10 ** 6 + i * 100000 + k, budget_emcs=10 ** 6)
             for i, sp in enumerate(specs) for k in range(sp.slots)]
    per_emcs_s = srv.fill_and_time(probe, 5)
    del srv
    torch.cuda.synchronize()
    cap = min(sp.slots / (budget * per_emcs_s) for sp in specs) * len(specs)   # requests/s
    lam = 0.8 * cap
    times, Ls = W.poisson_arrivals(n_req, lam, W.batch_seed(5))
    reqs = [Request(rid=i, L=int(Ls[i]), seed=W.batch_seed(5) + 7919 * i, budget_emcs=budget,
                    arrival=float(times[i])) for i in range(n_req)]
    srv = Server(specs, max_chunk=max_chunk)
    srv.run(reqs, realtime=True)
    st = srv.stats()
    return {"metric": "time-to-budget p50/p99 and aggregate spin updates/ns",
            "p50_s": st["p50_s"], "p99_s": st["p99_s"], "updates_per_ns": st["updates_per_ns"],
            "requests": st["requests"], "budget_emcs": budget, "lambda_per_s": lam,
            "capacity_per_s": cap, "full_pool_emcs_s": per_emcs_s,
            "slots": {sp.L: sp.slots for sp in specs}, "memory_budget_gb": mem_gb,
            "emcs_steps": st["emcs_steps"], "chunks": st["chunks"], "max_chunk": max_chunk,
            "pool_shapes": {sp.L: (sp.tuning or "default") for sp in specs},
            "config": {"workload": "serving: L uniform in {6,8,10,12,16}, 24 T 0.2..1.6, 4 replicas + "
                                   "4 reservoir clones, paper EMCS, couplings drawn on the device from each "
                                   "request's seed, 960-sweep reservoir pre-thermalisation at admission, "
                                   "Poisson arrivals at 0.8 x the measured capacity"}}


def autocorr_at(dev, t_max, n_samples=256):
    """C(tau) of the reservoir clones at T_max = t_max (the paper's L = 16
    grid ends at T_max = 2, App. A.2) after the 960-sweep pre-thermalisation,
    tau = 240 .. 960, same lattice size and reservoir as the workload."""
    import dataclasses
    import torch
    from paper_2605_25872_gb300 import Batch
    from paper_2605_25872_gb300.analysis import spin_autocorrelation
    cfg = dataclasses.replace(batch_config(n_samples), t_max=t_max)
    b = Batch(cfg, couplings=None, seeds=W.sample_seeds(W.batch_seed(WL.index) + 77777, n_samples), device=dev,
              stream=torch.cuda.Stream(dev))
    b.prethermalize(960)
    sums = b.reservoir_autocorrelation(4, 240).cpu().numpy()
    b.close()
    _, cmean, cerr = spin_autocorrelation(sums, cfg.n_replicas, cfg.n_res, cfg.V)
    return {"t_max": t_max, "tau_sweeps": [240, 480, 720, 960], "C": [float(x) for x in cmean],
            "C_err": [float(x) for x in cerr], "samples": n_samples}


def micsa_measure(dev, J, seeds, n_emcs=10):
    """The same workload with the MicSA local update (App. A.1; the paper's
    PTHR* for its late L=16 bins): EMCS and sweep-launch timing with CUDA
    events (graph replay of whole EMCS)."""
    import dataclasses
    import torch
    from paper_2605_25872_gb300 import Batch
    cfg = dataclasses.replace(batch_config(len(seeds)), rule="micsa")
    stream = torch.cuda.Stream(dev)
    b = Batch(cfg, couplings=J, seeds=seeds, device=dev, stream=stream)
    if WL.er_on and WL.res_pretherm_sweeps:
        b.prethermalize(WL.res_pretherm_sweeps)
    b.emcs(3, graph=True)
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    with torch.cuda.stream(stream):
        e0.record(stream)
        b.emcs(n_emcs, graph=True)
        e1.record(stream)
        b.sweep(WL.sweeps_per_emcs, WL.res_sweeps_per_emcs if WL.er_on else 0)
        e2.record(stream)
        b.houdayer()
        b.swap(True, WL.er_on)
        b.measure()
    stream.synchronize()
    pt, res = updates_per_emcs(len(seeds))
    ms = e0.elapsed_time(e1) / n_emcs
    ms_sweep = e1.elapsed_time(e2)
    b.close()
    return {"rule": "micsa", "updates_per_ns": (pt + res) / (ms * 1e6), "ms_per_emcs": ms,
            "sweep_ms": ms_sweep, "sweep_updates_per_ns": (pt + res) / (ms_sweep * 1e6)}


def mixed_group_measure(dev, slots=128, n_emcs=10):
    """Mixed lattice sizes advanced together: one resident batch per L in
    {6, 8, 10, 12, 16} (slots samples each, 24 temperatures, 4 replicas + 4
    reservoir clones, paper EMCS), every slot busy.  Times n_emcs EMCS as one
    group graph (pthr_group: one launch per EMCS step over every size) and
    as one graph per batch on its own stream."""
    import torch
    from paper_2605_25872_gb300 import Batch, BatchConfig, Group
    batches = []
    for L in W.SERVE_SIZES:
        cfg = BatchConfig(L=L, n_samples=slots, n_temps=24)
        b = Batch(cfg, couplings=None, seeds=W.sample_seeds(W.batch_seed(5) + 1000 * L, slots), device=dev,
                  stream=torch.cuda.Stream(dev))
        b.prethermalize(960)
        batches.append(b)
    torch.cuda.synchronize(dev)
    upd = sum(b.cfg.n_samples * b.cfg.n_replicas * (b.cfg.n_temps * b.cfg.sweeps_per_emcs
                                                      + b.cfg.n_res * b.cfg.res_sweeps_per_emcs) * b.cfg.V
              for b in batches)
    g = Group(batches)
    g.emcs(2)
    g.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.emcs(n_emcs)
    e1.record(g.stream)
    g.synchronize()
    ms_group = e0.elapsed_time(e1) / n_emcs
    launches = g.launches_per_emcs
    g.close()
    for b in batches:
        b.emcs(1, graph=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(n_emcs):
        for b in batches:
            b.emcs(1, graph=True)
    torch.cuda.synchronize(dev)
    ms_sep = (time.perf_counter() - t0) * 1e3 / n_emcs
    for b in batches:
        b.close()
    return {"sizes": list(W.SERVE_SIZES), "samples_per_size": slots,
            "group_launches_per_emcs": launches, "group_ms_per_emcs": ms_group,
            "group_updates_per_ns": upd / (ms_group * 1e6),
            "separate_graphs_ms_per_emcs": ms_sep, "separate_updates_per_ns": upd / (ms_sep * 1e6),
            "separate_launches_per_emcs": 4 * len(batches)}


def run_serve(args):
    import torch
    from paper_2605_25872_gb300.build import build
    build()
    torch.cuda.set_device(0)
    line = {"mode": "serve", **serve_measure(args.serve_budget, args.serve_requests, args.serve_mem_gb,
                                             args.serve_max_slots, args.serve_chunk,
                                             not args.serve_default_shapes)}
    print(json.dumps(line))
    return 0


def run_autotune(args):
    from paper_2605_25872_gb300.build import build
    from paper_2605_25872_gb300.autotune import autotune, autotune_schedule
    build()
    cfg = batch_config(args.samples)
    shape = autotune(cfg, emcs=3, use_cache=False, verbose=True)
    k, table = autotune_schedule(cfg)
    print(json.dumps({"mode": "autotune", "best_shape": shape, "acu_interval": k, "schedule": table}))
    return 0


def main():
    global WL
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--samples", type=int, default=WL.n_samples,
                    help="samples per GPU (profiling cases only; the headline uses 512)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the batched EMCS only (no plain form, e2e, CPU baseline)")
    ap.add_argument("--serve", action="store_true", help="serving mode (separate JSON line)")
    ap.add_argument("--serve-budget", type=int, default=10000,
                    help="EMCS per request (serving; 10^4 EMCS = the 10^5-sweep budget of the serving workload)")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-mem-gb", type=float, default=2.0)
    ap.add_argument("--serve-max-slots", type=int, default=128)
    ap.add_argument("--serve-default-shapes", action="store_true",
                    help="serving pools keep the library's default kernel shapes (else autotuned)")
    ap.add_argument("--serve-chunk", type=int, default=64,
                    help="most EMCS a pool runs between two host checks (serving)")
    ap.add_argument("--autotune", action="store_true", help="print the shape sweep for the workload")
    ap.add_argument("--workload", default="c4", choices=["c2", "c3", "c4"],
                    help="c4 (L=16 PTHR, the headline) or the batched L=8 / L=12 workloads")
    ap.add_argument("--spin-layout", default="bytes", choices=["bytes", "bits"],
                    help="spin storage in device memory (bits: 8x smaller; same results)")
    ap.add_argument("--tuned-schedule", action="store_true",
                    help="apply the schedule autotuner's cluster-move interval (a different Markov chain "
                         "schedule; profiling lines only)")
    ap.add_argument("--tuned", action="store_true",
                    help="apply the autotuned kernel shape of the workload before timing")
    ap.add_argument("--rule", default="metropolis", choices=["metropolis", "heatbath", "micsa"],
                    help="local update rule of the timed batch (profiling cases; the headline is Metropolis)")
    args = ap.parse_args()
    WL = W.WORKLOADS[args.workload]
    global RULE, SPINS
    RULE = args.rule
    SPINS = args.spin_layout
    if RULE != "metropolis" and not args.no_extras:
        ap.error("--rule other than metropolis is for --no-extras profiling runs")
    if args.tuned_schedule and not args.no_extras:
        ap.error("--tuned-schedule is for --no-extras profiling runs")
    if args.workload != "c4":
        global METRIC
        METRIC = METRIC_OTHER.format(L=WL.L)
    if args.samples == W.WORKLOADS["c4"].n_samples:
        args.samples = WL.n_samples
    if args.serve:
        return run_serve(args)
    if args.autotune:
        return run_autotune(args)
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
