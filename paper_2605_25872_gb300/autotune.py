"""Autotuner for the kernel shapes of a batch configuration.

It times whole EMCS (CUDA events on the batch's stream) for candidate shapes:
lattices per sweep block for PT and reservoir clones, sweep threads, and
cluster threads.  It does this on a scratch batch of the same configuration,
keeps the fastest shape, and caches it per (configuration, GPU).  Shapes
never change results, because every random number is keyed by (sample,
lattice, site, step), so tuning can run on synthetic couplings and the
winner can be applied to any batch of that configuration.
"""
from __future__ import annotations

import itertools
import json
import os

import numpy as np

from ._lib import PthrError
from .batch import Batch, BatchConfig

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning_cache.json")


def _key(cfg: BatchConfig, device_name: str) -> str:
    d = dict(cfg.__dict__)
    d.pop("seed", None)
    return device_name + "|" + json.dumps(d, sort_keys=True)


def sweep_lane_threads(L: int) -> list:
    """Sweep block sizes below the default: whole lattice lanes of Gt threads
    (Gt = the 4-site groups of one colour, or its largest divisor up to 512),
    one, two or four lanes.  Fewer lanes give each thread more lattices, so
    its couplings serve more updates, and give small batches more blocks."""
    G = L * L * ((L // 2 + 3) // 4)
    Gt = G if G <= 512 else max(d for d in range(1, 513) if G % d == 0)
    return [Gt * p for p in (1, 2, 4) if p < 512 // Gt]


def candidates(cfg: BatchConfig):
    """Sweep shapes (PT / reservoir lattices per block, sweep threads), then
    cluster threads."""
    npt = cfg.n_replicas * cfg.n_temps
    nres = cfg.n_replicas * max(cfg.n_res, 1)
    ks = sorted({k for k in (4, 8, 12, 16, 24, 32, 48, 64) if k <= npt} | {npt if npt <= 64 else 64})
    kr = sorted({k for k in (2, 4, 8, 16, 32) if k <= nres} | {nres if nres <= 64 else 64})
    for kp, krs, th in itertools.product(ks, kr, [0] + sweep_lane_threads(cfg.L)):
        shape = {"pt_lattices_per_block": kp, "res_lattices_per_block": krs}
        if th:
            shape["sweep_threads"] = th
        yield shape
    V = cfg.L ** 3
    for ct in (64, 128, 256, 384, 512):
        if ct <= max(64, V // 2):
            yield {"cluster_threads": ct}


def time_shape(b: Batch, shape: dict, emcs: int = 3, warmup: int = 1) -> float:
    import torch
    b.set_tuning(**shape)
    b.emcs(warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(b.stream):
        e0.record(b.stream)
        b.emcs(emcs)
        e1.record(b.stream)
    b.stream.synchronize()
    return e0.elapsed_time(e1) / emcs


def autotune(cfg: BatchConfig, emcs: int = 3, use_cache: bool = True, device="cuda",
             verbose: bool = False, warm_emcs: int = 20, pretherm_sweeps: int = 960) -> dict:
    """Return the fastest shape for cfg (measured on this GPU).  The scratch
    batch is brought to a representative state first (reservoir
    pre-thermalisation and warm_emcs EMCS): the cluster step's cost depends on
    the cluster structure of the replica pairs."""
    import torch
    name = torch.cuda.get_device_name(torch.device(device))
    key = _key(cfg, name)
    cache = {}
    if use_cache and os.path.exists(CACHE):
        with open(CACHE) as f:
            cache = json.load(f)
        if key in cache:
            return cache[key]["shape"]
    rng = np.random.default_rng(0)
    J = np.rint(rng.standard_normal((cfg.n_samples, 3, cfg.L ** 3)) * 2 ** 18) / 2 ** 18
    b = Batch(cfg, couplings=J.astype(np.float32), device=device)
    if cfg.er_on and cfg.n_res:
        b.prethermalize(pretherm_sweeps)
    b.emcs(warm_emcs)
    base = time_shape(b, {}, emcs)
    best, best_ms = {}, base
    results = [({}, base)]
    sweep_best = {}
    for shape in candidates(cfg):
        trial = dict(sweep_best)
        trial.update(shape)
        try:
            ms = time_shape(b, trial, emcs)
        except PthrError:
            continue
        results.append((trial, ms))
        if verbose:
            print(f"{trial}: {ms:.3f} ms/EMCS")
        if ms < best_ms:
            best, best_ms = trial, ms
            if "pt_lattices_per_block" in shape:
                sweep_best = {k: v for k, v in trial.items() if k != "cluster_threads"}
    b.close()
    entry = {"shape": best, "ms_per_emcs": best_ms, "default_ms_per_emcs": base,
             "tried": len(results)}
    if use_cache:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        cache[key] = entry
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    return best


def tuned_batch(cfg: BatchConfig, **kw) -> Batch:
    """A batch with the autotuned shape applied."""
    shape = autotune(cfg, device=kw.get("device", "cuda"))
    b = Batch(cfg, **kw)
    if shape:
        b.set_tuning(**shape)
    return b


def autotune_schedule(cfg: BatchConfig, intervals=(1, 2, 4, 8), max_cluster_share: float = 0.10,
                      emcs: int = 8, warm_emcs: int = 8, device="cuda"):
    """Cluster-move schedule by cost balance.

    The paper fixes its EMCS (10 local sweeps per cluster move, PT and ER
    step) from a balance between the costs of the steps (Sec. 3).  Here the
    interval between cluster moves (acu_interval, in EMCS) is chosen the same
    way on this GPU: every candidate is timed on a warmed scratch batch (CUDA
    events around the sweep and the cluster launches of each EMCS), and the
    smallest interval whose cluster step takes at most max_cluster_share of
    the EMCS time is returned with the measured table.  The interval changes
    the Markov chain, not only its speed, so it is a recommendation that the
    caller applies through BatchConfig.acu_interval.
    """
    import torch
    rng = np.random.default_rng(1)
    J = (np.rint(rng.standard_normal((cfg.n_samples, 3, cfg.L ** 3)) * 2 ** 18) / 2 ** 18).astype(np.float32)
    table = []
    for k in intervals:
        c = BatchConfig(**{**cfg.__dict__, "acu_interval": int(k)})
        st = torch.cuda.Stream(device)
        b = Batch(c, couplings=J, device=device, stream=st)
        if c.er_on and c.n_res:
            b.prethermalize(960)
        b.emcs(warm_emcs)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        sw = cl = tot = 0.0
        with torch.cuda.stream(st):
            for _ in range(emcs):
                ev[0].record(st)
                b.sweep(c.sweeps_per_emcs, c.res_sweeps_per_emcs if c.er_on else 0)
                ev[1].record(st)
                b.houdayer()
                ev[2].record(st)
                b.swap(True, c.er_on)
                b.measure()
                ev[3].record(st)
                st.synchronize()
                sw += ev[0].elapsed_time(ev[1])
                cl += ev[1].elapsed_time(ev[2])
                tot += ev[0].elapsed_time(ev[3])
        table.append({"acu_interval": int(k), "ms_per_emcs": tot / emcs, "cluster_ms_per_emcs": cl / emcs,
                      "sweep_ms_per_emcs": sw / emcs, "cluster_share": cl / tot})
        b.close()
    chosen = intervals[-1]
    for row in table:
        if row["cluster_share"] <= max_cluster_share:
            chosen = row["acu_interval"]
            break
    return chosen, table


def autotune_spin_layout(cfg: BatchConfig, emcs: int = 4, warm_emcs: int = 4, device="cuda",
                         memory_weight: float = 0.0):
    """Spin storage for cfg: times whole EMCS with the spins stored as bytes
    and as bits (same couplings and seeds, so the same trajectory) and returns
    (layout, table).  The layout is fixed when a batch is created, so this is
    a recommendation for BatchConfig.spin_layout.  With memory_weight > 0 the
    bit layout wins unless it is slower by more than that fraction (its
    workspace holds 8x fewer spin bytes: more resident samples per GB)."""
    import torch
    rng = np.random.default_rng(2)
    J = (np.rint(rng.standard_normal((cfg.n_samples, 3, cfg.L ** 3)) * 2 ** 18) / 2 ** 18).astype(np.float32)
    table = {}
    for layout in ("bytes", "bits"):
        c = BatchConfig(**{**cfg.__dict__, "spin_layout": layout})
        st = torch.cuda.Stream(device)
        b = Batch(c, couplings=J, device=device, stream=st)
        b.emcs(warm_emcs)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            b.emcs(emcs)
            e1.record(st)
        st.synchronize()
        table[layout] = {"ms_per_emcs": e0.elapsed_time(e1) / emcs, "workspace_bytes": b.nbytes}
        b.close()
    fast = table["bits"]["ms_per_emcs"] <= table["bytes"]["ms_per_emcs"] * (1.0 + memory_weight)
    return ("bits" if fast else "bytes"), table
