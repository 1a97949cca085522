"""Parity at the full sizes of the workloads, in the launch configuration
that bench.py times (default tuning), on sampled samples the oracle steps one
by one (a sample's trajectory does not depend on its slot)."""
import numpy as np
import pytest
import torch

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


def cfg_of(wl, cluster="acu"):
    return BatchConfig(L=wl.L, n_samples=wl.n_samples, n_temps=wl.n_temps, t_min=wl.t_min,
                       t_max=wl.t_max, n_replicas=wl.n_replicas, n_res=wl.n_res if wl.er_on else 0,
                       sweeps_per_emcs=wl.sweeps_per_emcs,
                       res_sweeps_per_emcs=wl.res_sweeps_per_emcs, er_on=wl.er_on, cluster=cluster)


def run_sampled(wl, n_emcs, picks):
    cfg = cfg_of(wl)
    J = W.gaussian_couplings(wl.L, wl.n_samples, W.batch_seed(wl.index))
    seeds = W.sample_seeds(W.batch_seed(wl.index), wl.n_samples)
    gpu = Batch(cfg, couplings=J, seeds=seeds)
    sub = BatchConfig(**{**cfg.__dict__, "n_samples": len(picks)})
    mir = Mirror(sub, J[picks], seeds[picks])
    ties_seen = set()
    if wl.res_pretherm_sweeps and wl.er_on:
        gpu.prethermalize(wl.res_pretherm_sweeps)
        t = mir.sweep(0, wl.res_pretherm_sweeps, pretherm=True)
        ties_seen |= {s for s, _ in t}
    for _ in range(n_emcs):
        gpu.emcs(1)
        ties, pt_ties = mir.emcs()
        ties_seen |= {s for s, _ in ties} | set(pt_ties)
    g = gpu.export_spins().cpu().numpy()[picks]
    o = mir.spins()
    gp = gpu.perm.cpu().numpy()[picks]
    ge = gpu.energies.cpu().numpy()[picks]
    gobs = gpu.obs.cpu().numpy()[picks]
    checked = 0
    for i in range(len(picks)):
        if i in ties_seen and not np.array_equal(g[i], o[i]):
            continue          # a counted near tie changed this trajectory
        np.testing.assert_array_equal(g[i], o[i])
        np.testing.assert_array_equal(gp[i], mir.perms()[i])
        np.testing.assert_array_equal(ge[i], mir.energies()[i])
        np.testing.assert_array_equal(gobs[i], mir.samples[i].obs)
        checked += 1
    assert checked >= len(picks) - 1
    assert gpu.poll(60000) == 0


def test_fullsize_pthr_L16_512_samples():
    """L=16, 512 samples x 32 T x 4 groups + reservoir, 960-sweep reservoir
    pre-thermalisation, one paper EMCS; samples 0, 257 and 511 checked."""
    run_sampled(W.WORKLOADS["c4"], 1, [0, 257, 511])


def test_fullsize_batched_L8_256_samples():
    run_sampled(W.WORKLOADS["c2"], 5, [0, 100, 255])


def test_fullsize_batched_L12_1024_samples():
    run_sampled(W.WORKLOADS["c3"], 3, [0, 700, 1023])
