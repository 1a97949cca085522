"""Edge cases of the configuration space against the FP64 oracle: the
smallest batch (L = 2, one sample, two temperatures, one replica group, no
cluster move, no reservoir), no temperature below the cluster-move cut, the
largest lattice (L = 24), ragged shapes that leave partial blocks
(7 samples, 13 temperatures, 3 reservoir clones), and a reset of a sample
range in the middle of a batch."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402

from test_gpu_parity import gpu_spins, make, run_emcs_parity  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


def test_smallest_batch():
    cfg = BatchConfig(L=2, n_samples=1, n_temps=2, n_replicas=1, n_res=0, er_on=False, cluster="off",
                      sweeps_per_emcs=3)
    gpu, mir, resyncs = run_emcs_parity(cfg, 60, seed=501)
    assert resyncs <= 1


def test_no_temperature_below_the_cluster_cut():
    """acu_t_below under T_min: the cluster step has no pair to move."""
    cfg = BatchConfig(L=6, n_samples=2, n_temps=5, n_replicas=4, n_res=2, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=3, acu_t_below=0.1)
    gpu, mir, resyncs = run_emcs_parity(cfg, 15, seed=502)
    assert resyncs <= 1
    assert int(gpu.cluster_stats.cpu().numpy().sum()) == 0


def test_largest_lattice_full_emcs():
    cfg = BatchConfig(L=24, n_samples=2, n_temps=4, n_replicas=4, n_res=1, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=2)
    gpu, mir, resyncs = run_emcs_parity(cfg, 3, seed=503)
    assert resyncs <= 1


@pytest.mark.parametrize("cluster", ["acu", "single"])
def test_ragged_shapes(cluster):
    cfg = BatchConfig(L=10, n_samples=7, n_temps=13, n_replicas=4, n_res=3, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=5, cluster=cluster)
    gpu, mir, resyncs = run_emcs_parity(cfg, 6, seed=504)
    assert resyncs <= 3          # each one explained by a near tie of that sample


def test_reset_of_a_middle_range_leaves_the_others_alone():
    cfg = BatchConfig(L=6, n_samples=5, n_temps=4, n_replicas=2, n_res=2, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=2)
    J = W.gaussian_couplings(6, 5, 505)
    seeds = W.sample_seeds(W.SEED_BASE + 505, 5)
    a = Batch(cfg, couplings=J, seeds=seeds)
    b = Batch(cfg, couplings=J, seeds=seeds)
    a.emcs(3)
    b.emcs(3)
    new_seeds = W.sample_seeds(W.SEED_BASE + 9505, 2)
    b.reset_samples(1, 2, seeds=new_seeds, couplings=W.gaussian_couplings(6, 2, 9505), pretherm_sweeps=4)
    a.emcs(2)
    b.emcs(2)
    ga, gb = gpu_spins(a), gpu_spins(b)
    for s in (0, 3, 4):
        np.testing.assert_array_equal(ga[s], gb[s])
        np.testing.assert_array_equal(a.obs.cpu().numpy()[s], b.obs.cpu().numpy()[s])
    assert b.emcs_counter.cpu().numpy().tolist() == [5, 2, 2, 5, 5]
    # the reset samples start like a fresh batch of those two samples
    c = Batch(BatchConfig(**{**cfg.__dict__, "n_samples": 2}), couplings=W.gaussian_couplings(6, 2, 9505),
              seeds=new_seeds)
    c.prethermalize(4)
    c.emcs(2)
    np.testing.assert_array_equal(gb[1:3], gpu_spins(c))
