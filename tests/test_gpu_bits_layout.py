"""GPU parity of the bit spin storage (spin_layout="bits", one bit per site
slot in the workspace).  The sweep and cluster kernels expand a lattice to
the byte layout in shared memory and pack it again on write-back; the
measurement, initialisation, import/export and autocorrelation kernels read
the bits directly.  Checked two ways: against the FP64 oracle on the same
inputs (as the byte layout is), and against the byte layout bit for bit --
both store the same spins, so every result must be identical.
"""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig, buffer_info  # noqa: E402
from paper_2605_25872_gb300 import _lib  # noqa: E402
from paper_2605_25872_gb300.batch import Group  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402
from test_gpu_parity import make, gpu_spins, run_emcs_parity  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


def bits(cfg: BatchConfig) -> BatchConfig:
    return dataclasses.replace(cfg, spin_layout="bits")


def pair(cfg: BatchConfig, seed: int):
    """The same samples (couplings, seeds) in both layouts, each batch on its
    own stream."""
    seeds = W.sample_seeds(W.SEED_BASE + seed, cfg.n_samples)
    J = W.gaussian_couplings(cfg.L, cfg.n_samples, seed)
    return (Batch(cfg, couplings=J, seeds=seeds, stream=torch.cuda.Stream()),
            Batch(bits(cfg), couplings=J, seeds=seeds, stream=torch.cuda.Stream()))


def assert_same_state(a: Batch, b: Batch):
    np.testing.assert_array_equal(a.export_spins().cpu().numpy(), b.export_spins().cpu().numpy())
    for name in ("energies", "perm", "age", "rt_state", "round_trips", "pt_accepted", "flips", "obs",
                 "emcs_counter", "cluster_stats", "chaos"):
        np.testing.assert_array_equal(getattr(a, name).cpu().numpy(), getattr(b, name).cpu().numpy(),
                                      err_msg=name)


def test_bit_storage_is_an_eighth_of_the_byte_storage():
    c = BatchConfig(L=16, n_samples=512, n_temps=32)
    assert buffer_info(bits(c), _lib.BUF_SPINS)[1] * 8 == buffer_info(c, _lib.BUF_SPINS)[1]
    b = Batch(bits(BatchConfig(L=12, n_samples=2, n_temps=4)))
    assert b.lattice_bytes() == 2 * 144 * 8 // 8


@pytest.mark.parametrize("L", [2, 4, 6, 12, 16])
def test_bits_init_state_matches_oracle(L):
    cfg = bits(BatchConfig(L=L, n_samples=3, n_temps=5, n_replicas=4, n_res=3))
    gpu, mir = make(cfg, seed=L)
    np.testing.assert_array_equal(gpu_spins(gpu), mir.spins())
    np.testing.assert_array_equal(gpu.energies.cpu().numpy(), mir.energies())


@pytest.mark.parametrize("L,cluster,rule,er", [(8, "acu", "metropolis", True), (6, "single", "heatbath", False),
                                               (12, "acu", "micsa", True), (4, "acu", "metropolis", True)])
def test_bits_full_emcs_parity(L, cluster, rule, er):
    """Spins, energies, permutations, ages, round trips, PT counters and the
    observable accumulators bit-exact against the oracle over whole EMCS."""
    cfg = bits(BatchConfig(L=L, n_samples=3, n_temps=8, n_replicas=4, n_res=2 if er else 0,
                           sweeps_per_emcs=2, res_sweeps_per_emcs=6, er_on=er, cluster=cluster, rule=rule))
    gpu, mir, resyncs = run_emcs_parity(cfg, 25, seed=40 + L)
    assert resyncs <= 2


@pytest.mark.parametrize("L,rule,cluster", [(6, "metropolis", "acu"), (12, "metropolis", "acu"),
                                            (16, "metropolis", "acu"), (10, "heatbath", "single"),
                                            (8, "micsa", "acu")])
def test_bits_equal_bytes_bit_for_bit(L, rule, cluster):
    cfg = BatchConfig(L=L, n_samples=3, n_temps=10, n_replicas=4, n_res=2, sweeps_per_emcs=3,
                      res_sweeps_per_emcs=12, rule=rule, cluster=cluster)
    a, b = pair(cfg, seed=70 + L)
    for x in (a, b):
        x.prethermalize(24)
        x.emcs(4)
        x.emcs(3, graph=True)
        x.measure(chaos=True)
        x.synchronize()
    assert_same_state(a, b)
    np.testing.assert_array_equal(a.cluster_labels().cpu().numpy(), b.cluster_labels().cpu().numpy())


def test_bits_import_export_round_trip_and_energies():
    cfg = bits(BatchConfig(L=12, n_samples=2, n_temps=4, n_replicas=2, n_res=1))
    gpu, mir = make(cfg, seed=5)
    spins = W.random_spins((cfg.n_samples, cfg.n_lat, cfg.V), 77)
    gpu.import_spins(torch.from_numpy(spins))
    np.testing.assert_array_equal(gpu_spins(gpu), spins)
    E = np.array([[O.energy(cfg.L, mir.samples[s].J, spins[s, lat]) for lat in range(cfg.n_lat)]
                  for s in range(cfg.n_samples)])
    np.testing.assert_array_equal(gpu.energies.cpu().numpy(), E)


def test_bits_reservoir_autocorrelation_equals_bytes():
    cfg = BatchConfig(L=8, n_samples=4, n_temps=6, n_replicas=4, n_res=4, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=8)
    a, b = pair(cfg, seed=91)
    for x in (a, b):
        x.prethermalize(32)
    ca = a.reservoir_autocorrelation(3, 16).cpu().numpy()
    cb = b.reservoir_autocorrelation(3, 16).cpu().numpy()
    np.testing.assert_array_equal(ca, cb)
    assert_same_state(a, b)


def test_group_of_mixed_layouts_equals_separate_batches():
    """A four-launch group whose batches use different layouts."""
    c6 = BatchConfig(L=6, n_samples=3, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                     res_sweeps_per_emcs=4)
    c8 = bits(BatchConfig(L=8, n_samples=2, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                          res_sweeps_per_emcs=4))
    g6, s6 = pair(c6, seed=3)
    g8, s8 = (Batch(c8, couplings=W.gaussian_couplings(8, 2, 4), seeds=W.sample_seeds(W.SEED_BASE + 4, 2),
                    stream=torch.cuda.Stream()) for _ in range(2))
    grp = Group([g6, g8])
    assert grp.launches_per_emcs == 4
    grp.emcs(5)
    grp.synchronize()
    s6.emcs(5)
    s8.emcs(5)
    for x in (s6, s8):
        x.synchronize()
    assert_same_state(g6, s6)
    assert_same_state(g8, s8)


def test_spin_layout_autotuner_times_both_layouts():
    from paper_2605_25872_gb300.autotune import autotune_spin_layout
    cfg = BatchConfig(L=8, n_samples=8, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=4)
    layout, table = autotune_spin_layout(cfg, emcs=2, warm_emcs=1)
    assert layout in ("bytes", "bits")
    assert table["bits"]["workspace_bytes"] < table["bytes"]["workspace_bytes"]
    assert all(t["ms_per_emcs"] > 0 for t in table.values())
    # any slowdown is accepted once memory counts for more than it
    assert autotune_spin_layout(cfg, emcs=1, warm_emcs=1, memory_weight=1e9)[0] == "bits"


def test_bits_reset_samples_and_checkpoint_equal_bytes():
    """The serving admission path (a slot becomes a new sample, pre-thermalised)
    and a checkpoint round trip in both layouts."""
    cfg = BatchConfig(L=12, n_samples=4, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=8)
    a, b = pair(cfg, seed=33)
    new_seeds = W.sample_seeds(W.SEED_BASE + 999, 2)
    new_J = W.gaussian_couplings(cfg.L, 2, 999)
    for x in (a, b):
        x.emcs(2)
        x.reset_samples(1, 2, seeds=new_seeds, couplings=new_J, pretherm_sweeps=16)
        x.emcs(2)
        x.synchronize()
    assert_same_state(a, b)
    blobs = [x.save() for x in (a, b)]
    for x in (a, b):
        x.emcs(3)
        x.synchronize()
    after = [x.export_spins().cpu().numpy() for x in (a, b)]
    np.testing.assert_array_equal(after[0], after[1])
    for x, blob in zip((a, b), blobs):
        x.load(blob)
        x.emcs(3)
        x.synchronize()
    # resume from the checkpoint repeats the same three EMCS exactly
    np.testing.assert_array_equal(a.export_spins().cpu().numpy(), after[0])
    np.testing.assert_array_equal(b.export_spins().cpu().numpy(), after[1])
    assert_same_state(a, b)
