"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Inputs (couplings, seeds, spin configurations) come from ``workloads``; every
expected value comes from ``oracle``.  Trajectory parity: with shared Philox
counters the spins must match bit for bit, except where a Metropolis/heat-bath
decision had an oracle margin |u - p| < 1e-6 (a near tie, counted); such a
divergence is resynchronised by pushing the oracle state into the GPU.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from mirror import Mirror, explained_by_ties

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402

TIE_RATE_MAX = 1e-5
# near ties and decisions of every sweep-parity run in this module, pooled:
# the 1e-5 rate bound is checked on each run large enough to resolve it
# (>= 1e6 decisions) and on the pool (test_pooled_near_tie_rate)
TIE_LEDGER = {"ties": 0, "decisions": 0}


def record_ties(mir):
    TIE_LEDGER["ties"] += mir.n_ties
    TIE_LEDGER["decisions"] += mir.decisions
    if mir.decisions >= 1_000_000:
        assert mir.n_ties < TIE_RATE_MAX * mir.decisions, (mir.n_ties, mir.decisions)


def assert_explained(L, g, o, ties, it):
    """Every (sample, lattice) whose spins differ had near ties in this call,
    and every differing site is a tie site or (first colour) its neighbour."""
    bad = np.argwhere(g != o)
    for s, lat in {(int(a), int(b)) for a, b, _ in bad}:
        sites = bad[(bad[:, 0] == s) & (bad[:, 1] == lat)][:, 2]
        assert (s, lat) in ties and explained_by_ties(L, sites, ties[(s, lat)]), \
            f"call {it}: sample {s} lattice {lat} differs at {sites[:10]} without a near tie"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


def make(cfg: BatchConfig, seed=7, on_grid=True, couplings="input", field_err_bound=False):
    seeds = W.sample_seeds(W.SEED_BASE + seed, cfg.n_samples)
    if couplings == "input":
        J = W.gaussian_couplings(cfg.L, cfg.n_samples, seed, on_grid=on_grid)
        gpu = Batch(cfg, couplings=J, seeds=seeds)
    else:
        J = np.stack([O.couplings_from_seed(cfg.L, int(s)) for s in seeds]).astype(np.float32)
        gpu = Batch(cfg, couplings=None, seeds=seeds)
    mir = Mirror(cfg, J, seeds, field_err_bound=field_err_bound)
    return gpu, mir


def gpu_spins(gpu):
    return gpu.export_spins().cpu().numpy()


def resync(gpu, mir):
    """Push the oracle state into the GPU (spins, permutations, ages, round-trip
    state and counters); energies are recomputed by the import."""
    gpu.perm.copy_(torch.from_numpy(mir.perms().astype(np.int32)))
    if mir.cfg.n_res:
        gpu.age.copy_(torch.from_numpy(mir.ages().astype(np.int32)))
    gpu.rt_state.copy_(torch.from_numpy(np.stack([s.rt_state for s in mir.samples])))
    gpu.round_trips.copy_(torch.from_numpy(np.stack([s.round_trips for s in mir.samples])))
    gpu.pt_accepted.copy_(torch.from_numpy(
        np.stack([s.pt_accepted for s in mir.samples]).reshape(gpu.pt_accepted.shape)))
    gpu.import_spins(torch.from_numpy(mir.spins()))


def check_sweep_parity(gpu, mir, n_calls, n_pt=1, n_res=1):
    """Sweep both sides call by call; returns (near ties that changed the
    trajectory, oracle decisions).  The near-tie count itself must stay below
    1e-5 of the decisions (record_ties)."""
    assert n_pt <= 1 and n_res <= 1   # one sweep per call: tie explanations are local
    diverged = 0
    for it in range(n_calls):
        gpu.sweep(n_pt, n_res)
        ties = mir.sweep(n_pt, n_res)
        g = gpu_spins(gpu)
        o = mir.spins()
        if not np.array_equal(g, o):
            assert_explained(mir.L, g, o, ties, it)
            diverged += 1
            resync(gpu, mir)
        else:
            np.testing.assert_array_equal(gpu.energies.cpu().numpy(), mir.energies())
    record_ties(mir)
    return diverged, mir.decisions


# ----------------------------------------------------------------------------- a1

def test_couplings_from_seed_match_oracle():
    cfg = BatchConfig(L=8, n_samples=6, n_temps=4, n_replicas=2, n_res=2, cluster="acu")
    gpu, mir = make(cfg, couplings="seed")
    Jg = gpu.J.cpu().numpy()
    Jo = np.stack([s.J for s in mir.samples])
    diff = Jg.astype(np.float64) != Jo
    # FP64 libm and CUDA math may differ in the last bit before the 2^-18 rounding
    assert diff.sum() <= 2
    assert np.all(np.abs(Jg.astype(np.float64) - Jo)[diff] <= 2.0 ** -18)


@pytest.mark.parametrize("L,n_temps,t_min,t_max", [(6, 13, 0.2, 1.6), (10, 7, 0.35, 2.0)])
def test_creation_tables_match_their_definitions(L, n_temps, t_min, t_max):
    """The creation-time tables equal, bit for bit, the oracle's temperature
    grid and 1/T_k, the IEEE quotients (V - 2n)/V and (3V - 2n)/(3V), and the
    FP32 sweep factor -2 log2(e) / T_k."""
    from paper_2605_25872_gb300 import _lib, buffer_info
    cfg = BatchConfig(L=L, n_samples=1, n_temps=n_temps, n_replicas=2, n_res=1, t_min=t_min,
                      t_max=t_max)
    gpu = Batch(cfg)
    off, n = buffer_info(cfg, _lib.BUF_TABLES)
    raw = gpu.ws[off:off + n].cpu().numpy()
    V, NT = cfg.V, n_temps
    nd = 2 * NT + 4 * V + 2
    d = raw[:8 * nd].view(np.float64)
    tb = raw[8 * nd:8 * nd + 4 * NT].view(np.float32)
    T, beta = O.temperatures(NT, t_min, t_max)
    np.testing.assert_array_equal(d[:NT], T)
    np.testing.assert_array_equal(d[NT:2 * NT], beta)
    m = np.arange(V + 1, dtype=np.float64)
    np.testing.assert_array_equal(d[2 * NT:2 * NT + V + 1], (V - 2 * m) / float(V))
    m3 = np.arange(3 * V + 1, dtype=np.float64)
    np.testing.assert_array_equal(d[2 * NT + V + 1:nd], (3 * V - 2 * m3) / (3.0 * V))
    np.testing.assert_array_equal(tb, ((-2.0 * 1.4426950408889634073599) / T).astype(np.float32))


@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 12, 16])
def test_init_state_matches_oracle(L):
    cfg = BatchConfig(L=L, n_samples=3, n_temps=5, n_replicas=4, n_res=3)
    gpu, mir = make(cfg, seed=L)
    np.testing.assert_array_equal(gpu_spins(gpu), mir.spins())
    np.testing.assert_array_equal(gpu.energies.cpu().numpy(), mir.energies())
    np.testing.assert_array_equal(gpu.perm.cpu().numpy(), mir.perms())
    np.testing.assert_array_equal(gpu.age.cpu().numpy(), mir.ages())


# ----------------------------------------------------------------------------- a2/a3/a4

@pytest.mark.parametrize("L,rule", [(2, "metropolis"), (4, "metropolis"), (6, "metropolis"),
                                    (8, "metropolis"), (10, "metropolis"), (12, "metropolis"),
                                    (14, "metropolis"), (16, "metropolis"), (18, "metropolis"),
                                    (20, "metropolis"), (22, "metropolis"), (24, "metropolis"),
                                    (8, "heatbath"), (6, "heatbath"), (18, "heatbath")])
def test_sweep_trajectory_parity(L, rule):
    cfg = BatchConfig(L=L, n_samples=2, n_temps=6, n_replicas=2, n_res=2, rule=rule,
                      t_min=0.2, t_max=1.6)
    gpu, mir = make(cfg, seed=100 + L)
    n = 150 if L < 12 else (60 if L <= 16 else 12)
    diverged, decisions = check_sweep_parity(gpu, mir, n)
    assert diverged <= max(1, TIE_RATE_MAX * decisions)
    if diverged == 0:
        np.testing.assert_array_equal(gpu.flips.cpu().numpy(), np.stack([s.flips for s in mir.samples]))


@pytest.mark.parametrize("L", [2, 4, 6, 8, 12, 16, 18])
def test_micsa_sweep_trajectory_parity(L):
    """MicSA (App. A.1): walkers per (clone, group, colour pass) keyed by the
    clone's position; bit-exact against the oracle up to counted near ties."""
    cfg = BatchConfig(L=L, n_samples=2, n_temps=6, n_replicas=2, n_res=2, rule="micsa",
                      t_min=0.2, t_max=1.6)
    gpu, mir = make(cfg, seed=400 + L)
    n = 100 if L < 12 else (40 if L <= 16 else 10)
    diverged, decisions = check_sweep_parity(gpu, mir, n)
    assert diverged <= max(1, TIE_RATE_MAX * decisions)
    if diverged == 0:
        np.testing.assert_array_equal(gpu.flips.cpu().numpy(), np.stack([s.flips for s in mir.samples]))


def test_sweep_parity_1000_sweeps_plain_config():
    """Config 1 shape (L=4, 12 temperatures, 4 replicas + 4 reservoir clones):
    10^3 sweeps of every clone, bit-exact up to counted near ties."""
    cfg = BatchConfig(L=4, n_samples=1, n_temps=12, n_replicas=4, n_res=4)
    gpu, mir = make(cfg, seed=1)
    diverged, decisions = check_sweep_parity(gpu, mir, 1000)
    assert diverged <= max(1, TIE_RATE_MAX * decisions)


def test_multi_sweep_launch_matches_single_sweeps():
    """Ten sweeps in one launch (shared-memory resident) equal the oracle's ten."""
    cfg = BatchConfig(L=8, n_samples=3, n_temps=8, n_replicas=4, n_res=2)
    gpu, mir = make(cfg, seed=5)
    for it in range(5):
        gpu.sweep(10, 24)
        ties = mir.sweep(10, 24)
        g, o = gpu_spins(gpu), mir.spins()
        if not np.array_equal(g, o):
            bad = {(int(a), int(b)) for a, b, _ in np.argwhere(g != o)}
            assert bad <= set(ties), "divergence without a near tie"
            resync(gpu, mir)
        else:
            np.testing.assert_array_equal(gpu.energies.cpu().numpy(), mir.energies())


def test_offgrid_couplings_parity_with_fp32_error_margin():
    """Couplings off the 2^-18 grid: the FP32 field is rounded, so the near-tie
    margin adds the FP32 error bound of the field (oracle, field_err_bound)."""
    cfg = BatchConfig(L=8, n_samples=2, n_temps=6, n_replicas=2, n_res=2)
    gpu, mir = make(cfg, seed=77, on_grid=False, field_err_bound=True)
    L = cfg.L
    diverged = 0
    for it in range(100):
        gpu.sweep(1, 1)
        ties = mir.sweep(1, 1)
        g, o = gpu_spins(gpu), mir.spins()
        bad = np.argwhere(g != o)
        if len(bad):
            for s, lat in {(int(a), int(b)) for a, b, _ in bad}:
                sites = bad[(bad[:, 0] == s) & (bad[:, 1] == lat)][:, 2]
                assert (s, lat) in ties and explained_by_ties(L, sites, ties[(s, lat)])
            diverged += 1
            resync(gpu, mir)
        else:
            np.testing.assert_allclose(gpu.energies.cpu().numpy(), mir.energies(), rtol=1e-9, atol=1e-9)
    assert diverged <= 5


# ----------------------------------------------------------------------------- a5/a6

@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 12, 16, 18, 24])
def test_cluster_labels_bit_exact(L):
    cfg = BatchConfig(L=L, n_samples=2, n_temps=5, n_replicas=4, n_res=1)
    gpu, mir = make(cfg, seed=30 + L)
    spins = W.random_spins((cfg.n_samples, cfg.n_lat, cfg.V), 1000 + L)
    spins[0, 0] = spins[0, cfg.n_slot]           # pair 0 at T_0: every q_i = +1
    gpu.import_spins(torch.from_numpy(spins))
    lab = gpu.cluster_labels().cpu().numpy()
    for s in range(cfg.n_samples):
        for p in range(cfg.n_replicas // 2):
            for k in range(cfg.n_temps):
                la = (2 * p) * cfg.n_slot + k
                lb = (2 * p + 1) * cfg.n_slot + k
                ref, _ = O.cc_labels(L, spins[s, la], spins[s, lb])
                np.testing.assert_array_equal(lab[s, p, k], ref)


@pytest.mark.parametrize("mode", ["acu", "single"])
@pytest.mark.parametrize("L", [4, 8, 12, 16])
def test_cluster_move_parity(mode, L):
    cfg = BatchConfig(L=L, n_samples=3, n_temps=8, n_replicas=4, n_res=2, cluster=mode)
    gpu, mir = make(cfg, seed=60 + L)
    spins = W.random_spins((cfg.n_samples, cfg.n_lat, cfg.V), 2000 + L)
    gpu.import_spins(torch.from_numpy(spins))
    for s, smp in enumerate(mir.samples):
        smp.spins[:] = spins[s]
        for lat in range(cfg.n_lat):
            smp.E_lat[lat] = O.energy(L, smp.J, smp.spins[lat])
    for rep in range(3):
        gpu.houdayer()
        stats = mir.houdayer()
        np.testing.assert_array_equal(gpu_spins(gpu), mir.spins())
        np.testing.assert_array_equal(gpu.energies.cpu().numpy(), mir.energies())
        cs = gpu.cluster_stats.cpu().numpy()
        for (s, p, k), (lab, n) in stats.items():
            if mode == "acu":
                assert cs[s, p, k, 0] == n
                sizes = np.sort(np.bincount(lab))[::-1]
                assert cs[s, p, k, 1] == sizes[0]
                assert cs[s, p, k, 2] == (sizes[1] if len(sizes) > 1 and sizes[1] > 0 else 0)
            else:
                assert cs[s, p, k, 3] == n
        gpu.swap(pt=False, er=False)      # next EMCS index: new random signs
        mir.swap(pt=False, er=False)


@pytest.mark.parametrize("kind", ["offgrid", "wide"])
def test_cluster_move_energies_outside_the_exact_grid(kind):
    """Cluster moves with couplings off the 2^-18 grid (both energies are
    recomputed and reduced in FP64: within 1e-9 of the oracle) and with on-grid
    couplings up to |J| = 32 (the sweep's energies take the FP64 path, the
    cluster step's cut-bond update stays exact: equal to the oracle)."""
    L = 8
    cfg = BatchConfig(L=L, n_samples=3, n_temps=8, n_replicas=4, n_res=2, cluster="acu")
    seeds = W.sample_seeds(W.SEED_BASE + 71, cfg.n_samples)
    if kind == "offgrid":
        J = W.gaussian_couplings(L, cfg.n_samples, 71, on_grid=False)
    else:
        J = (W.gaussian_couplings(L, cfg.n_samples, 71, on_grid=True) * 4.0).astype(np.float32)
    gpu = Batch(cfg, couplings=J, seeds=seeds)
    mir = Mirror(cfg, J, seeds)
    spins = W.random_spins((cfg.n_samples, cfg.n_lat, cfg.V), 2071)
    gpu.import_spins(torch.from_numpy(spins))
    for s, smp in enumerate(mir.samples):
        smp.spins[:] = spins[s]
        for lat in range(cfg.n_lat):
            smp.E_lat[lat] = O.energy(L, smp.J, smp.spins[lat])
    for rep in range(3):
        gpu.houdayer()
        mir.houdayer()
        np.testing.assert_array_equal(gpu_spins(gpu), mir.spins())
        Eg, Eo = gpu.energies.cpu().numpy(), mir.energies()
        if kind == "offgrid":
            np.testing.assert_allclose(Eg, Eo, rtol=1e-9, atol=1e-9)
        else:
            np.testing.assert_array_equal(Eg, Eo)
        gpu.swap(pt=False, er=False)
        mir.swap(pt=False, er=False)


# ----------------------------------------------------------------------------- a7/a8/a9 and full EMCS

def diverged_samples(gpu, mir):
    g = gpu_spins(gpu)
    bad = {int(a) for a, _, _ in np.argwhere(g != mir.spins())}
    bad |= {int(a) for a in np.argwhere((gpu.perm.cpu().numpy() != mir.perms()).any(axis=(1, 2))).ravel()}
    return bad


def run_emcs_parity(cfg, n_emcs, seed, switch=None):
    """switch = (EMCS index, rule): both sides change the local update rule
    there (the paper's PTHR*: Metropolis early, MicSA late)."""
    gpu, mir = make(cfg, seed=seed)
    resyncs = 0
    for e in range(n_emcs):
        if switch is not None and e == switch[0]:
            gpu.set_rule(switch[1])
            mir.rule = {"metropolis": O.RULE_METROPOLIS, "heatbath": O.RULE_HEATBATH,
                        "micsa": O.RULE_MICSA}[switch[1]]
        gpu.sweep(cfg.sweeps_per_emcs, cfg.res_sweeps_per_emcs if cfg.er_on else 0)
        if cfg.cluster != "off":
            gpu.houdayer()
        gpu.swap(True, cfg.er_on)
        gpu.measure()
        ties, pt_ties = mir.emcs()
        bad_samples = diverged_samples(gpu, mir)
        if bad_samples:
            # a near tie of a sample (local or PT) may change that sample only
            tie_samples = {s for s, _ in ties} | set(pt_ties)
            assert bad_samples <= tie_samples, \
                f"EMCS {e}: samples {bad_samples - tie_samples} diverged without a near tie of their own"
            resyncs += 1
            resync(gpu, mir)
            gpu.obs.copy_(torch.from_numpy(np.stack([s.obs for s in mir.samples])))
            continue
        np.testing.assert_array_equal(gpu.energies.cpu().numpy(), mir.energies())
        if cfg.n_res:
            np.testing.assert_array_equal(gpu.age.cpu().numpy(), mir.ages())
        np.testing.assert_array_equal(gpu.rt_state.cpu().numpy(), np.stack([s.rt_state for s in mir.samples]))
        np.testing.assert_array_equal(gpu.round_trips.cpu().numpy(), np.stack([s.round_trips for s in mir.samples]))
        np.testing.assert_array_equal(gpu.pt_accepted.cpu().numpy().reshape(cfg.n_samples, -1),
                                      np.stack([s.pt_accepted for s in mir.samples]))
        np.testing.assert_array_equal(gpu.obs.cpu().numpy(), np.stack([s.obs for s in mir.samples]))
        assert np.all(gpu.emcs_counter.cpu().numpy() == e + 1)
    record_ties(mir)
    return gpu, mir, resyncs


def test_full_emcs_parity_plain_config():
    """Config 1: L=4, 1 sample, 12 temperatures 0.2..1.6, 4 replicas (2
    Houdayer pairs) + 4 reservoir clones with 240 sweeps, 1 local sweep + ACU
    + PT + ER per EMCS; spins, permutations, energies, ages, round trips, PT
    counters and observable accumulators bit-exact."""
    cfg = BatchConfig(L=4, n_samples=1, n_temps=12, n_replicas=4, n_res=4, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=240)
    gpu, mir, resyncs = run_emcs_parity(cfg, 150, seed=1)
    assert resyncs <= 2
    assert mir.samples[0].pt_accepted.sum() > 0


@pytest.mark.parametrize("cluster,rule,er", [("acu", "metropolis", True), ("single", "metropolis", True),
                                             ("acu", "heatbath", False), ("off", "metropolis", False),
                                             ("acu", "micsa", True)])
def test_full_emcs_parity_batched(cluster, rule, er):
    cfg = BatchConfig(L=8, n_samples=4, n_temps=8, n_replicas=4, n_res=2 if er else 0,
                      sweeps_per_emcs=2, res_sweeps_per_emcs=6, er_on=er, cluster=cluster, rule=rule)
    gpu, mir, resyncs = run_emcs_parity(cfg, 40, seed=11)
    assert resyncs <= 2


def test_update_rule_switch_at_an_emcs_boundary():
    """PTHR*: Metropolis for 12 EMCS, then MicSA, against the oracle doing the
    same; the switch is refused inside an EMCS."""
    from paper_2605_25872_gb300 import _lib
    cfg = BatchConfig(L=8, n_samples=3, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=6)
    gpu, mir, resyncs = run_emcs_parity(cfg, 24, seed=77, switch=(12, "micsa"))
    assert resyncs <= 2 and gpu.cfg.rule == "micsa"
    gpu.sweep(1, 0)
    with pytest.raises(_lib.PthrError) as err:
        gpu.set_rule("metropolis")
    assert err.value.status == _lib.PTHR_E_STATE


def test_acu_interval_and_threshold():
    cfg = BatchConfig(L=6, n_samples=2, n_temps=10, n_replicas=2, n_res=2, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=3, acu_interval=3, acu_t_below=0.9)
    run_emcs_parity(cfg, 12, seed=3)


# ----------------------------------------------------------------------------- batch-level properties

def _state(gpu):
    return (gpu_spins(gpu), gpu.perm.cpu().numpy().copy(), gpu.energies.cpu().numpy().copy(),
            gpu.obs.cpu().numpy().copy())


def _same(a, b):
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_graph_replay_equals_direct_launches():
    cfg = BatchConfig(L=8, n_samples=6, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=3,
                      res_sweeps_per_emcs=5)
    J = W.gaussian_couplings(8, 6, 3)
    seeds = W.sample_seeds(99, 6)
    s = torch.cuda.Stream()
    a = Batch(cfg, couplings=J, seeds=seeds, stream=s)
    b = Batch(cfg, couplings=J, seeds=seeds, stream=s)
    a.emcs(7, graph=False)
    b.emcs(7, graph=True)
    s.synchronize()
    _same(_state(a), _state(b))


def test_tuning_does_not_change_results():
    cfg = BatchConfig(L=8, n_samples=3, n_temps=8, n_replicas=4, n_res=4, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=4)
    J = W.gaussian_couplings(8, 3, 4)
    seeds = W.sample_seeds(5, 3)
    ref = Batch(cfg, couplings=J, seeds=seeds)
    ref.emcs(5)
    for t in ({"pt_lattices_per_block": 1, "res_lattices_per_block": 3},
              {"pt_lattices_per_block": 7, "sweep_threads": 64, "cluster_threads": 128},
              {"pt_lattices_per_block": 32, "res_lattices_per_block": 16, "sweep_threads": 256}):
        b = Batch(cfg, couplings=J, seeds=seeds, tuning=t)
        b.emcs(5)
        _same(_state(ref), _state(b))
    # MicSA draws one Philox call per four positions: also independent of the shape
    cm = BatchConfig(**{**cfg.__dict__, "rule": "micsa"})
    ref = Batch(cm, couplings=J, seeds=seeds)
    ref.emcs(5)
    for t in ({"pt_lattices_per_block": 3, "res_lattices_per_block": 5}, {"pt_lattices_per_block": 13}):
        b = Batch(cm, couplings=J, seeds=seeds, tuning=t)
        b.emcs(5)
        _same(_state(ref), _state(b))


def test_save_load_resume_is_exact():
    cfg = BatchConfig(L=6, n_samples=3, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=4)
    J = W.gaussian_couplings(6, 3, 8)
    seeds = W.sample_seeds(8, 3)
    full = Batch(cfg, couplings=J, seeds=seeds)
    full.emcs(10)
    half = Batch(cfg, couplings=J, seeds=seeds)
    half.emcs(5)
    blob = half.save()
    again = Batch(cfg, couplings=J, seeds=seeds)
    again.load(blob)
    again.emcs(5)
    _same(_state(full), _state(again))


def test_sample_result_is_independent_of_slot_and_neighbours():
    """Serving property: a sample reset into any slot of a busy batch evolves
    exactly as it does alone (counter-based random numbers keyed by its seed)."""
    cfg1 = BatchConfig(L=6, n_samples=1, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                       res_sweeps_per_emcs=4)
    cfg4 = BatchConfig(**{**cfg1.__dict__, "n_samples": 4})
    J = W.gaussian_couplings(6, 4, 12)
    alone = Batch(cfg1, couplings=J[2:3], seeds=[777])
    alone.prethermalize(8)
    alone.emcs(6)
    mixed = Batch(cfg4, couplings=J, seeds=W.sample_seeds(1, 4))
    mixed.emcs(3)
    mixed.reset_samples(2, 1, seeds=[777], couplings=J[2:3], pretherm_sweeps=8)
    mixed.emcs(6)
    np.testing.assert_array_equal(gpu_spins(mixed)[2], gpu_spins(alone)[0])
    np.testing.assert_array_equal(mixed.obs.cpu().numpy()[2], alone.obs.cpu().numpy()[0])
    np.testing.assert_array_equal(mixed.energies.cpu().numpy()[2], alone.energies.cpu().numpy()[0])


def test_idle_slots_are_untouched():
    cfg = BatchConfig(L=6, n_samples=3, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=2)
    b = Batch(cfg, couplings=W.gaussian_couplings(6, 3, 1), seeds=W.sample_seeds(2, 3))
    before = gpu_spins(b)[1].copy()
    b.set_active(1, 1, False)
    b.emcs(4)
    after = gpu_spins(b)
    np.testing.assert_array_equal(after[1], before)
    assert b.emcs_counter.cpu().numpy().tolist() == [4, 0, 4]


def test_prethermalisation_matches_oracle():
    """Reservoir pre-thermalisation one sweep per call: the sweep index
    continues from call to call, so 30 calls of one sweep are the oracle's 30
    sweeps.  A divergence must be explained by a near tie of that call, and
    the GPU is then resynchronised."""
    cfg = BatchConfig(L=6, n_samples=2, n_temps=4, n_replicas=2, n_res=3)
    gpu, mir = make(cfg, seed=44)
    for it in range(30):
        gpu.prethermalize(1)
        ties = mir.sweep(0, 1, pretherm=True)
        g, o = gpu_spins(gpu), mir.spins()
        if not np.array_equal(g, o):
            assert_explained(cfg.L, g, o, ties, it)
            resync(gpu, mir)
        else:
            np.testing.assert_array_equal(gpu.energies.cpu().numpy(), mir.energies())
    record_ties(mir)
    assert gpu.poll(10000) == 0


def test_prethermalisation_continues_the_sweep_index():
    """Two pre-thermalisation calls of n sweeps equal one call of 2n (fresh
    random numbers, no replay), and a reset restarts the index."""
    cfg = BatchConfig(L=6, n_samples=2, n_temps=4, n_replicas=2, n_res=3)
    J = W.gaussian_couplings(6, 2, 45)
    seeds = W.sample_seeds(W.SEED_BASE + 45, 2)
    a = Batch(cfg, couplings=J, seeds=seeds)
    b = Batch(cfg, couplings=J, seeds=seeds)
    a.prethermalize(10)
    a.prethermalize(10)
    b.prethermalize(20)
    np.testing.assert_array_equal(gpu_spins(a), gpu_spins(b))
    c = Batch(cfg, couplings=J, seeds=seeds)
    c.prethermalize(10)
    c.reset_samples(0, 2, seeds=seeds, couplings=J, pretherm_sweeps=10)
    d = Batch(cfg, couplings=J, seeds=seeds)
    d.prethermalize(10)
    np.testing.assert_array_equal(gpu_spins(c), gpu_spins(d))
    assert not np.array_equal(gpu_spins(a), gpu_spins(d))


# ----------------------------------------------------------------------------- statistics

def test_gpu_chain_reproduces_exact_enumeration_2x2x2():
    """The GPU PTHR chain at L=2 (64 samples of one coupling set, different
    seeds) samples the Boltzmann weight: <e>, <q^2>, <q_l>, <S> per
    temperature within 5 standard errors of exact enumeration."""
    L, S, NT = 2, 64, 4
    J1 = W.gaussian_couplings(L, 1, 5)[0]
    J = np.repeat(J1[None], S, axis=0)
    cfg = BatchConfig(L=L, n_samples=S, n_temps=NT, t_min=0.4, t_max=1.6, n_replicas=4, n_res=4,
                      sweeps_per_emcs=1, res_sweeps_per_emcs=3)
    b = Batch(cfg, couplings=J, seeds=W.sample_seeds(321, S))
    b.emcs(100)
    b.reset_observables()
    b.emcs(2000, graph=False)
    obs = b.read_observables()
    n = obs[:, :, 0:1]
    per = np.stack([obs[:, :, 1] / (n[:, :, 0] * 4), obs[:, :, 4] / (n[:, :, 0] * 2),
                    obs[:, :, 5] / (n[:, :, 0] * 2), obs[:, :, 6] / (n[:, :, 0] * 2)], -1)
    est = per.mean(0)
    err = per.std(0, ddof=1) / np.sqrt(S)
    T, _ = O.temperatures(NT, 0.4, 1.6)
    exact = O.enumerate_l2(J1.astype(np.float64), T)[:, [0, 1, 2, 3]]
    z = np.abs(est - exact) / np.maximum(err, 1e-9)
    assert np.all(z < 5.0), z


def test_status_word_reads_ok():
    cfg = BatchConfig(L=8, n_samples=2, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=2)
    b = Batch(cfg, couplings=W.gaussian_couplings(8, 2, 1), seeds=W.sample_seeds(2, 2))
    b.emcs(3)
    assert b.poll(10000) == 0


def test_reservoir_autocorrelation_matches_oracle():
    """C(tau) at T_max (Sec. 3, ER): from a common state, the GPU's integer
    sums of s_i(t) s_i(t + tau) over every reservoir clone equal the oracle's,
    computed from its own snapshot and the same pre-thermalisation sweeps,
    for every sample whose oracle sweeps met no near tie."""
    cfg = BatchConfig(L=6, n_samples=4, n_temps=4, n_replicas=2, n_res=3)
    gpu, mir = make(cfg, seed=52)
    gpu.prethermalize(20)
    mir.sweep(0, 20, pretherm=True)
    resync(gpu, mir)                       # common starting point
    n_points, per = 4, 5
    got = gpu.reservoir_autocorrelation(n_points, per).cpu().numpy()
    snap = [np.stack([smp.spins[smp.lattice_at(g, cfg.n_temps + r)] for g in range(cfg.n_replicas)
                      for r in range(cfg.n_res)]).astype(np.int64) for smp in mir.samples]
    ref = np.zeros((cfg.n_samples, n_points), dtype=np.int64)
    tied = set()
    for p in range(n_points):
        ties = mir.sweep(0, per, pretherm=True)
        tied |= {s for s, _ in ties}
        for s, smp in enumerate(mir.samples):
            now = np.stack([smp.spins[smp.lattice_at(g, cfg.n_temps + r)] for g in range(cfg.n_replicas)
                            for r in range(cfg.n_res)]).astype(np.int64)
            ref[s, p] = int((snap[s] * now).sum())
    compared = [s for s in range(cfg.n_samples) if s not in tied]
    assert len(compared) >= 3
    np.testing.assert_array_equal(got[compared], ref[compared])
    assert np.all(np.abs(ref) <= cfg.n_replicas * cfg.n_res * cfg.V)
    assert gpu.poll(10000) == 0


def test_poll_times_out_while_a_long_launch_runs():
    """Failure detection on the host: pthr_poll(0) right after a long
    reservoir pre-thermalisation is enqueued returns PTHR_E_TIMEOUT without
    disturbing the stream; a later unbounded poll drains it and returns OK."""
    from paper_2605_25872_gb300 import _lib
    cfg = BatchConfig(L=16, n_samples=4, n_temps=4, n_replicas=2, n_res=4)
    b = Batch(cfg, couplings=W.gaussian_couplings(16, 4, 9), seeds=W.sample_seeds(10, 4))
    b.synchronize()
    b.prethermalize(20000)
    assert b.poll(0) == _lib.PTHR_E_TIMEOUT
    assert b.poll(-1) == _lib.PTHR_OK
    assert b.check_canaries() == -1


def test_guard_blocks_catch_a_write_past_a_buffer():
    """The guard block after a sub-buffer detects a write one byte past its
    end (made from the host through the workspace tensor: no kernel writes
    out of range)."""
    from paper_2605_25872_gb300 import _lib, buffer_info
    cfg = BatchConfig(L=6, n_samples=2, n_temps=4, n_replicas=2, n_res=1)
    b = Batch(cfg)
    assert b.check_canaries() == -1
    off, n = buffer_info(cfg, _lib.BUF_ENERGY)
    guard = off + ((n + 255) & ~255)
    saved = b.ws[guard].clone()
    b.ws[guard] = 0
    assert b.check_canaries() == _lib.BUF_ENERGY
    b.ws[guard] = saved
    assert b.check_canaries() == -1


def test_bounded_cluster_loop_reports_noconverge_without_changing_spins():
    """Failure detection without a fault: an iteration cap of 1 makes the
    union-find give up; the kernel latches PTHR_E_NOCONVERGE, returns, leaves
    the spins alone, and the context stays usable."""
    from paper_2605_25872_gb300 import _lib
    cfg = BatchConfig(L=8, n_samples=2, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=2)
    b = Batch(cfg, couplings=W.gaussian_couplings(8, 2, 3), seeds=W.sample_seeds(4, 2))
    b.sweep(3, 3)
    before = gpu_spins(b)
    e_before = b.energies.cpu().numpy().copy()
    b.set_tuning(cluster_iter_cap=1)
    b.houdayer()
    assert b.poll(10000) == _lib.PTHR_E_NOCONVERGE
    np.testing.assert_array_equal(gpu_spins(b), before)
    np.testing.assert_array_equal(b.energies.cpu().numpy(), e_before)
    b.set_tuning()
    b.houdayer()
    assert b.poll(10000) == 0


def test_autotuner_returns_a_valid_faster_or_default_shape():
    from paper_2605_25872_gb300.autotune import autotune
    cfg = BatchConfig(L=8, n_samples=8, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=4)
    shape = autotune(cfg, emcs=2, use_cache=False)
    J = W.gaussian_couplings(8, 8, 2)
    a = Batch(cfg, couplings=J, seeds=W.sample_seeds(3, 8))
    b = Batch(cfg, couplings=J, seeds=W.sample_seeds(3, 8), tuning=shape or None)
    a.emcs(3)
    b.emcs(3)
    _same(_state(a), _state(b))


def test_chaos_accumulators_match_oracle():
    """q^2 between the T_0 clone of group 2p and the T_k clone of group 2p+1,
    accumulated on the GPU, equals the oracle's overlap of the same clones."""
    cfg = BatchConfig(L=6, n_samples=2, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=1,
                      res_sweeps_per_emcs=2)
    gpu, mir = make(cfg, seed=21)
    ref = np.zeros((cfg.n_samples, cfg.n_temps, 2))
    for e in range(6):
        gpu.sweep(1, 2)
        gpu.houdayer()
        gpu.swap(True, True)
        gpu.measure(chaos=True)
        ties, pt_ties = mir.emcs()
        diverged = diverged_samples(gpu, mir)
        for s, smp in enumerate(mir.samples):
            for k in range(cfg.n_temps):
                for p in range(cfg.n_replicas // 2):
                    ref[s, k, 0] += 1.0
                    a = smp.spins[smp.lattice_at(2 * p, 0)]
                    bb = smp.spins[smp.lattice_at(2 * p + 1, k)]
                    q = O.pair_observables(cfg.L, smp.J, a, bb, 1.0)[0]
                    ref[s, k, 1] += q * q
        if diverged:
            # a near tie changed a trajectory: only that sample may differ;
            # continue from the oracle's state and accumulators
            assert diverged <= {s for s, _ in ties} | set(pt_ties)
            resync(gpu, mir)
            gpu.obs.copy_(torch.from_numpy(np.stack([s.obs for s in mir.samples])))
            gpu.chaos.copy_(torch.from_numpy(ref))
        np.testing.assert_array_equal(gpu.chaos.cpu().numpy(), ref)
    record_ties(mir)


def test_schedule_autotuner_reports_cluster_share():
    from paper_2605_25872_gb300.autotune import autotune_schedule
    cfg = BatchConfig(L=8, n_samples=8, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=4)
    k, table = autotune_schedule(cfg, intervals=(1, 4), emcs=4, warm_emcs=2)
    assert k in (1, 4) and len(table) == 2
    assert all(0.0 <= r["cluster_share"] < 1.0 for r in table)
    assert table[1]["cluster_ms_per_emcs"] < table[0]["cluster_ms_per_emcs"]


def test_pooled_near_tie_rate():
    """Near ties over every sweep-parity run of this module stay below 1e-5
    of the local decisions (the tolerance on FP32 vs FP64 accept decisions)."""
    if TIE_LEDGER["decisions"] == 0:
        pytest.skip("no parity run recorded in this session")
    assert TIE_LEDGER["ties"] < TIE_RATE_MAX * TIE_LEDGER["decisions"], TIE_LEDGER
