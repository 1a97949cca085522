"""Serving on the GPU: requests of mixed L admitted into busy pools give the
same result as the same request run alone."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402
from paper_2605_25872_gb300.serve import PoolSpec, Request, Server  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


def alone(spec, req):
    cfg = BatchConfig(L=spec.L, n_samples=1, n_temps=spec.n_temps, t_min=spec.t_min,
                      t_max=spec.t_max, n_replicas=spec.n_replicas, n_res=spec.n_res,
                      sweeps_per_emcs=spec.sweeps_per_emcs,
                      res_sweeps_per_emcs=spec.res_sweeps_per_emcs, er_on=True, cluster="acu")
    b = Batch(cfg, couplings=None if req.couplings is None else req.couplings[None],
              seeds=[req.seed])
    b.prethermalize(spec.pretherm_sweeps)
    b.emcs(req.budget_emcs)
    return b.obs[0].cpu().numpy(), b.round_trips[0].cpu().numpy()


SPECS = [PoolSpec(L=6, slots=3, n_temps=8, sweeps_per_emcs=2, res_sweeps_per_emcs=6, pretherm_sweeps=12),
         PoolSpec(L=8, slots=2, n_temps=8, sweeps_per_emcs=2, res_sweeps_per_emcs=6, pretherm_sweeps=12)]


def mixed_requests():
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(10):
        L = 6 if i % 2 else 8
        cpl = W.gaussian_couplings(L, 1, 500 + i)[0] if i % 3 else None
        reqs.append(Request(rid=i, L=L, seed=9000 + i, budget_emcs=int(rng.integers(3, 9)),
                            arrival=0.0, couplings=cpl))
    return reqs


@pytest.mark.parametrize("max_chunk", [1, 64])
def test_serving_result_alone_equals_in_the_mix(max_chunk):
    srv = Server(SPECS, max_chunk=max_chunk)
    done = srv.run(mixed_requests(), realtime=False)
    assert len(done) == 10
    for r in done:
        spec = srv.specs[r.L]
        obs, trips = alone(spec, r)
        np.testing.assert_array_equal(r.obs, obs)
        np.testing.assert_array_equal(r.round_trips, trips)
    st = srv.stats()
    assert st["p50_s"] > 0 and st["updates_per_ns"] > 0
    if max_chunk > 1:
        assert sum(st["chunks"].values()) < sum(st["emcs_steps"].values())


def test_served_requests_match_the_oracle():
    """Requests served in a busy mixed-L pool (admitted as slots free up,
    advanced in chunks) against the FP64 oracle run on the same seed and
    couplings: reservoir pre-thermalisation then the request's EMCS budget.
    Every request whose oracle run met no near tie has bit-identical
    observable accumulators and round-trip counts."""
    srv = Server(SPECS, max_chunk=64)
    done = srv.run(mixed_requests(), realtime=False)
    compared = 0
    for r in done:
        if r.couplings is None:
            continue            # couplings drawn on the device (checked in test_gpu_parity)
        spec = srv.specs[r.L]
        o = O.OracleSample(r.L, spec.n_temps, spec.t_min, spec.t_max, r.seed,
                           J=r.couplings.astype(np.float64), n_groups=spec.n_replicas,
                           n_res=spec.n_res, sweeps_per_emcs=spec.sweeps_per_emcs,
                           res_sweeps_per_emcs=spec.res_sweeps_per_emcs)
        o.prethermalize_reservoir(spec.pretherm_sweeps)
        o.emcs(r.budget_emcs)
        if o.n_ties.sum() == 0:
            np.testing.assert_array_equal(r.obs, o.obs)
            np.testing.assert_array_equal(r.round_trips, o.round_trips)
            compared += 1
    assert compared >= 3


def test_group_graph_equals_separate_batches():
    """pthr_group: one graph launch per EMCS over batches of different L gives
    the same state as advancing each batch on its own."""
    from paper_2605_25872_gb300 import Group
    cfgs = [BatchConfig(L=L, n_samples=3, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                        res_sweeps_per_emcs=4) for L in (6, 8, 12)]
    Js = [W.gaussian_couplings(c.L, 3, 40 + c.L) for c in cfgs]
    seeds = [W.sample_seeds(70 + c.L, 3) for c in cfgs]
    sep = [Batch(c, couplings=J, seeds=sd) for c, J, sd in zip(cfgs, Js, seeds)]
    grp_b = [Batch(c, couplings=J, seeds=sd, stream=torch.cuda.Stream()) for c, J, sd in zip(cfgs, Js, seeds)]
    for b in sep:
        b.emcs(5)
    g = Group(grp_b)
    assert g.launches_per_emcs == 4          # one launch per EMCS step for all sizes
    g.emcs(5)
    g.synchronize()
    for a, b in zip(sep, grp_b):
        np.testing.assert_array_equal(a.export_spins().cpu().numpy(), b.export_spins().cpu().numpy())
        np.testing.assert_array_equal(a.obs.cpu().numpy(), b.obs.cpu().numpy())
        np.testing.assert_array_equal(a.energies.cpu().numpy(), b.energies.cpu().numpy())


@pytest.mark.parametrize("rule", ["heatbath", "micsa"])
def test_group_graph_equals_separate_batches_other_rules(rule):
    from paper_2605_25872_gb300 import Group
    cfgs = [BatchConfig(L=L, n_samples=2, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                        res_sweeps_per_emcs=4, rule=rule) for L in (4, 10, 16)]
    Js = [W.gaussian_couplings(c.L, 2, 80 + c.L) for c in cfgs]
    seeds = [W.sample_seeds(90 + c.L, 2) for c in cfgs]
    sep = [Batch(c, couplings=J, seeds=sd) for c, J, sd in zip(cfgs, Js, seeds)]
    grp_b = [Batch(c, couplings=J, seeds=sd, stream=torch.cuda.Stream()) for c, J, sd in zip(cfgs, Js, seeds)]
    for b in sep:
        b.emcs(3)
    g = Group(grp_b)
    assert g.launches_per_emcs == 4
    g.emcs(3)
    g.synchronize()
    for a, b in zip(sep, grp_b):
        np.testing.assert_array_equal(a.export_spins().cpu().numpy(), b.export_spins().cpu().numpy())
        np.testing.assert_array_equal(a.obs.cpu().numpy(), b.obs.cpu().numpy())


def test_mixed_size_group_matches_the_oracle():
    """One graph of four launches per EMCS over batches of L = 4, 6 and 8
    (the EMCS of Sec. 3 for every sample whatever its size) against the FP64
    oracle, sample by sample: every sample whose oracle run met no near tie
    has the oracle's spins, permutations, energies and accumulators."""
    import sys
    sys.path.insert(0, __file__.rsplit("/", 1)[0])
    from mirror import Mirror
    from paper_2605_25872_gb300 import Group
    cfgs = [BatchConfig(L=L, n_samples=3, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                        res_sweeps_per_emcs=4) for L in (4, 6, 8)]
    Js = [W.gaussian_couplings(c.L, 3, 120 + c.L) for c in cfgs]
    seeds = [W.sample_seeds(W.SEED_BASE + 130 + c.L, 3) for c in cfgs]
    batches = [Batch(c, couplings=J, seeds=sd, stream=torch.cuda.Stream()) for c, J, sd in zip(cfgs, Js, seeds)]
    mirrors = [Mirror(c, J, sd) for c, J, sd in zip(cfgs, Js, seeds)]
    g = Group(batches)
    assert g.launches_per_emcs == 4
    n_emcs = 4
    g.emcs(n_emcs)
    g.synchronize()
    compared = 0
    for b, m in zip(batches, mirrors):
        tied = set()
        for _ in range(n_emcs):
            ties, pt_ties = m.emcs()
            tied |= {s for s, _ in ties} | set(pt_ties)
        spins = b.export_spins().cpu().numpy()
        for s in range(b.cfg.n_samples):
            if s in tied:
                continue
            np.testing.assert_array_equal(spins[s], m.spins()[s])
            np.testing.assert_array_equal(b.perm.cpu().numpy()[s], m.perms()[s])
            np.testing.assert_array_equal(b.energies.cpu().numpy()[s], m.energies()[s])
            np.testing.assert_array_equal(b.obs.cpu().numpy()[s], m.samples[s].obs)
            compared += 1
    assert compared >= 7


def test_group_outside_the_compiled_sizes_falls_back_to_per_batch_graphs():
    """A group with L = 18 (not compiled into the group kernels) and batches
    of different update rules is captured as each batch's own EMCS on its
    stream: same results as separate batches, more than four launches."""
    from paper_2605_25872_gb300 import Group
    cfgs = [BatchConfig(L=18, n_samples=1, n_temps=4, n_replicas=4, n_res=1, sweeps_per_emcs=1,
                        res_sweeps_per_emcs=2),
            BatchConfig(L=6, n_samples=2, n_temps=4, n_replicas=4, n_res=1, sweeps_per_emcs=1,
                        res_sweeps_per_emcs=2, rule="heatbath")]
    Js = [W.gaussian_couplings(c.L, c.n_samples, 160 + c.L) for c in cfgs]
    seeds = [W.sample_seeds(170 + c.L, c.n_samples) for c in cfgs]
    sep = [Batch(c, couplings=J, seeds=sd) for c, J, sd in zip(cfgs, Js, seeds)]
    grp_b = [Batch(c, couplings=J, seeds=sd, stream=torch.cuda.Stream()) for c, J, sd in zip(cfgs, Js, seeds)]
    for b in sep:
        b.emcs(2)
    g = Group(grp_b)
    assert g.launches_per_emcs == 8
    g.emcs(2)
    g.synchronize()
    for a, b in zip(sep, grp_b):
        np.testing.assert_array_equal(a.export_spins().cpu().numpy(), b.export_spins().cpu().numpy())
        np.testing.assert_array_equal(a.obs.cpu().numpy(), b.obs.cpu().numpy())
