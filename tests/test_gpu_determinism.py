"""Run-to-run determinism at the sizes where concurrency shows.

Every random number is keyed by (sample, lattice, site, step), the energies
are exact integer sums on the coupling grid and every accumulation runs in a
fixed order, so two batches with the same inputs must stay bit-identical
step by step.  Differences would come from a race between threads: the
union-find of the cluster kernel is the one place where many threads write
the same shared array, and a path-halving store during flattening once left
a site pointing at an intermediate ancestor instead of its root (a rare
wrong flip, seen in one pair out of thousands).  The small parity tests are
too small to meet such a race; these run many pairs per launch.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

P = pytest.importorskip("paper_2605_25872_gb300")
from paper_2605_25872_gb300 import Batch, BatchConfig  # noqa: E402
from paper_2605_25872_gb300.build import build  # noqa: E402

NAMES = ["energies", "perm", "age", "rt_state", "round_trips", "pt_accepted", "flips", "obs", "cluster_stats"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build()


def state(b):
    torch.cuda.synchronize()
    d = {n: getattr(b, n).cpu().numpy().copy() for n in NAMES}
    d["spins"] = b.export_spins().cpu().numpy()
    torch.cuda.synchronize()
    return d


def assert_same(a, b, where):
    for n in a:
        assert np.array_equal(a[n], b[n]), f"{where}: {n} differs at {np.argwhere(a[n] != b[n])[:5].tolist()}"


@pytest.mark.parametrize("L,S,NT,cluster,rule", [(16, 64, 32, "acu", "metropolis"), (12, 160, 24, "acu", "metropolis"),
                                                  (8, 256, 16, "single", "metropolis"), (16, 48, 32, "acu", "micsa"),
                                                  (10, 128, 24, "acu", "heatbath")])
def test_identical_inputs_give_identical_trajectories(L, S, NT, cluster, rule):
    cfg = BatchConfig(L=L, n_samples=S, n_temps=NT, n_replicas=4, n_res=4 if L == 16 else 0,
                      sweeps_per_emcs=10 if L == 16 else 1, res_sweeps_per_emcs=240 if L == 16 else 0,
                      er_on=L == 16, cluster=cluster, rule=rule)
    J = W.gaussian_couplings(L, S, 5)
    seeds = W.sample_seeds(W.SEED_BASE + 5, S)
    st = torch.cuda.Stream()
    bs = [Batch(cfg, couplings=J, seeds=seeds, stream=st) for _ in range(2)]
    if cfg.er_on:
        for b in bs:
            b.prethermalize(240)
    for e in range(3 if L == 16 else 12):
        for b in bs:
            b.sweep(cfg.sweeps_per_emcs, cfg.res_sweeps_per_emcs if cfg.er_on else 0)
            b.houdayer()
        assert_same(state(bs[0]), state(bs[1]), f"EMCS {e} after the cluster move")
        for b in bs:
            b.swap(True, cfg.er_on)
            b.measure()
    la, lb = (b.cluster_labels().cpu().numpy() for b in bs)
    np.testing.assert_array_equal(la, lb)
    # canonical labels: every label is a site labelled by itself, no larger than the site
    flat = la.reshape(-1, cfg.V)
    i = np.arange(cfg.V)
    assert np.all(flat <= i)
    assert np.all(np.take_along_axis(flat, flat, axis=1) == flat)
    for b in bs:
        assert b.poll(60000) == 0


def test_identical_groups_give_identical_trajectories():
    """The four-launch group of the serving mix: every kernel covers the blocks
    of five batches at once."""
    from paper_2605_25872_gb300.batch import Group
    groups = []
    for _ in range(2):
        bs = []
        for i, L in enumerate((6, 8, 10, 12, 16)):
            cfg = BatchConfig(L=L, n_samples=32, n_temps=24, n_replicas=4, n_res=4, sweeps_per_emcs=10,
                              res_sweeps_per_emcs=240)
            bs.append(Batch(cfg, couplings=W.gaussian_couplings(L, 32, 40 + i),
                            seeds=W.sample_seeds(W.SEED_BASE + 40 + i, 32), stream=torch.cuda.Stream()))
            bs[-1].prethermalize(240)
        torch.cuda.synchronize()
        g = Group(bs)
        assert g.launches_per_emcs == 4
        groups.append((g, bs))
    for e in range(3):
        for g, _ in groups:
            g.emcs(1)
            g.synchronize()
        for a, b in zip(groups[0][1], groups[1][1]):
            assert_same(state(a), state(b), f"EMCS {e}, L={a.cfg.L}")


def test_group_emcs_is_ordered_with_the_members_streams():
    """Per-batch calls and group EMCS mixed without host synchronisation give
    the state of the same calls with a synchronisation after each."""
    from paper_2605_25872_gb300.batch import Group

    def members():
        out = []
        for i, L in enumerate((8, 12)):
            cfg = BatchConfig(L=L, n_samples=24, n_temps=16, n_replicas=4, n_res=4, sweeps_per_emcs=4,
                              res_sweeps_per_emcs=96)
            out.append(Batch(cfg, couplings=W.gaussian_couplings(L, 24, 60 + i),
                             seeds=W.sample_seeds(W.SEED_BASE + 60 + i, 24), stream=torch.cuda.Stream()))
        torch.cuda.synchronize()
        return out

    free, synced = members(), members()
    gf, gs = Group(free), Group(synced)
    for b in free:
        b.prethermalize(480)          # still running when the group EMCS is queued
    gf.emcs(2)
    for b in free:
        b.emcs(1)                     # queued on the member streams after the group EMCS
    for b in synced:
        b.prethermalize(480)
    torch.cuda.synchronize()
    gs.emcs(2)
    torch.cuda.synchronize()
    for b in synced:
        b.emcs(1)
    torch.cuda.synchronize()
    for a, b in zip(free, synced):
        assert_same(state(a), state(b), f"L={a.cfg.L}")


def test_group_emcs_inside_a_callers_graph_capture():
    """pthr_group_emcs inside the caller's CUDA-graph capture: the four-launch
    group enqueues its kernels into the capture (a graph cannot be launched
    there), and replaying the caller's graph gives the state of direct calls."""
    from paper_2605_25872_gb300.batch import Group

    def members():
        out = []
        for i, L in enumerate((6, 10)):
            cfg = BatchConfig(L=L, n_samples=16, n_temps=12, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                              res_sweeps_per_emcs=24)
            out.append(Batch(cfg, couplings=W.gaussian_couplings(L, 16, 80 + i),
                             seeds=W.sample_seeds(W.SEED_BASE + 80 + i, 16), stream=torch.cuda.Stream()))
        torch.cuda.synchronize()
        return out

    direct, captured = members(), members()
    gd, gc = Group(direct), Group(captured)
    gd.emcs(3)
    gd.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gc.stream):
        gc.emcs(1)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(direct, captured):
        assert_same(state(a), state(b), f"L={a.cfg.L}")


def test_batch_emcs_inside_a_callers_graph_capture():
    """pthr_emcs(use_graph=1) while the caller captures the batch's stream
    enqueues the EMCS kernels into that capture instead of its own graph."""
    cfg = BatchConfig(L=8, n_samples=8, n_temps=8, n_replicas=4, n_res=2, sweeps_per_emcs=2,
                      res_sweeps_per_emcs=16)
    J, seeds = W.gaussian_couplings(8, 8, 90), W.sample_seeds(W.SEED_BASE + 90, 8)
    direct = Batch(cfg, couplings=J, seeds=seeds, stream=torch.cuda.Stream())
    captured = Batch(cfg, couplings=J, seeds=seeds, stream=torch.cuda.Stream())
    torch.cuda.synchronize()
    direct.emcs(4)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=captured.stream):
        captured.emcs(2, graph=True)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert_same(state(direct), state(captured), "captured EMCS")


def test_per_batch_graph_group_refuses_a_callers_capture():
    """A group outside the four-launch form (an L=18 member) returns
    PTHR_E_STATE inside a caller's capture, leaves the capture usable, and
    still steps normally afterwards."""
    from paper_2605_25872_gb300 import _lib
    from paper_2605_25872_gb300.batch import Group
    bs = []
    for i, L in enumerate((18, 6)):
        cfg = BatchConfig(L=L, n_samples=2, n_temps=6, n_replicas=4, n_res=2, sweeps_per_emcs=1,
                          res_sweeps_per_emcs=4)
        bs.append(Batch(cfg, couplings=W.gaussian_couplings(L, 2, 95 + i),
                        seeds=W.sample_seeds(W.SEED_BASE + 95 + i, 2), stream=torch.cuda.Stream()))
    torch.cuda.synchronize()
    g = Group(bs)
    assert g.launches_per_emcs > 4
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=g.stream):
        with pytest.raises(_lib.PthrError) as err:
            g.emcs(1)
        x = torch.zeros(4, device="cuda")
        x += 1                                  # the capture still records work
    assert err.value.status == _lib.PTHR_E_STATE
    graph.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 4.0
    g.emcs(1)
    g.synchronize()
    assert all(int(b.emcs_counter.cpu()[0]) == 1 for b in bs)
