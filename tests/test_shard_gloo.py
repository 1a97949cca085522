"""Multi-rank host logic on CPU (gloo, world size 2): sample ranges cover
the batch exactly once, seeds follow the global sample id (so results do not
depend on the rank count), and gathered / reduced accumulators equal the
single-process ones."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2605_25872_gb300.shard import gather_samples, reduce_sums, sample_range, shard_seeds


def test_sample_ranges_partition_the_batch():
    for n in (0, 1, 5, 512, 1023):
        for world in (1, 2, 3, 8):
            ids = []
            for r in range(world):
                f, c = sample_range(r, world, n)
                ids += list(range(f, f + c))
            assert ids == list(range(n))
    np.testing.assert_array_equal(np.concatenate([shard_seeds(100, r, 3, 10) for r in range(3)]),
                                  100 + np.arange(10, dtype=np.uint64))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n_total, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = sample_range(rank, world, n_total)
    rng = np.random.default_rng(123)
    full = rng.standard_normal((n_total, 6, 8))          # accumulators of every sample
    local = full[first:first + count]
    g = gather_samples(local)
    s = reduce_sums(local.sum(axis=0))
    np.save(os.path.join(out_dir, f"g{rank}.npy"), g)
    np.save(os.path.join(out_dir, f"s{rank}.npy"), s)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("n_total", [7, 16])
def test_gather_and_reduce_over_two_gloo_ranks(tmp_path, n_total):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_total, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    rng = np.random.default_rng(123)
    full = rng.standard_normal((n_total, 6, 8))
    for r in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / f"g{r}.npy"), full)
        np.testing.assert_allclose(np.load(tmp_path / f"s{r}.npy"), full.sum(axis=0), rtol=1e-12)


def _pthr_worker(rank, world, port, n_total, n_emcs, out_dir):
    """Each rank runs the FP64 oracle on its own shard of the samples (seeds
    and couplings from the global sample id) and the per-sample accumulators
    are gathered and the per-temperature sums reduced at the end."""
    import torch.distributed as dist
    import oracle as O
    import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    first, count = sample_range(rank, world, n_total)
    seeds = shard_seeds(W.SEED_BASE + 77, rank, world, n_total)
    J = W.gaussian_couplings(4, n_total, 77)[first:first + count]
    obs = []
    for s in range(count):
        smp = O.OracleSample(4, 6, 0.2, 1.6, int(seeds[s]), J=J[s].astype(np.float64), n_groups=4,
                             n_res=2, sweeps_per_emcs=1, res_sweeps_per_emcs=4)
        smp.prethermalize_reservoir(8)
        smp.emcs(n_emcs)
        obs.append(np.concatenate([smp.obs.ravel(), smp.round_trips.astype(np.float64)]))
    local = np.array(obs).reshape(count, -1) if count else np.zeros((0, 6 * 8 + 4))
    g = gather_samples(local)
    tot = reduce_sums(local.sum(axis=0))
    np.save(os.path.join(out_dir, f"pthr_g{rank}_{world}.npy"), g)
    np.save(os.path.join(out_dir, f"pthr_s{rank}_{world}.npy"), tot)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_oracle_pthr_equals_one_rank(tmp_path):
    """Sample sharding (independent disorder samples): PTHR run on two gloo
    ranks, each with its own contiguous shard, gives per-sample accumulators
    and reduced sums identical to the same run on one rank -- the result does
    not depend on the rank count (per-sample values bit for bit; the reduced
    sums up to the order of the floating-point additions)."""
    n_total, n_emcs = 5, 6
    ctx = mp.get_context("spawn")
    for world in (1, 2):
        port = _free_port()
        procs = [ctx.Process(target=_pthr_worker, args=(r, world, port, n_total, n_emcs, str(tmp_path)))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
    one = np.load(tmp_path / "pthr_g0_1.npy")
    assert one.shape[0] == n_total
    for r in range(2):
        np.testing.assert_array_equal(np.load(tmp_path / f"pthr_g{r}_2.npy"), one)
        # the reduction adds the same per-sample values in another order
        np.testing.assert_allclose(np.load(tmp_path / f"pthr_s{r}_2.npy"), np.load(tmp_path / "pthr_s0_1.npy"),
                                   rtol=1e-13, atol=1e-12)
