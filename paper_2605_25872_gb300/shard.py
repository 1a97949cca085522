"""Sharding of independent disorder samples over ranks (one GPU per rank).

Samples are independent (quenched disorder, Sec. 2), so the data path needs
no collective: rank r owns a contiguous range of global sample ids and keys
each sample's random numbers by its global id.  Results therefore do not
depend on the number of ranks.  The only exchange is off the hot loop: at
a measurement-bin boundary the per-sample accumulators are gathered (or the
per-temperature sums reduced) for the disorder average.
"""
from __future__ import annotations

import numpy as np


def sample_range(rank: int, world: int, n_total: int):
    """Contiguous (first, count) of global sample ids owned by `rank`; the
    first n_total % world ranks hold one extra sample."""
    if not (0 <= rank < world) or n_total < 0:
        raise ValueError("bad rank/world/n_total")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return first, count


def shard_seeds(batch_seed: int, rank: int, world: int, n_total: int) -> np.ndarray:
    """Philox keys of this rank's samples: batch_seed + global sample id."""
    first, count = sample_range(rank, world, n_total)
    return (np.uint64(batch_seed) + np.arange(first, first + count, dtype=np.uint64)).astype(np.uint64)


def gather_samples(local, group=None):
    """All-gather per-sample arrays (leading axis = this rank's samples) into
    the global array, in rank order, on every rank.  Host tensors (gloo)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(local))
    world = dist.get_world_size(group)
    counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(counts, torch.tensor([t.shape[0]], dtype=torch.int64), group=group)
    mx = int(max(int(c) for c in counts))
    pad = torch.zeros((mx,) + tuple(t.shape[1:]), dtype=t.dtype)
    pad[: t.shape[0]] = t
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return np.concatenate([p[: int(c)].numpy() for p, c in zip(parts, counts)], axis=0)


def reduce_sums(local_sums, group=None):
    """Sum of per-temperature accumulators over all ranks' samples."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(np.ascontiguousarray(local_sums, dtype=np.float64)).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()
