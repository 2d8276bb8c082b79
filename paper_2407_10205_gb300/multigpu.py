"""Replica sharding over ranks (one process per GPU) and the one exchange it needs.

Replicas are independent (each draws from its own Philox counter), so a run with R
replicas on W ranks gives rank k the replica range `shard(R, W, k)` and a seed shared by
all ranks; no collective touches the data path.  The only exchange is the final result:
the lowest energy over ranks (ties: earliest iteration, then lowest rank) and the spins
of the winning replica, gathered with torch.distributed (any backend).
"""
from __future__ import annotations

import numpy as np


def shard(total: int, world: int, rank: int) -> tuple[int, int]:
    """[first, first + count) of `total` replicas for `rank` of `world` (contiguous, sizes
    differing by at most one)."""
    base, extra = divmod(int(total), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def global_best(energy_k: int, step: int, spins: np.ndarray):
    """All-gather (energy, step) over the process group and broadcast the winner's spins.
    Returns (energy_k, step, winning rank, spins)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size()
    mine = torch.tensor([int(energy_k), int(step)], dtype=torch.int64)
    allv = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allv, mine)
    keys = [(int(v[0]), int(v[1]), r) for r, v in enumerate(allv)]
    e, s, winner = min(keys)
    buf = torch.from_numpy(np.ascontiguousarray(spins, dtype=np.int8).copy())
    dist.broadcast(buf, src=winner)
    return e, s, winner, buf.numpy()
