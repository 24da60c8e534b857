"""Several GPUs of one node as independent replicas.

The step does not shard: one domain lives on one GPU, and the batched
boiling curve's instances are independent. So N ranks (one process per GPU,
launched by torchrun) run N independent problems with no collective on the
data path. The only collectives are host-side bookkeeping: the slowest
rank's time (the job's time), and gathering the per-case results of a
boiling curve whose cases were dealt out to the ranks.
"""

from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's time is the slowest
    rank's); `dist` is torch.distributed with an initialised group, or None
    for one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, ms: float) -> float:
    """Whole-job throughput in units per second: every rank processed
    units_per_rank units, the job took the slowest rank's `ms`."""
    return world * units_per_rank / (ms * 1e-3)


def shard(items, rank: int, world: int) -> list:
    """The items rank `rank` of `world` handles: every world-th item from
    position rank (balanced to one item, order kept)."""
    return list(items)[rank::world]


def gather_shards(local: list, rank: int, world: int, dist=None) -> list:
    """Inverse of shard: the full list in the original order, on every rank."""
    if dist is None or world == 1:
        return list(local)
    parts = [None] * world
    dist.all_gather_object(parts, list(local))
    n = sum(len(p) for p in parts)
    out = [None] * n
    for r, p in enumerate(parts):
        out[r::world] = p
    return out
