"""Host logic of multi-GPU runs.  The time steps of one grid do not shard
cheaply (every transform would need an all-to-all transpose), so N GPUs run
independent work: replicas of one workload (weak scaling) or disjoint shards of
a batch's members (strong scaling).  No collective touches the data path; the
only collectives are the max of the timed region over ranks and the sum of the
units processed, on the host side of the benchmark."""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Members of a batch that rank `rank` of `world` advances: every
    world-th member starting at rank (sizes stay mixed on every rank)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return list(items)[rank::world]


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The slowest rank's time (the whole job ends when it ends)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device="cpu") -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
