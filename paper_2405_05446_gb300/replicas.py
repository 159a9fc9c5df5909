"""Replicas: one process per GPU, each with its own copy of the resident scenes,
rendering whole views. Views are independent, so there is no collective on the
data path; the only communication is the timing reduction at the end of a run.

`shard` deals a list of independent views out to the ranks (round robin, every
view exactly once); `aggregate` turns per-rank work and time into the whole-job
throughput, all units over the slowest rank's time. Both work with any
torch.distributed backend (gloo on the host, nccl on the GPUs)."""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int) -> list[int]:
    """Indices of the items rank `rank` of `world` renders: rank, rank + world, ..."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    return list(range(rank, n_items, world))


def aggregate(units: float, seconds: float, device=None) -> dict:
    """Whole-job throughput over all ranks: sum of units / max of seconds. Without
    an initialised process group it is this process's own numbers."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return {"units": units, "seconds": seconds, "value": units / seconds, "world": 1}
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    world = dist.get_world_size()
    return {"units": float(u.item()), "seconds": float(t.item()),
            "value": float(u.item()) / float(t.item()), "world": world}
