"""Distribution of partition models over ranks (one process per GPU).

The models of different partitions never exchange data while training
(Sec. 3.1 of the paper), so the only multi-rank logic is which rank trains
which partition and how a timing is agreed on: there is no collective on the
data path.
"""
from __future__ import annotations


def assign_lpt(costs, world: int) -> list[list[int]]:
    """Longest-processing-time assignment: partitions sorted by cost
    (e.g. voxel count) in decreasing order, each given to the currently
    least-loaded rank. Returns the partition indices of every rank, each in
    increasing order. Deterministic (ties go to the lower rank / index)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def rank_partitions(costs, world: int, rank: int) -> list[int]:
    """The partitions rank `rank` trains."""
    return assign_lpt(costs, world)[rank]


def max_over_ranks(value: float) -> float:
    """Max of a per-rank scalar over the default process group (the step
    time of the slowest rank); the value itself when not distributed."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
