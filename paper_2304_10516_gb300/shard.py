"""Distribution of partition models over ranks (one process per GPU).

The models of different partitions never exchange data while training
(Sec. 3.1 of the paper): which rank trains which partition and how a timing
is agreed on need no data-path collective. The exchanges of the paper's
visualisation pipeline are here too: sort-last compositing of the ranks'
images (Sec. 4.3: gather, then blend in depth order with the library's
dvnr_composite) and the global error (Sec. 5: sums of squared errors and
voxel counts reduced in FP64).
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


def _device_for(tensor_device):
    import torch
    import torch.distributed as dist

    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_images(rgba, depth: float):
    """All-gather every rank's image (h, w, 4) and the depth of its partition
    (e.g. its box's lo.z); returns (images, depths) in rank order on every
    rank. Images travel on the backend's device (GPU for NCCL, host for
    gloo) and come back on the device of `rgba`."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return [rgba], [float(depth)]
    world = dist.get_world_size()
    dev = _device_for(rgba.device)
    x = rgba.contiguous().to(dev)
    bufs = [torch.empty_like(x) for _ in range(world)]
    dist.all_gather(bufs, x)
    d = torch.tensor([float(depth)], dtype=torch.float64, device=dev)
    dbufs = [torch.empty_like(d) for _ in range(world)]
    dist.all_gather(dbufs, d)
    return [b.to(rgba.device) for b in bufs], [float(v.item()) for v in dbufs]


def composite_sort_last(rgba, depth: float, stream=None):
    """The image of all ranks' partitions: gather the ranks' images and blend
    them front to back on this rank's GPU (library kernel)."""
    from . import model as dv

    images, depths = gather_images(rgba, depth)
    return dv.composite(images, depths, stream=stream)


def sort_last_frame(depths, render_depth, composite, gather=None):
    """The frame of all ranks' partitions, composited sort-last (Sec. 4.3).

    Partitions at one depth (e.g. one z-layer of a box decomposition) cover
    disjoint pixels, so a rank's partitions at one depth form one image;
    partitions at different depths must blend in depth order, whichever rank
    holds them. For every depth of the global decomposition (`depths`, the
    same list on every rank), each rank renders its own partitions at that
    depth (`render_depth(d)`, an empty image when it holds none there) and the
    images of all ranks are gathered (`gather`, default gather_images); then
    `composite(images, depths)` blends all of them front to back (stable
    in depth order; images of one depth do not overlap)."""
    gather = gather or gather_images
    images, ds = [], []
    for d in depths:
        ims, dd = gather(render_depth(d), d)
        images += ims
        ds += dd
    return composite(images, ds)


def global_psnr(sse: float, count: int, value_range: float = 1.0):
    """PSNR over the voxels of all ranks (Sec. 5): the squared errors and
    voxel counts are summed over ranks in FP64 first (voxel-weighted)."""
    import math

    import torch
    import torch.distributed as dist

    t = torch.tensor([float(sse), float(count)], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized():
        t = t.to(_device_for(t.device))
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    s, n = float(t[0].item()), float(t[1].item())
    return 20 * math.log10(value_range) - 10 * math.log10(s / n), s, n
