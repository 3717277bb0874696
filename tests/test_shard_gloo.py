"""The N > 1 path on CPU: two gloo ranks split the 64 uneven partitions of the
partitioned workload by longest-processing-time and agree on the max step
time; no data-path collective exists (partitions are independent)."""
import os

import pytest

from paper_2304_10516_gb300 import shard, volumes


def _boxes():
    return volumes.uneven_boxes((512, 512, 512), (4, 4, 4), (96, 160), seed=1004)


def _cost(box):
    (lo, hi) = box
    return (hi[0] - lo[0] + 2) * (hi[1] - lo[1] + 2) * (hi[2] - lo[2] + 2)


def test_lpt_is_a_balanced_partition():
    costs = [_cost(b) for b in _boxes()]
    for world in (1, 2, 3, 8):
        parts = shard.assign_lpt(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: max load <= mean + max single cost
        assert max(loads) <= sum(costs) / world + max(costs)
    assert shard.assign_lpt([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [_cost(b) for b in _boxes()]
        mine = shard.rank_partitions(costs, world, rank)
        import torch

        # every rank sees the others' shares only through this check
        buf = [None] * world
        dist.all_gather_object(buf, mine)
        t = shard.max_over_ranks(1.0 + rank)
        out.put((rank, mine, buf, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_partitions_and_agree_on_time():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, mine0, all0, t0), (r1, mine1, all1, t1) = res
    assert all0 == all1 == [mine0, mine1]
    assert sorted(mine0 + mine1) == list(range(64)) and not set(mine0) & set(mine1)
    assert t0 == t1 == 2.0  # the slowest rank's time


def _exchange_worker(rank, world, port, out):
    import math

    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's image of its partition (rank-specific values) and depth
        img = torch.full((3, 5, 4), float(rank + 1)) * torch.arange(4.0)
        depth = [7.0, 2.0][rank]  # rank 1's partition is in front
        images, depths = shard.gather_images(img, depth)
        psnr, s, n = shard.global_psnr([0.5, 1.5][rank], [100, 300][rank], value_range=2.0)
        out.put((rank, [im.tolist() for im in images], depths, psnr, s, n,
                 20 * math.log10(2.0) - 10 * math.log10(2.0 / 400)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_images_and_errors():
    # the exchanges of the visualisation path: every rank receives all ranks'
    # images and depths in rank order (sort-last input), and the PSNR is
    # taken over the sum of both ranks' squared errors and voxel counts
    import socket

    import torch
    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_exchange_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [(torch.full((3, 5, 4), float(r + 1)) * torch.arange(4.0)).tolist() for r in range(2)]
    for rank, images, depths, psnr, s, n, psnr_want in res:
        assert images == want and depths == [7.0, 2.0]
        assert (s, n) == (2.0, 400.0) and abs(psnr - psnr_want) < 1e-12
