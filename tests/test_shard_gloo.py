"""The N > 1 path on CPU: two gloo ranks split the 64 uneven partitions of the
partitioned workload by longest-processing-time and agree on the max step
time; no data-path collective exists (partitions are independent)."""
import os

import numpy as np

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


# ------------------------------------------------------------------------
# The partitioned workload's multi-rank driver (bench.py blocks_measure) on
# two gloo ranks, with CPU stand-ins for the library's render and composite
# calls: LPT assignment of the 64 uneven blocks, per-depth-layer images
# gathered from all ranks, sort-last blending, and the global PSNR.

FRAME = 32  # pixels per side over the [0, 512)^2 footprint of the blocks


def _block_image(i, box):
    """Stand-in for a block rendered in the global frame: a premultiplied
    colour over the block's x-y footprint, zero elsewhere."""
    import torch

    (lo, hi) = box
    img = torch.zeros((FRAME, FRAME, 4), dtype=torch.float64)
    s = 512 // FRAME
    a = 0.1 + 0.8 * ((i * 37) % 11) / 10.0
    img[lo[1] // s: hi[1] // s, lo[0] // s: hi[0] // s] = torch.tensor(
        [a * ((i * 7) % 5) / 4.0, a * ((i * 3) % 7) / 6.0, a * 0.5, a], dtype=torch.float64)
    return img


def _blend(images, depths):
    """Stand-in for dvnr_composite: front to back in increasing depth
    (stable), C += (1 - A) C_i."""
    import torch

    order = sorted(range(len(images)), key=lambda k: depths[k])
    acc = torch.zeros_like(images[0])
    for k in order:
        acc = acc + (1.0 - acc[..., 3:4]) * images[k]
    return acc


def _block_sse(i):
    return 1e-3 * (1 + (i % 5)), 1000 + 17 * i  # (squared error, voxel count) of block i


def _frame_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        boxes = _boxes()
        costs = [_cost(b) for b in boxes]
        mine = shard.rank_partitions(costs, world, rank)
        layers = sorted({lo[2] for lo, _ in boxes})

        def render_layer(z):
            sel = [i for i in mine if boxes[i][0][2] == z]
            img = torch.zeros((FRAME, FRAME, 4), dtype=torch.float64)
            for i in sel:  # blocks of one layer cover disjoint pixels
                img = img + _block_image(i, boxes[i])
            return img

        frame = shard.sort_last_frame(layers, render_layer, _blend)
        sse = sum(_block_sse(i)[0] for i in mine)
        vox = sum(_block_sse(i)[1] for i in mine)
        psnr, s, n = shard.global_psnr(sse, vox)
        out.put((rank, mine, frame.tolist(), psnr, s, n))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_run_the_partitioned_frame():
    import math
    import socket

    import torch
    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_frame_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    boxes = _boxes()
    # the single-process frame: every block's image blended by its depth
    want = _blend([_block_image(i, b) for i, b in enumerate(boxes)], [b[0][2] for b in boxes])
    sse = sum(_block_sse(i)[0] for i in range(len(boxes)))
    vox = sum(_block_sse(i)[1] for i in range(len(boxes)))
    psnr_want = -10 * math.log10(sse / vox)
    (r0, mine0, f0, p0, s0, n0), (r1, mine1, f1, p1, s1, n1) = res
    assert sorted(mine0 + mine1) == list(range(len(boxes))) and mine0 and mine1
    for f in (f0, f1):
        np.testing.assert_allclose(np.array(f), want.numpy(), rtol=0, atol=1e-15)
    assert (s0, n0) == (s1, n1) and abs(n0 - vox) == 0 and abs(s0 - sse) < 1e-12
    assert abs(p0 - psnr_want) < 1e-9 and p0 == p1
    # the frame is not trivial: most pixels are covered, and blocks overlap in depth
    assert (want[..., 3] > 0).float().mean() > 0.9
