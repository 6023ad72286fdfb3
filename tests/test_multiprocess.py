"""The multi-GPU path of bench.py shards images over ranks with no data-path
collective; only the timing is reduced (max over ranks).  Checked here with
two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.image_seeds(images=4, seed=7, rank=rank)
    t = bench.max_over_ranks(0.5 + rank, dist, torch.device("cpu"))
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    if rank == 0:
        out.put((gathered, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_images_and_report_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert len(set(gathered[0]) & set(gathered[1])) == 0
    assert len(gathered[0]) == len(gathered[1]) == 4
    assert t == pytest.approx(1.5)


def _detect_rank(rank, world, port, out):
    """One rank: its own shard of a small mixed-size workload (the bench's
    make_workload with its rank), each image solved by the oracle (the CPU
    stand-in for this rank's GPU), the polylines gathered on rank 0."""
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = bench.make_workload("plain256", 3, 5, rank)
    res = []
    for img, k, B in items:
        x, d, s = oracle.detect(img, k, B)
        res.append((img.tobytes(), [int(v) for v in x], [int(v) for v in d], int(s)))
    t = bench.max_over_ranks(float(len(res)) + rank, dist, torch.device("cpu"))
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    if rank == 0:
        out.put((gathered, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_detect_their_own_shards_like_one_process():
    """Weak scaling over images: each rank detects only its shard, the
    shards are disjoint, and every gathered polyline equals what a single
    process computes on the same image."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_detect_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == pytest.approx(4.0)   # the slower rank's count + its rank
    imgs = [r[0] for shard in gathered for r in shard]
    assert len(imgs) == 6 and len(set(imgs)) == 6
    for rank, shard in enumerate(gathered):
        local = bench.make_workload("plain256", 3, 5, rank)
        for (img, k, B), (blob, x, d, s) in zip(local, shard):
            assert img.tobytes() == blob
            xo, do, so = oracle.detect(img, k, B)
            assert x == list(xo) and d == list(do) and s == int(so)
            assert oracle.path_score(img, k, x[0], np.asarray(d)) == so
