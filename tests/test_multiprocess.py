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
