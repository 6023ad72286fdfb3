#!/usr/bin/env python
"""Throughput of end-to-end curve detection (band FHT + bend-limited DP +
read-back) on synthetic 2048x2048 uint8 images, k=16 bands of 128 rows, bend
range 16, in Mpix/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole method over a batch of --images distinct
seeded images per GPU (inputs already resident in HBM; the batch is larger
than the 129 MB L2, so no flush is needed between steps).  Under torchrun
each rank takes its own images (weak scaling, no data-path collective).
Rank 0 prints one JSON line.  ``--impl reference`` times the CPU oracle (the
paper's method as a plain C program) on a bounded sample of the same
workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W_IMG, K, B = 2048, 2048, 16, 16
N_BAND = H // K
METRIC = "Mpix/s end-to-end band-FHT+DP (exact) and % HBM roofline; batched/learned vs plain"
WORKLOAD = "u8 2048x2048, k=16 bands of 128 rows, bend |d_{i+1}-d_i|<=16, Gaussian noise + 3 polylines"

# DRAM bytes (read + write) per image of engine_kernel<uint8> from the ncu
# capture summarised in profiles/engine_kernel_u8_2048x2048_k16_B16.md
# (48 images per launch); a launch's traffic is this times its images.  Set to
# None whenever the kernel changes until it is captured again.
NCU_TRAFFIC_BYTES_PER_IMAGE = (264.419328e6 + 1391.033e6) / 48


def algorithmic_bytes_per_image(h=H, w=W_IMG, k=K, bpp=1):
    """Bytes the method must move per image: read the image once, write and
    read one 4-byte DP value per state (x, d) of every band, and the path."""
    n = h // k
    return h * w * bpp + k * 8 * (2 * n - 1) * w + 4 * (2 * k + 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--images", type=int, default=32, help="images per step per GPU")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU baseline leg")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.file.flush()
        self.file.seek(0)
        rows = [l.strip().split(",") for l in self.file.read().splitlines() if l.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        for r in rows:
            r = [c.strip() for c in r]
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            for name, val in zip(self.NAMES, r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_images(count, first_seed):
    from paper_1912_01884_gb300 import synth
    return [synth.plain_gaussian(first_seed + j, H, W_IMG, K, B).img for j in range(count)]


def image_seeds(images, seed, rank):
    """Seeds of the images of one rank: every rank takes its own images
    (weak scaling; the images are independent problems)."""
    first = seed * 1000003 + rank * 10007
    return [first + j for j in range(images)]


def max_over_ranks(value, dist, device):
    """The slowest rank's time (the only cross-rank reduction of the run)."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(budget_s=12.0, max_images=8, seed=0):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload's images."""
    import oracle
    imgs = make_images(max_images, 900000 + seed)
    done, t0 = 0, time.perf_counter()
    for img in imgs:
        oracle.detect(img, K, B)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done * H * W_IMG / dt / 1e6, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
            "sample": "%d of the workload's 2048x2048 images, whole method, one thread" % done}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    imgs = make_images(args.steps + args.warmup, 700000 + args.seed)
    for img in imgs[:args.warmup]:
        oracle.detect(img, K, B)
    t0 = time.perf_counter()
    for img in imgs[args.warmup:]:
        oracle.detect(img, K, B)
    dt = time.perf_counter() - t0
    value = args.steps * H * W_IMG / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "images_per_step": 1, "h": H, "w": W_IMG, "k": K,
                   "B": B, "pixel": "u8"},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": 1, "kind": "oracle",
                         "sample": "1 image of the workload per step, whole method, one thread"},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1912_01884_gb300 as fd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    fd.load()
    I = args.images
    from paper_1912_01884_gb300 import synth
    imgs = [synth.plain_gaussian(sd, H, W_IMG, K, B).img for sd in image_seeds(I, args.seed, rank)]
    host = torch.from_numpy(np.stack(imgs)).pin_memory()
    dimg = host.to(dev)
    xs = torch.empty((I, K + 1), dtype=torch.int32, device=dev)
    ds = torch.empty((I, K), dtype=torch.int32, device=dev)
    sc = torch.empty((I, 1), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    plan = fd.BatchPlan([dimg[i] for i in range(I)], [K] * I, [B] * I, out=(xs, ds, sc),
                        stream=stream)
    hx = torch.empty_like(xs, device="cpu").pin_memory()
    hd = torch.empty_like(ds, device="cpu").pin_memory()
    hs = torch.empty_like(sc, device="cpu").pin_memory()

    def step():
        plan.run(stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()

    # --- device-resident throughput -------------------------------------
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = fd.launch_count()
    barrier()
    for e0, e1 in ev:
        e0.record(stream)
        step()
        e1.record(stream)
    barrier()
    launches = fd.launch_count() - l0
    clocks = sampler.stop()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_s = max_over_ranks(sum(step_ms) / 1e3, dist, dev)
    pix = I * H * W_IMG * world * args.steps
    value = pix / total_s / 1e6

    # --- end to end through the public API: H2D + detect + D2H -----------
    h2d = host.numel() * host.element_size()
    d2h = (hx.numel() + hd.numel() + hs.numel()) * 4
    for _ in range(2):
        dimg.copy_(host, non_blocking=True)
        step()
    barrier()
    t0 = time.perf_counter()
    e2e_ev = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dimg.copy_(host, non_blocking=True)
        step()
        hx.copy_(xs, non_blocking=True)
        hd.copy_(ds, non_blocking=True)
        hs.copy_(sc, non_blocking=True)
        e1.record(stream)
        stream.synchronize()
        e2e_ev.append((e0, e1))
    barrier()
    e2e_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in e2e_ev) / 1e3, dist, dev)
    e2e_value = pix / e2e_s / 1e6

    # --- roofline of the engine kernel (one launch per step) --------------
    hbm, peak_kind = peaks()
    alg = algorithmic_bytes_per_image() * I
    per_launch_s = total_s / args.steps
    achieved = alg / per_launch_s / 1e9

    # --- single-image latency (one image per launch, same kernels) --------
    ws1 = torch.empty(fd.workspace_bytes(fd.DTYPE_U8, H, W_IMG, K, B), dtype=torch.uint8,
                      device=dev)
    for _ in range(3):
        fd.detect_polyline(dimg[0], K, B, out=(xs[0], ds[0], sc[0]), ws=ws1, stream=stream)
    lat = []
    for i in range(min(I, 16)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fd.detect_polyline(dimg[i], K, B, out=(xs[i], ds[i], sc[i]), ws=ws1, stream=stream)
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    plan.status(stream=stream)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "images_per_step": I, "h": H, "w": W_IMG, "k": K,
                       "B": B, "pixel": "u8", "parallelism": "images sharded over ranks",
                       "l2": "inputs %d MB per step > 129 MB L2, no flush" % (h2d // 2**20)},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": (NCU_TRAFFIC_BYTES_PER_IMAGE * I
                                     if NCU_TRAFFIC_BYTES_PER_IMAGE else None),
                         "peak_kind": peak_kind,
                         "kernel": "engine_kernel (one persistent launch per step)"},
            "single_image_ms": statistics.median(lat),
            "e2e": {"value": e2e_value, "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        if world == 1 and not args.skip_cpu:
            out["cpu_baseline"] = cpu_baseline(seed=args.seed)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
