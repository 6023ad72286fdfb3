#!/usr/bin/env python
"""Throughput of end-to-end curve detection (band FHT + bend-limited DP +
read-back) in Mpix/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mixed|plain2048|float8192|plain256|angle2048|through2048|
                                horizontal2048|two2048|padded2048|learned1024]
                    [--images I] [--no-extras] [--skip-cpu]

Default workload: the mixed batch of 256 synthetic uint8 images (heights 512..4096,
widths 512..3072, bands of 32..256 rows, bend range 1/8 of the band height).
A step is one pass of the whole method over the batch of distinct seeded
images per GPU: one persistent kernel launch, replayed from a CUDA graph,
inputs already resident in HBM.  Each batch is larger than the 129 MB L2, so
no flush is needed between steps.  The same JSON line carries the 2048x2048
single-size batch and the 8192x8192 float response map as extra keys
(--no-extras omits them).  Under torchrun each rank takes its own images (weak
scaling, no data-path collective) and rank 0 prints one JSON line.
``--impl reference`` times the CPU oracle (the method as a plain C program)
on bounded samples of the same workload on the host cores; the paper has no
code of its own to run.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpix/s end-to-end band-FHT+DP (exact) and % HBM roofline; batched/learned vs plain"

WORKLOADS = {
    "mixed": dict(
        desc="mixed batch: 256 u8 images, h in 512..4096, w in 512..3072 (step 256), band "
             "height 32..256, bend = band/8, uniform noise 0..40 + 1 polyline of 200",
        images=256, dtype="u8"),
    "plain2048": dict(
        desc="u8 2048x2048, k=16 bands of 128 rows, bend |d_{i+1}-d_i|<=16, Gaussian noise + 3 "
             "polylines", images=32, dtype="u8"),
    "float8192": dict(
        desc="f32 8192x8192 ridge response, k=64 bands of 128 rows, bend 24", images=1,
        dtype="f32"),
    "plain256": dict(
        desc="u8 256x256, k=4 bands of 64 rows, bend 8, uniform noise + 1 polyline", images=2048,
        dtype="u8"),
    "angle2048": dict(
        desc="main problem: u8 2048x2048 bent edges with salt noise, rows smoothed with the "
             "binomial Gaussian r=2, k=16 bands of 128 rows, bend angle <= 10 degrees",
        images=32, dtype="u8"),
    "angle2048batch": dict(
        desc="main problem, batched: the angle2048 images (u8 2048x2048 bent edges, r=2, k=16, "
             "bend angle <= 10 degrees), each step smoothing every image's rows and running all "
             "32 in one persistent launch with the window table (fhtdp_batch_angle)",
        images=32, dtype="u8"),
    "through2048": dict(
        desc="Subproblem 3: u8 2048x2048 (the plain2048 images), k=16 bands of 128 rows, bend 16, "
             "the best polyline through one point per image on band border 8",
        images=32, dtype="u8"),
    "through2048batch": dict(
        desc="Subproblem 3, batched: the through2048 images and points (u8 2048x2048, k=16, bend "
             "16, one point per image on band border 8) in one persistent launch "
             "(fhtdp_batch_points)", images=32, dtype="u8"),
    "horizontal2048": dict(
        desc="mostly horizontal curves: u8 2048x2048 (the plain2048 images transposed), k=16 "
             "vertical strips of 128 columns, bend 16 (each step transposes its images and runs "
             "them as one batch)", images=32, dtype="u8"),
    "padded2048": dict(
        desc="vertices in the zero padding: u8 2048x2048 (the plain2048 images), k=16 bands of "
             "128 rows, bend 16, every vertex in [0, w + 128)", images=32, dtype="u8"),
    "two2048": dict(
        desc="two different extreme polylines: u8 2048x2048 (the plain2048 images), k=16, "
             "bend 16, the second polyline's top vertex at least 64 columns from the first's",
        images=32, dtype="u8"),
    "learned1024": dict(
        desc="u8 1024x1024 lanes over textured noise, k=16 bands of 64 rows, bend 12: learned "
             "window proposal (4-layer 32-channel bf16 CNN on the 4x downsample, windows of 16) "
             "+ pruned DP + full-DP fallback, against the plain DP", images=512, dtype="u8"),
}
# Workloads measured by the default run besides the headline one (N = 1).
EXTRAS = ("plain2048", "float8192")

# DRAM bytes (read + write) per pixel of the fused engine's launch on each
# batched workload, from the ncu captures summarised in profiles/; a launch's
# traffic is this times its pixels.  None where no capture of the current
# kernel exists (reset whenever the kernel changes until it is captured again).
NCU_TRAFFIC_BYTES_PER_PIXEL = {
    "mixed": 15.0048e9 / 1064894464,     # engine_kernel_u8<int, 1>: 4.445 + 10.559 GB
    "plain2048": 1.2455e9 / 134217728,   # engine_kernel_u8<int, 0>: 0.216 + 1.030 GB
    "float8192": 1.2905e9 / 67108864,    # engine_kernel_wide: 0.275 + 1.015 GB
}
# DRAM bytes of one dp_band_window_kernel band launch on the 2048x2048, k = 16
# workloads (profiles/dp_band_window_kernel_angle2048.md).
NCU_TRAFFIC_DP_WINDOW_LAUNCH = 4.14e6


# The main problem's smoothing half-width and bend angle (the paper's
# Fig. 3 example bends by at most 10 degrees).
ANGLE_R = 2
ANGLE_GAMMA = 0.17453292519943295   # 10 degrees in radians


# The through-point workload's query: border 8 of 16, at the first planted
# polyline's vertex there.
THROUGH_BORDER = 8
# The two-polyline workload's suppression radius on the top vertex.
TWO_SEPARATION = 64


def through_column(wl):
    return int(wl.planted[0][0][THROUGH_BORDER])


def algorithmic_bytes(h, w, k, bpp):
    """Bytes the method must move per image: read the image once, write and
    read one 4-byte DP value per state (x, d) of every band, and the path."""
    n = h // k
    return h * w * bpp + k * 8 * (2 * n - 1) * w + 4 * (2 * k + 2)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="mixed", choices=sorted(WORKLOADS))
    ap.add_argument("--images", type=int, default=0, help="images per step per GPU")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU baseline leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="omit the extra workloads of the default run")
    ap.add_argument("--lanes", type=int, default=0,
                    help="angle2048: streams a step spreads its images over (default 8)")
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
    """SM clocks and throttle reasons sampled during the timed region: through
    NVML (every 10 ms, read-only queries) where libnvidia-ml loads, else with
    nvidia-smi every 200 ms."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    # NVML clock-event reason bits (public NVML API constants)
    BITS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
            0x4: "sw_power_cap"}
    PERIOD_S = 0.01

    def __init__(self, gpu_index, uuid=None):
        self.gpu = gpu_index
        self.uuid = uuid
        self.proc = None
        self.file = None
        self.nvml = None
        self.thread = None
        self.samples = []
        self.smax = None
        self.stop_flag = threading.Event()

    def _nvml_open(self):
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            found = False
            if self.uuid:   # the CUDA device itself, whatever CUDA_VISIBLE_DEVICES says
                found = lib.nvmlDeviceGetHandleByUUID(self.uuid.encode(), ctypes.byref(h)) == 0
            if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu),
                                                               ctypes.byref(h)) != 0:
                return None
            self.reasons_fn = (getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or
                               getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None))
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:   # NVML_CLOCK_SM
                self.smax = float(mx.value)
            return lib, h
        except OSError:
            return None

    def _nvml_loop(self):
        lib, h = self.nvml
        clk = ctypes.c_uint()
        reasons = ctypes.c_ulonglong()
        while not self.stop_flag.is_set():
            ok = lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0
            rr = (self.reasons_fn is not None and
                  self.reasons_fn(h, ctypes.byref(reasons)) == 0)
            if ok:
                self.samples.append((float(clk.value), int(reasons.value) if rr else 0))
            time.sleep(self.PERIOD_S)

    def start(self):
        self.nvml = self._nvml_open()
        if self.nvml:
            self.thread = threading.Thread(target=self._nvml_loop, daemon=True)
            self.thread.start()
            return
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.thread is not None:
            self.stop_flag.set()
            self.thread.join(timeout=5)
            sm = [c for c, _ in self.samples]
            reasons = set()
            for _, r in self.samples:
                for bit, name in self.BITS.items():
                    if r & bit:
                        reasons.add(name)
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": self.smax,
                    "reasons": sorted(reasons), "samples": len(sm), "source": "nvml, 10 ms"}
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
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 200 ms"}


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


def make_workload(name, images, seed, rank):
    """[(img, k, B)] of one rank."""
    import numpy as np
    from paper_1912_01884_gb300 import synth
    seeds = image_seeds(images, seed, rank)
    if name == "plain2048":
        return [(w.img, w.k, w.B) for w in (synth.plain_gaussian(s) for s in seeds)]
    if name == "plain256":
        return [(w.img, w.k, w.B) for w in (synth.plain_uniform(s, 256, 256, 4, 8) for s in seeds)]
    if name == "float8192":
        return [(w.img, w.k, w.B) for w in (synth.ridge_response(s) for s in seeds)]
    if name in ("angle2048", "angle2048batch"):
        return [(w.img, w.k, None) for w in (synth.bent_edges(s) for s in seeds)]
    if name == "horizontal2048":
        return [(np.ascontiguousarray(w.img.T), w.k, w.B)
                for w in (synth.plain_gaussian(s) for s in seeds)]
    if name == "padded2048":
        return [(w.img, w.k, ("padded", w.B)) for w in (synth.plain_gaussian(s) for s in seeds)]
    if name == "two2048":
        return [(w.img, w.k, ("two", w.B, TWO_SEPARATION))
                for w in (synth.plain_gaussian(s) for s in seeds)]
    if name in ("through2048", "through2048batch"):
        return [(w.img, w.k, (w.B, THROUGH_BORDER, through_column(w)))
                for w in (synth.plain_gaussian(s) for s in seeds)]
    shapes = synth.mixed_batch_shapes(seed * 7919 + rank, images)
    return [(synth.plain_uniform(s, h, w, k, B).img, k, B)
            for s, (h, w, k, B) in zip(seeds, shapes)]


def oracle_one(item, horizontal=False):
    """The oracle on one image of a workload (the whole method)."""
    import numpy as np
    import oracle
    img, k, B = item
    if B is None:
        oracle.detect_angle(img, k, ANGLE_R, ANGLE_GAMMA)
    elif isinstance(B, tuple) and B[0] == "two":
        oracle.detect_two(img, k, B[1], B[2])
    elif isinstance(B, tuple) and B[0] == "padded":
        oracle.detect_padded(img, k, B[1])
    elif isinstance(B, tuple):
        oracle.detect_through(img, k, *B)
    elif horizontal:
        oracle.detect_horizontal(img, k, B)
    elif img.dtype == np.float32:
        oracle.detect_f32(img, k, B)
    else:
        oracle.detect(img, k, B)
    return img.size


def oracle_rate(items, budget_s, horizontal=False):
    """The oracle as it stands, one thread, on images of the workload until
    `budget_s` has passed: (Mpix/s, images done)."""
    done, pix, t0 = 0, 0, time.perf_counter()
    for item in items:
        pix += oracle_one(item, horizontal)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return pix / (time.perf_counter() - t0) / 1e6, done


def host_threads():
    """Threads for the all-core oracle leg (the host's cores, at most 64)."""
    return max(1, min(64, os.cpu_count() or 1))


def oracle_rate_threads(items, threads, horizontal=False):
    """The oracle as it stands on `items`, one image per task over `threads`
    host threads (its C calls release the interpreter lock): (Mpix/s, images)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        pix = sum(ex.map(lambda it: oracle_one(it, horizontal), items))
    return pix / (time.perf_counter() - t0) / 1e6, len(items)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(name, seed):
    """The oracle on bounded samples of the workload: one thread (images until
    12 s have passed) and every host core (two images per thread)."""
    horizontal = name == "horizontal2048"
    one_rate, one_done = oracle_rate(make_workload(name, 8, 900000 + seed, 0), 12.0, horizontal)
    th = host_threads()
    sample = make_workload(name, 2 * th, 950000 + seed, 0)
    all_rate, all_done = oracle_rate_threads(sample, th, horizontal)
    return {"value": all_rate, "unit": "Mpix/s", "cores": th, "kind": "oracle",
            "sample": "%d images of the workload, whole method, one image per task on %d host "
                      "threads" % (all_done, th),
            "single_thread": {"value": one_rate, "unit": "Mpix/s", "cores": 1,
                              "sample": "%d images of the workload, one thread" % one_done},
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    spec = WORKLOADS[args.workload]
    th = host_threads()
    hor = args.workload == "horizontal2048"
    # Each step: a bounded sample of the workload, one image per host thread.
    items = make_workload(args.workload, (args.steps + args.warmup) * th, 700000 + args.seed, 0)
    steps = [items[i * th:(i + 1) * th] for i in range(args.steps + args.warmup)]
    for st in steps[:args.warmup]:
        oracle_rate_threads(st, th, hor)
    t0 = time.perf_counter()
    pix = 0
    for st in steps[args.warmup:]:
        oracle_rate_threads(st, th, hor)
        pix += sum(it[0].size for it in st)
    dt = time.perf_counter() - t0
    value = pix / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if spec["dtype"] == "u8" else "f32",
        "data": "synthetic",
        "config": {"workload": spec["desc"], "images_per_step": th},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": th, "kind": "oracle",
                         "sample": "%d images of the workload per step, whole method, one "
                                   "image per task on %d host threads" % (th, th),
                         "nproc": os.cpu_count(), "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def gpu_uuid(dev):
    """NVML name of a CUDA device ("GPU-<uuid>"), or None."""
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except (AttributeError, RuntimeError):
        return None


class BatchBench:
    """One batched workload on this rank's GPU: its images resident in HBM,
    a tuned batch plan, and a CUDA graph of one step (one persistent launch)."""

    def __init__(self, name, images, seed, rank, dev):
        import numpy as np
        import torch
        import paper_1912_01884_gb300 as fd
        self.fd, self.torch, self.dev = fd, torch, dev
        self.name = name
        spec = WORKLOADS[name]
        self.items = make_workload(name, images, seed, rank)
        self.tdt = torch.float32 if spec["dtype"] == "f32" else torch.uint8
        self.esize = 4 if spec["dtype"] == "f32" else 1
        self.horizontal = name == "horizontal2048"
        # Inputs: one pinned host buffer and one device buffer, image after
        # image (each 256-byte aligned); outputs in flat device buffers.
        self.offs, total = [], 0
        for img, _, _ in self.items:
            self.offs.append(total)
            total += (img.size * self.esize + 255) // 256 * 256
        self.host = torch.empty(total, dtype=torch.uint8).pin_memory()
        for (img, _, _), o in zip(self.items, self.offs):
            self.host[o:o + img.size * self.esize].view(self.tdt).view(img.shape).copy_(
                torch.from_numpy(img))
        self.dbuf = self.host.to(dev)
        self.views = self._views(self.dbuf)
        self.ks = [k for _, k, _ in self.items]
        self.Bs = [B for _, _, B in self.items]
        # through-point batches: (B, border, column) per image
        self.points = None
        if name == "through2048batch":
            self.points = [(B[1], B[2]) for B in self.Bs]
            self.Bs = [B[0] for B in self.Bs]
        self.xs = torch.empty(sum(k + 1 for k in self.ks), dtype=torch.int32, device=dev)
        self.ds = torch.empty(sum(self.ks), dtype=torch.int32, device=dev)
        self.sc = torch.empty(len(self.items), dtype=torch.float32 if self.tdt == torch.float32
                              else torch.int32, device=dev)
        xo = np.cumsum([0] + [k + 1 for k in self.ks])
        do = np.cumsum([0] + self.ks)
        self.outs = ([self.xs[xo[i]:xo[i + 1]] for i in range(len(self.items))],
                     [self.ds[do[i]:do[i + 1]] for i in range(len(self.items))],
                     [self.sc[i:i + 1] for i in range(len(self.items))])
        self.stream = torch.cuda.Stream(dev)   # graphs are captured off the default stream
        if self.horizontal:
            # every step transposes its images (fhtdp_transpose) into buffers
            # that one batch plan runs over
            self.tviews = [torch.empty((img.shape[1], img.shape[0]), dtype=self.tdt, device=dev)
                           for img, _, _ in self.items]
            self.plan = fd.BatchPlan(self.tviews, self.ks, self.Bs, out=self.outs,
                                     stream=self.stream)
        else:
            self.plan = fd.BatchPlan(self.views, self.ks, self.Bs, out=self.outs,
                                     stream=self.stream)
        if self.points:
            self.plan.points(self.points, stream=self.stream)
        # Untimed set-up: the library's tuner picks the queue schedule and, per
        # band height, the tile width and register depth.
        self.width = self.plan.autotune(reps=2, stream=self.stream)
        self.pixels = sum(img.size for img, _, _ in self.items)
        self.alg = sum(algorithmic_bytes(img.shape[0], img.shape[1], k, self.esize)
                       for img, k, _ in self.items)

    def _views(self, buf):
        return [buf[o:o + img.size * self.esize].view(self.tdt).view(img.shape)
                for (img, _, _), o in zip(self.items, self.offs)]

    def enqueue(self, plan=None, src=None):
        """One step on self.stream: the whole batch, one persistent launch."""
        if self.horizontal:
            for v, t in zip(src or self.views, self.tviews):
                self.fd.transpose(v, out=t, stream=self.stream)
        (plan or self.plan).run(stream=self.stream)

    def capture(self):
        """A CUDA graph of one step; returns the launches it holds."""
        torch = self.torch
        self.enqueue()   # first use outside the capture
        torch.cuda.synchronize(self.dev)
        l0 = self.fd.launch_count()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.enqueue()
        return self.fd.launch_count() - l0

    def choices(self):
        ns = sorted(set(img.shape[0] // k for img, k, _ in self.items))
        if self.horizontal:
            ns = sorted(set(img.shape[1] // k for img, k, _ in self.items))
        ch = {n: self.plan.choice(n) for n in ns}
        first = next(iter(ch.values()))
        return {"schedule": first["schedule"], "width": first["width"],
                "per_band_height": {str(n): {"tile": c["tile"], "fht_register_levels": c["depth"]}
                                    for n, c in ch.items()}}

    def timed_replays(self, steps, warmup, barrier):
        """Device time of `steps` graph replays (CUDA events on the replay
        stream), after `warmup` untimed ones."""
        torch = self.torch
        with torch.cuda.stream(self.stream):   # replay() launches on the current stream
            for _ in range(warmup):
                self.graph.replay()
            barrier()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            # an NVTX range names the timed launches for profilers
            torch.cuda.nvtx.range_push("timed_" + self.name)
            for e0, e1 in ev:
                e0.record(self.stream)
                self.graph.replay()
                e1.record(self.stream)
            torch.cuda.nvtx.range_pop()
            barrier()
        self.plan.status(stream=self.stream)
        return sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3

    def e2e(self, steps, barrier):
        """End to end through the public API: every step copies its inputs from
        pinned host memory and reads its results back inside the timed region.
        Two input buffers (and a plan on each) let the copy of step i+1 run on
        a copy stream while step i computes; events order each buffer's copy,
        use and re-use."""
        torch, fd = self.torch, self.fd
        dbuf2 = torch.empty_like(self.dbuf)
        views2 = self._views(dbuf2)
        if self.horizontal:
            plan2 = self.plan
        else:
            plan2 = fd.BatchPlan(views2, self.ks, self.Bs, out=self.outs, stream=self.stream)
            if self.points:
                plan2.points(self.points, stream=self.stream)
            plan2.autotune(reps=1, stream=self.stream)
        plans, bufs, srcs = (self.plan, plan2), (self.dbuf, dbuf2), (self.views, views2)
        copy_stream = torch.cuda.Stream(self.dev)
        hx = torch.empty_like(self.xs, device="cpu").pin_memory()
        hd = torch.empty_like(self.ds, device="cpu").pin_memory()
        hs = torch.empty_like(self.sc, device="cpu").pin_memory()
        stream = self.stream

        def run(nsteps):
            copied = [torch.cuda.Event() for _ in range(2)]
            used = [torch.cuda.Event() for _ in range(2)]
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            copy_stream.wait_event(t0)
            with torch.cuda.stream(copy_stream):
                bufs[0].copy_(self.host, non_blocking=True)
            copied[0].record(copy_stream)
            for i in range(nsteps):
                b = i % 2
                if i + 1 < nsteps:   # next step's inputs, once that buffer is free
                    nb = 1 - b
                    if i >= 1:
                        copy_stream.wait_event(used[nb])
                    with torch.cuda.stream(copy_stream):
                        bufs[nb].copy_(self.host, non_blocking=True)
                    copied[nb].record(copy_stream)
                stream.wait_event(copied[b])
                self.enqueue(plans[b], srcs[b])
                used[b].record(stream)
                with torch.cuda.stream(stream):
                    hx.copy_(self.xs, non_blocking=True)
                    hd.copy_(self.ds, non_blocking=True)
                    hs.copy_(self.sc, non_blocking=True)
            t1.record(stream)
            stream.synchronize()
            return t0.elapsed_time(t1) / 1e3

        run(2)
        barrier()
        t = run(steps)
        barrier()
        h2d = self.dbuf.numel()
        d2h = (hx.numel() + hd.numel() + hs.numel()) * 4
        return t, h2d, d2h

    def single_image_ms(self):
        """Median latency of one image per launch (the first image)."""
        torch, fd = self.torch, self.fd
        img0, k0, B0 = self.views[0], self.ks[0], self.Bs[0]
        dcode = fd.DTYPE_F32 if self.tdt == torch.float32 else fd.DTYPE_U8
        if self.horizontal:
            ws1 = torch.empty(fd.horizontal_workspace_bytes(dcode, img0.shape[0], img0.shape[1],
                                                            k0, B0), dtype=torch.uint8,
                              device=self.dev)
            detect_one = fd.detect_polyline_horizontal
        else:
            ws1 = torch.empty(fd.workspace_bytes(dcode, img0.shape[0], img0.shape[1], k0, B0),
                              dtype=torch.uint8, device=self.dev)
            detect_one = fd.detect_polyline
        one = (self.outs[0][0], self.outs[1][0], self.outs[2][0])
        for _ in range(3):
            detect_one(img0, k0, B0, out=one, ws=ws1, stream=self.stream)
        lat = []
        for _ in range(8):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            detect_one(img0, k0, B0, out=one, ws=ws1, stream=self.stream)
            e1.record(self.stream)
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
        return statistics.median(lat)


def roofline(bb, per_step_s):
    """Roofline of the fused engine's launch (one per step): algorithmic
    bytes per launch over its CUDA-event time, against the measured HBM
    copy bandwidth; traffic from the ncu capture of the same kernel."""
    hbm, peak_kind = peaks()
    achieved = bb.alg / per_step_s / 1e9
    tpp = NCU_TRAFFIC_BYTES_PER_PIXEL.get(bb.name)
    kern = ("engine_kernel (float images, one persistent launch per step)"
            if bb.tdt == bb.torch.float32 else
            "engine_kernel_u8 (one persistent launch per step%s)"
            % (", after one transpose_kernel per image" if bb.horizontal else ""))
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": tpp * bb.pixels if tpp else None,
            "peak_kind": peak_kind, "algorithmic_bytes_per_launch": bb.alg, "kernel": kern}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1912_01884_gb300 as fd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    fd.load()
    spec = WORKLOADS[args.workload]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    bb = BatchBench(args.workload, args.images or spec["images"], args.seed, rank, dev)
    launches_per_step = bb.capture()
    barrier()
    # --- device-resident throughput: graph replays, clocks sampled ---------
    sampler = ClockSampler(local, gpu_uuid(dev))
    sampler.start()
    total_s = bb.timed_replays(args.steps, args.warmup, barrier)
    clocks = sampler.stop()
    total_s = max_over_ranks(total_s, dist, dev)
    value = bb.pixels * world * args.steps / total_s / 1e6
    # --- end to end through the public API: H2D + detect + D2H -----------
    e2e_s, h2d, d2h = bb.e2e(args.steps, barrier)
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = bb.pixels * world * args.steps / e2e_s / 1e6
    lat = bb.single_image_ms()
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if bb.tdt == torch.float32 else "int32", "data": "synthetic",
            "config": {"workload": spec["desc"], "images_per_step": len(bb.items),
                       "pixels_per_step": bb.pixels, "parallelism": "images sharded over ranks",
                       "l2": "inputs %d MB per step %s 129 MB L2, no flush"
                             % (bb.dbuf.numel() // 2**20, ">" if bb.dbuf.numel() > 129e6 else "<"),
                       "timing": "CUDA-graph replay of one step per timed step",
                       "tuned": bb.choices()},
            "roofline": roofline(bb, total_s / args.steps),
            "single_image_ms": lat,
            "e2e": {"value": e2e_value, "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
        }
    del bb
    torch.cuda.empty_cache()
    # --- extra workloads of the default run (one GPU) ----------------------
    if world == 1 and not args.no_extras and args.workload == "mixed":
        for name in EXTRAS:
            eb = BatchBench(name, WORKLOADS[name]["images"], args.seed, rank, dev)
            eb.capture()
            # at least ~100 ms of timed work, so that the clock samples cover it
            probe = eb.timed_replays(2, 1, barrier) / 2
            steps = int(min(400, max(args.steps, 0.1 / max(probe, 1e-6))))
            s_ = ClockSampler(local, gpu_uuid(dev))
            s_.start()
            t = eb.timed_replays(steps, max(args.warmup, 3), barrier)
            ck = s_.stop()
            out[name] = {"value": eb.pixels * steps / t / 1e6, "unit": "Mpix/s",
                         "ms_per_step": t / steps * 1e3, "steps": steps,
                         "images_per_step": len(eb.items), "workload": WORKLOADS[name]["desc"],
                         "roofline": roofline(eb, t / steps), "tuned": eb.choices(),
                         "clocks": ck}
            del eb
            torch.cuda.empty_cache()
    if rank == 0:
        if world == 1 and not args.skip_cpu:
            out["cpu_baseline"] = cpu_baseline(args.workload, args.seed)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


ANGLE_LANES = 8   # streams over which one step spreads its images (4: -4 %, 2: -21 %)


def run_standalone(args):
    """The calls that run on the standalone kernels, on a batch of images per
    step: the main problem (angle2048: smoothing + band FHT + bend-angle DP +
    read-back, one fhtdp_detect_polyline_angle call of 24 launches per image)
    or the through-point query (through2048: band FHT + DP with the point's
    band masked + read-back, one fhtdp_detect_through_point call per image).
    A step spreads the images over ANGLE_LANES streams, each with its own
    workspace, and is captured once as a CUDA graph that every timed step
    replays."""
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
    name = args.workload
    spec = WORKLOADS[name]
    I = args.images or spec["images"]
    items = make_workload(name, I, args.seed, rank)
    h, w = items[0][0].shape
    k = items[0][1]
    angle = name == "angle2048"
    host = torch.empty((I, h, w), dtype=torch.uint8).pin_memory()
    for j, (img, _, _) in enumerate(items):
        host[j].copy_(torch.from_numpy(img))
    imgs = host.to(dev)
    xs = torch.empty((I, k + 1), dtype=torch.int32, device=dev)
    ds = torch.empty((I, k), dtype=torch.int32, device=dev)
    sc = torch.empty((I, 1), dtype=torch.int32, device=dev)
    if angle:
        need = fd.angle_workspace_bytes(fd.DTYPE_U8, h, w, k, ANGLE_R)
    elif name == "horizontal2048":
        need = fd.horizontal_workspace_bytes(fd.DTYPE_U8, h, w, k, items[0][2])
    else:
        need = fd.through_workspace_bytes(fd.DTYPE_U8, h, w, k)
    two = name == "two2048"
    if two:   # two polylines per image
        xs2 = torch.empty((I, 2, k + 1), dtype=torch.int32, device=dev)
        ds2 = torch.empty((I, 2, k), dtype=torch.int32, device=dev)
        sc2 = torch.empty((I, 2), dtype=torch.int32, device=dev)
    lanes = min(args.lanes or ANGLE_LANES, I)
    wss = [torch.empty(need, dtype=torch.uint8, device=dev) for _ in range(lanes)]
    main = torch.cuda.Stream(dev)      # graphs are captured off the default stream
    torch.cuda.set_stream(main)
    side = [torch.cuda.Stream(dev) for _ in range(lanes)]

    def enqueue(src):
        # fork: every lane waits for the main stream, runs its images, joins
        for ln in range(lanes):
            side[ln].wait_stream(main)
            for j in range(ln, I, lanes):
                if angle:
                    fd.detect_polyline_angle(src[j], k, ANGLE_R, ANGLE_GAMMA,
                                             out=(xs[j], ds[j], sc[j]), ws=wss[ln],
                                             stream=side[ln])
                elif name == "horizontal2048":
                    fd.detect_polyline_horizontal(src[j], k, items[j][2],
                                                  out=(xs[j], ds[j], sc[j]), ws=wss[ln],
                                                  stream=side[ln])
                elif two:
                    fd.detect_two_polylines(src[j], k, items[j][2][1], items[j][2][2],
                                            out=(xs2[j], ds2[j], sc2[j]), ws=wss[ln],
                                            stream=side[ln])
                elif name == "padded2048":
                    fd.detect_polyline_padded(src[j], k, items[j][2][1],
                                              out=(xs[j], ds[j], sc[j]), ws=wss[ln],
                                              stream=side[ln])
                else:
                    B, jb, xp = items[j][2]
                    fd.detect_through_point(src[j], k, B, jb, xp, out=(xs[j], ds[j], sc[j]),
                                            ws=wss[ln], stream=side[ln])
        for ln in range(lanes):
            main.wait_stream(side[ln])

    enqueue(imgs)   # untimed: first-use set-up outside the capture
    torch.cuda.synchronize(dev)
    l0 = fd.launch_count()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=main):
        enqueue(imgs)
    launches_per_step = fd.launch_count() - l0

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        graph.replay()
    barrier()
    sampler = ClockSampler(local, gpu_uuid(dev))
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    for e0, e1 in ev:
        e0.record(main)
        graph.replay()
        e1.record(main)
    barrier()
    clocks = sampler.stop()
    total_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, dev)
    pix_rank = I * h * w
    value = pix_rank * world * args.steps / total_s / 1e6

    # End to end: each step copies its images from pinned host memory, runs
    # the graph on them and reads every result back, all inside the timed
    # region (copies on the main stream, ordered before the graph).
    rx, rd, rs = (xs2, ds2, sc2) if two else (xs, ds, sc)
    hx = torch.empty_like(rx, device="cpu").pin_memory()
    hd = torch.empty_like(rd, device="cpu").pin_memory()
    hs = torch.empty_like(rs, device="cpu").pin_memory()

    def e2e_run(nsteps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(main)
        for _ in range(nsteps):
            imgs.copy_(host, non_blocking=True)
            graph.replay()
            hx.copy_(rx, non_blocking=True)
            hd.copy_(rd, non_blocking=True)
            hs.copy_(rs, non_blocking=True)
        t1.record(main)
        main.synchronize()
        return t0.elapsed_time(t1) / 1e3

    e2e_run(1)
    barrier()
    e2e_s = max_over_ranks(e2e_run(args.steps), dist, dev)
    e2e_value = pix_rank * world * args.steps / e2e_s / 1e6

    # Stage times on one image through the modular calls (one stream), to
    # find the dominant kernel and its roofline.
    ws_tmp = torch.empty(fd.fht_workspace_bytes(fd.DTYPE_I32, h, w, k), dtype=torch.uint8,
                         device=dev)
    smooth = torch.empty((h, w), dtype=torch.int32, device=dev)
    hough = torch.empty((k, 2, h // k, w + h // k), dtype=torch.int32, device=dev)
    one = (xs[0], ds[0], sc[0])
    if angle:
        stages = {
            "gauss_rows": lambda: fd.gauss_rows(imgs[0], ANGLE_R, out=smooth, stream=main),
            "fht_bands": lambda: fd.fht_bands(smooth, k, out=hough, ws=ws_tmp, stream=main),
            "dp_angle": lambda: fd.polyline_dp_angle(hough, h, w, k, ANGLE_GAMMA, stream=main),
            "backtrack": lambda: fd.backtrack_angle(hough, h, w, k, ANGLE_GAMMA, out=one,
                                                    stream=main),
        }
    elif name == "horizontal2048":
        B0 = items[0][2]
        ws_e = torch.empty(fd.workspace_bytes(fd.DTYPE_U8, w, h, k, B0), dtype=torch.uint8,
                           device=dev)
        # the transposed image a horizontal call leaves at the start of its
        # workspace (row pitch h rounded up to 64)
        tp = (h + 63) // 64 * 64
        tr = wss[0][:w * tp].view(w, tp)[:, :h]
        stages = {
            "horizontal": lambda: fd.detect_polyline_horizontal(imgs[0], k, B0, out=one,
                                                                ws=wss[0], stream=main),
            "engine": lambda: fd.detect_polyline(tr, k, B0, out=one, ws=ws_e, stream=main),
        }
    else:
        B0 = items[0][2][1] if (two or name == "padded2048") else items[0][2][0]
        stages = {
            "fht_bands": lambda: fd.fht_bands(imgs[0], k, out=hough, ws=ws_tmp, stream=main),
            "dp": lambda: fd.polyline_dp(hough, h, w, k, B0, stream=main),
            "backtrack": lambda: fd.backtrack(hough, h, w, k, B0, out=one, stream=main),
        }
    stage_ms = {name: [] for name in stages}
    for rep in range(6):
        for sname, fn in stages.items():
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            fn()
            b.record(main)
            b.synchronize()
            if rep >= 2:
                stage_ms[sname].append(a.elapsed_time(b))
    stage_ms = {sname: statistics.median(v) for sname, v in stage_ms.items()}
    n = h // k
    D = 2 * n - 1
    # minimal DRAM bytes of each stage run on its own
    stage_bytes = {
        "gauss_rows": h * w * (1 + 4),
        "fht_bands": h * w * (4 if angle else 1) + k * 2 * n * (w + n) * 4,
        "dp_angle": (k - 1) * 3 * D * w * 4,
        "dp": (k - 1) * 3 * D * w * 4,
        "backtrack": D * w * 4,
        "horizontal": algorithmic_bytes(w, h, k, 1) + 2 * h * w,
        "engine": algorithmic_bytes(w, h, k, 1),
    }
    # The roofline kernel is the DP (the largest share of the launch list);
    # "backtrack" here is the standalone one-block read-back, not the argmax
    # + one-warp read-back that the detection calls run.
    top = "dp_angle" if angle else ("engine" if name == "horizontal2048" else "dp")
    hbm, peak_kind = peaks()
    achieved = stage_bytes[top] / (stage_ms[top] / 1e3) / 1e9

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": spec["desc"], "images_per_step": I,
                       "pixels_per_step": pix_rank, "parallelism": "images sharded over ranks",
                       "lanes": lanes,
                       **({"r": ANGLE_R, "gamma_rad": ANGLE_GAMMA} if angle else
                          {"B": items[0][2]} if name == "horizontal2048" else
                          {"B": items[0][2][1], "separation": TWO_SEPARATION} if two else
                          {"B": items[0][2][1], "vertex_domain": "[0, w + n)"}
                          if name == "padded2048" else
                          {"B": items[0][2][0], "border": THROUGH_BORDER}),
                       "l2": "inputs %d MB per step %s 129 MB L2, no flush"
                             % (host.numel() // 2**20, ">" if host.numel() > 129e6 else "<")},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm,
                         "traffic": NCU_TRAFFIC_DP_WINDOW_LAUNCH * (k - 1)
                                    if NCU_TRAFFIC_DP_WINDOW_LAUNCH and top != "engine" else None,
                         "peak_kind": peak_kind,
                         "kernel": ("engine_kernel_u8 (one image per launch, the transposed "
                                    "image)" if top == "engine" else
                                    "dp_band_window_kernel (the k-1 band launches of one image "
                                    "and the last-band kernel, timed together)")},
            "stages_ms_one_image": stage_ms,
            "pipeline_frac_of_hbm": sum(algorithmic_bytes(h, w, k, 1) for _ in range(I))
                                    / (total_s / args.steps) / 1e9 / hbm,
            "e2e": {"value": e2e_value, "unit": "Mpix/s", "h2d_bytes_per_step": host.numel(),
                    "d2h_bytes_per_step": (hx.numel() + hd.numel() + hs.numel()) * 4},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
        }
        if world == 1 and not args.skip_cpu:
            out["cpu_baseline"] = cpu_baseline(name, args.seed)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_angle_batch(args):
    """The main problem for a batch: every step smooths each image's rows
    (fhtdp_gauss_rows, int32) and runs all of them in one persistent launch
    of the int32 engine with the bend-angle window table (fhtdp_batch_angle),
    captured once as a CUDA graph that every timed step replays."""
    import torch
    import torch.distributed as dist

    import paper_1912_01884_gb300 as fd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    fd.load()
    name = args.workload
    spec = WORKLOADS[name]
    I = args.images or spec["images"]
    items = make_workload(name, I, args.seed, rank)
    h, w = items[0][0].shape
    k = items[0][1]
    n = h // k
    host = torch.empty((I, h, w), dtype=torch.uint8).pin_memory()
    for j, (img, _, _) in enumerate(items):
        host[j].copy_(torch.from_numpy(img))
    imgs = host.to(dev)
    smooth = torch.empty((I, h, w), dtype=torch.int32, device=dev)
    main = torch.cuda.Stream(dev)
    torch.cuda.set_stream(main)
    plan = fd.BatchPlan([smooth[j] for j in range(I)], [k] * I, [2 * n - 2] * I, stream=main)
    plan.angle(ANGLE_GAMMA)
    for j in range(I):   # untimed: the tuner runs on smoothed rows
        fd.gauss_rows(imgs[j], ANGLE_R, out=smooth[j], stream=main)
    plan.autotune(reps=2, stream=main)
    choice = plan.choice(n)

    def enqueue():
        for j in range(I):
            fd.gauss_rows(imgs[j], ANGLE_R, out=smooth[j], stream=main)
        plan.run(stream=main)

    enqueue()
    torch.cuda.synchronize(dev)
    l0 = fd.launch_count()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=main):
        enqueue()
    launches_per_step = fd.launch_count() - l0

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        graph.replay()
    barrier()
    sampler = ClockSampler(local, gpu_uuid(dev))
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    for e0, e1 in ev:
        e0.record(main)
        graph.replay()
        e1.record(main)
    barrier()
    clocks = sampler.stop()
    total_s = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, dev)
    pix_rank = I * h * w
    value = pix_rank * world * args.steps / total_s / 1e6

    # End to end: the images from pinned host memory and every result back.
    hx = torch.empty((I, k + 1), dtype=torch.int32).pin_memory()
    hd = torch.empty((I, k), dtype=torch.int32).pin_memory()
    hs = torch.empty((I, 1), dtype=torch.int32).pin_memory()

    def e2e_run(nsteps):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(main)
        for _ in range(nsteps):
            imgs.copy_(host, non_blocking=True)
            graph.replay()
            for j in range(I):
                hx[j].copy_(plan.x[j], non_blocking=True)
                hd[j].copy_(plan.d[j], non_blocking=True)
                hs[j].copy_(plan.score[j].reshape(-1), non_blocking=True)
        t1.record(main)
        main.synchronize()
        return t0.elapsed_time(t1) / 1e3

    e2e_run(1)
    barrier()
    e2e_s = max_over_ranks(e2e_run(args.steps), dist, dev)
    e2e_value = pix_rank * world * args.steps / e2e_s / 1e6

    # The dominant kernel: the engine launch alone (events on its stream),
    # against the bytes the method must move from the smoothed int32 rows.
    eng_ms = []
    for rep in range(8):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(main)
        plan.run(stream=main)
        b.record(main)
        b.synchronize()
        if rep >= 3:
            eng_ms.append(a.elapsed_time(b))
    eng_ms = statistics.median(eng_ms)
    eng_bytes = I * algorithmic_bytes(h, w, k, 4)
    hbm, peak_kind = peaks()
    achieved = eng_bytes / (eng_ms / 1e3) / 1e9

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": spec["desc"], "images_per_step": I,
                       "pixels_per_step": pix_rank, "parallelism": "images sharded over ranks",
                       "r": ANGLE_R, "gamma_rad": ANGLE_GAMMA,
                       "tuned": {"schedule": choice["schedule"], "width": choice["width"]},
                       "l2": "inputs %d MB per step %s 129 MB L2, no flush"
                             % (host.numel() // 2**20, ">" if host.numel() > 129e6 else "<")},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                         "algorithmic_bytes_per_launch": eng_bytes,
                         "kernel": "engine_kernel_wide<int, int> (window-table DP items, one "
                                   "launch per step; %.3f ms)" % eng_ms},
            "e2e": {"value": e2e_value, "unit": "Mpix/s", "h2d_bytes_per_step": host.numel(),
                    "d2h_bytes_per_step": (hx.numel() + hd.numel() + hs.numel()) * 4},
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clocks,
        }
        if world == 1 and not args.skip_cpu:
            out["cpu_baseline"] = cpu_baseline(name, args.seed)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_learned(args):
    """Trains the proposal network on images labelled by the exact method
    (Adam, batches of 32, learning rate 3e-3, then 1e-3 and 3e-4), then on a
    held-out batch reports, for each fallback rule, the exact-optimum hit rate,
    the fallback rate and the score gap, and times the learned pipeline
    (fhtdp_detect_learned) against the plain exact DP on the same batch, both
    with CUDA events on one stream."""
    import numpy as np
    import torch

    import paper_1912_01884_gb300 as fd
    from paper_1912_01884_gb300 import learned

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    fd.load()
    h = w = 1024
    k, B = 16, 12
    N = args.images or WORKLOADS["learned1024"]["images"]
    bs, train_steps = 32, 1500
    model = learned.LaneProposer(seed=args.seed, lr=3e-3)
    t0 = time.perf_counter()
    losses = []
    for step in range(train_steps):
        if step == int(train_steps * 0.6):
            model.lr = 1e-3
        if step == int(train_steps * 0.85):
            model.lr = 3e-4
        imgs = learned.lane_images(10 * args.seed + 1000 + step, bs, h, w, k, B)
        _, d, _ = learned.exact_paths(imgs, k, B)
        labels = torch.from_numpy(learned.bins_of(d.cpu().numpy()).astype(np.int32)).cuda()
        loss = model.train_step(imgs, labels, k)
        if step < 5 or step >= train_steps - 20:
            losses.append(float(loss.cpu()))
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    imgs = learned.lane_images(10**6 + 97 * args.seed, N, h, w, k, B)
    xe, de, se = learned.exact_paths(imgs, k, B)
    win = model.windows(model.propose(imgs, k), h // k)
    in_windows = float(((de >= win[..., 0]) & (de <= win[..., 1])).all(1).float().mean())
    # the confidence threshold, calibrated on other images to a 99.5 % hit rate
    conf, cal_hit, cal_fb = learned.calibrate_min_conf(
        model, learned.lane_images(2 * 10**6 + 97 * args.seed, N, h, w, k, B), k, B)
    plan = learned.LearnedPlan(imgs, k, B)
    rules = {}
    for name, margin, min_conf in (("margin0_conf0", 0.0, 0.0), ("margin0_conf0.5", 0.0, 0.5),
                                   ("margin0_conf0.8", 0.0, 0.8), ("margin100_conf0", 100.0, 0.0),
                                   ("calibrated", 0.0, conf)):
        plan.run(model, margin, min_conf)
        plan.status()
        hit = (plan.score == se) & (plan.x == xe).all(1) & (plan.d == de).all(1)
        gap = (se - plan.score).double() / se.double()
        rules[name] = {
            "exact_optimum_hit_rate": float(hit.float().mean()),
            "fallback_rate": float(plan.used_fallback.float().mean()),
            "score_gap_mean": float(gap.mean()), "score_gap_max": float(gap.max())}
    rules["calibrated"].update({"min_conf": conf, "calibration_hit_rate": cal_hit,
                                "calibration_fallback_rate": cal_fb,
                                "calibration": "%d other images, target hit rate 0.995" % N})

    stream = torch.cuda.Stream()
    plain = fd.BatchPlan([imgs[i] for i in range(N)], [k] * N, [B] * N, stream=stream)
    plain.autotune(reps=2, stream=stream)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    pix = N * h * w
    plain_ms = timed(lambda: plain.run(stream=stream))
    learned_ms = {m: timed(lambda m=m: plan.run(model, m[0], m[1], stream=stream))
                  for m in ((0.0, 0.0), (100.0, 0.0), (0.0, conf))}
    cnn_ms = timed(lambda: model.forward(imgs, k))
    value = pix / learned_ms[(0.0, conf)] / 1e3
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": learned_ms[(0.0, conf)], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32 DP, bf16 CNN",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["learned1024"]["desc"], "images_per_step": N},
            "learned": {"plain_dp_mpix_s": pix / plain_ms / 1e3,
                        "learned_mpix_s_calibrated": value,
                        "learned_mpix_s_margin0": pix / learned_ms[(0.0, 0.0)] / 1e3,
                        "learned_mpix_s_margin100": pix / learned_ms[(100.0, 0.0)] / 1e3,
                        "cnn_forward_ms": cnn_ms, "plain_dp_ms": plain_ms,
                        "speedup_vs_plain": plain_ms / learned_ms[(0.0, conf)],
                        "windows_contain_optimum": in_windows, "rules": rules,
                        "train_images": train_steps * bs, "train_seconds": train_s,
                        "loss_first": losses[0], "loss_last": float(np.mean(losses[-10:])),
                        "timing": "CUDA events over --steps back-to-back launches on one "
                                  "stream; learned = CNN + windows + pruned DP + device "
                                  "fallback decision + fallback DP"},
        }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("angle2048", "through2048", "two2048", "padded2048"):
        run_standalone(args)
    elif args.workload == "angle2048batch":
        run_angle_batch(args)
    elif args.workload == "learned1024":
        run_learned(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
