"""Learned window proposal in front of the exact method.

A 4-layer, 32-channel CNN (3x3 convolutions with dilations 1, 2, 4, 8, a
31-pixel receptive field on the 4x4-downsampled image, i.e. at least the 16
low-resolution rows of a band) predicts for every band one of 32 bins of 4
displacements.  The DP then searches only a 16-wide window around the
predicted bin (the pruned DP).  An image falls back to the full DP when its
pruned optimum does not exist, touches a window edge, or scores below a
confidence margin (a mean intensity per image row), or where the network's
own confidence in a band's bin is low.  The network is trained
on labels that the exact method produces.  The paper has none of this: it is
an addition in front of the method.

Every computation runs in the library's CUDA kernels (C ABI ``fhtdp_cnn_*``
and ``fhtdp_detect_learned``: tensor-core bf16 convolutions with FP32
accumulation, the band head, Adam on FP32 master weights, the pruned DP and
the fallback decision on the device).  PyTorch provides device memory and the
training images' random numbers.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import BatchPlan, _check, _stream, lib

C = 32                      # channels
DILATIONS = (1, 2, 4, 8)
BINS = 32                   # displacement bins of 4 (d + 64 in [4c, 4c + 3])
MARGIN = 6                  # window = the bin's 4 displacements +- 6


def _torch():
    import torch
    return torch


def bins_of(d):
    """Label bin of displacements d in [-63, 63]."""
    return (np.asarray(d) + 64) >> 2


def lane_images(seed: int, count: int, h: int = 1024, w: int = 1024, k: int = 16, B: int = 12,
                device="cuda"):
    """Training / evaluation images on the GPU, uint8 [count, h, w]: uniform
    noise 0..40 plus a smooth sinusoidal field of amplitude 20, and 2
    lane-like polylines of intensity 70..140 whose displacement follows a
    slowly varying curve with |d_{i+1} - d_i| <= B.  Drawn with torch's
    seeded generator (the same recipe as synth.lane_texture, generated on
    the device because training needs tens of thousands of images)."""
    torch = _torch()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    n = h // k
    img = torch.randint(0, 41, (count, h, w), generator=g, device=device).float()
    ph = torch.rand(count, 2, generator=g, device=device) * (2 * math.pi)
    xx = torch.arange(w, device=device, dtype=torch.float32)
    yy = torch.arange(h, device=device, dtype=torch.float32)
    fx = torch.sin(2 * math.pi * xx[None, :] / 173.0 + ph[:, :1])          # [N, w]
    fy = torch.cos(2 * math.pi * yy[None, :] / 211.0 + ph[:, 1:2])         # [N, h]
    img += 20.0 * (0.5 + 0.5 * fy[:, :, None] * fx[:, None, :])
    img = img.round().clamp(0, 255)
    rows = torch.arange(h, device=device)
    band = rows // n
    yb = (rows % n).float()
    for _line in range(2):
        a = torch.rand(count, 3, generator=g, device=device)
        base = (a[:, 0] - 0.5) * (n - 1)
        amp = a[:, 1] * min(B, n - 1) * 2.0
        ph2 = a[:, 2] * 2 * math.pi
        i = torch.arange(k, device=device, dtype=torch.float32)
        d = torch.round(base[:, None] + amp[:, None] * torch.sin(ph2[:, None]
                                                                 + 2 * math.pi * i / (2.5 * k)))
        d = d.clamp(-(n - 1), n - 1)
        for j in range(1, k):   # keep the bends within B
            d[:, j] = torch.maximum(torch.minimum(d[:, j], d[:, j - 1] + B), d[:, j - 1] - B)
        d = d.long()
        offs = torch.cat([torch.zeros(count, 1, dtype=torch.long, device=device),
                          torch.cumsum(d, 1)], 1)                         # [N, k+1]
        lo = -offs.min(1).values
        hi = (w - 1) - offs.max(1).values
        x0 = torch.randint(0, 1 << 30, (count,), generator=g, device=device)
        x0 = lo + x0 % (hi - lo + 1)
        xs = x0[:, None] + offs                                            # [N, k+1]
        val = torch.randint(70, 141, (count,), generator=g, device=device).float()
        # column of every row: x_i + round(d_i * y / (n-1)), halves up
        di = d[:, band]                                                     # [N, h]
        if n > 1:
            cols = xs[:, band] + torch.div(2 * di * yb.long() + (n - 1), 2 * (n - 1),
                                           rounding_mode="floor")
        else:
            cols = xs[:, band]
        img.scatter_(2, cols[:, :, None], val[:, None, None].expand(count, h, 1))
    return img.to(torch.uint8)


class LaneProposer:
    """The CNN's parameter block (FP32 master weights, Adam moments, bf16
    copies; C ABI fhtdp_cnn_*) and a training workspace for batches of
    `batch` images of h x w."""

    def __init__(self, seed: int = 0, device="cuda", lr: float = 3e-3):
        torch = _torch()
        self.device = device
        self.lr = lr
        self.step_count = 0
        self.params = torch.empty(lib().fhtdp_cnn_param_bytes(), dtype=torch.uint8, device=device)
        _check(lib().fhtdp_cnn_init(self.params.data_ptr(), int(seed), _stream(None)))
        self._ws = None
        self._ws_key = None

    def _workspace(self, n, h, w):
        torch = _torch()
        if self._ws_key != (n, h, w):
            self._ws = torch.empty(lib().fhtdp_cnn_workspace_bytes(n, h, w), dtype=torch.uint8,
                                   device=self.device)
            self._ws_key = (n, h, w)
        return self._ws

    def forward(self, imgs, bands):
        """(pred [N, bands] bins, conf [N, bands] softmax probabilities)."""
        torch = _torch()
        N, h, w = imgs.shape
        ws = self._workspace(N, h, w)
        pred = torch.empty(N, bands, dtype=torch.int32, device=self.device)
        conf = torch.empty(N, bands, dtype=torch.float32, device=self.device)
        _check(lib().fhtdp_cnn_forward(self.params.data_ptr(), imgs.data_ptr(), N, h, w, bands,
                                       ws.data_ptr(), ws.numel(), pred.data_ptr(),
                                       conf.data_ptr(), _stream(None)))
        return pred, conf

    def train_step(self, imgs, labels, bands):
        """One Adam step on a batch: imgs uint8 [N, H, W] (device), labels int32
        [N, bands] (bins).  Returns the loss (a device tensor)."""
        torch = _torch()
        N, h, w = imgs.shape
        self.forward(imgs, bands)
        ws = self._workspace(N, h, w)
        loss = torch.zeros(1, device=self.device)
        _check(lib().fhtdp_cnn_backward(self.params.data_ptr(), labels.data_ptr(), N, h, w, bands,
                                        ws.data_ptr(), ws.numel(), loss.data_ptr(),
                                        _stream(None)))
        self.step_count += 1
        _check(lib().fhtdp_cnn_step(self.params.data_ptr(), ws.data_ptr(), N, h, w,
                                    float(self.lr), self.step_count, _stream(None)))
        return loss

    def propose(self, imgs, bands):
        """Predicted bins [N, bands] (int32, device)."""
        return self.forward(imgs, bands)[0]

    def windows(self, pred, n):
        torch = _torch()
        win = torch.empty(pred.numel(), 2, dtype=torch.int32, device=self.device)
        _check(lib().fhtdp_cnn_bin_windows(pred.data_ptr(), pred.numel(), n, MARGIN,
                                           win.data_ptr(), _stream(None)))
        return win.view(*pred.shape, 2)


class LearnedPlan:
    """fhtdp_learned_plan over a batch of images [N, h, w] (one contiguous
    device tensor): proposal, pruned DP, device-side fallback to the full DP."""

    def __init__(self, imgs, k: int, B: int, window_half: int = MARGIN, stream=None):
        from . import Image
        torch = _torch()
        N, h, w = imgs.shape
        self.imgs, self.k, self.N = imgs, k, N
        dev = imgs.device
        self.x = torch.empty(N, k + 1, dtype=torch.int32, device=dev)
        self.d = torch.empty(N, k, dtype=torch.int32, device=dev)
        self.score = torch.empty(N, dtype=torch.int32, device=dev)
        self.used_fallback = torch.empty(N, dtype=torch.int32, device=dev)
        arr = (Image * N)()
        for i in range(N):
            arr[i] = Image(imgs[i].data_ptr(), h, w, w, k, B, self.x[i].data_ptr(),
                           self.d[i].data_ptr(), self.score[i:i + 1].data_ptr(), None)
        self._arr = arr
        handle = ctypes.c_void_p()
        _check(lib().fhtdp_learned_plan_create(ctypes.cast(arr, ctypes.c_void_p), N,
                                               int(window_half), ctypes.byref(handle)))
        self._plan = handle
        self.ws = torch.empty(lib().fhtdp_learned_workspace_bytes(handle), dtype=torch.uint8,
                              device=dev)
        _check(lib().fhtdp_learned_upload(handle, self.ws.data_ptr(), self.ws.numel(),
                                          _stream(stream)))

    def run(self, model, margin: float, min_conf: float = 0.0, stream=None):
        """Enqueues the detection; results in self.x, self.d, self.score and
        self.used_fallback."""
        _check(lib().fhtdp_detect_learned(self._plan, model.params.data_ptr(), float(margin),
                                          float(min_conf), self.used_fallback.data_ptr(),
                                          self.ws.data_ptr(), _stream(stream)))

    def status(self, stream=None):
        _check(lib().fhtdp_learned_status(self._plan, self.ws.data_ptr(), _stream(stream)))
        return 0

    def close(self):
        if self._plan:
            lib().fhtdp_learned_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exact_paths(imgs, k, B):
    """Exact DP of every image: (x [N, k+1], d [N, k], score [N]) device."""
    plan = BatchPlan([imgs[i] for i in range(imgs.shape[0])], [k] * imgs.shape[0],
                     [B] * imgs.shape[0])
    plan.run()
    plan.status()
    torch = _torch()
    return (torch.stack(plan.x), torch.stack(plan.d), torch.cat(plan.score))


CONF_GRID = tuple(round(0.5 + 0.02 * i, 2) for i in range(16)) + (0.85, 0.9)


def calibrate_min_conf(model, imgs, k, B, target: float = 0.995, margin: float = 0.0,
                       grid=CONF_GRID):
    """Calibrates the band-confidence threshold of the fallback rule on images
    held apart from those it is later used on: the smallest threshold of
    `grid` under which the learned detection returns the exact optimum for at
    least `target` of `imgs` (the largest one when none does).  Raising the
    threshold only adds fallbacks, so the hit rate does not fall along the
    grid.  Returns (min_conf, hit rate, fallback rate) on `imgs`."""
    xe, de, se = exact_paths(imgs, k, B)
    plan = LearnedPlan(imgs, k, B)
    try:
        for c in grid:
            plan.run(model, margin, c)
            plan.status()
            hit = float(((plan.score == se) & (plan.x == xe).all(1) &
                         (plan.d == de).all(1)).float().mean())
            fb = float(plan.used_fallback.float().mean())
            if hit >= target:
                break
        return c, hit, fb
    finally:
        plan.close()


def detect_learned(model, imgs, k, B, margin: float = 0.0, min_conf: float = 0.0):
    """Learned proposal + pruned DP + device-side fallback (fhtdp_detect_learned).
    Returns (x, d, score, used_fallback[N]); images that fall back carry the
    exact method's outputs."""
    plan = LearnedPlan(imgs, k, B)
    plan.run(model, margin, min_conf)
    plan.status()
    return plan.x, plan.d, plan.score, plan.used_fallback.bool()
