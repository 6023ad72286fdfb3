"""Learned window proposal in front of the exact method.

A 4-layer, 32-channel CNN (3x3 convolutions with dilations 1, 2, 4, 8, a
31-pixel receptive field on the 4x4-downsampled image, i.e. at least the 16
low-resolution rows of a band) predicts for every band one of 32 bins of 4
displacements.  The DP then searches only a 16-wide window around the
predicted bin (the pruned DP: ``BatchPlan(..., windows=...)``).  An image
falls back to the full DP when its pruned optimum does not exist or touches a
window edge.  The network is trained on labels that the exact method
produces.  The paper has none of this: it is an addition in front of the
method.

Every computation runs in the library's CUDA kernels (C ABI ``fhtdp_cnn_*``:
tensor-core bf16 convolutions with FP32 accumulation, the band head, Adam on
FP32 master weights).  PyTorch provides device memory, the random
initialisation and the training images' random numbers.
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
    """The CNN, its FP32 master weights, bf16 copies and Adam state."""

    def __init__(self, seed: int = 0, device="cuda", lr: float = 3e-3):
        torch = _torch()
        self.device = device
        self.lr = lr
        self.step_count = 0
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        self.params = []   # (weight fp32, bias fp32, bf16 copy, cin, dilation)
        for layer, dil in enumerate(DILATIONS):
            cin = 1 if layer == 0 else C
            taps = 16 if cin == 1 else 9 * cin
            fan_in = 9 * cin
            wt = torch.randn(taps, C, generator=g, device=device) * math.sqrt(2.0 / fan_in)
            if cin == 1:
                wt[9:] = 0.0
            b = torch.zeros(C, device=device)
            self.params.append([wt.contiguous(), b, torch.empty(taps, C, dtype=torch.bfloat16,
                                                                 device=device), cin, dil])
        self.moments = [[torch.zeros_like(p[0]), torch.zeros_like(p[0]), torch.zeros_like(p[1]),
                         torch.zeros_like(p[1])] for p in self.params]
        self.wflip = torch.empty(9 * C * C, dtype=torch.bfloat16, device=device)
        for p in self.params:
            _check(lib().fhtdp_cnn_to_bf16(p[0].data_ptr(), p[2].data_ptr(), p[0].numel(),
                                           _stream(None)))

    # -- forward --------------------------------------------------------------
    def downsample(self, imgs):
        torch = _torch()
        N, H, W = imgs.shape
        x = torch.empty(N, H // 4, W // 4, 1, dtype=torch.bfloat16, device=self.device)
        _check(lib().fhtdp_cnn_downsample4(imgs.data_ptr(), N, H, W, x.data_ptr(),
                                           _stream(None)))
        return x

    def forward(self, x):
        """Activations [x, a1, a2, a3, logits] (NHWC bf16)."""
        torch = _torch()
        N, H, W, _ = x.shape
        acts = [x]
        for layer, (wt, b, wb, cin, dil) in enumerate(self.params):
            y = torch.empty(N, H, W, C, dtype=torch.bfloat16, device=self.device)
            relu = 1 if layer < len(self.params) - 1 else 0
            _check(lib().fhtdp_cnn_conv3x3(acts[-1].data_ptr(), cin, N, H, W, dil, wb.data_ptr(),
                                           b.data_ptr(), relu, y.data_ptr(), _stream(None)))
            acts.append(y)
        return acts

    def head(self, logits, bands, labels=None, want_grad=False):
        """(loss, dlogits, pred) of the band head."""
        torch = _torch()
        N, H, W, _ = logits.shape
        loss = torch.zeros(1, device=self.device)
        pred = torch.empty(N, bands, dtype=torch.int32, device=self.device)
        dl = torch.empty_like(logits) if want_grad else None
        _check(lib().fhtdp_cnn_band_head(
            logits.data_ptr(), N, H, W, bands,
            labels.data_ptr() if labels is not None else None, 1.0 / (N * bands),
            dl.data_ptr() if dl is not None else None, loss.data_ptr(), pred.data_ptr(),
            _stream(None)))
        return loss, dl, pred

    # -- backward -------------------------------------------------------------
    def backward(self, acts, dlogits):
        """FP32 gradients [(dW, db)] of every layer."""
        torch = _torch()
        N, H, W, _ = acts[0].shape
        grads = [None] * len(self.params)
        dz = dlogits
        for layer in range(len(self.params) - 1, -1, -1):
            wt, b, wb, cin, dil = self.params[layer]
            dw = torch.zeros_like(wt)
            db = torch.zeros_like(b)
            _check(lib().fhtdp_cnn_conv3x3_wgrad(acts[layer].data_ptr(), cin, N, H, W, dil,
                                                 dz.data_ptr(), dw.data_ptr(), db.data_ptr(),
                                                 _stream(None)))
            grads[layer] = (dw, db)
            if layer == 0:
                break
            dx = torch.empty_like(acts[layer])
            _check(lib().fhtdp_cnn_conv3x3_dgrad(dz.data_ptr(), N, H, W, dil, wb.data_ptr(),
                                                 self.wflip.data_ptr(), dx.data_ptr(),
                                                 _stream(None)))
            _check(lib().fhtdp_cnn_relu_backward(acts[layer].data_ptr(), dx.data_ptr(),
                                                 dx.numel(), _stream(None)))
            dz = dx
        return grads

    def apply(self, grads):
        self.step_count += 1
        for (wt, b, wb, _, _), (m_w, v_w, m_b, v_b), (dw, db) in zip(self.params, self.moments,
                                                                   grads):
            _check(lib().fhtdp_cnn_adam(wt.data_ptr(), m_w.data_ptr(), v_w.data_ptr(),
                                        dw.data_ptr(), wt.numel(), self.lr, 0.9, 0.999, 1e-8,
                                        self.step_count, wb.data_ptr(), _stream(None)))
            _check(lib().fhtdp_cnn_adam(b.data_ptr(), m_b.data_ptr(), v_b.data_ptr(),
                                        db.data_ptr(), b.numel(), self.lr, 0.9, 0.999, 1e-8,
                                        self.step_count, None, _stream(None)))
        # The first layer's padding taps (9..15) have zero gradients, so Adam
        # leaves them at zero.

    def train_step(self, imgs, labels, bands):
        """One Adam step on a batch: imgs uint8 [N, H, W] (device), labels int32
        [N, bands] (bins).  Returns the loss (a device tensor)."""
        acts = self.forward(self.downsample(imgs))
        loss, dl, _ = self.head(acts[-1], bands, labels, want_grad=True)
        self.apply(self.backward(acts, dl))
        return loss

    def propose(self, imgs, bands):
        """Predicted bins [N, bands] (int32, device)."""
        acts = self.forward(self.downsample(imgs))
        return self.head(acts[-1], bands)[2]

    def windows(self, pred, n):
        torch = _torch()
        win = torch.empty(pred.numel(), 2, dtype=torch.int32, device=self.device)
        _check(lib().fhtdp_cnn_bin_windows(pred.data_ptr(), pred.numel(), n, MARGIN,
                                           win.data_ptr(), _stream(None)))
        return win.view(*pred.shape, 2)


def exact_paths(imgs, k, B):
    """Exact DP of every image: (x [N, k+1], d [N, k], score [N]) device."""
    plan = BatchPlan([imgs[i] for i in range(imgs.shape[0])], [k] * imgs.shape[0],
                     [B] * imgs.shape[0])
    plan.run()
    plan.status()
    torch = _torch()
    return (torch.stack(plan.x), torch.stack(plan.d), torch.cat(plan.score))


def detect_learned(model, imgs, k, B):
    """Learned proposal + pruned DP + fallback.  Returns (x, d, score,
    used_fallback[N]) with the exact method's outputs for fallback images."""
    torch = _torch()
    N, h, w = imgs.shape
    n = h // k
    pred = model.propose(imgs, k)
    win = model.windows(pred, n)
    plan = BatchPlan([imgs[i] for i in range(N)], [k] * N, [B] * N,
                     windows=[win[i] for i in range(N)])
    plan.run()
    plan.status()
    x = torch.stack(plan.x)
    d = torch.stack(plan.d)
    s = torch.cat(plan.score)
    # Fallback: no polyline inside the windows, or one touching a window edge
    # that is not the edge of the displacement range.
    wl, wh = win[..., 0], win[..., 1]
    edge = ((d == wl) & (wl > -(n - 1))) | ((d == wh) & (wh < n - 1))
    fb = (x[:, 0] < 0) | edge.any(1)
    idx = torch.nonzero(fb).flatten().cpu().numpy().tolist()
    if idx:
        fplan = BatchPlan([imgs[i] for i in idx], [k] * len(idx), [B] * len(idx))
        fplan.run()
        fplan.status()
        for j, i in enumerate(idx):
            x[i] = fplan.x[j]
            d[i] = fplan.d[j]
            s[i] = fplan.score[j][0]
    return x, d, s, fb
