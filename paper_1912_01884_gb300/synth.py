"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's images (its Fig. 6 link and the document dataset behind Fig. 3)
are not available, so every workload is synthetic: a noisy background with
bright polylines drawn over it, as in Sec. 3's synthetic examples.  This
module only draws random numbers and rasterises straight segments by
rounding; it holds none of the method's arithmetic (no Hough transform, no
dyadic line pattern, no DP), so the CUDA path and the CPU oracle can both be
fed from it without sharing any of the method's code.

Random numbers come from a counter-based SplitMix64 (Steele, Lea, Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): value i of
stream (seed, stream) is mix64(key + (i+1) * golden), so results are the same
on every machine and numpy version.  Normal deviates use Box-Muller.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based SplitMix64 stream; draws advance an internal counter."""

    def __init__(self, seed: int, stream: int = 0):
        key = np.array([(seed * 0x100000001B3 + stream * 0xC2B2AE3D27D4EB4F) & (2**64 - 1)],
                       dtype=np.uint64)
        self._key = _mix64(key)[0]
        self._ctr = 0

    def bits(self, count: int) -> np.ndarray:
        idx = np.arange(self._ctr + 1, self._ctr + 1 + count, dtype=np.uint64)
        self._ctr += count
        with np.errstate(over="ignore"):
            return _mix64(self._key + idx * _GOLDEN)

    def ints(self, count: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (int64)."""
        span = np.uint64(hi - lo + 1)
        r = (self.bits(count) >> np.uint64(32)) * span >> np.uint64(32)
        return r.astype(np.int64) + lo

    def int1(self, lo: int, hi: int) -> int:
        return int(self.ints(1, lo, hi)[0])

    def uniform(self, count: int) -> np.ndarray:
        """Uniform doubles in (0, 1)."""
        return ((self.bits(count) >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)

    def normal(self, count: int) -> np.ndarray:
        half = (count + 1) // 2
        u1 = self.uniform(half)
        u2 = self.uniform(half)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)])
        return z[:count]


@dataclass
class Workload:
    """One synthetic image and the parameters it is solved with."""
    img: np.ndarray            # h x w, uint8 / int32 / float32
    k: int                     # number of bands
    B: int                     # bend range |d_{i+1} - d_i| <= B
    planted: list = field(default_factory=list)   # [(x[k+1], d[k])] drawn polylines

    @property
    def h(self) -> int:
        return self.img.shape[0]

    @property
    def w(self) -> int:
        return self.img.shape[1]


def random_polyline(rng: Rng, h: int, w: int, k: int, bend: int, tries: int = 200):
    """x[k+1], d[k] of a k-link polyline whose vertices stay in [0, w), with
    |d_i| <= n-1 and |d_{i+1} - d_i| <= bend."""
    n = h // k
    dmax = n - 1
    for _ in range(tries):
        x0 = rng.int1(0, w - 1)
        d = [rng.int1(-dmax, dmax)]
        for _i in range(1, k):
            d.append(int(np.clip(d[-1] + rng.int1(-bend, bend), -dmax, dmax)))
        xs = np.concatenate([[x0], x0 + np.cumsum(d)])
        if xs.min() >= 0 and xs.max() < w:
            return xs.astype(np.int32), np.asarray(d, dtype=np.int32)
    x0 = rng.int1(0, w - 1)
    return np.full(k + 1, x0, dtype=np.int32), np.zeros(k, dtype=np.int32)


def raster_columns(x0: int, d: int, n: int) -> np.ndarray:
    """Columns of a straight segment over n rows from x0 to x0 + d, each row's
    column rounded to the nearest integer (halves round up)."""
    y = np.arange(n, dtype=np.int64)
    if n == 1:
        return np.array([x0], dtype=np.int64)
    return x0 + (2 * d * y + (n - 1)) // (2 * (n - 1))


def _draw(img, xs, ds, n, value, keep=None):
    for i, d in enumerate(ds):
        rows = np.arange(i * n, (i + 1) * n)
        cols = raster_columns(int(xs[i]), int(d), n)
        if keep is not None:
            m = keep[i * n:(i + 1) * n]
            rows, cols = rows[m], cols[m]
        img[rows, cols] = value


def plain_uniform(seed: int, h: int, w: int, k: int, B: int, lines: int = 1,
                  noise_hi: int = 40, value: int = 200) -> Workload:
    """Background i.i.d. uniform integers in [0, noise_hi] plus `lines`
    polylines of intensity `value` whose bends stay within B (the 256x256
    single-image workload and the mixed-size batch use this model)."""
    rng = Rng(seed, 1)
    img = rng.ints(h * w, 0, noise_hi).astype(np.uint8).reshape(h, w)
    planted = []
    for _ in range(lines):
        xs, ds = random_polyline(rng, h, w, k, B)
        _draw(img, xs, ds, h // k, value)
        planted.append((xs, ds))
    return Workload(img, k, B, planted)


def plain_gaussian(seed: int, h: int = 2048, w: int = 2048, k: int = 16, B: int = 16,
                   lines: int = 3, dropout: float = 0.3) -> Workload:
    """Gaussian background (mean 30, sd 12, rounded and clipped to [0, 255])
    plus `lines` polylines of intensity uniform in {90..160}; each polyline
    pixel is dropped with probability `dropout` (it keeps the background)."""
    rng = Rng(seed, 2)
    bg = np.clip(np.rint(30.0 + 12.0 * rng.normal(h * w)), 0, 255)
    img = bg.astype(np.uint8).reshape(h, w)
    planted = []
    for _ in range(lines):
        xs, ds = random_polyline(rng, h, w, k, B)
        value = rng.int1(90, 160)
        keep = rng.uniform(h) >= dropout
        _draw(img, xs, ds, h // k, value, keep)
        planted.append((xs, ds))
    return Workload(img, k, B, planted)


def lane_texture(seed: int, h: int = 1024, w: int = 1024, k: int = 16, B: int = 12,
                 lines: int = 2) -> Workload:
    """Textured background (uniform [0, 40] plus a smooth sinusoidal field of
    amplitude 20 with random phase) and `lines` lane-like polylines whose
    displacement follows a slowly varying curve (|d_{i+1} - d_i| <= B),
    intensity uniform in {70..140}."""
    rng = Rng(seed, 4)
    n = h // k
    noise = rng.ints(h * w, 0, 40).reshape(h, w).astype(np.float64)
    ph = rng.uniform(2) * 2.0 * math.pi
    yy, xx = np.mgrid[0:h, 0:w]
    field_ = 20.0 * (0.5 + 0.5 * np.sin(2 * math.pi * xx / 173.0 + ph[0])
                     * np.cos(2 * math.pi * yy / 211.0 + ph[1]))
    img = np.clip(np.rint(noise + field_), 0, 255).astype(np.uint8)
    planted = []
    for _ in range(lines):
        for _t in range(100):
            x0 = rng.int1(w // 8, 7 * w // 8)
            a = rng.uniform(3)
            base = (a[0] - 0.5) * (n - 1)
            amp = a[1] * min(B, n - 1) * 2.0
            ph2 = a[2] * 2 * math.pi
            d = []
            for i in range(k):
                v = int(round(base + amp * math.sin(ph2 + 2 * math.pi * i / (2.5 * k))))
                v = max(-(n - 1), min(n - 1, v))
                if d:
                    v = max(d[-1] - B, min(d[-1] + B, v))
                d.append(v)
            xs = np.concatenate([[x0], x0 + np.cumsum(d)])
            if xs.min() >= 0 and xs.max() < w:
                break
        else:
            xs, d = np.full(k + 1, x0), [0] * k
        value = rng.int1(70, 140)
        _draw(img, np.asarray(xs), d, n, value)
        planted.append((np.asarray(xs, dtype=np.int32), np.asarray(d, dtype=np.int32)))
    return Workload(img, k, B, planted)


def ridge_response(seed: int, h: int = 8192, w: int = 8192, k: int = 64, B: int = 24,
                   lines: int = 4, value: float = 3.0, width: float = 1.5) -> Workload:
    """Float32 ridge-response map: |N(0, 1)| background plus `lines` polylines
    that each add value * exp(-dx^2 / (2 width^2)) around the segment's exact
    column on every row."""
    rng = Rng(seed, 5)
    img = np.abs(rng.normal(h * w)).astype(np.float32).reshape(h, w)
    n = h // k
    planted = []
    reach = int(math.ceil(4 * width))
    offs = np.arange(-reach, reach + 1)
    for _ in range(lines):
        xs, ds = random_polyline(rng, h, w, k, B)
        for i, d in enumerate(ds):
            y = np.arange(n)
            centre = xs[i] + (d * y / (n - 1) if n > 1 else 0.0)
            cols = np.rint(centre)[:, None].astype(np.int64) + offs[None, :]
            wgt = value * np.exp(-((cols - centre[:, None]) ** 2) / (2 * width * width))
            ok = (cols >= 0) & (cols < w)
            rows = np.broadcast_to((i * n + y)[:, None], cols.shape)
            np.add.at(img, (rows[ok], cols[ok]), wgt[ok].astype(np.float32))
        planted.append((xs, ds))
    return Workload(img, k, B, planted)


def mixed_batch_shapes(seed: int, count: int = 256):
    """(h, w, k, B) of the mixed-size batch: h uniform in {512..4096} step 256,
    w uniform in {512..3072} step 256, n = h/k uniform in {32, 64, 128, 256},
    B = n/8."""
    rng = Rng(seed, 3)
    hs = 256 * rng.ints(count, 2, 16)
    ws = 256 * rng.ints(count, 2, 12)
    ns = 2 ** rng.ints(count, 5, 8)
    return [(int(h), int(w), int(h // n), int(n // 8)) for h, w, n in zip(hs, ws, ns)]


def mixed_batch(seed: int, count: int = 256, shapes=None):
    """Workloads of the mixed-size batch (uniform-noise model, one polyline)."""
    shapes = shapes or mixed_batch_shapes(seed, count)
    return [plain_uniform(seed * 100003 + j, h, w, k, B) for j, (h, w, k, B) in enumerate(shapes)]


def bent_edges(seed: int, h: int = 2048, w: int = 2048, k: int = 16, lines: int = 2,
               max_slope: float = 0.6, value: int = 70, salt: float = 0.004) -> Workload:
    """A bent-document-boundary image (Sec. 3, Fig. 3) for the main problem:
    Gaussian background (mean 30, sd 12, clipped to [0, 255]), `lines` smooth
    mostly-vertical curves x(y) = x0 + a y + b sin(2 pi y / period + phase)
    with |dx/dy| <= max_slope, each a 3-pixel ridge adding `value`, 0.6 *
    `value` and 0.2 * `value` at column offsets 0, +-1, +-2, and spiky noise:
    a fraction `salt` of all pixels set to 255 (the outliers the Welsh
    estimate is robust to).  `B` is -1: the image is solved with a bend angle,
    not an integer bend limit; `planted` holds the curves' columns per row."""
    rng = Rng(seed, 6)
    bg = np.clip(np.rint(30.0 + 12.0 * rng.normal(h * w)), 0, 255)
    img = bg.astype(np.int64).reshape(h, w)
    y = np.arange(h, dtype=np.float64)
    planted = []
    for _ in range(lines):
        period = h * (0.5 + rng.uniform(1)[0])
        b = (0.25 + 0.5 * rng.uniform(1)[0]) * max_slope * period / (2 * math.pi)
        a = (rng.uniform(1)[0] * 2 - 1) * 0.25 * max_slope
        phase = 2 * math.pi * rng.uniform(1)[0]
        x = a * y + b * np.sin(2 * math.pi * y / period + phase)
        x0 = w * (0.2 + 0.6 * rng.uniform(1)[0]) - 0.5 * (x.max() + x.min())
        cols = np.rint(x0 + x).astype(np.int64)
        for off, frac in ((0, 1.0), (-1, 0.6), (1, 0.6), (-2, 0.2), (2, 0.2)):
            c = cols + off
            ok = (c >= 0) & (c < w)
            img[np.arange(h)[ok], c[ok]] += int(round(value * frac))
        planted.append(cols)
    spikes = rng.uniform(h * w) < salt
    img = np.clip(img, 0, 255).reshape(-1)
    img[spikes] = 255
    return Workload(img.reshape(h, w).astype(np.uint8), k, -1, planted)


# The five workloads of the benchmark suite, by name.
WORKLOADS = {
    "u8_256x256_k4_B8": lambda seed: plain_uniform(seed, 256, 256, 4, 8),
    "u8_2048x2048_k16_B16": lambda seed: plain_gaussian(seed),
    "u8_1024x1024_k16_B12_lanes": lambda seed: lane_texture(seed),
    "f32_8192x8192_k64_B24": lambda seed: ridge_response(seed),
}
