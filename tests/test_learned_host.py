"""Host logic of the learned proposal that needs no GPU: the label bins, the
training images' recipe (generated on the CPU), and the calibration of
the fallback rule's confidence threshold, run against a fake plan whose hit
rate rises with the threshold as the device rule's does (each image falls
back, and is then exact, once the threshold exceeds its lowest band
confidence)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1912_01884_gb300 import learned  # noqa: E402


class _FakePlan:
    """Images with a lowest band confidence `conf[i]`; image i is pruned-exact
    when `exact[i]`, and it falls back (exact) when conf[i] < min_conf."""

    def __init__(self, conf, exact, xe, de, se):
        self.conf, self.exact = conf, exact
        self.xe, self.de, self.se = xe, de, se
        self.runs = []

    def run(self, model, margin, min_conf, stream=None):
        self.runs.append(min_conf)
        fb = self.conf < min_conf
        ok = fb | self.exact
        self.used_fallback = torch.from_numpy(fb.astype(np.int32))
        self.score = torch.where(torch.from_numpy(ok), self.se, self.se - 1)
        self.x, self.d = self.xe.clone(), self.de.clone()

    def status(self, stream=None):
        return 0

    def close(self):
        pass


def _install(monkeypatch, conf, exact):
    n = len(conf)
    xe = torch.zeros(n, 5, dtype=torch.int32)
    de = torch.zeros(n, 4, dtype=torch.int32)
    se = torch.full((n,), 100, dtype=torch.int32)
    plan = _FakePlan(np.asarray(conf), np.asarray(exact), xe, de, se)
    monkeypatch.setattr(learned, "exact_paths", lambda imgs, k, B: (xe, de, se))
    monkeypatch.setattr(learned, "LearnedPlan", lambda imgs, k, B: plan)
    return plan


def test_calibration_takes_the_smallest_threshold_that_reaches_the_target(monkeypatch):
    # 1000 images: 10 pruned answers are wrong, with lowest confidences
    # 0.515, 0.525, ..., 0.605; 90 right ones between 0.62 and 0.70
    conf = np.concatenate([np.linspace(0.515, 0.605, 10), np.full(990, 0.9)])
    exact = np.concatenate([np.zeros(10, bool), np.ones(990, bool)])
    conf[10:100] = np.linspace(0.62, 0.70, 90)
    plan = _install(monkeypatch, conf, exact)
    # under 0.56 five wrong answers fall back (hit 0.995), under 0.58 seven
    c, hit, fb = learned.calibrate_min_conf(None, None, 4, 2, target=0.996)
    assert c == 0.58 and plan.runs == [0.5, 0.52, 0.54, 0.56, 0.58]
    assert hit == pytest.approx(0.997) and fb == pytest.approx(0.007)
    c, hit, fb = learned.calibrate_min_conf(None, None, 4, 2, target=0.99)
    assert c == 0.5 and hit == pytest.approx(0.99) and fb == 0.0


def test_calibration_returns_the_largest_threshold_when_none_reaches_the_target(monkeypatch):
    conf = np.full(200, 0.95)
    exact = np.arange(200) % 10 != 0          # 10 % wrong at every threshold
    _install(monkeypatch, conf, exact)
    c, hit, fb = learned.calibrate_min_conf(None, None, 4, 2, target=0.995)
    assert c == learned.CONF_GRID[-1] and hit == pytest.approx(0.9) and fb == 0.0


def test_label_bins_cover_the_displacements_four_at_a_time():
    d = np.arange(-63, 64)
    b = learned.bins_of(d)
    assert b.min() == 0 and b.max() == learned.BINS - 1
    assert np.all(np.diff(b) >= 0)
    assert np.all(4 * b <= d + 64) and np.all(d + 64 <= 4 * b + 3)


def test_lane_images_follow_their_recipe_on_the_host():
    """The training images (generated on the CPU here): seeded, uint8, noise
    and field at most 60, and two lanes of intensity 70..140 whose pixels
    move at most one column from row to row."""
    args = dict(h=64, w=128, k=4, B=3, device="cpu")
    a = learned.lane_images(7, 3, **args)
    assert a.dtype == torch.uint8 and tuple(a.shape) == (3, 64, 128)
    assert torch.equal(a, learned.lane_images(7, 3, **args))
    assert not torch.equal(a, learned.lane_images(8, 3, **args))
    img = a.numpy().astype(int)
    bright = img >= 70
    assert np.all(img[~bright] <= 60) and np.all(img[bright] <= 140)
    counts = bright.sum(2)
    assert np.all((counts >= 1) & (counts <= 2))
    for n in range(3):
        for r in range(63):
            prev = np.flatnonzero(bright[n, r])
            for c in np.flatnonzero(bright[n, r + 1]):
                assert np.abs(prev - c).min() <= 1, (n, r, c)
