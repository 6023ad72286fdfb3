"""Host logic of the learned proposal that needs no GPU: the calibration of
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
