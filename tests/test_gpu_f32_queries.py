"""GPU parity of the queries of Secs. 2.2-2.3 and 3 on float32 images
(smoothing + bend angle, through-point with and without the angle, padded
vertices, two polylines), through the C ABI, against the oracle's float32
restatements: the chosen polylines bit-exact, scores within the relative
tolerance 1e-5 of float response maps."""
import math

import numpy as np
import pytest

import oracle
from helpers import to_device

pytestmark = pytest.mark.gpu

REL = 1e-5
SHAPES = [(64, 64, 4), (64, 37, 4), (128, 300, 2), (16, 5, 16), (8, 3, 4), (96, 77, 3),
          (32, 1, 2), (512, 130, 4), (16, 40, 16)]


def _img(h, w, seed):
    rng = np.random.default_rng(seed)
    return (np.abs(rng.standard_normal((h, w))) * 2.5).astype(np.float32)


def _close(s, so):
    if so == -math.inf:
        return s == -math.inf
    return abs(float(s) - so) <= REL * abs(so)


def _same(x, d, s, xo, do, so):
    x, d = x.cpu().numpy(), d.cpu().numpy()
    assert np.array_equal(x, xo) and np.array_equal(d, do)
    assert _close(s.cpu().numpy().reshape(-1)[0], so)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [0, 2])
def test_angle_f32_matches_oracle(lib, shape, r):
    h, w, k = shape
    img = _img(h, w, 11 * h + w + r)
    for gamma in (0.0, math.radians(10), 0.6, 2.0):
        x, d, s = lib.detect_polyline_angle(to_device(img), k, r, gamma)
        assert s.dtype == __import__("torch").float32
        _same(x, d, s, *oracle.detect_angle_f32(img, k, r, gamma))


def test_angle_f32_full_size_2048(lib):
    img = _img(2048, 2048, 5)
    x, d, s = lib.detect_polyline_angle(to_device(img), 16, 2, math.radians(10))
    _same(x, d, s, *oracle.detect_angle_f32(img, 16, 2, math.radians(10)))


@pytest.mark.parametrize("shape", SHAPES[:6])
def test_angle_through_f32_matches_oracle(lib, shape):
    h, w, k = shape
    img = _img(h, w, 13 * h + w)
    for j, xp in ((0, 0), (k // 2, w // 2), (k, w - 1)):
        x, d, s = lib.detect_through_point_angle(to_device(img), k, 1, 0.4, j, xp)
        _same(x, d, s, *oracle.detect_angle_through_f32(img, k, 1, 0.4, j, xp))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("B", [0, 3, 1000])
def test_through_f32_matches_oracle(lib, shape, B):
    h, w, k = shape
    img = _img(h, w, 17 * h + w + B)
    for j, xp in ((0, 0), (k // 2, w // 2), (k, w - 1), (1, w // 3)):
        if j > k:
            continue
        x, d, s = lib.detect_through_point(to_device(img), k, B, j, xp)
        _same(x, d, s, *oracle.detect_through_f32(img, k, B, j, xp))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("B", [0, 2, 1000])
def test_padded_f32_matches_oracle(lib, shape, B):
    h, w, k = shape
    img = _img(h, w, 19 * h + w + B)
    x, d, s = lib.detect_polyline_padded(to_device(img), k, B)
    _same(x, d, s, *oracle.detect_padded_f32(img, k, B))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("B", [0, 3, 1000])
def test_two_f32_matches_oracle(lib, shape, B):
    h, w, k = shape
    img = _img(h, w, 23 * h + w + B)
    for sep in sorted({1, 3, max(1, w // 4), w}):
        x, d, s = lib.detect_two_polylines(to_device(img), k, B, sep)
        xo, do, so = oracle.detect_two_f32(img, k, B, sep)
        x, d, s = x.cpu().numpy(), d.cpu().numpy(), s.cpu().numpy()
        assert np.array_equal(x, xo) and np.array_equal(d, do), (B, sep)
        assert _close(s[0], so[0]) and _close(s[1], so[1]), (B, sep)


def test_gauss_rows_f32_matches_oracle(lib):
    img = _img(9, 1500, 3)
    for r in (0, 1, 4, 12):
        out = lib.gauss_rows(to_device(img), r).cpu().numpy()
        assert out.dtype == np.float32
        assert np.array_equal(out, oracle.gauss_rows_f32(img, r)), r


def test_angle_f32_one_row_bands_smoothed_in_the_workspace(lib):
    """k = h: one-row bands take the separate smoothing launch."""
    img = _img(8, 50, 29)
    x, d, s = lib.detect_polyline_angle(to_device(img), 8, 3, 0.5)
    _same(x, d, s, *oracle.detect_angle_f32(img, 8, 3, 0.5))
