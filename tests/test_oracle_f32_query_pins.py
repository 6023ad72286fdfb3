"""Pins of the oracle's float32 queries (Secs. 2.2-2.3 and 3 on float32
images): on images of small integers every float32 sum is exact, so each
query must return exactly the brute-force answer (float64, pinned in its own
tests) over every admissible polyline; on real-valued images the float32
answer must be optimal to within the 1e-5 relative score tolerance of float
response maps, judged in float64 on the polyline it returns."""
import math

import numpy as np
import pytest

import oracle

REL = 1e-5


def _ints(seed, h, w, hi=256):
    return np.random.default_rng(seed).integers(0, hi, (h, w)).astype(np.float32)


def _reals(seed, h, w):
    rng = np.random.default_rng(seed)
    return np.abs(rng.standard_normal((h, w))).astype(np.float32)


@pytest.mark.parametrize("r", [0, 1, 2, 5])
def test_gauss_rows_f32_is_numpy_convolution_on_integers(r):
    img = _ints(r, 4, 29)
    wts = np.array([math.comb(2 * r, j) for j in range(2 * r + 1)], dtype=np.float64)
    out = oracle.gauss_rows_f32(img, r)
    for y in range(img.shape[0]):
        assert np.array_equal(out[y].astype(np.float64),
                              np.convolve(img[y].astype(np.float64), wts, mode="same"))


@pytest.mark.parametrize("r", [1, 3])
def test_gauss_rows_f32_within_rounding_of_float64_on_reals(r):
    img = _reals(10 + r, 3, 40)
    got = oracle.gauss_rows_f32(img, r).astype(np.float64)
    want = oracle.gauss_rows(img.astype(np.float64), r)
    # 2r + 1 products and sums of positive terms: relative error below
    # (2(2r + 1)) float32 half-ulps
    assert np.all(np.abs(got - want) <= (4 * r + 2) * 2.0 ** -24 * want + 1e-30)


@pytest.mark.parametrize("seed", range(4))
def test_angle_f32_equals_brute_force_on_integer_images(seed):
    h, w, k = [(8, 7, 4), (16, 9, 4), (16, 8, 2), (12, 6, 3)][seed]
    img = _ints(500 + seed, h, w)
    for r in (0, 1):
        sm = oracle.gauss_rows(img.astype(np.float64), r)
        for gamma in (0.0, 0.2, 0.7, 2.0):
            x, d, s = oracle.detect_angle_f32(img, k, r, gamma)
            bx, bd, bs, _ = oracle.brute_angle(sm, k, gamma)
            assert s == bs and np.array_equal(x, bx) and np.array_equal(d, bd), (r, gamma)


@pytest.mark.parametrize("seed", range(3))
def test_angle_through_f32_equals_brute_force_on_integer_images(seed):
    img = _ints(520 + seed, 16, 8)
    k = 4
    sm = oracle.gauss_rows(img.astype(np.float64), 1)
    for j in (0, 2, 4):
        for xp in (0, 3, 7):
            x, d, s = oracle.detect_angle_through_f32(img, k, 1, 0.4, j, xp)
            bx, bd, bs = oracle.brute_angle_through(sm, k, 0.4, j, xp)
            assert s == bs and np.array_equal(x, bx) and np.array_equal(d, bd), (j, xp)


@pytest.mark.parametrize("seed", range(3))
def test_through_f32_equals_brute_force_on_integer_images(seed):
    img = _ints(540 + seed, 16, 7)
    k = 4
    for B in (0, 2, 6):
        for j in (0, 1, 4):
            for xp in (0, 4, 6):
                x, d, s = oracle.detect_through_f32(img, k, B, j, xp)
                bx, bd, bs, _ = oracle.brute_through(img.astype(np.float64), k, B, j, xp)
                assert s == bs and np.array_equal(x, bx) and np.array_equal(d, bd), (B, j, xp)


@pytest.mark.parametrize("seed", range(3))
def test_padded_f32_equals_brute_force_on_integer_images(seed):
    img = _ints(560 + seed, 8, 5)
    for k, B in ((2, 1), (4, 2), (2, 6)):
        x, d, s = oracle.detect_padded_f32(img, k, B)
        bx, bd, bs, _ = oracle.brute_padded(img.astype(np.float64), k, B)
        assert s == bs and np.array_equal(x, bx) and np.array_equal(d, bd), (k, B)


@pytest.mark.parametrize("seed", range(3))
def test_two_f32_equals_brute_force_on_integer_images(seed):
    img = _ints(580 + seed, 16, 9)
    k = 4
    for B, sep in ((1, 2), (3, 4), (6, 9)):
        xs, ds, sc = oracle.detect_two_f32(img, k, B, sep)
        gx, gd, gs, _ = oracle.brute(img.astype(np.float64), k, B)
        assert sc[0] == gs and np.array_equal(xs[0], gx) and np.array_equal(ds[0], gd)
        bx, bd, bs = oracle.brute_apart(img.astype(np.float64), k, B, int(gx[0]), sep)
        assert sc[1] == bs and np.array_equal(xs[1], bx) and np.array_equal(ds[1], bd), (B, sep)


@pytest.mark.parametrize("seed", range(2))
def test_horizontal_f32_equals_brute_force_on_the_transposed_integer_image(seed):
    img = _ints(600 + seed, 7, 16)
    x, d, s = oracle.detect_horizontal_f32(img, 4, 2)
    bx, bd, bs, _ = oracle.brute(np.ascontiguousarray(img.T).astype(np.float64), 4, 2)
    assert s == bs and np.array_equal(x, bx) and np.array_equal(d, bd)


@pytest.mark.parametrize("seed", range(3))
def test_f32_queries_are_optimal_within_tolerance_on_real_images(seed):
    """On |N(0,1)| images the float32 decisions may differ from float64
    ones only between polylines whose exact scores agree to 1e-5."""
    h, w, k = 64, 48, 4
    img = _reals(620 + seed, h, w)
    img64 = img.astype(np.float64)
    # main problem, smoothing r = 2, 10 degrees
    x, d, s = oracle.detect_angle_f32(img, k, 2, math.radians(10))
    x6, d6, s6 = oracle.detect_angle(img64, k, 2, math.radians(10))
    sm = oracle.gauss_rows(img64, 2)
    assert abs(s - s6) <= REL * abs(s6)
    assert abs(oracle.path_score(sm, k, x[0], d) - s6) <= REL * abs(s6)
    # through a point, bend limit 3
    x, d, s = oracle.detect_through_f32(img, k, 3, 2, 20)
    x6, d6, s6 = oracle.detect_through(img64, k, 3, 2, 20)
    assert x[2] == 20 and abs(s - s6) <= REL * abs(s6)
    assert abs(oracle.path_score(img64, k, x[0], d) - s6) <= REL * abs(s6)
    # vertices in the padding
    x, d, s = oracle.detect_padded_f32(img, k, 3)
    x6, d6, s6 = oracle.detect_padded(img64, k, 3)
    assert abs(s - s6) <= REL * abs(s6)
    assert abs(oracle.path_score_padded(img64, k, x[0], d) - s6) <= REL * abs(s6)
    # two polylines: the first is the optimum, the second respects the
    # separation from the first
    xs, ds, sc = oracle.detect_two_f32(img, k, 3, 8)
    x6, d6, s6 = oracle.detect_two(img64, k, 3, 8)
    assert abs(sc[0] - s6[0]) <= REL * abs(s6[0])
    assert abs(int(xs[1][0]) - int(xs[0][0])) >= 8
    assert abs(oracle.path_score(img64, k, xs[1][0], ds[1]) - sc[1]) <= REL * abs(sc[1])
