"""Pins of the oracle's two-polyline query (Sec. 3, Figs. 6d, 7a: two
different extreme polylines, read as suppression on the top vertex) and of
mostly horizontal detection by transposition (Sec. 3, Fig. 7), against brute
force and sums written out along the horizontal line pattern."""
import numpy as np
import pytest

import oracle


def _img(h, w, seed, hi=256):
    return np.random.default_rng(seed).integers(0, hi, (h, w)).astype(np.float64)


@pytest.mark.parametrize("seed", range(6))
def test_second_polyline_equals_brute_force(seed):
    h, w, k = [(8, 9, 4), (16, 10, 4), (12, 8, 3), (16, 9, 2), (8, 12, 8), (16, 7, 4)][seed]
    n = h // k
    img = _img(h, w, 800 + seed, hi=5 if seed % 2 else 256)
    for B in (0, 1, 2 * n - 2):
        for sep in (1, 2, 4, w):
            xs, ds, sc = oracle.detect_two(img, k, B, sep)
            gx, gd, gs = oracle.detect(img, k, B)
            assert sc[0] == gs and list(xs[0]) == list(gx) and list(ds[0]) == list(gd)
            bx, bd, bs = oracle.brute_apart(img, k, B, int(gx[0]), sep)
            assert sc[1] == bs, (seed, B, sep)
            assert list(xs[1]) == list(bx) and list(ds[1]) == list(bd), (seed, B, sep)
            if bs != -np.inf:
                assert abs(int(xs[1][0]) - int(xs[0][0])) >= sep
                assert sc[1] <= sc[0]
                assert oracle.path_score(img, k, xs[1][0], ds[1]) == sc[1]
            else:
                assert list(xs[1]) == [-1] * (k + 1)


def test_two_distant_planted_polylines_are_both_found():
    """Two bright straight polylines far apart over weak noise: the optimum is
    the brighter, the second the other one."""
    rng = np.random.default_rng(9)
    n, k, w = 16, 4, 120
    img = rng.integers(0, 20, (n * k, w)).astype(np.float64)
    off = oracle.off_table(n)
    for x0, d, v in ((20, 3, 250.0), (90, -2, 200.0)):
        x = x0
        for i in range(k):
            for y in range(n):
                img[i * n + y, x + (off[d, y] if d >= 0 else -off[-d, y])] = v
            x += d
    xs, ds, sc = oracle.detect_two(img, k, 2, 10)
    assert xs[0][0] == 20 and list(ds[0]) == [3] * k
    assert xs[1][0] == 90 and list(ds[1]) == [-2] * k


def _horizontal_sum(img, k, y0, ds):
    """Sum along a mostly horizontal polyline written out directly: link i
    covers the n columns of strip i, row y_i + sign(d) off_|d|(t) at column
    i n + t."""
    h, w = img.shape
    n = w // k
    off = oracle.off_table(n)
    total, y = 0.0, y0
    for i, d in enumerate(ds):
        for t in range(n):
            total += img[y + (off[d, t] if d >= 0 else -off[-d, t]), i * n + t]
        y += d
    return total


@pytest.mark.parametrize("seed", range(4))
def test_horizontal_detection_equals_brute_force_along_rows(seed):
    h, w, k = [(9, 16, 4), (7, 12, 3), (10, 16, 2), (6, 8, 8)][seed]
    img = _img(h, w, 900 + seed)
    n = w // k
    for B in (0, 1, 2 * n - 2):
        y, d, s = oracle.detect_horizontal(img, k, B)
        by, bd, bs, _ = oracle.brute(np.ascontiguousarray(img.T), k, B)
        assert s == bs and list(y) == list(by) and list(d) == list(bd)
        assert _horizontal_sum(img, k, int(y[0]), list(d)) == s
        assert np.all((np.asarray(y) >= 0) & (np.asarray(y) < h))


def test_planted_horizontal_polyline_is_recovered():
    rng = np.random.default_rng(4)
    h, w, k = 40, 64, 4
    n = w // k
    img = rng.integers(0, 30, (h, w)).astype(np.float64)
    off = oracle.off_table(n)
    y, ds = 10, [2, 5, 3, -4]
    for i, d in enumerate(ds):
        for t in range(n):
            img[y + (off[d, t] if d >= 0 else -off[-d, t]), i * n + t] = 220.0
        y += d
    yy, dd, s = oracle.detect_horizontal(img, k, 10)
    assert yy[0] == 10 and list(dd) == ds
