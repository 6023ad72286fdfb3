"""Pins of the oracle's padded vertex domain (Sec. 2.2: Hough columns over
[0, w + h/k - 1]; Sec. 2.1: bands extended by h/k zero columns on the right):
brute force with the plain sum (zeros right of the image), the cyclic FHT
against that sum for every link inside the padded width, and the superset
relation with the in-image method."""
import numpy as np
import pytest

import oracle


def _img(h, w, seed, hi=256):
    return np.random.default_rng(seed).integers(0, hi, (h, w)).astype(np.float64)


@pytest.mark.parametrize("seed", range(5))
def test_padded_dp_equals_brute_force(seed):
    h, w, k = [(8, 5, 4), (16, 6, 4), (12, 4, 3), (16, 3, 2), (8, 2, 8)][seed]
    n = h // k
    img = _img(h, w, 1000 + seed, hi=4 if seed % 2 else 256)
    for B in (0, 1, 2 * n - 2):
        x, d, s = oracle.detect_padded(img, k, B)
        bx, bd, bs, visited = oracle.brute_padded(img, k, B)
        assert visited > 0
        assert s == bs and list(x) == list(bx) and list(d) == list(bd), (seed, B)
        assert oracle.path_score_padded(img, k, x[0], d) == s
        assert np.all((x >= 0) & (x < w + n))


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
def test_cyclic_fht_is_the_clipped_sum_inside_the_padded_width(n):
    """For a link with both ends in [0, w + n) the cyclic Hough value never
    wraps: it is the sum of the in-image pixels of the line."""
    w = 9
    img = _img(n, w, 77 + n)
    H = oracle.fht_recursive(img, 1)
    W = w + n
    for x in range(W):
        for d in range(-(n - 1), n):
            if not 0 <= x + d < W:
                continue
            want = oracle.path_score_padded(img, 1, x, [d])
            got = H[0, 0 if d >= 0 else 1, abs(d), x]
            assert got == want, (n, x, d)


@pytest.mark.parametrize("seed", range(3))
def test_padded_optimum_is_at_least_the_in_image_optimum(seed):
    img = _img(64, 30, 1100 + seed)
    for B in (0, 3, 20):
        _, _, sp = oracle.detect_padded(img, 4, B)
        _, _, si = oracle.detect(img, 4, B)
        assert sp >= si


def test_polyline_leaving_the_image_is_found_with_padding_vertices():
    """A bright line that runs off the right edge: only the padded domain
    can follow it, and its score is its in-image part."""
    n, k, w = 8, 4, 20
    img = np.zeros((n * k, w))
    off = oracle.off_table(n)
    x = 12
    for i in range(k):
        for y in range(n):
            c = x + off[3, y]
            if c < w:
                img[i * n + y, c] = 100.0
        x += 3
    xs, ds, s = oracle.detect_padded(img, k, 0)
    assert list(ds) == [3] * k and xs[0] == 12 and xs[-1] == 24
    assert s == img.sum()
    _, _, si = oracle.detect(img, k, 0)
    assert si < s
