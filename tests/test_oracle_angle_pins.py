"""Pins of the oracle's main-problem functions (Sec. 2.3: Gaussian row
smoothing and the bend-angle restriction of Eqs. 6-7) against facts fixed by
the paper and by mathematics: the tan form of Eqs. 6-7, Pascal's triangle and
numpy's convolution, the special cases gamma = 0 and gamma >= pi/2 (which
reduce to the already pinned integer bend limit), and brute force."""
import math

import numpy as np
import pytest

import oracle


def _eq67_interval(n, d, gamma):
    """[lo, hi] of Eqs. 6-7 in displacement form: n tg(max(-pi/4, a - g)) <=
    e <= n tg(min(pi/4, a + g)), a = atg(d / n), clipped to |e| <= n - 1.
    Returns None when a bound lies within 1e-7 of an integer (a boundary
    case the tan form cannot settle in double)."""
    a = math.atan(d / n)
    lo_f = n * math.tan(max(-math.pi / 4, a - gamma))
    hi_f = n * math.tan(min(math.pi / 4, a + gamma))
    for v in (lo_f, hi_f):
        if abs(v - round(v)) < 1e-7 and abs(round(v)) < n:
            return None
    return max(math.ceil(lo_f), -(n - 1)), min(math.floor(hi_f), n - 1)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 128, 256])
@pytest.mark.parametrize("gamma", [0.05, math.radians(10), 0.3, 0.8, 1.3])
def test_window_is_the_tan_form_of_eqs_6_7(n, gamma):
    t = oracle.angle_window(n, gamma)
    checked = 0
    for d in range(-(n - 1), n):
        want = _eq67_interval(n, d, gamma)
        if want is None:
            continue
        assert tuple(t[d + n - 1]) == want, (n, gamma, d)
        checked += 1
    assert checked >= (2 * n - 1) // 2


@pytest.mark.parametrize("n", [2, 8, 32, 128])
@pytest.mark.parametrize("gamma", [0.02, 0.2, 0.6])
def test_window_properties(n, gamma):
    t = oracle.angle_window(n, gamma).astype(np.int64)
    d = np.arange(-(n - 1), n)
    lo, hi = t[:, 0], t[:, 1]
    assert np.all(lo <= d) and np.all(d <= hi)           # a straight continuation is allowed
    assert np.all(np.diff(lo) >= 0) and np.all(np.diff(hi) >= 0)   # monotone in d
    assert np.array_equal(lo, -hi[::-1])                 # mirror symmetry d -> -d
    assert np.all(lo >= -(n - 1)) and np.all(hi <= n - 1)
    # every e inside is within gamma, both neighbours outside are not
    a = np.arctan(np.arange(-(n - 1), n) / n)
    for i in range(2 * n - 1):
        inside = np.abs(a - a[i]) <= gamma
        assert inside[lo[i] + n - 1:hi[i] + n].all()
        assert inside.sum() == hi[i] - lo[i] + 1


def test_window_limits():
    n = 16
    t0 = oracle.angle_window(n, 0.0)
    assert np.array_equal(t0[:, 0], np.arange(-(n - 1), n))
    assert np.array_equal(t0[:, 1], np.arange(-(n - 1), n))
    tf = oracle.angle_window(n, math.pi / 2)
    assert np.all(tf[:, 0] == -(n - 1)) and np.all(tf[:, 1] == n - 1)
    # a bend just below the angle between the vertical and the first step
    # admits only the straight continuation at d = 0
    g = math.atan(1 / n)
    assert tuple(oracle.angle_window(n, g * (1 - 1e-6))[n - 1]) == (0, 0)
    assert tuple(oracle.angle_window(n, g * (1 + 1e-6))[n - 1]) == (-1, 1)
    with pytest.raises(ValueError):
        oracle.angle_window(n, -0.1)


@pytest.mark.parametrize("r,row", [(0, [1]), (1, [1, 2, 1]), (2, [1, 4, 6, 4, 1]),
                                   (3, [1, 6, 15, 20, 15, 6, 1])])
def test_gauss_of_a_delta_is_a_pascal_row(r, row):
    img = np.zeros((3, 17))
    img[1, 8] = 1.0
    out = oracle.gauss_rows(img, r)
    want = np.zeros(17)
    want[8 - r:8 + r + 1] = row
    assert np.array_equal(out[1], want)
    assert not out[0].any() and not out[2].any()


@pytest.mark.parametrize("r", [0, 1, 2, 4, 6])
def test_gauss_is_numpy_convolution_with_binomial_weights(r):
    rng = np.random.default_rng(r)
    img = rng.integers(0, 256, (5, 23)).astype(np.float64)
    wts = np.array([math.comb(2 * r, j) for j in range(2 * r + 1)], dtype=np.float64)
    out = oracle.gauss_rows(img, r)
    for y in range(img.shape[0]):
        assert np.array_equal(out[y], np.convolve(img[y], wts, mode="same"))
    # the weights are 4^r times a distribution of variance r / 2
    t = np.arange(-r, r + 1)
    assert wts.sum() == 4 ** r
    assert abs((wts * t * t).sum() / wts.sum() - r / 2) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_angle_dp_equals_angle_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    h, w, k = [(8, 7, 4), (16, 9, 4), (12, 6, 3), (16, 10, 2), (8, 9, 2), (16, 6, 8)][seed]
    img = rng.integers(0, 256, (h, w)).astype(np.float64)
    n = h // k
    for gamma in (0.0, 0.13, 0.41, 0.9, 2.0):
        x, d, s = oracle.detect_angle(img, k, 0, gamma)
        bx, bd, bs, visited = oracle.brute_angle(img, k, gamma)
        assert visited > 0
        assert s == bs, (seed, gamma)
        assert np.array_equal(x, bx) and np.array_equal(d, bd), (seed, gamma)
        assert oracle.path_score(img, k, x[0], d) == s
        a = np.arctan(np.asarray(d) / n)
        assert np.all(np.abs(np.diff(a)) <= gamma)


@pytest.mark.parametrize("seed", range(3))
def test_angle_dp_with_smoothing_equals_brute_force_on_the_smoothed_image(seed):
    rng = np.random.default_rng(200 + seed)
    img = rng.integers(0, 256, (16, 9)).astype(np.float64)
    for r in (1, 2):
        x, d, s = oracle.detect_angle(img, 4, r, 0.3)
        bx, bd, bs, _ = oracle.brute_angle(oracle.gauss_rows(img, r), 4, 0.3)
        assert s == bs and np.array_equal(x, bx) and np.array_equal(d, bd)


@pytest.mark.parametrize("seed", range(3))
def test_gamma_zero_and_right_angle_reduce_to_the_integer_bend_limit(seed):
    """gamma = 0 admits only e = d, the integer limit B = 0; gamma >= pi/2
    admits every e, the limit B = 2n - 2 (both pinned against brute force
    in the DP's own tests)."""
    rng = np.random.default_rng(300 + seed)
    img = rng.integers(0, 256, (32, 21)).astype(np.float64)
    k = 4
    n = 8
    for gamma, B in ((0.0, 0), (math.pi / 2, 2 * n - 2), (3.0, 2 * n - 2)):
        xa, da, sa = oracle.detect_angle(img, k, 0, gamma)
        xb, db, sb = oracle.detect(img, k, B)
        assert sa == sb and np.array_equal(xa, xb) and np.array_equal(da, db)


def test_angle_dp_tables_and_read_back_pieces_agree():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, (32, 40)).astype(np.float64)
    k, n = 4, 8
    t = oracle.angle_window(n, 0.25)
    H = oracle.fht_recursive(oracle.gauss_rows(img, 1), k)
    V = oracle.dp_angle(H, 32, 40, k, t)
    x, d, s = oracle.backtrack_angle(V, 32, 40, k, t)
    assert (x, d, s)[2] == oracle.detect_angle(img, k, 1, 0.25)[2]
    assert s == V[0].max()
    # the score read back is the sum along the returned polyline
    assert oracle.path_score(oracle.gauss_rows(img, 1), k, x[0], d) == s


@pytest.mark.parametrize("seed", range(3))
def test_planted_bent_polyline_is_recovered_after_smoothing(seed):
    """A bright polyline with bend angles under gamma, on uniform noise and
    one pixel wide, is found exactly through the smoothing."""
    rng = np.random.default_rng(400 + seed)
    h, w, k = 64, 48, 8
    n = h // k
    gamma = 0.35
    img = rng.integers(0, 40, (h, w)).astype(np.float64)
    a = np.arctan(np.arange(-(n - 1), n) / n)
    ds = [int(rng.integers(-3, 4))]
    for _ in range(k - 1):
        ok = [e for e in range(-(n - 1), n) if abs(a[e + n - 1] - a[ds[-1] + n - 1]) <= gamma
              and abs(e) <= 3]
        ds.append(int(rng.choice(ok)))
    x0 = w // 2 - sum(ds) // 2
    off = oracle.off_table(n)
    x = x0
    for i, d in enumerate(ds):
        for y in range(n):
            c = x + (off[d, y] if d >= 0 else -off[-d, y])
            img[i * n + y, c] = 255.0
        x += d
    xs, got, s = oracle.detect_angle(img, k, 2, gamma)
    assert list(got) == ds and xs[0] == x0
