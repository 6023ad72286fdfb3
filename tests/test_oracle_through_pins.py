"""Pins of the oracle's through-point query (Subproblems 2-3, Sec. 2.2-2.3:
the extreme polyline through a given point P on a band border) against
brute force, against the global optimum, and against the paper's own
construction of the part above P by flipping the top bands about Ox."""
import numpy as np
import pytest

import oracle


def _img(h, w, seed, hi=256):
    return np.random.default_rng(seed).integers(0, hi, (h, w)).astype(np.float64)


@pytest.mark.parametrize("seed", range(5))
def test_through_dp_equals_brute_force(seed):
    h, w, k = [(8, 6, 4), (16, 7, 4), (12, 5, 3), (16, 8, 2), (8, 9, 8)][seed]
    n = h // k
    img = _img(h, w, 500 + seed, hi=6 if seed % 2 else 256)   # small ranges: many ties
    for B in (0, 1, 2 * n - 2):
        for j in range(k + 1):
            for xp in range(w):
                x, d, s = oracle.detect_through(img, k, B, j, xp)
                bx, bd, bs, visited = oracle.brute_through(img, k, B, j, xp)
                assert visited > 0
                assert s == bs, (seed, B, j, xp)
                assert list(x) == list(bx) and list(d) == list(bd), (seed, B, j, xp)
                assert x[j] == xp
                assert oracle.path_score(img, k, x[0], d) == s


@pytest.mark.parametrize("seed", range(4))
def test_best_point_on_any_border_is_the_global_optimum(seed):
    """The best polyline passes some point of every band border: the
    maximum over xp of the through-point score is the global optimum, and
    the query at the optimum's own vertex returns the optimum itself."""
    img = _img(64, 40, 600 + seed)
    k, B = 4, 3
    gx, gd, gs = oracle.detect(img, k, B)
    for j in range(k + 1):
        scores = [oracle.detect_through(img, k, B, j, xp)[2] for xp in range(40)]
        assert max(scores) == gs
        x, d, s = oracle.detect_through(img, k, B, j, int(gx[j]))
        assert s == gs and list(x) == list(gx) and list(d) == list(gd)


@pytest.mark.parametrize("seed", range(4))
def test_flip_construction_of_the_upper_part(seed):
    """Subproblem 2 (no bend limit): the best polyline through P is the best
    part below P (bands j..k-1 starting at xp) plus the best part above it,
    which the paper finds by flipping bands 0..j-1 about Ox and running the
    same search from xp.  The flipped link covers the same pixels (central
    symmetry of the dyadic pattern)."""
    rng = np.random.default_rng(700 + seed)
    n, k, w = 8, 5, 23
    img = rng.integers(0, 256, (n * k, w)).astype(np.float64)
    B = 2 * n - 2
    for j in range(1, k):
        for xp in (0, 7, w - 1):
            _, _, s = oracle.detect_through(img, k, B, j, xp)
            lower = img[j * n:]
            upper = img[:j * n][::-1]
            _, _, sl = oracle.detect_through(lower, k - j, B, 0, xp)
            xu, du, su = oracle.detect_through(upper, j, B, 0, xp)
            assert s == sl + su, (j, xp)
            # the flipped part read back in image order is a valid upper part
            xs_up = list(xu[::-1])
            assert xs_up[-1] == xp
            assert oracle.path_score(img[:j * n], j, xs_up[0], list(-np.asarray(du[::-1]))) == su


def test_through_rejects_points_outside():
    img = _img(16, 5, 1)
    with pytest.raises(ValueError):
        oracle.detect_through(img, 4, 1, 5, 0)
    with pytest.raises(ValueError):
        oracle.detect_through(img, 4, 1, 0, 5)


@pytest.mark.parametrize("seed", range(4))
def test_angle_through_dp_equals_brute_force(seed):
    """Subproblem 3 with the bend angle: the masked angle DP against brute
    force with the direct angle test, with and without smoothing."""
    h, w, k = [(8, 6, 4), (16, 7, 4), (12, 5, 3), (16, 6, 2)][seed]
    img = _img(h, w, 1200 + seed, hi=6 if seed % 2 else 256)
    for r in (0, 1):
        scored = oracle.gauss_rows(img, r)
        for gamma in (0.0, 0.2, 0.7, 2.0):
            for j in range(k + 1):
                for xp in (0, w // 2, w - 1):
                    x, d, s = oracle.detect_angle_through(img, k, r, gamma, j, xp)
                    bx, bd, bs = oracle.brute_angle_through(scored, k, gamma, j, xp)
                    assert s == bs, (seed, r, gamma, j, xp)
                    assert list(x) == list(bx) and list(d) == list(bd)
                    assert x[j] == xp


def test_angle_through_reduces_to_the_integer_through_query():
    """gamma >= pi/2 admits every bend: the unrestricted through query."""
    img = _img(32, 20, 1300)
    for j, xp in ((0, 3), (2, 10), (4, 19)):
        a = oracle.detect_angle_through(img, 4, 0, 2.0, j, xp)
        b = oracle.detect_through(img, 4, 14, j, xp)
        assert a[2] == b[2] and list(a[0]) == list(b[0]) and list(a[1]) == list(b[1])
