"""Property-based pins of the oracle's DP queries against brute force on
random tiny problems (shapes, value ranges with many ties, bend limits,
angles, points): the integer-limit method, the bend-angle method (with and
without smoothing), the through-point query and the padded vertex domain."""
import numpy as np
import pytest

import oracle

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies
given, settings = hypothesis.given, hypothesis.settings


@st.composite
def problems(draw):
    n = draw(st.sampled_from([1, 2, 4]))
    k = draw(st.integers(1, 4 if n < 4 else 3))
    w = draw(st.integers(1, 7))
    hi = draw(st.sampled_from([1, 3, 255]))
    vals = draw(st.lists(st.integers(0, hi), min_size=n * k * w, max_size=n * k * w))
    img = np.array(vals, dtype=np.float64).reshape(n * k, w)
    return img, k


SETTINGS = settings(max_examples=80, deadline=None)


@SETTINGS
@given(problems(), st.integers(0, 7))
def test_integer_limit_dp_is_brute_force(p, B):
    img, k = p
    x, d, s = oracle.detect(img, k, B)
    bx, bd, bs, _ = oracle.brute(img, k, B)
    assert s == bs and list(x) == list(bx) and list(d) == list(bd)


@SETTINGS
@given(problems(), st.floats(0.0, 1.7), st.integers(0, 1))
def test_angle_dp_is_brute_force(p, gamma, r):
    img, k = p
    x, d, s = oracle.detect_angle(img, k, r, gamma)
    bx, bd, bs, _ = oracle.brute_angle(oracle.gauss_rows(img, r), k, gamma)
    assert s == bs and list(x) == list(bx) and list(d) == list(bd)


@SETTINGS
@given(problems(), st.integers(0, 7), st.data())
def test_through_dp_is_brute_force(p, B, data):
    img, k = p
    j = data.draw(st.integers(0, k))
    xp = data.draw(st.integers(0, img.shape[1] - 1))
    x, d, s = oracle.detect_through(img, k, B, j, xp)
    bx, bd, bs, _ = oracle.brute_through(img, k, B, j, xp)
    assert s == bs and list(x) == list(bx) and list(d) == list(bd)
    assert x[j] == xp


@SETTINGS
@given(problems(), st.integers(0, 7))
def test_padded_dp_is_brute_force(p, B):
    img, k = p
    x, d, s = oracle.detect_padded(img, k, B)
    bx, bd, bs, _ = oracle.brute_padded(img, k, B)
    assert s == bs and list(x) == list(bx) and list(d) == list(bd)
