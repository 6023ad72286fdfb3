"""Pins of the CPU reference of the proposal network (it is not in the
paper): each gradient against central finite differences of its forward."""
import numpy as np

from oracle import cnn_ref


def _fd(f, a, idx, eps=1e-6):
    a1, a2 = a.copy(), a.copy()
    a1[idx] += eps
    a2[idx] -= eps
    return (f(a1) - f(a2)) / (2 * eps)


def test_conv_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    for cin, dil in ((3, 1), (3, 2), (1, 1)):
        x = rng.standard_normal((2, 5, 6, cin))
        w = rng.standard_normal((9, cin, 4))
        b = rng.standard_normal(4)
        g = rng.standard_normal((2, 5, 6, 4))        # d(loss)/d(output) of loss = sum(y * g)
        loss = lambda x_, w_=w, b_=b: float((cnn_ref.conv3x3(x_, w_, b_, dil) * g).sum())
        dx = cnn_ref.conv3x3_dgrad(g, w, dil)
        dw, db = cnn_ref.conv3x3_wgrad(x, g, dil)
        for idx in [(0, 0, 0, 0), (1, 4, 5, cin - 1), (0, 2, 3, 0)]:
            assert abs(_fd(loss, x, idx) - dx[idx]) < 1e-6
        for idx in [(0, 0, 0), (4, cin - 1, 3), (8, 0, 2)]:
            assert abs(_fd(lambda w_: loss(x, w_), w, idx) - dw[idx]) < 1e-6
        for i in range(4):
            assert abs(_fd(lambda b_: loss(x, w, b_), b, (i,)) - db[i]) < 1e-6


def test_band_head_gradient_and_pooling():
    rng = np.random.default_rng(1)
    z = rng.standard_normal((2, 8, 4, 32))
    labels = rng.integers(0, 32, (2, 2))
    pooled, loss, dz, pred = cnn_ref.band_head(z, 2, labels)
    # log-sum-exp pooling of a band is at least its maximum and at most max + log(count)
    zb = z.reshape(2, 2, 16, 32)
    assert np.all(pooled >= zb.max(2) - 1e-12)
    assert np.all(pooled <= zb.max(2) + np.log(16) + 1e-12)
    f = lambda z_: cnn_ref.band_head(z_, 2, labels)[1]
    for idx in [(0, 0, 0, 0), (1, 7, 3, 31), (0, 5, 2, labels[0, 1])]:
        assert abs(_fd(f, z, idx) - dz[idx]) < 1e-7
