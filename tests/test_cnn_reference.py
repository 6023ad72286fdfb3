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


def test_conv_forward_single_lit_pixel_is_the_flipped_dilated_kernel():
    """Worked by hand: one lit pixel at (3, 3) of a 7x7 single-channel image,
    weights 1..9 in tap order (tap = 3 ky + kx), dilation 2.  Output pixel p
    takes w[tap] from input p + 2 (ky - 1, kx - 1), so the lit pixel reaches
    p = (3, 3) - 2 (ky - 1, kx - 1): w[0] = 1 lands at (5, 5), w[2] = 3 at (5, 1),
    w[4] = 5 at (3, 3), w[6] = 7 at (1, 5), w[8] = 9 at (1, 1); every other
    output is the bias 0.5."""
    x = np.zeros((1, 7, 7, 1))
    x[0, 3, 3, 0] = 1.0
    w = np.arange(1.0, 10.0).reshape(9, 1, 1)
    y = cnn_ref.conv3x3(x, w, np.array([0.5]), 2)[0, :, :, 0]
    want = np.full((7, 7), 0.5)
    for (r, c), v in {(5, 5): 1, (5, 3): 2, (5, 1): 3, (3, 5): 4, (3, 3): 5, (3, 1): 6,
                      (1, 5): 7, (1, 3): 8, (1, 1): 9}.items():
        want[r, c] += v
    assert np.array_equal(y, want)


def test_conv_forward_equals_scipy_correlation_with_a_dilated_kernel():
    """Multi-channel dilated convolution against scipy's 2-D correlation
    ('same' size, zero boundary) with the 3x3 kernel spread to (2d+1)^2."""
    from scipy.signal import correlate2d
    rng = np.random.default_rng(3)
    for cin, cout, dil in ((3, 4, 1), (2, 3, 2), (1, 5, 4)):
        x = rng.standard_normal((2, 9, 11, cin))
        w = rng.standard_normal((9, cin, cout))
        b = rng.standard_normal(cout)
        y = cnn_ref.conv3x3(x, w, b, dil)
        for nimg in range(2):
            for co in range(cout):
                acc = np.full((9, 11), b[co])
                for ci in range(cin):
                    K = np.zeros((2 * dil + 1, 2 * dil + 1))
                    K[::dil, ::dil] = w[:, ci, co].reshape(3, 3)
                    acc += correlate2d(x[nimg, :, :, ci], K, mode="same")
                assert np.allclose(y[nimg, :, :, co], acc, rtol=0, atol=1e-12)
