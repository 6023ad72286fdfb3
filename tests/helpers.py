"""Shared helpers of the GPU parity tests: run the library through its Python
binding of the C ABI, and bring oracle arrays into the library's layout."""
import numpy as np

import oracle


def to_device(img):
    import torch
    return torch.from_numpy(np.ascontiguousarray(img)).cuda()


def hough_from_oracle(img, k, float32=False):
    """Oracle Hough images in the library layout [k][2][n][W]."""
    if float32:
        return oracle.fht_recursive(img, k, np.float32)
    return oracle.fht_recursive(img, k, np.float64)


def v_to_library_layout(Vo, n, W, dead):
    """Oracle DP values [k][2n-1][w] -> library layout [k][2][n][W] with the
    padding columns dead."""
    k, D, w = Vo.shape
    out = np.full((k, 2, n, W), dead, dtype=np.float64)
    for s in range(n):
        out[:, 0, s, :w] = Vo[:, s + n - 1, :]
        out[:, 1, s, :w] = Vo[:, n - 1 - s, :]
    return out


def check_path(img, k, B, x, d):
    """The returned polyline is admissible: vertices inside the image, |d| <=
    n-1, bends within B, x_{i+1} = x_i + d_i."""
    h, w = img.shape
    n = h // k
    x = np.asarray(x)
    d = np.asarray(d)
    assert len(x) == k + 1 and len(d) == k
    assert np.all((x >= 0) & (x < w))
    assert np.all(np.abs(d) <= n - 1)
    assert np.array_equal(np.diff(x), d)
    if k > 1:
        assert np.all(np.abs(np.diff(d)) <= B)
