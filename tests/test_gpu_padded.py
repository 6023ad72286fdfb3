"""GPU parity of the padded vertex domain (Sec. 2.2: vertices anywhere in
[0, w + h/k), zeros right of the image), through the C ABI, against the
CPU oracle (int32, bit-exact)."""
import numpy as np
import pytest

import oracle
from paper_1912_01884_gb300 import synth
from helpers import to_device

pytestmark = pytest.mark.gpu

SHAPES = [(256, 256, 4), (64, 37, 4), (128, 1000, 1), (512, 300, 2), (16, 5, 16),
          (8, 3, 4), (2048, 130, 16), (96, 77, 3), (32, 1, 2), (1024, 517, 4)]


def _img(h, w, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        return rng.integers(0, 256, (h, w)).astype(np.uint8)
    return rng.integers(-3000, 3000, (h, w)).astype(np.int32)


def _assert_padded(lib, img, k, B):
    x, d, s = lib.detect_polyline_padded(to_device(img), k, B)
    x, d, s = x.cpu().numpy(), d.cpu().numpy(), int(s.cpu().numpy()[0])
    xo, do, so = oracle.detect_padded(img, k, B)
    assert list(x) == list(xo) and list(d) == list(do), B
    assert s == so
    assert oracle.path_score_padded(img, k, x[0], d) == so


@pytest.mark.parametrize("dtype", ["u8", "i32"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("B", [0, 3, 1000])
def test_padded_matches_oracle(lib, shape, dtype, B):
    h, w, k = shape
    _assert_padded(lib, _img(h, w, dtype, 11 * h + w + B), k, B)


def test_padded_2048x2048_full_size(lib):
    wl = synth.plain_gaussian(3)
    _assert_padded(lib, wl.img, 16, 16)


def test_curve_running_off_the_right_edge(lib):
    n, k, w = 32, 8, 300
    img = np.random.default_rng(5).integers(0, 30, (n * k, w)).astype(np.uint8)
    off = oracle.off_table(n)
    x = 230
    for i in range(k):
        for y in range(n):
            c = x + off[10, y]
            if c < w:
                img[i * n + y, c] = 250
        x += 10
    _assert_padded(lib, img, k, 2)
    xs, _, _ = lib.detect_polyline_padded(to_device(img), k, 2)
    assert xs.cpu().numpy()[-1] >= w


def test_padded_rejects_bad_arguments_on_device(lib):
    import torch
    img = torch.zeros((64, 40), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_padded(img, 3, 2)
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_padded(img, 4, -1)
    with pytest.raises(TypeError):
        lib.detect_polyline_padded(img.double(), 4, 2)
