"""GPU parity of two different extreme polylines (Sec. 3, Figs. 6d and 7a,
suppression on the top vertex) and of mostly horizontal detection by
transposition (Sec. 3, Fig. 7), through the C ABI, against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1912_01884_gb300 import synth
from helpers import check_path, to_device

pytestmark = pytest.mark.gpu

SHAPES = [(256, 256, 4), (64, 37, 4), (128, 1000, 1), (512, 300, 2), (16, 5, 16),
          (8, 3, 4), (2048, 130, 16), (96, 77, 3), (32, 1, 2), (1024, 517, 4)]


def _img(h, w, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        return rng.integers(0, 256, (h, w)).astype(np.uint8)
    if dtype == "i32":
        return rng.integers(-3000, 3000, (h, w)).astype(np.int32)
    return np.abs(rng.standard_normal((h, w))).astype(np.float32) * np.float32(2.5)


def _assert_two(lib, img, k, B, sep):
    x, d, s = lib.detect_two_polylines(to_device(img), k, B, sep)
    x, d, s = x.cpu().numpy(), d.cpu().numpy(), s.cpu().numpy()
    xo, do, so = oracle.detect_two(img, k, B, sep)
    assert np.array_equal(x, xo) and np.array_equal(d, do), (B, sep)
    assert int(s[0]) == so[0]
    if so[1] == -np.inf:
        assert int(s[1]) == np.iinfo(np.int32).min and np.all(x[1] == -1)
    else:
        assert int(s[1]) == so[1]
        check_path(img, k, B, x[1], d[1])


@pytest.mark.parametrize("dtype", ["u8", "i32"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("B", [0, 3, 1000])
def test_two_polylines_match_oracle(lib, shape, dtype, B):
    h, w, k = shape
    img = _img(h, w, dtype, 7 * h + w + B)
    for sep in sorted({1, 3, max(1, w // 4), w}):
        _assert_two(lib, img, k, B, sep)


@pytest.mark.parametrize("seed", range(2))
def test_two_polylines_2048x2048_full_size(lib, seed):
    wl = synth.plain_gaussian(seed)
    _assert_two(lib, wl.img, 16, 16, 64)


def _assert_horizontal(lib, img, k, B):
    y, d, s = lib.detect_polyline_horizontal(to_device(img), k, B)
    y, d, s = y.cpu().numpy(), d.cpu().numpy(), s.cpu().numpy()[0]
    t = np.ascontiguousarray(img.T)
    if img.dtype == np.float32:
        yo, do, so32 = oracle.detect_f32(t, k, B)
        assert list(y) == list(yo) and list(d) == list(do)
        assert np.float32(s) == np.float32(so32)
    else:
        yo, do, so = oracle.detect_horizontal(img, k, B)
        assert list(y) == list(yo) and list(d) == list(do)
        assert int(s) == int(so)
    check_path(t, k, B, y, d)


@pytest.mark.parametrize("dtype", ["u8", "i32", "f32"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("B", [0, 3, 1000])
def test_horizontal_matches_oracle(lib, shape, dtype, B):
    w, h, k = shape          # the transposes of the vertical shapes
    _assert_horizontal(lib, _img(h, w, dtype, 3 * h + w + B), k, B)


@pytest.mark.parametrize("seed", range(2))
def test_horizontal_2048x2048_k16_B16_full_size(lib, seed):
    wl = synth.plain_gaussian(seed)
    _assert_horizontal(lib, np.ascontiguousarray(wl.img.T), 16, 16)


def test_horizontal_respects_pitch(lib):
    import torch
    img = _img(300, 128, "u8", 5)
    big = torch.zeros((300, 160), dtype=torch.uint8, device="cuda")
    big[:, :128] = to_device(img)
    y, d, s = lib.detect_polyline_horizontal(big[:, :128], 4, 5)
    yo, do, so = oracle.detect_horizontal(img, 4, 5)
    assert list(y.cpu().numpy()) == list(yo) and int(s.cpu().numpy()[0]) == int(so)


def test_two_and_horizontal_reject_bad_arguments_on_device(lib):
    import torch
    img = torch.zeros((64, 40), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.FhtdpError):
        lib.detect_two_polylines(img, 4, 2, 0)               # sep < 1
    with pytest.raises(lib.FhtdpError):
        lib.detect_two_polylines(img, 4, -1, 3)
    with pytest.raises(TypeError):
        lib.detect_two_polylines(img.double(), 4, 2, 3)
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_horizontal(img, 3, 2)             # 40 columns, k = 3
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_horizontal(img, 4, -1)


@pytest.mark.parametrize("dtype", ["u8", "i32", "f32"])
@pytest.mark.parametrize("h,w", [(1, 1), (33, 65), (300, 7), (2048, 2048), (31, 1000), (67, 64),
                                 (64, 132)])
@pytest.mark.parametrize("aligned", [True, False])
def test_transpose_matches_numpy(lib, dtype, h, w, aligned):
    """Both uint8 kernels: 4-byte words when both pitches are multiples of 4,
    bytes otherwise."""
    import torch
    img = _img(h, w, dtype, h + w)
    pad = (8 - h % 4) if aligned else (5 if (h + 5) % 4 else 6)
    out = torch.zeros((w, h + pad), dtype=to_device(img).dtype, device="cuda")
    lib.transpose(to_device(img), out=out[:, :h])
    got = out.cpu().numpy()
    assert np.array_equal(got[:, :h], img.T)
    assert not got[:, h:].any()


def test_batch_of_transposed_images_equals_horizontal_calls(lib):
    """The batched route for mostly horizontal images: transpose each, run
    one batch plan; equal to the single-image horizontal call."""
    imgs = [_img(200 + 40 * j, 256, "u8", 40 + j) for j in range(4)]
    dev = [to_device(m) for m in imgs]
    tr = [lib.transpose(m) for m in dev]
    plan = lib.BatchPlan(tr, [4] * 4, [6] * 4)
    plan.run()
    for i, m in enumerate(dev):
        y, d, s = lib.detect_polyline_horizontal(m, 4, 6)
        assert list(plan.x[i].cpu().numpy()) == list(y.cpu().numpy())
        assert list(plan.d[i].cpu().numpy()) == list(d.cpu().numpy())
        assert int(plan.score[i].cpu().numpy()[0]) == int(s.cpu().numpy()[0])
