"""The C-ABI library builds, loads, exports every declared entry point and
rejects bad arguments on the host (no GPU needed: nothing is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "fhtdp.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fhtdp_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    handle = lib.lib()
    names = _declared()
    assert "fhtdp_detect_polyline" in names and "fhtdp_fht_bands" in names
    for name in names:
        assert hasattr(handle, name), name


def test_version_and_sizes(lib):
    L = lib.lib()
    assert L.fhtdp_version() >= 100
    # [k][2][n][w+n] elements of 4 bytes
    assert L.fhtdp_hough_bytes(0, 2048, 2048, 16) == 16 * 2 * 128 * (2048 + 128) * 4
    assert L.fhtdp_hough_bytes(0, 100, 10, 3) == 0          # h not a multiple of k
    assert L.fhtdp_hough_bytes(0, 96, 10, 1) == 0           # n not a power of two
    assert L.fhtdp_hough_bytes(0, 512, 10, 1) == 0          # n > 256
    assert L.fhtdp_hough_bytes(7, 64, 10, 1) == 0           # unknown dtype
    assert L.fhtdp_workspace_bytes(0, 256, 256, 4, 8) > 0
    assert L.fhtdp_workspace_bytes(0, 256, 256, 4, -1) == 0


@pytest.mark.parametrize("args,code", [
    ((None, 0, 100, 10, 10, 3, 1), 1),         # h % k != 0
    ((None, 0, 96, 10, 10, 1, 1), 1),          # n = 96 not a power of two
    ((None, 0, 64, 10, 5, 4, 1), 1),           # pitch < w
    ((None, 0, 64, 10, 10, 4, -1), 1),         # B < 0
    ((None, 9, 64, 10, 10, 4, 1), 1),          # dtype
    ((None, 0, 64, 10, 10, 4, 1), 1),          # null image
])
def test_detect_rejects_bad_arguments_before_launch(lib, args, code):
    L = lib.lib()
    r = L.fhtdp_detect_polyline(*args, None, None, None, None, 0, None)
    assert r == code
    assert L.fhtdp_last_error().decode()


def test_detect_rejects_small_workspace(lib):
    L = lib.lib()
    fake = ctypes.c_void_p(16)      # never dereferenced: rejected before launch
    r = L.fhtdp_detect_polyline(fake, 0, 64, 10, 10, 4, 1, fake, fake, fake, fake, 8, None)
    assert r == 2 and "workspace" in L.fhtdp_last_error().decode()


def test_fht_and_dp_reject_bad_arguments(lib):
    L = lib.lib()
    assert L.fhtdp_fht_bands(None, 0, 64, 10, 10, 4, None, None, 0, None) == 1
    assert L.fhtdp_polyline_dp(None, 0, 64, 10, 4, 1, None) == 1
    assert L.fhtdp_polyline_dp(ctypes.c_void_p(16), 0, 64, 10, 4, -2, None) == 1
    assert L.fhtdp_backtrack(None, 0, 64, 10, 4, 1, None, None, None, None) == 1


def test_batch_autotune_rejects_bad_arguments(lib):
    """The queue tuner checks its plan and workspace on the host: without a
    plan, or with a workspace the plan was not bound to (no upload), it
    returns FHTDP_EINVAL before any launch."""
    L = lib.lib()
    width = ctypes.c_longlong(-1)
    assert L.fhtdp_batch_autotune(None, ctypes.c_void_p(16), 1, None, ctypes.byref(width)) == 1
    img = lib.Image(16, 64, 40, 40, 4, 2, 16, 16, 16, None)   # never dereferenced
    plan = ctypes.c_void_p()
    assert L.fhtdp_batch_plan_create(ctypes.byref(img), 1, 0, ctypes.byref(plan)) == 0
    try:
        r = L.fhtdp_batch_autotune(plan, ctypes.c_void_p(256), 1, None, ctypes.byref(width))
        assert r == 1 and "workspace" in L.fhtdp_last_error().decode()
        assert width.value == -1
    finally:
        L.fhtdp_batch_plan_destroy(plan)


def test_angle_window_is_computed_on_the_host_like_the_oracle(lib):
    """The library's bend-angle table (a host computation, no GPU) equals the
    oracle's pair-by-pair definition, boundary angles included."""
    import math
    import numpy as np
    import oracle
    for n in (1, 2, 8, 64, 128, 256):
        for g in (0.0, 0.02, math.radians(10), 0.3, 1.0, math.pi / 2, 3.0,
                  math.atan(1 / n), math.atan(5 / n) - math.atan(2 / n)):
            assert np.array_equal(lib.angle_window(n, g), oracle.angle_window(n, g)), (n, g)
    L = lib.lib()
    buf = (ctypes.c_int32 * 2)()
    assert L.fhtdp_angle_window(3, 0.1, buf) == 1          # n not a power of two
    assert L.fhtdp_angle_window(512, 0.1, buf) == 1        # n > 256
    assert L.fhtdp_angle_window(1, -0.5, buf) == 1
    assert L.fhtdp_angle_window(1, float("inf"), buf) == 1
    assert L.fhtdp_angle_window(1, 0.1, None) == 1


def test_angle_entries_reject_bad_arguments_before_launch(lib):
    L = lib.lib()
    fake = ctypes.c_void_p(16)      # never dereferenced: rejected before launch
    assert L.fhtdp_angle_workspace_bytes(0, 64, 10, 4, 2) > 0
    assert L.fhtdp_angle_workspace_bytes(2, 64, 10, 4, 2) > 0       # float images
    assert L.fhtdp_angle_workspace_bytes(3, 64, 10, 4, 2) == 0      # unknown dtype
    assert L.fhtdp_angle_workspace_bytes(0, 64, 10, 4, 13) == 0     # r > 12
    args = (fake, fake, fake, fake, 1 << 30, None)
    assert L.fhtdp_detect_polyline_angle(fake, 3, 64, 10, 10, 4, 2, 0.3, *args) == 1
    assert L.fhtdp_detect_polyline_angle(fake, 0, 64, 10, 10, 4, -1, 0.3, *args) == 1
    assert L.fhtdp_detect_polyline_angle(fake, 0, 64, 10, 10, 4, 2, -0.3, *args) == 1
    assert L.fhtdp_detect_polyline_angle(fake, 0, 64, 10, 10, 4, 2, float("nan"), *args) == 1
    assert L.fhtdp_detect_polyline_angle(fake, 0, 64, 10, 9, 4, 2, 0.3, *args) == 1   # pitch
    assert L.fhtdp_detect_polyline_angle(None, 0, 64, 10, 10, 4, 2, 0.3, *args) == 1
    assert L.fhtdp_detect_polyline_angle(fake, 0, 4096, 8, 8, 16, 10, 0.3, *args) == 1
    assert "4^r" in L.fhtdp_last_error().decode()
    r = L.fhtdp_detect_polyline_angle(fake, 0, 64, 10, 10, 4, 2, 0.3, fake, fake, fake, fake,
                                      64, None)
    assert r == 2 and "workspace" in L.fhtdp_last_error().decode()
    assert L.fhtdp_gauss_rows(fake, 3, 4, 4, 4, 1, fake, None) == 1
    assert L.fhtdp_gauss_rows(fake, 0, 4, 4, 3, 1, fake, None) == 1
    assert L.fhtdp_gauss_rows(None, 0, 4, 4, 4, 1, fake, None) == 1
    assert L.fhtdp_polyline_dp_angle(None, 0, 64, 10, 4, 0.3, None) == 1
    assert L.fhtdp_polyline_dp_angle(fake, 0, 96, 10, 1, 0.3, None) == 1
    assert L.fhtdp_backtrack_angle(fake, 0, 64, 10, 4, 0.3, None, fake, fake, None) == 1


def test_through_point_rejects_bad_arguments_before_launch(lib):
    L = lib.lib()
    fake = ctypes.c_void_p(16)      # never dereferenced: rejected before launch
    assert L.fhtdp_through_workspace_bytes(0, 64, 10, 4) > 0
    assert L.fhtdp_through_workspace_bytes(2, 64, 10, 4) > 0        # float images
    assert L.fhtdp_through_workspace_bytes(3, 64, 10, 4) == 0       # unknown dtype
    outs = (fake, fake, fake, fake, 1 << 30, None)
    for j, xp in ((5, 0), (-1, 0), (1, 10), (1, -1)):
        assert L.fhtdp_detect_through_point(fake, 0, 64, 10, 10, 4, 2, j, xp, *outs) == 1
    assert L.fhtdp_detect_through_point(fake, 3, 64, 10, 10, 4, 2, 1, 1, *outs) == 1
    assert L.fhtdp_detect_through_point(fake, 0, 64, 10, 10, 4, -1, 1, 1, *outs) == 1
    assert L.fhtdp_detect_through_point(None, 0, 64, 10, 10, 4, 2, 1, 1, *outs) == 1
    r = L.fhtdp_detect_through_point(fake, 0, 64, 10, 10, 4, 2, 1, 1, fake, fake, fake, fake,
                                     64, None)
    assert r == 2 and "workspace" in L.fhtdp_last_error().decode()


def test_two_and_horizontal_reject_bad_arguments_before_launch(lib):
    L = lib.lib()
    fake = ctypes.c_void_p(16)      # never dereferenced: rejected before launch
    outs = (fake, fake, fake, fake, 1 << 30, None)
    assert L.fhtdp_two_workspace_bytes(0, 64, 10, 4) > 0
    assert L.fhtdp_detect_two_polylines(fake, 0, 64, 10, 10, 4, 2, 0, *outs) == 1
    assert L.fhtdp_detect_two_polylines(fake, 3, 64, 10, 10, 4, 2, 1, *outs) == 1
    assert L.fhtdp_detect_two_polylines(fake, 0, 64, 10, 10, 4, -1, 1, *outs) == 1
    r = L.fhtdp_detect_two_polylines(fake, 0, 64, 10, 10, 4, 2, 1, fake, fake, fake, fake, 64,
                                     None)
    assert r == 2
    # horizontal: bands over the width (w = k n)
    assert L.fhtdp_horizontal_workspace_bytes(0, 10, 64, 4, 2) > 0
    assert L.fhtdp_horizontal_workspace_bytes(0, 64, 10, 4, 2) == 0
    assert L.fhtdp_detect_polyline_horizontal(fake, 0, 10, 64, 64, 3, 2, *outs) == 1
    assert L.fhtdp_detect_polyline_horizontal(fake, 0, 10, 64, 63, 4, 2, *outs) == 1   # pitch
    assert L.fhtdp_detect_polyline_horizontal(fake, 9, 10, 64, 64, 4, 2, *outs) == 1
    r = L.fhtdp_detect_polyline_horizontal(fake, 0, 10, 64, 64, 4, 2, fake, fake, fake, fake, 64,
                                           None)
    assert r == 2 and "workspace" in L.fhtdp_last_error().decode()


def test_transpose_rejects_bad_arguments_before_launch(lib):
    L = lib.lib()
    a, b = ctypes.c_void_p(16), ctypes.c_void_p(4096)
    assert L.fhtdp_transpose(a, 0, 4, 8, 7, b, 4, None) == 1      # pitch < w
    assert L.fhtdp_transpose(a, 0, 4, 8, 8, b, 3, None) == 1      # dst pitch < h
    assert L.fhtdp_transpose(a, 5, 4, 8, 8, b, 4, None) == 1      # dtype
    assert L.fhtdp_transpose(a, 0, 4, 8, 8, a, 4, None) == 1      # in place
    assert L.fhtdp_transpose(None, 0, 4, 8, 8, b, 4, None) == 1
    assert L.fhtdp_transpose(a, 0, 0, 8, 8, b, 4, None) == 1


def test_padded_rejects_bad_arguments_before_launch(lib):
    L = lib.lib()
    fake = ctypes.c_void_p(16)      # never dereferenced: rejected before launch
    outs = (fake, fake, fake, fake, 1 << 30, None)
    assert L.fhtdp_detect_polyline_padded(fake, 3, 64, 10, 10, 4, 2, *outs) == 1
    assert L.fhtdp_detect_polyline_padded(fake, 0, 64, 10, 10, 3, 2, *outs) == 1
    assert L.fhtdp_detect_polyline_padded(fake, 0, 64, 10, 10, 4, -1, *outs) == 1
    assert L.fhtdp_detect_polyline_padded(fake, 0, 64, 10, 9, 4, 2, *outs) == 1
    r = L.fhtdp_detect_polyline_padded(fake, 0, 64, 10, 10, 4, 2, fake, fake, fake, fake, 64,
                                       None)
    assert r == 2


def test_through_point_angle_rejects_bad_arguments_before_launch(lib):
    L = lib.lib()
    fake = ctypes.c_void_p(16)      # never dereferenced: rejected before launch
    outs = (fake, fake, fake, fake, 1 << 30, None)
    f = L.fhtdp_detect_through_point_angle
    assert f(fake, 0, 64, 10, 10, 4, 2, 0.3, 5, 0, *outs) == 1       # border > k
    assert f(fake, 0, 64, 10, 10, 4, 2, 0.3, 1, 10, *outs) == 1      # xp >= w
    assert f(fake, 0, 64, 10, 10, 4, 2, -0.3, 1, 1, *outs) == 1
    assert f(fake, 0, 64, 10, 10, 4, 13, 0.3, 1, 1, *outs) == 1
    assert f(fake, 3, 64, 10, 10, 4, 2, 0.3, 1, 1, *outs) == 1
    assert f(fake, 0, 64, 10, 10, 4, 2, 0.3, 1, 1, fake, fake, fake, fake, 64, None) == 2


def test_cnn_and_learned_entries_reject_bad_arguments_before_launch(lib):
    """The learned proposal's calls check their arguments on the host: a width
    that is not a multiple of 64, a channel count other than 1 or 32, a
    dilation outside 1..8, null buffers, shapes the band head or the
    downsample cannot take, and null plans (every case returns EINVAL with a
    message before anything is enqueued)."""
    L = lib.lib()
    f = ctypes.c_void_p(256)      # never dereferenced: rejected before any launch
    bad = [
        lambda: L.fhtdp_cnn_conv3x3(f, 32, 1, 6, 160, 2, f, None, 1, f, None),    # w % 64
        lambda: L.fhtdp_cnn_conv3x3(f, 16, 1, 6, 192, 2, f, None, 1, f, None),    # cin
        lambda: L.fhtdp_cnn_conv3x3(f, 32, 1, 6, 192, 9, f, None, 1, f, None),    # dil > 8
        lambda: L.fhtdp_cnn_conv3x3(f, 32, 1, 6, 192, 0, f, None, 1, f, None),    # dil < 1
        lambda: L.fhtdp_cnn_conv3x3(None, 32, 1, 6, 192, 2, f, None, 1, f, None),  # null x
        lambda: L.fhtdp_cnn_conv3x3(f, 32, 0, 6, 192, 2, f, None, 1, f, None),    # no image
        lambda: L.fhtdp_cnn_conv3x3_wgrad(f, 32, 1, 6, 100, 1, f, f, None, None),  # w % 64
        lambda: L.fhtdp_cnn_conv3x3_wgrad(f, 3, 1, 6, 128, 1, f, f, None, None),   # cin
        lambda: L.fhtdp_cnn_conv3x3_wgrad(f, 32, 1, 6, 128, 1, f, None, None, None),  # null dw
        lambda: L.fhtdp_cnn_conv3x3_dgrad(f, 1, 6, 63, 1, f, f, f, None),          # w % 64
        lambda: L.fhtdp_cnn_downsample4(f, 1, 6, 64, f, None),                      # h % 4
        lambda: L.fhtdp_cnn_band_head(f, 1, 10, 64, 4, None, 1.0, None, None, None, None),
        lambda: L.fhtdp_cnn_adam(f, f, f, f, 0, 1e-3, 0.9, 0.999, 1e-8, 1, None, None),
        lambda: L.fhtdp_cnn_adam(f, f, f, f, 8, 1e-3, 0.9, 0.999, 1e-8, 0, None, None),
        lambda: L.fhtdp_cnn_bin_windows(f, 4, 64, -1, f, None),                     # margin
        lambda: L.fhtdp_cnn_relu_backward(f, f, -1, None),
        lambda: L.fhtdp_cnn_init(None, 0, None),
        lambda: L.fhtdp_cnn_step(f, f, 0, 64, 64, 1e-3, 1, None),                   # n < 1
        lambda: L.fhtdp_detect_learned(None, f, 0.0, 0.5, f, f, None),
        lambda: L.fhtdp_learned_upload(None, f, 1 << 20, None),
        lambda: L.fhtdp_learned_status(None, f, None),
    ]
    for i, call in enumerate(bad):
        assert call() == 1, i
        assert L.fhtdp_last_error().decode(), i
    out = ctypes.c_void_p()
    assert L.fhtdp_learned_plan_create(None, 0, 6, ctypes.byref(out)) == 1
    assert not out.value
