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
