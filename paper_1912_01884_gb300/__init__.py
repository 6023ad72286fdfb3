"""fhtdp: end-to-end curves of limited curvature (arXiv 1912.01884) on GB300.

Thin Python binding of the C-ABI library ``libfhtdp.so`` (declared in
``include/fhtdp.h``).  This module only marshals arguments: PyTorch tensors
provide device memory and the current CUDA stream, and every step of the
method runs in the library's CUDA kernels.  There is no CPU fallback: if the
library cannot be loaded the calls raise.

Calls (same names as the C entry points, without the ``fhtdp_`` prefix):
  fht_bands(img, k)                  Sec. 2.1, Hough images [k, 2, n, w+n]
  polyline_dp(hough, h, w, k, B)     Sec. 2.2-2.3, Eqs. 3-4, in place
  backtrack(V, h, w, k, B)           Eq. 5 / main problem: (x, d, score)
  detect_polyline(img, k, B)         the whole method: (x, d, score)
  BatchPlan(images, ks, Bs)          many images in one persistent launch
  angle_window(n, gamma)             Sec. 2.3, Eqs. 6-7: bend-angle windows (host)
  gauss_rows(img, r)                 main problem step 1: binomial row smoothing
  polyline_dp_angle / backtrack_angle / detect_polyline_angle(img, k, r, gamma)
                                     the main problem with the bend angle
  detect_through_point(img, k, B, j, xp)               Subproblems 2-3
  detect_through_point_angle(img, k, r, gamma, j, xp)  Subproblem 3, bend angle
  detect_polyline_padded(img, k, B)  vertices in the zero padding (Sec. 2.2)
  detect_two_polylines(img, k, B, sep)                 two different polylines
  detect_polyline_horizontal(img, k, B), transpose(img)  mostly horizontal curves
The raw ctypes handle with the exact C signatures is ``lib()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = ["load", "lib", "build", "FhtdpError", "fht_bands", "polyline_dp", "backtrack",
           "detect_polyline", "detect_polyline_noalloc", "noalloc_status", "workspace_bytes",
           "launch_count",
           "BatchPlan", "Image",
           "workspace_status", "hough_bytes", "fht_workspace_bytes",
           "angle_window", "gauss_rows", "polyline_dp_angle", "backtrack_angle",
           "angle_workspace_bytes", "detect_polyline_angle", "through_workspace_bytes",
           "detect_through_point", "detect_through_point_angle", "detect_polyline_padded",
           "detect_two_polylines", "horizontal_workspace_bytes", "detect_polyline_horizontal",
           "transpose",
           "DTYPE_U8", "DTYPE_I32", "DTYPE_F32", "STATUS"]

DTYPE_U8, DTYPE_I32, DTYPE_F32 = 0, 1, 2
STATUS = {0: "FHTDP_OK", 1: "FHTDP_EINVAL", 2: "FHTDP_EWORKSPACE", 3: "FHTDP_ECUDA",
          4: "FHTDP_ETIMEOUT"}

_lock = threading.Lock()
_lib = None


class FhtdpError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(code, code), message))
        self.code = code


def build(force: bool = False) -> str:
    return _build.build(force=force)


_SIGS = {
    "fhtdp_last_error": (ctypes.c_char_p, []),
    "fhtdp_version": (ctypes.c_int, []),
    "fhtdp_launch_count": (ctypes.c_uint64, []),
    "fhtdp_hough_bytes": (ctypes.c_size_t, [ctypes.c_int] * 4),
    "fhtdp_fht_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int] * 4),
    "fhtdp_fht_bands": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5
                        + [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_polyline_dp": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5
                          + [ctypes.c_void_p]),
    "fhtdp_backtrack": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5
                        + [ctypes.c_void_p] * 4),
    "fhtdp_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int] * 5),
    "fhtdp_detect_polyline": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 6
                              + [ctypes.c_void_p] * 4 + [ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_workspace_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fhtdp_debug_inject": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_longlong]),
    "fhtdp_detect_polyline_noalloc": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 6
                                      + [ctypes.c_void_p] * 4),
    "fhtdp_detect_polyline_noalloc_status": (ctypes.c_int, [ctypes.c_void_p]),
    "fhtdp_batch_plan_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_void_p)]),
    "fhtdp_batch_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "fhtdp_batch_items": (ctypes.c_longlong, [ctypes.c_void_p]),
    "fhtdp_batch_upload": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "fhtdp_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fhtdp_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    "fhtdp_batch_plan_destroy": (None, [ctypes.c_void_p]),
    "fhtdp_batch_choice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4),
    "fhtdp_batch_configure": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 3
                              + [ctypes.c_void_p]),
    "fhtdp_batch_angle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "fhtdp_batch_points": (ctypes.c_int, [ctypes.c_void_p] * 4),
    "fhtdp_angle_window": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_void_p]),
    "fhtdp_gauss_rows": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5
                         + [ctypes.c_void_p, ctypes.c_void_p]),
    "fhtdp_polyline_dp_angle": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 4
                                + [ctypes.c_double, ctypes.c_void_p]),
    "fhtdp_backtrack_angle": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 4
                              + [ctypes.c_double] + [ctypes.c_void_p] * 4),
    "fhtdp_angle_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int] * 5),
    "fhtdp_detect_polyline_angle": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 6
                                    + [ctypes.c_double] + [ctypes.c_void_p] * 4
                                    + [ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_through_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int] * 4),
    "fhtdp_detect_through_point": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 8
                                   + [ctypes.c_void_p] * 4 + [ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_detect_through_point_angle": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 6
                                         + [ctypes.c_double, ctypes.c_int, ctypes.c_int]
                                         + [ctypes.c_void_p] * 4
                                         + [ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_detect_polyline_padded": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 6
                                     + [ctypes.c_void_p] * 4
                                     + [ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_two_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int] * 4),
    "fhtdp_detect_two_polylines": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 7
                                   + [ctypes.c_void_p] * 4 + [ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_horizontal_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int] * 5),
    "fhtdp_transpose": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 4
                        + [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "fhtdp_detect_polyline_horizontal": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 6
                                         + [ctypes.c_void_p] * 4
                                         + [ctypes.c_size_t, ctypes.c_void_p]),
    "fhtdp_cnn_downsample4": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 3
                              + [ctypes.c_void_p, ctypes.c_void_p]),
    "fhtdp_cnn_conv3x3": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5
                          + [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                             ctypes.c_void_p]),
    "fhtdp_cnn_conv3x3_dgrad": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 4
                                + [ctypes.c_void_p] * 4),
    "fhtdp_cnn_relu_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_longlong, ctypes.c_void_p]),
    "fhtdp_cnn_conv3x3_wgrad": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 5
                                + [ctypes.c_void_p] * 4),
    "fhtdp_cnn_band_head": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_int] * 4
                            + [ctypes.c_void_p, ctypes.c_float] + [ctypes.c_void_p] * 4),
    "fhtdp_cnn_adam": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int] + [ctypes.c_float] * 4
                       + [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "fhtdp_cnn_to_bf16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p]),
    "fhtdp_cnn_bin_windows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "fhtdp_cnn_status": (ctypes.c_int, [ctypes.c_int]),
    "fhtdp_cnn_param_bytes": (ctypes.c_size_t, []),
    "fhtdp_cnn_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p]),
    "fhtdp_cnn_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int] * 3),
    "fhtdp_cnn_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 4
                          + [ctypes.c_void_p, ctypes.c_size_t] + [ctypes.c_void_p] * 3),
    "fhtdp_cnn_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 4
                           + [ctypes.c_void_p, ctypes.c_size_t] + [ctypes.c_void_p] * 2),
    "fhtdp_cnn_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p] + [ctypes.c_int] * 3
                       + [ctypes.c_float, ctypes.c_int, ctypes.c_void_p]),
    "fhtdp_learned_plan_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(ctypes.c_void_p)]),
    "fhtdp_learned_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "fhtdp_learned_upload": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                            ctypes.c_void_p]),
    "fhtdp_detect_learned": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float,
                                            ctypes.c_float] + [ctypes.c_void_p] * 3),
    "fhtdp_learned_status": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "fhtdp_learned_plan_destroy": (None, [ctypes.c_void_p]),
}


class Image(ctypes.Structure):
    """struct fhtdp_image of the C ABI."""
    _fields_ = [("img", ctypes.c_void_p), ("h", ctypes.c_int), ("w", ctypes.c_int),
                ("pitch", ctypes.c_int), ("k", ctypes.c_int), ("B", ctypes.c_int),
                ("x_out", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("score_out", ctypes.c_void_p), ("d_window", ctypes.c_void_p)]


def load():
    """Load libfhtdp.so (building it in-tree if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            handle = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def lib():
    return load()


def _check(code: int):
    if code != 0:
        raise FhtdpError(code, lib().fhtdp_last_error().decode())


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    m = {torch.uint8: DTYPE_U8, torch.int32: DTYPE_I32, torch.float32: DTYPE_F32}
    if t.dtype not in m:
        raise TypeError("image dtype must be uint8, int32 or float32, got %s" % t.dtype)
    return m[t.dtype]


def _acc_dtype(code: int):
    torch = _torch()
    return torch.float32 if code == DTYPE_F32 else torch.int32


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _image(img):
    if not img.is_cuda:
        raise ValueError("image must be a CUDA tensor")
    if img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("image must be 2-D with unit column stride")
    return img.shape[0], img.shape[1], img.stride(0)


def launch_count() -> int:
    """Kernel launches the library has enqueued in this process."""
    return lib().fhtdp_launch_count()


def hough_bytes(dtype: int, h: int, w: int, k: int) -> int:
    return lib().fhtdp_hough_bytes(dtype, h, w, k)


def fht_workspace_bytes(dtype: int, h: int, w: int, k: int) -> int:
    return lib().fhtdp_fht_workspace_bytes(dtype, h, w, k)


def workspace_bytes(dtype: int, h: int, w: int, k: int, B: int) -> int:
    return lib().fhtdp_workspace_bytes(dtype, h, w, k, B)


def fht_bands(img, k: int, out=None, ws=None, stream=None):
    """Hough images of the k bands: tensor [k, 2, n, w + n] (int32 or float32)."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    if h % k:
        raise ValueError("h must be a multiple of k")
    n = h // k
    if out is None:
        out = torch.empty((k, 2, n, w + n), dtype=_acc_dtype(code), device=img.device)
    need = fht_workspace_bytes(code, h, w, k)
    if ws is None and need:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    _check(lib().fhtdp_fht_bands(img.data_ptr(), code, h, w, pitch, k, out.data_ptr(),
                                 ws.data_ptr() if ws is not None else None,
                                 ws.numel() if ws is not None else 0, _stream(stream)))
    return out


def polyline_dp(hough, h: int, w: int, k: int, B: int, stream=None):
    """Bend-limited DP in place over the Hough images; returns the tensor."""
    torch = _torch()
    code = DTYPE_F32 if hough.dtype == torch.float32 else DTYPE_I32
    _check(lib().fhtdp_polyline_dp(hough.data_ptr(), code, h, w, k, B, _stream(stream)))
    return hough


def _outputs(k, code, device):
    torch = _torch()
    x = torch.empty(k + 1, dtype=torch.int32, device=device)
    d = torch.empty(k, dtype=torch.int32, device=device)
    score = torch.empty(1, dtype=_acc_dtype(code), device=device)
    return x, d, score


def backtrack(V, h: int, w: int, k: int, B: int, out=None, stream=None):
    """(x[k+1], d[k], score[1]) device tensors from DP values."""
    torch = _torch()
    code = DTYPE_F32 if V.dtype == torch.float32 else DTYPE_I32
    x, d, score = out if out is not None else _outputs(k, code, V.device)
    _check(lib().fhtdp_backtrack(V.data_ptr(), code, h, w, k, B, x.data_ptr(), d.data_ptr(),
                                 score.data_ptr(), _stream(stream)))
    return x, d, score


def workspace_status(ws, stream=None) -> int:
    """Status of the last run that used `ws` (synchronises the stream):
    0, or raises FhtdpError (FHTDP_ETIMEOUT when a device-side wait gave up)."""
    _check(lib().fhtdp_workspace_status(ws.data_ptr(), _stream(stream)))
    return 0


class BatchPlan:
    """Many images of one pixel type in one persistent launch.

    ``images`` are 2-D CUDA tensors, ``ks`` and ``Bs`` their band counts and
    bend limits.  Outputs ``x[i]``, ``d[i]``, ``score[i]`` are allocated here,
    or are the rows of ``out = (X, D, S)``; ``windows[i]`` (optional) is a
    device int32 [k][2] tensor of allowed displacements per band (pruned DP).
    ``run()`` enqueues the whole batch (one memset, one kernel) and may be
    captured in a CUDA graph."""

    def __init__(self, images, ks, Bs, ws=None, stream=None, out=None, windows=None):
        torch = _torch()
        if not images:
            raise ValueError("empty batch")
        code = _dtype_code(images[0])
        dev = images[0].device
        self.images = list(images)
        self.x, self.d, self.score = [], [], []
        arr = (Image * len(images))()
        for i, (img, k, B) in enumerate(zip(images, ks, Bs)):
            if _dtype_code(img) != code:
                raise TypeError("one pixel type per batch")
            h, w, pitch = _image(img)
            x, d, sc = (out[0][i], out[1][i], out[2][i]) if out is not None else \
                _outputs(k, code, dev)
            self.x.append(x)
            self.d.append(d)
            self.score.append(sc)
            win = windows[i] if windows is not None else None
            arr[i] = Image(img.data_ptr(), h, w, pitch, k, B, x.data_ptr(), d.data_ptr(),
                           sc.data_ptr(), win.data_ptr() if win is not None else None)
        self.windows = windows
        self._arr = arr
        handle = ctypes.c_void_p()
        _check(lib().fhtdp_batch_plan_create(ctypes.cast(arr, ctypes.c_void_p), len(images),
                                             code, ctypes.byref(handle)))
        self._plan = handle
        need = lib().fhtdp_batch_workspace_bytes(handle)
        self.ws = ws if ws is not None else torch.empty(need, dtype=torch.uint8, device=dev)
        if self.ws.numel() < need:
            raise ValueError("workspace too small")
        self.items = lib().fhtdp_batch_items(handle)
        _check(lib().fhtdp_batch_upload(handle, self.ws.data_ptr(), self.ws.numel(),
                                        _stream(stream)))

    def run(self, stream=None):
        _check(lib().fhtdp_batch_run(self._plan, self.ws.data_ptr(), _stream(stream)))

    def status(self, stream=None):
        return workspace_status(self.ws, stream)

    def autotune(self, reps=3, stream=None):
        """Tunes the queue schedule and width and, per band height, the tile
        width and register FHT depth by timing runs (synchronises the stream);
        returns the chosen width in column tiles per band level or step."""
        t = ctypes.c_longlong(0)
        _check(lib().fhtdp_batch_autotune(self._plan, self.ws.data_ptr(), int(reps),
                                          _stream(stream), ctypes.byref(t)))
        return t.value

    def choice(self, n: int):
        """The plan's schedule ("groups", "chains", "chains-spread256", "chains-slow256" or
        "chains-spread256-slow256"), width, and the tile
        width and register FHT depth of its images of band height n."""
        mode, target = ctypes.c_int(0), ctypes.c_longlong(0)
        tile, depth = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().fhtdp_batch_choice(self._plan, int(n), ctypes.byref(mode),
                                        ctypes.byref(target), ctypes.byref(tile),
                                        ctypes.byref(depth)))
        return {"schedule": ("groups", "chains", "chains-spread256", "chains-slow256",
                             "chains-spread256-slow256")[mode.value], "width": target.value,
                "tile": tile.value, "depth": depth.value}

    def configure(self, n: int, tile: int, depth: int, stream=None):
        """Sets the tile width and register FHT depth of the images of band
        height n by hand (the tuner's per-height choices)."""
        _check(lib().fhtdp_batch_configure(self._plan, self.ws.data_ptr(), int(n), int(tile),
                                           int(depth), _stream(stream)))

    def points(self, points, stream=None):
        """Through-point queries (Subproblems 2-3): points[i] = (border j in
        1..k, column xp) for image i, or None for no restriction (uint8 images
        with at least two bands of at most 128 rows)."""
        arr = (ctypes.c_int32 * (2 * len(self.images)))()
        for i, pt in enumerate(points):
            arr[2 * i], arr[2 * i + 1] = (-1, 0) if pt is None else (int(pt[0]), int(pt[1]))
        _check(lib().fhtdp_batch_points(self._plan, self.ws.data_ptr(),
                                        ctypes.cast(arr, ctypes.c_void_p), _stream(stream)))

    def angle(self, gamma: float):
        """Bend-angle windows of gamma radians for every run of the plan (Sec.
        2.3): the images must be smoothed rows (gauss_rows), int32 or
        float32, all of one band height in 2..128."""
        _check(lib().fhtdp_batch_angle(self._plan, float(gamma)))

    def close(self):
        if self._plan:
            lib().fhtdp_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def detect_polyline_noalloc(img, k: int, B: int, out=None, stream=None):
    """detect_polyline for callers that cannot allocate device memory: the
    scratch is a fixed array inside the library (FHTDP_NOALLOC_SCRATCH_BYTES).
    Calls that overlap on the GPU race on that array."""
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    x, d, score = out if out is not None else _outputs(k, code, img.device)
    _check(lib().fhtdp_detect_polyline_noalloc(img.data_ptr(), code, h, w, pitch, k, B,
                                               x.data_ptr(), d.data_ptr(), score.data_ptr(),
                                               _stream(stream)))
    return x, d, score


def noalloc_status(stream=None) -> int:
    """Status of the last detect_polyline_noalloc run on the current device
    (synchronises the stream): 0, or raises FhtdpError (FHTDP_ETIMEOUT when a
    device-side wait gave up)."""
    _check(lib().fhtdp_detect_polyline_noalloc_status(_stream(stream)))
    return 0


def detect_polyline(img, k: int, B: int, out=None, ws=None, stream=None):
    """The whole method on one device image: (x[k+1], d[k], score[1])."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    need = workspace_bytes(code, h, w, k, B)
    if need == 0:   # invalid arguments: let the library name the problem
        _check(lib().fhtdp_detect_polyline(None, code, h, w, pitch, k, B, None, None, None,
                                           None, 0, _stream(stream)))
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    x, d, score = out if out is not None else _outputs(k, code, img.device)
    _check(lib().fhtdp_detect_polyline(img.data_ptr(), code, h, w, pitch, k, B, x.data_ptr(),
                                       d.data_ptr(), score.data_ptr(), ws.data_ptr(), ws.numel(),
                                       _stream(stream)))
    return x, d, score


# ---------------------------------------------------------------------------
# The main problem (Sec. 2.3): row smoothing and bend-angle windows.

def angle_window(n: int, gamma: float):
    """numpy int32 [2n-1][2]: row d + n - 1 holds the range of next
    displacements whose bend angle from d is at most gamma (host call)."""
    import numpy as np
    out = np.zeros((2 * n - 1, 2), dtype=np.int32)
    _check(lib().fhtdp_angle_window(int(n), float(gamma), out.ctypes.data))
    return out


def gauss_rows(img, r: int, out=None, stream=None):
    """Every row convolved with the binomial weights C(2r, r+t): [h, w], int32
    for uint8 / int32 images, float32 for float32 ones."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    if out is None:
        out = torch.empty((h, w), dtype=_acc_dtype(code), device=img.device)
    _check(lib().fhtdp_gauss_rows(img.data_ptr(), code, h, w, pitch, int(r), out.data_ptr(),
                                  _stream(stream)))
    return out


def polyline_dp_angle(hough, h: int, w: int, k: int, gamma: float, stream=None):
    """The DP with bend-angle windows in place over int32 or float32 Hough
    images."""
    code = DTYPE_F32 if hough.dtype == _torch().float32 else DTYPE_I32
    _check(lib().fhtdp_polyline_dp_angle(hough.data_ptr(), code, h, w, k, float(gamma),
                                         _stream(stream)))
    return hough


def backtrack_angle(V, h: int, w: int, k: int, gamma: float, out=None, stream=None):
    """(x[k+1], d[k], score[1]) read back with the bend-angle windows."""
    code = DTYPE_F32 if V.dtype == _torch().float32 else DTYPE_I32
    x, d, score = out if out is not None else _outputs(k, code, V.device)
    _check(lib().fhtdp_backtrack_angle(V.data_ptr(), code, h, w, k, float(gamma),
                                       x.data_ptr(), d.data_ptr(), score.data_ptr(),
                                       _stream(stream)))
    return x, d, score


def angle_workspace_bytes(dtype: int, h: int, w: int, k: int, r: int) -> int:
    return lib().fhtdp_angle_workspace_bytes(dtype, h, w, k, r)


def detect_polyline_angle(img, k: int, r: int, gamma: float, out=None, ws=None, stream=None):
    """Steps 1-3 of the main problem on one device image (uint8, int32 or
    float32): (x[k+1], d[k], score[1]), the score of the smoothed image."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    need = angle_workspace_bytes(code, h, w, k, r)
    if need == 0:   # invalid arguments: let the library name the problem
        _check(lib().fhtdp_detect_polyline_angle(None, code, h, w, pitch, k, int(r),
                                                 float(gamma), None, None, None, None, 0,
                                                 _stream(stream)))
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    x, d, score = out if out is not None else _outputs(k, code, img.device)
    _check(lib().fhtdp_detect_polyline_angle(img.data_ptr(), code, h, w, pitch, k, int(r),
                                             float(gamma), x.data_ptr(), d.data_ptr(),
                                             score.data_ptr(), ws.data_ptr(), ws.numel(),
                                             _stream(stream)))
    return x, d, score


# ---------------------------------------------------------------------------
# Subproblems 2-3: the extreme polyline through a given point.

def through_workspace_bytes(dtype: int, h: int, w: int, k: int) -> int:
    return lib().fhtdp_through_workspace_bytes(dtype, h, w, k)


def detect_through_point(img, k: int, B: int, j: int, xp: int, out=None, ws=None, stream=None):
    """The best polyline through (xp, j * h/k) on a band border (uint8 or
    int32 image): (x[k+1], d[k], score[1]) with x[j] = xp."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    need = through_workspace_bytes(code, h, w, k)
    if need == 0:   # invalid arguments: let the library name the problem
        _check(lib().fhtdp_detect_through_point(None, code, h, w, pitch, k, B, j, xp, None, None,
                                                None, None, 0, _stream(stream)))
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    x, d, score = out if out is not None else _outputs(k, code, img.device)
    _check(lib().fhtdp_detect_through_point(img.data_ptr(), code, h, w, pitch, k, B, int(j),
                                            int(xp), x.data_ptr(), d.data_ptr(),
                                            score.data_ptr(), ws.data_ptr(), ws.numel(),
                                            _stream(stream)))
    return x, d, score


# ---------------------------------------------------------------------------
# Two different extreme polylines; mostly horizontal curves.

def detect_two_polylines(img, k: int, B: int, sep: int, out=None, ws=None, stream=None):
    """The optimum and the best polyline whose top vertex is at least `sep`
    columns from it (uint8, int32 or float32 image): x [2, k+1], d [2, k],
    score [2]."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    need = lib().fhtdp_two_workspace_bytes(code, h, w, k)
    if need == 0:   # invalid arguments: let the library name the problem
        _check(lib().fhtdp_detect_two_polylines(None, code, h, w, pitch, k, B, sep, None, None,
                                                None, None, 0, _stream(stream)))
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    if out is None:
        out = (torch.empty((2, k + 1), dtype=torch.int32, device=img.device),
               torch.empty((2, k), dtype=torch.int32, device=img.device),
               torch.empty(2, dtype=_acc_dtype(code), device=img.device))
    x, d, score = out
    _check(lib().fhtdp_detect_two_polylines(img.data_ptr(), code, h, w, pitch, k, B, int(sep),
                                            x.data_ptr(), d.data_ptr(), score.data_ptr(),
                                            ws.data_ptr(), ws.numel(), _stream(stream)))
    return x, d, score


def horizontal_workspace_bytes(dtype: int, h: int, w: int, k: int, B: int) -> int:
    return lib().fhtdp_horizontal_workspace_bytes(dtype, h, w, k, B)


def detect_polyline_horizontal(img, k: int, B: int, out=None, ws=None, stream=None):
    """Mostly horizontal polyline over k vertical strips of w/k columns:
    (y[k+1], d[k], score[1])."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    need = horizontal_workspace_bytes(code, h, w, k, B)
    if need == 0:   # invalid arguments: let the library name the problem
        _check(lib().fhtdp_detect_polyline_horizontal(None, code, h, w, pitch, k, B, None, None,
                                                      None, None, 0, _stream(stream)))
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    y, d, score = out if out is not None else _outputs(k, code, img.device)
    _check(lib().fhtdp_detect_polyline_horizontal(img.data_ptr(), code, h, w, pitch, k, B,
                                                  y.data_ptr(), d.data_ptr(), score.data_ptr(),
                                                  ws.data_ptr(), ws.numel(), _stream(stream)))
    return y, d, score


def transpose(img, out=None, stream=None):
    """dst[x][y] = img[y][x] on the device (the row pitch of `out` may exceed h)."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    if out is None:
        out = torch.empty((w, h), dtype=img.dtype, device=img.device)
    if out.dim() != 2 or out.shape[0] != w or out.shape[1] != h or out.stride(1) != 1:
        raise ValueError("out must be a [w, h] view with unit column stride")
    _check(lib().fhtdp_transpose(img.data_ptr(), code, h, w, pitch, out.data_ptr(), out.stride(0),
                                 _stream(stream)))
    return out


def detect_polyline_padded(img, k: int, B: int, out=None, ws=None, stream=None):
    """The method with vertices anywhere in [0, w + h/k) (zeros right of the
    image), uint8, int32 or float32 image: (x[k+1], d[k], score[1])."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    need = through_workspace_bytes(code, h, w, k)
    if need == 0:   # invalid arguments: let the library name the problem
        _check(lib().fhtdp_detect_polyline_padded(None, code, h, w, pitch, k, B, None, None,
                                                  None, None, 0, _stream(stream)))
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    x, d, score = out if out is not None else _outputs(k, code, img.device)
    _check(lib().fhtdp_detect_polyline_padded(img.data_ptr(), code, h, w, pitch, k, B,
                                              x.data_ptr(), d.data_ptr(), score.data_ptr(),
                                              ws.data_ptr(), ws.numel(), _stream(stream)))
    return x, d, score


def detect_through_point_angle(img, k: int, r: int, gamma: float, j: int, xp: int, out=None,
                               ws=None, stream=None):
    """Subproblem 3: the best polyline through (xp, j * h/k) with bend angles
    at most gamma, rows smoothed with half-width r (uint8, int32 or float32 image)."""
    torch = _torch()
    h, w, pitch = _image(img)
    code = _dtype_code(img)
    need = angle_workspace_bytes(code, h, w, k, r)
    if need == 0:   # invalid arguments: let the library name the problem
        _check(lib().fhtdp_detect_through_point_angle(None, code, h, w, pitch, k, int(r),
                                                      float(gamma), int(j), int(xp), None, None,
                                                      None, None, 0, _stream(stream)))
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device=img.device)
    x, d, score = out if out is not None else _outputs(k, code, img.device)
    _check(lib().fhtdp_detect_through_point_angle(img.data_ptr(), code, h, w, pitch, k, int(r),
                                                  float(gamma), int(j), int(xp), x.data_ptr(),
                                                  d.data_ptr(), score.data_ptr(), ws.data_ptr(),
                                                  ws.numel(), _stream(stream)))
    return x, d, score
