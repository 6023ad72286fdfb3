"""CPU oracle of the band-FHT + bend-limited DP method (arXiv 1912.01884).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package; the library's product path never
does, and shares no code with it.  The arithmetic lives in ``oracle.c``
(plain C loops, double precision plus a float32 copy of the recursion and the
DP); this module compiles it with gcc and marshals numpy arrays.

Function map (paper passages in the C file's comments):
  off_table        Sec. 2.1, dyadic line pattern of the FHT (refs [10], [34])
  fht_direct       Sec. 2.1, Hough images by direct summation along each line
  fht_recursive    Sec. 2.1, Hough images by the dyadic recursion
  dp               Sec. 2.2-2.3, Eqs. 3-4 with the bend window (RangeMaxQ)
  backtrack        Sec. 2.2 Eq. 5, main problem steps 2-3
  path_score       Sec. 2.1, sum along a given polyline (plain definition)
  brute            every admissible polyline, tiny images only
  detect_windowed  the DP restricted to per-band displacement windows (the
                   pruned DP of the learned proposal, not in the paper)
  detect / detect_f32   the whole method (CPU baseline)
  gauss_rows       Sec. 2.3 main problem step 1, row-wise Gaussian smoothing
  angle_window     Sec. 2.3 Eqs. 6-7, the bend-angle range of displacements
  dp_angle / backtrack_angle / detect_angle
                   the main problem with the angle restriction
  brute_angle      every polyline passing the direct angle test, tiny images
  dp_through / detect_through / brute_through
                   Sec. 2.2-2.3 Subproblems 2-3: the extreme polyline through a
                   given point on a band border
  detect_angle_through / brute_angle_through
                   Sec. 2.3 Subproblem 3: through a given point with the bend angle
  detect_two / brute_apart
                   Sec. 3: two different extreme polylines (suppression on x_0)
  detect_horizontal  Sec. 3, Fig. 7: mostly horizontal polylines (transposition)
  detect_padded / brute_padded / path_score_padded
                   Sec. 2.2: vertices anywhere in the zero-padded band width
  gauss_rows_f32 / detect_angle_f32 / detect_angle_through_f32 /
  detect_through_f32 / detect_padded_f32 / detect_two_f32 /
  detect_horizontal_f32
                   the same queries on float32 images in float32 arithmetic
                   (the decisions of the library's float path)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_I32P = ctypes.POINTER(ctypes.c_int32)
_F64P = ctypes.POINTER(ctypes.c_double)
_F32P = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no fast-math,
    no floating-point contraction).  Returns the library path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_off_table.argtypes = [ctypes.c_int, _I32P]
            lib.oracle_fht_direct_f64.argtypes = [_F64P, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, _F64P]
            lib.oracle_fht_recursive_f64.argtypes = [_F64P, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, _F64P]
            lib.oracle_fht_recursive_f32.argtypes = [_F32P, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, _F32P]
            lib.oracle_dp_f64.argtypes = [_F64P] + [ctypes.c_int] * 4 + [_F64P]
            lib.oracle_dp_f32.argtypes = [_F32P] + [ctypes.c_int] * 4 + [_F32P]
            lib.oracle_backtrack_f64.argtypes = [_F64P] + [ctypes.c_int] * 4 + [_I32P, _I32P]
            lib.oracle_backtrack_f64.restype = ctypes.c_double
            lib.oracle_backtrack_f32.argtypes = [_F32P] + [ctypes.c_int] * 4 + [_I32P, _I32P]
            lib.oracle_backtrack_f32.restype = ctypes.c_double
            lib.oracle_path_score_f64.argtypes = [_F64P] + [ctypes.c_int] * 4 + [_I32P]
            lib.oracle_path_score_f64.restype = ctypes.c_double
            lib.oracle_brute_f64.argtypes = ([_F64P] + [ctypes.c_int] * 4
                                             + [_I32P, _I32P, ctypes.POINTER(ctypes.c_long)])
            lib.oracle_brute_f64.restype = ctypes.c_double
            lib.oracle_detect_f64.argtypes = [_F64P] + [ctypes.c_int] * 4 + [_I32P, _I32P]
            lib.oracle_detect_f64.restype = ctypes.c_double
            lib.oracle_detect_f32.argtypes = [_F32P] + [ctypes.c_int] * 4 + [_I32P, _I32P]
            lib.oracle_detect_f32.restype = ctypes.c_double
            lib.oracle_detect_win_f64.argtypes = ([_F64P] + [ctypes.c_int] * 4
                                                  + [_I32P, _I32P, _I32P])
            lib.oracle_detect_win_f64.restype = ctypes.c_double
            lib.oracle_brute_win_f64.argtypes = ([_F64P] + [ctypes.c_int] * 4
                                                 + [_I32P, _I32P, _I32P,
                                                    ctypes.POINTER(ctypes.c_long)])
            lib.oracle_brute_win_f64.restype = ctypes.c_double
            lib.oracle_gauss_rows_f64.argtypes = [_F64P] + [ctypes.c_int] * 3 + [_F64P]
            lib.oracle_angle_window.argtypes = [ctypes.c_int, ctypes.c_double, _I32P]
            lib.oracle_dp_angle_f64.argtypes = [_F64P] + [ctypes.c_int] * 3 + [_I32P, _F64P]
            lib.oracle_backtrack_angle_f64.argtypes = ([_F64P] + [ctypes.c_int] * 3
                                                       + [_I32P, _I32P, _I32P])
            lib.oracle_backtrack_angle_f64.restype = ctypes.c_double
            lib.oracle_brute_angle_f64.argtypes = ([_F64P] + [ctypes.c_int] * 3
                                                   + [ctypes.c_double, _I32P, _I32P,
                                                      ctypes.POINTER(ctypes.c_long)])
            lib.oracle_brute_angle_f64.restype = ctypes.c_double
            lib.oracle_detect_angle_f64.argtypes = ([_F64P] + [ctypes.c_int] * 4
                                                    + [ctypes.c_double, _I32P, _I32P])
            lib.oracle_detect_angle_f64.restype = ctypes.c_double
            lib.oracle_dp_through_f64.argtypes = [_F64P] + [ctypes.c_int] * 6 + [_F64P]
            lib.oracle_detect_through_f64.argtypes = ([_F64P] + [ctypes.c_int] * 6
                                                      + [_I32P, _I32P])
            lib.oracle_detect_through_f64.restype = ctypes.c_double
            lib.oracle_brute_through_f64.argtypes = ([_F64P] + [ctypes.c_int] * 6
                                                     + [_I32P, _I32P,
                                                        ctypes.POINTER(ctypes.c_long)])
            lib.oracle_brute_through_f64.restype = ctypes.c_double
            lib.oracle_detect_two_f64.argtypes = ([_F64P] + [ctypes.c_int] * 5
                                                  + [_I32P, _I32P, _F64P])
            lib.oracle_brute_apart_f64.argtypes = ([_F64P] + [ctypes.c_int] * 6
                                                   + [_I32P, _I32P])
            lib.oracle_brute_apart_f64.restype = ctypes.c_double
            lib.oracle_path_score_padded_f64.argtypes = [_F64P] + [ctypes.c_int] * 4 + [_I32P]
            lib.oracle_path_score_padded_f64.restype = ctypes.c_double
            lib.oracle_detect_padded_f64.argtypes = [_F64P] + [ctypes.c_int] * 4 + [_I32P, _I32P]
            lib.oracle_detect_padded_f64.restype = ctypes.c_double
            lib.oracle_brute_padded_f64.argtypes = ([_F64P] + [ctypes.c_int] * 4
                                                    + [_I32P, _I32P,
                                                       ctypes.POINTER(ctypes.c_long)])
            lib.oracle_brute_padded_f64.restype = ctypes.c_double
            lib.oracle_detect_angle_through_f64.argtypes = ([_F64P] + [ctypes.c_int] * 4
                                                            + [ctypes.c_double, ctypes.c_int,
                                                               ctypes.c_int, _I32P, _I32P])
            lib.oracle_detect_angle_through_f64.restype = ctypes.c_double
            lib.oracle_brute_angle_through_f64.argtypes = ([_F64P] + [ctypes.c_int] * 3
                                                           + [ctypes.c_double, ctypes.c_int,
                                                              ctypes.c_int, _I32P, _I32P])
            lib.oracle_brute_angle_through_f64.restype = ctypes.c_double
            lib.oracle_gauss_rows_f32.argtypes = [_F32P] + [ctypes.c_int] * 3 + [_F32P]
            lib.oracle_detect_angle_f32.argtypes = ([_F32P] + [ctypes.c_int] * 4
                                                    + [ctypes.c_double, _I32P, _I32P])
            lib.oracle_detect_angle_f32.restype = ctypes.c_double
            lib.oracle_detect_angle_through_f32.argtypes = ([_F32P] + [ctypes.c_int] * 4
                                                            + [ctypes.c_double, ctypes.c_int,
                                                               ctypes.c_int, _I32P, _I32P])
            lib.oracle_detect_angle_through_f32.restype = ctypes.c_double
            lib.oracle_detect_through_f32.argtypes = ([_F32P] + [ctypes.c_int] * 6
                                                      + [_I32P, _I32P])
            lib.oracle_detect_through_f32.restype = ctypes.c_double
            lib.oracle_detect_padded_f32.argtypes = [_F32P] + [ctypes.c_int] * 4 + [_I32P, _I32P]
            lib.oracle_detect_padded_f32.restype = ctypes.c_double
            lib.oracle_detect_two_f32.argtypes = ([_F32P] + [ctypes.c_int] * 5
                                                  + [_I32P, _I32P, _F64P])
            _lib = lib
    return _lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(img) -> np.ndarray:
    return np.ascontiguousarray(img, dtype=np.float64)


def _band_rows(img, k):
    h, w = img.shape
    if k < 1 or h % k:
        raise ValueError("h must be a multiple of k")
    n = h // k
    if n & (n - 1):
        raise ValueError("h/k must be a power of two")
    return h, w, n


def off_table(n: int) -> np.ndarray:
    """[n][n] int32: off[s, y] = column offset of the shift-s line on row y."""
    out = np.zeros((n, n), dtype=np.int32)
    if _load().oracle_off_table(n, _p(out, ctypes.c_int32)) != 0:
        raise ValueError("n must be a power of two")
    return out


def fht_direct(img, k: int) -> np.ndarray:
    """[k][2][n][W] float64 Hough images by direct summation (cyclic in W)."""
    img = _f64(img)
    h, w, n = _band_rows(img, k)
    H = np.empty((k, 2, n, w + n), dtype=np.float64)
    _load().oracle_fht_direct_f64(_p(img, ctypes.c_double), h, w, k, _p(H, ctypes.c_double))
    return H


def fht_recursive(img, k: int, dtype=np.float64) -> np.ndarray:
    """[k][2][n][W] Hough images by the dyadic recursion, in float64 or in
    float32 (the float32 summation tree the CUDA float path follows)."""
    dtype = np.dtype(dtype)
    src = np.ascontiguousarray(img, dtype=dtype)
    h, w, n = _band_rows(src, k)
    H = np.empty((k, 2, n, w + n), dtype=dtype)
    lib = _load()
    if dtype == np.float64:
        lib.oracle_fht_recursive_f64(_p(src, ctypes.c_double), h, w, k, _p(H, ctypes.c_double))
    elif dtype == np.float32:
        lib.oracle_fht_recursive_f32(_p(src, ctypes.c_float), h, w, k, _p(H, ctypes.c_float))
    else:
        raise TypeError("float64 or float32")
    return H


def dp(H: np.ndarray, h: int, w: int, k: int, B: int) -> np.ndarray:
    """[k][2n-1][w] DP values from Hough images (float64 or float32)."""
    n = h // k
    V = np.empty((k, 2 * n - 1, w), dtype=H.dtype)
    H = np.ascontiguousarray(H)
    lib = _load()
    if H.dtype == np.float64:
        lib.oracle_dp_f64(_p(H, ctypes.c_double), h, w, k, B, _p(V, ctypes.c_double))
    elif H.dtype == np.float32:
        lib.oracle_dp_f32(_p(H, ctypes.c_float), h, w, k, B, _p(V, ctypes.c_float))
    else:
        raise TypeError("float64 or float32")
    return V


def backtrack(V: np.ndarray, h: int, w: int, k: int, B: int):
    """(x[k+1], d[k], score) read back from the DP values."""
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    V = np.ascontiguousarray(V)
    lib = _load()
    if V.dtype == np.float64:
        s = lib.oracle_backtrack_f64(_p(V, ctypes.c_double), h, w, k, B,
                                     _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    else:
        s = lib.oracle_backtrack_f32(_p(V, ctypes.c_float), h, w, k, B,
                                     _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def path_score(img, k: int, x0: int, ds) -> float:
    """Sum of the pixels along the polyline (x0, d_0..d_{k-1}), float64;
    -inf if it is not admissible."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    d = np.ascontiguousarray(ds, dtype=np.int32)
    return _load().oracle_path_score_f64(_p(img, ctypes.c_double), h, w, k, int(x0),
                                         _p(d, ctypes.c_int32))


def brute(img, k: int, B: int):
    """(x, d, score, visited) of the lexicographically smallest optimum over
    every admissible polyline.  Tiny images only."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    visited = ctypes.c_long(0)
    s = _load().oracle_brute_f64(_p(img, ctypes.c_double), h, w, k, B,
                                 _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32),
                                 ctypes.byref(visited))
    return xs, ds, s, visited.value


def detect(img, k: int, B: int):
    """The whole method in float64: (x[k+1], d[k], score)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_f64(_p(img, ctypes.c_double), h, w, k, B,
                                  _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def detect_windowed(img, k: int, B: int, win):
    """The method restricted to per-band displacement windows win[k][2]
    (the pruned DP of the learned proposal): (x, d, score); x = -1 and score
    -inf when no admissible polyline lies inside the windows."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    wn = np.ascontiguousarray(win, dtype=np.int32).reshape(k, 2)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_win_f64(_p(img, ctypes.c_double), h, w, k, B,
                                      _p(wn, ctypes.c_int32), _p(xs, ctypes.c_int32),
                                      _p(ds, ctypes.c_int32))
    return xs, ds, s


def brute_windowed(img, k: int, B: int, win):
    """Brute force over the admissible polylines inside the windows."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    wn = np.ascontiguousarray(win, dtype=np.int32).reshape(k, 2)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    visited = ctypes.c_long(0)
    s = _load().oracle_brute_win_f64(_p(img, ctypes.c_double), h, w, k, B,
                                     _p(wn, ctypes.c_int32), _p(xs, ctypes.c_int32),
                                     _p(ds, ctypes.c_int32), ctypes.byref(visited))
    return xs, ds, s, visited.value


def detect_f32(img, k: int, B: int):
    """The whole method with float32 arithmetic and decisions (the decisions
    the float path of the library must reproduce): (x, d, score)."""
    src = np.ascontiguousarray(img, dtype=np.float32)
    h, w, _ = _band_rows(src, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_f32(_p(src, ctypes.c_float), h, w, k, B,
                                  _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def gauss_rows(img, r: int) -> np.ndarray:
    """Every row convolved with the binomial weights C(2r, r+t), |t| <= r,
    zero outside the row (unnormalised), float64."""
    img = _f64(img)
    h, w = img.shape
    out = np.empty_like(img)
    if _load().oracle_gauss_rows_f64(_p(img, ctypes.c_double), h, w, int(r),
                                     _p(out, ctypes.c_double)):
        raise ValueError("r must be >= 0")
    return out


def angle_window(n: int, gamma: float) -> np.ndarray:
    """[2n-1][2] int32: the range [lo(d), hi(d)] of next displacements whose
    bend angle from d is at most gamma (Eqs. 6-7), row d + n - 1."""
    out = np.zeros((2 * n - 1, 2), dtype=np.int32)
    if _load().oracle_angle_window(int(n), float(gamma), _p(out, ctypes.c_int32)):
        raise ValueError("n >= 1 and gamma >= 0 required")
    return out


def dp_angle(H: np.ndarray, h: int, w: int, k: int, lohi) -> np.ndarray:
    """V[k][2n-1][w] of the angle-restricted DP over Hough images H."""
    n = h // k
    H = np.ascontiguousarray(H, dtype=np.float64)
    t = np.ascontiguousarray(lohi, dtype=np.int32)
    V = np.empty((k, 2 * n - 1, w), dtype=np.float64)
    if _load().oracle_dp_angle_f64(_p(H, ctypes.c_double), h, w, k, _p(t, ctypes.c_int32),
                                   _p(V, ctypes.c_double)):
        raise ValueError("bad shape")
    return V


def backtrack_angle(V: np.ndarray, h: int, w: int, k: int, lohi):
    """(x[k+1], d[k], score) read back from V with the angle windows."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    t = np.ascontiguousarray(lohi, dtype=np.int32)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_backtrack_angle_f64(_p(V, ctypes.c_double), h, w, k,
                                           _p(t, ctypes.c_int32), _p(xs, ctypes.c_int32),
                                           _p(ds, ctypes.c_int32))
    return xs, ds, s


def brute_angle(img, k: int, gamma: float):
    """Brute force over every polyline whose bend angles pass the direct
    test |atan(d'/n) - atan(d/n)| <= gamma: (x, d, score, visited)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    visited = ctypes.c_long(0)
    s = _load().oracle_brute_angle_f64(_p(img, ctypes.c_double), h, w, k, float(gamma),
                                       _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32),
                                       ctypes.byref(visited))
    return xs, ds, s, visited.value


def detect_angle(img, k: int, r: int, gamma: float):
    """The main problem in float64: Gaussian rows (half-width r), band FHT,
    angle-restricted DP, read-back.  (x[k+1], d[k], score of the smoothed
    image)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_angle_f64(_p(img, ctypes.c_double), h, w, k, int(r),
                                        float(gamma), _p(xs, ctypes.c_int32),
                                        _p(ds, ctypes.c_int32))
    return xs, ds, s


def dp_through(H: np.ndarray, h: int, w: int, k: int, B: int, j: int, xp: int) -> np.ndarray:
    """V[k][2n-1][w] of the DP whose band-j states (j = k: band k-1's end
    points) off the point xp are dead."""
    n = h // k
    H = np.ascontiguousarray(H, dtype=np.float64)
    V = np.empty((k, 2 * n - 1, w), dtype=np.float64)
    if _load().oracle_dp_through_f64(_p(H, ctypes.c_double), h, w, k, B, int(j), int(xp),
                                     _p(V, ctypes.c_double)):
        raise ValueError("bad shape, point or bend")
    return V


def detect_through(img, k: int, B: int, j: int, xp: int):
    """The extreme polyline through (xp, j*n): (x[k+1], d[k], score)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    if not (0 <= j <= k and 0 <= xp < w):
        raise ValueError("point outside the image")
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_through_f64(_p(img, ctypes.c_double), h, w, k, B, int(j),
                                          int(xp), _p(xs, ctypes.c_int32),
                                          _p(ds, ctypes.c_int32))
    return xs, ds, s


def brute_through(img, k: int, B: int, j: int, xp: int):
    """Brute force over the admissible polylines with x_j = xp."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    visited = ctypes.c_long(0)
    s = _load().oracle_brute_through_f64(_p(img, ctypes.c_double), h, w, k, B, int(j),
                                         int(xp), _p(xs, ctypes.c_int32),
                                         _p(ds, ctypes.c_int32), ctypes.byref(visited))
    return xs, ds, s, visited.value


def detect_two(img, k: int, B: int, sep: int):
    """The optimum and the best polyline whose top vertex is at least `sep`
    columns from the optimum's: (x[2][k+1], d[2][k], scores[2])."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros((2, k + 1), dtype=np.int32)
    ds = np.zeros((2, k), dtype=np.int32)
    sc = np.zeros(2, dtype=np.float64)
    if _load().oracle_detect_two_f64(_p(img, ctypes.c_double), h, w, k, B, int(sep),
                                     _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32),
                                     _p(sc, ctypes.c_double)):
        raise ValueError("bad shape, bend or separation")
    return xs, ds, sc


def brute_apart(img, k: int, B: int, x0: int, sep: int):
    """Brute force: the best admissible polyline with |x_0 - x0| >= sep."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_brute_apart_f64(_p(img, ctypes.c_double), h, w, k, B, int(x0), int(sep),
                                       _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def detect_horizontal(img, k: int, B: int):
    """Mostly horizontal polylines (Fig. 7): the method on the transposed
    image, whose bands are the image's vertical strips of w/k columns.
    Returns (y[k+1], d[k], score): y_i is the row of the polyline on the
    first column of strip i, d_i = y_{i+1} - y_i."""
    return detect(np.ascontiguousarray(np.asarray(img).T), k, B)


def path_score_padded(img, k: int, x0: int, ds) -> float:
    """Sum along the polyline with vertices in [0, w + n) and zeros right of
    the image; -inf if it is not admissible."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    d = np.ascontiguousarray(ds, dtype=np.int32)
    return _load().oracle_path_score_padded_f64(_p(img, ctypes.c_double), h, w, k, int(x0),
                                                _p(d, ctypes.c_int32))


def detect_padded(img, k: int, B: int):
    """The method with every vertex in [0, w + n) (the zero-padded band
    width): (x[k+1], d[k], score)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_padded_f64(_p(img, ctypes.c_double), h, w, k, B,
                                         _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def brute_padded(img, k: int, B: int):
    """Brute force with vertices in [0, w + n): (x, d, score, visited)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    visited = ctypes.c_long(0)
    s = _load().oracle_brute_padded_f64(_p(img, ctypes.c_double), h, w, k, B,
                                        _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32),
                                        ctypes.byref(visited))
    return xs, ds, s, visited.value


def detect_angle_through(img, k: int, r: int, gamma: float, j: int, xp: int):
    """Subproblem 3: the best polyline through (xp, j*n) with bend angles at
    most gamma, on the row-smoothed image: (x[k+1], d[k], score)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    if not (0 <= j <= k and 0 <= xp < w):
        raise ValueError("point outside the image")
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_angle_through_f64(_p(img, ctypes.c_double), h, w, k, int(r),
                                                float(gamma), int(j), int(xp),
                                                _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def brute_angle_through(img, k: int, gamma: float, j: int, xp: int):
    """Brute force over polylines with x_j = xp passing the direct angle
    test, on the image as given (smooth it first for r > 0)."""
    img = _f64(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_brute_angle_through_f64(_p(img, ctypes.c_double), h, w, k, float(gamma),
                                               int(j), int(xp), _p(xs, ctypes.c_int32),
                                               _p(ds, ctypes.c_int32))
    return xs, ds, s


def _f32(img) -> np.ndarray:
    return np.ascontiguousarray(img, dtype=np.float32)


def gauss_rows_f32(img, r: int) -> np.ndarray:
    """gauss_rows in float32: products and sums rounded to float, t from -r
    to r."""
    img = _f32(img)
    h, w = img.shape
    out = np.empty_like(img)
    if _load().oracle_gauss_rows_f32(_p(img, ctypes.c_float), h, w, int(r),
                                     _p(out, ctypes.c_float)):
        raise ValueError("r must be >= 0")
    return out


def detect_angle_f32(img, k: int, r: int, gamma: float):
    """The main problem on a float32 image in float32: (x, d, score)."""
    img = _f32(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_angle_f32(_p(img, ctypes.c_float), h, w, k, int(r), float(gamma),
                                        _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def detect_angle_through_f32(img, k: int, r: int, gamma: float, j: int, xp: int):
    """Subproblem 3 with the bend angle on a float32 image in float32."""
    img = _f32(img)
    h, w, _ = _band_rows(img, k)
    if not (0 <= j <= k and 0 <= xp < w):
        raise ValueError("point outside the image")
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_angle_through_f32(_p(img, ctypes.c_float), h, w, k, int(r),
                                                float(gamma), int(j), int(xp),
                                                _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def detect_through_f32(img, k: int, B: int, j: int, xp: int):
    """The extreme polyline through (xp, j*n) on a float32 image in float32."""
    img = _f32(img)
    h, w, _ = _band_rows(img, k)
    if not (0 <= j <= k and 0 <= xp < w):
        raise ValueError("point outside the image")
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_through_f32(_p(img, ctypes.c_float), h, w, k, B, int(j), int(xp),
                                          _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def detect_padded_f32(img, k: int, B: int):
    """Vertices in [0, w + n) on a float32 image in float32."""
    img = _f32(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros(k + 1, dtype=np.int32)
    ds = np.zeros(k, dtype=np.int32)
    s = _load().oracle_detect_padded_f32(_p(img, ctypes.c_float), h, w, k, B,
                                         _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32))
    return xs, ds, s


def detect_two_f32(img, k: int, B: int, sep: int):
    """Two different extreme polylines on a float32 image in float32."""
    img = _f32(img)
    h, w, _ = _band_rows(img, k)
    xs = np.zeros((2, k + 1), dtype=np.int32)
    ds = np.zeros((2, k), dtype=np.int32)
    sc = np.zeros(2, dtype=np.float64)
    if _load().oracle_detect_two_f32(_p(img, ctypes.c_float), h, w, k, B, int(sep),
                                     _p(xs, ctypes.c_int32), _p(ds, ctypes.c_int32),
                                     _p(sc, ctypes.c_double)):
        raise ValueError("bad shape, bend or separation")
    return xs, ds, sc


def detect_horizontal_f32(img, k: int, B: int):
    """Mostly horizontal polylines on a float32 image in float32: detect_f32
    on the transposed image."""
    return detect_f32(np.ascontiguousarray(np.asarray(img, dtype=np.float32).T), k, B)
