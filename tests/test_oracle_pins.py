"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
independently of the oracle's own code: hand-worked tables and examples,
closed forms, invariants, special cases and brute force."""
import os

import numpy as np
import pytest

import oracle
from paper_1912_01884_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Dyadic line pattern (Sec. 2.1, refs [10], [34])
# --------------------------------------------------------------------------
def test_off_tables_match_hand_tables():
    with open(os.path.join(GOLDEN, "off_tables.txt")) as f:
        rows = [l.split(":") for l in f if l.strip() and not l.startswith("#")]
    for head, vals in rows:
        n, s = map(int, head.split())
        want = [int(v) for v in vals.split()]
        assert list(oracle.off_table(n)[s]) == want, (n, s)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 128, 256])
def test_off_table_properties(n):
    off = oracle.off_table(n).astype(np.int64)
    s = np.arange(n)[:, None]
    y = np.arange(n)[None, :]
    assert np.all(off[:, 0] == 0)                       # starts at the band's top vertex
    assert np.all(off[:, -1] == np.arange(n))           # ends s columns to the right
    steps = np.diff(off, axis=1)
    assert np.all((steps == 0) | (steps == 1))          # 8-connected, mostly vertical
    assert np.all(off[:, ::-1] == s - off)              # central symmetry of a straight line
    if n > 1:                                           # close to the ideal straight line
        dev = np.abs(off - s * y / (n - 1)).max()
        assert dev <= np.log2(n) / 6 + 1e-9


# --------------------------------------------------------------------------
# Hough images (Sec. 2.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("fht", ["direct", "recursive"])
@pytest.mark.parametrize("h,w,k,y0,x0", [(8, 5, 1, 3, 2), (16, 7, 2, 5, 0),
                                          (32, 9, 2, 15, 8), (4, 3, 4, 0, 1)])
def test_single_lit_pixel_closed_form(fht, h, w, k, y0, x0):
    """One lit pixel at (row b*n + y0, column x0): the "+" image of band b
    is 1 exactly where x + off_s(y0) = x0 (mod W), the "-" image where
    x - off_s(y0) = x0 (mod W); every other band is zero."""
    n = h // k
    W = w + n
    b = k - 1
    img = np.zeros((h, w))
    img[b * n + y0, x0] = 1.0
    H = oracle.fht_direct(img, k) if fht == "direct" else oracle.fht_recursive(img, k)
    off = oracle.off_table(n)
    want = np.zeros_like(H)
    for s in range(n):
        want[b, 0, s, (x0 - off[s, y0]) % W] = 1.0
        want[b, 1, s, (x0 + off[s, y0]) % W] = 1.0
    assert np.array_equal(H, want)


@pytest.mark.parametrize("seed", range(3))
def test_fht_invariants_and_two_definitions_agree(seed):
    rng = np.random.default_rng(seed)
    h, w, k = 64, 23, 4
    n, W = h // k, w + h // k
    img = rng.integers(0, 256, (h, w)).astype(np.float64)
    Hd = oracle.fht_direct(img, k)
    Hr = oracle.fht_recursive(img, k)
    assert np.array_equal(Hd, Hr)                       # exact for integers
    band_tot = img.reshape(k, n, w).sum(axis=(1, 2))
    # every shift row of each half sums to the band total (cyclic FHT)
    assert np.array_equal(Hd.sum(axis=3), np.broadcast_to(band_tot[:, None, None], (k, 2, n)))
    # shift 0 is the vertical line, identical for both signs: column sums
    colsum = np.zeros((k, W))
    colsum[:, :w] = img.reshape(k, n, w).sum(axis=1)
    assert np.array_equal(Hd[:, 0, 0], colsum)
    assert np.array_equal(Hd[:, 1, 0], colsum)
    # the shift-(n-1) "+" line is the 45-degree diagonal
    x = 3
    diag = sum(img[y, x + y] for y in range(n))
    assert Hd[0, 0, n - 1, x] == diag


def test_fht_matches_hand_example():
    img, hough, _ = _read_hand()
    H = oracle.fht_direct(img, 2)
    for (b, sg, s), vals in hough.items():
        assert list(H[b, sg, s]) == vals, (b, sg, s)
    assert np.array_equal(oracle.fht_recursive(img, 2), H)


def test_float32_recursion_is_the_pairwise_tree_along_each_line():
    """In float32 the recursion must add (top half) + (bottom half) at every
    level, i.e. a balanced pairwise sum along each line in row order."""
    rng = np.random.default_rng(7)
    h, w, k = 32, 11, 2
    n, W = h // k, w + h // k
    img = np.abs(rng.standard_normal((h, w))).astype(np.float32) * np.float32(3.7)
    H = oracle.fht_recursive(img, k, np.float32)
    off = oracle.off_table(n)
    pad = np.zeros((h, W), dtype=np.float32)
    pad[:, :w] = img
    for b in range(k):
        for sg, sgn in ((0, 1), (1, -1)):
            for s in range(n):
                for x in range(W):
                    v = pad[b * n + np.arange(n), (x + sgn * off[s]) % W].astype(np.float32)
                    while v.size > 1:
                        v = (v[0::2] + v[1::2]).astype(np.float32)
                    assert H[b, sg, s, x].view(np.uint32) == v[0].view(np.uint32)


# --------------------------------------------------------------------------
# DP + read-back (Sec. 2.2-2.3, Eqs. 3-5) against brute force
# --------------------------------------------------------------------------
def _read_hand():
    img_rows, hough, best = [], {}, {}
    with open(os.path.join(GOLDEN, "hand_4x3.txt")) as f:
        lines = [l.strip() for l in f if l.strip() and not l.startswith("#")]
    it = iter(lines)
    for l in it:
        if l.startswith("image"):
            _, hh, ww = l.split()
            for _ in range(int(hh)):
                img_rows.append([float(v) for v in next(it).split()])
        elif l.startswith("hough"):
            head, vals = l.split("=")
            _, b, sg, s = head.split()
            hough[(int(b), 0 if sg == "+" else 1, int(s))] = [float(v) for v in vals.split()]
        elif l.startswith("best"):
            kv = dict(t.split("=") for t in l.split()[1:])
            best[int(kv["B"])] = (float(kv["score"]), [int(v) for v in kv["x"].split(",")],
                                  [int(v) for v in kv["d"].split(",")])
    return np.array(img_rows), hough, best


def test_hand_example_optimum():
    img, _, best = _read_hand()
    for B, (score, xs, ds) in best.items():
        x, d, s = oracle.detect(img, 2, B)
        assert (s, list(x), list(d)) == (score, xs, ds), B
        x, d, s, _ = oracle.brute(img, 2, B)
        assert (s, list(x), list(d)) == (score, xs, ds), B


@pytest.mark.parametrize("h,w,k", [(4, 5, 2), (8, 6, 2), (8, 5, 4), (12, 6, 3),
                                   (16, 7, 4), (16, 8, 2), (8, 4, 1), (4, 6, 4)])
@pytest.mark.parametrize("seed", range(3))
def test_dp_backtrack_equals_brute_force(h, w, k, seed):
    """Every bend range from B=0 to beyond 2n-2; small value range so that
    ties are frequent and the lexicographic rule is exercised."""
    n = h // k
    rng = np.random.default_rng(1000 * seed + h * 31 + w)
    img = rng.integers(0, 4, (h, w)).astype(np.float64)
    for B in range(0, 2 * n + 1):
        xb, db, sb, visited = oracle.brute(img, k, B)
        assert visited > 0
        x, d, s = oracle.detect(img, k, B)
        assert s == sb and list(x) == list(xb) and list(d) == list(db), (B, x, d, xb, db)
        assert oracle.path_score(img, k, x[0], d) == s


def test_k1_is_global_max_of_one_hough_image():
    rng = np.random.default_rng(3)
    h, w = 16, 9
    img = rng.integers(0, 50, (h, w)).astype(np.float64)
    H = oracle.fht_direct(img, 1)
    best, arg = -np.inf, None
    for x in range(w):
        for d in range(-(h - 1), h):
            if 0 <= x + d < w:
                v = H[0, 0, d, x] if d >= 0 else H[0, 1, -d, x]
                if v > best:
                    best, arg = v, (x, d)
    x, d, s = oracle.detect(img, 1, 0)
    assert s == best and (x[0], d[0]) == arg and x[1] == arg[0] + arg[1]


def test_unrestricted_bend_is_the_column_maximum_dp_of_subproblem_2():
    """B >= 2n-2: each step takes the whole Hough column's maximum (Sec. 2.2,
    ArgMax_i and Eqs. 3-4), written here with a column max instead of a
    window."""
    rng = np.random.default_rng(4)
    h, w, k = 32, 13, 4
    n = h // k
    img = rng.integers(0, 100, (h, w)).astype(np.float64)
    H = oracle.fht_direct(img, k)

    def hv(b, x, d):
        return H[b, 0, d, x] if d >= 0 else H[b, 1, -d, x]

    colmax = None
    for b in range(k - 1, -1, -1):
        V = np.full((2 * n - 1, w), -np.inf)
        for d in range(-(n - 1), n):
            for x in range(w):
                if 0 <= x + d < w:
                    V[d + n - 1, x] = hv(b, x, d) + (0 if colmax is None else colmax[x + d])
        colmax = V.max(axis=0)
    for B in (2 * n - 2, 2 * n + 5):
        _, _, s = oracle.detect(img, k, B)
        assert s == V.max()


def test_zero_bend_is_the_best_straight_polyline():
    rng = np.random.default_rng(5)
    h, w, k = 32, 17, 4
    n = h // k
    img = rng.integers(0, 100, (h, w)).astype(np.float64)
    best = -np.inf
    for x0 in range(w):
        for d in range(-(n - 1), n):
            best = max(best, oracle.path_score(img, k, x0, [d] * k))
    x, d, s = oracle.detect(img, k, 0)
    assert s == best and len(set(d.tolist())) == 1


def test_one_row_bands_give_the_brightest_column():
    rng = np.random.default_rng(6)
    img = rng.integers(0, 100, (8, 11)).astype(np.float64)
    x, d, s = oracle.detect(img, 8, 3)
    col = img.sum(axis=0)
    assert s == col.max() and list(d) == [0] * 8 and x[0] == int(np.argmax(col))


@pytest.mark.parametrize("seed", range(6))
def test_exact_recovery_of_a_planted_polyline(seed):
    """A polyline drawn with the FHT's own line pattern, brightness 200 over
    noise <= 40: every other polyline loses at least one link row to the
    noise, so it scores <= 200(h-1) + 40 < 200h; the planted one is the
    unique optimum whenever its bends respect B."""
    h, w, k, B = 64, 40, 4, 3
    n = h // k
    rng = synth.Rng(seed, 99)
    img = rng.ints(h * w, 0, 40).reshape(h, w).astype(np.float64)
    xs, ds = synth.random_polyline(rng, h, w, k, B)
    off = oracle.off_table(n)
    for i, d in enumerate(ds):
        s = abs(int(d))
        for y in range(n):
            img[i * n + y, xs[i] + np.sign(d) * off[s, y]] = 200
    x, d, s = oracle.detect(img, k, B)
    assert s == 200 * h
    assert list(x) == list(xs) and list(d) == list(ds)


@pytest.mark.parametrize("seed", range(3))
def test_float32_decisions_score_within_tolerance_of_float64(seed):
    wl = synth.ridge_response(seed, 128, 96, 4, 6, lines=2)
    x64, d64, s64 = oracle.detect(wl.img, wl.k, wl.B)
    x32, d32, s32 = oracle.detect_f32(wl.img, wl.k, wl.B)
    assert abs(s32 - s64) <= 1e-5 * abs(s64)
    # the float32 choice is optimal to within the tolerance in exact arithmetic
    assert abs(oracle.path_score(wl.img, wl.k, x32[0], d32) - s64) <= 1e-5 * abs(s64)


@pytest.mark.parametrize("seed", range(4))
def test_windowed_dp_equals_windowed_brute_force(seed):
    """The DP restricted to per-band displacement windows (the pruned DP of
    the learned proposal) against brute force over the polylines inside the
    windows, including windows that leave no admissible polyline."""
    rng = np.random.default_rng(50 + seed)
    h, w, k = 16, 7, 4
    n = h // k
    img = rng.integers(0, 4, (h, w)).astype(np.float64)
    for B in (0, 1, 3, 6):
        for _ in range(6):
            lo = rng.integers(-(n - 1), n, k)
            hi = lo + rng.integers(0, 4, k)
            win = np.stack([lo, hi], axis=1)
            xb, db, sb, _ = oracle.brute_windowed(img, k, B, win)
            x, d, s = oracle.detect_windowed(img, k, B, win)
            assert s == sb and list(x) == list(xb) and list(d) == list(db), (B, win)
            if s != -np.inf:
                assert all(win[i, 0] <= d[i] <= win[i, 1] for i in range(k))
    # the full window is the unrestricted method
    full = np.tile([-(n - 1), n - 1], (k, 1))
    assert oracle.detect_windowed(img, k, 2, full)[2] == oracle.detect(img, k, 2)[2]


def test_hand_example_queries():
    """The pencil-worked answers of the through-point, two-polyline and
    bend-angle queries on the 4x3 example (tests/golden/hand_4x3.txt)."""
    with open(os.path.join(GOLDEN, "hand_4x3.txt")) as f:
        lines = [l.strip() for l in f if l.strip() and not l.startswith("#")]
    rows = []
    it = iter(lines)
    for l in it:
        if l.startswith("image"):
            rows = [[float(v) for v in next(it).split()] for _ in range(int(l.split()[1]))]
            break
    img = np.array(rows)

    def fields(l):
        return dict(kv.split("=") for kv in l.split()[1:])

    checked = 0
    for l in lines:
        kind = l.split()[0]
        if kind not in ("through", "two", "angle"):
            continue
        f = fields(l)
        want_x = [int(v) for v in f["x"].split(",")]
        want_d = [int(v) for v in f["d"].split(",")]
        if kind == "through":
            x, d, s = oracle.detect_through(img, 2, int(f["B"]), int(f["j"]), int(f["xp"]))
        elif kind == "two":
            xs, ds, sc = oracle.detect_two(img, 2, int(f["B"]), int(f["sep"]))
            x, d, s = xs[1], ds[1], sc[1]
        else:
            x, d, s = oracle.detect_angle(img, 2, 0, float(f["gamma"]))
        assert s == float(f["score"]), l
        assert list(x) == want_x and list(d) == want_d, l
        checked += 1
    assert checked == 10
