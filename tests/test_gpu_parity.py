"""GPU parity: every C-ABI call against the CPU oracle on the same seeded
inputs.  Integer images must agree bit for bit; float images must give the
same float32 Hough values and decisions as the oracle's float32 recursion
(so identical path indices) and an optimal score within a relative 1e-5 of
the oracle's float64 optimum."""
import numpy as np
import pytest

import oracle
from paper_1912_01884_gb300 import synth
from helpers import check_path, hough_from_oracle, to_device, v_to_library_layout

pytestmark = pytest.mark.gpu

REL_TOL = 1e-5
INT_DEAD = np.iinfo(np.int32).min

# (h, w, k): several tiles and ragged tails, every band height 1..256
SHAPES = [(256, 256, 4), (64, 37, 4), (128, 1000, 1), (512, 300, 2), (16, 5, 16),
          (8, 3, 4), (2048, 130, 16), (96, 77, 3), (32, 1, 2), (1024, 517, 4)]


def _img(shape, dtype, seed):
    h, w, _ = shape
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        return rng.integers(0, 256, (h, w)).astype(np.uint8)
    if dtype == "i32":
        return rng.integers(-5000, 5000, (h, w)).astype(np.int32)
    return np.abs(rng.standard_normal((h, w))).astype(np.float32) * np.float32(2.5)


@pytest.mark.parametrize("dtype", ["u8", "i32", "f32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_fht_bands_matches_oracle(lib, shape, dtype):
    h, w, k = shape
    img = _img(shape, dtype, h * 7 + w)
    H = lib.fht_bands(to_device(img), k).cpu().numpy()
    if dtype == "f32":
        Ho = hough_from_oracle(img, k, float32=True)
        assert np.array_equal(H.view(np.uint32), Ho.view(np.uint32))
    else:
        Ho = hough_from_oracle(img, k)
        assert np.array_equal(H.astype(np.float64), Ho)


def test_fht_bands_respects_pitch(lib):
    import torch
    img = _img((128, 300, 4), "u8", 3)
    big = torch.zeros((128, 320), dtype=torch.uint8, device="cuda")
    big[:, :300] = to_device(img)
    H = lib.fht_bands(big[:, :300], 4).cpu().numpy()
    assert np.array_equal(H.astype(np.float64), hough_from_oracle(img, 4))


@pytest.mark.parametrize("dtype", ["u8", "f32"])
@pytest.mark.parametrize("shape", SHAPES[:8])
@pytest.mark.parametrize("B", [0, 3, 1000])
def test_polyline_dp_and_backtrack_match_oracle(lib, shape, dtype, B):
    h, w, k = shape
    n = h // k
    img = _img(shape, dtype, h + 13 * w + B)
    H = lib.fht_bands(to_device(img), k)
    V = lib.polyline_dp(H, h, w, k, B)
    x, d, score = lib.backtrack(V, h, w, k, B)
    Vg = V.cpu().numpy()
    f32 = dtype == "f32"
    Ho = hough_from_oracle(img, k, float32=f32)
    Vo = oracle.dp(Ho, h, w, k, B)
    want = v_to_library_layout(Vo.astype(np.float64), n, w + n, -np.inf if f32 else INT_DEAD)
    if f32:
        assert np.array_equal(Vg.astype(np.float64), want)
    else:
        got = Vg.astype(np.float64)
        want = np.where(np.isneginf(want), INT_DEAD, want)
        assert np.array_equal(got, want)
    xo, do, so = oracle.backtrack(Vo, h, w, k, B)
    assert list(x.cpu().numpy()) == list(xo)
    assert list(d.cpu().numpy()) == list(do)
    assert float(score.cpu().numpy()[0]) == so


def _detect(lib, img, k, B):
    x, d, s = lib.detect_polyline(to_device(img), k, B)
    return x.cpu().numpy(), d.cpu().numpy(), s.cpu().numpy()[0]


def _assert_detect_parity(lib, img, k, B):
    x, d, s = _detect(lib, img, k, B)
    check_path(img, k, B, x, d)
    if img.dtype == np.float32:
        xo, do, so32 = oracle.detect_f32(img, k, B)
        assert list(x) == list(xo) and list(d) == list(do)
        assert np.float32(s) == np.float32(so32)
        _, _, so64 = oracle.detect(img, k, B)
        assert abs(float(s) - so64) <= REL_TOL * abs(so64)
    else:
        xo, do, so = oracle.detect(img, k, B)
        assert list(x) == list(xo) and list(d) == list(do)
        assert int(s) == int(so)
        assert oracle.path_score(img, k, x[0], d) == so


@pytest.mark.parametrize("seed", range(8))
def test_detect_256x256_u8_k4_B8(lib, seed):
    wl = synth.plain_uniform(seed, 256, 256, 4, 8)
    _assert_detect_parity(lib, wl.img, wl.k, wl.B)


@pytest.mark.parametrize("seed", range(2))
def test_detect_2048x2048_u8_k16_B16_full_size(lib, seed):
    wl = synth.plain_gaussian(seed)
    _assert_detect_parity(lib, wl.img, wl.k, wl.B)


def test_detect_1024x1024_lanes_k16_B12(lib):
    wl = synth.lane_texture(0)
    _assert_detect_parity(lib, wl.img, wl.k, wl.B)


@pytest.mark.parametrize("seed", range(2))
def test_detect_float_response_reduced(lib, seed):
    wl = synth.ridge_response(seed, 1024, 1536, 8, 24)
    _assert_detect_parity(lib, wl.img, wl.k, wl.B)


def test_detect_float_response_8192_full_size(lib):
    """Full 8192x8192 float32, k=64, B=24, against the oracle's float32
    decisions and float64 score of the chosen path."""
    wl = synth.ridge_response(0)
    x, d, s = _detect(lib, wl.img, wl.k, wl.B)
    check_path(wl.img, wl.k, wl.B, x, d)
    xo, do, so32 = oracle.detect_f32(wl.img, wl.k, wl.B)
    assert list(x) == list(xo) and list(d) == list(do)
    assert np.float32(s) == np.float32(so32)
    ps = oracle.path_score(wl.img, wl.k, x[0], d)
    assert abs(float(s) - ps) <= REL_TOL * abs(ps)


def test_detect_mixed_batch_sample(lib):
    """A sample of the mixed-size batch's images, one band height each."""
    shapes = synth.mixed_batch_shapes(0)
    picked = {}
    for j, sh in enumerate(shapes):
        n = sh[0] // sh[2]
        if n not in picked and sh[0] * sh[1] <= 2048 * 2048:
            picked[n] = (j, sh)
    for j, (h, w, k, B) in picked.values():
        wl = synth.plain_uniform(j, h, w, k, B)
        _assert_detect_parity(lib, wl.img, wl.k, wl.B)


@pytest.mark.parametrize("h,w,k,B", [
    (64, 50, 1, 0),        # one band: best single line
    (16, 40, 16, 2),       # one-row bands: vertical lines only
    (64, 1, 4, 3),         # a one-pixel-wide image
    (128, 90, 4, 0),       # straight polylines only
    (128, 90, 4, 254),     # unrestricted (B = 2n-2)
    (128, 90, 4, 100000),  # beyond unrestricted
    (512, 700, 2, 32),     # 256-row bands
    (256, 4099, 2, 17),    # ragged width
])
def test_detect_edge_cases(lib, h, w, k, B):
    # int32 images with negative pixels: a link leaving the image can sum
    # more (zeros of the padding) than any admissible one, so the read-back
    # must reject it in every band
    for dtype in ("u8", "i32", "f32"):
        img = _img((h, w, k), dtype, h + w + k + B)
        _assert_detect_parity(lib, img, k, B)


def test_detect_planted_polyline_is_recovered(lib):
    """Exact recovery through the library: a polyline drawn with the FHT's
    own line pattern at 200 over noise <= 40 is the unique optimum."""
    h, w, k, B = 512, 700, 8, 6
    n = h // k
    rng = synth.Rng(5, 77)
    img = rng.ints(h * w, 0, 40).reshape(h, w).astype(np.uint8)
    xs, ds = synth.random_polyline(rng, h, w, k, B)
    off = oracle.off_table(n)
    for i, dd in enumerate(ds):
        for y in range(n):
            img[i * n + y, xs[i] + np.sign(dd) * off[abs(int(dd)), y]] = 200
    x, d, s = _detect(lib, img, k, B)
    assert int(s) == 200 * h and list(x) == list(xs) and list(d) == list(ds)


def test_detect_is_repeatable_with_a_reused_workspace(lib):
    import torch
    wl = synth.plain_uniform(3, 256, 256, 4, 8)
    dimg = to_device(wl.img)
    ws = torch.empty(lib.workspace_bytes(0, 256, 256, 4, 8), dtype=torch.uint8, device="cuda")
    first = [t.cpu().numpy().copy() for t in lib.detect_polyline(dimg, 4, 8, ws=ws)]
    ws.fill_(0xAB)
    second = [t.cpu().numpy() for t in lib.detect_polyline(dimg, 4, 8, ws=ws)]
    for a, b in zip(first, second):
        assert np.array_equal(a, b)


def test_detect_rejects_bad_arguments_on_device(lib):
    import torch
    img = torch.zeros((100, 10), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.FhtdpError) as e:
        lib.detect_polyline(img, 3, 1)
    assert e.value.code == 1
    img = torch.zeros((64, 10), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.FhtdpError) as e:
        lib.detect_polyline(img, 4, 1, ws=torch.empty(8, dtype=torch.uint8, device="cuda"))
    assert e.value.code == 2


# --------------------------------------------------------------------------
# Batches: one persistent launch over many images of different shapes
# --------------------------------------------------------------------------
def _batch_parity(lib, wls):
    imgs = [to_device(wl.img) for wl in wls]
    plan = lib.BatchPlan(imgs, [wl.k for wl in wls], [wl.B for wl in wls])
    plan.run()
    _check_batch(plan, wls)
    return plan


def _check_batch(plan, wls):
    plan.status()
    for i, wl in enumerate(wls):
        x = plan.x[i].cpu().numpy()
        d = plan.d[i].cpu().numpy()
        s = plan.score[i].cpu().numpy()[0]
        check_path(wl.img, wl.k, wl.B, x, d)
        if wl.img.dtype == np.float32:
            xo, do, so = oracle.detect_f32(wl.img, wl.k, wl.B)
            assert np.float32(s) == np.float32(so), i
        else:
            xo, do, so = oracle.detect(wl.img, wl.k, wl.B)
            assert int(s) == int(so), i
        assert list(x) == list(xo) and list(d) == list(do), i


def test_batch_of_mixed_shapes_matches_oracle(lib):
    shapes = [(256, 256, 4, 8), (512, 300, 8, 4), (1024, 130, 16, 12), (128, 1000, 1, 0),
              (64, 37, 4, 100), (16, 5, 16, 2), (768, 512, 6, 16), (2048, 77, 32, 3)]
    wls = [synth.plain_uniform(40 + j, h, w, k, B) for j, (h, w, k, B) in enumerate(shapes)]
    plan = _batch_parity(lib, wls)
    # a second run of the same plan gives the same results
    first = [t.clone() for t in plan.x]
    plan.run()
    for a, b in zip(first, plan.x):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_batch_autotune_keeps_exact_results(lib):
    """The queue tuner times a few group widths and keeps one; the batch it
    leaves behind gives the oracle's results, also with a 256-row-band image
    (side stream) in the batch."""
    shapes = [(256, 256, 4, 8), (512, 300, 8, 4), (1024, 130, 16, 12), (768, 512, 6, 16),
              (512, 700, 2, 32), (2048, 77, 32, 3)]
    wls = [synth.plain_uniform(70 + j, h, w, k, B) for j, (h, w, k, B) in enumerate(shapes)]
    imgs = [to_device(wl.img) for wl in wls]
    plan = lib.BatchPlan(imgs, [wl.k for wl in wls], [wl.B for wl in wls])
    width = plan.autotune(reps=1)
    assert width >= 1
    _check_batch(plan, wls)   # outputs of the tuner's last run
    for t in plan.x:
        t.fill_(-7)
    plan.run()
    _check_batch(plan, wls)


def test_batch_of_float_images_matches_oracle(lib):
    wls = [synth.ridge_response(60 + j, 256 * (1 + j % 3), 200 + 96 * j, 2 * (1 + j % 3), 6)
           for j in range(5)]
    _batch_parity(lib, wls)


def test_batch_mixed_sizes_sample_up_to_128_row_bands(lib):
    """The mixed-size batch (h 512..4096, w 512..3072, n 32..128, B = n/8):
    every image through one launch, checked against the oracle."""
    shapes = [s for s in synth.mixed_batch_shapes(0) if s[0] // s[2] <= 128][:24]
    wls = [synth.plain_uniform(j, h, w, k, B) for j, (h, w, k, B) in enumerate(shapes)]
    _batch_parity(lib, wls)


def test_batch_run_is_captured_in_a_cuda_graph(lib):
    import torch
    wls = [synth.plain_uniform(70 + j, 256, 256 + 64 * j, 4, 8) for j in range(4)]
    imgs = [to_device(wl.img) for wl in wls]
    plan = lib.BatchPlan(imgs, [4] * 4, [8] * 4)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.run(stream=stream)
    for t in plan.x + plan.d + plan.score:
        t.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    for i, wl in enumerate(wls):
        xo, do, so = oracle.detect(wl.img, 4, 8)
        assert list(plan.x[i].cpu().numpy()) == list(xo)
        assert list(plan.d[i].cpu().numpy()) == list(do)
        assert int(plan.score[i].cpu().numpy()[0]) == int(so)


def test_batch_mixed_sizes_including_256_row_bands(lib):
    """Mixed-size batch images of every band height (32..256) in one run."""
    shapes = [s for s in synth.mixed_batch_shapes(1) if s[0] * s[1] <= 1536 * 1024]
    by_n = {}
    for s in shapes:
        by_n.setdefault(s[0] // s[2], []).append(s)
    picked = [s for n in sorted(by_n) for s in by_n[n][:3]]
    assert any(s[0] // s[2] == 256 for s in picked)
    wls = [synth.plain_uniform(100 + j, h, w, k, B) for j, (h, w, k, B) in enumerate(picked)]
    _batch_parity(lib, wls)


@pytest.mark.parametrize("shape", [(512, 300, 2), (256, 256, 4), (96, 77, 3)])
def test_huge_bend_limit_equals_the_unrestricted_dp(lib, shape):
    """B = 2^31 - 1 admits every continuation, like B = 2n - 2, on the
    standalone calls (256-row bands included) and the fused engine."""
    h, w, k = shape
    n = h // k
    img = _img(shape, "u8", 5 * h + w)
    big = 2**31 - 1
    x, d, s = lib.detect_polyline(to_device(img), k, big)
    xr, dr, sr = lib.detect_polyline(to_device(img), k, 2 * n - 2)
    assert list(x.cpu().numpy()) == list(xr.cpu().numpy()) and int(s.cpu()[0]) == int(sr.cpu()[0])
    H = lib.fht_bands(to_device(img), k)
    V = lib.polyline_dp(H, h, w, k, big)
    xb, db, sb = lib.backtrack(V, h, w, k, big)
    xo, do, so = oracle.detect(img, k, 2 * n - 2)
    assert list(xb.cpu().numpy()) == list(xo) and list(db.cpu().numpy()) == list(do)
    assert int(sb.cpu().numpy()[0]) == int(so)


# --------------------------------------------------------------------------
# 256-row bands in the fused engine: half-band FHT items + 64-column DP
# items (uint8 rows 16-byte aligned, B <= 127); the rest take the standalone
# kernels.
# --------------------------------------------------------------------------
def _padded_device(img, pitch):
    """A device view of img whose rows are `pitch` bytes apart."""
    import torch
    h, w = img.shape
    buf = torch.zeros((h, pitch), dtype=torch.uint8, device="cuda")
    buf[:, :w] = torch.from_numpy(np.ascontiguousarray(img)).cuda()
    return buf[:, :w]


@pytest.mark.parametrize("h,w,pitch,k,B", [
    (512, 704, 704, 2, 32),     # config-3 bend (n/8)
    (256, 64, 64, 1, 0),        # one band, one DP tile
    (256, 1, 16, 1, 5),         # a one-pixel-wide image
    (768, 1000, 1008, 3, 127),  # largest fused bend; ragged width
    (1024, 300, 304, 4, 16),
    (256, 130, 144, 1, 3),      # one band over two half-band tiles
    (512, 200, 208, 2, 1),
])
def test_detect_256_row_bands_fused(lib, h, w, pitch, k, B):
    img = np.random.default_rng(h + w + B).integers(0, 256, (h, w)).astype(np.uint8)
    x, d, s = lib.detect_polyline(_padded_device(img, pitch), k, B)
    x, d, s = x.cpu().numpy(), d.cpu().numpy(), s.cpu().numpy()[0]
    check_path(img, k, B, x, d)
    xo, do, so = oracle.detect(img, k, B)
    assert list(x) == list(xo) and list(d) == list(do) and int(s) == int(so)


def test_detect_256_row_bands_planted_polyline(lib):
    """Exact recovery with 256-row bands (the FHT's own line pattern at 200
    over noise <= 40), bends up to 32."""
    h, w, k, B = 1024, 512, 4, 32
    n = h // k
    rng = synth.Rng(9, 77)
    img = rng.ints(h * w, 0, 40).reshape(h, w).astype(np.uint8)
    xs, ds = synth.random_polyline(rng, h, w, k, B)
    off = oracle.off_table(n)
    for i, dd in enumerate(ds):
        for y in range(n):
            img[i * n + y, xs[i] + np.sign(dd) * off[abs(int(dd)), y]] = 200
    x, d, s = _detect(lib, img, k, B)
    assert int(s) == 200 * h and list(x) == list(xs) and list(d) == list(ds)


def test_batch_of_256_row_bands_runs_in_one_launch(lib):
    """A batch of 256-row-band images (and shorter bands) runs as one
    persistent launch, with no standalone kernel beside it."""
    import torch
    shapes = [(512, 512, 2, 32), (1024, 768, 4, 32), (256, 256, 1, 8), (768, 1024, 3, 127),
              (512, 640, 4, 16), (256, 512, 8, 4)]
    wls = [synth.plain_uniform(300 + j, h, w, k, B) for j, (h, w, k, B) in enumerate(shapes)]
    imgs = [to_device(wl.img) for wl in wls]
    plan = lib.BatchPlan(imgs, [wl.k for wl in wls], [wl.B for wl in wls])
    torch.cuda.synchronize()
    l0 = lib.launch_count()
    plan.run()
    torch.cuda.synchronize()
    assert lib.launch_count() - l0 == 1
    _check_batch(plan, wls)
    plan.run()
    _check_batch(plan, wls)


def test_batch_every_tile_width_and_register_depth_is_exact(lib):
    """Every per-band-height choice the tuner can make (tile width 128 or
    256 columns, 2 or 3 FHT levels in registers; 256-row bands: the depth of
    their halves) gives the oracle's results."""
    # widths that are multiples of 16 take the TMA strip (where the register
    # depth applies); 700 takes plain loads
    shapes = [(512, 704, 16, 4), (512, 304, 8, 8), (1024, 528, 8, 16), (512, 256, 2, 32),
              (256, 272, 32, 1), (256, 208, 64, 1), (512, 700, 16, 3)]
    wls = [synth.plain_uniform(400 + j, h, w, k, B) for j, (h, w, k, B) in enumerate(shapes)]
    imgs = [to_device(wl.img) for wl in wls]
    plan = lib.BatchPlan(imgs, [wl.k for wl in wls], [wl.B for wl in wls])
    variants = {32: [(128, 2), (128, 3), (256, 2), (256, 3)],
                64: [(128, 2), (128, 3), (256, 2), (256, 3)],
                128: [(128, 2), (128, 3)], 256: [(64, 2), (64, 3)],
                8: [(128, 2), (128, 3), (256, 3)], 4: [(128, 2), (256, 2)]}
    for n, choices in variants.items():
        for tile, depth in choices:
            plan.configure(n, tile, depth)
            assert plan.choice(n)["tile"] == tile and plan.choice(n)["depth"] == depth
            for t in plan.x:
                t.fill_(-7)
            plan.run()
            _check_batch(plan, wls)
    with pytest.raises(lib.FhtdpError):
        plan.configure(128, 256, 3)   # 128-row bands do not fit 256 columns
    with pytest.raises(lib.FhtdpError):
        plan.configure(4, 128, 3)     # 4-row bands have only 2 register levels
