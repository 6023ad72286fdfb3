"""GPU parity of the main problem (Sec. 2.3): the row smoothing, the DP with
bend-angle windows (Eqs. 6-7) and the read-back, through the C ABI, against
the CPU oracle on the same seeded inputs.  All arithmetic is int32 on the
GPU and exact in the oracle, so every value and every index must agree bit
for bit."""
import math

import numpy as np
import pytest

import oracle
from paper_1912_01884_gb300 import synth
from helpers import to_device, v_to_library_layout

pytestmark = pytest.mark.gpu

INT_DEAD = np.iinfo(np.int32).min
GAMMAS = [0.0, 0.1, math.radians(10), 0.3, 0.8, 2.0]

# (h, w, k): several tiles and ragged tails, band heights 1..256
SHAPES = [(256, 256, 4), (64, 37, 4), (128, 1000, 1), (512, 300, 2), (16, 5, 16),
          (8, 3, 4), (2048, 130, 16), (96, 77, 3), (32, 1, 2), (1024, 517, 4)]


def _img(h, w, dtype, seed):
    rng = np.random.default_rng(seed)
    if dtype == "u8":
        return rng.integers(0, 256, (h, w)).astype(np.uint8)
    return rng.integers(-3000, 3000, (h, w)).astype(np.int32)


def _check_angle_path(n, gamma, d):
    a = np.arctan(np.asarray(d, dtype=np.float64) / n)
    assert np.all(np.abs(np.diff(a)) <= gamma)


@pytest.mark.parametrize("dtype", ["u8", "i32"])
@pytest.mark.parametrize("h,w,r", [(7, 1, 2), (5, 1023, 1), (9, 1024, 2), (4, 1025, 5),
                                   (33, 2500, 3), (1, 17, 11), (2048, 2048, 2), (6, 40, 0)])
def test_gauss_rows_matches_oracle(lib, dtype, h, w, r):
    img = _img(h, w, dtype, h * 31 + w + r)
    if dtype == "i32" and r == 11:
        img = (img % 50).astype(np.int32)
    got = lib.gauss_rows(to_device(img), r).cpu().numpy()
    want = oracle.gauss_rows(img, r)
    assert np.array_equal(got.astype(np.float64), want)


def test_gauss_rows_respects_pitch(lib):
    import torch
    img = _img(40, 300, "u8", 5)
    big = torch.zeros((40, 333), dtype=torch.uint8, device="cuda")
    big[:, :300] = to_device(img)
    got = lib.gauss_rows(big[:, :300], 3).cpu().numpy()
    assert np.array_equal(got.astype(np.float64), oracle.gauss_rows(img, 3))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("gamma", GAMMAS)
def test_dp_angle_and_backtrack_match_oracle(lib, shape, gamma):
    h, w, k = shape
    n = h // k
    img = _img(h, w, "u8", h + 17 * w)
    H = lib.fht_bands(to_device(img), k)
    V = lib.polyline_dp_angle(H, h, w, k, gamma)
    x, d, score = lib.backtrack_angle(V, h, w, k, gamma)
    t = oracle.angle_window(n, gamma)
    Vo = oracle.dp_angle(oracle.fht_recursive(img, k), h, w, k, t)
    want = v_to_library_layout(Vo, n, w + n, -np.inf)
    want = np.where(np.isneginf(want), INT_DEAD, want)
    assert np.array_equal(V.cpu().numpy().astype(np.float64), want)
    xo, do, so = oracle.backtrack_angle(Vo, h, w, k, t)
    assert list(x.cpu().numpy()) == list(xo)
    assert list(d.cpu().numpy()) == list(do)
    assert float(score.cpu().numpy()[0]) == so


def _detect(lib, img, k, r, gamma):
    x, d, s = lib.detect_polyline_angle(to_device(img), k, r, gamma)
    return x.cpu().numpy(), d.cpu().numpy(), int(s.cpu().numpy()[0])


def _assert_detect_parity(lib, img, k, r, gamma):
    x, d, s = _detect(lib, img, k, r, gamma)
    xo, do, so = oracle.detect_angle(img, k, r, gamma)
    assert list(x) == list(xo) and list(d) == list(do), (r, gamma)
    assert s == so
    if so != -np.inf:
        n = img.shape[0] // k
        _check_angle_path(n, gamma, d)
        assert np.all((x >= 0) & (x < img.shape[1]))
        assert oracle.path_score(oracle.gauss_rows(img, r), k, x[0], d) == so


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("r", [0, 1, 2])
def test_detect_angle_256x256_u8(lib, seed, r):
    img = synth.bent_edges(seed, 256, 256, 4, lines=1).img
    for gamma in (0.1, 0.3, 0.8):
        _assert_detect_parity(lib, img, 4, r, gamma)


@pytest.mark.parametrize("shape", SHAPES)
def test_detect_angle_shapes_int32(lib, shape):
    h, w, k = shape
    img = _img(h, w, "i32", 3 * h + w)
    _assert_detect_parity(lib, img, k, 1, 0.3)


@pytest.mark.parametrize("seed", range(2))
def test_detect_angle_2048x2048_k16_full_size(lib, seed):
    """The benchmark's image: 2048x2048 uint8 bent edges, k = 16, r = 2,
    gamma = 10 degrees, every output against the oracle."""
    wl = synth.bent_edges(seed)
    _assert_detect_parity(lib, wl.img, 16, 2, math.radians(10))


def test_detect_angle_256_row_bands(lib):
    wl = synth.bent_edges(7, 1024, 700, 4)
    _assert_detect_parity(lib, wl.img, 4, 2, 0.2)


def test_gamma_limits_equal_the_integer_bend_limits(lib):
    """gamma = 0 is B = 0 and gamma >= pi/2 is the unrestricted DP, through
    the library's two different DP kernels."""
    wl = synth.plain_uniform(3, 512, 384, 8, 4)
    img = wl.img
    for gamma, B in ((0.0, 0), (math.pi / 2, 1000)):
        xa, da, sa = _detect(lib, img, 8, 0, gamma)
        xb, db, sb = lib.detect_polyline(to_device(img), 8, B)
        assert list(xa) == list(xb.cpu().numpy()) and list(da) == list(db.cpu().numpy())
        assert sa == int(sb.cpu().numpy()[0])


@pytest.mark.parametrize("h,w,k,gamma", [(8, 1, 8, 0.3), (16, 2, 4, 0.0), (4, 9, 4, 1.0),
                                         (256, 1, 1, 0.5), (512, 3, 2, 0.05)])
def test_detect_angle_edge_cases(lib, h, w, k, gamma):
    img = _img(h, w, "u8", h + w)
    _assert_detect_parity(lib, img, k, 1, gamma)


def test_detect_angle_width_one_single_row_bands(lib):
    """Width 1 with one-row bands: the only polyline is the vertical one (a
    straight continuation is always admissible, so unlike the pruned DP the
    angle DP always has a solution)."""
    img = _img(6, 1, "u8", 1)
    _assert_detect_parity(lib, img, 6, 0, 0.0)


def test_detect_angle_reuses_its_workspace(lib):
    import torch
    wl0 = synth.bent_edges(1, 512, 512, 8)
    wl1 = synth.bent_edges(2, 512, 512, 8)
    need = lib.angle_workspace_bytes(lib.DTYPE_U8, 512, 512, 8, 2)
    ws = torch.full((need,), 0xAB, dtype=torch.uint8, device="cuda")
    for wl in (wl0, wl1, wl0):
        x, d, s = lib.detect_polyline_angle(to_device(wl.img), 8, 2, 0.25, ws=ws)
        xo, do, so = oracle.detect_angle(wl.img, 8, 2, 0.25)
        assert list(x.cpu().numpy()) == list(xo) and int(s.cpu().numpy()[0]) == so


def test_detect_angle_rejects_bad_arguments_on_device(lib):
    import torch
    img = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_angle(img, 4, 13, 0.3)          # r > 12
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_angle(img, 4, 2, -0.1)          # negative angle
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_angle(img, 4, 2, float("nan"))
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_angle(img, 3, 2, 0.3)           # 64 rows, k = 3
    tall = torch.zeros((4096, 8), dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.FhtdpError):
        lib.detect_polyline_angle(tall, 16, 10, 0.3)        # 255 * 4^10 * 4096 >= 2^31
    with pytest.raises(TypeError):
        lib.detect_polyline_angle(img.double(), 4, 2, 0.3)
    small = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.FhtdpError) as e:
        lib.detect_polyline_angle(img, 4, 2, 0.3, ws=small)
    assert e.value.code == 2


# ---------------------------------------------------------------------------
# The main problem for a batch in one persistent launch (fhtdp_batch_angle):
# rows smoothed by fhtdp_gauss_rows, then the engine with the window table.

BATCH_CASES = [
    # (band height n, [(h, w)...], k from h / n)
    (128, [(256, 256), (512, 300), (2048, 130), (1024, 517)]),
    (64, [(64, 37), (256, 1), (192, 700), (128, 129)]),
    (16, [(16, 5), (64, 77), (48, 1000)]),
    (2, [(8, 3), (4, 40)]),
]


def _batch_angle(lib, imgs, n, r, gamma, tune=False):
    import torch
    sm = [lib.gauss_rows(to_device(im), r) for im in imgs]
    ks = [im.shape[0] // n for im in imgs]
    plan = lib.BatchPlan(sm, ks, [2 * n - 2] * len(imgs))
    plan.angle(gamma)
    if tune:
        plan.autotune(reps=1)
    plan.run()
    torch.cuda.synchronize()
    assert plan.status() == 0
    return plan


@pytest.mark.parametrize("case", range(len(BATCH_CASES)))
@pytest.mark.parametrize("gamma", GAMMAS)
def test_batch_angle_int32_matches_oracle(lib, case, gamma):
    n, shapes = BATCH_CASES[case]
    imgs = [_img(h, w, "i32", 7 * h + w + case) for h, w in shapes]
    plan = _batch_angle(lib, imgs, n, 1, gamma)
    for i, im in enumerate(imgs):
        xo, do, so = oracle.detect_angle(im, im.shape[0] // n, 1, gamma)
        assert list(plan.x[i].cpu().numpy()) == list(xo), (i, gamma)
        assert list(plan.d[i].cpu().numpy()) == list(do), (i, gamma)
        assert int(plan.score[i].cpu().numpy().reshape(-1)[0]) == int(so)


@pytest.mark.parametrize("case", range(len(BATCH_CASES)))
def test_batch_angle_float_matches_oracle(lib, case):
    n, shapes = BATCH_CASES[case]
    rng = np.random.default_rng(case)
    imgs = [(np.abs(rng.standard_normal((h, w))) * 2.5).astype(np.float32) for h, w in shapes]
    for gamma in (0.1, math.radians(10), 0.8):
        plan = _batch_angle(lib, imgs, n, 2, gamma)
        for i, im in enumerate(imgs):
            xo, do, so = oracle.detect_angle_f32(im, im.shape[0] // n, 2, gamma)
            assert list(plan.x[i].cpu().numpy()) == list(xo), (i, gamma)
            assert list(plan.d[i].cpu().numpy()) == list(do), (i, gamma)
            s = float(plan.score[i].cpu().numpy().reshape(-1)[0])
            assert abs(s - so) <= 1e-5 * abs(so)


def test_batch_angle_2048x2048_tuned_full_size(lib):
    """The bench's main-problem batch shape (bent edges, r = 2, 10 degrees),
    tuned, against the oracle on every image."""
    imgs = [synth.bent_edges(s).img for s in range(4)]
    plan = _batch_angle(lib, imgs, 128, 2, math.radians(10), tune=True)
    for i, im in enumerate(imgs):
        xo, do, so = oracle.detect_angle(im, 16, 2, math.radians(10))
        assert list(plan.x[i].cpu().numpy()) == list(xo)
        assert list(plan.d[i].cpu().numpy()) == list(do)
        assert int(plan.score[i].cpu().numpy().reshape(-1)[0]) == int(so)


def test_batch_angle_rejects_mixed_heights_and_uint8(lib):
    import torch
    a = torch.zeros((64, 40), dtype=torch.int32, device="cuda")
    b = torch.zeros((128, 40), dtype=torch.int32, device="cuda")
    plan = lib.BatchPlan([a, b], [4, 4], [2, 2])   # band heights 16 and 32
    with pytest.raises(lib.FhtdpError):
        plan.angle(0.2)
    u = torch.zeros((64, 40), dtype=torch.uint8, device="cuda")
    plan = lib.BatchPlan([u], [4], [2])
    with pytest.raises(lib.FhtdpError):
        plan.angle(0.2)
    plan = lib.BatchPlan([a], [4], [2])
    with pytest.raises(lib.FhtdpError):
        plan.angle(-1.0)
