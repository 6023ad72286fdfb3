"""GPU parity of the through-point query (Subproblems 2-3, Sec. 2.2-2.3):
the best polyline through a given point on a band border, through the C ABI,
against the CPU oracle on the same seeded inputs (int32, bit-exact)."""
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
    return rng.integers(-3000, 3000, (h, w)).astype(np.int32)


def _through(lib, img, k, B, j, xp):
    x, d, s = lib.detect_through_point(to_device(img), k, B, j, xp)
    return x.cpu().numpy(), d.cpu().numpy(), int(s.cpu().numpy()[0])


def _assert_parity(lib, img, k, B, j, xp):
    x, d, s = _through(lib, img, k, B, j, xp)
    xo, do, so = oracle.detect_through(img, k, B, j, xp)
    assert list(x) == list(xo) and list(d) == list(do), (B, j, xp)
    assert s == so
    assert x[j] == xp
    check_path(img, k, B, x, d)


@pytest.mark.parametrize("dtype", ["u8", "i32"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("B", [0, 3, 1000])
def test_through_point_matches_oracle(lib, shape, dtype, B):
    h, w, k = shape
    img = _img(h, w, dtype, h * 5 + w + B)
    for j in sorted({0, k // 2, k}):
        for xp in sorted({0, w // 3, w - 1}):
            _assert_parity(lib, img, k, B, j, xp)


@pytest.mark.parametrize("seed", range(2))
def test_through_point_2048x2048_k16_B16_full_size(lib, seed):
    """The benchmark's image and query: the point on border 8 at a planted
    polyline's vertex, and at a random column."""
    wl = synth.plain_gaussian(seed)
    xs, _ = wl.planted[0]
    _assert_parity(lib, wl.img, 16, 16, 8, int(xs[8]))
    _assert_parity(lib, wl.img, 16, 16, 8, 1000 + 37 * seed)


def test_through_the_global_optimum_is_the_global_optimum(lib):
    wl = synth.plain_uniform(11, 512, 384, 8, 4)
    gx, gd, gs = lib.detect_polyline(to_device(wl.img), 8, 4)
    gx = gx.cpu().numpy()
    for j in range(9):
        x, d, s = _through(lib, wl.img, 8, 4, j, int(gx[j]))
        assert list(x) == list(gx) and s == int(gs.cpu().numpy()[0])


def test_through_point_reuses_its_workspace(lib):
    import torch
    img = _img(256, 300, "u8", 9)
    need = lib.through_workspace_bytes(lib.DTYPE_U8, 256, 300, 4)
    ws = torch.full((need,), 0x5A, dtype=torch.uint8, device="cuda")
    for j, xp in ((1, 17), (3, 250), (1, 17)):
        x, d, s = lib.detect_through_point(to_device(img), 4, 5, j, xp, ws=ws)
        xo, do, so = oracle.detect_through(img, 4, 5, j, xp)
        assert list(x.cpu().numpy()) == list(xo) and int(s.cpu().numpy()[0]) == so


def test_through_point_rejects_bad_arguments_on_device(lib):
    import torch
    img = torch.zeros((64, 40), dtype=torch.uint8, device="cuda")
    for args in ((4, 2, 5, 0), (4, 2, -1, 0), (4, 2, 1, 40), (4, 2, 1, -1), (4, -1, 1, 3)):
        with pytest.raises(lib.FhtdpError):
            lib.detect_through_point(img, *args)
    with pytest.raises(TypeError):
        lib.detect_through_point(img.double(), 4, 2, 1, 3)


@pytest.mark.parametrize("shape", SHAPES[:8])
@pytest.mark.parametrize("gamma", [0.0, 0.2, 0.8])
def test_through_point_with_bend_angle_matches_oracle(lib, shape, gamma):
    """Subproblem 3 with the bend angle, rows smoothed with r = 1."""
    h, w, k = shape
    img = _img(h, w, "u8", 13 * h + w)
    for j in sorted({0, k // 2, k}):
        for xp in sorted({0, w // 2, w - 1}):
            x, d, s = lib.detect_through_point_angle(to_device(img), k, 1, gamma, j, xp)
            xo, do, so = oracle.detect_angle_through(img, k, 1, gamma, j, xp)
            assert list(x.cpu().numpy()) == list(xo) and list(d.cpu().numpy()) == list(do)
            assert int(s.cpu().numpy()[0]) == so
            assert x.cpu().numpy()[j] == xp


def test_through_point_with_bend_angle_2048x2048_full_size(lib):
    wl = synth.bent_edges(0)
    xp = int(wl.planted[1][8 * 128])
    x, d, s = lib.detect_through_point_angle(to_device(wl.img), 16, 2, 0.17453292519943295, 8, xp)
    xo, do, so = oracle.detect_angle_through(wl.img, 16, 2, 0.17453292519943295, 8, xp)
    assert list(x.cpu().numpy()) == list(xo) and int(s.cpu().numpy()[0]) == so


def test_batch_points_match_oracle(lib):
    """fhtdp_batch_points: several uint8 images of different shapes in one
    persistent launch, each with its own point (top border, a middle border,
    the bottom border) or none, against the oracle image by image; then new
    points on the same plan."""
    import torch
    shapes = [(256, 256, 4), (64, 37, 4), (512, 300, 4), (16, 5, 16), (2048, 130, 16),
              (96, 77, 3), (1024, 517, 8)]
    imgs = [_img(h, w, "u8", 31 * h + w) for h, w, _ in shapes]
    ks = [k for _, _, k in shapes]
    Bs = [3, 1000, 0, 2, 16, 5, 9]
    plan = lib.BatchPlan([to_device(im) for im in imgs], ks, Bs)
    for rnd in range(2):
        pts = []
        for i, (h, w, k) in enumerate(shapes):
            j = [1, k // 2, k, None][(i + rnd) % 4]   # border 0 is for the single call
            pts.append(None if j is None else (j, (w * (i + 1 + rnd)) // 7 % w))
        plan.points(pts)
        if rnd == 1:
            plan.autotune(reps=1)
        plan.run()
        torch.cuda.synchronize()
        assert plan.status() == 0
        for i, (im, k, B, pt) in enumerate(zip(imgs, ks, Bs, pts)):
            x = plan.x[i].cpu().numpy()
            d = plan.d[i].cpu().numpy()
            s = int(plan.score[i].cpu().numpy().reshape(-1)[0])
            if pt is None:
                xo, do, so = oracle.detect(im, k, B)
            else:
                xo, do, so = oracle.detect_through(im, k, B, *pt)
                assert x[pt[0]] == pt[1]
            assert list(x) == list(xo) and list(d) == list(do), (rnd, i, pt)
            assert s == so


def test_batch_points_rejects_bad_points(lib):
    import torch
    a = torch.zeros((64, 40), dtype=torch.uint8, device="cuda")
    plan = lib.BatchPlan([a], [4], [2])
    for bad in [(5, 0), (1, 40), (2, -1), (0, 3)]:   # border 0: the single call
        with pytest.raises(lib.FhtdpError):
            plan.points([bad])
    f = torch.zeros((64, 40), dtype=torch.float32, device="cuda")
    plan = lib.BatchPlan([f], [4], [2])
    with pytest.raises(lib.FhtdpError):
        plan.points([(1, 3)])
