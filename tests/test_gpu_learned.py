"""The learned window proposal on the GPU: each network kernel against the
float64 CPU reference (oracle.cnn_ref, pinned by finite differences), the
pruned (windowed) DP against the oracle's windowed DP, and the whole
pipeline: training lowers the loss, and every answer is either the exact
optimum (fallback) or the exact optimum inside the proposed windows."""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import cnn_ref

pytestmark = pytest.mark.gpu

ATOL, RTOL = 3e-2, 2e-2   # bf16 operands and bf16 outputs, FP32 accumulation


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)


def _np(t):
    return t.float().cpu().numpy().astype(np.float64)


def _close(got, want):
    assert np.all(np.abs(got - want) <= ATOL + RTOL * np.abs(want)), \
        np.max(np.abs(got - want) - RTOL * np.abs(want))


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("cin,dil", [(32, 1), (32, 2), (32, 8), (1, 1), (1, 4)])
def test_conv_forward_matches_reference(lib, cin, dil):
    import torch
    rng = np.random.default_rng(cin + dil)
    N, H, W = 2, 12, 128
    x = _bf16(rng.standard_normal((N, H, W, cin)))
    taps = 16 if cin == 1 else 9
    w = rng.standard_normal((taps, cin, 32)) * 0.2
    if cin == 1:
        w[9:] = 0
    wb = _bf16(w.reshape(-1, 32))
    b = torch.from_numpy(rng.standard_normal(32).astype(np.float32))
    y = torch.empty(N, H, W, 32, dtype=torch.bfloat16, device="cuda")
    xd, wd, bd = x.cuda(), wb.cuda(), b.cuda()
    assert lib.lib().fhtdp_cnn_conv3x3(xd.data_ptr(), cin, N, H, W, dil, wd.data_ptr(),
                                       bd.data_ptr(), 1, y.data_ptr(), _stream()) == 0
    ref = cnn_ref.conv3x3(_np(x), _np(wb).reshape(taps, cin, 32), b.numpy().astype(np.float64),
                          dil)
    _close(_np(y), np.maximum(ref, 0))


def test_conv_gradients_match_reference(lib):
    import torch
    rng = np.random.default_rng(5)
    N, H, W, dil = 2, 10, 64, 2
    x = _bf16(np.maximum(rng.standard_normal((N, H, W, 32)), 0))
    w = _bf16(rng.standard_normal((9 * 32, 32)) * 0.2)
    dz = _bf16(rng.standard_normal((N, H, W, 32)))
    dx = torch.empty(N, H, W, 32, dtype=torch.bfloat16, device="cuda")
    wf = torch.empty(9 * 32 * 32, dtype=torch.bfloat16, device="cuda")
    xd, wd, dzd = x.cuda(), w.cuda(), dz.cuda()
    assert lib.lib().fhtdp_cnn_conv3x3_dgrad(dzd.data_ptr(), N, H, W, dil, wd.data_ptr(),
                                             wf.data_ptr(), dx.data_ptr(), _stream()) == 0
    _close(_np(dx), cnn_ref.conv3x3_dgrad(_np(dz), _np(w).reshape(9, 32, 32), dil))
    dw = torch.zeros(9 * 32, 32, device="cuda")
    db = torch.zeros(32, device="cuda")
    assert lib.lib().fhtdp_cnn_conv3x3_wgrad(xd.data_ptr(), 32, N, H, W, dil, dzd.data_ptr(),
                                             dw.data_ptr(), db.data_ptr(), _stream()) == 0
    rw, rb = cnn_ref.conv3x3_wgrad(_np(x), _np(dz), dil)
    assert np.allclose(dw.cpu().numpy().reshape(9, 32, 32), rw, rtol=1e-3, atol=1e-3)
    assert np.allclose(db.cpu().numpy(), rb, rtol=1e-3, atol=1e-3)
    # the single-channel first layer
    x1 = _bf16(rng.standard_normal((N, H, W, 1)))
    dw1 = torch.zeros(16, 32, device="cuda")
    assert lib.lib().fhtdp_cnn_conv3x3_wgrad(x1.cuda().data_ptr(), 1, N, H, W, 1, dzd.data_ptr(),
                                             dw1.data_ptr(), None, _stream()) == 0
    rw1, _ = cnn_ref.conv3x3_wgrad(_np(x1), _np(dz), 1)
    assert np.allclose(dw1.cpu().numpy()[:9], rw1[:, 0], rtol=1e-3, atol=1e-3)
    assert np.all(dw1.cpu().numpy()[9:] == 0)


def test_band_head_matches_reference(lib):
    import torch
    rng = np.random.default_rng(6)
    N, H, W, bands = 3, 32, 64, 4
    z = _bf16(rng.standard_normal((N, H, W, 32)) * 2)
    labels = rng.integers(0, 32, (N, bands)).astype(np.int32)
    zd = z.cuda()
    dl = torch.empty_like(zd)
    loss = torch.zeros(1, device="cuda")
    pred = torch.empty(N, bands, dtype=torch.int32, device="cuda")
    lab = torch.from_numpy(labels).cuda()
    assert lib.lib().fhtdp_cnn_band_head(zd.data_ptr(), N, H, W, bands, lab.data_ptr(),
                                         1.0 / (N * bands), dl.data_ptr(), loss.data_ptr(),
                                         pred.data_ptr(), _stream()) == 0
    pooled, rl, rdz, rpred = cnn_ref.band_head(_np(z), bands, labels)
    assert abs(float(loss.cpu()) - rl) <= 1e-3 * max(1.0, abs(rl))
    assert np.array_equal(pred.cpu().numpy(), rpred)
    assert np.allclose(_np(dl), rdz, rtol=2e-2, atol=1e-6)


def test_pruned_dp_matches_the_oracle_windowed_dp(lib):
    import torch
    from paper_1912_01884_gb300 import synth
    rng = np.random.default_rng(7)
    wls, wins = [], []
    for j in range(6):
        wl = synth.plain_uniform(300 + j, 256, 320, 4, 8)
        n = 64
        c = rng.integers(-50, 50, 4)
        width = rng.integers(0, 20, 4)
        win = np.stack([c, c + width], 1).astype(np.int32)
        if j == 5:
            win[:] = [[-63, -60], [60, 63], [-63, -60], [60, 63]]   # no admissible polyline
        wls.append(wl)
        wins.append(win)
    imgs = [torch.from_numpy(w.img).cuda() for w in wls]
    plan = lib.BatchPlan(imgs, [4] * 6, [8] * 6, windows=[torch.from_numpy(w).cuda() for w in wins])
    plan.run()
    plan.status()
    for i, (wl, win) in enumerate(zip(wls, wins)):
        xo, do, so = oracle.detect_windowed(wl.img, 4, 8, win)
        x = plan.x[i].cpu().numpy()
        s = int(plan.score[i].cpu().numpy()[0])
        assert list(x) == list(xo), i
        if so == -np.inf:
            assert s == np.iinfo(np.int32).min
        else:
            assert s == int(so) and list(plan.d[i].cpu().numpy()) == list(do)


def test_learned_pipeline_trains_and_answers_exactly_or_within_windows(lib):
    import torch
    from paper_1912_01884_gb300 import learned
    h, w, k, B = 512, 512, 8, 12
    model = learned.LaneProposer(seed=1, lr=3e-3)
    losses = []
    for step in range(40):
        imgs = learned.lane_images(1000 + step, 32, h, w, k, B)
        _, d, _ = learned.exact_paths(imgs, k, B)
        labels = torch.from_numpy(learned.bins_of(d.cpu().numpy()).astype(np.int32)).cuda()
        losses.append(float(model.train_step(imgs, labels, k).cpu()))
    assert np.mean(losses[-5:]) < np.mean(losses[:5])
    imgs = learned.lane_images(5000, 24, h, w, k, B)
    x, d, s, fb = learned.detect_learned(model, imgs, k, B)
    xe, de, se = learned.exact_paths(imgs, k, B)
    win = model.windows(model.propose(imgs, k), h // k).cpu().numpy()
    for i in range(imgs.shape[0]):
        if bool(fb[i]):
            assert torch.equal(x[i], xe[i]) and int(s[i]) == int(se[i])
        else:
            xo, do, so = oracle.detect_windowed(imgs[i].cpu().numpy(), k, B, win[i])
            assert list(x[i].cpu().numpy()) == list(xo) and int(s[i]) == int(so)
