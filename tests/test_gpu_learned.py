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


@pytest.mark.parametrize("W,dil,relu,bias", [(192, 3, 0, False), (256, 8, 1, True),
                                             (64, 5, 1, True), (320, 1, 0, True)])
def test_conv_tensor_core_tiles_and_ragged_rows(lib, W, dil, relu, bias):
    """32-channel layers run 128-pixel tiles on tcgen05: rows that end inside
    a tile (192, 320), a row narrower than a tile (64), every dilation's halo
    inside the staged rows, with and without bias and ReLU; no wait gave up."""
    import torch
    rng = np.random.default_rng(W + dil)
    N, H = 3, 9
    x = _bf16(rng.standard_normal((N, H, W, 32)))
    w = rng.standard_normal((9, 32, 32)) * 0.2
    wb = _bf16(w.reshape(-1, 32))
    b = rng.standard_normal(32).astype(np.float32)
    bd = torch.from_numpy(b).cuda() if bias else None
    y = torch.full((N, H, W, 32), 7.0, dtype=torch.bfloat16, device="cuda")
    xd, wd = x.cuda(), wb.cuda()
    L = lib.lib()
    assert L.fhtdp_cnn_status(1) == 0
    assert L.fhtdp_cnn_conv3x3(xd.data_ptr(), 32, N, H, W, dil, wd.data_ptr(),
                               bd.data_ptr() if bias else None, relu, y.data_ptr(),
                               _stream()) == 0
    torch.cuda.synchronize()
    assert L.fhtdp_cnn_status(0) == 0
    ref = cnn_ref.conv3x3(_np(x), _np(wb).reshape(9, 32, 32),
                          b.astype(np.float64) if bias else np.zeros(32), dil)
    _close(_np(y), np.maximum(ref, 0) if relu else ref)


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


def test_wgrad_tensor_core_accumulates_over_many_segments(lib):
    """The tcgen05 weight gradient keeps its accumulators in tensor memory
    across the row segments a CTA takes (more segments than CTAs), with rows
    that end inside a segment and a wide dilation."""
    import torch
    rng = np.random.default_rng(11)
    N, H, W, dil = 4, 64, 320, 7
    x = _bf16(rng.standard_normal((N, H, W, 32)))
    dz = _bf16(rng.standard_normal((N, H, W, 32)) * 0.5)
    dw = torch.zeros(9 * 32, 32, device="cuda")
    db = torch.zeros(32, device="cuda")
    L = lib.lib()
    assert L.fhtdp_cnn_status(1) == 0
    assert L.fhtdp_cnn_conv3x3_wgrad(x.cuda().data_ptr(), 32, N, H, W, dil, dz.cuda().data_ptr(),
                                     dw.data_ptr(), db.data_ptr(), _stream()) == 0
    torch.cuda.synchronize()
    assert L.fhtdp_cnn_status(0) == 0
    rw, rb = cnn_ref.conv3x3_wgrad(_np(x), _np(dz), dil)
    assert np.allclose(dw.cpu().numpy().reshape(9, 32, 32), rw, rtol=1e-3, atol=1e-2)
    assert np.allclose(db.cpu().numpy(), rb, rtol=1e-3, atol=1e-2)


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


@pytest.mark.gpu
def test_trained_proposal_reaches_99_percent_hit_rate_and_resolves_most_images_pruned(lib):
    """The lane workload (1024x1024, k = 16, B = 12): after 1500 Adam steps
    on batches of 32 images labelled by the exact DP, the learned detection
    with fallback on low confidence (a band's bin probability below a
    threshold calibrated on 1024 other images to a 99.5% hit rate) returns
    the exact optimum for at least 99% of 1024 held-out images while most of
    them (at least half) are answered by the pruned DP alone, which searches
    16 of the 127 displacements of each band.  The untrained network under
    the same rule resolves almost none, so the pruned answers are what
    training gains.  The times of both paths are printed; the learned path
    is not faster than the exact engine on this GPU (the CNN's 3.6 GFLOP per
    image cost more than the whole exact DP)."""
    import torch
    from paper_1912_01884_gb300 import learned
    h = w = 1024
    k, B, bs, steps = 16, 12, 32, 1500
    model = learned.LaneProposer(seed=0, lr=3e-3)
    for step in range(steps):
        if step == int(steps * 0.6):
            model.lr = 1e-3
        if step == int(steps * 0.85):
            model.lr = 3e-4
        imgs = learned.lane_images(1000 + step, bs, h, w, k, B)
        _, d, _ = learned.exact_paths(imgs, k, B)
        labels = torch.from_numpy(learned.bins_of(d.cpu().numpy()).astype(np.int32)).cuda()
        model.train_step(imgs, labels, k)
    conf, chit, cfb = learned.calibrate_min_conf(
        model, learned.lane_images(2 * 10**6, 1024, h, w, k, B), k, B)
    print("calibrated min_conf %.2f (calibration images: hit %.4f fallback %.4f)"
          % (conf, chit, cfb))
    N = 1024
    imgs = learned.lane_images(10**6, N, h, w, k, B)
    xe, de, se = learned.exact_paths(imgs, k, B)
    plan = learned.LearnedPlan(imgs, k, B)

    def rates(net):
        plan.run(net, 0.0, conf)
        plan.status()
        hit = (plan.score == se) & (plan.x == xe).all(1) & (plan.d == de).all(1)
        return float(hit.float().mean()), float(plan.used_fallback.float().mean())

    hit, fb = rates(model)
    hit0, fb0 = rates(learned.LaneProposer(seed=5))
    print("trained: hit %.4f fallback %.4f; untrained: hit %.4f fallback %.4f"
          % (hit, fb, hit0, fb0))
    assert hit >= 0.99
    assert fb <= 0.5
    assert fb0 >= 0.95 and hit0 >= hit
    plain = lib.BatchPlan([imgs[i] for i in range(N)], [k] * N, [B] * N)
    t = {}
    for name, fn in (("plain", lambda: plain.run()), ("learned", lambda: plan.run(model, 0.0, conf))):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            fn()
        e1.record()
        torch.cuda.synchronize()
        t[name] = e0.elapsed_time(e1) / 3
    print("ms per %d images: plain %.3f learned %.3f" % (N, t["plain"], t["learned"]))


def _layer_params(lib, params):
    """Views of the parameter block (the layout of include/fhtdp.h): per layer
    FP32 weights, bias, Adam moments and the bf16 copy, each from a 256-byte
    boundary."""
    import torch
    views, off = [], 0
    buf = params
    for layer in range(4):
        rows = 16 if layer == 0 else 288
        parts = {}
        for name, count, dt, size in (("w", rows * 32, torch.float32, 4), ("b", 32, torch.float32, 4),
                                      ("mw", rows * 32, torch.float32, 4),
                                      ("vw", rows * 32, torch.float32, 4),
                                      ("mb", 32, torch.float32, 4), ("vb", 32, torch.float32, 4),
                                      ("w16", rows * 32, torch.bfloat16, 2)):
            parts[name] = buf[off:off + count * size].view(dt)
            off = (off + count * size + 255) // 256 * 256
        views.append(parts)
    assert off == buf.numel()
    return views


def test_cnn_forward_backward_step_equal_the_per_layer_calls(lib):
    """The whole-network calls give exactly what the per-layer calls (each
    pinned against the CPU reference above) give in sequence."""
    import torch
    from paper_1912_01884_gb300 import learned
    N, h, w, k = 2, 128, 256, 4
    imgs = learned.lane_images(11, N, h, w, k, 12)
    model = learned.LaneProposer(seed=3)
    P = _layer_params(lib, model.params)
    pred, conf = model.forward(imgs, k)
    # per-layer reference of the forward pass
    L = lib.lib()
    s = _stream()
    x = torch.empty(N, h // 4, w // 4, 1, dtype=torch.bfloat16, device="cuda")
    assert L.fhtdp_cnn_downsample4(imgs.data_ptr(), N, h, w, x.data_ptr(), s) == 0
    acts = [x]
    for layer, dil in enumerate((1, 2, 4, 8)):
        y = torch.empty(N, h // 4, w // 4, 32, dtype=torch.bfloat16, device="cuda")
        assert L.fhtdp_cnn_conv3x3(acts[-1].data_ptr(), 1 if layer == 0 else 32, N, h // 4, w // 4,
                                   dil, P[layer]["w16"].data_ptr(), P[layer]["b"].data_ptr(),
                                   1 if layer < 3 else 0, y.data_ptr(), s) == 0
        acts.append(y)
    rpred = torch.empty(N, k, dtype=torch.int32, device="cuda")
    assert L.fhtdp_cnn_band_head(acts[-1].data_ptr(), N, h // 4, w // 4, k, None, 1.0, None,
                                 None, rpred.data_ptr(), s) == 0
    assert torch.equal(pred, rpred)
    assert torch.all((conf > 0) & (conf <= 1))
    # backward + step against the per-layer gradient and Adam calls
    labels = torch.randint(0, 32, (N, k), dtype=torch.int32, device="cuda")
    before = [{n_: t.clone() for n_, t in p.items()} for p in P]
    loss = model.train_step(imgs, labels, k)
    dz = torch.empty_like(acts[-1])
    rloss = torch.zeros(1, device="cuda")
    assert L.fhtdp_cnn_band_head(acts[-1].data_ptr(), N, h // 4, w // 4, k, labels.data_ptr(),
                                 1.0 / (N * k), dz.data_ptr(), rloss.data_ptr(), None, s) == 0
    assert torch.allclose(loss, rloss, rtol=1e-6)
    # the block's FP32 gradients sit in the training workspace after the
    # activations and two gradient buffers and the flipped weights
    a256 = lambda v: (v + 255) // 256 * 256
    px = N * (h // 4) * (w // 4)
    off = a256(px * 2) + 6 * a256(px * 32 * 2) + a256(9 * 32 * 32 * 2)
    ws = model._ws
    wf = torch.empty(9 * 32 * 32, dtype=torch.bfloat16, device="cuda")
    gofs = []
    for layer in range(4):
        rows = 16 if layer == 0 else 288
        gofs.append(off)
        off += a256((rows * 32 + 32) * 4)
    for layer in range(3, -1, -1):
        dil = (1, 2, 4, 8)[layer]
        rows = 16 if layer == 0 else 288
        g = ws[gofs[layer]:gofs[layer] + (rows * 32 + 32) * 4].view(torch.float32)
        dw = torch.zeros(rows, 32, device="cuda")
        db = torch.zeros(32, device="cuda")
        assert L.fhtdp_cnn_conv3x3_wgrad(acts[layer].data_ptr(), 1 if layer == 0 else 32, N,
                                         h // 4, w // 4, dil, dz.data_ptr(), dw.data_ptr(),
                                         db.data_ptr(), s) == 0
        # the same gradient up to the order of the FP32 atomic sums
        assert torch.allclose(g[:rows * 32], dw.flatten(), rtol=1e-4, atol=1e-6), layer
        assert torch.allclose(g[rows * 32:], db, rtol=1e-4, atol=1e-6), layer
        # Adam on the block's own gradient from the same starting point gives
        # the block's new weights and their bf16 copy
        pw, mw, vw = (before[layer]["w"].clone(), before[layer]["mw"].clone(),
                      before[layer]["vw"].clone())
        wb = torch.empty(rows * 32, dtype=torch.bfloat16, device="cuda")
        gw = g[:rows * 32].clone()
        assert L.fhtdp_cnn_adam(pw.data_ptr(), mw.data_ptr(), vw.data_ptr(), gw.data_ptr(),
                                rows * 32, ctypes.c_float(model.lr), ctypes.c_float(0.9),
                                ctypes.c_float(0.999), ctypes.c_float(1e-8), 1, wb.data_ptr(),
                                s) == 0
        assert torch.equal(pw, P[layer]["w"]) and torch.equal(wb, P[layer]["w16"])
        if layer == 0:
            break
        dx = torch.empty_like(dz)
        assert L.fhtdp_cnn_conv3x3_dgrad(dz.data_ptr(), N, h // 4, w // 4, dil,
                                         before[layer]["w16"].data_ptr(), wf.data_ptr(),
                                         dx.data_ptr(), s) == 0
        assert L.fhtdp_cnn_relu_backward(acts[layer].data_ptr(), dx.data_ptr(), dx.numel(), s) == 0
        dz = dx


def _check_learned(lib, imgs, k, B, plan, margin):
    """Every answer of the learned detection: the exact optimum where it fell
    back, else the optimum inside the proposed windows; and the fallback rule."""
    import torch
    from paper_1912_01884_gb300 import learned
    N, h, w = imgs.shape
    n = h // k
    xe, de, se = learned.exact_paths(imgs, k, B)
    fb = plan.used_fallback.cpu().numpy()
    x, d, s = plan.x.cpu().numpy(), plan.d.cpu().numpy(), plan.score.cpu().numpy()
    for i in range(N):
        if fb[i]:
            assert list(x[i]) == list(xe[i].cpu().numpy()) and int(s[i]) == int(se[i]), i
        else:
            assert x[i][0] >= 0 and s[i] >= margin * h, i
    return fb


def test_learned_detection_falls_back_exactly_where_the_rule_says(lib):
    import torch
    from paper_1912_01884_gb300 import learned
    h, w, k, B = 512, 512, 8, 12
    model = learned.LaneProposer(seed=2, lr=3e-3)
    for step in range(20):
        imgs = learned.lane_images(2000 + step, 16, h, w, k, B)
        _, d, _ = learned.exact_paths(imgs, k, B)
        labels = torch.from_numpy(learned.bins_of(d.cpu().numpy()).astype(np.int32)).cuda()
        model.train_step(imgs, labels, k)
    imgs = learned.lane_images(7000, 24, h, w, k, B)
    plan = learned.LearnedPlan(imgs, k, B)
    pred = model.propose(imgs, k)
    win = model.windows(pred, h // k).cpu().numpy()
    conf = model.forward(imgs, k)[1].cpu().numpy()
    for margin, min_conf in ((0.0, 0.0), (60.0, 0.0), (0.0, 0.5), (1e9, 0.0)):
        plan.run(model, margin, min_conf)
        plan.status()
        fb = _check_learned(lib, imgs, k, B, plan, margin)
        x, d, s = plan.x.cpu().numpy(), plan.d.cpu().numpy(), plan.score.cpu().numpy()
        for i in range(imgs.shape[0]):
            xo, do, so = oracle.detect_windowed(imgs[i].cpu().numpy(), k, B, win[i])
            n = h // k
            edge = any((do[b] == win[i][b][0] and win[i][b][0] > -(n - 1)) or
                       (do[b] == win[i][b][1] and win[i][b][1] < n - 1) for b in range(k)) \
                if xo[0] >= 0 else True
            want_fb = xo[0] < 0 or edge or so < margin * h or conf[i].min() < min_conf
            assert bool(fb[i]) == bool(want_fb), (margin, min_conf, i)
            if not fb[i]:
                assert list(x[i]) == list(xo) and list(d[i]) == list(do) and int(s[i]) == int(so)
        if margin == 1e9:
            assert fb.all()


def test_learned_detection_is_captured_in_a_cuda_graph(lib):
    import torch
    from paper_1912_01884_gb300 import learned
    h, w, k, B = 256, 256, 4, 8
    model = learned.LaneProposer(seed=4)
    imgs = learned.lane_images(8000, 8, h, w, k, B)
    plan = learned.LearnedPlan(imgs, k, B)
    stream = torch.cuda.Stream()
    plan.run(model, 50.0, stream=stream)   # first use outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.run(model, 50.0, stream=stream)
    for t in (plan.x, plan.d, plan.score, plan.used_fallback):
        t.fill_(-7)
    with torch.cuda.stream(stream):
        g.replay()
    torch.cuda.synchronize()
    _check_learned(lib, imgs, k, B, plan, 50.0)
