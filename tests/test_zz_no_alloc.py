"""fhtdp_detect_polyline_noalloc: the detection for callers that cannot
allocate device memory (hosts that own all device memory, or real-time loops
where a cudaMalloc, which may synchronise the device, is not allowed).  Its
scratch is a fixed array inside the library, so it must give exactly what
fhtdp_detect_polyline gives with a caller workspace, call after call, even
though every call reuses the same array.  This file is collected last so that
a run stopping at its first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1912_01884_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    fn = lib.lib().fhtdp_detect_polyline_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 6 + [ctypes.c_void_p] * 4
    return fn


def _status(lib):
    fn = lib.lib().fhtdp_detect_polyline_noalloc_status
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p]
    return fn


def _call(lib, img, k, B):
    """The no-allocation entry point through the C ABI with raw pointers."""
    import torch
    h, w = img.shape
    x = torch.full((k + 1,), -1, dtype=torch.int32, device="cuda")
    d = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    score = torch.zeros(1, dtype=torch.float32 if img.dtype == torch.float32 else torch.int32,
                        device="cuda")
    code = {torch.uint8: 0, torch.int32: 1, torch.float32: 2}[img.dtype]
    stream = torch.cuda.current_stream().cuda_stream
    rc = _noalloc(lib)(img.data_ptr(), code, h, w, img.stride(0), k, B, x.data_ptr(),
                       d.data_ptr(), score.data_ptr(), ctypes.c_void_p(stream))
    assert rc == 0, lib.lib().fhtdp_last_error().decode()
    assert lib.lib().fhtdp_last_error().decode() == ""
    torch.cuda.synchronize()
    return x.cpu().numpy(), d.cpu().numpy(), score.cpu().numpy()[0]


def _workloads():
    # fused engine (bands of 64 and 128 rows, uint8 and float) and the
    # 256-row-band path, whose argmax key also lives in the shared array
    return [synth.plain_gaussian(11), synth.plain_uniform(12, 256, 256, 4, 8),
            synth.ridge_response(13, 1024, 768, 8, 24),
            synth.plain_uniform(14, 512, 512, 2, 32),
            synth.ridge_response(15, 512, 384, 2, 40)]


def test_noalloc_matches_detect_polyline_on_two_calls_in_a_row(lib):
    import torch
    for wl in _workloads():
        img = torch.from_numpy(wl.img).cuda()
        want = [t.cpu().numpy() for t in lib.detect_polyline(img, wl.k, wl.B)]
        for _ in range(2):   # two calls in a row share (and reuse) the built-in scratch
            x, d, s = _call(lib, img, wl.k, wl.B)
            assert np.array_equal(x, want[0]) and np.array_equal(d, want[1])
            if img.dtype == torch.float32:
                assert np.float32(s).view(np.uint32) == np.float32(want[2][0]).view(np.uint32)
            else:
                assert int(s) == int(want[2][0])
            assert _status(lib)(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0


def test_noalloc_matches_the_oracle(lib):
    import torch
    for wl in _workloads():
        img = torch.from_numpy(wl.img).cuda()
        x, d, s = _call(lib, img, wl.k, wl.B)
        if wl.img.dtype == np.float32:
            xo, do, so = oracle.detect_f32(wl.img, wl.k, wl.B)
            assert np.float32(s) == np.float32(so)
        else:
            xo, do, so = oracle.detect(wl.img, wl.k, wl.B)
            assert int(s) == int(so)
        assert list(x) == list(xo) and list(d) == list(do)


def test_noalloc_status_reports_a_wait_that_gave_up(lib):
    import torch
    wl = synth.plain_uniform(21, 512, 384, 4, 8)
    img = torch.from_numpy(wl.img).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # band k-1 = 3, tile 1 never publishes; its consumers' waits give up after ~1 ms
    lib.lib().fhtdp_debug_inject(3, 1, 2_000_000)
    x = torch.zeros(5, dtype=torch.int32, device="cuda")
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _noalloc(lib)(img.data_ptr(), 0, 512, 384, 384, 4, 8, x.data_ptr(), d.data_ptr(),
                       s.data_ptr(), stream)
    assert rc == 0
    assert _status(lib)(stream) == 4
    assert "gave up" in lib.lib().fhtdp_last_error().decode()
    # the next call clears the control block and is correct again
    xg, dg, sg = _call(lib, img, 4, 8)
    assert _status(lib)(stream) == 0
    xo, do, so = oracle.detect(wl.img, 4, 8)
    assert list(xg) == list(xo) and list(dg) == list(do) and int(sg) == int(so)


def test_noalloc_rejects_images_beyond_the_builtin_scratch(lib):
    fn = _noalloc(lib)
    h, w, k = 4096, 4096, 32
    need = lib.workspace_bytes(0, h, w, k, 16)
    limit = 16 << 20
    assert need > limit
    fake = ctypes.c_void_p(256)   # never dereferenced: rejected before any launch
    rc = fn(fake, 0, h, w, w, k, 16, fake, fake, fake, None)
    assert rc == 2
    assert "built-in scratch" in lib.lib().fhtdp_last_error().decode()
