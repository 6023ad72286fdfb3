"""Failure detection without a GPU fault: a tile that never publishes makes
its consumers' bounded waits run out; the run reports FHTDP_ETIMEOUT through
the workspace status, and the next run on the same context is correct."""
import numpy as np
import pytest

import oracle
from paper_1912_01884_gb300 import synth

pytestmark = pytest.mark.gpu


def test_missing_producer_times_out_and_the_context_recovers(lib):
    import torch
    wl = synth.plain_uniform(21, 512, 384, 4, 8)
    img = torch.from_numpy(wl.img).cuda()
    ws = torch.empty(lib.workspace_bytes(0, 512, 384, 4, 8), dtype=torch.uint8, device="cuda")
    # band k-1 = 3, tile 1 never publishes; waits give up after ~1 ms
    lib.lib().fhtdp_debug_inject(3, 1, 2_000_000)
    lib.detect_polyline(img, 4, 8, ws=ws)
    with pytest.raises(lib.FhtdpError) as e:
        lib.workspace_status(ws)
    assert e.value.code == 4
    # the same context and workspace work again
    x, d, s = lib.detect_polyline(img, 4, 8, ws=ws)
    lib.workspace_status(ws)
    xo, do, so = oracle.detect(wl.img, 4, 8)
    assert list(x.cpu().numpy()) == list(xo) and int(s.cpu().numpy()[0]) == int(so)


def test_batch_missing_producer_times_out(lib):
    import torch
    wls = [synth.plain_uniform(30 + j, 256, 300, 4, 8) for j in range(3)]
    plan = lib.BatchPlan([torch.from_numpy(w.img).cuda() for w in wls], [4] * 3, [8] * 3)
    lib.lib().fhtdp_debug_inject(3, 0, 2_000_000)
    plan.run()
    with pytest.raises(lib.FhtdpError) as e:
        plan.status()
    assert e.value.code == 4
    plan.run()
    plan.status()
    for i, w in enumerate(wls):
        xo, do, so = oracle.detect(w.img, 4, 8)
        assert list(plan.x[i].cpu().numpy()) == list(xo)
