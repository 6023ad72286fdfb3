"""Host-side logic of bench.py that needs no GPU: the workload table, the
synthetic items of every workload, the oracle dispatch of the CPU baseline,
and the reference arm (the oracle) end to end."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_workload_is_described():
    for name, spec in bench.WORKLOADS.items():
        assert spec["desc"] and spec["images"] >= 1 and spec["dtype"] in ("u8", "f32"), name


@pytest.mark.parametrize("name", ["plain256", "through2048", "two2048", "padded2048",
                                  "horizontal2048"])
def test_workload_items_have_the_expected_form(name):
    items = bench.make_workload(name, 1, 0, 0)
    assert len(items) == 1
    img, k, B = items[0]
    h, w = img.shape
    assert img.dtype == np.uint8 and h % k == 0
    if name == "through2048":
        B_, j, xp = B
        assert j == bench.THROUGH_BORDER and 0 <= xp < w and B_ >= 0
    elif name == "two2048":
        assert B[0] == "two" and B[2] == bench.TWO_SEPARATION
    elif name == "padded2048":
        assert B[0] == "padded" and B[1] >= 0
    else:
        assert isinstance(B, int)


def test_ranks_take_different_images():
    a = bench.make_workload("plain256", 2, 0, 0)
    b = bench.make_workload("plain256", 2, 0, 1)
    assert not np.array_equal(a[0][0], b[0][0])


def test_oracle_rate_dispatches_every_kind():
    rng = np.random.default_rng(0)
    img = rng.integers(0, 256, (32, 32)).astype(np.uint8)
    kinds = [(img, 4, None), (img, 4, ("two", 2, 4)), (img, 4, ("padded", 2)), (img, 4, (2, 1, 5)),
             (img, 4, 2), (img.astype(np.float32), 4, 2)]
    rate, done = bench.oracle_rate(kinds, 1e9)
    assert done == len(kinds) and rate > 0
    rate, done = bench.oracle_rate([(img, 4, 2)], 1e9, horizontal=True)
    assert done == 1 and rate > 0


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "plain256", "--steps", "2", "--warmup", "1"], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Mpix/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["higher_is_better"] is True and d["metric"] == bench.METRIC


def test_all_core_oracle_leg_runs_images_on_threads():
    items = bench.make_workload("plain256", 4, 3, 0)
    rate, done = bench.oracle_rate_threads(items, 2)
    assert done == 4 and rate > 0
    assert bench.host_threads() >= 1
    assert isinstance(bench.cpu_model(), str)


def test_mixed_workload_is_the_default_and_spans_every_band_height():
    args = sys.argv
    try:
        sys.argv = ["bench.py"]
        assert bench.parse().workload == "mixed"
    finally:
        sys.argv = args
    from paper_1912_01884_gb300 import synth
    ns = {h // k for h, w, k, B in synth.mixed_batch_shapes(0, 256)}
    assert ns == {32, 64, 128, 256}


def test_clock_sampler_without_a_gpu_reports_why():
    s = bench.ClockSampler(0)
    s.start()
    r = s.stop()
    assert "reasons" in r
