"""The bench's CPU-side contract: the reference arm (the CPU oracle, as the
reference) prints one JSON line with the keys the driver reads, and the
threaded input generation the bench uses gives the same points as the
single-threaded generator."""
import json
import os
import subprocess
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "200000",
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "Gpoints/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_threaded_generation_is_identical():
    a = synth.points("kuzmin", (1 << 22) + 12345, 8)
    b = synth.points("kuzmin", (1 << 22) + 12345, 8, workers=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    x1, y1, o1, d1 = synth.batched_sets(nsets=40, lo=64, hi=50_000, seed=9)
    x2, y2, o2, d2 = synth.batched_sets(nsets=40, lo=64, hi=50_000, seed=9, workers=4)
    assert np.array_equal(o1, o2) and d1 == d2
    assert np.array_equal(x1, x2) and np.array_equal(y1, y2)


def test_cpu_batched_baseline_sample():
    """The batched section's CPU baseline: a bounded prefix of the sets, each
    hulled by the oracle on a thread pool."""
    sys.path.insert(0, ROOT)
    import bench
    x, y, offs, _ = synth.batched_sets(nsets=64, lo=64, hi=20_000, seed=4)
    r = bench.cpu_batched_baseline(x, y, offs, max_points=100_000)
    k = int(r["sample"].split()[2])
    assert 1 <= k <= 64 and int(offs[k]) <= 100_000 or k == 1
    assert r["hulls_per_s"] > 0 and r["cores"] >= 1 and r["kind"] == "oracle"


def test_clock_sampler_summary():
    """nvidia-smi csv lines (no header, no units) reduce to the median SM
    clock and power, the ceiling and the active throttle reasons of one GPU;
    unparsable power readings are skipped, other GPUs' lines ignored."""
    sys.path.insert(0, ROOT)
    import bench
    lines = [
        "0, 1900, 2070, 700.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2000, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
        "1, 500, 2070, 100.0, 0x0, Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    s = bench.ClockSampler.summarize(lines, 0)
    assert s["samples"] == 3 and s["sm_mhz"] == 2000 and s["sm_max_mhz"] == 2070
    assert s["power_w"] == (700.5 + 900.0) / 2
    assert s["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler.summarize(["garbage"], 0) is None
