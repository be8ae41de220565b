"""GPU parity of the persistent segment worklist.

Below the level where the level loop hands over, Alg. 1's recursion runs in
one persistent kernel: partition tasks of the big segments (Sec. 3's
classification and compaction, the children's farthest points of Sec. 4)
and small segments finished in shared memory, a child starting as soon as
its parent's last task is done.  Neither the hull nor the per-level
counters may depend on where the handover happens: never (the level loop to
the end), at a middle level, or at level 0 (the whole recursion in the
worklist, including level-0 segments that read the caller's arrays).
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

NEVER, MIDDLE, LEVEL0 = 0, 1 << 16, 1 << 40


@pytest.fixture(scope="module")
def vq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_09417_gb300 as v
    v.load()
    return v


@pytest.fixture(autouse=True)
def _default_config(vq):
    cfg = vq.vq_get_config()
    yield
    vq.vq_set_config(cfg)


def gpu_hull(vq, x, y):
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float64)).cuda()
    return vq.vq_hull2d(xd, yd).cpu().numpy()


def same_stats(gs, st):
    assert gs["levels"] == st["levels"]
    assert gs["read"] == st["read"]
    assert gs["written"] == st["written"]
    assert gs["segments"] == st["segments"]


@pytest.mark.parametrize("dist", synth.DISTRIBUTIONS)
@pytest.mark.parametrize("n", [3, 1000, 70_001, 1_000_000])
def test_handover_level(vq, dist, n):
    """Every handover level, with and without the pre-filter: the oracle's
    hull, and (plain Alg. 1 counts) the oracle's per-level counters."""
    x, y = synth.points(dist, n, 7000 + n)
    want, st = oracle.hull(x, y, stats=True)
    for pre in (0, 1):
        for wl in (NEVER, MIDDLE, LEVEL0):
            vq.vq_set_config(worklist_points=wl, prefilter=pre)
            got = gpu_hull(vq, x, y)
            assert got.shape == want.shape and np.array_equal(got, want), (pre, wl)
            if pre == 0:
                same_stats(vq.vq_last_stats(), st)


@pytest.mark.parametrize("small_max", [2, 64, 1024])
@pytest.mark.parametrize("ppt", [8, 16])
def test_thresholds(vq, small_max, ppt):
    """Small-segment thresholds down to 2 (every segment of three points or
    more is a big one: many tiny partition tasks) and both tile sizes."""
    for dist, n in (("disk", 300_000), ("circle", 50_000), ("kuzmin", 123_457)):
        x, y = synth.points(dist, n, 9 + small_max + ppt)
        want, st = oracle.hull(x, y, stats=True)
        vq.vq_set_config(points_per_thread=ppt, small_max=small_max, worklist_points=LEVEL0, prefilter=0)
        got = gpu_hull(vq, x, y)
        assert np.array_equal(got, want), (dist, small_max, ppt)
        same_stats(vq.vq_last_stats(), st)


def test_degenerate_inputs(vq):
    """Coincident, collinear and duplicated points through the worklist."""
    vq.vq_set_config(worklist_points=LEVEL0)
    rng = np.random.default_rng(5)
    cases = [
        (np.zeros(5000), np.zeros(5000)),
        (np.arange(7000, dtype=np.float64), 2.0 * np.arange(7000, dtype=np.float64)),
        tuple(np.repeat(np.stack(synth.points("circle", 3000, 1)), 3, axis=1)),
        (np.round(rng.random(200_000) * 64) / 64, np.round(rng.random(200_000) * 64) / 64),
    ]
    for x, y in cases:
        assert np.array_equal(gpu_hull(vq, x, y), oracle.hull(x, y))


def test_fp64_tier(vq):
    """Coordinates of 2^45 and more (outside the FP32 tier): the worklist's
    FP64-key partition tasks and finisher."""
    x, y = synth.points("disk", 400_000, 77)
    x = x * 2.0 ** 45 + 3.0
    y = y * 2.0 ** 45 - 5.0
    vq.vq_set_config(worklist_points=LEVEL0, prefilter=0)
    assert np.array_equal(gpu_hull(vq, x, y), oracle.hull(x, y))


def test_batched(vq):
    """Sets of every distribution and of uneven sizes in one call, handed
    over at level 0 and at a middle level."""
    x, y, offs, _ = synth.batched_sets(nsets=48, lo=64, hi=400_000, seed=47)
    for wl in (LEVEL0, MIDDLE):
        vq.vq_set_config(worklist_points=wl)
        hi, ho = vq.vq_hull2d_batched(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(),
                                      torch.from_numpy(offs).cuda())
        hi, ho = hi.cpu().numpy(), ho.cpu().numpy()
        for s in range(48):
            a, b = offs[s], offs[s + 1]
            assert np.array_equal(hi[ho[s]:ho[s + 1]], oracle.hull(x[a:b], y[a:b])), (wl, s)


def test_queue_overflow_reruns(vq):
    """A queue too small for the recursion: the call runs again with the
    level loop alone and still returns the oracle's hull."""
    x, y = synth.points("disk", 1_000_000, 3)
    want = oracle.hull(x, y)
    vq.vq_set_config(worklist_points=LEVEL0, prefilter=0)
    os.environ["VQ_WL_QUEUE_CAP"] = "40"
    try:
        vq.vq_profile_read(reset=True)
        got = gpu_hull(vq, x, y)
        assert vq.vq_profile_read()["worklist_reruns"] == 1
    finally:
        del os.environ["VQ_WL_QUEUE_CAP"]
    assert np.array_equal(got, want)
    vq.vq_profile_read(reset=True)
    assert np.array_equal(gpu_hull(vq, x, y), want)
    assert vq.vq_profile_read()["worklist_reruns"] == 0


def test_repeated_calls_and_layouts(vq):
    """Calls of different sizes in turn (the queue's tags move with the
    workspace layout) and repeated calls of one size (new epochs)."""
    vq.vq_set_config(worklist_points=LEVEL0)
    pts = [synth.points(d, n, 11 + n) for d, n in (("square", 250_000), ("disk", 60_000), ("kuzmin", 250_000))]
    want = [oracle.hull(x, y) for x, y in pts]
    for _ in range(3):
        for (x, y), h in zip(pts, want):
            assert np.array_equal(gpu_hull(vq, x, y), h)


def test_profile_times_the_worklist(vq):
    """With per-kernel timing on, the worklist's time is reported (the
    level loop's kernels still launch at level 0, and find nothing to do)."""
    x, y = synth.points("disk", 1_000_000, 2)
    vq.vq_set_config(worklist_points=LEVEL0, profile=1)
    vq.vq_profile_read(reset=True)
    assert np.array_equal(gpu_hull(vq, x, y), oracle.hull(x, y))
    p = vq.vq_profile_read()
    assert p["k5_ms"] > 0.0
