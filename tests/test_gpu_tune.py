"""GPU tests of the autotuner and of the partition kernel's block shapes:
the autotuner picks one of its candidate configurations (points per lane,
small-segment threshold, pre-filter, block shape), installs it, and the hull
under the chosen configuration still equals the oracle's; every block shape
gives the oracle's hull."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_09417_gb300 as v
    v.load()
    return v


def test_autotune(vq):
    before = vq.vq_get_config()
    try:
        x, y = synth.points("disk", 2_000_000, 91)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        cfg, ms = vq.vq_autotune(xd, yd, reps=2)
        assert ms > 0
        assert cfg.points_per_thread in (8, 16)
        assert cfg.small_max in (256, 1024)
        assert cfg.prefilter in (0, 1)
        assert cfg.k1_shape in (0, 1, 2)
        now = vq.vq_get_config()
        assert (now.points_per_thread, now.small_max, now.prefilter, now.k1_shape) == \
            (cfg.points_per_thread, cfg.small_max, cfg.prefilter, cfg.k1_shape)
        assert now.timeout_ns == before.timeout_ns
        got = vq.vq_hull2d(xd, yd).cpu().numpy()
        assert np.array_equal(got, oracle.hull(x, y))
    finally:
        vq.vq_set_config(before)


@pytest.mark.parametrize("ppt", [4, 8, 16])
@pytest.mark.parametrize("shape", [0, 1, 2])
def test_block_shapes(vq, ppt, shape):
    before = vq.vq_get_config()
    try:
        vq.vq_set_config(points_per_thread=ppt, k1_shape=shape, prefilter=0)
        for dist, n in (("disk", 300_000), ("circle", 60_000)):
            x, y = synth.points(dist, n, 17 + shape)
            got = vq.vq_hull2d(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
            assert np.array_equal(got, oracle.hull(x, y)), (dist, ppt, shape)
    finally:
        vq.vq_set_config(before)
