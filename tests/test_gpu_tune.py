"""GPU test of the autotuner: it picks one of its candidate configurations,
installs it, and the hull under the chosen configuration still equals the
oracle's."""
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
        now = vq.vq_get_config()
        assert (now.points_per_thread, now.small_max, now.prefilter) == \
            (cfg.points_per_thread, cfg.small_max, cfg.prefilter)
        assert now.timeout_ns == before.timeout_ns
        got = vq.vq_hull2d(xd, yd).cpu().numpy()
        assert np.array_equal(got, oracle.hull(x, y))
    finally:
        vq.vq_set_config(before)
