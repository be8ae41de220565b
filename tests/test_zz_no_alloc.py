"""vq_hull2d_noalloc: the entry point for callers that cannot allocate.

It must give exactly the hull of vq_hull2d (the allocating entry point) on
consecutive calls, although every call reuses the same fixed device array
and starts from whatever the previous call left there.  Collected last, so
that a run stopping at its first failure has already run every other test;
it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_09417_gb300 as v
    v.load()
    return v


def _noalloc_via_cabi(lib, xd, yd, out):
    h = ctypes.c_int64(-1)
    st = lib.vq_hull2d_noalloc(xd.data_ptr(), yd.data_ptr(), xd.shape[0], out.data_ptr(), ctypes.byref(h),
                               torch.cuda.current_stream().cuda_stream)
    return st, h.value


def test_noalloc_matches_allocating_entry_point(vq):
    lib = vq.load()
    # two calls in a row with different inputs (the second call starts from
    # the first call's leftovers in the shared array), then a repeat
    cases = [("disk", 1_000_000, 2), ("circle", 300_000, 5), ("disk", 1_000_000, 2)]
    for dist, n, seed in cases:
        x, y = synth.points(dist, n, seed)
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        want = vq.vq_hull2d(xd, yd).cpu().numpy()
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        st, h = _noalloc_via_cabi(lib, xd, yd, out)
        assert st == 0, vq.status_string(st)
        got = out[:h].cpu().numpy()
        assert np.array_equal(got, want), (dist, n, h, want.shape[0])


def test_noalloc_limits(vq):
    lib = vq.load()
    h = ctypes.c_int64(-1)
    # beyond the fixed array: rejected before any device work
    assert lib.vq_hull2d_noalloc(1, 1, (1 << 20) + 1, 1, ctypes.byref(h), None) == -3
    assert lib.vq_hull2d_noalloc(None, None, 0, None, ctypes.byref(h), None) == 0 and h.value == 0
    # the largest accepted size works
    n = 1 << 20
    x, y = synth.points("square", n, 8)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    st, hh = _noalloc_via_cabi(lib, xd, yd, out)
    assert st == 0
    assert np.array_equal(out[:hh].cpu().numpy(), vq.vq_hull2d(xd, yd).cpu().numpy())
