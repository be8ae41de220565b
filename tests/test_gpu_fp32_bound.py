"""GPU pin of the FP32 tier's error bound.

Almost every point of every level is classified by the FP32 tier of the
exact left-of test (Sec. 2.1): orient(a, b, u) evaluated in FP32 on the
line's truncated origin and rounded direction and on the point truncated to
24 bits, with a per-point bound E.  The tier decides a sign only when
|d| > E, so every hull claimed exact rests on |d - orient| <= E.  This test
runs the device's own evaluation (vq_debug_orient_f32, the code the kernels
inline) on more than a million near-degenerate triples and checks the bound
against the exact orient, computed by the oracle's big-integer sums.
"""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2510_09417_gb300 as v
    v.load()
    return v


def near_degenerate_triples(rng, m):
    """(m, 6) triples a, b, u with every |coordinate| < 2^40: points on or a
    few ulps off the line a->b at magnitudes 2^-60 .. 2^39, directions of a
    few ulps (FP32 direction subnormal or zero), a far origin with a short
    direction, lattice points, and generic points."""
    k = rng.integers(-60, 40, m)
    s = np.ldexp(1.0, k)[:, None]
    kind = rng.integers(0, 6, m)
    a = (rng.random((m, 2)) * 2 - 1) * s
    b = (rng.random((m, 2)) * 2 - 1) * s
    # short directions: b a few ulps (of a) away from a
    short = kind == 1
    b[short] = a[short] + rng.integers(-3, 4, (short.sum(), 2)) * np.spacing(np.abs(a[short]))
    # a far origin and a direction many orders of magnitude shorter
    far = kind == 2
    a[far] = (rng.random((far.sum(), 2)) * 2 - 1) * 2.0 ** 39
    b[far] = a[far] + (rng.random((far.sum(), 2)) * 2 - 1) * np.ldexp(1.0, rng.integers(-30, 10, (far.sum(), 1)))
    # lattice points up to 2^39, u on the lattice line
    lat = kind == 3
    g = rng.integers(-(1 << 20), 1 << 20, (lat.sum(), 2)).astype(np.float64)
    step = rng.integers(-(1 << 18), 1 << 18, (lat.sum(), 2)).astype(np.float64)
    a[lat] = g
    b[lat] = g + step
    w = rng.random(m) * 1.5 - 0.25
    u = a + w[:, None] * (b - a)
    u[lat] = a[lat] + rng.integers(-4, 5, (lat.sum(), 1)) * (b[lat] - a[lat])
    # a few ulps off the line (not for the generic kind)
    near = kind != 5
    u[near] += rng.integers(-4, 5, (near.sum(), 2)) * np.spacing(np.abs(u[near]))
    gen = kind == 5
    u[gen] = (rng.random((gen.sum(), 2)) * 2 - 1) * s[gen]
    tri = np.concatenate([a, b, u], axis=1)
    tri = np.where(np.abs(tri) < 2.0 ** 40, tri, np.copysign(2.0 ** 39, tri))
    return tri


def test_fp32_tier_bound_holds(vq):
    rng = np.random.default_rng(2510)
    tri = near_degenerate_triples(rng, 1_200_000)
    assert np.all(np.isfinite(tri)) and np.all(np.abs(tri) < 2.0 ** 40)
    d, e = vq.vq_debug_orient_f32(torch.from_numpy(tri).cuda())
    d, e = d.cpu().numpy(), e.cpu().numpy()
    assert np.all(np.isfinite(d)) and np.all(e >= 0)
    out, bad = oracle.orient_bound_check(tri, d, e)
    assert out == 0, f"{out} triples with |d - orient| > E"
    assert bad == 0, f"{bad} signs claimed wrong"
    # the test reaches both sides of the margin: many decided (mostly the
    # generic sixth of the triples), most of the near-degenerate ones not
    decided = np.abs(d) > e
    assert 0.1 < decided.mean() < 0.9, decided.mean()
