"""GPU pin of the FP32 tier's error bound.

Almost every point of every level is classified by the FP32 tier of the
exact left-of test (Sec. 2.1): orient(a, b, u) evaluated in FP32 on the
line's truncated origin and rounded direction and on the point truncated to
24 bits, with a per-point bound E.  The tier decides a sign only when
|d| > E, so every hull claimed exact rests on |d - orient| <= E.  This test
runs the device's own evaluation (vq_debug_orient_f32, the code the kernels
inline) on more than a million near-degenerate triples and checks the bound
against the exact orient, computed by the oracle's big-integer sums.  The
same holds for the second FP32 tier, which evaluates the test in coordinates
relative to the line's origin for the points the first leaves undecided
(nearly collinear, far from the origin: points on a circle), and which must
decide most of the circle-arc triples that the first cannot.
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
    # a few ulps off the line (not for the generic kind nor the arcs)
    near = (kind != 5) & (kind != 4)
    u[near] += rng.integers(-4, 5, (near.sum(), 2)) * np.spacing(np.abs(u[near]))
    gen = kind == 5
    u[gen] = (rng.random((gen.sum(), 2)) * 2 - 1) * s[gen]
    # points on a circle arc between a and b (hull-dense data: nearly
    # collinear with the chord, far from the origin relative to its length)
    arc = kind == 4
    na = int(arc.sum())
    th = rng.random(na) * 2 * np.pi
    dth = np.ldexp(1.0, rng.integers(-30, -4, na))
    rad = np.ldexp(1.0, rng.integers(-20, 39, na))[:, None]
    ang = np.stack([th, th + dth, th + dth * rng.random(na)], 1)
    pts = np.stack([np.cos(ang), np.sin(ang)], 2) * rad[:, :, None]
    a[arc], b[arc], u[arc] = pts[:, 0], pts[:, 1], pts[:, 2]
    tri = np.concatenate([a, b, u], axis=1)
    tri = np.where(np.abs(tri) < 2.0 ** 40, tri, np.copysign(2.0 ** 39, tri))
    return tri


def test_fp32_tiers_bound_holds(vq):
    """Both FP32 tiers on the same 1.2M triples (tier 0: absolute
    coordinates; tier 1: relative to the line's origin): the bound holds for
    each, and the relative tier decides far more of the circle arcs."""
    rng = np.random.default_rng(2510)
    m = 1_200_000
    tri = near_degenerate_triples(rng, m)
    assert np.all(np.isfinite(tri)) and np.all(np.abs(tri) < 2.0 ** 40)
    arcs = _arc_rows(2510, m)
    got = {}
    for tier in (0, 1):
        d, e = vq.vq_debug_orient_f32(torch.from_numpy(tri).cuda(), tier=tier)
        d, e = d.cpu().numpy(), e.cpu().numpy()
        assert np.all(np.isfinite(d)) and np.all(e >= 0)
        out, bad = oracle.orient_bound_check(tri, d, e)
        assert out == 0, f"tier {tier}: {out} triples with |d - orient| > E"
        assert bad == 0, f"tier {tier}: {bad} signs claimed wrong"
        got[tier] = np.abs(d) > e
    # both sides of the margin are reached: many decided, many not
    assert 0.1 < got[0].mean() < 0.9, got[0].mean()
    # the arcs: the absolute tier decides few, the relative one many
    assert got[1][arcs].mean() > 0.3 and got[1][arcs].mean() > 3 * got[0][arcs].mean(), \
        (got[0][arcs].mean(), got[1][arcs].mean())


def _arc_rows(rng_seed, m):
    """The rows of near_degenerate_triples(default_rng(rng_seed), m) that
    are circle arcs (the generator draws the kinds first)."""
    rng = np.random.default_rng(rng_seed)
    rng.integers(-60, 40, m)
    return rng.integers(0, 6, m) == 4


def test_round_f32_is_ieee_nearest_even(vq):
    """The FP32 tiers round FP64 differences to FP32 with integer operations;
    the result must be IEEE 754 round-to-nearest-even, bit for bit (numpy's
    float64 -> float32 cast is that rounding): normal values, exact ties at
    the 29 dropped bits, values at and across the subnormal boundary, FP32
    overflow, signed zeros, infinities and NaNs."""
    rng = np.random.default_rng(77)
    m = 1 << 20
    e = rng.integers(-160, 130, m)
    v = np.ldexp(rng.random(m) + 0.5, e) * np.where(rng.random(m) < 0.5, -1.0, 1.0)
    # ties and near-ties: FP32 values plus exactly half an FP32 ulp (+- 1 FP64 ulp)
    f = rng.standard_normal(m // 4).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    half = (f.astype(np.float64) + up) / 2
    ties = np.concatenate([half, np.nextafter(half, np.inf), np.nextafter(half, -np.inf)])
    # the subnormal range and its boundary, and rounding that carries
    sub = np.ldexp(rng.random(m // 4), rng.integers(-152, -124, m // 4))
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028234663852886e38, 3.4028235677973366e38,
                        3.4028235677973362e38, -3.4028236e38, 2.0 ** -149, 2.0 ** -150, 2.0 ** -150 * 1.0000001,
                        2.0 ** -126, 2.0 ** -126 * (1 - 2.0 ** -25), 1.0 - 2.0 ** -25, 1.0 + 2.0 ** -24,
                        1.0 + 3 * 2.0 ** -24, 5e-324, -5e-324, 2.0 ** -1022])
    x = np.concatenate([v, ties, sub, -sub, special])
    got = vq.vq_debug_round_f32(torch.from_numpy(x).cuda()).cpu().numpy()
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(got), nan)
    gb, wb = got.view(np.uint32)[~nan], want.view(np.uint32)[~nan]
    bad = np.flatnonzero(gb != wb)
    assert bad.size == 0, (x[~nan][bad[:5]], gb[bad[:5]], wb[bad[:5]])
