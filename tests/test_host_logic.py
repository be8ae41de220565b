"""Host-side arithmetic that the device code relies on, checked on the CPU.

* The finalize kernel's fallback visits, for a segment spanning tiles
  [tb, te), the last tile of every partition warp's run inside it.  The
  partition kernel splits T tiles over nw warps as [T g / nw, T (g+1) / nw);
  the warp holding tile u is g = ceil((u + 1) nw / T) - 1.  The closed form
  is compared with a brute-force walk over all warps.
* The partition kernel widens FP32 bounds to FP64 with integer operations
  (rebias the exponent, renormalise subnormals).  The same bit construction
  is compared with numpy's float32 -> float64 conversion.
"""
import random

import numpy as np


def runs_closed(T, nw, tb, te):
    g0 = min(nw - 1, ((tb + 1) * nw + T - 1) // T - 1)
    g1 = min(nw - 1, (te * nw + T - 1) // T - 1)
    out = []
    for g in range(g0, g1 + 1):
        b, e = T * g // nw, T * (g + 1) // nw
        last = min(e, te) - 1
        if last < max(b, tb):
            continue
        out.append(last)
    return out


def runs_brute(T, nw, tb, te):
    out = []
    for g in range(nw):
        b, e = T * g // nw, T * (g + 1) // nw
        lo, hi = max(b, tb), min(e, te)
        if hi > lo:
            out.append(hi - 1)
    return out


def test_run_enumeration_matches_brute_force():
    rng = random.Random(1)
    for _ in range(20000):
        T = rng.randint(1, 300)
        nw = rng.randint(1, 400)
        tb = rng.randint(0, T - 1)
        te = rng.randint(tb + 1, T)
        assert runs_closed(T, nw, tb, te) == runs_brute(T, nw, tb, te), (T, nw, tb, te)


def widen_bits(u):
    """The integer construction of the device's f2d_exact, on uint32 bits."""
    s = (u >> 31) << 63
    e = (u >> 23) & 0xFF
    m = u & 0x7FFFFF
    if e == 0xFF:
        b = 0x7FF0000000000000 | (m << 29)
    elif e != 0:
        b = ((e + 896) << 52) | (m << 29)
    elif m == 0:
        b = 0
    else:
        p = m.bit_length() - 1
        b = ((p + 874) << 52) | ((m - (1 << p)) << (52 - p))
    return s | b


def test_float_widening_bits():
    rng = np.random.default_rng(3)
    special = [0, 1, 2, 0x3FF, 0x7FFFFF, 0x800000, 0x800001, 0x3F800000, 0x7F7FFFFF, 0x7F800000,
               0x7FC00000, 0x7F800001]
    us = np.array(special + [u | 0x80000000 for u in special] +
                  list(rng.integers(0, 2**32, 200000, dtype=np.uint64)), dtype=np.uint64)
    f = us.astype(np.uint32).view(np.float32)
    want = f.astype(np.float64).view(np.uint64)
    for u, wnt, fv in zip(us.tolist(), want.tolist(), f.tolist()):
        got = widen_bits(int(u))
        if np.isnan(fv):
            assert (got >> 52) & 0x7FF == 0x7FF and got & ((1 << 52) - 1), hex(u)
        else:
            assert got == wnt, hex(u)


def trunc_f32_bits(v):
    """The device's FP64 -> FP32 truncation, the same integer construction:
    top 23 fraction bits kept, exponent rebiased; magnitudes below 2^-126 go
    to exactly -2^-126 (negative values) or +2^-126 (positive and zeros)."""
    b = np.asarray(v, dtype=np.float64).view(np.uint64)
    hi = (b >> np.uint64(32)) & np.uint64(0xffffffff)
    lo = b & np.uint64(0xffffffff)
    a = hi & np.uint64(0x7fffffff)
    shifted = (((a << np.uint64(32)) | lo) >> np.uint64(29)) & np.uint64(0xffffffff)
    f = np.where(a < np.uint64(0x38100000), np.uint64(0x00800000),
                 (shifted - np.uint64(0xC0000000)) & np.uint64(0xffffffff))
    neg = np.where((a | lo) != 0, hi & np.uint64(0x80000000), np.uint64(0))
    return (f | neg).astype(np.uint32).view(np.float32)


def test_truncation_is_monotone_with_its_bound():
    """The level-0 pre-filter compares truncated coordinates with truncated
    thresholds and concludes x > t from trunc(x) > trunc(t): that needs the
    truncation to be monotone, including below 2^-126 and at both zeros.
    The FP32 tier's bound |v~ - v| <= 2^-23 |v| + 2^-125 must hold too."""
    rng = np.random.default_rng(3)
    mags = 10.0 ** rng.uniform(-320, 36, 400_000)
    vals = np.concatenate([mags * rng.choice([-1.0, 1.0], mags.size),
                           [0.0, -0.0, 2.0 ** -126, -2.0 ** -126, 2.0 ** -127, -2.0 ** -127,
                            5e-324, -5e-324, 1.0, -1.0, 2.0 ** 39, -2.0 ** 39]])
    vals = vals[np.isfinite(vals)]
    v = np.sort(vals)
    t = trunc_f32_bits(v).astype(np.float64)
    assert np.all(np.diff(t) >= 0)
    assert np.all(np.abs(t - v) <= np.abs(v) * 2.0 ** -23 + 2.0 ** -125)
    # equal doubles (the two zeros) truncate alike
    assert trunc_f32_bits(np.array([0.0]))[0] == trunc_f32_bits(np.array([-0.0]))[0]
    # the contrapositive the filter uses: trunc(x) > trunc(t) implies x > t
    x = rng.choice(v, 200_000)
    y = rng.choice(v, 200_000)
    gt = trunc_f32_bits(x) > trunc_f32_bits(y)
    assert np.all(x[gt] > y[gt])


def test_prefilter_triple_index():
    """The finalize kernel stores the orientation of the triple (i < j < k)
    of five chain positions at base_i[i] + base_j[j] - base_j[i + 1] + k - j - 1;
    that must enumerate the ten triples in lexicographic order."""
    import itertools
    base_i = [0, 6, 9, 10]
    base_j = [0, 0, 3, 5, 6]
    for t, (i, j, k) in enumerate(itertools.combinations(range(5), 3)):
        assert base_i[i] + (base_j[j] - base_j[i + 1]) + (k - j - 1) == t


def test_strictly_right_of_every_edge_means_strictly_inside():
    """The lemma behind dropping points at level 0: a point strictly right
    of every directed edge of a closed polygon (any vertex order, convex or
    not) lies strictly inside the convex hull of its vertices.  Checked in
    exact rational arithmetic on random small polygons and random points."""
    from fractions import Fraction as F

    def orient(a, b, c):
        v = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        return (v > 0) - (v < 0)

    def hull_strict_inside(pts, u):
        # u strictly inside conv(pts) iff for every pair (a, b) with all
        # points on one closed side, u is strictly on that side
        n = len(pts)
        for i in range(n):
            for j in range(n):
                if pts[i] == pts[j]:
                    continue
                s = [orient(pts[i], pts[j], p) for p in pts]
                if all(x <= 0 for x in s) and orient(pts[i], pts[j], u) >= 0:
                    return False
        return True

    rng = random.Random(5)
    found = 0
    for _ in range(8000):
        k = rng.randint(3, 8)
        poly = [(F(rng.randint(-6, 6)), F(rng.randint(-6, 6))) for _ in range(k)]
        u = (F(rng.randint(-12, 12), 2), F(rng.randint(-12, 12), 2))
        if all(orient(poly[i], poly[(i + 1) % k], u) < 0 for i in range(k)):
            found += 1
            assert hull_strict_inside(poly, u), (poly, u)
    assert found > 50


def test_server_admission_policy(tmp_path):
    """The serving handle's host policies (vq_admit.h): admission (the
    longest FIFO prefix within the free request slots and the memory budget,
    the server's fixed reserve included; nothing when the head does not fit)
    and the pinned staging area's first-fit extents.  Compiled with the host
    compiler."""
    import os
    import shutil
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        import pytest
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "admit_check"
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-I", os.path.join(root, "paper_2510_09417_gb300", "csrc"),
                           os.path.join(root, "tests", "admit_check.cpp"), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {l.split()[0]: tuple(int(v) for v in l.split()[1:]) for l in out if l.strip()}
    assert got["all"] == (4, 1000, 68 * 1000 + 4000)
    assert got["slots"] == (2, 300, 68 * 300 + 2000)
    assert got["no_slot"] == (0, 0, 0)
    assert got["budget"] == (2, 300, 68 * 300 + 2000)
    assert got["head_too_big"] == (0, 0, 0)
    assert got["empty"] == (0, 0, 0)
    assert got["reserve_fits"] == (2, 300, 68 * 300 + 2000)
    assert got["reserve_short"] == (1, 100, 68 * 100 + 1000)
    # a lane's batch stops before the request that would take it past
    # max(cap, head's points); a big head runs alone
    assert got["batch_cap"] == (3, 600)
    assert got["batch_big_head"] == (1, 5000)
    assert got["batch_all"] == (5, 5650)
    assert got["batch_none"] == (0, 0)
    # pinned staging extents: three of 300 fit in 1000 (first fit: 0, 300,
    # 600), a fourth does not; a freed hole of 300 cannot hold 301; returning
    # everything merges into one extent of 1000
    assert got["ext_take"] == (1, 1, 1, 0, 0, 300, 600, 100)
    assert got["ext_hole"] == (0, 2, 300)
    assert got["ext_merge"] == (1, 1000)
