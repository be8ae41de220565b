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
