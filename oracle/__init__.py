"""CPU oracle for the planar Quickhull (VQhull, arxiv 2510.09417).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg are the only callers.  The CUDA library and
its Python binding never import this package, and this package never imports
them.

The arithmetic lives in ``vq_oracle.c`` (sequential Quickhull after Alg. 1,
exact predicates of Sec. 2.1, hull verifier); this module compiles it with
gcc and marshals numpy arrays through ctypes.  ctypes releases the GIL, so
``verify`` splits its O(n log h) scan over a thread pool.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vq_oracle.c")
_LIB = os.path.join(_HERE, f"liborc.{platform.machine()}.so")
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 512

VERIFY_CODES = {
    0: "ok", 1: "count", 2: "index range", 3: "start vertex", 4: "not strictly convex",
    5: "chains not monotone", 6: "point outside", 7: "vertex not lowest index",
    8: "degenerate hull wrong", -4: "out of memory",
}


class Stats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int64),
        ("read", ctypes.c_int64 * MAX_LEVELS),
        ("written", ctypes.c_int64 * MAX_LEVELS),
        ("segments", ctypes.c_int64 * MAX_LEVELS),
        ("exact_calls", ctypes.c_int64),
        ("paper_bytes", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile liborc.so next to its source (gcc, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call([
                "gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    d, i64, i32p = ctypes.c_double, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.orc_orient_sign.argtypes = [d] * 6
    lib.orc_orient_sign.restype = ctypes.c_int
    lib.orc_cross_sign.argtypes = [d] * 8
    lib.orc_cross_sign.restype = ctypes.c_int
    lib.orc_dot_sign.argtypes = [d] * 8
    lib.orc_dot_sign.restype = ctypes.c_int
    lib.orc_set_filter.argtypes = [ctypes.c_int]
    lib.orc_exact_count.restype = ctypes.c_longlong
    lib.orc_hull.argtypes = [dp, dp, i64, i32p, ctypes.POINTER(Stats)]
    lib.orc_hull.restype = i64
    lib.orc_verify.argtypes = [dp, dp, i64, i32p, i64, i64, i64, ctypes.POINTER(i64)]
    lib.orc_verify.restype = ctypes.c_int
    lib.orc_farthest.argtypes = [dp, dp, ctypes.c_int32, ctypes.c_int32, i32p, i64]
    lib.orc_farthest.restype = ctypes.c_int32
    lib.orc_orient_bound_check.argtypes = [dp, i64, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                           ctypes.POINTER(i64)]
    lib.orc_orient_bound_check.restype = i64
    lib.orc_stats_size.restype = i64
    assert lib.orc_stats_size() == ctypes.sizeof(Stats)
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def orient_sign(a, b, c) -> int:
    """Exact sign of orient(a,b,c) = (b-a) x (c-a) (Sec. 2.1 left-of test)."""
    return _load().orc_orient_sign(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                   float(c[0]), float(c[1]))


def cross_sign(p0, p1, q0, q1) -> int:
    """Exact sign of (p1-p0) x (q1-q0) (Sec. 2.1 farther-than test)."""
    v = [float(t) for pt in (p0, p1, q0, q1) for t in pt]
    return _load().orc_cross_sign(*v)


def dot_sign(p0, p1, q0, q1) -> int:
    """Exact sign of (p1-p0) . (q1-q0)."""
    v = [float(t) for pt in (p0, p1, q0, q1) for t in pt]
    return _load().orc_dot_sign(*v)


def farthest(x, y, a: int, b: int, cand) -> int:
    """Farthest of the candidate indices from the line a->b: max orient(a,b,u),
    then the smaller projection on b - a, then the lowest index."""
    lib = _load()
    x, y = _f64(x), _f64(y)
    c = np.ascontiguousarray(cand, dtype=np.int32)
    return int(lib.orc_farthest(_dp(x), _dp(y), int(a), int(b), _ip(c), c.shape[0]))


def orient_bound_check(tri, d, e) -> tuple[int, int]:
    """For triples tri[k] = (ax, ay, bx, by, cx, cy) and approximations d[k]
    with bounds e[k] of orient(a,b,c) (Sec. 2.1 left-of test): the number
    of k whose exact orient lies outside [d - e, d + e], and the number with
    |d| > e whose sign is wrong.  Exact sums of products."""
    t = np.ascontiguousarray(tri, dtype=np.float64).reshape(-1, 6)
    dd = np.ascontiguousarray(d, dtype=np.float32)
    ee = np.ascontiguousarray(e, dtype=np.float32)
    assert dd.shape[0] == ee.shape[0] == t.shape[0]
    bad = ctypes.c_int64(0)
    fp = ctypes.POINTER(ctypes.c_float)
    out = _load().orc_orient_bound_check(_dp(t), t.shape[0], dd.ctypes.data_as(fp), ee.ctypes.data_as(fp),
                                         ctypes.byref(bad))
    return int(out), int(bad.value)


def set_filter(on: bool) -> None:
    """Turn the FP64 error-bound filter in front of the exact sums on or off."""
    _load().orc_set_filter(1 if on else 0)


def hull(x, y, stats: bool = False):
    """Hull vertex indices (int32), clockwise from the lexicographic minimum.

    Raises ValueError on non-finite input.  With stats=True also returns a
    dict of per-level partition counts and the paper's byte model.
    """
    lib = _load()
    x, y = _f64(x), _f64(y)
    n = x.shape[0]
    assert y.shape[0] == n
    out = np.empty(max(n, 1), dtype=np.int32)
    st = Stats()
    h = lib.orc_hull(_dp(x), _dp(y), n, _ip(out), ctypes.byref(st))
    if h == -2:
        raise ValueError("non-finite coordinate")
    if h < 0:
        raise MemoryError("oracle out of memory")
    res = out[:h].copy()
    if not stats:
        return res
    L = int(st.levels)
    info = {
        "levels": L,
        "read": [int(st.read[i]) for i in range(L)],
        "written": [int(st.written[i]) for i in range(L)],
        "segments": [int(st.segments[i]) for i in range(L)],
        "exact_calls": int(st.exact_calls),
        "paper_bytes": float(st.paper_bytes),
    }
    return res, info


def verify(x, y, hull_idx, threads: int | None = None) -> tuple[int, int]:
    """Check a hull against its definition.  Returns (code, bad) with code 0
    when the hull is exactly the strict-vertex hull, clockwise from the
    lowest-index lexicographic minimum, lowest indices at duplicates."""
    lib = _load()
    x, y = _f64(x), _f64(y)
    H = np.ascontiguousarray(hull_idx, dtype=np.int32)
    n = x.shape[0]
    h = H.shape[0]
    if threads is None:
        threads = min(16, os.cpu_count() or 1)
    chunks = max(1, min(threads, n // 200_000 + 1))
    bounds = [(n * k // chunks, n * (k + 1) // chunks) for k in range(chunks)]

    def run(b):
        bad = ctypes.c_int64(-1)
        hp = _ip(H) if h > 0 else ctypes.POINTER(ctypes.c_int32)()
        rc = lib.orc_verify(_dp(x), _dp(y), n, hp, h, b[0], b[1], ctypes.byref(bad))
        return rc, int(bad.value)

    if chunks == 1:
        return run(bounds[0])
    with ThreadPoolExecutor(max_workers=chunks) as ex:
        for rc, bad in ex.map(run, bounds):
            if rc != 0:
                return rc, bad
    return 0, -1
