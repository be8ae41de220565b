"""Seeded synthetic point sets for the planar hull workloads.

This module only draws inputs. It holds none of the hull arithmetic, and both
the CPU oracle and the CUDA path take their inputs from here.

The distributions stand in for the three 1e8-point evaluation sets that the
paper takes from PBBS (Sec. 5.2 "The Datasets"): Kuzmin, points on a circle,
and points in a disk. A uniform square is added as the plain case. Those
files are not available here, so the sets are regenerated from their
definitions with a seeded counter-based generator.

Random bits come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014). Value i of stream (seed, k)
is mix64(base(seed, k) + (i + 1) * GAMMA), so any slice can be regenerated
on its own. A uniform double in [0, 1) is (bits >> 11) * 2**-53.

Coordinates are FP64 in structure-of-arrays layout, which is the layout the
paper uses (Sec. 5.4).
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53_INV = 1.0 / 9007199254740992.0

DISTRIBUTIONS = ("square", "disk", "circle", "kuzmin")

# Seeds of the five measured workloads (single hulls, batched sets, serving).
WORKLOAD_SEEDS = {
    ("square", 1_000_000): 1,
    ("square", 100_000_000): 1,
    ("disk", 100_000_000): 2,
    ("circle", 100_000_000): 3,
    ("kuzmin", 100_000_000): 4,
}
BATCHED_SEED = 5
SERVING_SEED = 6

_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _stream_base(seed: int, stream: int) -> np.uint64:
    key = np.array([((int(seed) & 0xFFFFFFFFFFFF) << 16) | (int(stream) & 0xFFFF)], dtype=np.uint64)
    return _mix64(key)[0]


def splitmix_bits(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Raw 64-bit words i = start .. start+count-1 of stream (seed, stream)."""
    base = _stream_base(seed, stream)
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = base + i * GAMMA
    return _mix64(z)


def uniform01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Doubles k * 2**-53, k uniform in [0, 2**53)."""
    bits = splitmix_bits(seed, stream, start, count)
    return (bits >> np.uint64(11)).astype(np.float64) * _TWO53_INV


def _fill(dist: str, seed: int, x: np.ndarray, y: np.ndarray, start: int) -> None:
    m = x.shape[0]
    u0 = uniform01(seed, 0, start, m)
    if dist == "square":
        x[:] = u0
        y[:] = uniform01(seed, 1, start, m)
    elif dist == "circle":
        theta = (2.0 * math.pi) * u0
        np.cos(theta, out=x)
        np.sin(theta, out=y)
    elif dist == "disk":
        r = np.sqrt(u0)
        theta = (2.0 * math.pi) * uniform01(seed, 1, start, m)
        np.multiply(r, np.cos(theta), out=x)
        np.multiply(r, np.sin(theta), out=y)
    elif dist == "kuzmin":
        one_minus = 1.0 - u0
        r = np.sqrt(1.0 / (one_minus * one_minus) - 1.0)
        theta = (2.0 * math.pi) * uniform01(seed, 1, start, m)
        np.multiply(r, np.cos(theta), out=x)
        np.multiply(r, np.sin(theta), out=y)
    else:
        raise ValueError(f"unknown distribution {dist!r}")


def points(dist: str, n: int, seed: int, out_x: np.ndarray | None = None,
           out_y: np.ndarray | None = None, workers: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """n FP64 points of `dist` as two contiguous arrays (x, y).

    square: (u, u') in [0,1)^2.  disk: r = sqrt(u), theta = 2*pi*u'.
    circle: (cos theta, sin theta), theta = 2*pi*u.
    kuzmin: r = sqrt(1/(1-u)^2 - 1), theta = 2*pi*u'.
    workers > 1 fills chunks on that many threads (numpy releases the GIL in
    its array loops); every value depends only on its index, so the output
    is the same for any worker count.
    """
    n = int(n)
    x = np.empty(n, dtype=np.float64) if out_x is None else out_x
    y = np.empty(n, dtype=np.float64) if out_y is None else out_y
    starts = range(0, n, _CHUNK)
    if workers > 1 and n > _CHUNK:
        with ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(lambda s: _fill(dist, seed, x[s:min(n, s + _CHUNK)], y[s:min(n, s + _CHUNK)], s), starts))
    else:
        for s in starts:
            _fill(dist, seed, x[s:min(n, s + _CHUNK)], y[s:min(n, s + _CHUNK)], s)
    return x, y


def workload(dist: str, n: int, workers: int = 1) -> tuple[np.ndarray, np.ndarray]:
    """One of the named single-hull workloads with its fixed seed."""
    return points(dist, n, WORKLOAD_SEEDS[(dist, int(n))], workers=workers)


def batched_sets(nsets: int = 4096, lo: int = 64, hi: int = 1_000_000,
                 seed: int = BATCHED_SEED, workers: int = 1):
    """Independent sets with sizes log-uniform in [lo, hi].

    Set s has size round(exp(ln lo + u * ln(hi/lo))) and a distribution drawn
    uniformly from the four above; its points use seed (seed << 20) + s.
    Returns (x, y, offsets int64[nsets+1], dists list).
    """
    u = uniform01(seed, 0, 0, nsets)
    pick = uniform01(seed, 1, 0, nsets)
    sizes = np.rint(np.exp(math.log(lo) + u * math.log(hi / lo))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    dists = [DISTRIBUTIONS[min(3, int(p * 4))] for p in pick]
    offsets = np.zeros(nsets + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    x = np.empty(total, dtype=np.float64)
    y = np.empty(total, dtype=np.float64)

    def fill(s):
        a, b = int(offsets[s]), int(offsets[s + 1])
        points(dists[s], b - a, (seed << 20) + s, x[a:b], y[a:b])

    if workers > 1:
        with ThreadPoolExecutor(max_workers=workers) as ex:
            list(ex.map(fill, range(nsets)))
    else:
        for s in range(nsets):
            fill(s)
    return x, y, offsets, dists


def serving_requests(count: int, rate_per_s: float, lo: int = 100,
                     hi: int = 10_000_000, seed: int = SERVING_SEED):
    """Poisson arrivals of hull requests.

    Returns a list of dicts {t: arrival seconds, n, dist, seed}. Inter-arrival
    gaps are exponential with mean 1/rate; sizes are log-uniform in [lo, hi].
    The points of request i are points(dist, n, seed) and are drawn by the
    caller when it submits.
    """
    g = uniform01(seed, 0, 0, count)
    u = uniform01(seed, 1, 0, count)
    pick = uniform01(seed, 2, 0, count)
    gaps = -np.log1p(-g) / float(rate_per_s)
    t = np.cumsum(gaps)
    sizes = np.clip(np.rint(np.exp(math.log(lo) + u * math.log(hi / lo))), lo, hi).astype(np.int64)
    out = []
    for i in range(count):
        out.append({"t": float(t[i]), "n": int(sizes[i]),
                    "dist": DISTRIBUTIONS[min(3, int(pick[i] * 4))],
                    "seed": (seed << 24) + i})
    return out
