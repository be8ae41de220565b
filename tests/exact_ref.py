"""Independent exact references used to pin the oracle (CPU, pure Python).

Nothing here is shared with the oracle or with the CUDA path.  Coordinates
are turned into Python integers on a common binary scale (every finite double
is an integer times 2**e), so every predicate below is exact integer
arithmetic.  Two hull constructions follow from the definition of the
result rather than from Quickhull:

* ``brute_hull``: O(n^3) edge test.  A pair (i, j) of distinct sites is a
  clockwise hull edge iff no site lies strictly to its left and every site
  on its line lies within the closed segment [i, j].
* ``monotone_chain``: Andrew's monotone chain (Inf. Proc. Letters 9(5),
  1979) over sites sorted by (x, y), keeping strict turns only.

Both return strict vertices, one index per coordinate pair (the lowest),
clockwise with y up, starting at the lexicographic minimum.
"""
from __future__ import annotations

import math


def exact_ints(x, y):
    """Integers X, Y with x[i] = X[i] * 2**e and y[i] = Y[i] * 2**e."""
    vals = [float(v) for v in x] + [float(v) for v in y]
    exps = []
    for v in vals:
        if v != 0.0:
            num, den = v.as_integer_ratio()
            exps.append(-(den.bit_length() - 1))
    e = min(exps) if exps else 0
    out = []
    for v in vals:
        num, den = v.as_integer_ratio()
        shift = -e - (den.bit_length() - 1)
        out.append(num << shift)
    n = len(x)
    return out[:n], out[n:]


def orient(X, Y, a, b, c) -> int:
    """orient(a,b,c) = (b-a) x (c-a) as an exact integer."""
    return (X[b] - X[a]) * (Y[c] - Y[a]) - (Y[b] - Y[a]) * (X[c] - X[a])


def _sites(X, Y):
    """Lowest index per distinct coordinate pair, sorted by (x, y)."""
    first = {}
    for i, key in enumerate(zip(X, Y)):
        if key not in first:
            first[key] = i
    return sorted(first.values(), key=lambda i: (X[i], Y[i]))


def brute_hull(x, y):
    n = len(x)
    if n == 0:
        return []
    X, Y = exact_ints(x, y)
    S = _sites(X, Y)
    if len(S) == 1:
        return [S[0]]
    nxt = {}
    for i in S:
        for j in S:
            if i == j:
                continue
            ok = True
            for k in S:
                o = orient(X, Y, i, j, k)
                if o > 0:
                    ok = False
                    break
                if o == 0:
                    # k must lie on the closed segment [i, j]
                    if not (min(X[i], X[j]) <= X[k] <= max(X[i], X[j]) and
                            min(Y[i], Y[j]) <= Y[k] <= max(Y[i], Y[j])):
                        ok = False
                        break
            if ok:
                assert i not in nxt, "two clockwise edges leave one vertex"
                nxt[i] = j
    start = S[0]
    out = [start]
    cur = nxt[start]
    while cur != start:
        out.append(cur)
        cur = nxt[cur]
        assert len(out) <= len(S)
    return out


def monotone_chain(x, y):
    n = len(x)
    if n == 0:
        return []
    X, Y = exact_ints(x, y)
    S = _sites(X, Y)
    if len(S) <= 2:
        return list(S)

    def cross(o, a, b):
        return (X[a] - X[o]) * (Y[b] - Y[o]) - (Y[a] - Y[o]) * (X[b] - X[o])

    upper = []  # lexmin -> lexmax, clockwise: keep right turns only
    for i in S:
        while len(upper) >= 2 and cross(upper[-2], upper[-1], i) >= 0:
            upper.pop()
        upper.append(i)
    lower = []  # lexmax -> lexmin
    for i in reversed(S):
        while len(lower) >= 2 and cross(lower[-2], lower[-1], i) >= 0:
            lower.pop()
        lower.append(i)
    hull = upper[:-1] + lower[:-1]
    if len(hull) == 2 and hull[0] == hull[1]:
        return hull[:1]
    return hull


def orient_sign_exact(a, b, c) -> int:
    X, Y = exact_ints([a[0], b[0], c[0]], [a[1], b[1], c[1]])
    v = orient(X, Y, 0, 1, 2)
    return (v > 0) - (v < 0)


def cross_sign_exact(p0, p1, q0, q1) -> int:
    X, Y = exact_ints([p0[0], p1[0], q0[0], q1[0]], [p0[1], p1[1], q0[1], q1[1]])
    v = (X[1] - X[0]) * (Y[3] - Y[2]) - (Y[1] - Y[0]) * (X[3] - X[2])
    return (v > 0) - (v < 0)


def dot_sign_exact(p0, p1, q0, q1) -> int:
    X, Y = exact_ints([p0[0], p1[0], q0[0], q1[0]], [p0[1], p1[1], q0[1], q1[1]])
    v = (X[1] - X[0]) * (X[3] - X[2]) + (Y[1] - Y[0]) * (Y[3] - Y[2])
    return (v > 0) - (v < 0)


def polygon_area2(x, y, idx) -> float:
    """Twice the signed area (negative for clockwise)."""
    s = 0.0
    for k in range(len(idx)):
        a, b = idx[k], idx[(k + 1) % len(idx)]
        s += x[a] * y[b] - x[b] * y[a]
    return s


def renyi_sulanke_disk(n: int) -> float:
    """Leading term of the expected vertex count of the hull of n uniform
    points in the unit disk (Renyi and Sulanke 1963):
    2*pi * (2 / (3*pi))**(1/3) * Gamma(5/3) * n**(1/3), about 3.3826 n^(1/3)."""
    return 2.0 * math.pi * (2.0 / (3.0 * math.pi)) ** (1.0 / 3.0) * math.gamma(5.0 / 3.0) * n ** (1.0 / 3.0)


def renyi_sulanke_square(n: int) -> float:
    """Leading term for n uniform points in a square: (8/3) ln n (a polygon
    with r vertices gives (2r/3) ln n)."""
    return 8.0 / 3.0 * math.log(n)
