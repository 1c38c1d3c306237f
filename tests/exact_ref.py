"""Independent exact references used to pin the oracle.

Everything here is exact rational arithmetic (``fractions.Fraction``) on the
float32 inputs, written as a *constructive* computation (the actual set T n C is
built by clipping), which is a different method from the sign-only
decomposition used by the oracle.  Slow; only for small test inputs.
"""
from fractions import Fraction as Fr

import numpy as np


def fr3(p):
    return tuple(Fr(float(np.float32(x))) for x in p)


def sub(a, b):
    return (a[0] - b[0], a[1] - b[1], a[2] - b[2])


def add(a, b):
    return (a[0] + b[0], a[1] + b[1], a[2] + b[2])


def mul(a, t):
    return (a[0] * t, a[1] * t, a[2] * t)


def dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2],
            a[0] * b[1] - a[1] * b[0])


def sgn(x):
    return (x > 0) - (x < 0)


def orient3d(a, b, c, d):
    a, b, c, d = fr3(a), fr3(b), fr3(c), fr3(d)
    return sgn(dot(sub(a, d), cross(sub(b, d), sub(c, d))))


def orient2d(a, b, c):
    a = [Fr(float(np.float32(x))) for x in a]
    b = [Fr(float(np.float32(x))) for x in b]
    c = [Fr(float(np.float32(x))) for x in c]
    return sgn((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))


def _clip(poly, tri, n):
    """Clip convex polygon (list of points in the plane) by triangle tri (same
    plane, normal n) using closed half-planes."""
    for i in range(3):
        u, v = tri[i], tri[(i + 1) % 3]
        m = cross(n, sub(v, u))          # inward for a triangle oriented by n
        out = []
        k = len(poly)
        for j in range(k):
            p, q = poly[j], poly[(j + 1) % k]
            fp, fq = dot(m, sub(p, u)), dot(m, sub(q, u))
            if fp >= 0:
                out.append(p)
            if (fp > 0 and fq < 0) or (fp < 0 and fq > 0):
                t = fp / (fp - fq)
                out.append(add(p, mul(sub(q, p), t)))
        poly = out
        if not poly:
            break
    return poly


def _interval(tri, n, p0, d):
    lo, hi = None, None
    for i in range(3):
        u, v = tri[i], tri[(i + 1) % 3]
        m = cross(n, sub(v, u))
        c0, c1 = dot(m, sub(p0, u)), dot(m, d)
        if c1 == 0:
            if c0 < 0:
                return None
            continue
        t = -c0 / c1
        if c1 > 0:
            lo = t if lo is None else max(lo, t)
        else:
            hi = t if hi is None else min(hi, t)
    return lo, hi


def intersection_points(T, C):
    """Exact description of T n C for non-degenerate triangles: returns
    ('empty',), ('points', [pts]) (convex hull = T n C)."""
    nT = cross(sub(T[1], T[0]), sub(T[2], T[0]))
    nC = cross(sub(C[1], C[0]), sub(C[2], C[0]))
    d = cross(nT, nC)
    if d == (0, 0, 0):
        if dot(nT, sub(C[0], T[0])) != 0:
            return ("empty",)
        # coplanar: orient C consistently with nT's side for clipping
        Cc = list(C) if dot(nC, nT) > 0 else [C[0], C[2], C[1]]
        poly = _clip(list(T), Cc, nT)
        return ("points", poly) if poly else ("empty",)
    # line of the two planes: p0 solves nT.x = nT.T0, nC.x = nC.C0, d.x = 0
    rows = [nT, nC, d]
    rhs = [dot(nT, T[0]), dot(nC, C[0]), Fr(0)]
    det = dot(rows[0], cross(rows[1], rows[2]))
    cols = []
    for k in range(3):
        M = [list(r) for r in rows]
        for i in range(3):
            M[i][k] = rhs[i]
        cols.append(dot(tuple(M[0]), cross(tuple(M[1]), tuple(M[2]))) / det)
    p0 = tuple(cols)
    it = _interval(T, nT, p0, d)
    ic = _interval(C, nC, p0, d)
    if it is None or ic is None:
        return ("empty",)
    lo = max(it[0], ic[0])
    hi = min(it[1], ic[1])
    if lo > hi:
        return ("empty",)
    return ("points", [add(p0, mul(d, lo)), add(p0, mul(d, hi))])


def tri_intersect(T, C, ti, ci):
    """Reference for the mesh self-intersection predicate (Algorithm 3 with
    the supplementary case analysis, read exactly):
    s=3 -> True; zero-area triangle -> True; s=0: T n C non-empty;
    s=1: T n C contains a point other than the shared vertex;
    s=2: the triangles are coplanar and T n C leaves the shared edge's line."""
    s = len(set(int(x) for x in ti) & set(int(x) for x in ci))
    if s >= 3:
        return True
    T = [fr3(p) for p in T]
    C = [fr3(p) for p in C]
    for X in (T, C):
        if cross(sub(X[1], X[0]), sub(X[2], X[0])) == (0, 0, 0):
            return True
    res = intersection_points(T, C)
    if res[0] == "empty":
        return False
    pts = res[1]
    if s == 0:
        return True
    ti, ci = [int(x) for x in ti], [int(x) for x in ci]
    if s == 1:
        a = [i for i in range(3) if ti[i] in ci][0]
        A = T[a]
        return any(p != A for p in pts)
    nT = cross(sub(T[1], T[0]), sub(T[2], T[0]))
    nC = cross(sub(C[1], C[0]), sub(C[2], C[0]))
    if cross(nT, nC) != (0, 0, 0):
        return False
    sh = [i for i in range(3) if ti[i] in ci]
    A, B = T[sh[0]], T[sh[1]]
    return any(cross(sub(p, A), sub(B, A)) != (0, 0, 0) for p in pts)
