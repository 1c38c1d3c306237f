"""Pins for the oracle's exact predicates and its triangle-pair test.

The oracle's orient3d/orient2d (double filter + exact integer fallback) are
checked against rational arithmetic; its self-intersection predicate
(Section 5.2, Algorithm 3, supplementary Section 3) against the hand-built
figure cases and a constructive rational clipping reference on seeded pairs of
the kinds the paper's detector study uses (coplanar, vertex- and edge-sharing,
random; Table 'self-intersection quantitative').  The bar is the paper's
detector goal with the slack removed: no false negatives and no false
positives.
"""
import json
import os

import numpy as np
import pytest

import oracle
from tests import exact_ref

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_points(rng, n, kind):
    if kind == "uniform":
        return rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    if kind == "grid":
        return rng.integers(-3, 4, size=(n, 3)).astype(np.float32)
    if kind == "wide":  # mixed magnitudes, exercises inexact double differences
        m = rng.uniform(-1, 1, size=(n, 3)) * 10.0 ** rng.integers(-30, 20, size=(n, 3))
        return m.astype(np.float32)
    raise ValueError(kind)


def _near_coplanar(rng, n):
    """Four points on a random plane, rounded to float32: orient3d is tiny."""
    out = []
    for _ in range(n):
        o = rng.normal(size=3)
        u, v = rng.normal(size=3), rng.normal(size=3)
        st = rng.normal(size=(4, 2))
        P = o + st[:, :1] * u + st[:, 1:] * v
        out.append(P.astype(np.float32))
    return out


@pytest.mark.parametrize("kind", ["uniform", "grid", "wide"])
def test_orient3d_matches_rational(kind):
    rng = np.random.default_rng(11)
    for _ in range(300):
        P = _rand_points(rng, 4, kind)
        ref = exact_ref.orient3d(*P)
        assert oracle.orient3d(*P, exact=True) == ref
        assert oracle.orient3d(*P) == ref


def test_orient3d_near_degenerate_and_exact_zero():
    rng = np.random.default_rng(12)
    zeros = 0
    for P in _near_coplanar(rng, 300):
        ref = exact_ref.orient3d(*P)
        zeros += ref == 0
        assert oracle.orient3d(*P, exact=True) == ref
        assert oracle.orient3d(*P) == ref
    # exactly coplanar: integer points on the plane x + y + z = 3
    for _ in range(200):
        xy = rng.integers(-5, 6, size=(4, 2))
        P = np.concatenate([xy, (3 - xy.sum(1))[:, None]], 1).astype(np.float32)
        assert exact_ref.orient3d(*P) == 0
        assert oracle.orient3d(*P) == 0


def test_orient3d_extreme_exponents():
    # differences that are not representable in double: 1 + 2^-60 style
    a = np.array([1.0, 0.0, 0.0], np.float32)
    b = np.array([0.0, 1.0, 0.0], np.float32)
    c = np.array([0.0, 0.0, 1.0], np.float32)
    for e in (-40, -80, -120, -140):
        d = np.array([1 / 3, 1 / 3, 1 / 3], np.float32) + np.float32(2.0 ** e)
        d = d.astype(np.float32)
        assert oracle.orient3d(a, b, c, d) == exact_ref.orient3d(a, b, c, d)
    tiny = np.float32(2.0 ** -149)
    P = np.array([[tiny, 0, 0], [0, tiny, 0], [0, 0, tiny], [0, 0, 0]], np.float32)
    assert oracle.orient3d(*P) == exact_ref.orient3d(*P) != 0
    big = np.float32(3e38)
    P = np.array([[big, 0, 0], [0, big, 0], [0, 0, big], [-big, -big, -big]], np.float32)
    assert oracle.orient3d(*P, exact=True) == exact_ref.orient3d(*P)


@pytest.mark.parametrize("kind", ["uniform", "grid", "wide"])
def test_orient2d_matches_rational(kind):
    rng = np.random.default_rng(13)
    for _ in range(300):
        P = _rand_points(rng, 3, kind)[:, :2]
        ref = exact_ref.orient2d(*P)
        assert oracle.orient2d(*P, exact=True) == ref
        assert oracle.orient2d(*P) == ref


def test_figure_cases_golden():
    with open(os.path.join(HERE, "golden", "tritri_figure_cases.json")) as fh:
        cases = json.load(fh)["cases"]
    for c in cases:
        T = np.array(c["T"], np.float32)
        C = np.array(c["C"], np.float32)
        got = oracle.tri_intersect(T, C, c["ti"], c["ci"])
        assert got == c["expect"], c["name"]
        # the constructive reference agrees with the labels, too
        assert exact_ref.tri_intersect(T, C, c["ti"], c["ci"]) == c["expect"], c["name"]
        # the predicate is symmetric in its two faces
        assert oracle.tri_intersect(C, T, c["ci"], c["ti"]) == c["expect"], c["name"]


def _pair_stream(rng, n):
    """Seeded triangle pairs in the categories of the paper's detector study:
    random, coplanar, sharing one vertex, sharing an edge; with integer-grid
    variants that create exact degeneracies."""
    for i in range(n):
        kind = i % 8
        if kind == 0:   # generic random, no sharing
            P = rng.uniform(-1, 1, size=(6, 3))
            yield P[:3], P[3:], (0, 1, 2), (3, 4, 5)
        elif kind == 1:  # coplanar on z = 0, integer grid
            P = np.concatenate([rng.integers(-3, 4, size=(6, 2)), np.zeros((6, 1))], 1)
            yield P[:3], P[3:], (0, 1, 2), (3, 4, 5)
        elif kind == 2:  # shared vertex, coplanar grid
            P = np.concatenate([rng.integers(-3, 4, size=(5, 2)), np.zeros((5, 1))], 1)
            yield P[[0, 1, 2]], P[[0, 3, 4]], (0, 1, 2), (0, 3, 4)
        elif kind == 3:  # shared vertex, 3-D grid
            P = rng.integers(-2, 3, size=(5, 3))
            yield P[[0, 1, 2]], P[[0, 3, 4]], (0, 1, 2), (0, 3, 4)
        elif kind == 4:  # shared edge, coplanar grid
            P = np.concatenate([rng.integers(-3, 4, size=(4, 2)), np.zeros((4, 1))], 1)
            yield P[[0, 1, 2]], P[[1, 0, 3]], (0, 1, 2), (1, 0, 3)
        elif kind == 5:  # shared edge, 3-D grid
            P = rng.integers(-2, 3, size=(4, 3))
            yield P[[0, 1, 2]], P[[1, 0, 3]], (0, 1, 2), (1, 0, 3)
        elif kind == 6:  # 3-D grid, no sharing: touching / edge-on cases
            P = rng.integers(-2, 3, size=(6, 3))
            yield P[:3], P[3:], (0, 1, 2), (3, 4, 5)
        else:            # sharp: nearly coplanar float pairs sharing a vertex
            o = rng.normal(size=3)
            u, v = rng.normal(size=3), rng.normal(size=3)
            st = rng.normal(size=(5, 2))
            P = o + st[:, :1] * u + st[:, 1:] * v
            P = P + rng.normal(size=P.shape) * 1e-7
            yield P[[0, 1, 2]], P[[0, 3, 4]], (0, 1, 2), (0, 3, 4)


def test_random_pairs_match_constructive_reference():
    rng = np.random.default_rng(2024)
    tp = tn = 0
    for T, C, ti, ci in _pair_stream(rng, 2400):
        T = np.asarray(T, np.float32)
        C = np.asarray(C, np.float32)
        ref = exact_ref.tri_intersect(T, C, ti, ci)
        got = oracle.tri_intersect(T, C, ti, ci)
        assert got == ref, (T.tolist(), C.tolist(), ti, ci)
        tp += ref
        tn += not ref
    assert tp > 300 and tn > 300  # both labels well represented


def _naive_orient3d(a, b, c, d):
    a, b, c, d = [np.asarray(x, np.float64) for x in (a, b, c, d)]
    A, B, C = a - d, b - d, c - d
    det = (A[2] * (B[0] * C[1] - C[0] * B[1]) + B[2] * (C[0] * A[1] - A[0] * C[1])
           + C[2] * (A[0] * B[1] - B[0] * A[1]))
    return int(np.sign(det))


def _on_plane(rng, n, scale):
    x = rng.integers(-8, 9, 3).astype(np.float64) * scale
    k = int(np.argmax(np.abs(n)))
    r = [i for i in range(3) if i != k]
    x[k] = -(n[r[0]] * x[r[0]] + n[r[1]] * x[r[1]]) / n[k]
    return x


def test_orient3d_exponent_gap_adversarial():
    """Coplanar points of very different magnitudes plus a tiny offset: the
    double differences round, and plain double evaluation often returns the
    wrong sign.  The filter must hand those to the exact path."""
    rng = np.random.default_rng(77)
    naive_wrong = 0
    for _ in range(1500):
        n = rng.integers(-3, 4, 3)
        if not n.any():
            continue
        a, b, c = (_on_plane(rng, n, 2.0 ** rng.integers(10, 40)) for _ in range(3))
        d = (_on_plane(rng, n, 2.0 ** rng.integers(-40, -10))
             + rng.integers(-1, 2, 3) * 2.0 ** rng.integers(-80, -40))
        P = [np.asarray(x, np.float32) for x in (a, b, c, d)]
        ref = exact_ref.orient3d(*P)
        nv = _naive_orient3d(*P)
        naive_wrong += nv != ref and nv != 0
        assert oracle.orient3d(*P) == ref
    assert naive_wrong > 20


def test_orient2d_exponent_gap_adversarial():
    rng = np.random.default_rng(78)
    naive_wrong = 0
    for _ in range(1500):
        k = rng.integers(1, 5)
        pts = []
        for sc in (2.0 ** rng.integers(10, 40), 2.0 ** rng.integers(10, 40)):
            t = rng.integers(-8, 9) * sc
            pts.append((t, k * t))
        t = rng.integers(-8, 9) * 2.0 ** rng.integers(-40, -10)
        pts.append((t + rng.integers(-1, 2) * 2.0 ** rng.integers(-80, -40), k * t))
        P = [np.asarray(p, np.float32) for p in pts]
        ref = exact_ref.orient2d(*P)
        a, b, c = [np.asarray(p, np.float64) for p in P]
        nv = int(np.sign((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])))
        naive_wrong += nv != ref and nv != 0
        assert oracle.orient2d(*P) == ref
    assert naive_wrong > 5
