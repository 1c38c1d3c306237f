"""The float-float skinny term behind the edge-cost keys (Eq. 1, Sec. 5.1).

The cost kernel evaluates each produced triangle's 1 - C_ijk in float-float
arithmetic and keeps a key only when the bound kTriBound = 2^-40 per triangle
proves it equal to the float64 evaluation's key.  These tests pin the bound's
ingredients against arithmetic that shares nothing with the kernel:
  * the kernel's float64 term equals the oracle's 1 - C_ijk bit for bit;
  * against the exact value (decimal arithmetic at 120 digits), the float-float
    term is within the analysis' 112.4 u^2 (u = 2^-24) and the float64 term
    within 0.81 u^2, on mesh-like triangles, slivers down to a height/length
    ratio of 1e-12, near-equilateral ones, scales 2^-16 .. 2^28 and corners
    whose float differences are inexact;
  * against the float64 term, the float-float term is within the 114 u^2 the
    analysis states in total, well inside kTriBound;
  * outside the certified range (D < 2^-60, D > 2^60, coincident corners,
    non-finite corners) the float-float term is NaN, so the key falls back to
    float64.
"""
import decimal
from fractions import Fraction

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

U2 = 2.0 ** -48


def _mesh_like(rng, n, h=5e-3):
    P0 = rng.uniform(-1, 1, (n, 3))
    return np.concatenate([P0, P0 + rng.normal(0, h, (n, 3)), P0 + rng.normal(0, h, (n, 3))], 1)


def _equilateral(rng, n, side=1e-2, jitter=1e-6):
    c = rng.uniform(-1, 1, (n, 3))
    e1 = rng.normal(size=(n, 3))
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(e1, rng.normal(size=(n, 3)))
    e2 /= np.linalg.norm(e2, axis=1, keepdims=True)
    pts = [c + side * (np.cos(a) * e1 + np.sin(a) * e2) / np.sqrt(3)
           for a in (0.0, 2 * np.pi / 3, 4 * np.pi / 3)]
    T = np.concatenate(pts, 1)
    return T + rng.normal(0, jitter * side, T.shape)


def _slivers(rng, n):
    P0 = rng.uniform(-1, 1, (n, 3))
    d = rng.normal(0, 5e-3, (n, 3))
    perp = np.cross(d, rng.normal(size=(n, 3)))
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    ratio = 10.0 ** rng.uniform(-12, -1, (n, 1))
    lam = rng.uniform(-0.5, 1.5, (n, 1))
    L = np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([P0, P0 + d, P0 + lam * d + ratio * L * perp], 1)


def _near_zero(rng, n):
    # coordinates of both signs near 0: float differences that are not exact
    return rng.uniform(-1e-3, 1e-3, (n, 9)) * (10.0 ** rng.uniform(-3, 0, (n, 1)))


def _families(seed=7, n=20000):
    rng = np.random.default_rng(seed)
    fams = {"mesh": _mesh_like(rng, n), "equilateral": _equilateral(rng, n),
            "sliver": _slivers(rng, n), "near_zero": _near_zero(rng, n)}
    for k in (-16, -10, 10, 28):
        fams[f"scaled_2^{k}"] = _mesh_like(rng, n // 4) * 2.0 ** k
    return {k: v.astype(np.float32) for k, v in fams.items()}


def _exact_t(tri):
    """1 - C of one triangle from exact rationals; the square roots at 120
    digits (the caller's decimal context)."""
    P = [Fraction(float(x)) for x in tri]
    a = [P[3 + i] - P[i] for i in range(3)]
    b = [P[6 + i] - P[i] for i in range(3)]
    c = [P[6 + i] - P[3 + i] for i in range(3)]
    n = [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
    n2 = sum(x * x for x in n)
    D = sum(x * x for x in a) + sum(x * x for x in b) + sum(x * x for x in c)
    C = 2 * decimal.Decimal(3).sqrt() * _dec(n2).sqrt() / _dec(D)
    return decimal.Decimal(1) - C


def _dec(f):
    return decimal.Decimal(f.numerator) / decimal.Decimal(f.denominator)


def test_float64_term_is_the_oracles():
    import paper_2509_05595_gb300 as pamo
    T = np.concatenate(list(_families().values()))
    t64, _ = pamo.pamo_skinny_terms(T)
    t64 = t64.cpu().numpy()
    want = np.array([1.0 - oracle.tri_quality(r[0:3].astype(np.float64), r[3:6].astype(np.float64),
                                              r[6:9].astype(np.float64)) for r in T])
    assert np.array_equal(t64.view(np.uint64), want.view(np.uint64))


def test_float_float_term_within_its_bound():
    import paper_2509_05595_gb300 as pamo
    worst = {}
    for name, T in _families().items():
        t64, tff = pamo.pamo_skinny_terms(T)
        t64, tff = t64.cpu().numpy(), tff.cpu().numpy()
        assert np.isfinite(tff).all(), name  # every family lies in the certified range
        # against the float64 term: exact difference of the binary values
        hi = tff[:, 0].astype(np.float64) + tff[:, 1].astype(np.float64)  # exact
        d = np.abs(hi - t64)
        assert d.max() <= 114 * U2, (name, d.max() / U2)
        # against the exact value, on a sample
        idx = np.random.default_rng(11).choice(len(T), 300, replace=False)
        e_ff = e_64 = 0.0
        with decimal.localcontext() as ctx:
            ctx.prec = 120
            for i in idx:
                t = _exact_t(T[i])
                tf = decimal.Decimal(float(tff[i, 0])) + decimal.Decimal(float(tff[i, 1]))
                e_ff = max(e_ff, abs(float(tf - t)))
                e_64 = max(e_64, abs(float(decimal.Decimal(float(t64[i])) - t)))
        assert e_ff <= 112.4 * U2, (name, e_ff / U2)
        assert e_64 <= 0.81 * U2, (name, e_64 / U2)
        worst[name] = (d.max() / U2, e_ff / U2, e_64 / U2)
    print("max |ff - f64|, |ff - exact|, |f64 - exact| in u^2:",
          {k: tuple(round(x, 3) for x in v) for k, v in worst.items()})


def test_outside_the_certified_range_is_nan():
    import paper_2509_05595_gb300 as pamo
    rng = np.random.default_rng(3)
    base = _mesh_like(rng, 64)  # D about 2^-12
    cases = {
        "tiny": base * 2.0 ** -28,        # D about 2^-68
        "huge": base * 2.0 ** 40,         # D about 2^68
        "coincident": np.tile(rng.uniform(-1, 1, (64, 3)), (1, 3)),
        "non_finite": np.where(np.arange(9) == 4, np.inf, base),
        "nan": np.where(np.arange(9) == 0, np.nan, base),
    }
    for name, T in cases.items():
        T = T.astype(np.float32)
        t64, tff = pamo.pamo_skinny_terms(T)
        tff = tff.cpu().numpy()
        assert np.isnan(tff[:, 0]).all(), name
    t64, tff = pamo.pamo_skinny_terms(np.zeros((0, 9), np.float32))
    assert t64.numel() == 0 and tff.numel() == 0
