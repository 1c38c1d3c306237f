"""The error analysis of the certified float-float skinny term (Eq. 1), checked
on the CPU: tests/ff_emulation.py runs the kernel's steps in exact float32
arithmetic (the GPU test test_gpu_skinny_ff.py shows the kernel's pairs equal
the emulation's bit for bit), and these tests search its error.

  * fma32, the emulator's one non-native operation, equals the correctly
    rounded float32 of a*b + c computed in rationals, including exact ties;
  * the term is within the analysis' total of 114 u^2 (u = 2^-24) of the
    oracle's float64 1 - C_ijk on every family and on adversarial ones (far
    from the origin, D at both ends of the certified range, needles, exact
    collinear triangles), and within 112.4 u^2 of the exact value (120-digit
    decimal arithmetic) on the worst cases found and on samples;
  * outside the certified range the high part is NaN.
"""
import decimal
from fractions import Fraction

import numpy as np

import ff_emulation
import oracle
import skinny_cases

U2 = 2.0 ** -48


def _rn32(q):
    """Correctly rounded float32 of a rational (ties to even)."""
    f = np.float32(float(q))
    best = None
    for c in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
        d = abs(Fraction(float(c)) - q)
        even = (np.array([c], np.float32).view(np.uint32)[0] & 1) == 0
        if best is None or d < best[0] or (d == best[0] and even):
            best = (d, c)
    return np.float32(best[1])


def _oracle_t64(T):
    return np.array([1.0 - oracle.tri_quality(r[0:3].astype(np.float64), r[3:6].astype(np.float64),
                                              r[6:9].astype(np.float64)) for r in T])


def _adversarial(seed=5, n=4000):
    rng = np.random.default_rng(seed)
    out = {}
    # far from the origin: large coordinates, small triangles, inexact differences
    off = rng.choice([-1.0, 1.0], (n, 1)) * 10.0 ** rng.uniform(3, 6, (n, 1))
    base = skinny_cases.mesh_like(rng, n, h=1.0)
    out["far"] = base + np.tile(off, (1, 9))
    # D near the ends of the certified range (2^-60, 2^60)
    m = skinny_cases.mesh_like(rng, n)
    D = np.array([np.sum((r[3:6] - r[0:3]) ** 2) + np.sum((r[6:9] - r[0:3]) ** 2)
                  + np.sum((r[6:9] - r[3:6]) ** 2) for r in m])
    out["near_low"] = m * np.sqrt(2.0 ** -58 / D)[:, None]
    out["near_high"] = m * np.sqrt(2.0 ** 58 / D)[:, None]
    # needles: two corners almost coincident
    P0 = rng.uniform(-1, 1, (n, 3))
    P1 = P0 + rng.normal(0, 5e-3, (n, 3))
    out["needle"] = np.concatenate([P0, P1, P1 + rng.normal(0, 1e-9, (n, 3))], 1)
    # exactly collinear: P2 = P0 + 2 (P1 - P0) with float-exact coordinates
    q0 = np.round(rng.uniform(-1, 1, (n, 3)) * 2 ** 10) / 2 ** 10
    q1 = q0 + np.round(rng.normal(0, 1e-2, (n, 3)) * 2 ** 16) / 2 ** 16
    out["collinear"] = np.concatenate([q0, q1, q0 + 2 * (q1 - q0)], 1)
    return {k: v.astype(np.float32) for k, v in out.items()}


def test_fma32_is_correctly_rounded():
    rng = np.random.default_rng(0)
    n = 3000
    a = rng.standard_normal(n).astype(np.float32)
    b = rng.standard_normal(n).astype(np.float32)
    cases = [-(a.astype(np.float64) * b).astype(np.float32),           # cancellation
             rng.standard_normal(n).astype(np.float32) * np.float32(1e-8),
             rng.standard_normal(n).astype(np.float32)]
    for c in cases:
        got = ff_emulation.fma32(a, b, c)
        for i in range(0, n, 5):
            want = _rn32(Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i])))
            assert got[i] == want, (a[i], b[i], c[i])
    # products that land exactly on a float32 midpoint, nudged either way by c
    u = 1 + 2.0 ** -12
    for x, y, z in [(u, u, 2.0 ** -80), (u, u, -2.0 ** -80), (u, u, 0.0), (u, -u, 2.0 ** -80),
                    (u, -u, -2.0 ** -80), (1 + 2.0 ** -13, 1 + 2.0 ** -11, 2.0 ** -90),
                    (1 + 2.0 ** -13, 1 + 2.0 ** -11, -2.0 ** -90)]:
        A, B, C = (np.array([v], np.float32) for v in (x, y, z))
        want = _rn32(Fraction(float(A[0])) * Fraction(float(B[0])) + Fraction(float(C[0])))
        assert ff_emulation.fma32(A, B, C)[0] == want, (x, y, z)


def test_float_float_term_within_the_analysis():
    fams = dict(skinny_cases.families(n=8000))
    fams.update(_adversarial())
    worst = {}
    for name, T in fams.items():
        tff = ff_emulation.skinny_term_ff(T)
        assert np.isfinite(tff).all(), name
        t64 = _oracle_t64(T)
        d = np.abs(tff[:, 0].astype(np.float64) + tff[:, 1].astype(np.float64) - t64)
        assert d.max() <= 114 * U2, (name, d.max() / U2)
        # against the exact value: the 20 worst rows and a sample
        rows = np.unique(np.concatenate([np.argsort(d)[-20:],
                                         np.random.default_rng(2).choice(len(T), 60, replace=False)]))
        e_ff = e_64 = 0.0
        with decimal.localcontext() as ctx:
            ctx.prec = 120
            for i in rows:
                t = skinny_cases.exact_t(T[i])
                tf = decimal.Decimal(float(tff[i, 0])) + decimal.Decimal(float(tff[i, 1]))
                e_ff = max(e_ff, abs(float(tf - t)))
                e_64 = max(e_64, abs(float(decimal.Decimal(float(t64[i])) - t)))
        assert e_ff <= 112.4 * U2, (name, e_ff / U2)
        assert e_64 <= 0.81 * U2, (name, e_64 / U2)
        worst[name] = (d.max() / U2, e_ff / U2, e_64 / U2)
    print("max |ff - f64|, |ff - exact|, |f64 - exact| in u^2:",
          {k: tuple(round(x, 3) for x in v) for k, v in worst.items()})


def test_outside_the_certified_range_is_nan():
    for name, T in skinny_cases.out_of_range().items():
        assert np.isnan(ff_emulation.skinny_term_ff(T)[:, 0]).all(), name
