"""The float-float skinny term behind the edge-cost keys (Eq. 1, Sec. 5.1).

The cost kernel evaluates each produced triangle's 1 - C_ijk in float-float
arithmetic and keeps a key only when the bound kTriBound = 2^-40 per triangle
proves it equal to the float64 evaluation's key.  These tests pin the bound's
ingredients against arithmetic that shares nothing with the kernel:
  * the kernel's float64 term equals the oracle's 1 - C_ijk bit for bit;
  * the kernel's float-float pairs equal, bit for bit, an exact float32
    emulation of the same steps (tests/ff_emulation.py), whose error the CPU
    tests (test_skinny_ff_emulation.py) search without a GPU;
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

import numpy as np
import pytest

import ff_emulation
import oracle
import skinny_cases

pytestmark = pytest.mark.gpu

U2 = 2.0 ** -48


def test_float64_term_is_the_oracles():
    import paper_2509_05595_gb300 as pamo
    T = np.concatenate(list(skinny_cases.families().values()))
    t64, _ = pamo.pamo_skinny_terms(T)
    t64 = t64.cpu().numpy()
    want = np.array([1.0 - oracle.tri_quality(r[0:3].astype(np.float64), r[3:6].astype(np.float64),
                                              r[6:9].astype(np.float64)) for r in T])
    assert np.array_equal(t64.view(np.uint64), want.view(np.uint64))


def test_float_float_pairs_are_the_emulations():
    import paper_2509_05595_gb300 as pamo
    fams = dict(skinny_cases.families())
    fams.update(skinny_cases.out_of_range())
    for name, T in fams.items():
        _, tff = pamo.pamo_skinny_terms(T)
        got = tff.cpu().numpy()
        want = ff_emulation.skinny_term_ff(T)
        finite = ~np.isnan(want[:, 0])
        assert np.array_equal(np.isnan(got[:, 0]), ~finite), name
        assert np.array_equal(got[finite].view(np.uint32), want[finite].view(np.uint32)), name


def test_float_float_term_within_its_bound():
    import paper_2509_05595_gb300 as pamo
    worst = {}
    for name, T in skinny_cases.families().items():
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
    import paper_2509_05595_gb300 as pamo
    for name, T in skinny_cases.out_of_range().items():
        _, tff = pamo.pamo_skinny_terms(T)
        assert np.isnan(tff.cpu().numpy()[:, 0]).all(), name
    t64, tff = pamo.pamo_skinny_terms(np.zeros((0, 9), np.float32))
    assert t64.numel() == 0 and tff.numel() == 0
