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
  * outside the certified range the high part is NaN;
  * per edge, on the round-0 edges of real meshes: the float-float sum of the
    edge's terms lies within B = nt (2^-40 + 3.2 u^2 sum|t|) of the oracle's
    float64 sum, and the kernel's interval test (B rounded upwards in float32,
    the interval's ends rounded outwards in float64, both ends through
    fl(w_s x + Tq) to key bits), emulated exactly, certifies only keys equal to
    the oracle's.
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


# ---- the per-edge certification (the edge-cost kernel's key decision) ------

def _rd64(q):
    f = float(q)
    return f if Fraction(f) <= q else float(np.nextafter(f, -np.inf))


def _ru64(q):
    f = float(q)
    return f if Fraction(f) >= q else float(np.nextafter(f, np.inf))


def _ru32(q):
    f = np.float32(float(q))
    while Fraction(float(f)) < q:
        f = np.nextafter(f, np.float32(np.inf))
    while Fraction(float(np.nextafter(f, np.float32(-np.inf)))) >= q:
        f = np.nextafter(f, np.float32(-np.inf))
    return f


def _fma64(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _key_bits(cost):
    with np.errstate(over="ignore"):
        cf = np.float32(cost)
    if np.isnan(cost) or np.isinf(cf):
        return 0xFFFFFFFF
    if not cf > 0:
        cf = np.float32(0)
    return int(np.array([cf], np.float32).view(np.uint32)[0])


def _produced(V, F, ab, vbar):
    """Per edge, its produced triangles [vbar, p, q] in ascending face order."""
    around = [[] for _ in range(len(V))]
    for f, t in enumerate(F):
        for v in t:
            around[v].append(f)
    tris, owner = [], []
    for e, (a, b) in enumerate(ab):
        fa, fb = set(around[a]), set(around[b])
        for f in sorted(fa ^ fb):
            others = [v for v in F[f] if v != a and v != b]
            tris.append(np.concatenate([vbar[e], V[others[0]], V[others[1]]]))
            owner.append(e)
    return np.array(tris, np.float32), np.array(owner)


def _meshes():
    import meshgen
    out = {"bumped_icosphere_l4": meshgen.bumped_icosphere(level=4, seed=0)[:2],
           "torus_48x24": meshgen.torus(48, 24)[:2],
           "nested_shells_l3": meshgen.nested_shells(level=3)[:2]}
    return {k: (np.asarray(V, np.float32), np.asarray(F, np.int32)) for k, (V, F) in out.items()}


def test_edge_skinny_sum_within_its_bound_and_certified_keys_are_the_oracles():
    """On the round-0 edges of real meshes: the float-float sum of an edge's
    terms lies within B = nt (2^-40 + 3.2 u^2 sum|t|) of the oracle's float64
    sum Cs, and every key the kernel's interval test certifies equals the
    oracle's key."""
    w_e, w_s = oracle.W_E, oracle.W_S
    C1 = float.fromhex("0x1.99999ap-47")
    for name, (V, F) in _meshes().items():
        et = oracle.edge_table(V, F)
        ab, vbar = et["ab"], et["vbar"]
        T, owner = _produced(V, F, ab, vbar)
        tff = ff_emulation.skinny_term_ff(T)
        assert np.isfinite(tff).all(), name
        # the lane's float-float sum, in the produced triangles' order
        ne = len(ab)
        cs = (np.zeros(ne, np.float32), np.zeros(ne, np.float32))
        nt = np.bincount(owner, minlength=ne)
        starts = np.concatenate([[0], np.cumsum(nt)[:-1]])
        for k in range(nt.max()):
            sel = np.nonzero(nt > k)[0]
            rows = starts[sel] + k
            s0, s1 = ff_emulation.add((cs[0][sel], cs[1][sel]), (tff[rows, 0], tff[rows, 1]))
            cs[0][sel], cs[1][sel] = s0, s1
        # the non-skinny part, restated from the oracle's scale and fma order
        lo_b, hi_b = V.astype(np.float64).min(0), V.astype(np.float64).max(0)
        ext = float(np.max(hi_b - lo_b))
        scale = 1.0 / ext
        s2, wes = scale * scale, w_e * scale
        worst, certified = 0.0, 0
        for e in range(ne):
            Tq = _fma64(wes, et["l"][e], s2 * et["Q"][e])
            assert _fma64(w_s, et["Cs"][e], Tq) == et["cost"][e], (name, e)  # restatement check
            terms = tff[starts[e]:starts[e] + nt[e]]
            A_exact = sum(abs(Fraction(float(t))) for t in terms[:, 0])
            B_min = nt[e] * (Fraction(2) ** -40 + Fraction(C1) * A_exact)
            Cs_ff = Fraction(float(cs[0][e])) + Fraction(float(cs[1][e]))
            err = abs(Cs_ff - Fraction(et["Cs"][e]))
            assert err <= B_min, (name, e, float(err / B_min))
            worst = max(worst, float(err / B_min))
            # the kernel's B (float32, rounded upwards) and its interval test
            A = np.float32(0)
            for t in terms[:, 0]:
                A = _ru32(Fraction(float(A)) + abs(Fraction(float(t))))
            A = _ru32(Fraction(float(A)) * (1 + Fraction(2) ** -22))
            B = _ru32(nt[e] * Fraction(float(_ru32(Fraction(C1) * Fraction(float(A))
                                                      + Fraction(2) ** -40))))
            Bd = Fraction(float(B))
            lo = _rd64(Fraction(_rd64(Cs_ff)) - Bd)
            hi = _ru64(Fraction(_ru64(Cs_ff)) + Bd)
            k0 = _key_bits(_fma64(w_s, lo if w_s >= 0 else hi, Tq))
            k1 = _key_bits(_fma64(w_s, hi if w_s >= 0 else lo, Tq))
            if k0 == k1 and k0 != 0xFFFFFFFF:
                certified += 1
                assert k0 == _key_bits(et["cost"][e]), (name, e)
        print(f"{name}: {ne} edges, {certified} keys certified, "
              f"max |Cs_ff - Cs| / B = {worst:.2e}")
        assert certified >= 0.99 * ne, name
