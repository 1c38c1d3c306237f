"""Pins for the oracle's edge cost (Eq. 1) and its quadric term.

Each pin is fixed by the paper or by mathematics, not by retyping the oracle's
expressions: quadrics vanish on planar patches; the QEM value equals the sum
of squared distances to the incident face planes (Garland-Heckbert, cited in
Section 5.1); C_ijk is 1 for an equilateral triangle and at most 1 otherwise;
all terms are invariant under power-of-two rescaling of the input, which the
normalisation to [0,1]^3 (start of Section 4) implies exactly.
"""
import struct

import mpmath
import numpy as np
import pytest

import meshgen
import oracle

mpmath.mp.dps = 50


def _mpv(p):
    return [mpmath.mpf(float(x)) for x in p]


def _plane(p0, p1, p2):
    a, b, c = _mpv(p0), _mpv(p1), _mpv(p2)
    u = [b[i] - a[i] for i in range(3)]
    w = [c[i] - a[i] for i in range(3)]
    n = [u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]]
    ln = mpmath.sqrt(sum(x * x for x in n))
    n = [x / ln for x in n]
    return n, -sum(n[i] * a[i] for i in range(3))


def _quality_mp(q0, q1, q2):
    a, b, c = _mpv(q0), _mpv(q1), _mpv(q2)
    u = [b[i] - a[i] for i in range(3)]
    w = [c[i] - a[i] for i in range(3)]
    t = [c[i] - b[i] for i in range(3)]
    n = [u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]]
    area = mpmath.sqrt(sum(x * x for x in n)) / 2
    den = sum(x * x for x in u) + sum(x * x for x in t) + sum(x * x for x in w)
    return 4 * mpmath.sqrt(3) * area / den if den > 0 else mpmath.mpf(0)


def test_planar_patch_quadric_and_zero_qem():
    V, F = meshgen.box_grid(4)
    K = oracle.vertex_quadrics(V, F)
    top = np.where((V[:, 2] == 1.0) & (V[:, 0] > 0) & (V[:, 0] < 1) &
                   (V[:, 1] > 0) & (V[:, 1] < 1))[0]
    assert len(top) == 9
    for v in top:
        k = (F == v).any(1).sum()
        # plane z = 1: n = (0,0,1), d = -1 -> [0..0, 1, -1, 1] per face
        assert K[v].tolist() == [0, 0, 0, 0, 0, 0, 0, k, -k, k]
    T = oracle.edge_table(V, F)
    inner = np.isin(T["ab"][:, 0], top) & np.isin(T["ab"][:, 1], top)
    assert inner.sum() >= 8
    assert (T["Q"][inner] == 0.0).all()              # zero QEM inside planar regions
    assert (T["vbar"][inner][:, 2] == 1.0).all()      # placement stays on the plane
    for i in np.where(inner)[0]:                     # singular -> a, b or midpoint
        a, b = V[T["ab"][i, 0]], V[T["ab"][i, 1]]
        m = ((a.astype(np.float64) + b) * 0.5).astype(np.float32)
        assert any((T["vbar"][i] == p).all() for p in (a, b, m))


def test_quality_closed_forms():
    eq = [np.array([0, 0, 0.]), np.array([1, 0, 0.]), np.array([0.5, np.sqrt(3) / 2, 0])]
    assert abs(oracle.tri_quality(*eq) - 1.0) <= 2 * np.finfo(float).eps
    rng = np.random.default_rng(5)
    for _ in range(200):
        q = [rng.normal(size=3) for _ in range(3)]
        c = oracle.tri_quality(*q)
        assert c <= 1.0 + 4e-16
        assert abs(c - float(_quality_mp(*q))) <= 4e-15
        s = 2.0 ** rng.integers(-20, 20)
        assert oracle.tri_quality(*[x * s for x in q]) == c
    # collinear and coincident corners
    assert oracle.tri_quality(np.zeros(3), np.ones(3), 2 * np.ones(3)) == 0.0
    assert oracle.tri_quality(np.zeros(3), np.zeros(3), np.zeros(3)) == 0.0


def _sliver(rng, ratio):
    """A triangle whose apex lies ratio * |u| off the line of its base u,
    anywhere along it (needles and caps), in a random orientation and corner
    order, as float64 corners."""
    p0, p1 = rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3)
    u = p1 - p0
    n = rng.normal(size=3)
    n -= n.dot(u) / u.dot(u) * u
    n /= np.linalg.norm(n)
    p2 = p0 + rng.uniform(-0.5, 1.5) * u + ratio * np.linalg.norm(u) * n
    q = [p0, p1, p2]
    return [q[i] for i in rng.permutation(3)]


# Error bound of C_ijk as Eq. 1 writes it (area from the cross product, the
# three squared lengths summed), for any triangle: each cross-product
# component is off by at most ~eps |u||w| (the edge differences, one product
# and one fused multiply-add), so |u x w| by at most 3 sqrt(3) eps |u||w|;
# C = 2 sqrt(3) |u x w| / den with den >= |u|^2 + |w|^2 >= 2 |u||w| gives
# |C - C_exact| <= 9 eps plus the few-ulp relative error of the quotient.
# The absolute bound holds however thin the triangle is, so a sliver's C_ijk
# (nearly 0) stays right.  An area from |u|^2 |w|^2 - (u.w)^2 instead would be
# off by about sqrt(eps) ~ 1e-8 on these slivers.
QUALITY_ABS_BOUND = 9 * np.finfo(float).eps


@pytest.mark.parametrize("ratio", [1e-3, 1e-6, 1e-9, 1e-12])
def test_quality_on_slivers_against_mpmath(ratio):
    rng = np.random.default_rng(int(-np.log10(ratio)))
    worst = 0.0
    for _ in range(120):
        q = _sliver(rng, ratio)
        c = oracle.tri_quality(*q)
        e = _quality_mp(*q)
        assert e > 0 and c > 0
        worst = max(worst, abs(c - float(e)))
    assert worst <= QUALITY_ABS_BOUND, worst


def test_quality_on_float32_exact_slivers():
    # base along (a, b, 0), apex 2^-k above the base's midpoint: every corner is
    # exact in float32 (as mesh positions are), the exact C_ijk is far from 0,
    # and |u|^2 |w|^2 - (u.w)^2 rounds to exactly 0 in float64 for k >= 27
    for a, b in ((1, 1), (3, 1), (2, 5)):
        for k in (10, 20, 27, 35, 50):
            q = [np.zeros(3), np.array([a / 4, b / 4, 0.0]),
                 np.array([a / 8, b / 8, 2.0 ** -k])]
            assert all((np.float32(x) == x).all() for x in q)
            e = float(_quality_mp(*q))
            c = oracle.tri_quality(*q)
            assert abs(c - e) <= QUALITY_ABS_BOUND and c > 0
            assert abs(c - e) <= 1e-12 * e


@pytest.mark.slow
def test_fma_order_moves_keys_only_through_the_placement():
    """Reading R13 fixes one float64 evaluation order of Eq. 1 (explicit fused
    multiply-adds).  Against the same formulas with every fused multiply-add
    split into a multiply and an add, on the 1,310,720-face benchmark mesh
    (round 0, 1,966,080 edges): eligibility, link results and the
    solved/fallback choice of every placement agree, and every key that moves
    does so because the float32 placement moved -- the Cramer solve is
    ill-conditioned on this fine, smooth mesh, so its last float32 bit depends
    on the order in most edges.  Counts (stated beside R13): 1,711,870
    placements and 1,249,136 keys differ."""
    V, F, _ = meshgen.mesh_config("bumped_icosphere_l8")
    A = oracle.edge_table(V, F)
    B = oracle.edge_table(V, F, plain_products=True)
    assert (A["ab"] == B["ab"]).all() and (A["link_ok"] == B["link_ok"]).all()
    assert (np.isnan(A["vsolve"][:, 0]) == np.isnan(B["vsolve"][:, 0])).all()
    assert ((A["key"] == ~np.uint64(0)) == (B["key"] == ~np.uint64(0))).all()
    moved_key = A["key"] != B["key"]
    moved_vbar = (A["vbar"] != B["vbar"]).any(1)
    assert not (moved_key & ~moved_vbar).any()
    # the two float64 solves agree to the conditioning of the 3x3 systems
    solved = ~np.isnan(A["vsolve"][:, 0])
    rel = (np.linalg.norm(A["vsolve"][solved] - B["vsolve"][solved], axis=1)
           / np.linalg.norm(A["vsolve"][solved], axis=1))
    assert rel.max() < 1e-3
    assert moved_vbar.sum() == 1711870 and moved_key.sum() == 1249136


@pytest.fixture(scope="module")
def torus_table():
    V, F, _ = meshgen.mesh_config("torus_64x32")
    return V, F, oracle.edge_table(V, F)


def test_edge_ids_are_sorted_unique_mesh_edges(torus_table):
    V, F, T = torus_table
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    ref = np.unique(np.sort(e, 1), axis=0)
    assert (T["ab"] == ref).all()
    lo = (T["key"] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    assert (lo == np.arange(len(lo))).all()


def test_qem_equals_sum_of_squared_plane_distances(torus_table):
    V, F, T = torus_table
    rng = np.random.default_rng(3)
    for i in rng.choice(len(T["ab"]), 40, replace=False):
        a, b = T["ab"][i]
        v = _mpv(T["vbar"][i])
        q = mpmath.mpf(0)
        for x in (a, b):   # K_a + K_b: faces on edge ab count twice
            for f in np.where((F == x).any(1))[0]:
                n, d = _plane(*V[F[f]])
                q += (sum(n[k] * v[k] for k in range(3)) + d) ** 2
        assert abs(T["Q"][i] - float(q)) <= 1e-12
        # the placement is no worse than the fallback candidates
        for cand in (V[a], V[b]):
            c = _mpv(cand)
            qc = mpmath.mpf(0)
            for x in (a, b):
                for f in np.where((F == x).any(1))[0]:
                    n, d = _plane(*V[F[f]])
                    qc += (sum(n[k] * c[k] for k in range(3)) + d) ** 2
            assert float(q) <= float(qc) + 1e-12


def test_length_and_skinny_terms(torus_table):
    V, F, T = torus_table
    rng = np.random.default_rng(4)
    for i in rng.choice(len(T["ab"]), 40, replace=False):
        a, b = T["ab"][i]
        pa, pb = _mpv(V[a]), _mpv(V[b])
        l = mpmath.sqrt(sum((pb[k] - pa[k]) ** 2 for k in range(3)))
        assert abs(T["l"][i] - float(l)) <= 2 * np.finfo(float).eps * float(l)
        ring = np.where((F == a).any(1) | (F == b).any(1))[0]
        produced = [f for f in ring if not ((F[f] == a).any() and (F[f] == b).any())]
        assert len(produced) == len(ring) - 2
        cs = mpmath.mpf(0)
        for f in produced:
            q = [T["vbar"][i] if x in (a, b) else V[x] for x in F[f]]
            cs += 1 - _quality_mp(*q)
        assert abs(T["Cs"][i] - float(cs)) <= 1e-13


def test_cost_combination_and_key_bits(torus_table):
    V, F, T = torus_table
    ext = (V.astype(np.float64).max(0) - V.astype(np.float64).min(0)).max()
    s = 1.0 / ext
    want = s * s * T["Q"] + oracle.W_E * s * T["l"] + oracle.W_S * T["Cs"]
    assert np.allclose(T["cost"], want, rtol=1e-14, atol=0)
    hi = (T["key"] >> np.uint64(32)).astype(np.uint32)
    bits = np.array([struct.unpack("<I", struct.pack("<f", np.float32(c)))[0]
                     for c in T["cost"]], np.uint32)
    assert (hi == bits).all()


@pytest.mark.parametrize("k", [-3, 1, 5])
def test_power_of_two_scale_invariance(torus_table, k):
    V, F, T = torus_table
    T2 = oracle.edge_table((V * np.float32(2.0 ** k)).astype(np.float32), F)
    assert (T2["key"] == T["key"]).all()
    assert (T2["vbar"] == T["vbar"] * np.float32(2.0 ** k)).all()


def test_link_condition_special_meshes():
    V, F = meshgen.tetrahedron()
    assert not oracle.edge_table(V, F)["link_ok"].any()
    V, F = meshgen.octahedron()
    T = oracle.edge_table(V, F)
    assert len(T["ab"]) == 12 and T["link_ok"].all()
    # split octahedron face (0,2,4) 1-to-3 around a new valence-3 vertex 6
    V2 = np.concatenate([V, np.array([[0.3, 0.3, 0.3]], np.float32)])
    keep = [f for f in F.tolist() if sorted(f) != [0, 2, 4]]
    F2 = np.array(keep + [[6, 0, 2], [6, 2, 4], [6, 4, 0]], np.int32)
    T = oracle.edge_table(V2, F2)
    bad = {tuple(x) for x in T["ab"][~T["link_ok"]].tolist()}
    assert bad == {(0, 2), (2, 4), (0, 4)}


@pytest.mark.parametrize("mesh,tol", [("torus", 1e-10), ("sphere4", 1e-8), ("sphere6", 1e-5)])
def test_placement_float64_error_statement(mesh, tol):
    # Precision of the placement (R2): the float64 Cramer solve against a
    # 50-digit solve of the same float64 system; the error grows with the
    # conditioning of A (flatter neighbourhoods at finer levels), bounded below
    V, F = {"torus": lambda: meshgen.torus(),
            "sphere4": lambda: meshgen.bumped_icosphere(4, 3),
            "sphere6": lambda: meshgen.bumped_icosphere(6, 0)}[mesh]()
    T = oracle.edge_table(V, F)
    K = oracle.vertex_quadrics(V, F)
    solved = np.where(~np.isnan(T["vsolve"][:, 0]))[0]
    idx = np.random.default_rng(1).choice(solved, min(800, len(solved)), replace=False)
    worst, flips = 0.0, 0
    for i in idx:
        a, b = T["ab"][i]
        k = K[a] + K[b]
        A = mpmath.matrix([[k[0], k[1], k[2]], [k[1], k[4], k[5]], [k[2], k[5], k[7]]])
        v = mpmath.lu_solve(A, mpmath.matrix([-k[3], -k[6], -k[8]]))
        vm = np.array([float(x) for x in v])
        worst = max(worst, np.linalg.norm(T["vsolve"][i] - vm) / np.linalg.norm(vm))
        flips += int((np.float32(vm) != T["vbar"][i]).any())
    assert worst < tol
    assert flips <= 0.1 * len(idx)


@pytest.mark.parametrize("mesh", ["torus", "sphere5", "sphere7"])
def test_cost_float64_error_statement(mesh):
    """Precision of the cost itself (Eq. 1): at the oracle's float32 placement,
    the float64 cost against Eq. 1 evaluated in 40-digit arithmetic from its
    definitions -- Q as the sum of squared distances to the incident face
    planes, the exact edge length, the exact skinny term.  Measured: relative
    error below 5e-13 on all three meshes, and every sampled float32 key equal
    to the correctly rounded exact cost, so a key differs from the plain
    definition's only through the placement (reading R13)."""
    mpmath.mp.dps = 40
    V, F = {"torus": lambda: meshgen.torus(),
            "sphere5": lambda: meshgen.bumped_icosphere(5, 0),
            "sphere7": lambda: meshgen.bumped_icosphere(7, 0)}[mesh]()
    T = oracle.edge_table(V, F)
    s = 1 / mpmath.mpf(float((V.astype(np.float64).max(0) - V.astype(np.float64).min(0)).max()))
    faces_of = {}
    for f, t in enumerate(F):
        for x in t:
            faces_of.setdefault(int(x), []).append(f)
    worst, flips = 0.0, 0
    idx = np.random.default_rng(11).choice(len(T["ab"]), 300, replace=False)
    for i in idx:
        a, b = map(int, T["ab"][i])
        v = _mpv(T["vbar"][i])
        Q = mpmath.mpf(0)
        for x in (a, b):  # K_a + K_b: the faces on ab count twice
            for f in faces_of[x]:
                n, d = _plane(*V[F[f]])
                Q += (sum(n[k] * v[k] for k in range(3)) + d) ** 2
        pa, pb = _mpv(V[a]), _mpv(V[b])
        l = mpmath.sqrt(sum((pb[k] - pa[k]) ** 2 for k in range(3)))
        Cs = mpmath.mpf(0)
        for f in sorted(set(faces_of[a]) | set(faces_of[b])):
            if a in F[f] and b in F[f]:
                continue
            Cs += 1 - _quality_mp(*[T["vbar"][i] if x in (a, b) else V[x] for x in F[f]])
        C = s * s * Q + mpmath.mpf(oracle.W_E) * s * l + mpmath.mpf(oracle.W_S) * Cs
        worst = max(worst, abs(T["cost"][i] - float(C)) / float(C))
        flips += int(np.float32(float(C)) != np.float32(T["cost"][i]))
    mpmath.mp.dps = 50
    assert worst < 1e-11, worst
    assert flips <= 1
