"""Pins for the oracle's round rule (Algorithm 1, Sections 5.1-5.3).

Selection is checked against the pairwise definition of independent regions
(an edge wins iff its key is below every other eligible key whose 1-ring shares
a triangle with its own) and against the per-vertex (pull) form of the
propagation; whole runs against the invariants the paper fixes: closed,
manifold, Euler characteristic and components preserved, face count at most
the target, and no self-intersection by an all-pairs exact scan.
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests.meshcheck import components, euler, is_closed_manifold


def _rings(F, ab):
    inc = {}
    for f, tri in enumerate(F.tolist()):
        for v in tri:
            inc.setdefault(v, set()).add(f)
    return [inc[a] | inc[b] for a, b in ab.tolist()], inc


@pytest.mark.parametrize("mesh", ["torus", "sphere3", "box"])
def test_round0_winners_pairwise_definition(mesh):
    if mesh == "torus":
        V, F, _ = meshgen.mesh_config("torus_64x32")
    elif mesh == "sphere3":
        V, F = meshgen.bumped_icosphere(3, 7)
    else:
        V, F = meshgen.box_grid(8)
    T = oracle.edge_table(V, F)
    r = oracle.simplify(V, F, len(F) - 1, max_rounds=1)
    got = {tuple(p) for p in r.rounds[0]["winner_pairs"].tolist()}
    rings, inc = _rings(F, T["ab"])
    elig = T["key"] != np.uint64(0xFFFFFFFFFFFFFFFF)
    by_face = {}
    for i in np.where(elig)[0]:
        for f in rings[i]:
            by_face.setdefault(f, []).append(i)
    want = set()
    for i in np.where(elig)[0]:
        rivals = {j for f in rings[i] for j in by_face[f]}
        if all(T["key"][i] < T["key"][j] for j in rivals if j != i):
            want.add(tuple(T["ab"][i].tolist()))
    assert got == want and len(got) > 0
    # pull form: vkey = min key over incident eligible edges; winner iff its key
    # equals the minimum vkey over the closed neighbourhoods of a and b
    vkey = np.full(len(V), np.uint64(0xFFFFFFFFFFFFFFFF))
    for i in np.where(elig)[0]:
        for v in T["ab"][i]:
            vkey[v] = min(vkey[v], T["key"][i])
    pull = set()
    for i in np.where(elig)[0]:
        a, b = T["ab"][i]
        verts = set(F[list(inc[a] | inc[b])].ravel().tolist())
        if all(T["key"][i] == min(vkey[w] for w in verts) for _ in [0]):
            pull.add((int(a), int(b)))
    assert pull == want
    # winners' regions are face-disjoint and their endpoints non-adjacent
    ids = [i for i in range(len(T["ab"])) if tuple(T["ab"][i].tolist()) in got]
    seen = set()
    for i in ids:
        assert not (rings[i] & seen)
        seen |= rings[i]


def _check_mesh(V, F, chi, comps):
    assert is_closed_manifold(F, len(V))
    assert euler(F, len(V)) == chi
    assert components(F, len(V)) == comps
    _, n = oracle.self_intersections(V, F, brute=True)
    assert n == 0


def test_torus_run_invariants(torus_mesh):
    V, F, target = torus_mesh
    r = oracle.simplify(V, F, target)
    assert r.status == 0 and len(r.F) <= target
    _check_mesh(r.V, r.F, 0, 1)
    for a, b in zip(r.rounds, r.rounds[1:]):
        c = a["committed"]
        assert b["nF"] == a["nF"] - 2 * c
        assert b["nV"] == a["nV"] - c
        assert b["nE"] == a["nE"] - 3 * c
    for d in r.rounds:
        assert d["committed"] + d["undone"] == d["winners"]


@pytest.mark.parametrize("rounds", [1, 5, 20])
def test_torus_intermediate_rounds_valid(torus_mesh, rounds):
    V, F, target = torus_mesh
    r = oracle.simplify(V, F, target, max_rounds=rounds)
    assert len(r.rounds) == rounds
    _check_mesh(r.V, r.F, 0, 1)


def test_check_scope_equivalence_with_undos():
    """Checking only changed faces (grid or brute force) gives the same run as
    checking every face pair, because M_1 is intersection-free (Alg. 3)."""
    V, F = meshgen.nested_shells(3, check=False)
    target = len(F) // 12
    runs = [oracle.simplify(V, F, target, check_mode=m)
            for m in (oracle.CHECK_GRID, oracle.CHECK_CHANGED_BRUTE, oracle.CHECK_ALL_PAIRS)]
    assert sum(d["undone"] for d in runs[0].rounds) > 0
    for r in runs[1:]:
        assert (r.V == runs[0].V).all() and (r.F == runs[0].F).all()
        for x, y in zip(r.rounds, runs[0].rounds):
            for k in ("winners", "committed", "undone", "undo_iters"):
                assert x[k] == y[k]
            assert (x["committed_pairs"] == y["committed_pairs"]).all()
    _check_mesh(runs[0].V, runs[0].F, 4, 2)


def test_shells_flags_follow_undos():
    V, F = meshgen.nested_shells(4, check=False)
    r = oracle.simplify(V, F, len(F) // 50)
    _check_mesh(r.V, r.F, 4, 2)
    hold = 0
    seen_undo = False
    for cur, nxt in zip(r.rounds, r.rounds[1:]):
        seen_undo |= cur["undone"] > 0
        if cur["committed"] > 0:
            hold = 0
            assert nxt["flagged"] == cur["undone"]   # Sec. 5.3: one round of flags
        else:
            hold += 1
            if hold >= oracle.TOLERANCE:
                hold = 0
                assert nxt["flagged"] == 0         # tolerance reached: cleared
            else:
                assert nxt["flagged"] >= cur["flagged"]
    assert seen_undo


def test_box_with_planar_sides():
    V, F = meshgen.box_grid(8)
    r = oracle.simplify(V, F, 40)
    _check_mesh(r.V, r.F, 2, 1)
    assert len(r.F) <= 40 or r.status == 4


def test_stall_on_tetrahedron_and_octahedron_to_tetrahedron():
    V, F = meshgen.tetrahedron()
    r = oracle.simplify(V, F, 2)
    assert r.status == 4 and len(r.F) == 4 and r.rounds[0]["eligible"] == 0
    V, F = meshgen.octahedron()
    r = oracle.simplify(V, F, 4)
    assert r.status == 0 and len(r.F) == 4
    _check_mesh(r.V, r.F, 2, 1)


# ------------------------------------------------ termination refinements
# Section 5.1 names two termination criteria: a target face count (the default
# above) and a target edge cost.  exact_target keeps only the winners needed to
# land on N_t; max_cost makes costlier edges ineligible.
def _same_rounds(a, b):
    for k in oracle.ROUND_FIELDS:
        if a[k] != b[k]:
            return False
    return all(np.array_equal(a[k], b[k])
               for k in ("winner_pairs", "committed_pairs", "undone_pairs"))


def test_exact_target_single_collapse_is_the_global_minimum():
    # N_t = |F| - 2: one collapse is needed, so the trimmed round keeps the
    # edge with the smallest key of the whole mesh (always a winner)
    V, F = meshgen.bumped_icosphere(3, 7)
    T = oracle.edge_table(V, F)
    r = oracle.simplify(V, F, len(F) - 2, exact_target=1)
    e = int(np.argmin(T["key"]))
    assert len(r.rounds) == 1 and r.rounds[0]["winners"] == 1
    assert r.rounds[0]["winner_pairs"].tolist() == [T["ab"][e].tolist()]
    assert len(r.F) == len(F) - 2


def test_exact_target_lands_on_target_and_only_trims_when_needed(torus_mesh):
    V, F, _ = torus_mesh
    target = 1000
    plain = oracle.simplify(V, F, target)
    exact = oracle.simplify(V, F, target, exact_target=1)
    assert len(plain.F) < target           # Algorithm 1 overshoots here
    assert exact.status == 0 and len(exact.F) == target
    k = next(i for i, (a, b) in enumerate(zip(plain.rounds, exact.rounds))
             if not _same_rounds(a, b))
    a, b = plain.rounds[k], exact.rounds[k]
    need = (b["nF"] - target + 1) // 2
    assert b["winners"] == need < a["winners"]
    kept = {tuple(p) for p in b["winner_pairs"].tolist()}
    assert kept <= {tuple(p) for p in a["winner_pairs"].tolist()}
    V2, F2 = exact.V, exact.F
    assert is_closed_manifold(F2, len(V2)) and euler(F2, len(V2)) == 0


def test_max_cost_round0_eligibility_and_normal_end(torus_mesh):
    V, F, target = torus_mesh
    T = oracle.edge_table(V, F)
    finite = T["key"] != np.uint64(0xFFFFFFFFFFFFFFFF)
    c = float(np.quantile(T["cost"][finite], 0.3))
    r = oracle.simplify(V, F, 0, max_cost=c)
    want = int((finite & (T["cost"].astype(np.float32) <= np.float32(c))).sum())
    assert r.rounds[0]["eligible"] == want
    assert r.status == 0 and len(r.F) > 0          # ended by the cost target
    assert r.rounds[-1]["eligible"] == 0
    assert is_closed_manifold(r.F, len(r.V)) and euler(r.F, len(r.V)) == 0
    # nothing costs less than zero: max_cost = 0 stops at once, unchanged
    z = oracle.simplify(V, F, target, max_cost=0.0)
    assert z.status == 0 and len(z.rounds) == 1 and np.array_equal(z.F, F)
    # +infinity is the default rule
    d, i = oracle.simplify(V, F, target), oracle.simplify(V, F, target, max_cost=np.inf)
    assert all(_same_rounds(a, b) for a, b in zip(d.rounds, i.rounds))


def _bad_pct(V, F, alpha):
    P = np.asarray(V, np.float64)[np.asarray(F)]
    m = np.full(len(F), 180.0)
    for i in range(3):
        u = P[:, (i + 1) % 3] - P[:, i]
        w = P[:, (i + 2) % 3] - P[:, i]
        c = (u * w).sum(1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(w, axis=1))
        m = np.minimum(m, np.degrees(np.arccos(np.clip(c, -1, 1))))
    return 100.0 * (m < alpha).mean()


@pytest.mark.parametrize("mesh", ["box16", "torus"])
def test_edge_cost_terms_reduce_bad_triangles(mesh):
    # the edge-cost ablation of the paper: with both extra terms of Eq. 1 the
    # output has the fewest triangles whose smallest angle is below 10 degrees,
    # and QEM alone is clearly worse (flat regions, where QEM is constant)
    V, F = meshgen.box_grid(16) if mesh == "box16" else meshgen.torus()
    target = len(F) // 10
    bad = {}
    for name, (w_e, w_s) in {"full": (0.001, 0.005), "no_ce": (0.0, 0.005),
                             "no_cs": (0.001, 0.0), "none": (0.0, 0.0)}.items():
        r = oracle.simplify(V, F, target, w_e=w_e, w_s=w_s, keep_pairs=False)
        assert is_closed_manifold(r.F, len(r.V))
        bad[name] = _bad_pct(r.V, r.F, 10.0)
    assert bad["full"] <= min(bad["no_ce"], bad["no_cs"], bad["none"])
    assert bad["none"] >= bad["full"] + 2.0


def test_recompute_quadrics_is_memoryless(torus_mesh):
    # With recompute_quadrics (R16) a round's costs depend only on the current
    # mesh (and the flags, empty while nothing is undone), so k rounds equal k
    # fresh one-round runs chained, each starting from face-plane quadrics.
    V, F, target = torus_mesh
    Vk, Fk = V, F
    for k in range(1, 6):
        step = oracle.simplify(Vk, Fk, target, max_rounds=1, keep_pairs=False)
        assert step.rounds[0]["undone"] == 0
        Vk, Fk = step.V, step.F
        full = oracle.simplify(V, F, target, max_rounds=k, keep_pairs=False, recompute_quadrics=1)
        assert np.array_equal(full.F, Fk) and np.array_equal(full.V, Vk), k
    # and it is a different rule from carrying K_a + K_b once collapses happened
    carry = oracle.simplify(V, F, target, keep_pairs=False)
    fresh = oracle.simplify(V, F, target, keep_pairs=False, recompute_quadrics=1)
    assert not (np.array_equal(carry.F, fresh.F) and np.array_equal(carry.V, fresh.V))
    assert is_closed_manifold(fresh.F, len(fresh.V)) and euler(fresh.F, len(fresh.V)) == 0
