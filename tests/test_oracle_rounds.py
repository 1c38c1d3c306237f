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
