"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: integer and index results bit-exact --
per-round winner / committed / undone collapse sets, every counter, and the
output connectivity; positions bit-identical (float32 bits), which implies
the required 1e-12 x bbox-diagonal bound; edge keys bit-identical (the FP64
cost runs without contraction on both sides).
"""
import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2509_05595_gb300 as pamo  # noqa: E402
from tests.meshcheck import components, euler, is_closed_manifold  # noqa: E402
from tests.test_oracle_predicates import _near_coplanar, _on_plane, _pair_stream  # noqa: E402


def _bits(a):
    return np.ascontiguousarray(a, np.float32).view(np.uint32)


# ---------------------------------------------------------------- predicates
def test_orient_batches_match_oracle():
    rng = np.random.default_rng(101)
    P3 = [rng.uniform(-1, 1, (4, 3)) for _ in range(2000)]
    P3 += [p for p in _near_coplanar(rng, 2000)]
    P3 += [rng.integers(-3, 4, (4, 3)) for _ in range(2000)]
    for _ in range(2000):  # exponent-gap adversarial cases
        n = rng.integers(-3, 4, 3)
        if not n.any():
            continue
        a, b, c = (_on_plane(rng, n, 2.0 ** rng.integers(10, 40)) for _ in range(3))
        d = (_on_plane(rng, n, 2.0 ** rng.integers(-40, -10))
             + rng.integers(-1, 2, 3) * 2.0 ** rng.integers(-80, -40))
        P3.append(np.array([a, b, c, d]))
    P3 = np.array([np.asarray(p, np.float32) for p in P3], np.float32)
    got = pamo.pamo_orient3d_batch(torch.from_numpy(P3.reshape(-1, 12))).cpu().numpy()
    want = np.array([oracle.orient3d(*p, exact=True) for p in P3])
    assert (got == want).all()
    assert (want == 0).sum() > 500 and (want != 0).sum() > 1000
    P2 = P3[:, :3, :2].reshape(-1, 6).copy()
    got = pamo.pamo_orient2d_batch(torch.from_numpy(P2)).cpu().numpy()
    want = np.array([oracle.orient2d(*p.reshape(3, 2), exact=True) for p in P2])
    assert (got == want).all()


def test_triangle_pair_predicate_matches_oracle():
    rng = np.random.default_rng(202)
    Ps, Is = [], []
    for T, C, ti, ci in _pair_stream(rng, 20000):
        Ps.append(np.concatenate([np.asarray(T, np.float32).ravel(),
                                  np.asarray(C, np.float32).ravel()]))
        Is.append(np.array(list(ti) + list(ci), np.int32))
    P = np.array(Ps, np.float32)
    idx = np.array(Is, np.int32)
    got = pamo.pamo_tri_intersect_batch(torch.from_numpy(P), torch.from_numpy(idx)).cpu().numpy()
    want = np.array([oracle.tri_intersect(p[:9].reshape(3, 3), p[9:].reshape(3, 3),
                                          i[:3], i[3:]) for p, i in zip(P, idx)])
    assert (got == want).all(), np.where(got != want)[0][:10]
    assert want.sum() > 3000 and (~want).sum() > 3000


# ---------------------------------------------------------------- round 0
def _ctx_round0(V, F):
    c = pamo.Ctx(torch.from_numpy(V), torch.from_numpy(F))
    c.round_cost()
    _, _, K, E = c.export(keys=True)
    c.close()
    return K.cpu().numpy().view(np.uint64), E.cpu().numpy()


@pytest.mark.parametrize("mesh", ["torus", "sphere4", "box8", "shells3"])
def test_round0_keys_bit_exact(mesh):
    V, F = {
        "torus": lambda: meshgen.torus(),
        "sphere4": lambda: meshgen.bumped_icosphere(4, 3),
        "box8": lambda: meshgen.box_grid(8),
        "shells3": lambda: meshgen.nested_shells(3, check=False),
    }[mesh]()
    K, E = _ctx_round0(V, F)
    T = oracle.edge_table(V, F)
    assert (E == T["ab"]).all()
    assert (K == T["key"]).all(), np.where(K != T["key"])[0][:10]


# ---------------------------------------------------------------- full runs
def _gpu_run(V, F, target, **opts):
    c = pamo.Ctx(torch.from_numpy(V), torch.from_numpy(F), record_rounds=1, **opts)
    stats, status = c.run(target)
    n, _ = c.rounds()
    rounds = []
    for r in range(n):
        d = c.round_info(r)
        for kind, name in ((0, "winner_pairs"), (1, "committed_pairs"), (2, "undone_pairs")):
            d[name] = c.round_pairs(r, kind)
        rounds.append(d)
    Vo, Fo = c.export()
    c.close()
    return Vo.cpu().numpy(), Fo.cpu().numpy(), rounds, stats, status


def _assert_same_run(V, F, target, check_mode=oracle.CHECK_GRID, gpu_mode=0, gpu_only=None,
                     ref=None, **opts):
    """opts (w_e, w_s, exact_target, max_cost) go to both sides; gpu_only
    (speed-only knobs) to the GPU run alone; ref: an oracle run of the same
    arguments made earlier."""
    if ref is None:
        ref = oracle.simplify(V, F, target, check_mode=check_mode, **opts)
    gV, gF, rounds, stats, status = _gpu_run(V, F, target, check_mode=gpu_mode, **opts,
                                             **(gpu_only or {}))
    assert len(rounds) == len(ref.rounds)
    for r, (g, o) in enumerate(zip(rounds, ref.rounds)):
        for k in oracle.ROUND_FIELDS:
            assert g[k] == o[k], (r, k, g[k], o[k])
        for k in ("winner_pairs", "committed_pairs", "undone_pairs"):
            assert np.array_equal(g[k], o[k]), (r, k)
    assert status == ("PAMO_OK" if ref.status == 0 else "PAMO_ESTALL")
    assert np.array_equal(gF, ref.F)
    assert np.array_equal(_bits(gV), _bits(ref.V))
    return ref, stats


def test_torus_full_run_bit_exact(torus_mesh):
    V, F, target = torus_mesh
    ref, stats = _assert_same_run(V, F, target)
    assert stats["rounds"] == len(ref.rounds) and len(ref.F) <= target


@pytest.mark.parametrize("level,seed", [(4, 0), (5, 9)])
def test_bumped_sphere_full_run_bit_exact(level, seed):
    V, F = meshgen.bumped_icosphere(level, seed)
    _assert_same_run(V, F, len(F) // 100)


@pytest.mark.parametrize("level,div", [(3, 12), (4, 50), (5, 60)])
def test_nested_shells_with_undos_bit_exact(level, div):
    V, F = meshgen.nested_shells(level, check=False)
    ref, stats = _assert_same_run(V, F, len(F) // div)
    assert sum(d["undone"] for d in ref.rounds) > 0
    assert stats["undone"] == sum(d["undone"] for d in ref.rounds)


def test_candidate_overflow_fallback_bit_exact(monkeypatch):
    """Tiny candidate buffers force the fused-check fallback in every check
    iteration; the run must not change."""
    monkeypatch.setenv("PAMO_CAND_CAP_DIVISOR", "1000000")
    V, F = meshgen.nested_shells(4, check=False)
    _assert_same_run(V, F, len(F) // 50)


def test_planar_box_exercises_exact_predicates():
    V, F = meshgen.box_grid(8)
    _assert_same_run(V, F, 40)


def test_all_faces_check_mode_matches():
    V, F = meshgen.nested_shells(3, check=False)
    _assert_same_run(V, F, len(F) // 12, check_mode=oracle.CHECK_ALL_PAIRS, gpu_mode=1)


# ---------------------------------------------------------------- boundary
def test_simplify_entry_point_and_host_variant(torus_mesh):
    V, F, target = torus_mesh
    ref = oracle.simplify(V, F, target, keep_pairs=False)
    Vo, Fo, stats, status = pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F), target)
    assert status == "PAMO_OK"
    assert np.array_equal(Fo.cpu().numpy(), ref.F)
    assert np.array_equal(_bits(Vo.cpu().numpy()), _bits(ref.V))
    Vh, Fh, stats_h, status_h = pamo.pamo_simplify_host(V, F, target)
    assert np.array_equal(Fh, ref.F) and np.array_equal(_bits(Vh), _bits(ref.V))
    assert stats_h["rounds"] == stats["rounds"] == len(ref.rounds)


def test_stall_and_degenerate_targets():
    V, F = meshgen.tetrahedron()
    Vo, Fo, stats, status = pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F), 2)
    assert status == "PAMO_ESTALL" and len(Fo) == 4
    V, F = meshgen.octahedron()
    Vo, Fo, stats, status = pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F), 4)
    ref = oracle.simplify(V, F, 4)
    assert status == "PAMO_OK" and np.array_equal(Fo.cpu().numpy(), ref.F)
    V, F, _ = meshgen.mesh_config("torus_64x32")
    Vo, Fo, stats, status = pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F), len(F))
    assert stats["rounds"] == 0 and np.array_equal(Fo.cpu().numpy(), F)


def test_invalid_inputs_rejected():
    V, F, _ = meshgen.mesh_config("torus_64x32")
    with pytest.raises(pamo.PamoError, match="ENOTMANIFOLD"):
        pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F[:-2]), 100)  # open
    bad = F.copy()
    bad[5, 1] = len(V) + 7
    with pytest.raises(pamo.PamoError, match="EINVAL"):
        pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(bad), 100)
    Vn = V.copy()
    Vn[3, 2] = np.nan
    with pytest.raises(pamo.PamoError, match="EINVAL"):
        pamo.pamo_simplify(torch.from_numpy(Vn), torch.from_numpy(F), 100)
    flipped = F.copy()
    flipped[10] = flipped[10, [0, 2, 1]]
    with pytest.raises(pamo.PamoError, match="ENOTMANIFOLD"):
        pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(flipped), 100)


def test_self_intersection_check_matches_oracle():
    # two overlapping spheres: many genuine intersections
    V1, F1 = meshgen.bumped_icosphere(4, 1)
    V2, F2 = meshgen.bumped_icosphere(4, 2)
    V = np.concatenate([V1, V2 + np.float32(0.7)]).astype(np.float32)
    F = np.concatenate([F1, F2 + len(V1)]).astype(np.int32)
    pairs, n = oracle.self_intersections(V, F)
    gn, gp = pamo.pamo_check_self_intersections(torch.from_numpy(V), torch.from_numpy(F))
    assert gn == n > 100
    got = {tuple(p) for p in gp.cpu().numpy().tolist()}
    assert got == {tuple(p) for p in pairs.tolist()}
    # and a clean mesh reports none
    V, F = meshgen.nested_shells(4, check=False)
    gn, _ = pamo.pamo_check_self_intersections(torch.from_numpy(V), torch.from_numpy(F))
    assert gn == 0


def _deep_tree_soup(stack=1500):
    """A triangle soup whose LBVH is as deep as Morton keys let it be: flat
    triangles in the 30 cells whose Morton codes are single bits (a comb of
    depth 30 in the radix tree), and a stack of `stack` parallel slanted
    triangles inside cell (0, 0, 0) -- equal Morton keys, split by leaf index
    below the comb -- whose boxes overlap about 500 deep but which never meet.
    Two large triangles fix the box to [0, 1]^3.  All corners are exact in
    float32."""
    cell = 1.0 / 1023.0
    tris = [[[0, 0, 0], [1, 0, 0], [0, 1, 0]], [[1, 1, 1], [0.5, 1, 1], [1, 0.5, 1]]]
    for axis in range(3):
        for j in range(10):
            c = np.full(3, 0.25 * cell)
            c[axis] = (2 ** j + 0.25) * cell
            z = np.float32(c[2])
            tris.append([[c[0], c[1], z], [c[0] + 0.25 * cell, c[1], z],
                         [c[0], c[1] + 0.25 * cell, z]])
    a, b, h = 2.0 ** -13, 2.0 ** -14, 2.0 ** -15
    for i in range(stack):
        x0, y0, z0 = 2.0 ** -12, 2.0 ** -12, 2.0 ** -12 + i * 2.0 ** -24
        tris.append([[x0, y0, z0], [x0 + a, y0, z0 + b], [x0, y0 + a, z0 + h]])
    V = np.asarray(tris, np.float32).reshape(-1, 3)
    F = np.arange(len(V), dtype=np.int32).reshape(-1, 3)
    return V, F


def test_check_on_a_deep_tree_matches_oracle():
    V, F = _deep_tree_soup()
    pairs, n = oracle.self_intersections(V, F)
    assert n == 0
    gn, _ = pamo.pamo_check_self_intersections(torch.from_numpy(V), torch.from_numpy(F))
    assert gn == 0
    # and with one stacked triangle tilted through its neighbours
    V2 = V.copy()
    k = 3 * (2 + 30 + 700)
    V2[k + 1, 2] += np.float32(2.0 ** -16)
    pairs, n = oracle.self_intersections(V2, F)
    gn, gp = pamo.pamo_check_self_intersections(torch.from_numpy(V2), torch.from_numpy(F))
    assert gn == n > 0
    assert {tuple(p) for p in gp.cpu().numpy().tolist()} == {tuple(p) for p in pairs.tolist()}


# ---------------------------------------------------------------- full size
@pytest.fixture(scope="module")
def sphere_l8():
    return meshgen.mesh_config("bumped_icosphere_l8")


@pytest.fixture(scope="module")
def sphere_l8_ref(sphere_l8):
    V, F, target = sphere_l8
    return oracle.simplify(V, F, target)


def test_full_size_round0_keys_bit_exact(sphere_l8):
    V, F, _ = sphere_l8
    K, E = _ctx_round0(V, F)
    T = oracle.edge_table(V, F)
    assert (E == T["ab"]).all()
    assert (K == T["key"]).all()


def test_full_size_run_bit_exact(sphere_l8, sphere_l8_ref):
    """The benchmark workload itself, 1,310,720 -> <= 13,107 faces: every
    round's winner, committed and undone sets and counters, the output faces
    and the position bits equal the oracle's (Algorithm 1, Eq. 1)."""
    V, F, target = sphere_l8
    ref, stats = _assert_same_run(V, F, target, ref=sphere_l8_ref)
    assert len(ref.rounds) > 40 and len(ref.F) <= target


def test_full_size_run_properties(sphere_l8, sphere_l8_ref):
    """1,310,720 -> <= 13,107 faces in the launch configuration the benchmark
    times (pamo_simplify, validation off): bit-identical to the oracle,
    manifold, genus 0, one component, under the target, and free of
    self-intersections by both the GPU check and the oracle's exact scan."""
    V, F, target = sphere_l8
    Vo, Fo, stats, status = pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F),
                                               target, validate_input=0)
    Vo, Fo = Vo.cpu().numpy(), Fo.cpu().numpy()
    ref = sphere_l8_ref
    assert np.array_equal(Fo, ref.F) and np.array_equal(_bits(Vo), _bits(ref.V))
    assert stats["rounds"] == len(ref.rounds)
    assert status == "PAMO_OK" and len(Fo) <= target
    assert is_closed_manifold(Fo, len(Vo))
    assert euler(Fo, len(Vo)) == 2 and components(Fo, len(Vo)) == 1
    gn, _ = pamo.pamo_check_self_intersections(torch.from_numpy(Vo), torch.from_numpy(Fo))
    assert gn == 0
    _, n = oracle.self_intersections(Vo, Fo)
    assert n == 0


def test_nested_shells_l6_full_parity():
    """163,840 faces of near-contact shells (many undos): the full run is
    bit-identical to the oracle."""
    V, F = meshgen.nested_shells(6, check=False)
    ref, _ = _assert_same_run(V, F, len(F) // 100)
    assert sum(d["undone"] for d in ref.rounds) > 100


@pytest.fixture(scope="module")
def shells_l8():
    return meshgen.mesh_config("nested_shells_l8")


def test_nested_shells_full_size_round0_keys(shells_l8):
    V, F, _ = shells_l8
    K, E = _ctx_round0(V, F)
    T = oracle.edge_table(V, F)
    assert (E == T["ab"]).all()
    assert (K == T["key"]).all()


@pytest.fixture(scope="module")
def shells_l8_ref(shells_l8):
    V, F, target = shells_l8
    return oracle.simplify(V, F, target)


def test_nested_shells_full_size_run_bit_exact(shells_l8, shells_l8_ref):
    """The near-contact stress at full size, 2,621,440 faces -> 0.1 %: per-round
    sets and counters (including the undo iterations of Section 5.3), output
    faces and position bits equal the oracle's."""
    V, F, target = shells_l8
    ref, stats = _assert_same_run(V, F, target, ref=shells_l8_ref)
    assert sum(d["undone"] for d in ref.rounds) > 0
    assert stats["undone"] == sum(d["undone"] for d in ref.rounds)


def test_nested_shells_full_size_run_properties(shells_l8, shells_l8_ref):
    """2,621,440 faces -> 0.1 % through pamo_simplify (validation off): the
    oracle's output, two closed manifold shells that nearly touch; the output
    must stay manifold, keep both components and be free of
    self-intersections, checked by the GPU and by the oracle's exact scan."""
    V, F, target = shells_l8
    Vo, Fo, stats, status = pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F),
                                               target, validate_input=0)
    Vo, Fo = Vo.cpu().numpy(), Fo.cpu().numpy()
    assert np.array_equal(Fo, shells_l8_ref.F)
    assert np.array_equal(_bits(Vo), _bits(shells_l8_ref.V))
    assert status in ("PAMO_OK", "PAMO_ESTALL")
    if status == "PAMO_OK":
        assert len(Fo) <= target
    assert stats["undone"] > 0
    assert is_closed_manifold(Fo, len(Vo))
    assert euler(Fo, len(Vo)) == 4 and components(Fo, len(Vo)) == 2
    gn, _ = pamo.pamo_check_self_intersections(torch.from_numpy(Vo), torch.from_numpy(Fo))
    assert gn == 0
    _, n = oracle.self_intersections(Vo, Fo)
    assert n == 0
