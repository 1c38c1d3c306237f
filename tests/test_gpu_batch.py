"""GPU batch path (many meshes per pass): every mesh of the batch must come
out bit-identical to the oracle simplifying that mesh alone -- same faces,
same position bits, same status, same number of rounds.

The batch runs Algorithm 1 once per round over the disjoint union of all
meshes; what must not leak between meshes is each one's normalisation
(Section 4 start), flags and tolerance count (Section 5.3), termination, and
the intersection check (pairs are only tested within a mesh).
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
from tests.test_gpu_parity import _bits  # noqa: E402


def _run_batch(meshes, targets, **opts):
    V, voff, F, foff = pamo.concat_meshes(meshes)
    Vo, vo, Fo, fo, status, rounds, stats = pamo.pamo_simplify_batch(
        torch.from_numpy(V), voff, torch.from_numpy(F), foff, targets, **opts)
    Vo, Fo = Vo.cpu().numpy(), Fo.cpu().numpy()
    out = [(Vo[vo[m]:vo[m + 1]], Fo[fo[m]:fo[m + 1]]) for m in range(len(meshes))]
    return out, status, rounds, stats


def _assert_batch_matches_oracle(meshes, targets, **opts):
    out, status, rounds, stats = _run_batch(meshes, targets, **opts)
    for m, ((V, F), t) in enumerate(zip(meshes, targets)):
        ref = oracle.simplify(V, F, t, keep_pairs=False, **opts)
        gV, gF = out[m]
        assert np.array_equal(gF, ref.F), m
        assert np.array_equal(_bits(gV), _bits(ref.V)), m
        assert status[m] == ("PAMO_OK" if ref.status == 0 else "PAMO_ESTALL"), m
        assert rounds[m] == len(ref.rounds), (m, rounds[m], len(ref.rounds))
    return out, status, rounds, stats


def test_mixed_batch_bit_exact():
    meshes = [meshgen.torus(32, 16, 1.0, 0.3, 0.002, 1),
              meshgen.bumped_icosphere(4, 5),
              meshgen.torus(64, 32, 1.0, 0.45, 0.002, 2),
              meshgen.nested_shells(3, check=False),   # undo loops
              meshgen.box_grid(6),                     # exact-predicate paths
              meshgen.bumped_icosphere(3, 8)]
    targets = [len(F) // 10 for _, F in meshes]
    targets[3] = len(meshes[3][1]) // 12
    _assert_batch_matches_oracle(meshes, targets)


def test_batch_with_idle_and_stalling_meshes():
    octa = meshgen.octahedron()
    meshes = [meshgen.bumped_icosphere(3, 1), octa, meshgen.torus(24, 12, 1.0, 0.3, 0.002, 3),
              meshgen.bumped_icosphere(3, 2)]
    # mesh 1 cannot reach 2 faces (stall); mesh 3's target is above its size
    targets = [len(meshes[0][1]) // 20, 2, len(meshes[2][1]) // 10, 10 ** 9]
    out, status, rounds, _ = _assert_batch_matches_oracle(meshes, targets)
    assert status[1] == "PAMO_ESTALL" and rounds[3] == 0
    assert np.array_equal(out[3][1], meshes[3][1])


def test_generated_batch_bit_exact():
    meshes = meshgen.batch_meshes(count=10, seed0=4000, fmin=2000, fmax=30000)
    targets = [len(F) // 100 for _, F in meshes]
    _assert_batch_matches_oracle(meshes, targets)


@pytest.mark.parametrize("opts", [dict(check_mode=1), dict(max_cost=2e-3),
                                  dict(w_e=0.0, w_s=0.0)])
def test_batch_options_bit_exact(opts):
    meshes = [meshgen.bumped_icosphere(3, 11), meshgen.nested_shells(3, check=False),
              meshgen.torus(32, 16, 1.0, 0.25, 0.002, 5)]
    targets = [len(F) // 15 for _, F in meshes]
    out, status, rounds, _ = _run_batch(meshes, targets, **opts)
    # the oracle's check scope does not change its results (C-15)
    oopts = {k: v for k, v in opts.items() if k != "check_mode"}
    for m, ((V, F), t) in enumerate(zip(meshes, targets)):
        ref = oracle.simplify(V, F, t, keep_pairs=False, **oopts)
        assert np.array_equal(out[m][1], ref.F), m
        assert np.array_equal(_bits(out[m][0]), _bits(ref.V)), m
        assert rounds[m] == len(ref.rounds), m


def test_batch_rejects_bad_input():
    V, F = meshgen.bumped_icosphere(3, 0)
    bad = F.copy()
    bad[5, 1] = len(V)  # outside its own mesh
    Vc, voff, Fc, foff = pamo.concat_meshes([(V, F), (V, bad)])
    with pytest.raises(pamo.PamoError, match="EINVAL"):
        pamo.pamo_simplify_batch(torch.from_numpy(Vc), voff, torch.from_numpy(Fc), foff,
                                 [100, 100])
    Vc, voff, Fc, foff = pamo.concat_meshes([(V, F), (V, F)])
    with pytest.raises(pamo.PamoError, match="EINVAL"):
        pamo.pamo_simplify_batch(torch.from_numpy(Vc), voff, torch.from_numpy(Fc), foff,
                                 [100, 100], exact_target=1)


def test_autotune_picks_knobs_and_keeps_results():
    meshes = [meshgen.bumped_icosphere(4, 12), meshgen.torus(48, 24, 1.0, 0.35, 0.002, 9),
              meshgen.bumped_icosphere(3, 13)]
    targets = [len(F) // 50 for _, F in meshes]
    V, voff, F, foff = pamo.concat_meshes(meshes)
    best, trials = pamo.pamo_autotune_batch(torch.from_numpy(V), voff, torch.from_numpy(F),
                                            foff, targets)
    assert len(trials) == 6 and all(t > 0 for t in trials)
    assert best.resort_percent in (25, 50, 75, 100) and best.grid_blocks_per_sm in (4, 6, 8)
    out, status, rounds, _ = _run_batch(meshes, targets, resort_percent=best.resort_percent,
                                        grid_blocks_per_sm=best.grid_blocks_per_sm)
    for m, ((Vm, Fm), t) in enumerate(zip(meshes, targets)):
        ref = oracle.simplify(Vm, Fm, t, keep_pairs=False)
        assert np.array_equal(out[m][1], ref.F) and np.array_equal(_bits(out[m][0]), _bits(ref.V))


def test_batch_in_one_graph_launch_bit_exact():
    """options.device_loop: the whole batch as one graph launch, every mesh's
    Section 5.3 bookkeeping (flags, tolerance, stall, target, status) kept by
    device kernels; every mesh still equals the oracle simplifying it alone."""
    octa = meshgen.octahedron()
    tet = meshgen.tetrahedron()
    meshes = [meshgen.torus(32, 16, 1.0, 0.3, 0.002, 1), meshgen.nested_shells(4, check=False),
              octa, tet, meshgen.box_grid(6), meshgen.bumped_icosphere(4, 5)]
    targets = [len(meshes[0][1]) // 10, len(meshes[1][1]) // 50, 4, 2, 30,
               len(meshes[5][1]) // 20]
    V, voff, F, foff = pamo.concat_meshes(meshes)
    Vo, vo, Fo, fo, status, rounds, stats = pamo.pamo_simplify_batch(
        torch.from_numpy(V), voff, torch.from_numpy(F), foff, targets, device_loop=1)
    Vo, Fo = Vo.cpu().numpy(), Fo.cpu().numpy()
    for m, ((Vm, Fm), t) in enumerate(zip(meshes, targets)):
        ref = oracle.simplify(Vm, Fm, t, keep_pairs=False)
        assert np.array_equal(Fo[fo[m]:fo[m + 1]], ref.F), m
        assert np.array_equal(_bits(Vo[vo[m]:vo[m + 1]]), _bits(ref.V)), m
        assert status[m] == ("PAMO_OK" if ref.status == 0 else "PAMO_ESTALL"), m
        assert rounds[m] == len(ref.rounds), m
    assert "PAMO_ESTALL" in list(status)  # the tetrahedron cannot collapse
