"""GPU parity of the option variants: the two termination refinements of
Section 5.1 (exact target face count, target edge cost) and the Eq. 1
ablation switches (w_e = 0, w_s = 0, both) of the edge-cost study.

Same bar as the plain path: per-round collapse sets, counters, output
connectivity and position bits identical to the oracle's.
"""
import numpy as np
import pytest

import meshgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from tests.test_gpu_parity import _assert_same_run  # noqa: E402


@pytest.mark.parametrize("mesh", ["torus", "sphere5", "shells4", "shells4_stall"])
def test_exact_target_bit_exact(mesh):
    V, F, target = {
        "torus": lambda: (*meshgen.mesh_config("torus_64x32")[:2], 1000),
        "sphere5": lambda: (*meshgen.bumped_icosphere(5, 9), 2 * 1023),
        "shells4": lambda: (*meshgen.nested_shells(4, check=False), 2400),
        # the trimmed winners get undone near the end: a stall, on both sides
        "shells4_stall": lambda: (*meshgen.nested_shells(4, check=False), 1400),
    }[mesh]()
    ref, stats = _assert_same_run(V, F, target, exact_target=1)
    if ref.status == 0:
        assert len(ref.F) == target  # even face counts: exactly N_t


def test_exact_target_single_collapse_is_global_minimum():
    V, F = meshgen.bumped_icosphere(4, 3)
    ref, _ = _assert_same_run(V, F, len(F) - 2, exact_target=1)
    T = oracle.edge_table(V, F)
    e = int(np.argmin(T["key"]))
    assert ref.rounds[0]["winners"] == 1
    assert ref.rounds[0]["winner_pairs"].tolist() == [T["ab"][e].tolist()]


@pytest.mark.parametrize("q", [0.0, 0.2, 0.6])
def test_max_cost_bit_exact(q):
    V, F = meshgen.bumped_icosphere(5, 4)
    T = oracle.edge_table(V, F)
    c = float(np.quantile(T["cost"], q)) if q > 0 else 0.0
    ref, _ = _assert_same_run(V, F, 64, max_cost=c)
    assert ref.status == 0  # the cost target ends the run normally
    assert ref.rounds[-1]["eligible"] == 0


@pytest.mark.parametrize("w_e,w_s", [(0.0, 0.005), (0.001, 0.0), (0.0, 0.0)])
def test_cost_ablation_switches_bit_exact(w_e, w_s):
    V, F = meshgen.bumped_icosphere(5, 2)
    _assert_same_run(V, F, len(F) // 50, w_e=w_e, w_s=w_s)
    Vt, Ft, target = meshgen.mesh_config("torus_64x32")
    _assert_same_run(Vt, Ft, target, w_e=w_e, w_s=w_s)


@pytest.mark.parametrize("knobs", [dict(resort_percent=100), dict(resort_percent=50),
                                   dict(grid_blocks_per_sm=2), dict(grid_blocks_per_sm=8)])
def test_speed_knobs_do_not_change_results(knobs):
    V, F = meshgen.bumped_icosphere(5, 6)
    _assert_same_run(V, F, len(F) // 100, **{"gpu_only": knobs})


@pytest.mark.parametrize("mesh", ["torus", "sphere5", "shells4"])
def test_recompute_quadrics_bit_exact(mesh):
    V, F, target = {
        "torus": lambda: meshgen.mesh_config("torus_64x32"),
        "sphere5": lambda: (*meshgen.bumped_icosphere(5, 3), 400),
        "shells4": lambda: (*meshgen.nested_shells(4, check=False), 2400),
    }[mesh]()
    _assert_same_run(V, F, target, recompute_quadrics=1)


def test_input_intersection_check_refuses_bad_input():
    from tests.test_gpu_parity import pamo as _pamo
    # seeds whose shells overlap (the generator's own disjointness check fails)
    V, F = meshgen.nested_shells(4, seeds=(2000, 6000), check=False)
    assert oracle.self_intersections(V, F)[1] > 0
    with pytest.raises(_pamo.PamoError, match="EINTERSECT"):
        _pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F), len(F) // 10,
                            check_input_intersections=1)
    # an intersection-free input is accepted and simplified exactly as the
    # oracle does it (the input check changes nothing else)
    Vg, Fg = meshgen.nested_shells_seeded(4, 2001)
    ref = oracle.simplify(Vg, Fg, len(Fg) // 10, keep_pairs=False)
    Vo, Fo, st, status = _pamo.pamo_simplify(torch.from_numpy(Vg), torch.from_numpy(Fg),
                                             len(Fg) // 10, check_input_intersections=1)
    assert status == ("PAMO_OK" if ref.status == 0 else "PAMO_ESTALL")
    assert st["rounds"] == len(ref.rounds) > 0
    assert np.array_equal(Fo.cpu().numpy(), ref.F)
    assert np.array_equal(Vo.cpu().numpy().view(np.uint32), ref.V.view(np.uint32))


def test_cached_memory_reuse_and_release_do_not_change_results():
    """Back-to-back calls reuse the library's pooled device memory and pinned
    mirrors (of other sizes too); releasing the cache between calls changes
    nothing either."""
    from tests.test_gpu_parity import pamo as _pamo
    Vs, Fs = meshgen.bumped_icosphere(5, 7)
    Vt, Ft, tt = meshgen.mesh_config("torus_64x32")
    Vd, Fd = torch.from_numpy(Vs).cuda(), torch.from_numpy(Fs).cuda()
    first = _pamo.pamo_simplify(Vd, Fd, len(Fs) // 20)
    outs = []
    for k in range(3):
        _pamo.pamo_simplify(torch.from_numpy(Vt), torch.from_numpy(Ft), tt)  # other sizes
        if k == 1:
            _pamo.pamo_release_cached_memory()
        outs.append(_pamo.pamo_simplify(Vd, Fd, len(Fs) // 20))
    for o in outs:
        assert o[3] == first[3] and o[2]["rounds"] == first[2]["rounds"]
        assert torch.equal(o[0], first[0]) and torch.equal(o[1], first[1])
    _pamo.pamo_release_cached_memory()


@pytest.mark.parametrize("case", ["shells_undos", "fallback", "box", "exact_target", "max_cost",
                                  "stall", "sphere"])
def test_device_round_loop_matches_oracle(case, monkeypatch):
    """With options.device_loop every round runs on the device (one graph:
    conditional loops over rounds and undo iterations, the Section 5.3 flag
    and stall bookkeeping in kernels).  Its output, status and round count
    equal the oracle's in every branch of that loop."""
    from tests.test_gpu_parity import pamo as _pamo
    opts = {}
    if case in ("shells_undos", "fallback"):
        V, F = meshgen.nested_shells(5, check=False)
        target = len(F) // 60
        if case == "fallback":  # tiny candidate buffers: the fused fallback check every time
            monkeypatch.setenv("PAMO_CAND_CAP_DIVISOR", "1000000")
    elif case == "box":
        V, F = meshgen.box_grid(8)
        target = 40
    elif case == "exact_target":
        V, F = meshgen.bumped_icosphere(5, 2)
        target, opts = 1001, dict(exact_target=1)
    elif case == "max_cost":
        V, F = meshgen.bumped_icosphere(5, 4)
        c = float(np.quantile(oracle.edge_table(V, F)["cost"], 0.6))
        target, opts = 64, dict(max_cost=c)
    elif case == "stall":
        V, F = meshgen.tetrahedron()
        target = 2
    else:
        V, F = meshgen.bumped_icosphere(6, 5)
        target = len(F) // 100
    ref = oracle.simplify(V, F, target, keep_pairs=False, **opts)
    Vo, Fo, st, status = _pamo.pamo_simplify(torch.from_numpy(V), torch.from_numpy(F), target,
                                             device_loop=1, **opts)
    assert status == ("PAMO_OK" if ref.status == 0 else "PAMO_ESTALL")
    assert st["rounds"] == len(ref.rounds)
    assert np.array_equal(Fo.cpu().numpy(), ref.F)
    assert np.array_equal(Vo.cpu().numpy().view(np.uint32), ref.V.view(np.uint32))
    assert st["committed"] == sum(r["committed"] for r in ref.rounds)
    assert st["undone"] == sum(r["undone"] for r in ref.rounds)
    if case == "shells_undos":
        assert st["undone"] > 0 and st["undo_iters_hist"][0] < st["rounds"]
