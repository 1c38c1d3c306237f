"""Host-side parts of the Python binding (no GPU): the batch layout helper
and the marshalling of options into the C struct."""
import ctypes

import numpy as np

import meshgen
import paper_2509_05595_gb300 as pamo


def test_concat_meshes_layout():
    a = meshgen.tetrahedron()
    b = meshgen.octahedron()
    V, voff, F, foff = pamo.concat_meshes([a, b, a])
    assert V.dtype == np.float32 and F.dtype == np.int32
    assert voff.tolist() == [0, 4, 10, 14] and foff.tolist() == [0, 4, 12, 16]
    # each mesh's faces index its own vertices from 0, unchanged
    assert np.array_equal(F[foff[1]:foff[2]], np.asarray(b[1], np.int32))
    assert np.array_equal(V[voff[2]:voff[3]], np.asarray(a[0], np.float32))
    assert F[foff[2]:foff[3]].max() < 4


def test_options_marshal_every_field():
    o = pamo.Options(w_e=0.25, w_s=0.5, tolerance=7, max_rounds=99, stall_limit=5,
                     validate_input=0, check_mode=1, record_rounds=1, profile=3,
                     exact_target=1, max_cost=2.5, grid_blocks_per_sm=8, resort_percent=30,
                     proposal_threshold=0.75, check_input_intersections=1,
                     recompute_quadrics=1, device_loop=1)
    c = o.c()
    for name in ("w_e", "w_s", "tolerance", "max_rounds", "stall_limit", "validate_input",
                 "check_mode", "record_rounds", "profile", "exact_target", "max_cost",
                 "grid_blocks_per_sm", "resort_percent", "check_input_intersections",
                 "recompute_quadrics", "device_loop"):
        assert getattr(c, name) == getattr(o, name), name
    assert abs(c.proposal_threshold - 0.75) < 1e-7
    assert not c.proposal  # no network: a null pointer


def test_default_options_match_the_library():
    lib = pamo.lib()
    d = pamo._Options()
    lib.pamo_default_options(ctypes.byref(d))
    o = pamo.Options().c()
    for name, _ in pamo._Options._fields_:
        if name == "proposal":
            continue
        assert getattr(o, name) == getattr(d, name), name


def test_noalloc_check_rejects_host_arguments_before_any_call():
    """The allocation-free check converts nothing: anything but CUDA tensors
    is refused in Python, before the library is called."""
    import pytest
    torch = pytest.importorskip("torch")
    V, F = meshgen.octahedron()
    out = np.zeros((4, 2), np.int32)
    with pytest.raises(ValueError, match="torch CUDA tensor"):
        pamo.pamo_check_self_intersections_noalloc(V, F, out)
    with pytest.raises(ValueError, match="CUDA tensor"):
        pamo.pamo_check_self_intersections_noalloc(torch.from_numpy(V), torch.from_numpy(F),
                                                  torch.from_numpy(out))
