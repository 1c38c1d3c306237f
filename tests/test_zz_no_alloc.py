"""The allocation-free self-intersection check.

pamo_check_self_intersections_noalloc serves callers that cannot allocate
device memory while they run (for example code whose device memory is owned
and budgeted elsewhere): it uses a fixed scratch array inside the library.
Here it must report exactly what pamo_check_self_intersections reports, on two
calls in a row (the shared scratch keeps the previous call's contents, so the
second call checks that nothing leaks between calls), take no device memory
while it runs, and refuse bad face indices and wrongly typed arguments.  This
file is collected last so that a -x run has executed every other test first.
"""
import numpy as np
import pytest

import meshgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2509_05595_gb300 as pamo  # noqa: E402


def _overlapping_spheres():
    V1, F1 = meshgen.bumped_icosphere(4, 1)
    V2, F2 = meshgen.bumped_icosphere(4, 2)
    V = np.concatenate([V1, V2 + np.float32(0.7)]).astype(np.float32)
    F = np.concatenate([F1, F2 + len(V1)]).astype(np.int32)
    return V, F


def _check_both(V, F, out):
    Vd = torch.from_numpy(V).cuda()
    Fd = torch.from_numpy(F).cuda()
    n_ref, pairs_ref = pamo.pamo_check_self_intersections(Vd, Fd)
    n = pamo.pamo_check_self_intersections_noalloc(Vd, Fd, out)
    torch.cuda.synchronize()
    assert n == n_ref
    got = {tuple(p) for p in out[: min(n, out.shape[0])].cpu().numpy().tolist()}
    assert got == {tuple(p) for p in pairs_ref.cpu().numpy().tolist()}
    return n


def test_noalloc_check_matches_allocating_check_twice_in_a_row():
    out = torch.full((1 << 16, 2), -1, dtype=torch.int32, device="cuda")
    V, F = _overlapping_spheres()                 # 10,240 faces, many crossings
    n1 = _check_both(V, F, out)
    assert n1 > 100
    V2, F2 = meshgen.nested_shells(4, check=False)  # 10,240 faces, none
    n2 = _check_both(V2, F2, out)
    assert n2 == 0
    n3 = _check_both(V, F, out)                   # and back: same answer
    assert n3 == n1


def test_noalloc_check_rejects_oversized_mesh():
    V, F = meshgen.bumped_icosphere(6, 0)         # 81,920 faces > 32,768
    out = torch.empty((16, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(pamo.PamoError, match="EINVAL"):
        pamo.pamo_check_self_intersections_noalloc(torch.from_numpy(V).cuda(),
                                                  torch.from_numpy(F).cuda(), out)


def test_noalloc_check_takes_no_device_memory():
    """Free device memory is the same before and after repeated calls once the
    library's cached pool memory has been handed back: nothing was allocated,
    not even memory that the call would free again into the pool."""
    out = torch.full((1 << 12, 2), -1, dtype=torch.int32, device="cuda")
    V, F = _overlapping_spheres()
    Vd, Fd = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    n0 = pamo.pamo_check_self_intersections_noalloc(Vd, Fd, out)  # set-up on this device
    torch.cuda.synchronize()
    pamo.pamo_release_cached_memory()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert pamo.pamo_check_self_intersections_noalloc(Vd, Fd, out) == n0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_checks_reject_face_indices_out_of_range():
    """A face index outside [0, nV) is refused with PAMO_EINVAL before the mesh
    is read, by both checks; the next call works."""
    V, F = meshgen.nested_shells(3, check=False)
    out = torch.empty((64, 2), dtype=torch.int32, device="cuda")
    Vd = torch.from_numpy(V).cuda()
    for bad_index in (len(V), -1, 1 << 30):
        Fb = F.copy()
        Fb[17, 2] = bad_index
        Fd = torch.from_numpy(Fb).cuda()
        with pytest.raises(pamo.PamoError, match="EINVAL"):
            pamo.pamo_check_self_intersections_noalloc(Vd, Fd, out)
        with pytest.raises(pamo.PamoError, match="EINVAL"):
            pamo.pamo_check_self_intersections(Vd, Fd)
    Fd = torch.from_numpy(F).cuda()
    assert pamo.pamo_check_self_intersections_noalloc(Vd, Fd, out) == 0


def test_noalloc_check_rejects_wrong_tensors():
    V, F = meshgen.nested_shells(3, check=False)
    Vd, Fd = torch.from_numpy(V).cuda(), torch.from_numpy(F).cuda()
    out = torch.empty((64, 2), dtype=torch.int32, device="cuda")
    bad = [(Vd.double(), Fd, out), (Vd, Fd.long(), out), (Vd, Fd, out.reshape(-1)),
           (Vd, Fd, out.t()), (Vd[:, :2], Fd, out), (Vd.t().contiguous().t(), Fd, out)]
    for args in bad:
        with pytest.raises(ValueError):
            pamo.pamo_check_self_intersections_noalloc(*args)
