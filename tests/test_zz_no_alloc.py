"""The allocation-free self-intersection check.

pamo_check_self_intersections_noalloc serves callers that cannot allocate
device memory while they run (for example code whose device memory is owned
and budgeted elsewhere): it uses a fixed scratch array inside the library.
Here it must report exactly what pamo_check_self_intersections reports, on two
calls in a row (the shared scratch keeps the previous call's contents, so the
second call checks that nothing leaks between calls).  This file is collected
last so that a -x run has executed every other test first.
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
