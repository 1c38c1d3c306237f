"""The seeded input generators that both the oracle and the CUDA path read:
the sizes of the stated recipes, closed oriented manifolds with the right
Euler characteristic, outward orientation, and bit-for-bit determinism."""
import numpy as np
import pytest

import meshgen
from tests.meshcheck import components, euler, is_closed_manifold


def _signed_volume(V, F):
    V = np.asarray(V, np.float64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_sizes_and_topology(level):
    V, F = meshgen.icosphere(level)
    assert len(F) == 20 * 4 ** level and len(V) == 10 * 4 ** level + 2
    assert is_closed_manifold(F, len(V)) and euler(F, len(V)) == 2
    assert np.allclose(np.linalg.norm(V, axis=1), 1.0, atol=1e-6)
    assert _signed_volume(V, F) > 0  # counter-clockwise = outward


def test_torus_recipe():
    V, F = meshgen.torus()
    assert len(V) == 2048 and len(F) == 4096
    assert is_closed_manifold(F, len(V)) and euler(F, len(V)) == 0
    assert components(F, len(V)) == 1
    assert _signed_volume(V, F) > 0
    V2, F2, target = meshgen.mesh_config("torus_64x32")
    assert target == 410 and np.array_equal(V, V2) and np.array_equal(F, F2)


def test_bumped_icosphere_recipe_and_determinism():
    V, F = meshgen.bumped_icosphere(5, 9)
    V2, F2 = meshgen.bumped_icosphere(5, 9)
    assert V.dtype == np.float32 and F.dtype == np.int32
    assert np.array_equal(V.view(np.uint32), V2.view(np.uint32)) and np.array_equal(F, F2)
    r = np.linalg.norm(V.astype(np.float64), axis=1)
    # radius 1 plus 32 outward bumps of amplitude at most 0.05 each
    assert r.min() >= 1.0 - 1e-6 and r.max() <= 1.0 + 32 * 0.05
    assert not np.array_equal(V, meshgen.bumped_icosphere(5, 10)[0])  # the seed matters
    assert is_closed_manifold(F, len(V)) and euler(F, len(V)) == 2


def test_nested_shells_are_two_spheres_inside_one_another():
    V, F = meshgen.nested_shells_seeded(3, 2001)
    assert len(F) == 2 * 20 * 4 ** 3
    assert is_closed_manifold(F, len(V)) and euler(F, len(V)) == 4
    assert components(F, len(V)) == 2
    # the inner shell is reversed: the enclosed volume is the thick solid's
    n = len(V) // 2
    r = np.linalg.norm(V.astype(np.float64), axis=1)
    assert (r[n:] < r[:n]).all()
    assert _signed_volume(V, F) > 0


def test_batch_recipe_first_meshes():
    meshes = meshgen.batch_meshes(count=12)
    assert len(meshes) == 12
    for i, (V, F) in enumerate(meshes):
        assert is_closed_manifold(F, len(V)), i
        assert euler(F, len(V)) in (0, 2)
        assert 2000 / 4 <= len(F) <= 500000 * 4  # log-uniform target, rounded to a level
    again = meshgen.batch_meshes(count=12)
    for (V, F), (V2, F2) in zip(meshes, again):
        assert np.array_equal(V, V2) and np.array_equal(F, F2)


def test_special_meshes():
    for make, chi, nf in ((meshgen.tetrahedron, 2, 4), (meshgen.octahedron, 2, 8)):
        V, F = make()
        assert len(F) == nf and is_closed_manifold(F, len(V)) and euler(F, len(V)) == chi
    V, F = meshgen.box_grid(3)
    assert is_closed_manifold(F, len(V)) and euler(F, len(V)) == 2
    # exactly planar sides: every coordinate on a face of the box is 0 or the size
    on_side = (np.isclose(V, 0.0) | np.isclose(V, 1.0)).any(axis=1)
    assert on_side.all()
