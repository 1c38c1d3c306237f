"""Seeded synthetic input meshes for the simplification path.

These generators build closed, manifold, intersection-free triangle meshes that
stand in for the paper's Thingi10K workload (Section 7.1 evaluates on Thingi10K
meshes of about 0.7M faces on average, with 2M- and 7M-face examples in the
teaser).  They hold none of the simplification method's arithmetic: no quadric,
cost, predicate or collapse is computed here.  Both the CUDA path and the CPU
oracle read the bytes produced here, so both sides see identical inputs.

Every mesh is returned as ``(V, F)``: ``V`` float32 ``[nV, 3]`` row-major,
``F`` int32 ``[nF, 3]`` with counter-clockwise corners seen from outside.
Geometry is computed in float64 and rounded once to float32.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "torus", "icosphere", "bumped_icosphere", "nested_shells", "tetrahedron",
    "octahedron", "box_grid", "batch_meshes", "mesh_config", "CONFIGS",
]


def torus(nu: int = 64, nv: int = 32, R: float = 1.0, r: float = 0.3,
          noise: float = 0.002, seed: int = 0):
    """UV torus with ``nu`` x ``nv`` quads, each split along (i,j)-(i+1,j+1).

    Vertex (i, j) sits at major angle 2*pi*i/nu and minor angle 2*pi*j/nv and
    is moved along the analytic normal by N(0, (noise*r)^2) (seeded PCG64).
    """
    rng = np.random.default_rng(seed)
    i = np.arange(nu, dtype=np.float64)[:, None]
    j = np.arange(nv, dtype=np.float64)[None, :]
    th = 2.0 * np.pi * i / nu
    ph = 2.0 * np.pi * j / nv
    nrm = np.stack(np.broadcast_arrays(np.cos(ph) * np.cos(th),
                                       np.cos(ph) * np.sin(th),
                                       np.sin(ph) + 0.0 * th), axis=-1)
    ring = (R + r * np.cos(ph)) + 0.0 * th
    p = np.stack([ring * np.cos(th), ring * np.sin(th),
                  (r * np.sin(ph)) + 0.0 * th], axis=-1)
    d = rng.normal(0.0, noise * r, size=(nu, nv))
    p = p + nrm * d[..., None]
    V = p.reshape(-1, 3).astype(np.float32)
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    v00 = ii * nv + jj
    v10 = ((ii + 1) % nu) * nv + jj
    v11 = ((ii + 1) % nu) * nv + (jj + 1) % nv
    v01 = ii * nv + (jj + 1) % nv
    t0 = np.stack([v00, v10, v11], axis=-1)
    t1 = np.stack([v00, v11, v01], axis=-1)
    F = np.stack([t0, t1], axis=2).reshape(-1, 3).astype(np.int32)
    return V, F


def _icosahedron():
    g = (1.0 + np.sqrt(5.0)) / 2.0
    V = np.array([[-1, g, 0], [1, g, 0], [-1, -g, 0], [1, -g, 0],
                  [0, -1, g], [0, 1, g], [0, -1, -g], [0, 1, -g],
                  [g, 0, -1], [g, 0, 1], [-g, 0, -1], [-g, 0, 1]],
                 dtype=np.float64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]],
                 dtype=np.int64)
    return V, F


def icosphere(level: int):
    """Unit icosphere after ``level`` rounds of 1-to-4 midpoint subdivision.

    Children of face (a, b, c) are emitted in the order (a, ab, ca),
    (ab, b, bc), (ca, bc, c), (ab, bc, ca).  New midpoint vertices are numbered
    after the old ones, in ascending order of their (min, max) edge key, and
    projected onto the unit sphere.  Returns float64 positions.
    """
    V, F = _icosahedron()
    for _ in range(level):
        nv = V.shape[0]
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        pairs = np.stack([np.stack([a, b], 1), np.stack([b, c], 1),
                          np.stack([c, a], 1)], 1)          # [F, 3, 2]
        lo = pairs.min(axis=2)
        hi = pairs.max(axis=2)
        key = lo * nv + hi
        uniq, inv = np.unique(key.ravel(), return_inverse=True)
        inv = inv.reshape(-1, 3) + nv
        ulo, uhi = uniq // nv, uniq % nv
        mid = V[ulo] + V[uhi]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        V = np.concatenate([V, mid], axis=0)
        ab, bc, ca = inv[:, 0], inv[:, 1], inv[:, 2]
        F = np.stack([np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1),
                      np.stack([ca, bc, c], 1), np.stack([ab, bc, ca], 1)],
                     axis=1).reshape(-1, 3)
    return V, F


def _bumps(rng, k: int, amp_lo: float, amp_hi: float | None):
    c = rng.normal(size=(k, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    if amp_hi is None:
        a = np.full(k, amp_lo)
    else:
        a = rng.uniform(amp_lo, amp_hi, size=k)
    w = rng.uniform(0.1, 0.3, size=k)
    return c, a, w


def _radius(P, base: float, c, a, w):
    dots = np.clip(P @ c.T, -1.0, 1.0)
    th = np.arccos(dots)
    return base + (a[None, :] * np.exp(-th * th / (2.0 * w[None, :] ** 2))).sum(1)


def bumped_icosphere(level: int = 8, seed: int = 0, nbumps: int = 32,
                     amp=(0.01, 0.05), base: float = 1.0):
    """Icosphere radially displaced by a sum of Gaussian bumps (in angle).

    r(p) = base + sum_k a_k exp(-theta_k(p)^2 / (2 w_k^2)), theta_k the angle
    between p and the bump centre c_k; c_k uniform on the sphere, a_k ~ U(amp),
    w_k ~ U(0.1, 0.3) rad.  A radial graph over the sphere is closed, manifold
    and free of self-intersections.
    """
    P, F = icosphere(level)
    rng = np.random.default_rng(seed)
    lo, hi = (amp, None) if np.isscalar(amp) else amp
    c, a, w = _bumps(rng, nbumps, lo, hi)
    r = _radius(P, base, c, a, w)
    return (P * r[:, None]).astype(np.float32), F.astype(np.int32)


def nested_shells(level: int = 8, seeds=(0, 1), radii=(1.0, 0.99),
                  amp: float = 0.004, nbumps: int = 32, check: bool = True):
    """Two bumped icospheres with the same connectivity, the inner one reversed.

    The pair bounds a thick solid.  Both shells are radial graphs over the same
    spherical triangulation, so r_in < r_out at every vertex implies the shells
    are disjoint; the generator asserts that inequality and reports the
    minimum radial gap (``nested_shells.last_min_gap``).
    """
    P, F = icosphere(level)
    rs = []
    for s, base in zip(seeds, radii):
        rng = np.random.default_rng(s)
        c, a, w = _bumps(rng, nbumps, amp, None)
        rs.append(_radius(P, base, c, a, w))
    gap = rs[0] - rs[1]
    nested_shells.last_min_gap = float(gap.min())
    if check and not (gap > 0).all():
        raise ValueError(f"nested shells overlap: min radial gap {gap.min():.3e}")
    Vo = (P * rs[0][:, None]).astype(np.float32)
    Vi = (P * rs[1][:, None]).astype(np.float32)
    nv = P.shape[0]
    Fo = F
    Fi = F[:, [0, 2, 1]] + nv
    V = np.concatenate([Vo, Vi], 0)
    return V, np.concatenate([Fo, Fi], 0).astype(np.int32)


nested_shells.last_min_gap = float("nan")


def nested_shells_seeded(level: int, seed: int, **kw):
    """Nested shells (nested_shells) for one seed of a seeded family: the outer
    shell uses ``seed``; the inner one the first of seed + 4000 + 10007 k,
    k = 0, 1, ..., for which the shells are disjoint."""
    for k in range(64):
        try:
            return nested_shells(level, seeds=(seed, seed + 4000 + 10007 * k), check=True, **kw)
        except ValueError:
            continue
    raise ValueError(f"no disjoint inner shell for seed {seed}")


def tetrahedron():
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], np.float32)
    F = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], np.int32)
    return V, F


def octahedron():
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0],
                  [0, 0, 1], [0, 0, -1]], np.float32)
    F = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                  [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]], np.int32)
    return V, F


def box_grid(n: int = 4, size=(1.0, 1.0, 1.0)):
    """Closed axis-aligned box whose six sides are planar n x n quad grids.

    Each side is exactly planar (one coordinate is constant), which makes
    planar-patch collapses available.  Grid coordinates are dyadic when
    ``n`` is a power of two and the sizes are dyadic.
    """
    sx, sy, sz = size
    verts = {}
    V = []

    def vid(p):
        if p not in verts:
            verts[p] = len(V)
            V.append(p)
        return verts[p]

    F = []
    # integer lattice coordinates on the box surface, scaled at the end
    sides = [  # (fixed axis, fixed value, u axis, v axis, flip)
        (0, 0, 1, 2, True), (0, n, 1, 2, False),
        (1, 0, 0, 2, False), (1, n, 0, 2, True),
        (2, 0, 0, 1, True), (2, n, 0, 1, False),
    ]
    for ax, val, ua, va, flip in sides:
        for i in range(n):
            for j in range(n):
                q = []
                for (di, dj) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                    p = [0, 0, 0]
                    p[ax] = val
                    p[ua] = i + di
                    p[va] = j + dj
                    q.append(vid(tuple(p)))
                t0, t1 = (q[0], q[1], q[2]), (q[0], q[2], q[3])
                if flip:
                    t0, t1 = (t0[0], t0[2], t0[1]), (t1[0], t1[2], t1[1])
                F.extend([t0, t1])
    V = np.array(V, np.float64) / n * np.array(size)
    return V.astype(np.float32), np.array(F, np.int32)


def batch_meshes(count: int = 256, seed0: int = 4000, fmin: int = 2000,
                 fmax: int = 500000):
    """Seeded batch of tori and bumped icospheres with log-uniform face counts."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        is_torus = rng.random() < 0.5
        f = float(np.exp(rng.uniform(np.log(fmin), np.log(fmax))))
        if is_torus:
            rr = rng.uniform(0.2, 0.5)
            nv = max(3, int(round(np.sqrt(f / 4.0))))
            out.append(torus(2 * nv, nv, 1.0, rr, 0.002, seed0 + i))
        else:
            lvl = int(np.clip(np.round(np.log(f / 20.0) / np.log(4.0)), 3, 7))
            out.append(bumped_icosphere(lvl, seed0 + i))
    return out


CONFIGS = {
    "torus_64x32": dict(target=410),
    "bumped_icosphere_l8": dict(target=13107),
    "nested_shells_l8": dict(target=2621),
}


def mesh_config(name: str):
    """(V, F, target_faces) for a named workload."""
    if name == "torus_64x32":
        V, F = torus()
    elif name == "bumped_icosphere_l8":
        V, F = bumped_icosphere(8, 0)
    elif name == "nested_shells_l8":
        V, F = nested_shells(8)
    else:
        raise KeyError(name)
    return V, F, CONFIGS[name]["target"]
