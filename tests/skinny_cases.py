"""Seeded triangle families for the skinny-term tests (Eq. 1's 1 - C_ijk), and
its exact value.  Each row of a family is [placement, corner, corner] as
float32, the layout of pamo_skinny_terms."""
import decimal
from fractions import Fraction

import numpy as np


def mesh_like(rng, n, h=5e-3):
    P0 = rng.uniform(-1, 1, (n, 3))
    return np.concatenate([P0, P0 + rng.normal(0, h, (n, 3)), P0 + rng.normal(0, h, (n, 3))], 1)


def equilateral(rng, n, side=1e-2, jitter=1e-6):
    c = rng.uniform(-1, 1, (n, 3))
    e1 = rng.normal(size=(n, 3))
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(e1, rng.normal(size=(n, 3)))
    e2 /= np.linalg.norm(e2, axis=1, keepdims=True)
    pts = [c + side * (np.cos(a) * e1 + np.sin(a) * e2) / np.sqrt(3)
           for a in (0.0, 2 * np.pi / 3, 4 * np.pi / 3)]
    T = np.concatenate(pts, 1)
    return T + rng.normal(0, jitter * side, T.shape)


def slivers(rng, n):
    P0 = rng.uniform(-1, 1, (n, 3))
    d = rng.normal(0, 5e-3, (n, 3))
    perp = np.cross(d, rng.normal(size=(n, 3)))
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    ratio = 10.0 ** rng.uniform(-12, -1, (n, 1))
    lam = rng.uniform(-0.5, 1.5, (n, 1))
    L = np.linalg.norm(d, axis=1, keepdims=True)
    return np.concatenate([P0, P0 + d, P0 + lam * d + ratio * L * perp], 1)


def near_zero(rng, n):
    # coordinates of both signs near 0: float differences that are not exact
    return rng.uniform(-1e-3, 1e-3, (n, 9)) * (10.0 ** rng.uniform(-3, 0, (n, 1)))


def families(seed=7, n=20000):
    """Mesh-like, near-equilateral, sliver (height/length 1e-12 .. 0.1), near-zero
    and scaled (2^-16 .. 2^28) triangles, all inside the certified range."""
    rng = np.random.default_rng(seed)
    fams = {"mesh": mesh_like(rng, n), "equilateral": equilateral(rng, n),
            "sliver": slivers(rng, n), "near_zero": near_zero(rng, n)}
    for k in (-16, -10, 10, 28):
        fams[f"scaled_2^{k}"] = mesh_like(rng, n // 4) * 2.0 ** k
    return {k: v.astype(np.float32) for k, v in fams.items()}


def out_of_range(seed=3, n=64):
    """Triangles outside the certified range: D below 2^-60 or above 2^60,
    coincident corners, an infinite or a NaN coordinate."""
    rng = np.random.default_rng(seed)
    base = mesh_like(rng, n)  # D about 2^-12
    cases = {
        "tiny": base * 2.0 ** -28,        # D about 2^-68
        "huge": base * 2.0 ** 40,         # D about 2^68
        "coincident": np.tile(rng.uniform(-1, 1, (n, 3)), (1, 3)),
        "non_finite": np.where(np.arange(9) == 4, np.inf, base),
        "nan": np.where(np.arange(9) == 0, np.nan, base),
    }
    return {k: v.astype(np.float32) for k, v in cases.items()}


def _dec(f):
    return decimal.Decimal(f.numerator) / decimal.Decimal(f.denominator)


def exact_t(tri):
    """1 - C of one triangle from exact rationals; the square roots in the
    caller's decimal context (use 120 digits)."""
    P = [Fraction(float(x)) for x in tri]
    a = [P[3 + i] - P[i] for i in range(3)]
    b = [P[6 + i] - P[i] for i in range(3)]
    c = [P[6 + i] - P[3 + i] for i in range(3)]
    n = [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]
    n2 = sum(x * x for x in n)
    D = sum(x * x for x in a) + sum(x * x for x in b) + sum(x * x for x in c)
    C = 2 * decimal.Decimal(3).sqrt() * _dec(n2).sqrt() / _dec(D)
    return decimal.Decimal(1) - C
