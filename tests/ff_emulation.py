"""Exact float32 emulation of the certified float-float skinny term (Eq. 1's
1 - C_ijk as the edge-cost kernel evaluates it), for tests.

NumPy's float32 addition, subtraction, multiplication, division and square
root round to nearest-even like the kernel's __fadd_rn / __fmul_rn /
__frcp_rn / __fsqrt_rn.  The fused multiply-add has no NumPy counterpart, so
fma32 computes it exactly: the product of two float32 values is exact in
float64, TwoSum gives the exact float64 pair (s, e) of product + addend, and
rounding s to float32 is the rounding of s + e except when s lies exactly on a
midpoint between two float32 values, where the sign of e decides.

The steps follow the algorithm the kernel implements (TwoSum, Fast2Sum, the
FMA form of TwoProduct, the pair products and sums, the scaling by a power of
two, the corrected square root and quotient); nothing here is shared with the
kernel's source.
"""
import numpy as np

F32 = np.float32
F64 = np.float64


def fma32(a, b, c):
    """round_to_nearest_even_float32(a * b + c), exactly, elementwise."""
    a, b, c = (np.asarray(x, F32) for x in (a, b, c))
    p = a.astype(F64) * b.astype(F64)          # exact (24 + 24 bits)
    c64 = c.astype(F64)
    s = p + c64
    bb = s - p
    e = (p - (s - bb)) + (c64 - bb)             # s + e == p + c exactly
    with np.errstate(over="ignore", invalid="ignore"):
        f = s.astype(F32)                       # round_to_nearest_even(s)
        r = s - f.astype(F64)                   # exact: s is within half a float32 ulp of f
        toward = np.where(r > 0, F32(np.inf), F32(-np.inf)).astype(F32)
        n = np.nextafter(f, toward)             # the other float32 neighbour of s
        mid = (f.astype(F64) + n.astype(F64)) * 0.5
        # Away from a float32 midpoint, s + e rounds like s (|e| is at most half
        # a float64 ulp of s, and a midpoint is itself a float64).  On a
        # midpoint the sign of e decides; e == 0 keeps the even choice f.
        tie = (r != 0) & (s == mid)
        hi = np.maximum(f, n)
        lo = np.minimum(f, n)
        f = np.where(tie & (e > 0), hi, np.where(tie & (e < 0), lo, f))
    return f.astype(F32)


def two_sum(a, b):
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    e = ((a - (s - bb).astype(F32)).astype(F32) + (b - bb).astype(F32)).astype(F32)
    return s, e


def fast_two_sum(a, b):
    s = (a + b).astype(F32)
    return s, (b - (s - a).astype(F32)).astype(F32)


def mul(x, y):
    p = (x[0] * y[0]).astype(F32)
    e = fma32(x[0], y[0], -p)
    e = fma32(x[0], y[1], e)
    e = fma32(x[1], y[0], e)
    return p, e


def sqr(x):
    p = (x[0] * x[0]).astype(F32)
    e = fma32((x[0] + x[0]).astype(F32), x[1], fma32(x[0], x[0], -p))
    return fast_two_sum(p, e)


def add_nonneg(x, y):
    s = two_sum(x[0], y[0])
    w = (s[1] + (x[1] + y[1]).astype(F32)).astype(F32)
    return fast_two_sum(s[0], w)


def add(x, y):
    s = two_sum(x[0], y[0])
    w = (s[1] + (x[1] + y[1]).astype(F32)).astype(F32)
    return two_sum(s[0], w)


def cross_term(x1, y1, x2, y2):
    p, q = mul(x1, y1), mul(x2, y2)
    s = two_sum(p[0], -q[0])
    z = ((p[1] - q[1]).astype(F32) + s[1]).astype(F32)
    return two_sum(s[0], z)


def norm2(x, y, z):
    return add_nonneg(add_nonneg(sqr(x), sqr(y)), sqr(z))


def scale(x, t):
    return (x[0] * t).astype(F32), (x[1] * t).astype(F32)


K_D = 2.0 * 1.7320508075688772          # 2 sqrt(3), the nearest double
K_H = F32(K_D)
K_L = F32(K_D - float(K_H))


def skinny_term_ff(T):
    """1 - C_ijk of triangles T ([n, 9] float32: the placement, then the two
    other corners) as the kernel's float-float pairs ([n, 2] float32); NaN in
    the high part outside the certified range D_h in [2^-60, 2^60]."""
    T = np.asarray(T, F32)
    p0, p1, p2 = T[:, 0:3], T[:, 3:6], T[:, 6:9]
    with np.errstate(all="ignore"):
        a = [two_sum(p1[:, k], -p0[:, k]) for k in range(3)]
        b = [two_sum(p2[:, k], -p0[:, k]) for k in range(3)]
        c = [two_sum(p2[:, k], -p1[:, k]) for k in range(3)]
        D = add_nonneg(add_nonneg(norm2(*a), norm2(*b)), norm2(*c))
        ok = (D[0] >= F32(2.0 ** -60)) & (D[0] <= F32(2.0 ** 60))
        # tau = 2^k with tau D_h in [1, 2): exponent field 254 - e(D_h)
        e = (np.where(ok, D[0], F32(1)).view(np.int32) >> 23) & 0xFF
        tau = ((254 - e) << 23).astype(np.int32).view(F32)
        nx = scale(cross_term(a[1], b[2], a[2], b[1]), tau)
        ny = scale(cross_term(a[2], b[0], a[0], b[2]), tau)
        nz = scale(cross_term(a[0], b[1], a[1], b[0]), tau)
        Ds = scale(D, tau)
        N = norm2(nx, ny, nz)
        r = np.sqrt(N[0]).astype(F32)
        v = (fma32(-r, r, N[0]) + N[1]).astype(F32)
        corr = (v * (F32(0.5) * (F32(1) / r).astype(F32)).astype(F32)).astype(F32)
        corr = np.where(N[0] >= F32(2.0 ** -100), corr, F32(0)).astype(F32)
        s = fast_two_sum(r, corr)
        Mu = mul((np.full_like(r, K_H), np.full_like(r, K_L)), s)
        M = fast_two_sum(Mu[0], Mu[1])
        rD = (F32(1) / Ds[0]).astype(F32)
        q1 = (M[0] * rD).astype(F32)
        ph = (q1 * Ds[0]).astype(F32)
        pl = fma32(q1, Ds[0], -ph)
        res = (M[0] - ph).astype(F32)
        res = (res - pl).astype(F32)
        res = (res + M[1]).astype(F32)
        res = fma32(-q1, Ds[1], res)
        q2 = (res * rD).astype(F32)
        t0 = two_sum(np.full_like(q1, F32(1)), -q1)
        t = two_sum(t0[0], (t0[1] - q2).astype(F32))
    hi = np.where(ok, t[0], F32(np.nan)).astype(F32)
    lo = np.where(ok, t[1], F32(0)).astype(F32)
    return np.stack([hi, lo], axis=1)
