// The skinny term of Eq. 1, 1 - C_ijk with C_ijk = 4 sqrt(3) A / (l_ij^2 +
// l_jk^2 + l_ki^2), evaluated in float-float arithmetic (an unevaluated sum of
// two float32 values) with an a-priori bound on its distance from the float64
// evaluation.
//
// Why: the edge key holds float(C_ab) only, and this GPU's float64 pipe takes a
// warp instruction every 64 cycles while its float32 pipe takes one every
// cycle.  About three quarters of the float64 work of an edge cost is in its
// produced triangles.  So the triangles are evaluated here on the float32 pipe,
// and the caller certifies the key: if every cost the bound allows rounds to
// the same float, that float is the key of the float64 evaluation too;
// otherwise the caller evaluates the edge in float64.
//
// Building blocks (all exact, barring overflow, on round-to-nearest float32):
//   two_sum       Knuth's TwoSum: s + e = a + b
//   fast_two_sum  Dekker's Fast2Sum (|a| >= |b|): s + e = a + b
//   TwoProduct    with a fused multiply-add: p + e = a * b (up to 2^-150)
//
// Error analysis.  u = 2^-24; every float32 operation is fl(x) = x (1 + d),
// |d| <= u, up to an absolute 2^-150 in the subnormal range.  P0 is the
// placement, P1, P2 the other corners; a = P1 - P0, b = P2 - P0, c = P2 - P1,
// D = |a|^2 + |b|^2 + |c|^2, n = a x b, C = 2 sqrt(3) |n| / D.  C is symmetric
// in the corners, so the corner order of the face does not matter here.
//   a, b, c      two_sum per component: exact pairs (h, l), |l| <= u |h|
//   x*y          p = x_h y_h, e = (x_h y_h - p) + x_h y_l + x_l y_h by fused
//                multiply-adds; x_l y_l is dropped: |p + e - xy| <= 6.01 u^2 |x||y|
//   n_x          x1 y1 - x2 y2 from two such products, two_sum of the high
//                parts, the low parts added, two_sum: |err| <= 13.05 u^2 M_x,
//                M_x = |a_y b_z| + |a_z b_y| <= |a||b|, so |n~ - n| <= 22.61 u^2 |a||b|
//   x^2          p = x_h^2, e = (x_h^2 - p) + 2 x_h x_l: |err| <= 4.02 u^2 x^2
//   x + y        for x, y >= 0 (normalised pairs): two_sum of the high parts,
//                the low parts added, fast_two_sum: |err| <= 3.02 u^2 (x + y)
//   |v|^2        (x^2 + y^2) + z^2: relative error <= 10.06 u^2
//   D            (|a|^2 + |b|^2) + |c|^2: relative error <= 16.1 u^2
//   scaling      tau = 2^k with tau D_h in [1, 2), applied to n and D (exact;
//                C does not change, and |tau n| <= tau D / 2 < 1 cannot overflow)
//   N = |tau n~|^2           relative error <= 10.06 u^2
//   s = sqrt(N)  r = RN(sqrt(N_h)), the correction (N_h - r^2 + N_l) / (2r)
//                (N_h - r^2 is exact by a fused multiply-add):
//                |s~ - sqrt(N)| <= 5.8 u^2 sqrt(N); below N_h = 2^-100 the
//                correction is skipped and C~ moves by under 1 u^2
//   so |s~ - tau |n|| <= 33.51 u^2 tau |a||b|
//   K = 2 sqrt(3) as a pair: relative error <= 1.04 u^2;  M = K s~: 7.05 u^2
//   q = M / D    q1 = M_h RN(1/D_h), the residual M - q1 D by TwoProduct
//                (M_h - p_h is exact by Sterbenz), q2 = residual RN(1/D_h):
//                |q1 + q2 - M/D| <= 22 u^2 M/D
//   Since D >= |a|^2 + |b|^2 >= 2 |a||b|:
//     |2 sqrt(3) s~ / (tau D) - C| <= sqrt(3) 33.51 u^2 = 58.04 u^2,
//     |M/D - C| <= 58.04 u^2 + (7.05 + 16.1) u^2 C,  C <= 1 (Weitzenboeck),
//     |C~ - C| <= 103.2 u^2
//   t = 1 - q    two_sum(1, -q1), q2 subtracted from the low part, two_sum:
//                |t~ - (1 - C~)| <= 5.2 u^2
//   subnormal results in the low parts: under 4 u^2 in all, given D_h >= 2^-60
// The float64 evaluation (same corners, its own order, unit 2^-53 = u^2/32):
// |C_f64 - C| <= 24.7 * 2^-53, and 1 - C_f64 rounds by at most 2^-53, so
// |t_f64 - (1 - C)| <= 0.81 u^2.  In all |t~ - t_f64| <= 114 u^2; the bound
// used is kTriBound = 2^-40 = 256 u^2.
//
// The certified range: D_h in [2^-60, 2^60] (this also rules out NaN, infinite
// and overflowing inputs, which reach D).  Outside it the function returns NaN
// and the caller evaluates the triangle in float64.
#pragma once
#include <cuda_runtime.h>

namespace pamo {
namespace ff {

constexpr float kTriBound = 0x1p-40f;  // |t~ - t_f64| per triangle (see above)

struct FF {
  float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// x * y for normalised pairs; the result is not normalised (|e| <= 3.01 u |p|)
__device__ __forceinline__ FF mul(FF x, FF y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return {p, e};
}

// x^2 for a normalised pair, normalised
__device__ __forceinline__ FF sqr(FF x) {
  const float p = __fmul_rn(x.h, x.h);
  const float e = __fmaf_rn(__fadd_rn(x.h, x.h), x.l, __fmaf_rn(x.h, x.h, -p));
  return fast_two_sum(p, e);
}

// x + y for non-negative normalised pairs, normalised
__device__ __forceinline__ FF add_nonneg(FF x, FF y) {
  const FF s = two_sum(x.h, y.h);
  const float w = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
  return fast_two_sum(s.h, w);
}

// x + y for normalised pairs of any sign, normalised:
// |err| <= 3.02 u^2 (|x| + |y|)
__device__ __forceinline__ FF add(FF x, FF y) {
  const FF s = two_sum(x.h, y.h);
  const float w = __fadd_rn(s.l, __fadd_rn(x.l, y.l));
  return two_sum(s.h, w);
}

// x1 y1 - x2 y2 for normalised pairs, normalised
__device__ __forceinline__ FF cross_term(FF x1, FF y1, FF x2, FF y2) {
  const FF p = mul(x1, y1), q = mul(x2, y2);
  const FF s = two_sum(p.h, -q.h);
  const float z = __fadd_rn(__fsub_rn(p.l, q.l), s.l);
  return two_sum(s.h, z);
}

__device__ __forceinline__ FF norm2(FF x, FF y, FF z) {
  return add_nonneg(add_nonneg(sqr(x), sqr(y)), sqr(z));
}

__device__ __forceinline__ FF scale(FF x, float t) {
  return {__fmul_rn(x.h, t), __fmul_rn(x.l, t)};
}

// 1 - C of the triangle (P0, P1, P2) as a normalised pair (t.x + t.y), within
// kTriBound of the float64 evaluation; NaN outside the certified range.
__device__ __forceinline__ float2 skinny_term_ff(float p0x, float p0y, float p0z, float p1x,
                                                 float p1y, float p1z, float p2x, float p2y,
                                                 float p2z) {
  constexpr double kK = 2.0 * 1.7320508075688772;  // 2 sqrt(3), nearest double
  constexpr float kKh = (float)kK;
  constexpr float kKl = (float)(kK - (double)kKh);
  const FF ax = two_sum(p1x, -p0x), ay = two_sum(p1y, -p0y), az = two_sum(p1z, -p0z);
  const FF bx = two_sum(p2x, -p0x), by = two_sum(p2y, -p0y), bz = two_sum(p2z, -p0z);
  const FF cx = two_sum(p2x, -p1x), cy = two_sum(p2y, -p1y), cz = two_sum(p2z, -p1z);
  const FF D = add_nonneg(add_nonneg(norm2(ax, ay, az), norm2(bx, by, bz)), norm2(cx, cy, cz));
  if (!(D.h >= 0x1p-60f && D.h <= 0x1p60f)) return make_float2(__int_as_float(0x7fc00000), 0.f);
  // tau = 2^k with tau D_h in [1, 2): exponent field 254 - e(D_h)
  const float tau = __int_as_float((254 - ((__float_as_int(D.h) >> 23) & 0xff)) << 23);
  const FF nx = scale(cross_term(ay, bz, az, by), tau);
  const FF ny = scale(cross_term(az, bx, ax, bz), tau);
  const FF nz = scale(cross_term(ax, by, ay, bx), tau);
  const FF Ds = scale(D, tau);
  const FF N = norm2(nx, ny, nz);
  // s = sqrt(N)
  const float r = __fsqrt_rn(N.h);
  float corr = 0.f;
  if (N.h >= 0x1p-100f) {
    const float v = __fadd_rn(__fmaf_rn(-r, r, N.h), N.l);
    corr = __fmul_rn(v, __fmul_rn(0.5f, __frcp_rn(r)));
  }
  const FF s = fast_two_sum(r, corr);
  const FF Mu = mul({kKh, kKl}, s);
  const FF M = fast_two_sum(Mu.h, Mu.l);
  // q = M / Ds
  const float rD = __frcp_rn(Ds.h);
  const float q1 = __fmul_rn(M.h, rD);
  const float ph = __fmul_rn(q1, Ds.h);
  const float pl = __fmaf_rn(q1, Ds.h, -ph);
  float res = __fsub_rn(M.h, ph);
  res = __fsub_rn(res, pl);
  res = __fadd_rn(res, M.l);
  res = __fmaf_rn(-q1, Ds.l, res);
  const float q2 = __fmul_rn(res, rD);
  // t = 1 - q
  const FF t0 = two_sum(1.0f, -q1);
  const FF t = two_sum(t0.h, __fsub_rn(t0.l, q2));
  return make_float2(t.h, t.l);
}

}  // namespace ff
}  // namespace pamo
