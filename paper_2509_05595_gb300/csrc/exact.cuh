// Exact orientation predicates and the mesh triangle-pair test on the GPU.
//
// Filtering follows Shewchuk (1997): the determinant is evaluated in floating
// point with the usual difference form and accepted when it exceeds an error
// bound proportional to its permanent.  A float32 stage handles almost every
// call; a float64 stage catches most of the rest; the exact stage expands the
// determinant of [p 1] rows into monomials of the float32 inputs.  A product
// of two float32 values is exact in float64 (48 significant bits), and a third
// factor is split exactly with an FMA, so every monomial becomes a two-term
// expansion; the sign of their sum is taken from an exact grow-expansion
// (Shewchuk's Two-Sum accumulation).  No step rounds, so the sign is exact.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pamo {
namespace exact {

// ---- error-free transformations (double) ----------------------------------
__device__ __forceinline__ void two_sum(double a, double b, double& x, double& y) {
  x = __dadd_rn(a, b);
  double bv = __dsub_rn(x, a);
  double av = __dsub_rn(x, bv);
  double br = __dsub_rn(b, bv);
  double ar = __dsub_rn(a, av);
  y = __dadd_rn(ar, br);
}

__device__ __forceinline__ void two_prod(double a, double b, double& x, double& y) {
  x = __dmul_rn(a, b);
  y = __fma_rn(a, b, -x);
}

// h := h + b for a nonoverlapping expansion h (increasing magnitude), zero
// components dropped.  Returns the new length.
__device__ __forceinline__ int grow(double* h, int n, double b) {
  double q = b;
  int m = 0;
  for (int i = 0; i < n; i++) {
    double s, e;
    two_sum(q, h[i], s, e);
    q = s;
    if (e != 0.0) h[m++] = e;
  }
  if (q != 0.0 || m == 0) h[m++] = q;
  return m;
}

__device__ __forceinline__ int sign_of(const double* h, int n) {
  double t = h[n - 1];
  return (t > 0.0) - (t < 0.0);
}

// ---- orient3d: sign of det[a-d; b-d; c-d] ---------------------------------
// Exact stage: det[a 1; b 1; c 1; d 1] = det[abc] - det[abd] + det[acd] - det[bcd]
// and det[pqr] = sum over permutations of signed px*qy*rz.
__device__ __noinline__ int orient3d_exact(const float3 a, const float3 b, const float3 c,
                                          const float3 d) {
  double h[50];
  int n = 0;
  const float3* P[4] = {&a, &b, &c, &d};
  // (i, j, k, sign of the 3x3 minor in the 4x4 expansion)
  const int tri[4][4] = {{0, 1, 2, 1}, {0, 1, 3, -1}, {0, 2, 3, 1}, {1, 2, 3, -1}};
  for (int t = 0; t < 4; t++) {
    const float3& p = *P[tri[t][0]];
    const float3& q = *P[tri[t][1]];
    const float3& r = *P[tri[t][2]];
    const double s = (double)tri[t][3];
    // det[p;q;r] = px(qy rz - qz ry) - py(qx rz - qz rx) + pz(qx ry - qy rx)
    const double m[6][3] = {
        {p.x, q.y, r.z}, {-(double)p.x, q.z, r.y}, {-(double)p.y, q.x, r.z},
        {p.y, q.z, r.x}, {p.z, q.x, r.y},          {-(double)p.z, q.y, r.x}};
    for (int i = 0; i < 6; i++) {
      double uv = __dmul_rn(s * m[i][0], m[i][1]);  // exact: 24 x 24 bits
      double hi, lo;
      two_prod(uv, m[i][2], hi, lo);
      n = grow(h, n, lo);
      n = grow(h, n, hi);
    }
  }
  return sign_of(h, n);
}

// Out of line, like orient2d: the pair test calls both from many places, and
// inlined copies made the pair kernel's code large enough that instruction
// fetch stalled it
__device__ __noinline__ int orient3d(const float3 a, const float3 b, const float3 c,
                                     const float3 d) {
  // float32 stage, valid when no product can underflow: every non-zero
  // difference lies in [2^-40, 2^40]
  {
    const float adx = __fsub_rn(a.x, d.x), ady = __fsub_rn(a.y, d.y), adz = __fsub_rn(a.z, d.z);
    const float bdx = __fsub_rn(b.x, d.x), bdy = __fsub_rn(b.y, d.y), bdz = __fsub_rn(b.z, d.z);
    const float cdx = __fsub_rn(c.x, d.x), cdy = __fsub_rn(c.y, d.y), cdz = __fsub_rn(c.z, d.z);
    const float dv[9] = {adx, ady, adz, bdx, bdy, bdz, cdx, cdy, cdz};
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 9; i++) {
      float m = fabsf(dv[i]);
      ok &= (m == 0.0f) || (m >= 9.094947e-13f && m <= 1.0995116e12f);
    }
    if (ok) {
      const float bdxcdy = __fmul_rn(bdx, cdy), cdxbdy = __fmul_rn(cdx, bdy);
      const float cdxady = __fmul_rn(cdx, ady), adxcdy = __fmul_rn(adx, cdy);
      const float adxbdy = __fmul_rn(adx, bdy), bdxady = __fmul_rn(bdx, ady);
      const float det = __fadd_rn(__fadd_rn(__fmul_rn(adz, __fsub_rn(bdxcdy, cdxbdy)),
                                            __fmul_rn(bdz, __fsub_rn(cdxady, adxcdy))),
                                  __fmul_rn(cdz, __fsub_rn(adxbdy, bdxady)));
      const float perm =
          __fadd_rn(__fadd_rn(__fmul_rn(__fadd_rn(fabsf(bdxcdy), fabsf(cdxbdy)), fabsf(adz)),
                              __fmul_rn(__fadd_rn(fabsf(cdxady), fabsf(adxcdy)), fabsf(bdz))),
                    __fmul_rn(__fadd_rn(fabsf(adxbdy), fabsf(bdxady)), fabsf(cdz)));
      const float eb = __fmul_rn(4.7683716e-07f /* 8 * 2^-24 */, perm);
      if (det > eb) return 1;
      if (-det > eb) return -1;
    }
  }
  // float64 stage: float32 inputs cannot under- or overflow here
  {
    const double adx = (double)a.x - d.x, ady = (double)a.y - d.y, adz = (double)a.z - d.z;
    const double bdx = (double)b.x - d.x, bdy = (double)b.y - d.y, bdz = (double)b.z - d.z;
    const double cdx = (double)c.x - d.x, cdy = (double)c.y - d.y, cdz = (double)c.z - d.z;
    const double bdxcdy = __dmul_rn(bdx, cdy), cdxbdy = __dmul_rn(cdx, bdy);
    const double cdxady = __dmul_rn(cdx, ady), adxcdy = __dmul_rn(adx, cdy);
    const double adxbdy = __dmul_rn(adx, bdy), bdxady = __dmul_rn(bdx, ady);
    const double det = __dadd_rn(__dadd_rn(__dmul_rn(adz, __dsub_rn(bdxcdy, cdxbdy)),
                                           __dmul_rn(bdz, __dsub_rn(cdxady, adxcdy))),
                                 __dmul_rn(cdz, __dsub_rn(adxbdy, bdxady)));
    const double perm =
        __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(fabs(bdxcdy), fabs(cdxbdy)), fabs(adz)),
                            __dmul_rn(__dadd_rn(fabs(cdxady), fabs(adxcdy)), fabs(bdz))),
                  __dmul_rn(__dadd_rn(fabs(adxbdy), fabs(bdxady)), fabs(cdz)));
    const double eb = __dmul_rn(8.881784197001252e-16 /* 8 * 2^-53 */, perm);
    if (det > eb) return 1;
    if (-det > eb) return -1;
  }
  return orient3d_exact(a, b, c, d);
}

// ---- orient2d on two coordinates: sign of (b-a) x (c-a) -------------------
__device__ __noinline__ int orient2d_exact(float au, float av, float bu, float bv, float cu,
                                          float cv) {
  // det[a 1; b 1; c 1] = au bv - au cv - av bu + av cu + bu cv - bv cu; each
  // product of two float32 values is exact in float64
  double h[8];
  int n = 0;
  n = grow(h, n, __dmul_rn(au, bv));
  n = grow(h, n, -__dmul_rn(au, cv));
  n = grow(h, n, -__dmul_rn(av, bu));
  n = grow(h, n, __dmul_rn(av, cu));
  n = grow(h, n, __dmul_rn(bu, cv));
  n = grow(h, n, -__dmul_rn(bv, cu));
  return sign_of(h, n);
}

__device__ __noinline__ int orient2d(float au, float av, float bu, float bv, float cu,
                                     float cv) {
  {
    const float x1 = __fsub_rn(bu, au), y1 = __fsub_rn(bv, av);
    const float x2 = __fsub_rn(cu, au), y2 = __fsub_rn(cv, av);
    const float m[4] = {x1, y1, x2, y2};
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      float t = fabsf(m[i]);
      ok &= (t == 0.0f) || (t >= 9.094947e-13f && t <= 1.0995116e12f);
    }
    if (ok) {
      const float l = __fmul_rn(x1, y2), r = __fmul_rn(y1, x2);
      const float det = __fsub_rn(l, r);
      const float eb = __fmul_rn(2.3841858e-07f /* 4 * 2^-24 */, __fadd_rn(fabsf(l), fabsf(r)));
      if (det > eb) return 1;
      if (-det > eb) return -1;
    }
  }
  {
    const double x1 = (double)bu - au, y1 = (double)bv - av;
    const double x2 = (double)cu - au, y2 = (double)cv - av;
    const double l = __dmul_rn(x1, y2), r = __dmul_rn(y1, x2);
    const double det = __dsub_rn(l, r);
    const double eb = __dmul_rn(4.440892098500626e-16 /* 4 * 2^-53 */, __dadd_rn(fabs(l), fabs(r)));
    if (det > eb) return 1;
    if (-det > eb) return -1;
  }
  return orient2d_exact(au, av, bu, bv, cu, cv);
}

// ---- the triangle-pair predicate ------------------------------------------
__device__ __forceinline__ float comp(const float3& p, int k) {
  return k == 0 ? p.x : (k == 1 ? p.y : p.z);
}

// orientation of (a, b, c) after dropping axis k (the other two in cyclic order)
__device__ __forceinline__ int o2(const float3& a, const float3& b, const float3& c, int k) {
  const int u = k == 2 ? 0 : k + 1, w = k == 0 ? 2 : (k == 1 ? 0 : 1);
  return orient2d(comp(a, u), comp(a, w), comp(b, u), comp(b, w), comp(c, u), comp(c, w));
}

// Face descriptor computed once per face: a projection axis that keeps the
// triangle's area and its orientation there (0 = zero-area triangle).
struct FaceInfo {
  int axis;
  int o;
};

__device__ __forceinline__ FaceInfo face_info(const float3& a, const float3& b, const float3& c) {
  FaceInfo r{0, 0};
  // prefer the axis of largest normal component (any axis with non-zero
  // orientation gives the same answers; this one is usually decided in float32)
  const float ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
  const float vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
  const float nx = fabsf(uy * vz - uz * vy), ny = fabsf(uz * vx - ux * vz),
              nz = fabsf(ux * vy - uy * vx);
  int order[3];
  if (nz >= nx && nz >= ny) {
    order[0] = 2; order[1] = nx >= ny ? 0 : 1; order[2] = nx >= ny ? 1 : 0;
  } else if (nx >= ny) {
    order[0] = 0; order[1] = ny >= nz ? 1 : 2; order[2] = ny >= nz ? 2 : 1;
  } else {
    order[0] = 1; order[1] = nx >= nz ? 0 : 2; order[2] = nx >= nz ? 2 : 0;
  }
  for (int i = 0; i < 3; i++) {
    int s = o2(a, b, c, order[i]);
    if (s != 0) {
      r.axis = order[i];
      r.o = s;
      return r;
    }
  }
  return r;
}

__device__ __forceinline__ bool same_pt(const float3& a, const float3& b) {
  return a.x == b.x && a.y == b.y && a.z == b.z;
}

// closed coplanar segments pq and uw, projected along axis k
__device__ __forceinline__ bool segseg2(const float3& p, const float3& q, const float3& u,
                                        const float3& w, int k) {
  const int s1 = o2(p, q, u, k), s2 = o2(p, q, w, k);
  if (s1 * s2 > 0) return false;
  const int s3 = o2(u, w, p, k), s4 = o2(u, w, q, k);
  if (s3 * s4 > 0) return false;
  if (s1 == 0 && s2 == 0) {  // collinear: compare extents along a varying axis
    const int ax0 = k == 2 ? 0 : k + 1, ax1 = k == 0 ? 2 : (k == 1 ? 0 : 1);
    const int ax = comp(p, ax0) != comp(q, ax0) ? ax0 : ax1;
    const float lo = fmaxf(fminf(comp(p, ax), comp(q, ax)), fminf(comp(u, ax), comp(w, ax)));
    const float hi = fminf(fmaxf(comp(p, ax), comp(q, ax)), fmaxf(comp(u, ax), comp(w, ax)));
    return lo <= hi;
  }
  return true;
}

// closed segment pq (p != q) against closed triangle xyz with info fi (o != 0)
__device__ __forceinline__ bool segtri(const float3& p, const float3& q, const float3& x,
                                       const float3& y, const float3& z, FaceInfo fi) {
  const int sp = orient3d(x, y, z, p);
  const int sq = orient3d(x, y, z, q);
  if (sp * sq > 0) return false;
  if (sp == 0 && sq == 0) {
    const int k = fi.axis, o = fi.o;
    if (o2(x, y, p, k) * o >= 0 && o2(y, z, p, k) * o >= 0 && o2(z, x, p, k) * o >= 0) return true;
    if (o2(x, y, q, k) * o >= 0 && o2(y, z, q, k) * o >= 0 && o2(z, x, q, k) * o >= 0) return true;
    return segseg2(p, q, x, y, k) || segseg2(p, q, y, z, k) || segseg2(p, q, z, x, k);
  }
  const int s1 = orient3d(p, q, x, y);
  const int s2 = orient3d(p, q, y, z);
  if (s1 * s2 < 0) return false;
  const int s3 = orient3d(p, q, z, x);
  return !((s1 > 0 || s2 > 0 || s3 > 0) && (s1 < 0 || s2 < 0 || s3 < 0));
}

// does the segment from A towards P start inside the closed angle DAE of the
// non-degenerate triangle (A, D, E) with info fi?
__device__ __forceinline__ bool ray_in_angle(const float3& A, const float3& P, const float3& D,
                                             const float3& E, FaceInfo fi) {
  if (same_pt(A, P)) return false;
  if (orient3d(A, D, E, P) != 0) return false;
  // (A, D, E) is a cyclic rotation of the face's corner order, so its
  // projected orientation is fi.o
  return o2(A, D, P, fi.axis) * fi.o >= 0 && o2(A, P, E, fi.axis) * fi.o >= 0;
}

// Self-intersection test of two faces of a mesh: t/c corner positions, ti/ci
// vertex indices, ft/fc their FaceInfo.  Cases by the number s of shared
// vertex indices (Algorithm 3, supplementary Section 3): s = 3 intersects;
// a zero-area face intersects; s = 2: coplanar and the far corners not on
// strictly opposite sides of the shared edge; s = 1: the faces meet somewhere
// other than the shared vertex; s = 0: the closed faces meet.
__device__ __forceinline__ bool faces_intersect(const float3* t, const int* ti, FaceInfo ft,
                                                const float3* c, const int* ci, FaceInfo fc) {
  int s = 0, it = -1, ic = -1, st0 = -1, sc0 = -1;
  for (int i = 0; i < 3; i++) {
    bool shared = false;
    for (int j = 0; j < 3; j++)
      if (ti[i] == ci[j]) {
        shared = true;
        if (st0 < 0) { st0 = i; sc0 = j; }
      }
    if (shared) s++;
    else it = i;
  }
  if (s >= 3) return true;
  if (ft.o == 0 || fc.o == 0) return true;
  if (s == 2) {
    for (int j = 0; j < 3; j++) {
      bool shared = false;
      for (int i = 0; i < 3; i++) shared |= (ci[j] == ti[i]);
      if (!shared) ic = j;
    }
    const float3& A = t[(it + 1) % 3];
    const float3& B = t[(it + 2) % 3];
    if (orient3d(A, B, t[it], c[ic]) != 0) return false;
    // coplanar: side of the far corners w.r.t. line AB in T's projection
    const int k = ft.axis;
    return o2(A, B, t[it], k) * o2(A, B, c[ic], k) >= 0;
  }
  if (s == 1) {
    const float3& A = t[st0];
    const float3& B = t[(st0 + 1) % 3];
    const float3& C = t[(st0 + 2) % 3];
    const float3& D = c[(sc0 + 1) % 3];
    const float3& E = c[(sc0 + 2) % 3];
    // Early outs: if D and E lie strictly on one side of T's plane, the other
    // face meets that plane only at A, so the faces share nothing but A (and
    // symmetrically for B, C against the other face's plane).
    const int sD = orient3d(A, B, C, D), sE = orient3d(A, B, C, E);
    if (sD * sE > 0) return false;
    const int sB = orient3d(A, D, E, B), sC = orient3d(A, D, E, C);
    if (sB * sC > 0) return false;
    if (segtri(B, C, A, D, E, fc)) return true;
    if (segtri(D, E, A, B, C, ft)) return true;
    if (ray_in_angle(A, B, D, E, fc)) return true;
    if (ray_in_angle(A, C, D, E, fc)) return true;
    if (ray_in_angle(A, D, B, C, ft)) return true;
    if (ray_in_angle(A, E, B, C, ft)) return true;
    return false;
  }
  // s = 0.  Early outs: a face whose corners all lie strictly on one side of
  // the other face's plane cannot meet it.
  {
    const int a0 = orient3d(t[0], t[1], t[2], c[0]);
    const int a1 = orient3d(t[0], t[1], t[2], c[1]);
    const int a2 = orient3d(t[0], t[1], t[2], c[2]);
    if ((a0 > 0 && a1 > 0 && a2 > 0) || (a0 < 0 && a1 < 0 && a2 < 0)) return false;
    const int b0 = orient3d(c[0], c[1], c[2], t[0]);
    const int b1 = orient3d(c[0], c[1], c[2], t[1]);
    const int b2 = orient3d(c[0], c[1], c[2], t[2]);
    if ((b0 > 0 && b1 > 0 && b2 > 0) || (b0 < 0 && b1 < 0 && b2 < 0)) return false;
  }
  for (int i = 0; i < 3; i++)
    if (segtri(t[i], t[(i + 1) % 3], c[0], c[1], c[2], fc)) return true;
  for (int i = 0; i < 3; i++)
    if (segtri(c[i], c[(i + 1) % 3], t[0], t[1], t[2], ft)) return true;
  return false;
}

}  // namespace exact
}  // namespace pamo
