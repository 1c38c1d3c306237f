// Oracle for parallel intersection-free edge-collapse simplification.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
// CPU-baseline leg may load this library.  The product path never calls it.
// It shares no code, header, table or helper with the CUDA library.
//
// Plain, slow, single-threaded restatement of the simplification stage of
// PaMO (arXiv 2509.05595):
//   * Algorithm 1 (ParallelSimplification): rounds of cost -> propagation ->
//     collapse of independent regions -> repeat{intersection check; undo}.
//   * Eq. 1 (edge cost): C_ab = Q_ab + w_e * l_ab + w_s * sum(1 - C_ijk),
//     C_ijk = 4 sqrt(3) A / (l_ij^2 + l_jk^2 + l_ki^2), w_e = 0.001, w_s = 0.005.
//     Q_ab is the Garland-Heckbert quadric error (the paper cites QEM only).
//   * Section 5.1: the 64-bit key (float cost bits << 32 | edge id), the
//     triangle cost as the minimum over edges whose 1-ring holds the triangle,
//     an edge wins iff every triangle of its 1-ring holds its key, and the link
//     condition (Dey et al.) on collapses.
//   * Section 5.2 / Algorithm 3 / supplementary Section 3: intersection check
//     with the case analysis by the number of shared vertices.
//   * Section 5.3: undo and the invalid-edge flags with tolerance 4.
// Readings where the paper is silent:
//   R1 quadrics: unweighted face planes, vertex sums in ascending face order;
//      a collapse adds the two endpoint quadrics.
//   R2 placement: Cramer solve of A v = -b, singular if |det| <= 1e-12 m^3;
//      fallback = best of (a, b, midpoint) by Q, ties in that order; the
//      result is rounded to float and Q / skinny terms use the rounded point.
//   R3 skinny term: the triangles the collapse produces, ascending face index.
//   R4 scale: costs are those of the [0,1]^3-normalised mesh (Section 4 start),
//      i.e. C = s^2 Q + w_e s l + w_s sum(1-C_ijk), s = 1 / (max bbox extent).
//   R5 ids: edges are the sorted unique (min,max) vertex pairs; ties -> lower id.
//   R6 eligibility: flagged, link-failing or non-finite-cost edges hold no key.
//   R7 collapse: survivor min(a,b), faces keep slot and corner order.
//   R8 compaction after the undo loop, stable.
//   R9 intersection: exact predicates; a zero-area triangle intersects anything
//      it is tested against; s=1 means "the triangles meet beyond the shared
//      vertex"; s=2 means "coplanar and the far corners not strictly on
//      opposite sides of the shared edge"; s=3 intersects.
//   R10 flags: undone edges are invalid next round; after a round with no
//      committed collapse the flags accumulate, cleared after `tolerance`
//      such rounds.
//   R11 check scope: faces changed this round against all faces (the same
//      pairs as all faces against all faces, the previous mesh being
//      intersection-free).
//   R12 an intersecting pair undoes the collapses that tagged either face.
//   R13 evaluation order of Eq. 1: products accumulate with explicit std::fma
//      in a fixed order (one rounding each); the skinny term is the formula
//      as printed: A = |u x w| / 2 with u, w the edges from the first corner,
//      and the three squared edge lengths summed.  or_set_plain_products(1)
//      replaces every fused multiply-add by a multiply and an add (two
//      roundings), to measure how much the fixed fma order moves the keys.
//   R14 target edge cost (Section 5.1 names it beside the face target): an
//      edge whose float cost is above (float)max_cost is not eligible; the
//      run ends normally when no edge is eligible and no flag is pending.
//   R15 exact target: when a round's winners would remove more faces than
//      |F| - N_t, only the ceil((|F| - N_t) / 2) winners with the lowest keys
//      collapse (off by default: Algorithm 1 collapses every winner).
//   R16 quadric memory (option): by default a collapse adds the two endpoint
//      quadrics (R1); with recompute_quadrics every round starts from the
//      face-plane quadrics of the current mesh instead.
//
// Floating point: compiled with -ffp-contract=off (no implicit contraction),
// IEEE double throughout the cost with explicit std::fma where the order says
// so, float only for stored positions.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Exact integer arithmetic for predicates.
// Every finite float x is an integer multiple of 2^-149, so X = x * 2^149 is an
// integer of at most 278 bits.  Degree-3 polynomials in such integers fit in
// 1024 bits.  Sign-magnitude, 32 limbs of 32 bits, little-endian.
// ---------------------------------------------------------------------------
struct Big {
  int neg = 0;
  int n = 0;            // used limbs (no leading zero limbs)
  uint32_t d[34] = {0};
};

static void big_trim(Big& a) {
  while (a.n > 0 && a.d[a.n - 1] == 0) a.n--;
  if (a.n == 0) a.neg = 0;
}

static Big big_from_float(float f) {
  Big r;
  uint32_t bits;
  std::memcpy(&bits, &f, 4);
  uint32_t ex = (bits >> 23) & 0xff;
  uint32_t fr = bits & 0x7fffff;
  uint64_t m;
  int shift;  // value * 2^149 = m * 2^shift
  if (ex == 0) {
    m = fr;
    shift = 0;
  } else {
    m = fr | 0x800000u;
    shift = (int)ex - 1;  // x = m * 2^(ex-150); * 2^149 -> m * 2^(ex-1)
  }
  int limb = shift / 32, off = shift % 32;
  unsigned __int128 v = (unsigned __int128)m << off;
  r.d[limb] = (uint32_t)v;
  r.d[limb + 1] = (uint32_t)(v >> 32);
  r.d[limb + 2] = (uint32_t)(v >> 64);
  r.n = limb + 3;
  r.neg = (bits >> 31) ? 1 : 0;
  big_trim(r);
  return r;
}

static int big_cmp_mag(const Big& a, const Big& b) {
  if (a.n != b.n) return a.n < b.n ? -1 : 1;
  for (int i = a.n - 1; i >= 0; i--)
    if (a.d[i] != b.d[i]) return a.d[i] < b.d[i] ? -1 : 1;
  return 0;
}

static Big big_add_mag(const Big& a, const Big& b) {
  Big r;
  int n = std::max(a.n, b.n);
  uint64_t c = 0;
  for (int i = 0; i < n; i++) {
    uint64_t s = c + (i < a.n ? a.d[i] : 0) + (i < b.n ? b.d[i] : 0);
    r.d[i] = (uint32_t)s;
    c = s >> 32;
  }
  r.n = n;
  if (c) r.d[r.n++] = (uint32_t)c;
  return r;
}

static Big big_sub_mag(const Big& a, const Big& b) {  // |a| >= |b|
  Big r;
  int64_t br = 0;
  for (int i = 0; i < a.n; i++) {
    int64_t s = (int64_t)a.d[i] - (i < b.n ? b.d[i] : 0) - br;
    br = s < 0;
    if (s < 0) s += ((int64_t)1 << 32);
    r.d[i] = (uint32_t)s;
  }
  r.n = a.n;
  big_trim(r);
  return r;
}

static Big big_add(const Big& a, const Big& b) {
  Big r;
  if (a.neg == b.neg) {
    r = big_add_mag(a, b);
    r.neg = a.neg;
  } else if (big_cmp_mag(a, b) >= 0) {
    r = big_sub_mag(a, b);
    r.neg = a.neg;
  } else {
    r = big_sub_mag(b, a);
    r.neg = b.neg;
  }
  big_trim(r);
  return r;
}

static Big big_neg(Big a) {
  if (a.n) a.neg ^= 1;
  return a;
}

static Big big_sub(const Big& a, const Big& b) { return big_add(a, big_neg(b)); }

static Big big_mul(const Big& a, const Big& b) {
  Big r;
  if (a.n == 0 || b.n == 0) return r;
  uint64_t acc[68] = {0};
  for (int i = 0; i < a.n; i++) {
    uint64_t carry = 0;
    for (int j = 0; j < b.n; j++) {
      uint64_t t = (uint64_t)a.d[i] * b.d[j] + acc[i + j] + carry;
      acc[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
    int k = i + b.n;
    while (carry) {
      uint64_t t = acc[k] + carry;
      acc[k] = (uint32_t)t;
      carry = t >> 32;
      k++;
    }
  }
  int n = a.n + b.n;
  if (n > 34) {  // cannot happen for degree <= 3 in float inputs
    std::fprintf(stderr, "oracle: bigint overflow\n");
    std::abort();
  }
  for (int i = 0; i < n; i++) r.d[i] = (uint32_t)acc[i];
  r.n = n;
  r.neg = a.neg ^ b.neg;
  big_trim(r);
  return r;
}

static int big_sign(const Big& a) { return a.n == 0 ? 0 : (a.neg ? -1 : 1); }

// orient3d(a,b,c,d) = det [a-d; b-d; c-d] (rows), exact.
static int orient3d_exact(const float* a, const float* b, const float* c,
                          const float* d) {
  Big A[3], B[3], C[3];
  for (int k = 0; k < 3; k++) {
    Big dk = big_from_float(d[k]);
    A[k] = big_sub(big_from_float(a[k]), dk);
    B[k] = big_sub(big_from_float(b[k]), dk);
    C[k] = big_sub(big_from_float(c[k]), dk);
  }
  Big m0 = big_sub(big_mul(B[1], C[2]), big_mul(B[2], C[1]));
  Big m1 = big_sub(big_mul(B[0], C[2]), big_mul(B[2], C[0]));
  Big m2 = big_sub(big_mul(B[0], C[1]), big_mul(B[1], C[0]));
  Big det = big_add(big_sub(big_mul(A[0], m0), big_mul(A[1], m1)),
                    big_mul(A[2], m2));
  return big_sign(det);
}

// orient2d on coordinates (u,v) of three points: (b-a) x (c-a), exact.
static int orient2d_exact(float au, float av, float bu, float bv, float cu,
                          float cv) {
  Big a0 = big_from_float(au), a1 = big_from_float(av);
  Big x1 = big_sub(big_from_float(bu), a0), y1 = big_sub(big_from_float(bv), a1);
  Big x2 = big_sub(big_from_float(cu), a0), y2 = big_sub(big_from_float(cv), a1);
  return big_sign(big_sub(big_mul(x1, y2), big_mul(y1, x2)));
}

// Semi-static filters (Shewchuk 1997, "Adaptive precision floating-point
// arithmetic and fast robust geometric predicates", error bounds A).  When the
// double-precision value is farther from zero than the bound, its sign is the
// exact sign; otherwise the exact integer evaluation decides.
static const double kEps = 1.1102230246251565e-16;  // 2^-53
static const double kO3dBound = (7.0 + 56.0 * kEps) * kEps;
static const double kCcwBound = (3.0 + 16.0 * kEps) * kEps;

static int orient3d(const float* a, const float* b, const float* c,
                    const float* d) {
  double adx = (double)a[0] - d[0], ady = (double)a[1] - d[1], adz = (double)a[2] - d[2];
  double bdx = (double)b[0] - d[0], bdy = (double)b[1] - d[1], bdz = (double)b[2] - d[2];
  double cdx = (double)c[0] - d[0], cdy = (double)c[1] - d[1], cdz = (double)c[2] - d[2];
  double bdxcdy = bdx * cdy, cdxbdy = cdx * bdy;
  double cdxady = cdx * ady, adxcdy = adx * cdy;
  double adxbdy = adx * bdy, bdxady = bdx * ady;
  double det = adz * (bdxcdy - cdxbdy) + bdz * (cdxady - adxcdy) +
               cdz * (adxbdy - bdxady);
  double perm = (std::fabs(bdxcdy) + std::fabs(cdxbdy)) * std::fabs(adz) +
                (std::fabs(cdxady) + std::fabs(adxcdy)) * std::fabs(bdz) +
                (std::fabs(adxbdy) + std::fabs(bdxady)) * std::fabs(cdz);
  double eb = kO3dBound * perm;
  // det above is the expansion of det[a-d; b-d; c-d] along its z column,
  // which equals orient3d_exact's row-wise determinant.
  if (det > eb) return 1;
  if (-det > eb) return -1;
  return orient3d_exact(a, b, c, d);
}

static int orient2d(float au, float av, float bu, float bv, float cu, float cv) {
  double l = ((double)bu - au) * ((double)cv - av);
  double r = ((double)bv - av) * ((double)cu - au);
  double det = l - r;
  double eb = kCcwBound * (std::fabs(l) + std::fabs(r));
  if (det > eb) return 1;
  if (-det > eb) return -1;
  return orient2d_exact(au, av, bu, bv, cu, cv);
}

// ---------------------------------------------------------------------------
// Triangle-triangle intersection (Section 5.2, Algorithm 3, supplementary
// Section 3), decided exactly.  See R9 above.
// ---------------------------------------------------------------------------
struct P3 {
  float v[3];
};

static int orient2d_axis(const P3& a, const P3& b, const P3& c, int k) {
  // drop axis k, keep the other two in cyclic order
  int u = (k + 1) % 3, w = (k + 2) % 3;
  return orient2d(a.v[u], a.v[w], b.v[u], b.v[w], c.v[u], c.v[w]);
}

static bool degenerate(const P3& a, const P3& b, const P3& c) {
  for (int k = 0; k < 3; k++)
    if (orient2d_axis(a, b, c, k) != 0) return false;
  return true;
}

// a projection axis in which triangle (a,b,c) keeps nonzero area
static int good_axis(const P3& a, const P3& b, const P3& c, int* o) {
  for (int k = 0; k < 3; k++) {
    int s = orient2d_axis(a, b, c, k);
    if (s != 0) {
      *o = s;
      return k;
    }
  }
  *o = 0;
  return -1;
}

static bool same_point(const P3& a, const P3& b) {
  return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2];
}

// closed 2-D segment pq vs closed segment uw (projection axis k)
static bool seg_seg_2d(const P3& p, const P3& q, const P3& u, const P3& w, int k) {
  int o1 = orient2d_axis(p, q, u, k), o2 = orient2d_axis(p, q, w, k);
  int o3 = orient2d_axis(u, w, p, k), o4 = orient2d_axis(u, w, q, k);
  if (o1 * o2 > 0 || o3 * o4 > 0) return false;
  if (o1 == 0 && o2 == 0) {
    int a0 = (k + 1) % 3, a1 = (k + 2) % 3;
    int ax = (p.v[a0] != q.v[a0]) ? a0 : a1;
    float lo = std::max(std::min(p.v[ax], q.v[ax]), std::min(u.v[ax], w.v[ax]));
    float hi = std::min(std::max(p.v[ax], q.v[ax]), std::max(u.v[ax], w.v[ax]));
    return lo <= hi;
  }
  return true;
}

// closed segment pq (p != q) vs closed non-degenerate triangle xyz
static bool seg_tri(const P3& p, const P3& q, const P3& x, const P3& y,
                    const P3& z) {
  int sp = orient3d(x.v, y.v, z.v, p.v);
  int sq = orient3d(x.v, y.v, z.v, q.v);
  if (sp * sq > 0) return false;
  if (sp == 0 && sq == 0) {
    int o;
    int k = good_axis(x, y, z, &o);
    const P3* pts[2] = {&p, &q};
    for (int i = 0; i < 2; i++) {
      const P3& r = *pts[i];
      int a = orient2d_axis(x, y, r, k), b = orient2d_axis(y, z, r, k),
          c = orient2d_axis(z, x, r, k);
      if (a * o >= 0 && b * o >= 0 && c * o >= 0) return true;
    }
    if (seg_seg_2d(p, q, x, y, k)) return true;
    if (seg_seg_2d(p, q, y, z, k)) return true;
    if (seg_seg_2d(p, q, z, x, k)) return true;
    return false;
  }
  int a = orient3d(p.v, q.v, x.v, y.v);
  int b = orient3d(p.v, q.v, y.v, z.v);
  int c = orient3d(p.v, q.v, z.v, x.v);
  bool pos = a > 0 || b > 0 || c > 0;
  bool neg = a < 0 || b < 0 || c < 0;
  return !(pos && neg);
}

// Does the segment from shared vertex A towards P leave A inside the closed
// angle DAE of non-degenerate triangle A D E?  (supplementary Section 3.1,
// "angle-overlap test", evaluated exactly)
static bool ray_in_sector(const P3& A, const P3& P, const P3& D, const P3& E) {
  if (same_point(A, P)) return false;
  if (orient3d(A.v, D.v, E.v, P.v) != 0) return false;
  int o;
  int k = good_axis(A, D, E, &o);
  int s1 = orient2d_axis(A, D, P, k);
  int s2 = orient2d_axis(A, P, E, k);
  return s1 * o >= 0 && s2 * o >= 0;
}

// T = (t[0],t[1],t[2]), C = (c[0],c[1],c[2]); ti/ci vertex indices.
static bool tri_intersect(const P3* t, const int32_t* ti, const P3* c,
                          const int32_t* ci) {
  int s = 0;
  int mt[3] = {-1, -1, -1};  // mt[i] = j if t[i] is c[j]
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      if (ti[i] == ci[j]) {
        mt[i] = j;
        s++;
      }
  if (s >= 3) return true;  // duplicate face (Algorithm 3 final branch)
  if (degenerate(t[0], t[1], t[2]) || degenerate(c[0], c[1], c[2])) return true;
  if (s == 2) {
    // shared edge AB, far corners Ct (of T) and Dc (of C)
    int it = -1, jc = -1;
    for (int i = 0; i < 3; i++)
      if (mt[i] < 0) it = i;
    bool used[3] = {false, false, false};
    for (int i = 0; i < 3; i++)
      if (mt[i] >= 0) used[mt[i]] = true;
    for (int j = 0; j < 3; j++)
      if (!used[j]) jc = j;
    const P3& A = t[(it + 1) % 3];
    const P3& B = t[(it + 2) % 3];
    const P3& Ct = t[it];
    const P3& Dc = c[jc];
    if (orient3d(A.v, B.v, Ct.v, Dc.v) != 0) return false;  // supp. Sec. 3.2
    int o;
    int k = good_axis(A, B, Ct, &o);
    int sd = orient2d_axis(A, B, Dc, k);
    return sd * o >= 0;  // same side or on the line: supp. Sec. 3.1 same-side
  }
  if (s == 1) {
    int ia = -1;
    for (int i = 0; i < 3; i++)
      if (mt[i] >= 0) ia = i;
    int ja = mt[ia];
    const P3& A = t[ia];
    const P3& B = t[(ia + 1) % 3];
    const P3& Cc = t[(ia + 2) % 3];
    const P3& D = c[(ja + 1) % 3];
    const P3& E = c[(ja + 2) % 3];
    if (ray_in_sector(A, B, D, E)) return true;
    if (ray_in_sector(A, Cc, D, E)) return true;
    if (ray_in_sector(A, D, B, Cc)) return true;
    if (ray_in_sector(A, E, B, Cc)) return true;
    if (seg_tri(B, Cc, A, D, E)) return true;
    if (seg_tri(D, E, A, B, Cc)) return true;
    return false;
  }
  for (int i = 0; i < 3; i++)
    if (seg_tri(t[i], t[(i + 1) % 3], c[0], c[1], c[2])) return true;
  for (int i = 0; i < 3; i++)
    if (seg_tri(c[i], c[(i + 1) % 3], t[0], t[1], t[2])) return true;
  return false;
}

// ---------------------------------------------------------------------------
// Edge cost (Eq. 1) with the QEM term (Garland-Heckbert).
// ---------------------------------------------------------------------------
static const double kSqrt3 = 1.7320508075688772;

struct Quadric {
  double k[10];  // xx xy xz xd yy yz yd zz zd dd
};

static Quadric face_quadric(const float* p0, const float* p1, const float* p2) {
  Quadric q;
  for (int i = 0; i < 10; i++) q.k[i] = 0.0;
  double ux = (double)p1[0] - (double)p0[0], uy = (double)p1[1] - (double)p0[1],
         uz = (double)p1[2] - (double)p0[2];
  double vx = (double)p2[0] - (double)p0[0], vy = (double)p2[1] - (double)p0[1],
         vz = (double)p2[2] - (double)p0[2];
  double nx = uy * vz - uz * vy;
  double ny = uz * vx - ux * vz;
  double nz = ux * vy - uy * vx;
  double len = std::sqrt((nx * nx + ny * ny) + nz * nz);
  if (len == 0.0) return q;
  nx = nx / len;
  ny = ny / len;
  nz = nz / len;
  double d = -((nx * (double)p0[0] + ny * (double)p0[1]) + nz * (double)p0[2]);
  q.k[0] = nx * nx;
  q.k[1] = nx * ny;
  q.k[2] = nx * nz;
  q.k[3] = nx * d;
  q.k[4] = ny * ny;
  q.k[5] = ny * nz;
  q.k[6] = ny * d;
  q.k[7] = nz * nz;
  q.k[8] = nz * d;
  q.k[9] = d * d;
  return q;
}

// Evaluation order (reading R13): products are accumulated with fused
// multiply-adds (std::fma: one rounding), written out explicitly so that the
// order is fixed.  With g_plain_products set, each fused multiply-add is a
// multiply followed by an add instead (the same expression, two roundings).
static bool g_plain_products = false;

static double mad(double a, double b, double c) {
  if (g_plain_products) return a * b + c;
  return std::fma(a, b, c);
}

// Cramer's rule expanded along the first row.
static double det3(double a00, double a01, double a02, double a10, double a11,
                   double a12, double a20, double a21, double a22) {
  double m0 = mad(a11, a22, -(a12 * a21));
  double m1 = mad(a10, a22, -(a12 * a20));
  double m2 = mad(a10, a21, -(a11 * a20));
  return mad(a02, m2, mad(-a01, m1, a00 * m0));
}

// Q(v) = v^T A v + 2 b^T v + c for the summed quadric K
static double quadric_eval(const double* K, double x, double y, double z) {
  double ax = mad(K[2], z, mad(K[1], y, K[0] * x));
  double ay = mad(K[5], z, mad(K[4], y, K[1] * x));
  double az = mad(K[7], z, mad(K[5], y, K[2] * x));
  double bv = mad(K[8], z, mad(K[6], y, K[3] * x));
  return mad(2.0, bv, mad(z, az, mad(y, ay, x * ax))) + K[9];
}

static double dot3(double ax, double ay, double az, double bx, double by, double bz) {
  return mad(az, bz, mad(ay, by, ax * bx));
}

// C_ijk = 4 sqrt(3) A / (l_ij^2 + l_jk^2 + l_ki^2) of Eq. 1 for the triangle
// (q0, q1, q2): A is half the length of the cross product of the edges
// q1 - q0 and q2 - q0, the denominator the three squared edge lengths summed
// in the order (q0q1, q1q2, q2q0).
static double tri_quality(const double* q0, const double* q1, const double* q2) {
  double ux = q1[0] - q0[0], uy = q1[1] - q0[1], uz = q1[2] - q0[2];
  double tx = q2[0] - q1[0], ty = q2[1] - q1[1], tz = q2[2] - q1[2];
  double wx = q2[0] - q0[0], wy = q2[1] - q0[1], wz = q2[2] - q0[2];
  double nx = mad(uy, wz, -(uz * wy));
  double ny = mad(uz, wx, -(ux * wz));
  double nz = mad(ux, wy, -(uy * wx));
  double area = 0.5 * std::sqrt(dot3(nx, ny, nz, nx, ny, nz));
  double den = (dot3(ux, uy, uz, ux, uy, uz) + dot3(tx, ty, tz, tx, ty, tz)) +
               dot3(wx, wy, wz, wx, wy, wz);
  if (den > 0.0) return ((4.0 * kSqrt3) * area) / den;
  return 0.0;
}

// ---------------------------------------------------------------------------
// Mesh state and the round rule (Algorithm 1).
// ---------------------------------------------------------------------------
struct Options {
  double w_e, w_s;
  double max_cost;  // target edge cost (Section 5.1): +inf = off
  int32_t tolerance, max_rounds, stall_limit, check_mode;
  int32_t exact_target;  // keep only the lowest-key winners needed for N_t
  int32_t recompute_quadrics;  // R16: vertex quadrics from the current faces every round
  // check_mode: 0 = changed faces vs all faces (cell grid),
  //             1 = changed faces vs all faces (brute force),
  //             2 = all face pairs, brute force (Algorithm 3 as printed),
  //             3 = no intersection check (debug)
};

struct EdgeInfo {
  int32_t a, b;          // a < b
  uint64_t key;          // ~0 when ineligible
  float vbar[3];
  double vsolve[3];  // the float64 solve before rounding (NaN when the fallback is taken)
  double Q, l, Cs, cost;
  int32_t link_ok, flagged;
};

struct RoundLog {
  int64_t nV, nF, nE, link_rejects, flagged, eligible, winners, committed,
      undone, undo_iters, pairs_found;
  std::vector<int32_t> winner_pairs, committed_pairs, undone_pairs;
};

struct Run {
  std::vector<float> V;
  std::vector<int32_t> F;
  std::vector<double> K;
  std::vector<RoundLog> logs;
  int status = 0;  // 0 ok, 4 stalled
  double scale = 1.0;
};

struct Mesh {
  int64_t nV = 0, nF = 0;
  std::vector<float> V;     // 3 per vertex
  std::vector<int32_t> F;   // 3 per face
  std::vector<double> K;    // 10 per vertex
};

// incident faces per vertex, ascending face index
static void vertex_faces(const Mesh& m, std::vector<int64_t>& off,
                         std::vector<int32_t>& idx) {
  off.assign(m.nV + 1, 0);
  for (int64_t f = 0; f < m.nF; f++)
    for (int c = 0; c < 3; c++) off[m.F[3 * f + c] + 1]++;
  for (int64_t v = 0; v < m.nV; v++) off[v + 1] += off[v];
  idx.assign(off[m.nV], 0);
  std::vector<int64_t> cur(off.begin(), off.end() - 1);
  for (int64_t f = 0; f < m.nF; f++)
    for (int c = 0; c < 3; c++) idx[cur[m.F[3 * f + c]]++] = (int32_t)f;
}

static void init_quadrics(Mesh& m, const std::vector<int64_t>& off,
                          const std::vector<int32_t>& idx) {
  m.K.assign(10 * m.nV, 0.0);
  for (int64_t v = 0; v < m.nV; v++) {
    for (int64_t s = off[v]; s < off[v + 1]; s++) {
      const int32_t* f = &m.F[3 * (int64_t)idx[s]];
      Quadric q = face_quadric(&m.V[3 * (int64_t)f[0]], &m.V[3 * (int64_t)f[1]],
                               &m.V[3 * (int64_t)f[2]]);
      for (int i = 0; i < 10; i++) m.K[10 * v + i] = m.K[10 * v + i] + q.k[i];
    }
  }
}

static std::vector<std::pair<int32_t, int32_t>> sorted_edges(const Mesh& m) {
  std::vector<std::pair<int32_t, int32_t>> e;
  e.reserve(3 * m.nF);
  for (int64_t f = 0; f < m.nF; f++)
    for (int c = 0; c < 3; c++) {
      int32_t u = m.F[3 * f + c], w = m.F[3 * f + (c + 1) % 3];
      e.push_back({std::min(u, w), std::max(u, w)});
    }
  std::sort(e.begin(), e.end());
  e.erase(std::unique(e.begin(), e.end()), e.end());
  return e;
}

static bool face_has(const int32_t* f, int32_t v) {
  return f[0] == v || f[1] == v || f[2] == v;
}

static std::vector<int32_t> neighbours(const Mesh& m, const std::vector<int64_t>& off,
                                       const std::vector<int32_t>& idx, int32_t v) {
  std::vector<int32_t> n;
  for (int64_t s = off[v]; s < off[v + 1]; s++) {
    const int32_t* f = &m.F[3 * (int64_t)idx[s]];
    for (int c = 0; c < 3; c++)
      if (f[c] != v) n.push_back(f[c]);
  }
  std::sort(n.begin(), n.end());
  n.erase(std::unique(n.begin(), n.end()), n.end());
  return n;
}

// faces in the 1-ring of edge (a,b): union of faces incident to a or b,
// ascending face index
static std::vector<int32_t> edge_ring(const std::vector<int64_t>& off,
                                      const std::vector<int32_t>& idx, int32_t a,
                                      int32_t b) {
  std::vector<int32_t> r(idx.begin() + off[a], idx.begin() + off[a + 1]);
  r.insert(r.end(), idx.begin() + off[b], idx.begin() + off[b + 1]);
  std::sort(r.begin(), r.end());
  r.erase(std::unique(r.begin(), r.end()), r.end());
  return r;
}

// Link condition of Dey et al. for a closed 2-manifold: the common neighbours
// of a and b are exactly the two apexes c, d of the faces on ab, and the faces
// (a,c,d) and (b,c,d) do not both exist.
static bool link_condition(const Mesh& m, const std::vector<int64_t>& off,
                           const std::vector<int32_t>& idx, int32_t a, int32_t b) {
  std::vector<int32_t> na = neighbours(m, off, idx, a);
  std::vector<int32_t> nb = neighbours(m, off, idx, b);
  std::vector<int32_t> common;
  std::set_intersection(na.begin(), na.end(), nb.begin(), nb.end(),
                        std::back_inserter(common));
  std::vector<int32_t> apex;
  for (int64_t s = off[a]; s < off[a + 1]; s++) {
    const int32_t* f = &m.F[3 * (int64_t)idx[s]];
    if (face_has(f, b))
      for (int c = 0; c < 3; c++)
        if (f[c] != a && f[c] != b) apex.push_back(f[c]);
  }
  std::sort(apex.begin(), apex.end());
  if (common.size() != 2 || apex.size() != 2 || common != apex) return false;
  int32_t c = apex[0], d = apex[1];
  bool acd = false, bcd = false;
  for (int64_t s = off[c]; s < off[c + 1]; s++) {
    const int32_t* f = &m.F[3 * (int64_t)idx[s]];
    if (face_has(f, d) && face_has(f, a)) acd = true;
    if (face_has(f, d) && face_has(f, b)) bcd = true;
  }
  return !(acd && bcd);
}

static void edge_cost(const Mesh& m, const std::vector<int64_t>& off,
                      const std::vector<int32_t>& idx, double scale,
                      const Options& o, EdgeInfo& e) {
  int32_t a = e.a, b = e.b;
  double K[10];
  for (int i = 0; i < 10; i++) K[i] = m.K[10 * (int64_t)a + i] + m.K[10 * (int64_t)b + i];
  const float* pa = &m.V[3 * (int64_t)a];
  const float* pb = &m.V[3 * (int64_t)b];
  // optimal placement: solve A v = -b (Cramer), R2
  double r0 = -K[3], r1 = -K[6], r2 = -K[8];
  double mx = std::max(std::max(std::max(std::fabs(K[0]), std::fabs(K[1])),
                                std::max(std::fabs(K[2]), std::fabs(K[4]))),
                       std::max(std::fabs(K[5]), std::fabs(K[7])));
  double det = det3(K[0], K[1], K[2], K[1], K[4], K[5], K[2], K[5], K[7]);
  e.vsolve[0] = e.vsolve[1] = e.vsolve[2] = std::numeric_limits<double>::quiet_NaN();
  bool solved = false;
  float v[3];
  if (mx != 0.0 && !(std::fabs(det) <= 1e-12 * ((mx * mx) * mx))) {
    double x = det3(r0, K[1], K[2], r1, K[4], K[5], r2, K[5], K[7]) / det;
    double y = det3(K[0], r0, K[2], K[1], r1, K[5], K[2], r2, K[7]) / det;
    double z = det3(K[0], K[1], r0, K[1], K[4], r1, K[2], K[5], r2) / det;
    e.vsolve[0] = x;
    e.vsolve[1] = y;
    e.vsolve[2] = z;
    v[0] = (float)x;
    v[1] = (float)y;
    v[2] = (float)z;
    solved = std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
  }
  double Q;
  if (solved) {
    Q = quadric_eval(K, v[0], v[1], v[2]);
  } else {
    float cand[3][3];
    for (int k = 0; k < 3; k++) {
      cand[0][k] = pa[k];
      cand[1][k] = pb[k];
      cand[2][k] = (float)(((double)pa[k] + (double)pb[k]) * 0.5);
    }
    int best = 0;
    double bq = quadric_eval(K, cand[0][0], cand[0][1], cand[0][2]);
    for (int c = 1; c < 3; c++) {
      double q = quadric_eval(K, cand[c][0], cand[c][1], cand[c][2]);
      if (q < bq) {
        bq = q;
        best = c;
      }
    }
    for (int k = 0; k < 3; k++) v[k] = cand[best][k];
    Q = bq;
  }
  double dx = (double)pb[0] - (double)pa[0], dy = (double)pb[1] - (double)pa[1],
         dz = (double)pb[2] - (double)pa[2];
  double l = std::sqrt(dot3(dx, dy, dz, dx, dy, dz));
  // skinny term over the triangles the collapse produces, R3
  double Cs = 0.0;
  std::vector<int32_t> ring = edge_ring(off, idx, a, b);
  double vb[3] = {v[0], v[1], v[2]};
  for (int32_t f : ring) {
    const int32_t* fv = &m.F[3 * (int64_t)f];
    if (face_has(fv, a) && face_has(fv, b)) continue;
    double q[3][3];
    for (int c = 0; c < 3; c++) {
      if (fv[c] == a || fv[c] == b) {
        for (int k = 0; k < 3; k++) q[c][k] = vb[k];
      } else {
        for (int k = 0; k < 3; k++) q[c][k] = (double)m.V[3 * (int64_t)fv[c] + k];
      }
    }
    Cs = Cs + (1.0 - tri_quality(q[0], q[1], q[2]));
  }
  double s2 = scale * scale, wes = o.w_e * scale;
  double cost = mad(o.w_s, Cs, mad(wes, l, s2 * Q));
  e.Q = Q;
  e.l = l;
  e.Cs = Cs;
  e.cost = cost;
  e.vbar[0] = v[0];
  e.vbar[1] = v[1];
  e.vbar[2] = v[2];
  float cf = (float)cost;
  if (std::isnan(cost) || std::isinf(cf)) {
    e.key = ~0ull;
    return;
  }
  if (!(cf > 0.0f)) cf = 0.0f;  // negative rounding residue and -0 -> +0
  uint32_t hi;
  std::memcpy(&hi, &cf, 4);
  e.key = ((uint64_t)hi << 32);  // low word (edge id) added by the caller
}

// AABB of a face
struct Box {
  float lo[3], hi[3];
};

static Box face_box(const Mesh& m, int64_t f) {
  Box b;
  for (int k = 0; k < 3; k++) {
    b.lo[k] = b.hi[k] = m.V[3 * (int64_t)m.F[3 * f] + k];
    for (int c = 1; c < 3; c++) {
      float x = m.V[3 * (int64_t)m.F[3 * f + c] + k];
      b.lo[k] = std::min(b.lo[k], x);
      b.hi[k] = std::max(b.hi[k], x);
    }
  }
  return b;
}

static bool box_overlap(const Box& a, const Box& b) {
  for (int k = 0; k < 3; k++)
    if (a.lo[k] > b.hi[k] || b.lo[k] > a.hi[k]) return false;
  return true;
}

static bool faces_intersect(const Mesh& m, int64_t f, int64_t g) {
  P3 t[3], c[3];
  int32_t ti[3], ci[3];
  for (int i = 0; i < 3; i++) {
    ti[i] = m.F[3 * f + i];
    ci[i] = m.F[3 * g + i];
    for (int k = 0; k < 3; k++) {
      t[i].v[k] = m.V[3 * (int64_t)ti[i] + k];
      c[i].v[k] = m.V[3 * (int64_t)ci[i] + k];
    }
  }
  return tri_intersect(t, ti, c, ci);
}

// Uniform cell grid over the alive faces: a face is listed in every cell its
// AABB touches (faces touching more than 512 cells go to a list scanned for
// every query).  Two overlapping boxes always share a cell, so the candidate
// set is a superset of the box-overlap set.
struct CellGrid {
  double org[3], h;
  std::vector<std::pair<uint64_t, int32_t>> cells;
  std::vector<int32_t> big;
};

static void cell_range(const CellGrid& g, const Box& b, int64_t lo[3], int64_t hi[3]) {
  for (int k = 0; k < 3; k++) {
    lo[k] = (int64_t)std::floor(((double)b.lo[k] - g.org[k]) / g.h);
    hi[k] = (int64_t)std::floor(((double)b.hi[k] - g.org[k]) / g.h);
  }
}

static uint64_t cell_key(int64_t x, int64_t y, int64_t z) {
  return ((uint64_t)(x & 0x1fffff) << 42) | ((uint64_t)(y & 0x1fffff) << 21) |
         (uint64_t)(z & 0x1fffff);
}

static void build_grid(const Mesh& m, const std::vector<char>& alive, CellGrid& g) {
  g.cells.clear();
  g.big.clear();
  double lo[3] = {1e300, 1e300, 1e300};
  std::vector<double> ext;
  for (int64_t f = 0; f < m.nF; f++) {
    if (!alive[f]) continue;
    Box b = face_box(m, f);
    double e = 0;
    for (int k = 0; k < 3; k++) {
      lo[k] = std::min(lo[k], (double)b.lo[k]);
      e = std::max(e, (double)b.hi[k] - (double)b.lo[k]);
    }
    ext.push_back(e);
  }
  if (ext.empty()) {
    g.h = 1.0;
    g.org[0] = g.org[1] = g.org[2] = 0.0;
    return;
  }
  std::nth_element(ext.begin(), ext.begin() + ext.size() / 2, ext.end());
  g.h = std::max(ext[ext.size() / 2] * 2.0, 1e-30);
  for (int k = 0; k < 3; k++) g.org[k] = lo[k];
  for (int64_t f = 0; f < m.nF; f++) {
    if (!alive[f]) continue;
    Box b = face_box(m, f);
    int64_t a[3], c[3];
    cell_range(g, b, a, c);
    double cnt = 1;
    for (int k = 0; k < 3; k++) cnt *= (double)(c[k] - a[k] + 1);
    if (cnt > 512) {
      g.big.push_back((int32_t)f);
      continue;
    }
    for (int64_t x = a[0]; x <= c[0]; x++)
      for (int64_t y = a[1]; y <= c[1]; y++)
        for (int64_t z = a[2]; z <= c[2]; z++)
          g.cells.push_back({cell_key(x, y, z), (int32_t)f});
  }
  std::sort(g.cells.begin(), g.cells.end());
}

// faces g != f, alive, whose box overlaps f's box (each listed once)
static void grid_candidates(const Mesh& m, const CellGrid& g, const std::vector<char>& alive,
                            int64_t f, std::vector<int32_t>& out,
                            std::vector<int64_t>& stamp, int64_t tick) {
  out.clear();
  Box bf = face_box(m, f);
  auto consider = [&](int32_t c) {
    if (c == f || !alive[c] || stamp[c] == tick) return;
    stamp[c] = tick;
    if (box_overlap(bf, face_box(m, c))) out.push_back(c);
  };
  for (int32_t c : g.big) consider(c);
  int64_t a[3], c[3];
  cell_range(g, bf, a, c);
  double cnt = 1;
  for (int k = 0; k < 3; k++) cnt *= (double)(c[k] - a[k] + 1);
  if (cnt > 512) {  // a huge query box: scan everything
    for (int64_t h = 0; h < m.nF; h++) consider((int32_t)h);
    return;
  }
  for (int64_t x = a[0]; x <= c[0]; x++)
    for (int64_t y = a[1]; y <= c[1]; y++)
      for (int64_t z = a[2]; z <= c[2]; z++) {
        uint64_t key = cell_key(x, y, z);
        auto it = std::lower_bound(g.cells.begin(), g.cells.end(),
                                   std::make_pair(key, (int32_t)INT32_MIN));
        for (; it != g.cells.end() && it->first == key; ++it) consider(it->second);
      }
}

static uint64_t pair_key(int32_t a, int32_t b) {
  return ((uint64_t)(uint32_t)std::min(a, b) << 32) | (uint32_t)std::max(a, b);
}

static void analyse_edges(const Mesh& m, const std::vector<int64_t>& off,
                          const std::vector<int32_t>& idx, double scale,
                          const Options& o, const std::vector<uint64_t>& flags,
                          std::vector<EdgeInfo>& edges) {
  std::vector<std::pair<int32_t, int32_t>> es = sorted_edges(m);
  edges.assign(es.size(), EdgeInfo());
  for (size_t i = 0; i < es.size(); i++) {
    EdgeInfo& e = edges[i];
    e.a = es[i].first;
    e.b = es[i].second;
    e.link_ok = link_condition(m, off, idx, e.a, e.b) ? 1 : 0;
    e.flagged = std::binary_search(flags.begin(), flags.end(), pair_key(e.a, e.b)) ? 1 : 0;
    edge_cost(m, off, idx, scale, o, e);
    if (e.key != ~0ull) e.key |= (uint64_t)(uint32_t)i;
  }
}

static double input_scale(const float* V, int64_t nV) {
  if (nV == 0) return 1.0;
  double lo[3], hi[3];
  for (int k = 0; k < 3; k++) lo[k] = hi[k] = V[k];
  for (int64_t v = 1; v < nV; v++)
    for (int k = 0; k < 3; k++) {
      lo[k] = std::min(lo[k], (double)V[3 * v + k]);
      hi[k] = std::max(hi[k], (double)V[3 * v + k]);
    }
  double ext = std::max(std::max(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
  return ext > 0.0 ? 1.0 / ext : 1.0;
}

static uint32_t float_bits_of_max_cost(double max_cost) {
  if (!(max_cost < INFINITY)) return 0x7f800000u;  // +inf: every finite cost
  float f = (float)max_cost;
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
}

static void simplify(Mesh m, int64_t target, const Options& o, Run& run) {
  run.scale = input_scale(m.V.data(), m.nV);
  std::vector<int64_t> off;
  std::vector<int32_t> idx;
  vertex_faces(m, off, idx);
  init_quadrics(m, off, idx);
  std::vector<uint64_t> flags;  // invalid edges as sorted vertex pairs
  int hold = 0, zero_streak = 0;
  int round = 0;
  run.status = 0;
  while (m.nF > target) {
    if (round >= o.max_rounds) {
      run.status = 4;
      break;
    }
    RoundLog L{};
    L.nV = m.nV;
    L.nF = m.nF;
    vertex_faces(m, off, idx);
    if (o.recompute_quadrics) init_quadrics(m, off, idx);  // R16
    // --- edge costs (Algorithm 1, first parallel loop; Eq. 1)
    std::vector<EdgeInfo> edges;
    analyse_edges(m, off, idx, run.scale, o, flags, edges);
    L.nE = (int64_t)edges.size();
    // target edge cost (R14): an edge whose float cost exceeds (float)max_cost
    // is not eligible; compared on the key's float bits (non-negative floats
    // order as unsigned integers)
    const uint32_t max_bits = float_bits_of_max_cost(o.max_cost);
    std::vector<char> elig(edges.size(), 0);
    for (size_t i = 0; i < edges.size(); i++) {
      if (!edges[i].link_ok) L.link_rejects++;
      if (edges[i].flagged) L.flagged++;
      elig[i] = edges[i].link_ok && !edges[i].flagged && edges[i].key != ~0ull &&
                (uint32_t)(edges[i].key >> 32) <= max_bits;
      if (elig[i]) L.eligible++;
    }
    // --- cost propagation onto the 1-ring triangles (push form, Sec. 5.1)
    std::vector<uint64_t> tkey(m.nF, ~0ull);
    std::vector<std::vector<int32_t>> rings(edges.size());
    for (size_t i = 0; i < edges.size(); i++) {
      if (!elig[i]) continue;
      rings[i] = edge_ring(off, idx, edges[i].a, edges[i].b);
      for (int32_t t : rings[i]) tkey[t] = std::min(tkey[t], edges[i].key);
    }
    // --- independent regions: all ring triangles hold the edge's key
    std::vector<int32_t> winners;
    for (size_t i = 0; i < edges.size(); i++) {
      if (!elig[i]) continue;
      bool win = true;
      for (int32_t t : rings[i])
        if (tkey[t] != edges[i].key) {
          win = false;
          break;
        }
      if (win) winners.push_back((int32_t)i);
    }
    // exact-target mode (R15): when the winners would remove more faces than
    // |F| - N_t, keep the ceil((|F| - N_t) / 2) lowest keys, in edge-id order
    if (o.exact_target) {
      const int64_t need = (m.nF - target + 1) / 2;
      if ((int64_t)winners.size() > need) {
        std::vector<int32_t> by_key = winners;
        std::sort(by_key.begin(), by_key.end(),
                  [&](int32_t x, int32_t y) { return edges[x].key < edges[y].key; });
        by_key.resize(need);
        std::sort(by_key.begin(), by_key.end());
        winners.swap(by_key);
      }
    }
    L.winners = (int64_t)winners.size();
    for (int32_t w : winners) {
      L.winner_pairs.push_back(edges[w].a);
      L.winner_pairs.push_back(edges[w].b);
    }
    // --- collapse all winners into M_s (M_1 = m stays untouched)
    Mesh s = m;
    std::vector<int32_t> tag(m.nF, -1);        // collapse (winner slot) per face
    std::vector<char> fdead(m.nF, 0), vdead(m.nV, 0), standing(winners.size(), 1);
    std::vector<std::vector<int32_t>> wring(winners.size());
    for (size_t w = 0; w < winners.size(); w++) {
      const EdgeInfo& e = edges[winners[w]];
      wring[w] = rings[winners[w]];
      for (int k = 0; k < 3; k++) s.V[3 * (int64_t)e.a + k] = e.vbar[k];
      for (int i = 0; i < 10; i++)
        s.K[10 * (int64_t)e.a + i] = m.K[10 * (int64_t)e.a + i] + m.K[10 * (int64_t)e.b + i];
      vdead[e.b] = 1;
      for (int32_t f : wring[w]) {
        int32_t* fv = &s.F[3 * (int64_t)f];
        if (face_has(fv, e.a) && face_has(fv, e.b)) {
          fdead[f] = 1;
        } else {
          for (int c = 0; c < 3; c++)
            if (fv[c] == e.b) fv[c] = e.a;
        }
        tag[f] = (int32_t)w;
      }
    }
    // --- repeat { intersection check; undo } until clean (Sec. 5.2, 5.3)
    if (o.check_mode != 3) {
      std::vector<int64_t> stamp(m.nF, -1);
      int64_t tick = 0;
      std::vector<int32_t> cand;
      while (true) {
        std::vector<char> alive(m.nF);
        for (int64_t f = 0; f < m.nF; f++) alive[f] = !fdead[f];
        std::vector<char> undo(winners.size(), 0);
        int64_t npairs = 0;
        if (o.check_mode == 2) {
          for (int64_t f = 0; f < m.nF; f++) {
            if (!alive[f]) continue;
            for (int64_t g = f + 1; g < m.nF; g++) {
              if (!alive[g]) continue;
              if (!box_overlap(face_box(s, f), face_box(s, g))) continue;
              if (faces_intersect(s, f, g)) {
                npairs++;
                if (tag[f] >= 0) undo[tag[f]] = 1;
                if (tag[g] >= 0) undo[tag[g]] = 1;
              }
            }
          }
        } else {
          CellGrid grid;
          if (o.check_mode == 0) build_grid(s, alive, grid);
          for (int64_t f = 0; f < m.nF; f++) {
            if (!alive[f] || tag[f] < 0) continue;
            cand.clear();
            if (o.check_mode == 0) {
              grid_candidates(s, grid, alive, f, cand, stamp, ++tick);
            } else {
              Box bf = face_box(s, f);
              for (int64_t g = 0; g < m.nF; g++)
                if (g != f && alive[g] && box_overlap(bf, face_box(s, g)))
                  cand.push_back((int32_t)g);
            }
            for (int32_t g : cand) {
              if (tag[g] >= 0 && g < f) continue;  // pair seen from g's side
              if (faces_intersect(s, f, g)) {
                npairs++;
                undo[tag[f]] = 1;
                if (tag[g] >= 0) undo[tag[g]] = 1;
              }
            }
          }
        }
        L.pairs_found += npairs;
        bool any = false;
        for (size_t w = 0; w < winners.size(); w++)
          if (undo[w]) any = true;
        if (!any) break;
        L.undo_iters++;
        for (size_t w = 0; w < winners.size(); w++) {
          if (!undo[w]) continue;
          const EdgeInfo& e = edges[winners[w]];
          standing[w] = 0;
          for (int32_t f : wring[w]) {
            for (int c = 0; c < 3; c++) s.F[3 * (int64_t)f + c] = m.F[3 * (int64_t)f + c];
            fdead[f] = 0;
            tag[f] = -1;
          }
          for (int k = 0; k < 3; k++) {
            s.V[3 * (int64_t)e.a + k] = m.V[3 * (int64_t)e.a + k];
            s.V[3 * (int64_t)e.b + k] = m.V[3 * (int64_t)e.b + k];
          }
          for (int i = 0; i < 10; i++) s.K[10 * (int64_t)e.a + i] = m.K[10 * (int64_t)e.a + i];
          vdead[e.b] = 0;
        }
      }
    }
    // --- commit: stable compaction (R8), flags for the next round (R10)
    std::vector<uint64_t> undone_pairs;
    for (size_t w = 0; w < winners.size(); w++) {
      const EdgeInfo& e = edges[winners[w]];
      if (standing[w]) {
        L.committed++;
        L.committed_pairs.push_back(e.a);
        L.committed_pairs.push_back(e.b);
      } else {
        L.undone++;
        L.undone_pairs.push_back(e.a);
        L.undone_pairs.push_back(e.b);
        undone_pairs.push_back(pair_key(e.a, e.b));
      }
    }
    std::vector<int32_t> vmap(m.nV, -1);
    Mesh n;
    for (int64_t v = 0; v < m.nV; v++) {
      if (vdead[v]) continue;
      vmap[v] = (int32_t)n.nV++;
      for (int k = 0; k < 3; k++) n.V.push_back(s.V[3 * v + k]);
      for (int i = 0; i < 10; i++) n.K.push_back(s.K[10 * v + i]);
    }
    for (int64_t f = 0; f < m.nF; f++) {
      if (fdead[f]) continue;
      for (int c = 0; c < 3; c++) n.F.push_back(vmap[s.F[3 * f + c]]);
      n.nF++;
    }
    std::vector<uint64_t> next;
    if (L.committed > 0) {
      hold = 0;
      zero_streak = 0;
    } else {
      next = flags;
      hold++;
      zero_streak++;
    }
    next.insert(next.end(), undone_pairs.begin(), undone_pairs.end());
    if (L.committed == 0 && hold >= o.tolerance) {
      next.clear();
      hold = 0;
    }
    for (uint64_t& p : next) {
      int32_t a = vmap[(int32_t)(p >> 32)], b = vmap[(int32_t)(uint32_t)p];
      p = pair_key(a, b);
    }
    std::sort(next.begin(), next.end());
    next.erase(std::unique(next.begin(), next.end()), next.end());
    bool stall_empty = (L.eligible == 0 && flags.empty());
    flags.swap(next);
    m = std::move(n);
    run.logs.push_back(std::move(L));
    round++;
    if (stall_empty || zero_streak >= o.stall_limit) {
      // with a target edge cost, running out of eligible edges is the normal end
      const bool cost_end = stall_empty && std::isfinite(o.max_cost);
      if (m.nF > target && !cost_end) run.status = 4;
      break;
    }
  }
  run.V = m.V;
  run.F = m.F;
  run.K = m.K;
}

static Options to_options(const double* w, const int32_t* iopt) {
  Options o;
  o.w_e = w[0];
  o.w_s = w[1];
  o.tolerance = iopt[0];
  o.max_rounds = iopt[1];
  o.stall_limit = iopt[2];
  o.check_mode = iopt[3];
  o.exact_target = iopt[4];
  o.recompute_quadrics = iopt[5];
  o.max_cost = w[2];
  return o;
}

static Mesh to_mesh(const float* V, int64_t nV, const int32_t* F, int64_t nF) {
  Mesh m;
  m.nV = nV;
  m.nF = nF;
  m.V.assign(V, V + 3 * nV);
  m.F.assign(F, F + 3 * nF);
  return m;
}

}  // namespace

// ---------------------------------------------------------------------------
// C interface used by the tests (ctypes).
// ---------------------------------------------------------------------------
extern "C" {

int or_orient3d(const float* p) { return orient3d(p, p + 3, p + 6, p + 9); }
int or_orient3d_exact(const float* p) { return orient3d_exact(p, p + 3, p + 6, p + 9); }
int or_orient2d(const float* p) { return orient2d(p[0], p[1], p[2], p[3], p[4], p[5]); }
int or_orient2d_exact(const float* p) {
  return orient2d_exact(p[0], p[1], p[2], p[3], p[4], p[5]);
}

// p: 18 floats (T's three corners then C's), idx: 6 vertex indices
int or_tri_intersect(const float* p, const int32_t* idx) {
  P3 t[3], c[3];
  for (int i = 0; i < 3; i++)
    for (int k = 0; k < 3; k++) {
      t[i].v[k] = p[3 * i + k];
      c[i].v[k] = p[9 + 3 * i + k];
    }
  return tri_intersect(t, idx, c, idx + 3) ? 1 : 0;
}

// Vertex quadrics of a mesh (10 doubles per vertex).
void or_vertex_quadrics(const float* V, int64_t nV, const int32_t* F, int64_t nF,
                        double* K) {
  Mesh m = to_mesh(V, nV, F, nF);
  std::vector<int64_t> off;
  std::vector<int32_t> idx;
  vertex_faces(m, off, idx);
  init_quadrics(m, off, idx);
  std::memcpy(K, m.K.data(), sizeof(double) * 10 * nV);
}

// Round-0 edge table.  Returns the number of edges; the arrays (capacity cap)
// receive endpoints, key, placement, the Eq. 1 terms and eligibility bits.
int64_t or_edge_table(const float* V, int64_t nV, const int32_t* F, int64_t nF,
                      const double* w, int64_t cap, int32_t* ab, uint64_t* key,
                      float* vbar, double* terms, int32_t* bits, double* vsolve) {
  Mesh m = to_mesh(V, nV, F, nF);
  std::vector<int64_t> off;
  std::vector<int32_t> idx;
  vertex_faces(m, off, idx);
  init_quadrics(m, off, idx);
  Options o{};
  o.w_e = w[0];
  o.w_s = w[1];
  std::vector<EdgeInfo> edges;
  analyse_edges(m, off, idx, input_scale(V, nV), o, {}, edges);
  int64_t n = (int64_t)edges.size();
  for (int64_t i = 0; i < n && i < cap; i++) {
    const EdgeInfo& e = edges[i];
    ab[2 * i] = e.a;
    ab[2 * i + 1] = e.b;
    bool elig = e.link_ok && e.key != ~0ull;
    key[i] = elig ? e.key : ~0ull;
    for (int k = 0; k < 3; k++) vbar[3 * i + k] = e.vbar[k];
    if (vsolve)
      for (int k = 0; k < 3; k++) vsolve[3 * i + k] = e.vsolve[k];
    terms[4 * i] = e.Q;
    terms[4 * i + 1] = e.l;
    terms[4 * i + 2] = e.Cs;
    terms[4 * i + 3] = e.cost;
    bits[i] = e.link_ok;
  }
  return n;
}

void* or_run(const float* V, int64_t nV, const int32_t* F, int64_t nF,
             int64_t target, const double* w, const int32_t* iopt) {
  Run* r = new Run();
  simplify(to_mesh(V, nV, F, nF), target, to_options(w, iopt), *r);
  return r;
}

void or_free(void* h) { delete (Run*)h; }
int or_status(void* h) { return ((Run*)h)->status; }
int64_t or_rounds(void* h) { return (int64_t)((Run*)h)->logs.size(); }
int64_t or_nv(void* h) { return (int64_t)((Run*)h)->V.size() / 3; }
int64_t or_nf(void* h) { return (int64_t)((Run*)h)->F.size() / 3; }
double or_scale(void* h) { return ((Run*)h)->scale; }

void or_mesh(void* h, float* V, int32_t* F, double* K) {
  Run* r = (Run*)h;
  std::memcpy(V, r->V.data(), sizeof(float) * r->V.size());
  std::memcpy(F, r->F.data(), sizeof(int32_t) * r->F.size());
  if (K) std::memcpy(K, r->K.data(), sizeof(double) * r->K.size());
}

// 11 counters per round: nV nF nE link_rejects flagged eligible winners
// committed undone undo_iters pairs_found
void or_round_info(void* h, int64_t r, int64_t* out) {
  const RoundLog& L = ((Run*)h)->logs[r];
  int64_t v[11] = {L.nV, L.nF, L.nE, L.link_rejects, L.flagged, L.eligible,
                   L.winners, L.committed, L.undone, L.undo_iters, L.pairs_found};
  std::memcpy(out, v, sizeof(v));
}

// kind 0 = winners, 1 = committed, 2 = undone; vertex pairs in that round's
// input numbering.  Returns the number of pairs.
int64_t or_round_pairs(void* h, int64_t r, int kind, int32_t* out, int64_t cap) {
  const RoundLog& L = ((Run*)h)->logs[r];
  const std::vector<int32_t>& p =
      kind == 0 ? L.winner_pairs : (kind == 1 ? L.committed_pairs : L.undone_pairs);
  int64_t n = (int64_t)p.size() / 2;
  if (out) std::memcpy(out, p.data(), sizeof(int32_t) * std::min<int64_t>(2 * n, 2 * cap));
  return n;
}

// C_ijk of Eq. 1 for one triangle (9 doubles).
double or_tri_quality(const double* q) { return tri_quality(q, q + 3, q + 6); }

// 1: every fused multiply-add of the cost becomes a multiply and an add (R13)
void or_set_plain_products(int on) { g_plain_products = on != 0; }

// All intersecting face pairs of a mesh (Algorithm 3 applied to every face).
// brute = 1 tests every face pair, else box-overlap candidates from the cell
// grid.  Returns the count; writes up to cap pairs.
int64_t or_self_intersections(const float* V, int64_t nV, const int32_t* F,
                              int64_t nF, int32_t* out, int64_t cap, int brute) {
  Mesh m = to_mesh(V, nV, F, nF);
  if (brute) {
    int64_t n = 0;
    for (int64_t f = 0; f < nF; f++)
      for (int64_t c = f + 1; c < nF; c++)
        if (faces_intersect(m, f, c)) {
          if (out && n < cap) {
            out[2 * n] = (int32_t)f;
            out[2 * n + 1] = (int32_t)c;
          }
          n++;
        }
    return n;
  }
  std::vector<char> alive(nF, 1);
  CellGrid g;
  build_grid(m, alive, g);
  std::vector<int64_t> stamp(nF, -1);
  std::vector<int32_t> cand;
  int64_t n = 0, tick = 0;
  for (int64_t f = 0; f < nF; f++) {
    grid_candidates(m, g, alive, f, cand, stamp, ++tick);
    for (int32_t c : cand) {
      if (c < f) continue;
      if (faces_intersect(m, f, c)) {
        if (out && n < cap) {
          out[2 * n] = (int32_t)f;
          out[2 * n + 1] = c;
        }
        n++;
      }
    }
  }
  return n;
}

}  // extern "C"
