// Edge costs of one round (Algorithm 1, first parallel loop; Eq. 1):
//   C_ab = s^2 Q_ab + w_e s l_ab + w_s sum(1 - C_ijk)
// with the Garland-Heckbert quadric error Q_ab at the optimal placement, the
// edge length, and the skinny term over the triangles the collapse produces;
// s = 1 / (largest extent of the input box) puts the costs in the [0,1]^3 frame
// the paper normalises to (start of Section 4).  The same kernel evaluates the
// link condition (Dey et al., cited in Section 5.1) and the invalid-edge flags
// (Section 5.3) and packs the 64-bit key (float cost bits << 32 | edge id).
//
// All float64 arithmetic is IEEE round-to-nearest in a fixed evaluation order
// (the library is compiled with --fmad=false, so only the explicit __fma_rn
// calls fuse), so the keys are reproducible bit for bit.
#include "common.cuh"
#include "skinny_ff.cuh"

namespace pamo {

namespace {

constexpr double kSqrt3 = 1.7320508075688772;

// float -> double on the integer pipe (exact for normal floats; zero,
// subnormals, inf and NaN take the hardware conversion).  The float64 unit is
// the scarce resource of this kernel.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u || e == 0xffu) return (double)f;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

// Fixed evaluation order with explicit fused multiply-adds (one rounding each).
__device__ __forceinline__ double det3(double a00, double a01, double a02, double a10, double a11,
                                       double a12, double a20, double a21, double a22) {
  const double m0 = __fma_rn(a11, a22, -(a12 * a21));
  const double m1 = __fma_rn(a10, a22, -(a12 * a20));
  const double m2 = __fma_rn(a10, a21, -(a11 * a20));
  return __fma_rn(a02, m2, __fma_rn(-a01, m1, a00 * m0));
}

// v^T A v + 2 b^T v + c of the summed quadric
__device__ __forceinline__ double qeval(const double* K, double x, double y, double z) {
  const double ax = __fma_rn(K[2], z, __fma_rn(K[1], y, K[0] * x));
  const double ay = __fma_rn(K[5], z, __fma_rn(K[4], y, K[1] * x));
  const double az = __fma_rn(K[7], z, __fma_rn(K[5], y, K[2] * x));
  const double bv = __fma_rn(K[8], z, __fma_rn(K[6], y, K[3] * x));
  return __fma_rn(2.0, bv, __fma_rn(z, az, __fma_rn(y, ay, x * ax))) + K[9];
}

__device__ __forceinline__ double dot3(double ax, double ay, double az, double bx, double by,
                                       double bz) {
  return __fma_rn(az, bz, __fma_rn(ay, by, ax * bx));
}

// Finite doubles compare with zero on their bit patterns (a finite double is
// > 0 iff its bits are > 0 as a signed integer): the test runs on the integer
// pipe, off the float64 pipe.
__device__ __forceinline__ bool pos_finite(double x) { return __double_as_longlong(x) > 0; }

// C_ijk = 4 sqrt(3) A / (l_ij^2 + l_jk^2 + l_ki^2) of Eq. 1 for the triangle
// (q0, q1, q2): A = |u x w| / 2 with u = q1 - q0, w = q2 - q0, and the three
// squared edge lengths summed in the order (q0q1, q1q2, q2q0).  Evaluated as
// (2 sqrt(3) |u x w|) / den, which rounds to the same bits as
// (4 sqrt(3) (|u x w| / 2)) / den: 4 sqrt(3) and 2 sqrt(3) are exact
// multiples of the float64 sqrt(3), and halving |u x w| is exact (for float32
// corners it is zero or far above the subnormal range).
__device__ __forceinline__ double quality(double x0, double y0, double z0, double x1, double y1,
                                          double z1, double x2, double y2, double z2) {
  constexpr double k2Sqrt3 = 2.0 * kSqrt3;
  const double ux = x1 - x0, uy = y1 - y0, uz = z1 - z0;
  const double tx = x2 - x1, ty = y2 - y1, tz = z2 - z1;
  const double wx = x2 - x0, wy = y2 - y0, wz = z2 - z0;
  const double nx = __fma_rn(uy, wz, -(uz * wy));
  const double ny = __fma_rn(uz, wx, -(ux * wz));
  const double nz = __fma_rn(ux, wy, -(uy * wx));
  const double n2 = dot3(nx, ny, nz, nx, ny, nz);
  const double den = (dot3(ux, uy, uz, ux, uy, uz) + dot3(tx, ty, tz, tx, ty, tz)) +
                     dot3(wx, wy, wz, wx, wy, wz);
  return pos_finite(den) ? (k2Sqrt3 * sqrt(n2)) / den : 0.0;
}

// per-mesh eligible counts of a batch: one atomic per group of lanes with the
// same mesh (m < 0: nothing to count); every lane of the warp must call it
__device__ __forceinline__ void count_by_mesh(int m, int32_t* __restrict__ melig) {
  const unsigned peers = __match_any_sync(0xffffffffu, m);
  if (m >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&melig[m], __popc(peers));
}

__device__ __forceinline__ bool has(const int4& f, int v) {
  return f.x == v || f.y == v || f.z == v;
}

__device__ __forceinline__ bool is_flagged(const unsigned long long* flags, int n,
                                           unsigned long long k) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t m = (lo + hi) >> 1;
    unsigned long long x = flags[m];
    if (x == k) return true;
    if (x < k) lo = m + 1;
    else hi = m;
  }
  return false;
}

// Clean edges (neither endpoint is a survivor of the last round or adjacent to
// one) keep last round's cost bits, placement and link result: the edge's two
// vertex rings, quadrics and positions are unchanged and the ring's relative
// face order is kept by the stable compaction, so recomputing would give the
// same bits.  Dirty edges go to a list for k_edge_cost.
__global__ void __launch_bounds__(kBlock) k_edge_reuse(
    const int2* __restrict__ E, const uint8_t* __restrict__ vdirty,
    const int32_t* __restrict__ ivmap, const int2* __restrict__ E_prev,
    const int32_t* __restrict__ e_off_prev, const uint32_t* __restrict__ cbits_prev,
    const float4* __restrict__ vbar_prev, const uint8_t* __restrict__ link_prev,
    const unsigned long long* __restrict__ flags, unsigned long long* __restrict__ key,
    float4* __restrict__ vbar, uint32_t* __restrict__ cbits, uint8_t* __restrict__ link,
    int32_t* __restrict__ dlist, RoundCounters* __restrict__ dc,
    const int32_t* __restrict__ vmesh, const uint8_t* __restrict__ mactive,
    int32_t* __restrict__ melig, unsigned long long* __restrict__ vkey) {
  const int nE = dc->nE;
  // the per-vertex minima of the selection start from "no key" (nothing
  // reads them before the selection)
  {
    const int nV = dc->nV;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nV;
         v += (int64_t)gridDim.x * blockDim.x)
      vkey[v] = ~0ull;
  }
  const int nflags = dc->nflags;
  const unsigned max_bits = dc->max_bits;
  const bool all_dirty = !dc->have_prev;
  int link_bad = 0, flagged = 0, eligible = 0;
  const int lane = threadIdx.x & 31;
  // the whole warp iterates together (block-uniform base) for the ballots
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nE;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = base + threadIdx.x;
    bool dirty = false;
    int counted = -1;  // mesh of an eligible clean edge (batch)
    if (e < nE) {
      const int2 ab = E[e];
      dirty = all_dirty || vdirty[ab.x] || vdirty[ab.y];
      if (!dirty) {
        const int ua = ivmap[ab.x], ub = ivmap[ab.y];
        int lo = e_off_prev[ua], hi = e_off_prev[ua + 1];
        while (lo < hi) {  // previous edges of ua are sorted by their other end
          const int m = (lo + hi) >> 1;
          if (E_prev[m].y < ub) lo = m + 1;
          else hi = m;
        }
        const uint32_t cb = cbits_prev[lo];
        const uint8_t lk = link_prev[lo];
        cbits[e] = cb;
        link[e] = lk;
        vbar[e] = vbar_prev[lo];
        const bool flag = nflags > 0 &&
                          is_flagged(flags, nflags,
                                     ((unsigned long long)(unsigned)ab.x << 32) | (unsigned)ab.y);
        const int m = vmesh ? vmesh[ab.x] : 0;
        const bool active = !vmesh || mactive[m];
        unsigned long long k = ~0ull;
        if (cb != 0xffffffffu && cb <= max_bits && lk && !flag && active) {
          k = ((unsigned long long)cb << 32) | (unsigned long long)(uint32_t)e;
          eligible++;
          counted = m;
        }
        key[e] = k;
        link_bad += !lk;
        flagged += flag;
      }
    }
    if (vmesh) count_by_mesh(counted, melig);
    // dirty edges: warp-aggregated append to the work list
    const unsigned m = __ballot_sync(0xffffffffu, dirty);
    if (m) {
      int b0 = 0;
      if (lane == __ffs(m) - 1) b0 = atomicAdd(&dc->n_dirty, __popc(m));
      b0 = __shfl_sync(0xffffffffu, b0, __ffs(m) - 1);
      if (dirty) dlist[b0 + __popc(m & ((1u << lane) - 1u))] = (int32_t)e;
    }
  }
  link_bad = __reduce_add_sync(0xffffffffu, link_bad);
  flagged = __reduce_add_sync(0xffffffffu, flagged);
  eligible = __reduce_add_sync(0xffffffffu, eligible);
  if (lane == 0) {
    if (link_bad) atomicAdd(&dc->link_rejects, (unsigned long long)link_bad);
    if (flagged) atomicAdd(&dc->flagged, (unsigned long long)flagged);
    if (eligible) atomicAdd(&dc->eligible, (unsigned long long)eligible);
  }
}

// Produced triangles of one warp's edges, flattened over the warp's lanes.
// An edge produces val(a) + val(b) - 4 triangles on a closed manifold, and a
// lane walking its own edge's two incidence lists meets the two faces on ab
// at its own iterations, so a per-lane loop leaves about a third of the
// float64 pipe's lane slots idle.  Instead each lane writes its produced face
// ids (ascending) to shared memory, the warp evaluates 1 - C_ijk for all of
// them 32 at a time, and each lane then adds up its own terms in the same
// ascending order -- the same roundings as the per-lane loop.
constexpr int kFlatCap = 320;  // produced triangles per warp; more: per-lane loop
struct FlatTris {
  union {
    double t[kFlatCap];             // 1 - C_ijk in float64 (edges evaluated in float64)
    float2 tf[kFlatCap];            // 1 - C_ijk as a float pair (certified edges)
  };
  float vx[32], vy[32], vz[32];     // the owner edge's placement
  int face[kFlatCap];
  int a[32], b[32];
  short slot[kFlatCap];             // triangles of the edges evaluated in float64
  unsigned char own[kFlatCap];      // lane of the owner edge
};

// Key bits of a cost: float(cost) clamped at 0, ~0 when not finite.  On finite
// floats the map is monotone, which the certification below relies on.
__device__ __forceinline__ uint32_t key_bits(double cost) {
  float cf = __double2float_rn(cost);
  if (isnan(cost) || isinf(cf)) return 0xffffffffu;
  if (!(cf > 0.0f)) cf = 0.0f;
  return __float_as_uint(cf);
}

// 1 - C_ijk of face t with corners a and b moved to (vx, vy, vz), float-float
__device__ __forceinline__ float2 skinny_term_ff(const int4& t, int a, int b, float vx, float vy,
                                                 float vz, const float4* __restrict__ pos) {
  // the placement is the one corner that is a or b; C_ijk is symmetric
  int p = t.x, q = t.y;
  if (t.x == a || t.x == b) { p = t.y; q = t.z; }
  else if (t.y == a || t.y == b) { p = t.z; q = t.x; }
  const float4 P = pos[p], R = pos[q];
  return ff::skinny_term_ff(vx, vy, vz, P.x, P.y, P.z, R.x, R.y, R.z);
}

// 1 - C_ijk of face t with corners a and b moved to (vx, vy, vz)
__device__ __forceinline__ double skinny_term(const int4& t, int a, int b, double vx, double vy,
                                              double vz, const float4* __restrict__ pos) {
  double q[9];
  const int cs[3] = {t.x, t.y, t.z};
#pragma unroll
  for (int k = 0; k < 3; k++) {
    if (cs[k] == a || cs[k] == b) {
      q[3 * k] = vx; q[3 * k + 1] = vy; q[3 * k + 2] = vz;
    } else {
      const float4 p = pos[cs[k]];
      q[3 * k] = f2d(p.x); q[3 * k + 1] = f2d(p.y); q[3 * k + 2] = f2d(p.z);
    }
  }
  return 1.0 - quality(q[0], q[1], q[2], q[3], q[4], q[5], q[6], q[7], q[8]);
}

// 14 blocks of 64 per SM (72 registers): the kernel waits on dependent
// gathers (incidence lists, faces, positions), so more resident warps pay
// more than the few spilled registers cost
__global__ void __launch_bounds__(kItemBlock, 14) k_edge_cost(
    const int32_t* __restrict__ dlist, const int2* __restrict__ E, const float4* __restrict__ pos,
    const double* __restrict__ Kv, const int4* __restrict__ F, const int32_t* __restrict__ off,
    const int32_t* __restrict__ idx, const int32_t* __restrict__ nbr,
    const unsigned long long* __restrict__ flags,
    double s2_in, double wes_in, double ws, unsigned long long* __restrict__ key,
    float4* __restrict__ vbar, uint32_t* __restrict__ cbits, uint8_t* __restrict__ link,
    RoundCounters* __restrict__ dc, const int32_t* __restrict__ vmesh,
    const double* __restrict__ mcost, const uint8_t* __restrict__ mactive,
    int32_t* __restrict__ melig) {
  __shared__ FlatTris flat[kItemBlock / 32];
  FlatTris& S = flat[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int ndirty = dc->n_dirty;
  const int nflags = dc->nflags;
  const unsigned max_bits = dc->max_bits;
  int link_bad = 0, flagged = 0, eligible = 0, ntri = 0, nf64 = 0;
  // block-uniform iterations: the triangle stage and the per-mesh count are
  // warp-wide operations
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < ndirty;
       base += (int64_t)gridDim.x * blockDim.x) {
  const int64_t i = base + threadIdx.x;
  const bool live = i < ndirty;
  int counted = -1;
  int64_t e = 0;
  int a = 0, b = 0, m = 0, a0 = 0, a1 = 0, b0 = 0, b1 = 0, nt = 0;
  double s2 = 0.0, wes = 0.0, Q = 0.0, l = 0.0;
  float vx = 0.f, vy = 0.f, vz = 0.f;
  bool link_ok = false, flag = false;
  if (live) {
    e = dlist[i];
    const int2 ab = E[e];
    a = ab.x;
    b = ab.y;
    m = vmesh ? vmesh[a] : 0;
    // the mesh's own [0,1]^3 scale (a batch); one mesh: the arguments
    s2 = vmesh ? mcost[2 * m] : s2_in;
    wes = vmesh ? mcost[2 * m + 1] : wes_in;
    a0 = off[a]; a1 = off[a + 1]; b0 = off[b]; b1 = off[b + 1];
    // ---- link condition: exactly two common neighbours (the apexes of the
    // two faces on ab) and not both faces (a,c,d), (b,c,d) present.
    // common = the pairs of equal entries of the neighbour multisets of a and
    // b (the corner after a, resp. b, in each incident face; sorted, at the
    // incidence lists' offsets); the faces on ab are the face ids both sorted
    // incidence lists hold, in ascending order
    int common = 0;
    for (int i = a0, j = b0; i < a1 && j < b1;) {
      const int x = nbr[i], y = nbr[j];
      if (x != y) {
        i += x < y;
        j += y < x;
        continue;
      }
      int ra = 0, rb = 0;
      for (; i < a1 && nbr[i] == x; i++) ra++;
      for (; j < b1 && nbr[j] == x; j++) rb++;
      common += ra * rb;
    }
    int fab[2] = {-1, -1}, na = 0;
    for (int i = a0, j = b0; i < a1 && j < b1;) {
      const int x = idx[i], y = idx[j];
      if (x == y) {
        if (na < 2) fab[na] = x;
        na++;
      }
      i += x <= y;
      j += y <= x;
    }
    // the collapse produces every face around a or b but the na on ab
    nt = (a1 - a0) + (b1 - b0) - 2 * na;
    link_ok = (common == 2) && (na == 2);
    if (link_ok) {
      // the apexes: third corners of the two faces on ab
      const int4 f0 = F[fab[0]], f1 = F[fab[1]];
      const int c = f0.x != a && f0.x != b ? f0.x : (f0.y != a && f0.y != b ? f0.y : f0.z);
      const int d = f1.x != a && f1.x != b ? f1.x : (f1.y != a && f1.y != b ? f1.y : f1.z);
      bool acd = false, bcd = false;
      for (int i = off[c]; i < off[c + 1]; i++) {
        const int4 f = F[idx[i]];
        if (has(f, d)) {
          acd |= has(f, a);
          bcd |= has(f, b);
        }
      }
      link_ok = !(acd && bcd);
    }
    flag = nflags > 0 &&
           is_flagged(flags, nflags, ((unsigned long long)(unsigned)a << 32) | (unsigned)b);
    // ---- Q_ab at the optimal placement (Cramer solve of A v = -b)
    double K[10];
    {
      const double2* ka = reinterpret_cast<const double2*>(Kv + 10 * (int64_t)a);
      const double2* kb = reinterpret_cast<const double2*>(Kv + 10 * (int64_t)b);
#pragma unroll
      for (int i = 0; i < 5; i++) {
        double2 x = ka[i], y = kb[i];
        K[2 * i] = x.x + y.x;
        K[2 * i + 1] = x.y + y.y;
      }
    }
    const float4 pa = pos[a], pb = pos[b];
    const double r0 = -K[3], r1 = -K[6], r2 = -K[8];
    const double mx = fmax(fmax(fmax(fabs(K[0]), fabs(K[1])), fmax(fabs(K[2]), fabs(K[4]))),
                           fmax(fabs(K[5]), fabs(K[7])));
    const double det = det3(K[0], K[1], K[2], K[1], K[4], K[5], K[2], K[5], K[7]);
    bool solved = false;
    if (mx != 0.0 && !(fabs(det) <= 1e-12 * ((mx * mx) * mx))) {
      const double x = det3(r0, K[1], K[2], r1, K[4], K[5], r2, K[5], K[7]) / det;
      const double y = det3(K[0], r0, K[2], K[1], r1, K[5], K[2], r2, K[7]) / det;
      const double z = det3(K[0], K[1], r0, K[1], K[4], r1, K[2], K[5], r2) / det;
      vx = __double2float_rn(x);
      vy = __double2float_rn(y);
      vz = __double2float_rn(z);
      solved = isfinite(vx) && isfinite(vy) && isfinite(vz);
    }
    if (solved) {
      Q = qeval(K, f2d(vx), f2d(vy), f2d(vz));
    } else {
      // best of a, b, midpoint by Q; ties keep the earlier candidate
      const float mxp = __double2float_rn(((double)pa.x + (double)pb.x) * 0.5);
      const float myp = __double2float_rn(((double)pa.y + (double)pb.y) * 0.5);
      const float mzp = __double2float_rn(((double)pa.z + (double)pb.z) * 0.5);
      Q = qeval(K, f2d(pa.x), f2d(pa.y), f2d(pa.z));
      vx = pa.x; vy = pa.y; vz = pa.z;
      const double qb = qeval(K, f2d(pb.x), f2d(pb.y), f2d(pb.z));
      if (qb < Q) { Q = qb; vx = pb.x; vy = pb.y; vz = pb.z; }
      const double qm = qeval(K, f2d(mxp), f2d(myp), f2d(mzp));
      if (qm < Q) { Q = qm; vx = mxp; vy = myp; vz = mzp; }
    }
    // ---- l_ab
    const double dx = f2d(pb.x) - f2d(pa.x), dy = f2d(pb.y) - f2d(pa.y),
                 dz = f2d(pb.z) - f2d(pa.z);
    l = sqrt(dot3(dx, dy, dz, dx, dy, dz));
  }
  // ---- skinny term: faces around a or b, except the two on ab, ascending
  // face id (merge of the two sorted incidence lists)
  int incl = nt;  // warp prefix of the produced-triangle counts
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  const int T = __shfl_sync(0xffffffffu, incl, 31);
  const int o = incl - nt;
  const double vxd = f2d(vx), vyd = f2d(vy), vzd = f2d(vz);
  const double Tq = __fma_rn(wes, l, s2 * Q);  // the cost without its skinny term
  double Cs = 0.0;                             // the skinny sum in float64
  uint32_t cb = 0xffffffffu;                   // key bits (non-finite: never eligible)
  bool f64 = true;                             // the key comes from Cs
  if (T <= kFlatCap) {  // warp-uniform
    if (live) {
      S.a[lane] = a;
      S.b[lane] = b;
      S.vx[lane] = vx;
      S.vy[lane] = vy;
      S.vz[lane] = vz;
      int i = a0, j = b0, k = o;
      while (i < a1 || j < b1) {
        const int fi = i < a1 ? idx[i] : 0x7fffffff;
        const int fj = j < b1 ? idx[j] : 0x7fffffff;
        if (fi == fj) {  // a face on edge ab: deleted by the collapse
          i++;
          j++;
          continue;
        }
        S.face[k] = fi < fj ? fi : fj;
        S.own[k] = (unsigned char)lane;
        k++;
        if (fi < fj) i++;
        else j++;
      }
    }
    __syncwarp();
    for (int s = lane; s < T; s += 32) {
      const int L = S.own[s];
      S.tf[s] = skinny_term_ff(F[S.face[s]], S.a[L], S.b[L], S.vx[L], S.vy[L], S.vz[L], pos);
    }
    __syncwarp();
    if (live) {
      // The lane's sum in float-float.  Its distance from the float64 sum Cs
      // (terms within kTriBound each; both sums' roundings, at most
      // 3.02 u^2 and 2^-53 of the running magnitude per addition) is below
      // B = nt (kTriBound + 3.2 u^2 sum|t|), all rounded upwards.
      ff::FF cs = {0.f, 0.f};
      float A = 0.f;
      for (int k = 0; k < nt; k++) {
        const float2 t = S.tf[o + k];
        cs = ff::add(cs, {t.x, t.y});
        A = __fadd_ru(A, fabsf(t.x));
      }
      A = __fmul_ru(A, 1.0f + 0x1p-22f);
      const float B = __fmul_ru((float)nt, __fmaf_ru(0x1.99999ap-47f, A, ff::kTriBound));
      // Cs lies in [lo, hi]; x -> fl(w_s x + Tq) and key_bits are monotone, so
      // equal keys at both ends are the key of the float64 evaluation
      const double h = f2d(cs.h), hl = f2d(cs.l), Bd = f2d(B);
      const double lo = __dsub_rd(__dadd_rd(h, hl), Bd);
      const double hi = __dadd_ru(__dadd_ru(h, hl), Bd);
      const uint32_t k0 = key_bits(__fma_rn(ws, ws >= 0.0 ? lo : hi, Tq));
      const uint32_t k1 = key_bits(__fma_rn(ws, ws >= 0.0 ? hi : lo, Tq));
      if (k0 == k1 && k0 != 0xffffffffu) {
        cb = k0;
        f64 = false;
      }
    }
    // edges the bound leaves open: their triangles in float64, compacted over
    // the warp, each lane's terms then summed in order as before
    const bool redo = live && f64;
    if (__ballot_sync(0xffffffffu, redo)) {
      const int rn = redo ? nt : 0;
      int rinc = rn;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, rinc, d);
        if (lane >= d) rinc += y;
      }
      const int RT = __shfl_sync(0xffffffffu, rinc, 31);
      const int ro = rinc - rn;
      for (int k = 0; k < rn; k++) S.slot[ro + k] = (short)(o + k);
      __syncwarp();
      for (int s = lane; s < RT; s += 32) {
        const int sl = S.slot[s];
        const int L = S.own[sl];
        S.t[sl] = skinny_term(F[S.face[sl]], S.a[L], S.b[L], f2d(S.vx[L]), f2d(S.vy[L]),
                              f2d(S.vz[L]), pos);
      }
      __syncwarp();
      if (redo)
        for (int k = 0; k < nt; k++) Cs = Cs + S.t[o + k];
    }
    __syncwarp();  // the next iteration overwrites the warp's slots
  } else if (live) {
    int i = a0, j = b0;
    while (i < a1 || j < b1) {
      const int fi = i < a1 ? idx[i] : 0x7fffffff;
      const int fj = j < b1 ? idx[j] : 0x7fffffff;
      if (fi == fj) {
        i++;
        j++;
        continue;
      }
      int f;
      if (fi < fj) { f = fi; i++; }
      else { f = fj; j++; }
      Cs = Cs + skinny_term(F[f], a, b, vxd, vyd, vzd, pos);
    }
  }
  if (live) {
    ntri += nt;
    if (f64) {
      cb = key_bits(__fma_rn(ws, Cs, Tq));
      nf64++;
    }
    unsigned long long k = ~0ull;
    if (cb != 0xffffffffu && cb <= max_bits && link_ok && !flag && (!vmesh || mactive[m])) {
      k = ((unsigned long long)cb << 32) | (unsigned long long)(uint32_t)e;
      eligible++;
      counted = m;
    }
    key[e] = k;
    cbits[e] = cb;
    link[e] = link_ok ? 1 : 0;
    vbar[e] = make_float4(vx, vy, vz, 0.0f);
    link_bad += !link_ok;
    flagged += flag;
  }
  if (vmesh) count_by_mesh(counted, melig);
  }
  // block totals of the round counters
  link_bad = __reduce_add_sync(0xffffffffu, link_bad);
  flagged = __reduce_add_sync(0xffffffffu, flagged);
  eligible = __reduce_add_sync(0xffffffffu, eligible);
  ntri = __reduce_add_sync(0xffffffffu, ntri);
  nf64 = __reduce_add_sync(0xffffffffu, nf64);
  if ((threadIdx.x & 31) == 0) {
    if (ntri) atomicAdd(&dc->cost_tris, (unsigned long long)ntri);
    if (nf64) atomicAdd(&dc->cost_f64, nf64);
    if (link_bad) atomicAdd(&dc->link_rejects, (unsigned long long)link_bad);
    if (flagged) atomicAdd(&dc->flagged, (unsigned long long)flagged);
    if (eligible) atomicAdd(&dc->eligible, (unsigned long long)eligible);
  }
}

// Verification support: both evaluations of 1 - C_ijk for given triangles
__global__ void k_skinny_terms(const float* __restrict__ tri, int64_t n, double* __restrict__ t64,
                               float2* __restrict__ tff) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* p = tri + 9 * i;
    t64[i] = 1.0 - quality(f2d(p[0]), f2d(p[1]), f2d(p[2]), f2d(p[3]), f2d(p[4]), f2d(p[5]),
                           f2d(p[6]), f2d(p[7]), f2d(p[8]));
    tff[i] = ff::skinny_term_ff(p[0], p[1], p[2], p[3], p[4], p[5], p[6], p[7], p[8]);
  }
}

}  // namespace

pamo_status edge_costs(pamo_ctx* c) {
  const double s2 = c->scale * c->scale, wes = c->opt.w_e * c->scale;
  const bool batch = c->n_mesh > 1;
  static const int g_reuse = occ_grid(k_edge_reuse);
  static const int g_cost = occ_grid(k_edge_cost, kItemBlock);
  k_edge_reuse<<<g_reuse, kBlock, 0, c->st>>>(c->E, c->vdirty, c->ivmap, c->E_prev, c->e_off_prev,
                                        c->cbits_prev, c->vbar_prev, c->link_prev, c->flags,
                                        c->key, c->vbar, c->cbits, c->link, c->dlist, c->dc,
                                        batch ? c->vmesh : nullptr, c->mactive, c->mcount,
                                        c->vkey); note_launch();
  k_edge_cost<<<g_cost, kItemBlock, 0, c->st>>>(c->dlist, c->E, c->pos, c->K, c->F, c->vf_off, c->vf_idx,
                                       c->vf_nbr, c->flags, s2, wes, c->opt.w_s, c->key, c->vbar, c->cbits,
                                       c->link, c->dc, batch ? c->vmesh : nullptr, c->mcost,
                                       c->mactive, c->mcount); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo

extern "C" pamo_status pamo_skinny_terms(const float* d_tri, int64_t n, double* d_t64,
                                         float* d_tff, void* stream) {
  if (n < 0 || (n > 0 && (!d_tri || !d_t64 || !d_tff))) {
    pamo::set_error("pamo_skinny_terms: n >= 0 and three device arrays required");
    return PAMO_EINVAL;
  }
  if (n == 0) return PAMO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t blocks = (n + pamo::kBlock - 1) / pamo::kBlock;
  pamo::k_skinny_terms<<<(int)(blocks < 4096 ? blocks : 4096), pamo::kBlock, 0, st>>>(
      d_tri, n, d_t64, reinterpret_cast<float2*>(d_tff));
  pamo::note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}
