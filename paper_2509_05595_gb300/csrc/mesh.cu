// Mesh-level passes of a simplification round: input validation, the
// vertex -> incident-face adjacency (ascending face id), the canonical edge
// list (sorted unique (a<b) pairs; an edge's id is its rank, which is the
// tie-breaking id of the 64-bit key in Section 5.1), the initial vertex
// quadrics (Garland-Heckbert planes, summed in ascending face order), and the
// stable compaction that commits a round.
//
// Per-round kernels take their element counts from the device state block
// (so a round can be replayed as a CUDA graph) and loop grid-stride over a
// fixed grid; the commit kernels are gated by the "clean" result of the last
// intersection check.
#include <cstring>
#include <vector>

#include "common.cuh"

namespace pamo {

namespace {

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

// bad (nullable): set to 1 when a face index lies outside [0, nV)
__global__ void k_load(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ Fi,
                       int64_t nF, float4* __restrict__ pos, int4* __restrict__ F,
                       int* __restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nV) pos[i] = make_float4(V[3 * i], V[3 * i + 1], V[3 * i + 2], 0.0f);
  if (i < nF) {
    const int a = Fi[3 * i], b = Fi[3 * i + 1], c = Fi[3 * i + 2];
    if (bad && (a < 0 || b < 0 || c < 0 || a >= nV || b >= nV || c >= nV)) atomicOr(bad, 1);
    F[i] = make_int4(a, b, c, 0);
  }
}

__global__ void k_store(const float4* __restrict__ pos, int64_t nV, const int4* __restrict__ F,
                        int64_t nF, float* __restrict__ V, int32_t* __restrict__ Fo) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nV) {
    float4 p = pos[i];
    V[3 * i] = p.x;
    V[3 * i + 1] = p.y;
    V[3 * i + 2] = p.z;
  }
  if (i < nF) {
    int4 f = F[i];
    Fo[3 * i] = f.x;
    Fo[3 * i + 1] = f.y;
    Fo[3 * i + 2] = f.z;
  }
}

__device__ __forceinline__ unsigned fkey(float x) {  // order-preserving
  unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_bbox(const float4* __restrict__ pos, int64_t nV, unsigned* __restrict__ out) {
  unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nV;
       i += (int64_t)gridDim.x * blockDim.x) {
    float4 p = pos[i];
    float c[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
      unsigned u = fkey(c[k]);
      lo[k] = min(lo[k], u);
      hi[k] = max(hi[k], u);
    }
  }
#pragma unroll
  for (int k = 0; k < 3; k++) {
    lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
    hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
  }
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      atomicMin(&out[k], lo[k]);
      atomicMax(&out[3 + k], hi[k]);
    }
  }
}

// ---- batches: many meshes handled as one disjoint union --------------------
// The vertices (faces) of mesh m are [off[m], off[m+1]) of the union; the
// input faces of a mesh index its own vertices from 0.
__device__ __forceinline__ int seg_of(const int64_t* __restrict__ off, int M, int64_t i) {
  int lo = 0, hi = M - 1;  // the last m with off[m] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_load_batch(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ Fi,
                             int64_t nF, const int64_t* __restrict__ voff,
                             const int64_t* __restrict__ foff, int M, float4* __restrict__ pos,
                             int4* __restrict__ F, int32_t* __restrict__ vmesh,
                             int* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nV) {
    pos[i] = make_float4(V[3 * i], V[3 * i + 1], V[3 * i + 2], 0.0f);
    vmesh[i] = seg_of(voff, M, i);
  }
  if (i < nF) {
    const int m = seg_of(foff, M, i);
    const int64_t base = voff[m], nv = voff[m + 1] - base;
    int c[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const int32_t x = Fi[3 * i + k];
      if (x < 0 || x >= nv) {
        atomicOr(bad, 1);
        c[k] = (int)base;  // stays inside the mesh; the call fails with EINVAL
      } else {
        c[k] = (int)(base + x);
      }
    }
    F[i] = make_int4(c[0], c[1], c[2], 0);
  }
}

// bounding box of each mesh: one block per mesh, order-preserving encodings
__global__ void k_mesh_bbox(const float4* __restrict__ pos, const int64_t* __restrict__ voff,
                            unsigned* __restrict__ out) {
  __shared__ unsigned red[6][kBlock / 32];
  const int m = blockIdx.x;
  unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0, 0, 0};
  for (int64_t i = voff[m] + threadIdx.x; i < voff[m + 1]; i += blockDim.x) {
    const float4 p = pos[i];
    const float c[3] = {p.x, p.y, p.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const unsigned u = fkey(c[k]);
      lo[k] = min(lo[k], u);
      hi[k] = max(hi[k], u);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; k++) {
    lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
    hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
    if (lane == 0) {
      red[k][wid] = lo[k];
      red[3 + k][wid] = hi[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    unsigned r = red[k][0];
    for (int w = 1; w < kBlock / 32; w++) r = k < 3 ? min(r, red[k][w]) : max(r, red[k][w]);
    out[6 * m + k] = r;
  }
}

// output faces in each mesh's own vertex numbering
__global__ void k_store_batch(const float4* __restrict__ pos, int64_t nV,
                              const int4* __restrict__ F, int64_t nF,
                              const int32_t* __restrict__ vmesh, const int32_t* __restrict__ vbase,
                              float* __restrict__ V, int32_t* __restrict__ Fo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nV) {
    const float4 p = pos[i];
    V[3 * i] = p.x;
    V[3 * i + 1] = p.y;
    V[3 * i + 2] = p.z;
  }
  if (i < nF) {
    const int4 f = F[i];
    const int b = vbase[vmesh[f.x]];
    Fo[3 * i] = f.x - b;
    Fo[3 * i + 1] = f.y - b;
    Fo[3 * i + 2] = f.z - b;
  }
}

// last round's flags in the committed numbering (~0 where a vertex died); in a
// batch the flags of meshes that committed nothing carry over, and the
// vertices of other meshes may have moved
__global__ void k_remap_flags(const unsigned long long* __restrict__ flags,
                              const RoundCounters* __restrict__ dc,
                              const int32_t* __restrict__ vmap,
                              unsigned long long* __restrict__ out) {
  if (!dc->go) return;
  const int n = dc->nflags;
  GRID_STRIDE(i, n) {
    const unsigned long long p = flags[i];
    const int a = vmap[(int)(p >> 32)], b = vmap[(int)(p & 0xffffffffu)];
    out[i] = (a < 0 || b < 0) ? ~0ull
                              : ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
  }
}

// ---- validation (eager, host sizes) ---------------------------------------
__global__ void k_check_faces(const int4* __restrict__ F, int64_t nF, int64_t nV,
                              const float4* __restrict__ pos, int* __restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nF) {
    int4 f = F[i];
    if (f.x < 0 || f.y < 0 || f.z < 0 || f.x >= nV || f.y >= nV || f.z >= nV) atomicOr(bad, 1);
    else if (f.x == f.y || f.y == f.z || f.z == f.x) atomicOr(bad, 2);
  }
  if (i < nV) {
    float4 p = pos[i];
    if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) atomicOr(bad, 4);
  }
}

// closed, oriented, edge- and vertex-manifold around every vertex:
// the "next" neighbours (x of faces (u,x,y)) are distinct, the "previous"
// neighbours (y) are distinct and equal as sets (every u->x has x->u), and the
// link map x -> y is one cycle.
__global__ void k_check_vertices(const int4* __restrict__ F, const int32_t* __restrict__ off,
                                 const int32_t* __restrict__ idx, int64_t nV,
                                 int* __restrict__ bad) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nV) return;
  const int b = off[v], e = off[v + 1];
  const int deg = e - b;
  if (deg < 3) {
    atomicOr(bad, 8);
    return;
  }
  for (int s = b; s < e; s++) {
    int4 f = F[idx[s]];
    int x, y;
    if (f.x == v) { x = f.y; y = f.z; }
    else if (f.y == v) { x = f.z; y = f.x; }
    else { x = f.x; y = f.y; }
    int nx = 0, ny = 0, ysx = 0;
    for (int t = b; t < e; t++) {
      int4 g = F[idx[t]];
      int gx, gy;
      if (g.x == v) { gx = g.y; gy = g.z; }
      else if (g.y == v) { gx = g.z; gy = g.x; }
      else { gx = g.x; gy = g.y; }
      nx += gx == x;
      ny += gy == y;
      ysx += gy == x;
    }
    if (nx != 1 || ny != 1 || ysx != 1) {
      atomicOr(bad, 16);
      return;
    }
  }
  // walk the link from the first face
  int4 f0 = F[idx[b]];
  int start = f0.x == v ? f0.y : (f0.y == v ? f0.z : f0.x);
  int cur = start, steps = 0;
  do {
    int nxt = -1;
    for (int t = b; t < e; t++) {
      int4 g = F[idx[t]];
      int gx, gy;
      if (g.x == v) { gx = g.y; gy = g.z; }
      else if (g.y == v) { gx = g.z; gy = g.x; }
      else { gx = g.x; gy = g.y; }
      if (gx == cur) { nxt = gy; break; }
    }
    cur = nxt;
    steps++;
  } while (cur != start && cur >= 0 && steps <= deg);
  if (steps != deg || cur != start) atomicOr(bad, 32);
}

// ---- vertex -> faces ------------------------------------------------------
__global__ void k_count_corners(const int4* __restrict__ F, const int* nF_dev, int nF_host,
                                int32_t* __restrict__ cnt) {
  const int n = dev_n(nF_dev, nF_host);
  GRID_STRIDE(f, n) {
    const int4 t = F[f];
    atomicAdd(&cnt[t.x], 1);
    atomicAdd(&cnt[t.y], 1);
    atomicAdd(&cnt[t.z], 1);
  }
}

// each corner takes a slot of its vertex's segment by counting the vertex's
// corner count down to zero (slot order is arbitrary: the segments are sorted
// next), which leaves the counts zeroed
__global__ void k_fill_corners(const int4* __restrict__ F, const int* nF_dev, int nF_host,
                               const int32_t* __restrict__ off, int32_t* __restrict__ cnt,
                               int32_t* __restrict__ idx) {
  const int n = dev_n(nF_dev, nF_host);
  GRID_STRIDE(f, n) {
    const int4 t = F[f];
    idx[off[t.x] + atomicSub(&cnt[t.x], 1) - 1] = (int32_t)f;
    idx[off[t.y] + atomicSub(&cnt[t.y], 1) - 1] = (int32_t)f;
    idx[off[t.z] + atomicSub(&cnt[t.z], 1) - 1] = (int32_t)f;
  }
}

__device__ __forceinline__ int next_after(const int4& f, int v) {
  return f.x == v ? f.y : (f.y == v ? f.z : f.x);
}

// insertion sort of each vertex's incident faces (typically 4..10 entries)
__global__ void k_sort_segments(const int32_t* __restrict__ off, const int* nV_dev, int nV_host,
                                int32_t* __restrict__ idx) {
  const int nV = dev_n(nV_dev, nV_host);
  GRID_STRIDE(v, nV) {
    const int b = off[v], e = off[v + 1];
    if (e - b <= 16) {
      int a[16];
      const int n = e - b;
      for (int i = 0; i < n; i++) {
        const int x = idx[b + i];
        int j = i;
        while (j > 0 && a[j - 1] > x) {
          a[j] = a[j - 1];
          j--;
        }
        a[j] = x;
      }
      for (int i = 0; i < n; i++) idx[b + i] = a[i];
    } else {
      for (int i = b + 1; i < e; i++) {
        const int x = idx[i];
        int j = i;
        while (j > b && idx[j - 1] > x) {
          idx[j] = idx[j - 1];
          j--;
        }
        idx[j] = x;
      }
    }
  }
}

// The same sort, and each vertex's neighbour multiset: the corner after v in
// each incident face, in ascending order, in v's segment of nbr (on a closed
// manifold mesh these are v's distinct neighbours).  cnt[v] = how many exceed
// v: the last cnt[v] entries are v's edges to higher-numbered neighbours.
__global__ void k_sort_segments_nbr(const int4* __restrict__ F, const int32_t* __restrict__ off,
                                    const int* nV_dev, int32_t* __restrict__ idx,
                                    int32_t* __restrict__ nbr, int32_t* __restrict__ cnt) {
  const int nV = *nV_dev;
  GRID_STRIDE(v, nV) {
    const int b = off[v], e = off[v + 1];
    int m = 0;
    if (e - b <= 16) {
      int a[16], x[16];
      const int n = e - b;
      for (int i = 0; i < n; i++) {
        const int y = idx[b + i];
        int j = i;
        while (j > 0 && a[j - 1] > y) {
          a[j] = a[j - 1];
          j--;
        }
        a[j] = y;
      }
      for (int i = 0; i < n; i++) {
        idx[b + i] = a[i];
        const int y = next_after(F[a[i]], (int)v);
        m += y > v;
        int j = i;
        while (j > 0 && x[j - 1] > y) {
          x[j] = x[j - 1];
          j--;
        }
        x[j] = y;
      }
      for (int i = 0; i < n; i++) nbr[b + i] = x[i];
    } else {
      for (int i = b + 1; i < e; i++) {
        const int y = idx[i];
        int j = i;
        while (j > b && idx[j - 1] > y) {
          idx[j] = idx[j - 1];
          j--;
        }
        idx[j] = y;
      }
      for (int i = b; i < e; i++) {
        const int y = next_after(F[idx[i]], (int)v);
        m += y > v;
        int j = i;
        while (j > b && nbr[j - 1] > y) {
          nbr[j] = nbr[j - 1];
          j--;
        }
        nbr[j] = y;
      }
    }
    cnt[v] = m;
  }
}

// ---- edges ----------------------------------------------------------------

// the edge count; a closed triangle mesh has exactly 3F/2 edges, anything
// else means a non-manifold mesh (the host reports it at the next sync)
__device__ __forceinline__ void edge_total(const int32_t* __restrict__ eoff,
                                           RoundCounters* __restrict__ dc, int64_t cap) {
  const int ne = eoff[dc->nV];
  dc->ne_actual = ne;
  dc->nV_edges = dc->nV;
  const int want = (3 * dc->nF) / 2;
  if (ne != want || ne > cap) dc->bad |= 64;
  dc->nE = ne <= cap ? ne : (int)cap;
}

// Each vertex copies its sorted edges to higher-numbered neighbours (the last
// cnt[v] entries of its neighbour segment, from k_sort_segments_nbr) to its
// offset; the per-vertex counts are zeroed for the
// next corner count (the next round's vertices are a prefix of these), and
// one thread sets the edge total (only the counters read it before the next
// kernel).
__global__ void k_write_edges(const int32_t* __restrict__ off, const int32_t* __restrict__ nbr,
                              RoundCounters* __restrict__ dc, const int32_t* __restrict__ eoff,
                              int64_t cap, int2* __restrict__ E, int32_t* __restrict__ cnt) {
  const int nV = dc->nV;
  if (blockIdx.x == 0 && threadIdx.x == 0) edge_total(eoff, dc, cap);
  GRID_STRIDE(v, nV) {
    const int m = cnt[v];
    cnt[v] = 0;
    const int base = eoff[v], b = off[v + 1] - m;
    for (int k = 0; k < m && base + k < cap; k++) E[base + k] = make_int2((int)v, nbr[b + k]);
  }
}

// start of a round: zero the round's counters (the words after the persistent
// sizes) and make last round's edge data the reuse source of this round's costs
__global__ void k_save_prev(RoundCounters* __restrict__ dc, const int2* __restrict__ E,
                            const int32_t* __restrict__ e_off, const uint32_t* __restrict__ cbits,
                            const float4* __restrict__ vbar, const uint8_t* __restrict__ link,
                            int2* __restrict__ E_prev, int32_t* __restrict__ e_off_prev,
                            uint32_t* __restrict__ cbits_prev, float4* __restrict__ vbar_prev,
                            uint8_t* __restrict__ link_prev, int32_t* __restrict__ mcount,
                            int mcount_n) {
  const int nE = dc->nE, nO = dc->nV_edges + 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) dc->round_no++;  // outside the zeroed words
  GRID_STRIDE(i, mcount_n) mcount[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x < (sizeof(RoundCounters) - PAMO_ROUND_ZERO_OFFSET) / 4)
    reinterpret_cast<int*>(reinterpret_cast<char*>(dc) + PAMO_ROUND_ZERO_OFFSET)[threadIdx.x] = 0;
  GRID_STRIDE(i, nE) {
    E_prev[i] = E[i];
    cbits_prev[i] = cbits[i];
    vbar_prev[i] = vbar[i];
    link_prev[i] = link[i];
  }
  GRID_STRIDE(i, nO) e_off_prev[i] = e_off[i];
}

// ---- quadrics (Garland-Heckbert; Q_ab of Eq. 1) ---------------------------
// plane of a face through its first corner, unit normal; coefficient order
// xx xy xz xd yy yz yd zz zd dd
__global__ void k_face_quadrics(const float4* __restrict__ pos, const int4* __restrict__ F,
                                const int* nF_dev, int64_t nF_host, double* __restrict__ q) {
  const int64_t nF = nF_dev ? (int64_t)*nF_dev : nF_host;
  GRID_STRIDE(f, nF) {
  int4 t = F[f];
  float4 p0 = pos[t.x], p1 = pos[t.y], p2 = pos[t.z];
  double ux = (double)p1.x - (double)p0.x, uy = (double)p1.y - (double)p0.y,
         uz = (double)p1.z - (double)p0.z;
  double vx = (double)p2.x - (double)p0.x, vy = (double)p2.y - (double)p0.y,
         vz = (double)p2.z - (double)p0.z;
  double nx = uy * vz - uz * vy;
  double ny = uz * vx - ux * vz;
  double nz = ux * vy - uy * vx;
  double len = sqrt((nx * nx + ny * ny) + nz * nz);
  double* o = q + 10 * f;
  if (len == 0.0) {
#pragma unroll
    for (int i = 0; i < 10; i++) o[i] = 0.0;
    continue;
  }
  nx = nx / len;
  ny = ny / len;
  nz = nz / len;
  double d = -((nx * (double)p0.x + ny * (double)p0.y) + nz * (double)p0.z);
  o[0] = nx * nx;
  o[1] = nx * ny;
  o[2] = nx * nz;
  o[3] = nx * d;
  o[4] = ny * ny;
  o[5] = ny * nz;
  o[6] = ny * d;
  o[7] = nz * nz;
  o[8] = nz * d;
  o[9] = d * d;
  }
}

__global__ void k_vertex_quadrics(const double* __restrict__ q, const int32_t* __restrict__ off,
                                  const int32_t* __restrict__ idx, const int* nV_dev,
                                  int64_t nV_host, double* __restrict__ K) {
  const int64_t nV = nV_dev ? (int64_t)*nV_dev : nV_host;
  GRID_STRIDE(v, nV) {
  double s[10];
#pragma unroll
  for (int i = 0; i < 10; i++) s[i] = 0.0;
  for (int j = off[v]; j < off[v + 1]; j++) {
    const double* f = q + 10 * (int64_t)idx[j];
#pragma unroll
    for (int i = 0; i < 10; i++) s[i] = s[i] + f[i];
  }
#pragma unroll
  for (int i = 0; i < 10; i++) K[10 * v + i] = s[i];
  }
}

// ---- commit (stable compaction), gated by the last check (the gate sizes
// go/goV/goF/goW are set with the check's outcome) ---------------------------

__global__ void k_compact_vertices(const float4* __restrict__ pos_s, const double* __restrict__ K_s,
                                   const uint8_t* __restrict__ vdead,
                                   const int32_t* __restrict__ dead_before, const int* n_dev,
                                   float4* __restrict__ pos, double* __restrict__ K,
                                   int32_t* __restrict__ vmap, int32_t* __restrict__ ivmap,
                                   const int32_t* __restrict__ vmesh,
                                   int32_t* __restrict__ vmesh_out,
                                   const uint32_t* __restrict__ vgap,
                                   uint32_t* __restrict__ vgap_out) {
  const int nV = *n_dev;
  GRID_STRIDE(v, nV) {
    if (vdead[v]) {
      vmap[v] = -1;
      continue;
    }
    const int64_t n = v - dead_before[v];
    vmap[v] = (int32_t)n;
    ivmap[n] = (int32_t)v;
    pos[n] = pos_s[v];
    if (vmesh) vmesh_out[n] = vmesh[v];
    vgap_out[n] = vgap[v];
    const double2* src = reinterpret_cast<const double2*>(K_s + 10 * v);
    double2* dst = reinterpret_cast<double2*>(K + 10 * n);
#pragma unroll
    for (int i = 0; i < 5; i++) dst[i] = src[i];
  }
}

__global__ void k_compact_faces(const int4* __restrict__ F_s, const uint8_t* __restrict__ fdead,
                                const int32_t* __restrict__ dead_before, const int* n_dev,
                                const int32_t* __restrict__ vmap, int4* __restrict__ F) {
  const int nF = *n_dev;
  GRID_STRIDE(f, nF) {
    if (fdead[f]) continue;
    const int4 t = F_s[f];
    F[f - dead_before[f]] = make_int4(vmap[t.x], vmap[t.y], vmap[t.z], 0);
  }
}

// Undone winners as remapped vertex pairs, in winner (= ascending edge) order,
// which the monotone vertex map keeps sorted; uscan is the exclusive scan of
// the undone marks (total at [nW]).  After a round that committed something
// they are the next round's flags (Section 5.3) and go straight to flags; a
// round without a commit keeps them in flags_next for the host merge.  Also
// sets the committed / undone counts and the sizes of the committed mesh.
__global__ void k_undone_pairs(const int32_t* __restrict__ wlist, const int2* __restrict__ E,
                               const uint8_t* __restrict__ standing, const int32_t* __restrict__ uscan,
                               RoundCounters* __restrict__ dc, const int32_t* __restrict__ vmap,
                               unsigned long long* __restrict__ flags,
                               unsigned long long* __restrict__ flags_next,
                               const int32_t* __restrict__ vmesh, int32_t* __restrict__ mcount,
                               int M) {
  const int nW = dc->goW;  // 0 when the round does not commit
  const int nund = dc->go ? uscan[dc->nW] : 0;
  const int committed = dc->nW - nund;
  // a batch keeps every list apart for the per-mesh merge on the host
  unsigned long long* out = (committed > 0 && !vmesh) ? flags : flags_next;
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nW;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = base + threadIdx.x;
    int m = -1;
    bool st = false;
    if (w < nW) {
      const int2 e = E[wlist[w]];
      st = standing[w] != 0;
      if (!st)
        out[uscan[w]] = ((unsigned long long)(unsigned)vmap[e.x] << 32) | (unsigned)vmap[e.y];
      if (vmesh) m = vmesh[e.x];
    }
    if (vmesh) {  // per-mesh committed / undone counts, one atomic per group of lanes
      const int key = m < 0 ? -1 : (st ? m : M + m);
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (key >= 0 && lane == __ffs(peers) - 1)
        atomicAdd(&mcount[M + key], __popc(peers));  // [M, 2M) committed, [2M, 3M) undone
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (!dc->go) {
      dc->goVn = 0;
      dc->goFn = 0;
    } else {
      dc->nund = nund;
      dc->committed = committed;
      dc->goVn = dc->nV - committed;
      dc->goFn = dc->nF - 2 * committed;
      if (committed > 0 && !vmesh) dc->nflags = nund;
    }
  }
}

// clear two byte arrays over the new vertices, and move the per-vertex words
// that the compaction wrote to scratch (clearance; a batch's vertex -> mesh
// map, when set) back to their arrays
__global__ void k_clear2(uint8_t* __restrict__ a, uint8_t* __restrict__ b, const int* n_dev,
                         uint32_t* __restrict__ w0, const uint32_t* __restrict__ w0_src,
                         int32_t* __restrict__ w1, const int32_t* __restrict__ w1_src) {
  const int n = *n_dev;
  GRID_STRIDE(i, n) {
    a[i] = 0;
    b[i] = 0;
    w0[i] = w0_src[i];
    if (w1) w1[i] = w1_src[i];
  }
}

// survivors of committed collapses (new numbering)
__global__ void k_mark_survivors(const int32_t* __restrict__ wlist, const int2* __restrict__ E,
                                 const uint8_t* __restrict__ standing, const int* n_dev,
                                 const int32_t* __restrict__ vmap, uint8_t* __restrict__ vsurv) {
  const int nW = *n_dev;
  GRID_STRIDE(w, nW) {
    if (standing[w]) vsurv[vmap[E[wlist[w]].x]] = 1;
  }
}

// a vertex is dirty when it is a survivor or shares a face with one
__global__ void k_mark_dirty(const int4* __restrict__ F, const int* n_dev,
                             const uint8_t* __restrict__ vsurv, uint8_t* __restrict__ vdirty) {
  const int nF = *n_dev;
  GRID_STRIDE(f, nF) {
    const int4 t = F[f];
    if (vsurv[t.x] | vsurv[t.y] | vsurv[t.z]) {
      vdirty[t.x] = 1;
      vdirty[t.y] = 1;
      vdirty[t.z] = 1;
    }
  }
}

__global__ void k_commit_sizes(RoundCounters* __restrict__ dc) {
  if (!dc->go) return;
  dc->nV = dc->goVn;
  dc->nF = dc->goFn;
  dc->have_prev = 1;
  dc->last_committed = dc->committed;
}

}  // namespace

pamo_status load_mesh(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF, float4* pos,
                      int4* F, cudaStream_t st) {
  k_load<<<grid_for(nV > nF ? nV : nF), kBlock, 0, st>>>(d_V, nV, d_F, nF, pos, F, nullptr); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status load_mesh_checked(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                              float4* pos, int4* F, int* d_bad, cudaStream_t st) {
  PAMO_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  k_load<<<grid_for(nV > nF ? nV : nF), kBlock, 0, st>>>(d_V, nV, d_F, nF, pos, F, d_bad); note_launch();
  PAMO_CUDA(cudaGetLastError());
  int hb = 0;
  PAMO_CUDA(cudaMemcpyAsync(&hb, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  if (hb) {
    set_error("a face index is outside [0, nV)");
    return PAMO_EINVAL;
  }
  return PAMO_OK;
}

static void decode_bbox(const unsigned out[6], float lo[3], float hi[3]) {
  for (int k = 0; k < 3; k++) {
    unsigned a = out[k], b = out[3 + k];
    a = (a & 0x80000000u) ? (a & 0x7fffffffu) : ~a;
    b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
    std::memcpy(&lo[k], &a, 4);
    std::memcpy(&hi[k], &b, 4);
  }
}

pamo_status load_mesh_batch(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                            const int64_t* d_voff, const int64_t* d_foff, int M, float4* pos,
                            int4* F, int32_t* vmesh, int* d_bad, cudaStream_t st) {
  PAMO_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  k_load_batch<<<grid_for(nV > nF ? nV : nF), kBlock, 0, st>>>(d_V, nV, d_F, nF, d_voff, d_foff, M,
                                                               pos, F, vmesh, d_bad); note_launch();
  PAMO_CUDA(cudaGetLastError());
  int hb = 0;
  PAMO_CUDA(cudaMemcpyAsync(&hb, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  PAMO_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  if (hb) {
    set_error("a face index is outside its mesh's vertex range");
    return PAMO_EINVAL;
  }
  return PAMO_OK;
}

pamo_status mesh_bbox_batch(const float4* pos, const int64_t* d_voff, int M, unsigned* d_out,
                            float* lo, float* hi, cudaStream_t st) {
  k_mesh_bbox<<<M, kBlock, 0, st>>>(pos, d_voff, d_out); note_launch();
  PAMO_CUDA(cudaGetLastError());
  std::vector<unsigned> h(6 * (size_t)M);
  PAMO_CUDA(cudaMemcpyAsync(h.data(), d_out, sizeof(unsigned) * 6 * M, cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  for (int m = 0; m < M; m++) decode_bbox(&h[6 * (size_t)m], lo + 3 * (size_t)m, hi + 3 * (size_t)m);
  return PAMO_OK;
}

pamo_status store_mesh_batch(const float4* pos, int64_t nV, const int4* F, int64_t nF,
                             const int32_t* vmesh, const int32_t* d_vbase, float* d_V,
                             int32_t* d_F, cudaStream_t st) {
  k_store_batch<<<grid_for(nV > nF ? nV : nF), kBlock, 0, st>>>(pos, nV, F, nF, vmesh, d_vbase,
                                                                d_V, d_F); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status store_mesh(const float4* pos, int64_t nV, const int4* F, int64_t nF, float* d_V,
                       int32_t* d_F, cudaStream_t st) {
  k_store<<<grid_for(nV > nF ? nV : nF), kBlock, 0, st>>>(pos, nV, F, nF, d_V, d_F); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}


// mesh_bbox with caller-provided device scratch (6 words); allocates nothing
pamo_status mesh_bbox_into(const float4* pos, int64_t nV, unsigned* d_tmp, float lo[3], float hi[3],
                           cudaStream_t st) {
  unsigned init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0, 0, 0};
  PAMO_CUDA(cudaMemcpyAsync(d_tmp, init, sizeof(init), cudaMemcpyHostToDevice, st));
  unsigned g = grid_for(nV);
  if (g > 1024) g = 1024;
  k_bbox<<<g, kBlock, 0, st>>>(pos, nV, d_tmp); note_launch();
  PAMO_CUDA(cudaGetLastError());
  unsigned out[6];
  PAMO_CUDA(cudaMemcpyAsync(out, d_tmp, sizeof(out), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  decode_bbox(out, lo, hi);
  return PAMO_OK;
}

pamo_status mesh_bbox(const float4* pos, int64_t nV, float lo[3], float hi[3], Buf& tmp,
                      cudaStream_t st) {
  PAMO_TRY(buf_reserve(tmp, 64, st));
  return mesh_bbox_into(pos, nV, (unsigned*)tmp.p, lo, hi, st);
}

// vertex -> incident faces of the current mesh (device sizes); with
// neighbours, also each vertex's sorted higher-numbered neighbours and their
// counts in vcount, which build_edges must consume next
pamo_status build_vertex_faces(pamo_ctx* c, bool neighbours) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  const int G = c->grid;
  // vcount is zero here: zeroed at allocation, after each use as fill
  // cursors below, and by k_write_edges after its use as edge counts (the
  // neighbour sort writes those counts only when build_edges follows)
  k_count_corners<<<G, kBlock, 0, st>>>(c->F, &dc->nF, 0, c->vcount); note_launch();
  PAMO_TRY(scan_dev_i32(c->vcount, &dc->nV, c->vf_off, c->scan_sums, G, st));
  static const int g_fill = occ_grid(k_fill_corners);
  static const int g_sort = occ_grid(k_sort_segments);
  static const int g_nbr = occ_grid(k_sort_segments_nbr);
  k_fill_corners<<<g_fill, kBlock, 0, st>>>(c->F, &dc->nF, 0, c->vf_off, c->vcount, c->vf_idx); note_launch();
  if (neighbours) {
    k_sort_segments_nbr<<<g_nbr, kBlock, 0, st>>>(c->F, c->vf_off, &dc->nV, c->vf_idx, c->vf_nbr,
                                                  c->vcount); note_launch();
  } else {
    k_sort_segments<<<g_sort, kBlock, 0, st>>>(c->vf_off, &dc->nV, 0, c->vf_idx); note_launch();
  }
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status validate_mesh(pamo_ctx* c) {
  cudaStream_t st = c->st;
  int* bad = &c->dc->bad;
  PAMO_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  int64_t n = c->nV > c->nF ? c->nV : c->nF;
  k_check_faces<<<grid_for(n), kBlock, 0, st>>>(c->F, c->nF, c->nV, c->pos, bad); note_launch();
  PAMO_CUDA(cudaGetLastError());
  int hb = 0;
  PAMO_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  if (hb & 1) { set_error("face index out of range"); return PAMO_EINVAL; }
  if (hb & 2) { set_error("face with a repeated corner"); return PAMO_ENOTMANIFOLD; }
  if (hb & 4) { set_error("non-finite vertex coordinate"); return PAMO_EINVAL; }
  PAMO_TRY(build_vertex_faces(c, false));
  k_check_vertices<<<grid_for(c->nV), kBlock, 0, st>>>(c->F, c->vf_off, c->vf_idx, c->nV, bad); note_launch();
  PAMO_CUDA(cudaGetLastError());
  PAMO_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  PAMO_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  if (hb & 8) { set_error("vertex with fewer than 3 incident faces (isolated or open)"); return PAMO_ENOTMANIFOLD; }
  if (hb & 16) { set_error("mesh is not closed, oriented and edge-manifold"); return PAMO_ENOTMANIFOLD; }
  if (hb & 32) { set_error("a vertex link is not a single cycle"); return PAMO_ENOTMANIFOLD; }
  return PAMO_OK;
}

pamo_status save_prev(pamo_ctx* c) {
  k_save_prev<<<c->grid, kBlock, 0, c->st>>>(c->dc, c->E, c->e_off, c->cbits, c->vbar, c->link,
                                             c->E_prev, c->e_off_prev, c->cbits_prev, c->vbar_prev,
                                             c->link_prev, c->mcount,
                                             c->n_mesh > 1 ? 3 * c->n_mesh : 0); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

// canonical edge list of the current mesh (device sizes); sets dc->nE.
// Follows build_vertex_faces(c, true), whose neighbour lists it copies.
pamo_status build_edges(pamo_ctx* c) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  const int G = c->grid;
  static const int g_write = occ_grid(k_write_edges);
  PAMO_TRY(scan_dev_i32(c->vcount, &dc->nV, c->e_off, c->scan_sums, G, st));
  k_write_edges<<<g_write, kBlock, 0, st>>>(c->vf_off, c->vf_nbr, dc, c->e_off, c->Emax, c->E,
                                            c->vcount); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status init_quadrics(pamo_ctx* c) {
  cudaStream_t st = c->st;
  PAMO_TRY(buf_reserve(c->quad_tmp, sizeof(double) * 10 * (size_t)c->nF, st));
  double* q = (double*)c->quad_tmp.p;
  k_face_quadrics<<<grid_for(c->nF), kBlock, 0, st>>>(c->pos, c->F, nullptr, c->nF, q); note_launch();
  k_vertex_quadrics<<<grid_for(c->nV), kBlock, 0, st>>>(q, c->vf_off, c->vf_idx, nullptr, c->nV,
                                                        c->K); note_launch();
  PAMO_CUDA(cudaGetLastError());
  buf_free(c->quad_tmp, st);
  return PAMO_OK;
}

// the option recompute_quadrics: vertex quadrics of M_1 from its current faces
// (device sizes, every round, before the costs)
pamo_status recompute_quadrics(pamo_ctx* c) {
  cudaStream_t st = c->st;
  k_face_quadrics<<<c->grid, kBlock, 0, st>>>(c->pos, c->F, &c->dc->nF, 0, c->qface); note_launch();
  k_vertex_quadrics<<<c->grid, kBlock, 0, st>>>(c->qface, c->vf_off, c->vf_idx, &c->dc->nV, 0,
                                                c->K); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

// Commit M_s as the next M_1 when the last check was clean (device gate):
// stable compaction, undone pairs, flags, dirty vertices.  The new sizes
// become current in commit_sizes.
pamo_status commit_compact(pamo_ctx* c) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  const int G = c->grid;
  // the commit's independent scans in one set of launches: dead vertices and
  // dead faces before each (new id = old id - dead before it), undone winners
  // (next round's flags), and the live leaves of the LBVH order
  {
    ScanSeg seg[4];
    int ns = 0;
    seg[ns++] = ScanSeg{c->vdead, nullptr, &dc->goV, c->dbuf, c->scan_sums, 0};
    seg[ns++] = ScanSeg{c->fdead, nullptr, &dc->goF, c->dbufF, c->scan_sums2, 0};
    seg[ns++] = ScanSeg{c->standing, nullptr, &dc->goW, c->wscan, c->scan_sums2 + c->scan_span, 1};
    if (c->opt.check_mode != 3)
      seg[ns++] = ScanSeg{c->fdead, (const int32_t*)c->bvh.vals.p, &dc->goF,
                          (int32_t*)c->bvh.posn.p, c->scan_sums2 + 2 * c->scan_span, 1};
    PAMO_TRY(scan_dev_u8_multi(seg, ns, G, st));
  }
  const bool batch = c->n_mesh > 1;
  k_compact_vertices<<<G, kBlock, 0, st>>>(c->pos_s, c->K_s, c->vdead, c->dbuf, &dc->goV, c->pos,
                                           c->K, c->vmap, c->ivmap, batch ? c->vmesh : nullptr,
                                           c->vmesh_tmp, c->vgap, c->vgap_tmp); note_launch();
  // faces, corners remapped
  k_compact_faces<<<G, kBlock, 0, st>>>(c->F_s, c->fdead, c->dbufF, &dc->goF, c->vmap, c->F); note_launch();
  // undone winners -> next round's flag candidates (sorted vertex pairs)
  k_undone_pairs<<<G, kBlock, 0, st>>>(c->wlist, c->E, c->standing, c->wscan, dc, c->vmap, c->flags,
                                       c->flags_next, batch ? c->vmesh : nullptr, c->mcount,
                                       c->n_mesh); note_launch();
  if (batch) {  // goVn is set by k_undone_pairs
    k_remap_flags<<<G, kBlock, 0, st>>>(c->flags, dc, c->vmap, c->flags_old); note_launch();
  }
  // dirty vertices of the next round (survivors and their neighbours); the
  // compacted clearance (and vertex -> mesh map) back from scratch
  k_clear2<<<G, kBlock, 0, st>>>(c->vsurv, c->vdirty, &dc->goVn, c->vgap, c->vgap_tmp,
                                 batch ? c->vmesh : nullptr, c->vmesh_tmp); note_launch();
  k_mark_survivors<<<G, kBlock, 0, st>>>(c->wlist, c->E, c->standing, &dc->goW, c->vmap, c->vsurv); note_launch();
  k_mark_dirty<<<G, kBlock, 0, st>>>(c->F, &dc->goFn, c->vsurv, c->vdirty); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

// the new sizes become current (after everything that still needs the old ones)
pamo_status commit_sizes(pamo_ctx* c) {
  k_commit_sizes<<<1, 1, 0, c->st>>>(c->dc); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo
