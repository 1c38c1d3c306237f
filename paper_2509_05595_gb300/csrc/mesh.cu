// Mesh-level passes of a simplification round: input validation, the
// vertex -> incident-face adjacency (ascending face id), the canonical edge
// list (sorted unique (a<b) pairs; an edge's id is its rank, which is the
// tie-breaking id of the 64-bit key in Section 5.1), the initial vertex
// quadrics (Garland-Heckbert planes, summed in ascending face order), and the
// stable compaction that commits a round.
#include <cstring>

#include "common.cuh"

namespace pamo {

namespace {

__global__ void k_load(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ Fi,
                       int64_t nF, float4* __restrict__ pos, int4* __restrict__ F) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nV) pos[i] = make_float4(V[3 * i], V[3 * i + 1], V[3 * i + 2], 0.0f);
  if (i < nF) F[i] = make_int4(Fi[3 * i], Fi[3 * i + 1], Fi[3 * i + 2], 0);
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

// ---- validation -----------------------------------------------------------
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
__global__ void k_count_corners(const int4* __restrict__ F, int64_t nF, int32_t* __restrict__ cnt) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nF) return;
  int4 t = F[f];
  atomicAdd(&cnt[t.x], 1);
  atomicAdd(&cnt[t.y], 1);
  atomicAdd(&cnt[t.z], 1);
}

__global__ void k_fill_corners(const int4* __restrict__ F, int64_t nF,
                               const int32_t* __restrict__ off, int32_t* __restrict__ cur,
                               int32_t* __restrict__ idx) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nF) return;
  int4 t = F[f];
  idx[off[t.x] + atomicAdd(&cur[t.x], 1)] = (int32_t)f;
  idx[off[t.y] + atomicAdd(&cur[t.y], 1)] = (int32_t)f;
  idx[off[t.z] + atomicAdd(&cur[t.z], 1)] = (int32_t)f;
}

// insertion sort of each vertex's incident faces (typically 4..10 entries)
__global__ void k_sort_segments(const int32_t* __restrict__ off, int64_t nV,
                                int32_t* __restrict__ idx) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nV) return;
  const int b = off[v], e = off[v + 1];
  if (e - b <= 16) {
    int a[16];
    int n = e - b;
    for (int i = 0; i < n; i++) {
      int x = idx[b + i];
      int j = i;
      while (j > 0 && a[j - 1] > x) {
        a[j] = a[j - 1];
        j--;
      }
      a[j] = x;
    }
    for (int i = 0; i < n; i++) idx[b + i] = a[i];
    return;
  }
  for (int i = b + 1; i < e; i++) {
    int x = idx[i];
    int j = i;
    while (j > b && idx[j - 1] > x) {
      idx[j] = idx[j - 1];
      j--;
    }
    idx[j] = x;
  }
}

// ---- edges ----------------------------------------------------------------
__device__ __forceinline__ int next_after(const int4& f, int v) {
  return f.x == v ? f.y : (f.y == v ? f.z : f.x);
}

__global__ void k_count_edges(const int4* __restrict__ F, const int32_t* __restrict__ off,
                              const int32_t* __restrict__ idx, int64_t nV,
                              int32_t* __restrict__ cnt) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nV) return;
  int c = 0;
  for (int s = off[v]; s < off[v + 1]; s++) c += next_after(F[idx[s]], (int)v) > v;
  cnt[v] = c;
}

__global__ void k_write_edges(const int4* __restrict__ F, const int32_t* __restrict__ off,
                              const int32_t* __restrict__ idx, int64_t nV,
                              const int32_t* __restrict__ eoff, int2* __restrict__ E) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nV) return;
  const int base = eoff[v];
  int n = 0;
  for (int s = off[v]; s < off[v + 1]; s++) {
    int x = next_after(F[idx[s]], (int)v);
    if (x <= v) continue;
    // insertion into the sorted run E[base .. base+n)
    int j = n;
    while (j > 0 && E[base + j - 1].y > x) {
      E[base + j] = E[base + j - 1];
      j--;
    }
    E[base + j] = make_int2((int)v, x);
    n++;
  }
}

// ---- quadrics (Garland-Heckbert; Q_ab of Eq. 1) ---------------------------
// plane of a face through its first corner, unit normal; coefficient order
// xx xy xz xd yy yz yd zz zd dd
__global__ void k_face_quadrics(const float4* __restrict__ pos, const int4* __restrict__ F,
                                int64_t nF, double* __restrict__ q) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nF) return;
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
    return;
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

__global__ void k_vertex_quadrics(const double* __restrict__ q, const int32_t* __restrict__ off,
                                  const int32_t* __restrict__ idx, int64_t nV,
                                  double* __restrict__ K) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nV) return;
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

// ---- commit (stable compaction) -------------------------------------------
__global__ void k_compact_vertices(const float4* __restrict__ pos_s, const double* __restrict__ K_s,
                                   const uint8_t* __restrict__ vdead,
                                   const int32_t* __restrict__ dead_before, int64_t nV,
                                   float4* __restrict__ pos, double* __restrict__ K,
                                   int32_t* __restrict__ vmap, int32_t* __restrict__ ivmap) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nV) return;
  if (vdead[v]) {
    vmap[v] = -1;
    return;
  }
  int64_t n = v - dead_before[v];
  vmap[v] = (int32_t)n;
  ivmap[n] = (int32_t)v;
  pos[n] = pos_s[v];
  const double2* src = reinterpret_cast<const double2*>(K_s + 10 * v);
  double2* dst = reinterpret_cast<double2*>(K + 10 * n);
#pragma unroll
  for (int i = 0; i < 5; i++) dst[i] = src[i];
}

__global__ void k_compact_faces(const int4* __restrict__ F_s, const uint8_t* __restrict__ fdead,
                                const int32_t* __restrict__ dead_before, int64_t nF,
                                const int32_t* __restrict__ vmap, int4* __restrict__ F) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nF || fdead[f]) return;
  int4 t = F_s[f];
  F[f - dead_before[f]] = make_int4(vmap[t.x], vmap[t.y], vmap[t.z], 0);
}

// flags of the next round: undone winners as remapped vertex pairs, in winner
// (= ascending edge) order, which the monotone vertex map keeps sorted
__global__ void k_undone_pairs(const int32_t* __restrict__ wlist, const int2* __restrict__ E,
                               const uint8_t* __restrict__ standing, const int32_t* __restrict__ uscan,
                               int64_t nW, const int32_t* __restrict__ vmap,
                               unsigned long long* __restrict__ out) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nW || standing[w]) return;
  int2 e = E[wlist[w]];
  out[uscan[w]] = ((unsigned long long)(unsigned)vmap[e.x] << 32) | (unsigned)vmap[e.y];
}

// survivors of committed collapses (new numbering)
__global__ void k_mark_survivors(const int32_t* __restrict__ wlist, const int2* __restrict__ E,
                                 const uint8_t* __restrict__ standing, int64_t nW,
                                 const int32_t* __restrict__ vmap, uint8_t* __restrict__ vsurv) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nW || !standing[w]) return;
  vsurv[vmap[E[wlist[w]].x]] = 1;
}

// a vertex is dirty when it is a survivor or shares a face with one
__global__ void k_mark_dirty(const int4* __restrict__ F, int64_t nF, const uint8_t* __restrict__ vsurv,
                             uint8_t* __restrict__ vdirty) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nF) return;
  const int4 t = F[f];
  if (vsurv[t.x] | vsurv[t.y] | vsurv[t.z]) {
    vdirty[t.x] = 1;
    vdirty[t.y] = 1;
    vdirty[t.z] = 1;
  }
}

__global__ void k_not(const uint8_t* __restrict__ in, int64_t n, uint8_t* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[i] ? 0 : 1;
}

}  // namespace

pamo_status load_mesh(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF, float4* pos,
                      int4* F, cudaStream_t st) {
  k_load<<<grid_for(nV > nF ? nV : nF), kBlock, 0, st>>>(d_V, nV, d_F, nF, pos, F); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status store_mesh(const float4* pos, int64_t nV, const int4* F, int64_t nF, float* d_V,
                       int32_t* d_F, cudaStream_t st) {
  k_store<<<grid_for(nV > nF ? nV : nF), kBlock, 0, st>>>(pos, nV, F, nF, d_V, d_F); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status mesh_bbox(const float4* pos, int64_t nV, float lo[3], float hi[3], Buf& tmp,
                      cudaStream_t st) {
  PAMO_TRY(buf_reserve(tmp, 64, st));
  unsigned init[6] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0, 0, 0};
  PAMO_CUDA(cudaMemcpyAsync(tmp.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
  unsigned g = grid_for(nV);
  if (g > 1024) g = 1024;
  k_bbox<<<g, kBlock, 0, st>>>(pos, nV, (unsigned*)tmp.p); note_launch();
  PAMO_CUDA(cudaGetLastError());
  unsigned out[6];
  PAMO_CUDA(cudaMemcpyAsync(out, tmp.p, sizeof(out), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < 3; k++) {
    unsigned a = out[k], b = out[3 + k];
    a = (a & 0x80000000u) ? (a & 0x7fffffffu) : ~a;
    b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
    std::memcpy(&lo[k], &a, 4);
    std::memcpy(&hi[k], &b, 4);
  }
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
  for (int k = 0; k < 3; k++) {
    unsigned a = out[k], b = out[3 + k];
    a = (a & 0x80000000u) ? (a & 0x7fffffffu) : ~a;
    b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
    std::memcpy(&lo[k], &a, 4);
    std::memcpy(&hi[k], &b, 4);
  }
  return PAMO_OK;
}

pamo_status build_vertex_faces(pamo_ctx* c) {
  cudaStream_t st = c->st;
  PAMO_CUDA(cudaMemsetAsync(c->vcount, 0, sizeof(int32_t) * (c->nV + 1), st));
  k_count_corners<<<grid_for(c->nF), kBlock, 0, st>>>(c->F, c->nF, c->vcount); note_launch();
  PAMO_TRY(exclusive_scan_i32(c->vcount, c->vf_off, c->nV, c->scan_tmp, st));
  PAMO_CUDA(cudaMemsetAsync(c->vcount, 0, sizeof(int32_t) * (c->nV + 1), st));
  k_fill_corners<<<grid_for(c->nF), kBlock, 0, st>>>(c->F, c->nF, c->vf_off, c->vcount, c->vf_idx); note_launch();
  k_sort_segments<<<grid_for(c->nV), kBlock, 0, st>>>(c->vf_off, c->nV, c->vf_idx); note_launch();
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
  PAMO_TRY(build_vertex_faces(c));
  k_check_vertices<<<grid_for(c->nV), kBlock, 0, st>>>(c->F, c->vf_off, c->vf_idx, c->nV, bad); note_launch();
  PAMO_CUDA(cudaGetLastError());
  PAMO_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  if (hb & 8) { set_error("vertex with fewer than 3 incident faces (isolated or open)"); return PAMO_ENOTMANIFOLD; }
  if (hb & 16) { set_error("mesh is not closed, oriented and edge-manifold"); return PAMO_ENOTMANIFOLD; }
  if (hb & 32) { set_error("a vertex link is not a single cycle"); return PAMO_ENOTMANIFOLD; }
  return PAMO_OK;
}

pamo_status build_edges(pamo_ctx* c) {
  cudaStream_t st = c->st;
  k_count_edges<<<grid_for(c->nV), kBlock, 0, st>>>(c->F, c->vf_off, c->vf_idx, c->nV, c->vcount); note_launch();
  PAMO_TRY(exclusive_scan_i32(c->vcount, c->e_off, c->nV, c->scan_tmp, st));
  k_write_edges<<<grid_for(c->nV), kBlock, 0, st>>>(c->F, c->vf_off, c->vf_idx, c->nV, c->e_off,
                                                    c->E); note_launch();
  PAMO_CUDA(cudaGetLastError());
  // a closed triangle mesh has exactly 3F/2 edges; anything else means the
  // mesh is not closed and oriented, and later passes must not run
  int32_t ne = 0;
  PAMO_CUDA(cudaMemcpyAsync(&ne, c->e_off + c->nV, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
  PAMO_CUDA(cudaStreamSynchronize(c->st));
  if ((int64_t)ne != (3 * c->nF) / 2) {
    set_error("edge count is not 3F/2: the mesh is not a closed oriented manifold");
    return PAMO_ENOTMANIFOLD;
  }
  c->nE = ne;
  return PAMO_OK;
}

pamo_status init_quadrics(pamo_ctx* c) {
  cudaStream_t st = c->st;
  PAMO_TRY(buf_reserve(c->quad_tmp, sizeof(double) * 10 * (size_t)c->nF, st));
  double* q = (double*)c->quad_tmp.p;
  k_face_quadrics<<<grid_for(c->nF), kBlock, 0, st>>>(c->pos, c->F, c->nF, q); note_launch();
  k_vertex_quadrics<<<grid_for(c->nV), kBlock, 0, st>>>(q, c->vf_off, c->vf_idx, c->nV, c->K); note_launch();
  PAMO_CUDA(cudaGetLastError());
  buf_free(c->quad_tmp, st);
  return PAMO_OK;
}

pamo_status commit_compact(pamo_ctx* c, int64_t* n_undone) {
  cudaStream_t st = c->st;
  // vertices: new id = old id - (dead vertices before it)
  PAMO_TRY(exclusive_scan_u8(c->vdead, c->dbuf, c->nV, c->scan_tmp, st));
  k_compact_vertices<<<grid_for(c->nV), kBlock, 0, st>>>(c->pos_s, c->K_s, c->vdead, c->dbuf,
                                                         c->nV, c->pos, c->K, c->vmap, c->ivmap); note_launch();
  PAMO_CUDA(cudaGetLastError());
  // faces, corners remapped
  PAMO_TRY(exclusive_scan_u8(c->fdead, c->dbuf, c->nF, c->scan_tmp, st));
  k_compact_faces<<<grid_for(c->nF), kBlock, 0, st>>>(c->F_s, c->fdead, c->dbuf, c->nF, c->vmap,
                                                      c->F); note_launch();
  PAMO_CUDA(cudaGetLastError());
  int64_t nW = c->nW;
  // undone winners -> next round's flag candidates (sorted vertex pairs)
  *n_undone = 0;
  if (nW > 0) {
    k_not<<<grid_for(nW), kBlock, 0, st>>>(c->standing, nW, c->alive_tmp); note_launch();
    PAMO_TRY(exclusive_scan_u8(c->alive_tmp, c->wscan, nW, c->scan_tmp, st));
    k_undone_pairs<<<grid_for(nW), kBlock, 0, st>>>(c->wlist, c->E, c->standing, c->wscan, nW,
                                                    c->vmap, c->flags_next); note_launch();
    PAMO_CUDA(cudaGetLastError());
    int32_t hn = 0;
    PAMO_CUDA(cudaMemcpyAsync(&hn, c->wscan + nW, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaStreamSynchronize(st));
    *n_undone = hn;
  }
  // dirty vertices of the next round (survivors and their neighbours), in the
  // new numbering over the new faces
  const int64_t committed = nW - *n_undone;
  const int64_t nV_new = c->nV - committed, nF_new = c->nF - 2 * committed;
  PAMO_CUDA(cudaMemsetAsync(c->vsurv, 0, nV_new, st));
  PAMO_CUDA(cudaMemsetAsync(c->vdirty, 0, nV_new, st));
  if (committed > 0) {
    k_mark_survivors<<<grid_for(nW), kBlock, 0, st>>>(c->wlist, c->E, c->standing, nW, c->vmap,
                                                      c->vsurv); note_launch();
    k_mark_dirty<<<grid_for(nF_new), kBlock, 0, st>>>(c->F, nF_new, c->vsurv, c->vdirty); note_launch();
    PAMO_CUDA(cudaGetLastError());
  }
  return PAMO_OK;
}

}  // namespace pamo
