// Cost propagation, independent-region selection, collapse and undo
// (Algorithm 1 second and third loops, Section 5.1; UndoCollapse, Section 5.3).
//
// Propagation in the paper pushes every edge key onto the triangles of its
// 1-ring with atomicMin and lets an edge win when every triangle of its
// 1-ring still holds its key.  The triangles in the 1-ring of e = (a, b) are
// exactly the faces incident to a or b, so the minimum that reaches triangle t
// equals min over t's three corners of vkey[v] = min{ key_e : e incident to v }.
// This kernel computes vkey with one 64-bit atomicMin per endpoint (2 per edge
// instead of ~12 per edge), and an edge wins iff its key equals vkey[w] for
// every vertex w of every face around a or b: the same winner set.
#include "common.cuh"

namespace pamo {

namespace {

__global__ void k_vertex_min(const int2* __restrict__ E, const unsigned long long* __restrict__ key,
                             int64_t nE, unsigned long long* __restrict__ vkey) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE) return;
  const unsigned long long k = key[e];
  if (k == ~0ull) return;
  const int2 ab = E[e];
  atomicMin(&vkey[ab.x], k);
  atomicMin(&vkey[ab.y], k);
}

__global__ void k_select(const int2* __restrict__ E, const unsigned long long* __restrict__ key,
                         int64_t nE, const unsigned long long* __restrict__ vkey,
                         const int4* __restrict__ F, const int32_t* __restrict__ off,
                         const int32_t* __restrict__ idx, uint8_t* __restrict__ win) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nE) return;
  const unsigned long long k = key[e];
  uint8_t w = 0;
  if (k != ~0ull) {
    const int2 ab = E[e];
    if (vkey[ab.x] == k && vkey[ab.y] == k) {
      w = 1;
      for (int pass = 0; pass < 2 && w; pass++) {
        const int v = pass ? ab.y : ab.x;
        for (int s = off[v]; s < off[v + 1]; s++) {
          const int4 f = F[idx[s]];
          if (vkey[f.x] < k || vkey[f.y] < k || vkey[f.z] < k) {
            w = 0;
            break;
          }
        }
      }
    }
  }
  win[e] = w;
}

__global__ void k_gather_winners(const uint8_t* __restrict__ win, const int32_t* __restrict__ scan,
                                 int64_t nE, int32_t* __restrict__ wlist) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nE && win[e]) wlist[scan[e]] = (int32_t)e;
}

// Collapse winner w (edge a<b): survivor a takes vbar and K_a + K_b, b dies,
// the two faces on ab die, the other faces around b swap b for a; every face
// around a or b is tagged with w.  Regions of distinct winners share no face.
__global__ void k_collapse(const int32_t* __restrict__ wlist, int64_t nW, const int2* __restrict__ E,
                           const float4* __restrict__ vbar, const double* __restrict__ K,
                           const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                           const int4* __restrict__ F, float4* __restrict__ pos_s,
                           double* __restrict__ K_s, int4* __restrict__ F_s,
                           uint8_t* __restrict__ fdead, uint8_t* __restrict__ vdead,
                           int32_t* __restrict__ ftag, uint8_t* __restrict__ standing,
                           int32_t* __restrict__ qlist, int* __restrict__ qcount) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nW) return;
  const int e = wlist[w];
  const int a = E[e].x, b = E[e].y;
  pos_s[a] = vbar[e];
  {
    const double2* ka = reinterpret_cast<const double2*>(K + 10 * (int64_t)a);
    const double2* kb = reinterpret_cast<const double2*>(K + 10 * (int64_t)b);
    double2* ko = reinterpret_cast<double2*>(K_s + 10 * (int64_t)a);
#pragma unroll
    for (int i = 0; i < 5; i++) {
      double2 x = ka[i], y = kb[i];
      ko[i] = make_double2(x.x + y.x, x.y + y.y);
    }
  }
  vdead[b] = 1;
  standing[w] = 1;
  // the faces this collapse changes (alive ones) go to the query list as one
  // contiguous, spatially coherent run
  const int na = off[a + 1] - off[a], nb = off[b + 1] - off[b];
  int q = atomicAdd(qcount, na + nb - 4);
  for (int s = off[a]; s < off[a + 1]; s++) {
    const int f = idx[s];
    const int4 t = F[f];
    if (t.x == b || t.y == b || t.z == b) fdead[f] = 1;
    else qlist[q++] = f;
    ftag[f] = (int32_t)w;
  }
  for (int s = off[b]; s < off[b + 1]; s++) {
    const int f = idx[s];
    int4 t = F[f];
    if (t.x == a || t.y == a || t.z == a) continue;  // on edge ab: already dead
    if (t.x == b) t.x = a;
    if (t.y == b) t.y = a;
    if (t.z == b) t.z = a;
    F_s[f] = t;
    ftag[f] = (int32_t)w;
    qlist[q++] = f;
  }
}

// Undo every marked, still-standing collapse: its region returns to M_1.
__global__ void k_undo(const int32_t* __restrict__ wlist, int64_t nW, const int2* __restrict__ E,
                       const float4* __restrict__ pos, const double* __restrict__ K,
                       const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                       const int4* __restrict__ F, float4* __restrict__ pos_s,
                       double* __restrict__ K_s, int4* __restrict__ F_s,
                       uint8_t* __restrict__ fdead, uint8_t* __restrict__ vdead,
                       int32_t* __restrict__ ftag, uint8_t* __restrict__ standing,
                       uint8_t* __restrict__ undo, RoundCounters* __restrict__ dc) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (dc->cand_overflow) return;  // marks incomplete: the host reruns the fused check
  int n = 0;
  if (w < nW && undo[w]) {
    undo[w] = 0;
    if (standing[w]) {
      standing[w] = 0;
      n = 1;
      const int e = wlist[w];
      const int a = E[e].x, b = E[e].y;
      pos_s[a] = pos[a];
      pos_s[b] = pos[b];
      const double2* src = reinterpret_cast<const double2*>(K + 10 * (int64_t)a);
      double2* dst = reinterpret_cast<double2*>(K_s + 10 * (int64_t)a);
#pragma unroll
      for (int i = 0; i < 5; i++) dst[i] = src[i];
      vdead[b] = 0;
      for (int pass = 0; pass < 2; pass++) {
        const int v = pass ? b : a;
        for (int s = off[v]; s < off[v + 1]; s++) {
          const int f = idx[s];
          F_s[f] = F[f];
          fdead[f] = 0;
          ftag[f] = -1;
        }
      }
    }
  }
  n = __reduce_add_sync(0xffffffffu, n);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&dc->n_undo, n);
}

}  // namespace

pamo_status select_winners(pamo_ctx* c) {
  cudaStream_t st = c->st;
  PAMO_CUDA(cudaMemsetAsync(c->vkey, 0xff, sizeof(unsigned long long) * c->nV, st));
  k_vertex_min<<<grid_for(c->nE), kBlock, 0, st>>>(c->E, c->key, c->nE, c->vkey); note_launch();
  k_select<<<grid_for(c->nE), kBlock, 0, st>>>(c->E, c->key, c->nE, c->vkey, c->F, c->vf_off,
                                               c->vf_idx, c->win); note_launch();
  PAMO_TRY(exclusive_scan_u8(c->win, c->wscan, c->nE, c->scan_tmp, st));
  k_gather_winners<<<grid_for(c->nE), kBlock, 0, st>>>(c->win, c->wscan, c->nE, c->wlist); note_launch();
  PAMO_CUDA(cudaGetLastError());
  int32_t n = 0;
  PAMO_CUDA(cudaMemcpyAsync(&n, c->wscan + c->nE, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  c->nW = n;
  return PAMO_OK;
}

pamo_status collapse_winners(pamo_ctx* c) {
  cudaStream_t st = c->st;
  // M_s starts as a copy of M_1
  PAMO_CUDA(cudaMemcpyAsync(c->pos_s, c->pos, sizeof(float4) * c->nV, cudaMemcpyDeviceToDevice, st));
  PAMO_CUDA(cudaMemcpyAsync(c->K_s, c->K, sizeof(double) * 10 * c->nV, cudaMemcpyDeviceToDevice, st));
  PAMO_CUDA(cudaMemcpyAsync(c->F_s, c->F, sizeof(int4) * c->nF, cudaMemcpyDeviceToDevice, st));
  PAMO_CUDA(cudaMemsetAsync(c->fdead, 0, c->nF, st));
  PAMO_CUDA(cudaMemsetAsync(c->vdead, 0, c->nV, st));
  PAMO_CUDA(cudaMemsetAsync(c->ftag, 0xff, sizeof(int32_t) * c->nF, st));
  PAMO_CUDA(cudaMemsetAsync(c->undo, 0, c->nW > 0 ? c->nW : 1, st));
  PAMO_CUDA(cudaMemsetAsync(&c->dc->n_query, 0, sizeof(int), st));
  if (c->nW > 0) {
    k_collapse<<<grid_for(c->nW), kBlock, 0, st>>>(c->wlist, c->nW, c->E, c->vbar, c->K, c->vf_off,
                                                   c->vf_idx, c->F, c->pos_s, c->K_s, c->F_s,
                                                   c->fdead, c->vdead, c->ftag, c->standing,
                                                   c->qlist, &c->dc->n_query); note_launch();
    PAMO_CUDA(cudaGetLastError());
  }
  return PAMO_OK;
}

pamo_status undo_marked(pamo_ctx* c) {
  if (c->nW == 0) return PAMO_OK;
  k_undo<<<grid_for(c->nW), kBlock, 0, c->st>>>(c->wlist, c->nW, c->E, c->pos, c->K, c->vf_off,
                                                 c->vf_idx, c->F, c->pos_s, c->K_s, c->F_s,
                                                 c->fdead, c->vdead, c->ftag, c->standing,
                                                 c->undo, c->dc); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo
