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

#define GRID_STRIDE(i, n) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (n); \
       i += (int64_t)gridDim.x * blockDim.x)

__global__ void k_vertex_min(const int2* __restrict__ E, const unsigned long long* __restrict__ key,
                             const RoundCounters* __restrict__ dc,
                             unsigned long long* __restrict__ vkey) {
  const int nE = dc->nE;
  GRID_STRIDE(e, nE) {
    const unsigned long long k = key[e];
    if (k == ~0ull) continue;
    const int2 ab = E[e];
    atomicMin(&vkey[ab.x], k);
    atomicMin(&vkey[ab.y], k);
  }
}

__global__ void k_select(const int2* __restrict__ E, const unsigned long long* __restrict__ key,
                         const RoundCounters* __restrict__ dc,
                         const unsigned long long* __restrict__ vkey,
                         const int4* __restrict__ F, const int32_t* __restrict__ off,
                         const int32_t* __restrict__ idx, uint8_t* __restrict__ win) {
  const int nE = dc->nE;
  GRID_STRIDE(e, nE) {
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
}

__global__ void k_gather_winners(const uint8_t* __restrict__ win, const int32_t* __restrict__ scan,
                                 RoundCounters* __restrict__ dc, int32_t* __restrict__ wlist) {
  const int nE = dc->nE;
  GRID_STRIDE(e, nE) {
    if (win[e]) wlist[scan[e]] = (int32_t)e;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) dc->nW = scan[nE];
}

// Collapse winner w (edge a<b): survivor a takes vbar and K_a + K_b, b dies,
// the two faces on ab die, the other faces around b swap b for a; every face
// around a or b is tagged with w.  Regions of distinct winners share no face.
__global__ void k_collapse(const int32_t* __restrict__ wlist, const RoundCounters* __restrict__ dc,
                           const int2* __restrict__ E,
                           const float4* __restrict__ vbar, const double* __restrict__ K,
                           const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                           const int4* __restrict__ F, float4* __restrict__ pos_s,
                           double* __restrict__ K_s, int4* __restrict__ F_s,
                           uint8_t* __restrict__ fdead, uint8_t* __restrict__ vdead,
                           int32_t* __restrict__ ftag, uint8_t* __restrict__ standing,
                           uint8_t* __restrict__ undo, int32_t* __restrict__ qlist,
                           int* __restrict__ qcount, const uint8_t* __restrict__ keep) {
  const int nW = dc->nW;
  GRID_STRIDE(w, nW) {
  if (keep && !keep[w]) {  // deferred by the learned proposal: treated as undone
    standing[w] = 0;
    undo[w] = 0;
    continue;
  }
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
  undo[w] = 0;
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
}

__global__ void k_stage_ms(const RoundCounters* __restrict__ dc, const float4* __restrict__ pos,
                           const double* __restrict__ K, const int4* __restrict__ F,
                           float4* __restrict__ pos_s, double* __restrict__ K_s,
                           int4* __restrict__ F_s, uint8_t* __restrict__ vdead,
                           uint8_t* __restrict__ fdead, int32_t* __restrict__ ftag,
                           uint32_t* __restrict__ vgap) {
  const int nV = dc->nV, nF = dc->nF;
  GRID_STRIDE(v, nV) {
    pos_s[v] = pos[v];
    vgap[v] = 0x7f800000u;  // +inf; refilled by this round's check
    const double2* src = reinterpret_cast<const double2*>(K + 10 * v);
    double2* dst = reinterpret_cast<double2*>(K_s + 10 * v);
#pragma unroll
    for (int i = 0; i < 5; i++) dst[i] = src[i];
    vdead[v] = 0;
  }
  GRID_STRIDE(f, nF) {
    F_s[f] = F[f];
    fdead[f] = 0;
    ftag[f] = -1;
  }
}

// Undo every marked, still-standing collapse: its region returns to M_1, and
// its faces (each once) are appended to rlist, the queries of the next
// re-check.
__global__ void k_undo(const int32_t* __restrict__ wlist, const int2* __restrict__ E,
                       const float4* __restrict__ pos, const double* __restrict__ K,
                       const int32_t* __restrict__ off, const int32_t* __restrict__ idx,
                       const int4* __restrict__ F, float4* __restrict__ pos_s,
                       double* __restrict__ K_s, int4* __restrict__ F_s,
                       uint8_t* __restrict__ fdead, uint8_t* __restrict__ vdead,
                       int32_t* __restrict__ ftag, uint8_t* __restrict__ standing,
                       uint8_t* __restrict__ undo, RoundCounters* __restrict__ dc,
                       int32_t* __restrict__ rlist) {
  if (dc->cand_overflow) return;  // marks incomplete: the host reruns the fused check
  const int nW = dc->nW;
  int n = 0;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nW;
       base += (int64_t)gridDim.x * blockDim.x) {
  const int64_t w = base + threadIdx.x;
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
      // the region's faces: those around a, then those around b without a
      int nr = off[a + 1] - off[a];
      for (int s = off[b]; s < off[b + 1]; s++) {
        const int4 t = F[idx[s]];
        nr += !(t.x == a || t.y == a || t.z == a);
      }
      int q = atomicAdd(&dc->rest_end, nr);
      for (int pass = 0; pass < 2; pass++) {
        const int v = pass ? b : a;
        for (int s = off[v]; s < off[v + 1]; s++) {
          const int f = idx[s];
          const int4 t = F[f];
          F_s[f] = t;
          fdead[f] = 0;
          ftag[f] = -1;
          if (pass == 0 || !(t.x == a || t.y == a || t.z == a)) rlist[q++] = f;
        }
      }
    }
  }
  }
  n = __reduce_add_sync(0xffffffffu, n);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(&dc->n_undo, n);
}

// outcome of one check iteration: clean when nothing was undone (and the
// candidate buffers held every pair)
__global__ void k_check_result(RoundCounters* __restrict__ dc) {
  // after an overflow the fused check recounts the pairs
  if (!dc->cand_overflow) dc->pairs_total += dc->n_pairs;
  const bool undone = dc->n_undo > 0;
  dc->undo_iters += undone ? 1 : 0;
  const int go = (!undone && !dc->cand_overflow) ? 1 : 0;
  dc->clean = go;
  // commit gate: the compaction that follows runs on these sizes (0 = no-op)
  dc->go = go;
  dc->goV = go ? dc->nV : 0;
  dc->goF = go ? dc->nF : 0;
  dc->goW = go ? dc->nW : 0;
}

// Exact-target mode: when the winners would remove more faces than nF - N_t,
// keep the need = ceil((nF - N_t) / 2) winners with the lowest keys, in edge
// order.  One block: an MSB-first radix select (8 passes of 8 bits) finds the
// need-th smallest key T (keys are unique: the low word is the edge id), then
// an ordered in-place compaction keeps the winners with key <= T.  It runs at
// most in the last round or two of a simplification; otherwise it returns at
// once.
constexpr int kTrimBlock = 1024;

__device__ __forceinline__ int block_excl_scan_1024(int v, int& total) {
  __shared__ int ws[kTrimBlock / 32 + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int w = ws[lane];  // kTrimBlock / 32 == 32 warps
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    ws[lane] = wi - w;
    if (lane == 31) ws[32] = wi;
  }
  __syncthreads();
  const int r = ws[wid] + inc - v;
  total = ws[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kTrimBlock) k_trim(const unsigned long long* __restrict__ key,
                                                     int32_t* __restrict__ wlist,
                                                     RoundCounters* __restrict__ dc) {
  const int nW = dc->nW;
  const int excess = dc->nF - dc->target;
  const int need = excess > 0 ? (excess + 1) / 2 : 0;
  if (nW <= need) return;  // every winner is needed
  __shared__ int hist[256];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_rank;
  unsigned long long prefix = 0, mask = 0;
  int rank = need;  // 1-based rank of the wanted key among those matching prefix
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (int w = threadIdx.x; w < nW; w += blockDim.x) {
      const unsigned long long k = key[wlist[w]];
      if ((k & mask) == prefix) atomicAdd(&hist[(int)((k >> shift) & 0xffu)], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int below = 0, d = 0;
      for (; d < 255; d++) {
        if (below + hist[d] >= rank) break;
        below += hist[d];
      }
      s_prefix = prefix | ((unsigned long long)d << shift);
      s_rank = rank - below;
    }
    __syncthreads();
    prefix = s_prefix;
    rank = s_rank;
    mask |= 0xffull << shift;
    __syncthreads();
  }
  const unsigned long long T = prefix;  // the need-th smallest key
  int base = 0;
  for (int start = 0; start < nW; start += blockDim.x) {
    const int w = start + threadIdx.x;
    int e = -1, keep = 0;
    if (w < nW) {
      e = wlist[w];
      keep = key[e] <= T ? 1 : 0;
    }
    int total;
    const int ex = block_excl_scan_1024(keep, total);  // synchronises: reads done
    if (keep) wlist[base + ex] = e;  // base + ex <= w: never ahead of a read
    base += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) dc->nW = base;
}

}  // namespace

pamo_status trim_winners(pamo_ctx* c) {
  k_trim<<<1, kTrimBlock, 0, c->st>>>(c->key, c->wlist, c->dc); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status select_winners(pamo_ctx* c) {
  cudaStream_t st = c->st;
  const int G = c->grid;
  // vkey was reset to "no key" by k_edge_reuse
  k_vertex_min<<<G, kBlock, 0, st>>>(c->E, c->key, c->dc, c->vkey); note_launch();
  static const int g_select = occ_grid(k_select);
  k_select<<<g_select, kBlock, 0, st>>>(c->E, c->key, c->dc, c->vkey, c->F, c->vf_off, c->vf_idx, c->win); note_launch();
  PAMO_TRY(scan_dev_u8(c->win, &c->dc->nE, c->wscan, c->scan_sums, G, st));
  k_gather_winners<<<G, kBlock, 0, st>>>(c->win, c->wscan, c->dc, c->wlist); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status collapse_winners(pamo_ctx* c) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  const int G = c->grid;
  // M_s starts as a copy of M_1: nothing dead, no face tagged
  k_stage_ms<<<G, kBlock, 0, st>>>(dc, c->pos, c->K, c->F, c->pos_s, c->K_s, c->F_s, c->vdead,
                                   c->fdead, c->ftag, c->vgap); note_launch();
  static const int g_collapse = occ_grid(k_collapse);
  k_collapse<<<g_collapse, kBlock, 0, st>>>(c->wlist, dc, c->E, c->vbar, c->K, c->vf_off, c->vf_idx, c->F,
                                   c->pos_s, c->K_s, c->F_s, c->fdead, c->vdead, c->ftag,
                                   c->standing, c->undo, c->qlist, &dc->n_query,
                                   (c->opt.proposal || c->sched_on) ? c->pkeep : nullptr); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status undo_marked(pamo_ctx* c) {
  k_undo<<<c->grid, kBlock, 0, c->st>>>(c->wlist, c->E, c->pos, c->K, c->vf_off, c->vf_idx, c->F,
                                        c->pos_s, c->K_s, c->F_s, c->fdead, c->vdead, c->ftag,
                                        c->standing, c->undo, c->dc, c->rlist); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status check_result(pamo_ctx* c) {
  k_check_result<<<1, 1, 0, c->st>>>(c->dc); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo
