// The learned proposal (no counterpart in the paper): per-edge features, and
// the deferral of winners the network predicts the intersection check would
// reject (Sections 5.2-5.3 undo them; deferring skips the collapse, the
// check and the undo for this round, and the edge competes again next
// round, invalid for the next round like an undone edge).  Winners are
// independent, so deferring some leaves the others as they are.  Every
// collapse that is committed still passes the exact check.
//
// Features of an edge e = (a, b) of the current mesh, with its placement v,
// length l and cost (all float32; "produced" triangles are the faces around
// a or b except the two on ab, with a and b moved to v):
//   0 log10 of the cost (Eq. 1)          8 mean cos(old normal, new normal)
//   1 log2 of s l (normalised length)    9 min C_ijk of the produced triangles
//   2 |v - midpoint| / l                10 mean (1 - C_ijk)
//   3 valence of a / 6                  11 log2 of (largest distance of v to
//                                          the planes of the old faces) /
//                                          clearance (see 14), in [-10, 10]
//   4 valence of b / 6                  12 log2 of the one-ring area / l^2
//   5 (valence a + valence b - 4) / 6   13 new / old one-ring area
//   6 cos of the dihedral across ab     14 log2 of the clearance / l: the
//   7 min cos(old normal, new normal)      smallest plane distance to a
//                                          non-adjacent face with an overlapping
//                                          box in the last check (clamped to
//                                          [-10, 10]; 10 when there is none)
//                                       15 a or b survived a collapse last round
#include "common.cuh"

namespace pamo {

namespace {

constexpr int kF = PAMO_MLP_IN;

__device__ __forceinline__ float3 f3(const float4& p) { return make_float3(p.x, p.y, p.z); }
__device__ __forceinline__ float3 sub3(float3 a, float3 b) {
  return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3f(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float norm3(float3 a) { return sqrtf(dot3f(a, a)); }

__device__ __forceinline__ float tri_q(float3 u, float3 w, float3 n) {
  // 4 sqrt(3) A / (sum of squared edge lengths), A = |n| / 2
  const float den = dot3f(u, u) + dot3f(w, w) + dot3f(sub3(w, u), sub3(w, u));
  return den > 0.f ? 3.4641016f * norm3(n) / den : 0.f;
}

__device__ void edge_features(int e, const int2* __restrict__ E, const float4* __restrict__ pos,
                              const int4* __restrict__ F, const int32_t* __restrict__ off,
                              const int32_t* __restrict__ idx, const uint32_t* __restrict__ cbits,
                              const float4* __restrict__ vbar, const uint32_t* __restrict__ vgap,
                              const uint8_t* __restrict__ vsurv, float s, float* f) {
  const int2 ab = E[e];
  const int a = ab.x, b = ab.y;
  const float3 pa = f3(pos[a]), pb = f3(pos[b]), v = f3(vbar[e]);
  const float l = fmaxf(norm3(sub3(pb, pa)), 1e-30f);
  const float cost = __uint_as_float(cbits[e] == 0xffffffffu ? 0x7f7fffffu : cbits[e]);
  const int va = off[a + 1] - off[a], vb = off[b + 1] - off[b];
  const float3 mid = make_float3(0.5f * (pa.x + pb.x), 0.5f * (pa.y + pb.y), 0.5f * (pa.z + pb.z));
  float mincos = 1.f, sumcos = 0.f, minq = 1.f, sumskin = 0.f, aold = 0.f, anew = 0.f;
  float dmax = 0.f;  // how far v leaves the old surface
  int ntri = 0, nab = 0;
  float3 nab_n[2] = {make_float3(0.f, 0.f, 0.f), make_float3(0.f, 0.f, 0.f)};
  for (int pass = 0; pass < 2; pass++) {
    const int x = pass ? b : a;
    for (int s0 = off[x]; s0 < off[x + 1]; s0++) {
      const int fid = idx[s0];
      const int4 t = F[fid];
      const bool on_ab = (t.x == a || t.y == a || t.z == a) && (t.x == b || t.y == b || t.z == b);
      if (pass == 1 && (t.x == a || t.y == a || t.z == a)) continue;  // counted from a
      const float3 q0 = f3(pos[t.x]), q1 = f3(pos[t.y]), q2 = f3(pos[t.z]);
      const float3 n_old = cross3(sub3(q1, q0), sub3(q2, q0));
      const float lo_ = norm3(n_old);
      aold += 0.5f * lo_;
      if (lo_ > 0.f) dmax = fmaxf(dmax, fabsf(dot3f(n_old, sub3(v, q0))) / lo_);
      if (on_ab) {
        if (nab < 2) nab_n[nab] = n_old;
        nab++;
        continue;
      }
      const float3 r0 = (t.x == a || t.x == b) ? v : q0;
      const float3 r1 = (t.y == a || t.y == b) ? v : q1;
      const float3 r2 = (t.z == a || t.z == b) ? v : q2;
      const float3 u = sub3(r1, r0), w = sub3(r2, r0);
      const float3 n_new = cross3(u, w);
      const float ln = norm3(n_new), lo = norm3(n_old);
      const float c = (ln > 0.f && lo > 0.f) ? dot3f(n_new, n_old) / (ln * lo) : -1.f;
      mincos = fminf(mincos, c);
      sumcos += c;
      const float q = tri_q(u, w, n_new);
      minq = fminf(minq, q);
      sumskin += 1.f - q;
      anew += 0.5f * ln;
      ntri++;
    }
  }
  float dih = 1.f;
  if (nab == 2) {
    const float l0 = norm3(nab_n[0]), l1 = norm3(nab_n[1]);
    dih = (l0 > 0.f && l1 > 0.f) ? dot3f(nab_n[0], nab_n[1]) / (l0 * l1) : -1.f;
  }
  const float nt = (float)max(ntri, 1);
  f[0] = log10f(fmaxf(cost, 1e-12f));
  f[1] = log2f(fmaxf(s * l, 1e-12f));
  f[2] = norm3(sub3(v, mid)) / l;
  f[3] = va / 6.f;
  f[4] = vb / 6.f;
  f[5] = (va + vb - 4) / 6.f;
  f[6] = dih;
  f[7] = mincos;
  f[8] = sumcos / nt;
  f[9] = minq;
  f[10] = sumskin / nt;
  const float gap = __uint_as_float(min(vgap[a], vgap[b]));
  f[11] = fminf(fmaxf(log2f(fmaxf(dmax, 1e-30f) / fmaxf(gap, 1e-30f)), -10.f), 10.f);
  f[12] = log2f(fmaxf(aold / (l * l), 1e-12f));
  f[13] = aold > 0.f ? anew / aold : 0.f;
  f[14] = fminf(fmaxf(log2f(fmaxf(gap, 1e-30f) / l), -10.f), 10.f);
  f[15] = (vsurv[a] | vsurv[b]) ? 1.f : 0.f;
}

// features of the edges list[0..*n) (or of edges 0..*n when list is null)
__global__ void k_features(const int32_t* __restrict__ list, const int* __restrict__ n_dev,
                           const int2* __restrict__ E, const float4* __restrict__ pos,
                           const int4* __restrict__ F, const int32_t* __restrict__ off,
                           const int32_t* __restrict__ idx, const uint32_t* __restrict__ cbits,
                           const float4* __restrict__ vbar, const uint32_t* __restrict__ vgap,
                           const uint8_t* __restrict__ vsurv, float s, float* __restrict__ X) {
  const int n = *n_dev;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int e = list ? list[i] : (int)i;
    float f[kF];
    edge_features(e, E, pos, F, off, idx, cbits, vbar, vgap, vsurv, s, f);
    float4* o = reinterpret_cast<float4*>(X + (int64_t)kF * i);
#pragma unroll
    for (int q = 0; q < kF / 4; q++) o[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
  }
}

// deferral marks: a winner is kept unless the network predicts an undo (not
// after a round that committed nothing, so that every winner keeps a chance
// and the stall rule of Section 5.3 still ends a run).  A deferred winner is
// not collapsed and counts as undone, so it is an invalid edge for the next
// round like the undone ones (Section 5.3).
__global__ void k_defer_mark(RoundCounters* __restrict__ dc, const float* __restrict__ prob,
                             float threshold, uint8_t* __restrict__ keep) {
  const int n = dc->nW;
  const bool on = dc->last_committed != 0;
  int d = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool defer = on && prob[i] > threshold;
    keep[i] = defer ? 0 : 1;
    d += defer;
  }
  d = __reduce_add_sync(0xffffffffu, d);
  if ((threadIdx.x & 31) == 0 && d) atomicAdd(&dc->deferred, d);
}

// scheduled deferrals: a winner whose vertex pair is in this round's sorted
// part of the schedule is not collapsed and counts as undone, like a
// predicted reject
__global__ void k_defer_sched(RoundCounters* __restrict__ dc, const int32_t* __restrict__ wlist,
                              const int2* __restrict__ E, const unsigned long long* __restrict__ keys,
                              const int64_t* __restrict__ off, int rounds,
                              uint8_t* __restrict__ keep) {
  const int n = dc->nW, r = dc->round_no - 1;
  const unsigned long long* sched = keys + (r < rounds ? off[r] : 0);
  const int ns = r < rounds ? (int)(off[r + 1] - off[r]) : 0;
  int d = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int2 ab = E[wlist[i]];
    const unsigned long long k = ((unsigned long long)(unsigned)ab.x << 32) | (unsigned)ab.y;
    int lo = 0, hi = ns;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sched[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    const bool defer = lo < ns && sched[lo] == k;
    keep[i] = defer ? 0 : 1;
    d += defer;
  }
  d = __reduce_add_sync(0xffffffffu, d);
  if ((threadIdx.x & 31) == 0 && d) atomicAdd(&dc->deferred, d);
}

}  // namespace

pamo_status defer_scheduled(pamo_ctx* c) {
  k_defer_sched<<<c->grid, kBlock, 0, c->st>>>(c->dc, c->wlist, c->E, c->dsched, c->dsched_off,
                                                c->n_sched, c->pkeep); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status edge_features_list(pamo_ctx* c, const int32_t* list, const int* n_dev, float* X,
                               cudaStream_t st) {
  static const int g = occ_grid(k_features);
  k_features<<<g, kBlock, 0, st>>>(list, n_dev, c->E, c->pos, c->F, c->vf_off, c->vf_idx, c->cbits,
                                   c->vbar, c->vgap, c->vsurv, (float)c->scale, X); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

// features + network + deferral over this round's winners (device sizes)
pamo_status propose(pamo_ctx* c) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  const pamo_mlp* m = (const pamo_mlp*)c->opt.proposal;
  const int G = c->grid;
  PAMO_TRY(edge_features_list(c, c->wlist, &dc->nW, c->pX, st));
  PAMO_TRY(mlp_forward_dev(m, c->pX, &dc->nW, c->pprob, c->Emax, st));
  k_defer_mark<<<G, kBlock, 0, st>>>(dc, c->pprob, c->opt.proposal_threshold, c->pkeep); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo
