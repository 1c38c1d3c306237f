// C ABI of the simplifier (include/pamo.h): context lifecycle and the round
// loop of Algorithm 1 ("ParallelSimplification"):
//   while |F(M_1)| > N_t:
//     costs (Eq. 1) -> propagation / independent regions (Sec. 5.1)
//     -> collapse into M_s -> repeat { IntersectionCheck; UndoCollapse }
//     -> M_1 <- M_s (stable compaction) and invalid-edge flags (Sec. 5.3).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "common.cuh"

namespace pamo {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

static cudaEvent_t pool_event(pamo_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void kc_begin(pamo_ctx* c, int cls) {
  c->kc_launch0[cls] = launch_count();
  if (c->opt.profile & (1 << cls)) {
    cudaEvent_t e = pool_event(c);
    cudaEventRecord(e, c->st);
    c->kc_open[cls] = e;
  }
}

void kc_end(pamo_ctx* c, int cls, double bytes) {
  c->class_launches[cls] += launch_count() - c->kc_launch0[cls];
  c->class_bytes[cls] += bytes;
  c->bytes_model += bytes;
  if ((c->opt.profile & (1 << cls)) && c->kc_open[cls]) {
    cudaEvent_t e = pool_event(c);
    cudaEventRecord(e, c->st);
    c->kc_pending.push_back({cls, {c->kc_open[cls], e}});
    c->kc_open[cls] = nullptr;
  }
}

// call after the stream has been synchronised
void kc_resolve(pamo_ctx* c) {
  for (auto& p : c->kc_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.second.first, p.second.second) == cudaSuccess)
      c->class_ms[p.first] += ms;
    c->ev_pool.push_back(p.second.first);
    c->ev_pool.push_back(p.second.second);
  }
  c->kc_pending.clear();
}

pamo_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return PAMO_ENOMEM;
  return PAMO_ECUDA;
}

pamo_status buf_reserve(Buf& b, size_t bytes, cudaStream_t st) {
  if (bytes <= b.bytes && b.p) return PAMO_OK;
  if (b.p) {
    cudaError_t e = cudaFreeAsync(b.p, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    b.p = nullptr;
    b.bytes = 0;
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(&b.p, bytes, st);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return cuda_fail(e, "cudaMallocAsync");
  }
  b.bytes = bytes;
  return PAMO_OK;
}

void buf_free(Buf& b, cudaStream_t st) {
  if (b.p) cudaFreeAsync(b.p, st);
  b.p = nullptr;
  b.bytes = 0;
}

namespace {

template <typename T>
pamo_status alloc(T** p, size_t count, cudaStream_t st) {
  cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (count > 0 ? count : 1), st);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMallocAsync");
  }
  return PAMO_OK;
}

template <typename T>
void release(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync((void*)p, st);
  p = nullptr;
}

void free_ctx_buffers(pamo_ctx* c) {
  cudaStream_t st = c->st;
  release(c->pos, st); release(c->pos_s, st);
  release(c->K, st); release(c->K_s, st);
  release(c->F, st); release(c->F_s, st);
  release(c->vf_off, st); release(c->vf_idx, st); release(c->vcount, st);
  release(c->E, st); release(c->e_off, st); release(c->key, st); release(c->vbar, st);
  release(c->vkey, st); release(c->win, st); release(c->wscan, st); release(c->wlist, st);
  release(c->standing, st); release(c->undo, st); release(c->ftag, st); release(c->qlist, st);
  release(c->fdead, st); release(c->vdead, st); release(c->vmap, st); release(c->dbuf, st);
  release(c->alive_tmp, st); release(c->flags, st); release(c->flags_next, st);
  release(c->dc, st);
  release(c->E_prev, st); release(c->e_off_prev, st); release(c->cbits, st);
  release(c->cbits_prev, st); release(c->vbar_prev, st); release(c->link, st);
  release(c->link_prev, st); release(c->ivmap, st); release(c->vsurv, st); release(c->vdirty, st);
  release(c->dlist, st);
  for (int r = 0; r < 3; r++) release(c->cand[r], st);
  buf_free(c->scan_tmp, st);
  buf_free(c->quad_tmp, st);
  bvh_free(c->bvh, st);
  if (c->hc) cudaFreeHost(c->hc);
  c->hc = nullptr;
  for (auto& p : c->kc_pending) {
    c->ev_pool.push_back(p.second.first);
    c->ev_pool.push_back(p.second.second);
  }
  c->kc_pending.clear();
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
}

pamo_status check_options(const pamo_options* o) {
  if (!(o->w_e >= 0.0) || !(o->w_s >= 0.0)) {
    set_error("weights must be non-negative");
    return PAMO_EINVAL;
  }
  if (o->tolerance < 1 || o->max_rounds < 0 || o->stall_limit < 1) {
    set_error("tolerance and stall_limit must be >= 1, max_rounds >= 0");
    return PAMO_EINVAL;
  }
  if (o->check_mode != 0 && o->check_mode != 1 && o->check_mode != 3) {
    set_error("check_mode must be 0, 1 or 3");
    return PAMO_EINVAL;
  }
  return PAMO_OK;
}

pamo_status create(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                   const pamo_options* opt, cudaStream_t st, pamo_ctx** out) {
  *out = nullptr;
  if (!d_V || !d_F || nV < 4 || nF < 4) {
    set_error("need device arrays and a closed mesh (nV >= 4, nF >= 4)");
    return PAMO_EINVAL;
  }
  if (nF % 2 != 0 || nF >= (int64_t)1 << 30 || nV >= (int64_t)1 << 30) {
    set_error("face count must be even (closed mesh) and sizes below 2^30");
    return PAMO_EINVAL;
  }
  pamo_options o;
  if (opt) o = *opt;
  else pamo_default_options(&o);
  PAMO_TRY(check_options(&o));
  pamo_ctx* c = new pamo_ctx();
  c->st = st;
  c->opt = o;
  c->nV0 = c->nV = nV;
  c->nF0 = c->nF = nF;
  c->Emax = (3 * nF) / 2 + 2;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  }
  const int64_t mx = std::max(nV, nF);
  pamo_status s = PAMO_OK;
#define A(ptr, n) if (s == PAMO_OK) s = alloc(&c->ptr, (size_t)(n), st)
  A(pos, nV); A(pos_s, nV); A(K, 10 * nV); A(K_s, 10 * nV); A(F, nF); A(F_s, nF);
  A(vf_off, nV + 1); A(vf_idx, 3 * nF); A(vcount, nV + 1);
  A(E, c->Emax); A(e_off, nV + 1); A(key, c->Emax); A(vbar, c->Emax); A(vkey, nV);
  A(win, c->Emax); A(wscan, c->Emax + 1); A(wlist, c->Emax); A(standing, c->Emax);
  A(undo, c->Emax); A(ftag, nF); A(qlist, nF); A(fdead, nF); A(vdead, nV); A(vmap, nV + 1);
  A(dbuf, mx + 1); A(alive_tmp, mx); A(flags, c->Emax); A(flags_next, c->Emax); A(dc, 1);
  A(E_prev, c->Emax); A(e_off_prev, nV + 1); A(cbits, c->Emax); A(cbits_prev, c->Emax);
  A(vbar_prev, c->Emax); A(link, c->Emax); A(link_prev, c->Emax); A(ivmap, nV);
  A(vsurv, nV); A(vdirty, nV); A(dlist, c->Emax);
  // candidate pairs of the split check: a changed face has at most 3
  // edge-neighbours; vertex-neighbours and other overlaps are bounded
  // generously, and an overflow falls back to the fused check
  c->cand_cap[0] = 4 * nF; c->cand_cap[1] = 12 * nF; c->cand_cap[2] = 3 * nF;
  if (const char* e = std::getenv("PAMO_CAND_CAP_DIVISOR")) {  // test hook for the fallback
    const long d = std::atol(e);
    if (d > 1)
      for (int r = 0; r < 3; r++) c->cand_cap[r] = std::max<int64_t>(1, c->cand_cap[r] / d);
  }
  A(cand[0], c->cand_cap[0]); A(cand[1], c->cand_cap[1]); A(cand[2], c->cand_cap[2]);
#undef A
  if (s == PAMO_OK) {
    cudaError_t e = cudaMallocHost((void**)&c->hc, sizeof(RoundCounters));
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMallocHost");
  }
  if (s == PAMO_OK) s = load_mesh(d_V, nV, d_F, nF, c->pos, c->F, st);
  if (s == PAMO_OK) {
    cudaError_t e = cudaMemsetAsync(c->dc, 0, sizeof(RoundCounters), st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemsetAsync");
  }
  if (s == PAMO_OK && o.validate_input) s = validate_mesh(c);
  if (s == PAMO_OK && !o.validate_input) s = build_vertex_faces(c);
  if (s == PAMO_OK) s = mesh_bbox(c->pos, nV, c->bb_lo, c->bb_hi, c->scan_tmp, st);
  if (s == PAMO_OK) {
    // s = 1 / (largest extent of the input box), the [0,1]^3 normalisation
    double ext = 0.0;
    for (int k = 0; k < 3; k++) ext = std::max(ext, (double)c->bb_hi[k] - (double)c->bb_lo[k]);
    c->scale = ext > 0.0 ? 1.0 / ext : 1.0;
    s = init_quadrics(c);
  }
  if (s != PAMO_OK) {
    free_ctx_buffers(c);
    cudaStreamSynchronize(st);
    delete c;
    return s;
  }
  *out = c;
  return PAMO_OK;
}

pamo_status sync_counters(pamo_ctx* c) {
  PAMO_CUDA(cudaMemcpyAsync(c->hc, c->dc, sizeof(RoundCounters), cudaMemcpyDeviceToHost, c->st));
  PAMO_CUDA(cudaStreamSynchronize(c->st));
  return PAMO_OK;
}

pamo_status round_cost(pamo_ctx* c) {
  if (c->stage != 0) {
    set_error("pamo_round_cost: previous round not committed");
    return PAMO_EINVAL;
  }
  cudaStream_t st = c->st;
  const double nV = (double)c->nV, nF = (double)c->nF, nE = 1.5 * nF;
  kc_begin(c, PAMO_KC_ADJACENCY);
  // last round's edges and their costs become the reuse source
  std::swap(c->E, c->E_prev);
  std::swap(c->e_off, c->e_off_prev);
  std::swap(c->cbits, c->cbits_prev);
  std::swap(c->vbar, c->vbar_prev);
  std::swap(c->link, c->link_prev);
  if (c->rounds > 0) PAMO_TRY(build_vertex_faces(c));
  PAMO_TRY(build_edges(c));
  // F read; CSR written and read back; edges and offsets written
  kc_end(c, PAMO_KC_ADJACENCY, 16 * nF + 2 * (4 * nV + 12 * nF) + 8 * nE + 4 * nV);
  PAMO_CUDA(cudaMemsetAsync(c->dc, 0, sizeof(RoundCounters), st));
  if (!c->h_flags.empty()) {
    PAMO_CUDA(cudaMemcpyAsync(c->flags, c->h_flags.data(),
                              sizeof(unsigned long long) * c->h_flags.size(),
                              cudaMemcpyHostToDevice, st));
    c->h_flags.clear();
  }
  kc_begin(c, PAMO_KC_COST);
  PAMO_TRY(edge_costs(c));
  // E, positions, quadrics, CSR and faces read once; keys and placements written
  kc_end(c, PAMO_KC_COST, nE * (8 + 8 + 16) + nV * (16 + 80 + 4) + nF * (16 + 12));
  c->stage = 1;
  return PAMO_OK;
}

pamo_status round_select(pamo_ctx* c) {
  if (c->stage != 1) {
    set_error("pamo_round_select: call pamo_round_cost first");
    return PAMO_EINVAL;
  }
  const double nV = (double)c->nV, nF = (double)c->nF, nE = (double)c->nE;
  kc_begin(c, PAMO_KC_SELECT);
  PAMO_TRY(select_winners(c));
  // edges+keys read twice, vkey written and read, CSR+faces read, flags scanned
  kc_end(c, PAMO_KC_SELECT, nE * (2 * 16 + 1 + 1 + 4 + 1 + 4) + nV * (8 + 8 + 4) + nF * (16 + 12) +
                                4.0 * c->nW);
  c->stage = 2;
  return PAMO_OK;
}

pamo_status round_collapse(pamo_ctx* c) {
  if (c->stage != 2) {
    set_error("pamo_round_collapse: call pamo_round_select first");
    return PAMO_EINVAL;
  }
  const double nV = (double)c->nV, nF = (double)c->nF;
  kc_begin(c, PAMO_KC_COLLAPSE);
  PAMO_TRY(collapse_winners(c));
  // M_1 -> M_s copy, flag resets, and each winner's region (~12 faces)
  kc_end(c, PAMO_KC_COLLAPSE, 2 * (16 * nV + 80 * nV + 16 * nF) + nF * 5 + nV +
                                  (double)c->nW * (12 * (16 + 4 + 16) + 2 * 96));
  c->stage = 3;
  return PAMO_OK;
}

pamo_status round_check_undo(pamo_ctx* c) {
  if (c->stage != 3) {
    set_error("pamo_round_check_undo: call pamo_round_collapse first");
    return PAMO_EINVAL;
  }
  cudaStream_t st = c->st;
  c->undo_iters = 0;
  int64_t pairs_total = 0;
  if (c->nW > 0 && c->opt.check_mode != 3) {
    const double nF = (double)c->nF, nV = (double)c->nV;
    // leaf keys, 4 sort passes (read+write 8 B/face, histogram), tree, refit
    const double b_build = nF * (16 + 9) + nV * 16 + 4 * nF * (8 + 8 + 4) + nF * (4 + 32 + 8) +
                           nF * (16 + 4 + 64 + 1);
    const double b_refit = nF * (16 + 4 + 64 + 1 + 4) + nV * 16;
    // node boxes, faces, positions, per-face info / tags / liveness read once
    const double b_query = nF * (64 + 16 + 1 + 4 + 1) + nV * 16;
    kc_begin(c, PAMO_KC_BVH);
    PAMO_TRY(bvh_build(c->bvh, c->pos_s, c->F_s, c->fdead, (int)c->nF, c->bb_lo, c->bb_hi, st));
    kc_end(c, PAMO_KC_BVH, b_build);
    const int all = c->opt.check_mode == 1;
    // every iteration undoes at least one collapse, so nW + 1 iterations bound it
    for (int64_t it = 0; it <= c->nW; it++) {
      PAMO_CUDA(cudaMemsetAsync(&c->dc->n_pairs, 0, 2 * sizeof(int), st));  // n_pairs, n_undo
      kc_begin(c, PAMO_KC_QUERY);
      PAMO_TRY(bvh_check_split(c->bvh, c->pos_s, c->F_s, c->fdead, c->ftag, all, c->qlist,
                               &c->dc->n_query, c->undo, c->dc, c->cand, c->cand_cap,
                               c->dc->ncand, c->sm_count * 8, st));
      kc_end(c, PAMO_KC_QUERY, b_query);
      kc_begin(c, PAMO_KC_COLLAPSE);
      PAMO_TRY(undo_marked(c));  // skipped on the device if a bucket overflowed
      kc_end(c, PAMO_KC_COLLAPSE, (double)c->nW * 2);
      PAMO_TRY(sync_counters(c));
      if (c->hc->cand_overflow) {
        // candidate buffers too small this time: the fused check finds every
        // pair of the same mesh state, then the undo runs
        PAMO_CUDA(cudaMemsetAsync(&c->dc->n_pairs, 0, 2 * sizeof(int), st));
        PAMO_CUDA(cudaMemsetAsync(&c->dc->cand_overflow, 0, sizeof(int), st));
        PAMO_TRY(bvh_check(c->bvh, c->pos_s, c->F_s, c->fdead, c->ftag, all, c->qlist,
                           &c->dc->n_query, c->nF, c->undo, c->dc, nullptr, 0, st));
        PAMO_TRY(undo_marked(c));
        PAMO_TRY(sync_counters(c));
      }
      if (c->hc->overflow) {
        set_error("BVH traversal stack overflow");
        return PAMO_EINTERNAL;
      }
      pairs_total += c->hc->n_pairs;
      if (c->hc->n_undo == 0) break;  // clean (or pairs not caused by this round)
      c->undo_iters++;
      kc_begin(c, PAMO_KC_BVH);
      PAMO_TRY(bvh_refit(c->bvh, c->pos_s, c->F_s, c->fdead, st));
      kc_end(c, PAMO_KC_BVH, b_refit);
    }
  }
  c->stage = 4;
  c->last_pairs = pairs_total;
  return PAMO_OK;
}

pamo_status round_commit(pamo_ctx* c) {
  if (c->stage != 4 && !(c->stage == 3 && c->opt.check_mode == 3)) {
    set_error("pamo_round_commit: call pamo_round_check_undo first");
    return PAMO_EINVAL;
  }
  cudaStream_t st = c->st;
  const int64_t nV_in = c->nV, nF_in = c->nF, nE_in = c->nE, nW = c->nW;
  const int64_t nflags_in = c->nflags;
  // per-round record (before the edge list is rebuilt)
  RoundRecord rec;
  if (c->opt.record_rounds && nW > 0) {
    std::vector<int32_t> wl(nW);
    std::vector<uint8_t> stand(nW);
    std::vector<int2> Eh(c->nE);
    PAMO_CUDA(cudaMemcpyAsync(wl.data(), c->wlist, sizeof(int32_t) * nW, cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaMemcpyAsync(stand.data(), c->standing, nW, cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaMemcpyAsync(Eh.data(), c->E, sizeof(int2) * c->nE, cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaStreamSynchronize(st));
    for (int64_t w = 0; w < nW; w++) {
      int2 e = Eh[wl[w]];
      rec.win.push_back(e.x);
      rec.win.push_back(e.y);
      std::vector<int32_t>& dst = stand[w] ? rec.com : rec.und;
      dst.push_back(e.x);
      dst.push_back(e.y);
    }
  }
  int64_t nund = 0;
  kc_begin(c, PAMO_KC_COMMIT);
  PAMO_TRY(commit_compact(c, &nund));
  // M_s read (positions, quadrics, faces, liveness), M_1 written, vertex map
  // keep the BVH leaf order for the compacted faces (only valid if this
  // round's check built the tree over these nF_in faces)
  if (c->bvh.order_ok && c->bvh.n == nF_in)
    PAMO_TRY(bvh_compact_order(c->bvh, c->fdead, c->dbuf, (int)(nF_in - 2 * (nW - nund)),
                               c->scan_tmp, st));
  else
    c->bvh.order_ok = false;
  kc_end(c, PAMO_KC_COMMIT, (double)nV_in * (16 + 80 + 1 + 4) * 2 + (double)nF_in * (16 + 1 + 4) * 2);
  PAMO_TRY(sync_counters(c));
  kc_resolve(c);
  // float64 operations of the edge costs evaluated this round
  c->class_flops[PAMO_KC_COST] += 114.0 * c->hc->n_dirty + 32.0 * (double)c->hc->cost_tris;
  const int64_t committed = nW - nund;
  c->nV = nV_in - committed;
  c->nF = nF_in - 2 * committed;
  // invalid-edge flags for the next round (Sec. 5.3)
  if (committed > 0) {
    c->hold = 0;
    c->zero_streak = 0;
    std::swap(c->flags, c->flags_next);
    c->nflags = nund;
  } else {
    c->hold++;
    c->zero_streak++;
    std::vector<unsigned long long> a(nflags_in), b(nund), m;
    if (nflags_in)
      PAMO_CUDA(cudaMemcpyAsync(a.data(), c->flags, sizeof(unsigned long long) * nflags_in,
                                cudaMemcpyDeviceToHost, st));
    if (nund)
      PAMO_CUDA(cudaMemcpyAsync(b.data(), c->flags_next, sizeof(unsigned long long) * nund,
                                cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaStreamSynchronize(st));
    std::merge(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(m));
    m.erase(std::unique(m.begin(), m.end()), m.end());
    if (c->hold >= c->opt.tolerance) {
      m.clear();
      c->hold = 0;
    }
    c->nflags = (int64_t)m.size();
    c->h_flags = m;
  }
  const int64_t eligible = (int64_t)c->hc->eligible;
  const int64_t info[11] = {nV_in, nF_in, nE_in, (int64_t)c->hc->link_rejects,
                            (int64_t)c->hc->flagged, eligible, nW, committed, nund,
                            c->undo_iters, c->last_pairs};
  if (c->opt.record_rounds) {
    std::memcpy(rec.info, info, sizeof(info));
    c->rec.push_back(std::move(rec));
  }
  c->committed_total += committed;
  c->undone_total += nund;
  c->link_total += info[3];
  c->win_total += nW;
  c->undo_hist[std::min(c->undo_iters, 7)]++;
  c->rounds++;
  c->have_prev = true;
  c->stage = 0;
  const bool stall_empty = (eligible == 0 && nflags_in == 0);
  if (stall_empty || c->zero_streak >= c->opt.stall_limit) c->stalled = true;
  return PAMO_OK;
}

pamo_status run(pamo_ctx* c, int64_t target) {
  while (c->nF > target) {
    if (c->rounds >= c->opt.max_rounds) {
      c->status = PAMO_ESTALL;
      break;
    }
    PAMO_TRY(round_cost(c));
    PAMO_TRY(round_select(c));
    PAMO_TRY(round_collapse(c));
    PAMO_TRY(round_check_undo(c));
    PAMO_TRY(round_commit(c));
    if (c->stalled) {
      if (c->nF > target) c->status = PAMO_ESTALL;
      break;
    }
  }
  return PAMO_OK;
}

void fill_stats(const pamo_ctx* c, pamo_stats* s, double ms) {
  if (!s) return;
  std::memset(s, 0, sizeof(*s));
  s->rounds = (int32_t)c->rounds;
  for (int i = 0; i < 8; i++) s->undo_iters_hist[i] = c->undo_hist[i];
  s->committed = c->committed_total;
  s->undone = c->undone_total;
  s->link_rejects = c->link_total;
  s->winners = c->win_total;
  s->nV_out = c->nV;
  s->nF_out = c->nF;
  s->ms_total = ms;
  s->bytes_model = c->bytes_model;
  for (int i = 0; i < 8; i++) {
    s->class_ms[i] = c->class_ms[i];
    s->class_launches[i] = c->class_launches[i];
    s->class_bytes[i] = c->class_bytes[i];
    s->class_flops[i] = c->class_flops[i];
  }
}

}  // namespace
}  // namespace pamo

using namespace pamo;

extern "C" {

void pamo_default_options(pamo_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->w_e = 0.001;
  o->w_s = 0.005;
  o->tolerance = 4;
  o->max_rounds = 100000;
  o->stall_limit = 12;
  o->validate_input = 1;
  o->check_mode = 0;
  o->record_rounds = 0;
  o->profile = 0;
}

const char* pamo_last_error(void) { return g_err.c_str(); }

pamo_status pamo_ctx_create(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                            const pamo_options* opt, void* stream, pamo_ctx** out) {
  if (!out) {
    set_error("out is NULL");
    return PAMO_EINVAL;
  }
  return create(d_V, nV, d_F, nF, opt, (cudaStream_t)stream, out);
}

#define CTX_GUARD(c)                 \
  if (!(c)) {                        \
    set_error("context is NULL");    \
    return PAMO_EINVAL;              \
  }

pamo_status pamo_round_cost(pamo_ctx* c) {
  CTX_GUARD(c);
  return round_cost(c);
}

pamo_status pamo_round_select(pamo_ctx* c, int64_t* n_winners) {
  CTX_GUARD(c);
  pamo_status s = round_select(c);
  if (s == PAMO_OK && n_winners) *n_winners = c->nW;
  return s;
}

pamo_status pamo_round_collapse(pamo_ctx* c) {
  CTX_GUARD(c);
  return round_collapse(c);
}

pamo_status pamo_round_check_undo(pamo_ctx* c, int32_t* undo_iters) {
  CTX_GUARD(c);
  pamo_status s = round_check_undo(c);
  if (s == PAMO_OK && undo_iters) *undo_iters = c->undo_iters;
  return s;
}

pamo_status pamo_round_commit(pamo_ctx* c, int64_t* nF_now) {
  CTX_GUARD(c);
  pamo_status s = round_commit(c);
  if (s == PAMO_OK && nF_now) *nF_now = c->nF;
  return s;
}

pamo_status pamo_ctx_sizes(const pamo_ctx* c, int64_t* nV, int64_t* nF, int64_t* nE) {
  CTX_GUARD(c);
  if (nV) *nV = c->nV;
  if (nF) *nF = c->nF;
  if (nE) *nE = c->nE;
  return PAMO_OK;
}

pamo_status pamo_ctx_export(pamo_ctx* c, float* d_V, int32_t* d_F, uint64_t* d_keys,
                            int32_t* d_edges) {
  CTX_GUARD(c);
  if (d_V && d_F) PAMO_TRY(store_mesh(c->pos, c->nV, c->F, c->nF, d_V, d_F, c->st));
  if (d_keys)
    PAMO_CUDA(cudaMemcpyAsync(d_keys, c->key, sizeof(uint64_t) * c->nE, cudaMemcpyDeviceToDevice,
                              c->st));
  if (d_edges)
    PAMO_CUDA(cudaMemcpyAsync(d_edges, c->E, sizeof(int2) * c->nE, cudaMemcpyDeviceToDevice, c->st));
  PAMO_CUDA(cudaStreamSynchronize(c->st));
  return PAMO_OK;
}

pamo_status pamo_ctx_round_info(const pamo_ctx* c, int64_t r, int64_t* out) {
  CTX_GUARD(c);
  if (r < 0 || r >= (int64_t)c->rec.size() || !out) {
    set_error("round index out of range (or rounds not recorded)");
    return PAMO_EINVAL;
  }
  std::memcpy(out, c->rec[r].info, sizeof(c->rec[r].info));
  return PAMO_OK;
}

pamo_status pamo_ctx_round_pairs(const pamo_ctx* c, int64_t r, int32_t kind, int32_t* h_out,
                                 int64_t cap, int64_t* n) {
  CTX_GUARD(c);
  if (r < 0 || r >= (int64_t)c->rec.size() || kind < 0 || kind > 2) {
    set_error("round index or kind out of range (or rounds not recorded)");
    return PAMO_EINVAL;
  }
  const std::vector<int32_t>& v = kind == 0 ? c->rec[r].win : (kind == 1 ? c->rec[r].com : c->rec[r].und);
  const int64_t m = (int64_t)v.size() / 2;
  if (n) *n = m;
  if (h_out) std::memcpy(h_out, v.data(), sizeof(int32_t) * 2 * std::min(m, cap));
  return PAMO_OK;
}

pamo_status pamo_ctx_rounds(const pamo_ctx* c, int64_t* rounds) {
  CTX_GUARD(c);
  if (rounds) *rounds = c->rounds;
  return (pamo_status)c->status;
}

pamo_status pamo_ctx_run(pamo_ctx* c, int64_t target, pamo_stats* stats) {
  CTX_GUARD(c);
  cudaEvent_t e0, e1;
  PAMO_CUDA(cudaEventCreate(&e0));
  PAMO_CUDA(cudaEventCreate(&e1));
  PAMO_CUDA(cudaEventRecord(e0, c->st));
  const long long l0 = launch_count();
  pamo_status s = run(c, target);
  PAMO_CUDA(cudaEventRecord(e1, c->st));
  PAMO_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  kc_resolve(c);
  fill_stats(c, stats, ms);
  if (stats) stats->launches = launch_count() - l0;
  if (s != PAMO_OK) return s;
  return (pamo_status)c->status;
}

void pamo_ctx_destroy(pamo_ctx* c) {
  if (!c) return;
  free_ctx_buffers(c);
  cudaStreamSynchronize(c->st);
  delete c;
}

pamo_status pamo_simplify(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                          int64_t target, const pamo_options* opt, void* stream, float* d_Vout,
                          int64_t* nV_out, int32_t* d_Fout, int64_t* nF_out, pamo_stats* stats) {
  if (!d_Vout || !d_Fout || !nV_out || !nF_out) {
    set_error("output arguments must not be NULL");
    return PAMO_EINVAL;
  }
  if (target < 0) {
    set_error("target_faces must be >= 0");
    return PAMO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  PAMO_CUDA(cudaEventCreate(&e0));
  PAMO_CUDA(cudaEventCreate(&e1));
  PAMO_CUDA(cudaEventRecord(e0, st));
  pamo_ctx* c = nullptr;
  const long long l0 = launch_count();
  pamo_status s = create(d_V, nV, d_F, nF, opt, st, &c);
  if (s == PAMO_OK) s = run(c, target);
  if (s == PAMO_OK) s = store_mesh(c->pos, c->nV, c->F, c->nF, d_Vout, d_Fout, st);
  float ms = 0.f;
  if (s == PAMO_OK) {
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    *nV_out = c->nV;
    *nF_out = c->nF;
    kc_resolve(c);
    fill_stats(c, stats, ms);
    if (stats) stats->launches = launch_count() - l0;
    s = (pamo_status)c->status;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (c) pamo_ctx_destroy(c);
  return s;
}

pamo_status pamo_simplify_host(const float* h_V, int64_t nV, const int32_t* h_F, int64_t nF,
                               int64_t target, const pamo_options* opt, void* stream,
                               float* h_Vout, int64_t* nV_out, int32_t* h_Fout, int64_t* nF_out,
                               pamo_stats* stats) {
  if (!h_V || !h_F || !h_Vout || !h_Fout || !nV_out || !nF_out || nV <= 0 || nF <= 0) {
    set_error("host arrays and sizes required");
    return PAMO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float* dV = nullptr;
  int32_t* dF = nullptr;
  float* dVo = nullptr;
  int32_t* dFo = nullptr;
  pamo_status s = alloc(&dV, 3 * nV, st);
  if (s == PAMO_OK) s = alloc(&dF, 3 * nF, st);
  if (s == PAMO_OK) s = alloc(&dVo, 3 * nV, st);
  if (s == PAMO_OK) s = alloc(&dFo, 3 * nF, st);
  if (s == PAMO_OK) {
    cudaError_t e = cudaMemcpyAsync(dV, h_V, sizeof(float) * 3 * nV, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dF, h_F, sizeof(int32_t) * 3 * nF, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync H2D");
  }
  pamo_status r = PAMO_OK;
  if (s == PAMO_OK) {
    r = pamo_simplify(dV, nV, dF, nF, target, opt, stream, dVo, nV_out, dFo, nF_out, stats);
    if (r == PAMO_OK || r == PAMO_ESTALL) {
      cudaError_t e = cudaMemcpyAsync(h_Vout, dVo, sizeof(float) * 3 * *nV_out,
                                      cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_Fout, dFo, sizeof(int32_t) * 3 * *nF_out, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync D2H");
    }
  }
  release(dV, st);
  release(dF, st);
  release(dVo, st);
  release(dFo, st);
  cudaStreamSynchronize(st);
  return s != PAMO_OK ? s : r;
}

pamo_status pamo_check_self_intersections(const float* d_V, int64_t nV, const int32_t* d_F,
                                          int64_t nF, void* stream, int64_t* n_pairs,
                                          int32_t* d_pairs, int64_t cap) {
  if (!d_V || !d_F || nV <= 0 || nF <= 0 || !n_pairs || nF >= (int64_t)1 << 30) {
    set_error("device mesh and n_pairs required");
    return PAMO_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float4* pos = nullptr;
  int4* F = nullptr;
  RoundCounters* dc = nullptr;
  Buf tmp;
  Bvh b;
  pamo_status s = alloc(&pos, nV, st);
  if (s == PAMO_OK) s = alloc(&F, nF, st);
  if (s == PAMO_OK) s = alloc(&dc, 1, st);
  if (s == PAMO_OK) s = load_mesh(d_V, nV, d_F, nF, pos, F, st);
  float lo[3], hi[3];
  if (s == PAMO_OK) s = mesh_bbox(pos, nV, lo, hi, tmp, st);
  if (s == PAMO_OK) {
    cudaError_t e = cudaMemsetAsync(dc, 0, sizeof(RoundCounters), st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemsetAsync");
  }
  if (s == PAMO_OK) s = bvh_build(b, pos, F, nullptr, (int)nF, lo, hi, st);
  if (s == PAMO_OK)
    s = bvh_check(b, pos, F, nullptr, nullptr, 1, nullptr, nullptr, 0, nullptr, dc, d_pairs, cap, st);
  RoundCounters h{};
  if (s == PAMO_OK) {
    cudaError_t e = cudaMemcpyAsync(&h, dc, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync");
  }
  if (s == PAMO_OK && h.overflow) {
    set_error("BVH traversal stack overflow");
    s = PAMO_EINTERNAL;
  }
  if (s == PAMO_OK) *n_pairs = h.n_pairs;
  bvh_free(b, st);
  buf_free(tmp, st);
  release(pos, st);
  release(F, st);
  release(dc, st);
  cudaStreamSynchronize(st);
  return s;
}

pamo_status pamo_tri_intersect_batch(const float* d_P, const int32_t* d_idx, int64_t n,
                                     uint8_t* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_P || !d_idx || !d_out))) {
    set_error("bad batch arguments");
    return PAMO_EINVAL;
  }
  return tri_batch(d_P, d_idx, n, d_out, (cudaStream_t)stream);
}

pamo_status pamo_orient3d_batch(const float* d_P, int64_t n, int8_t* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_P || !d_out))) {
    set_error("bad batch arguments");
    return PAMO_EINVAL;
  }
  return orient3d_batch(d_P, n, d_out, (cudaStream_t)stream);
}

pamo_status pamo_orient2d_batch(const float* d_P, int64_t n, int8_t* d_out, void* stream) {
  if (n < 0 || (n > 0 && (!d_P || !d_out))) {
    set_error("bad batch arguments");
    return PAMO_EINVAL;
  }
  return orient2d_batch(d_P, n, d_out, (cudaStream_t)stream);
}

}  // extern "C"
