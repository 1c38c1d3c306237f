// C ABI of the simplifier (include/pamo.h): context lifecycle and the round
// loop of Algorithm 1 ("ParallelSimplification"):
//   while |F(M_1)| > N_t:
//     costs (Eq. 1) -> propagation / independent regions (Sec. 5.1)
//     -> collapse into M_s -> repeat { IntersectionCheck; UndoCollapse }
//     -> M_1 <- M_s (stable compaction) and invalid-edge flags (Sec. 5.3).
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace pamo {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

pamo_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return PAMO_ENOMEM;
  return PAMO_ECUDA;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 152;
}

int default_grid() { return 4 * sm_count(); }

// ---- memory -----------------------------------------------------------------
// Device buffers come from a stream-ordered pool owned by the library (one per
// device) whose release threshold keeps freed memory for the next call: a
// simplification allocates its whole working set up front and frees it at the
// end, and the default pool (threshold 0) would hand that memory back to the
// CUDA driver at the next synchronisation and map it again for the next call.
// Pinned host mirrors are recycled the same way.  pamo_release_cached_memory
// returns what no live context uses.
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mem_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
std::vector<std::pair<void*, size_t>> g_pinned;  // cached pinned host blocks
constexpr size_t kPinnedCacheMax = 32;
}  // namespace

pamo_status device_pool(cudaMemPool_t* out) {
  int dev = 0;
  PAMO_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range for the memory pool table");
    return PAMO_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mem_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    PAMO_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = UINT64_MAX;
    PAMO_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools[dev] = pool;
  }
  *out = g_pools[dev];
  return PAMO_OK;
}

pamo_status device_alloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  PAMO_TRY(device_pool(&pool));
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 16, pool, st);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMallocFromPoolAsync");
  }
  return PAMO_OK;
}

// a pinned host block of at least `bytes` (the smallest cached one that fits)
pamo_status pinned_get(void** p, size_t bytes) {
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    int best = -1;
    for (int i = 0; i < (int)g_pinned.size(); i++)
      if (g_pinned[i].second >= bytes && (best < 0 || g_pinned[i].second < g_pinned[best].second))
        best = i;
    if (best >= 0) {
      *p = g_pinned[best].first;
      g_pinned.erase(g_pinned.begin() + best);
      return PAMO_OK;
    }
  }
  // portable: the cache may hand the block to a context on another device
  cudaError_t e = cudaHostAlloc(p, bytes, cudaHostAllocPortable);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaHostAlloc");
  }
  return PAMO_OK;
}

// back to the cache; the caller has synchronised every copy into the block
void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    if (g_pinned.size() < kPinnedCacheMax) {
      g_pinned.emplace_back(p, bytes);
      return;
    }
  }
  cudaFreeHost(p);
}

pamo_status release_cached_memory() {
  std::vector<std::pair<void*, size_t>> blocks;
  cudaError_t first = cudaSuccess;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    blocks.swap(g_pinned);
    for (int d = 0; d < kMaxDevices; d++)
      if (g_pools[d]) {
        cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
        if (first == cudaSuccess) first = e;
      }
  }
  for (auto& b : blocks) cudaFreeHost(b.first);
  if (first != cudaSuccess) return cuda_fail(first, "cudaMemPoolTrimTo");
  return PAMO_OK;
}

// two timing events, destroyed on every exit path
struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  cudaError_t create() {
    cudaError_t e = cudaEventCreate(&a);
    return e == cudaSuccess ? cudaEventCreate(&b) : e;
  }
};

pamo_status buf_reserve(Buf& b, size_t bytes, cudaStream_t st) {
  if (bytes <= b.bytes && b.p) return PAMO_OK;
  if (b.p) {
    cudaError_t e = cudaFreeAsync(b.p, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    b.p = nullptr;
    b.bytes = 0;
  }
  if (bytes == 0) bytes = 16;
  PAMO_TRY(device_alloc(&b.p, bytes, st));
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
  void* q = nullptr;
  pamo_status s = device_alloc(&q, sizeof(T) * (count > 0 ? count : 1), st);
  *p = (T*)q;
  return s;
}

template <typename T>
void release(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync((void*)p, st);
  p = nullptr;
}

void free_graphs(pamo_ctx* c) {
  for (int g = 0; g < 2; g++)
    if (c->gA[g]) {
      cudaGraphExecDestroy(c->gA[g]);
      c->gA[g] = nullptr;
    }
  if (c->gB) {
    cudaGraphExecDestroy(c->gB);
    c->gB = nullptr;
  }
  if (c->gL) {
    cudaGraphExecDestroy(c->gL);
    c->gL = nullptr;
  }
  for (auto& g : c->gev)
    for (auto& k : g)
      for (auto& e : k)
        if (e) {
          cudaEventDestroy(e);
          e = nullptr;
        }
}

void free_ctx_buffers(pamo_ctx* c) {
  cudaStream_t st = c->st;
  free_graphs(c);
  release(c->pos, st); release(c->pos_s, st);
  release(c->K, st); release(c->K_s, st);
  release(c->F, st); release(c->F_s, st);
  release(c->vf_off, st); release(c->vf_idx, st); release(c->vf_nbr, st); release(c->vcount, st);
  release(c->E, st); release(c->e_off, st); release(c->key, st); release(c->vbar, st);
  release(c->vkey, st); release(c->win, st); release(c->wscan, st); release(c->wlist, st);
  release(c->standing, st); release(c->undo, st); release(c->ftag, st); release(c->qlist, st);
  release(c->fdead, st); release(c->vdead, st); release(c->vmap, st); release(c->dbuf, st);
  release(c->flags, st); release(c->flags_next, st);
  release(c->dc, st);
  release(c->E_prev, st); release(c->e_off_prev, st); release(c->cbits, st);
  release(c->cbits_prev, st); release(c->vbar_prev, st); release(c->link, st);
  release(c->link_prev, st); release(c->ivmap, st); release(c->vsurv, st); release(c->vdirty, st);
  release(c->dlist, st); release(c->scan_sums, st); release(c->scan_sums2, st);
  release(c->dbufF, st);
  release(c->vmesh, st); release(c->vmesh_tmp, st); release(c->voff_d, st); release(c->foff_d, st);
  release(c->mframe, st); release(c->mcost, st); release(c->mactive, st); release(c->mcount, st);
  release(c->mvbase, st); release(c->flags_old, st);
  release(c->vgap, st); release(c->vgap_tmp, st); release(c->pX, st);
  release(c->pprob, st); release(c->pkeep, st); release(c->qface, st);
  release(c->dsched, st); release(c->dsched_off, st); release(c->rlist, st);
  release(c->loop, st); release(c->flags_tmp, st); release(c->mstate, st);
  pinned_put(c->loop_h, sizeof(LoopState));
  c->loop_h = nullptr;
  pinned_put(c->mstate_h, sizeof(MeshState) * (size_t)c->n_mesh);
  c->mstate_h = nullptr;
  pinned_put(c->mcount_h, sizeof(int32_t) * 3 * (size_t)c->n_mesh);
  c->mcount_h = nullptr;
  for (int r = 0; r < 3; r++) release(c->cand[r], st);
  buf_free(c->scan_tmp, st);
  buf_free(c->quad_tmp, st);
  bvh_free(c->bvh, st);
  pinned_put(c->hc, sizeof(RoundCounters));
  c->hc = nullptr;
  for (auto& p : c->kc_pending) {
    c->ev_pool.push_back(p.second.first);
    c->ev_pool.push_back(p.second.second);
  }
  c->kc_pending.clear();
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
}

// the context's stream waits for the caller's work so far
pamo_status enter(pamo_ctx* c) {
  PAMO_CUDA(cudaEventRecord(c->join_ev, c->ust));
  PAMO_CUDA(cudaStreamWaitEvent(c->st, c->join_ev, 0));
  return PAMO_OK;
}

// the caller's stream waits for the context's work so far
pamo_status join(pamo_ctx* c) {
  PAMO_CUDA(cudaEventRecord(c->join_ev, c->st));
  PAMO_CUDA(cudaStreamWaitEvent(c->ust, c->join_ev, 0));
  return PAMO_OK;
}

void destroy_ctx(pamo_ctx* c) {
  // no copy into the pinned mirrors may be in flight when they are recycled
  cudaStreamSynchronize(c->st);
  free_ctx_buffers(c);
  cudaStreamSynchronize(c->st);
  for (cudaEvent_t& e : c->round_ev)
    if (e) cudaEventDestroy(e);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  cudaStreamDestroy(c->st);
  delete c;
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
  if (o->exact_target != 0 && o->exact_target != 1) {
    set_error("exact_target must be 0 or 1");
    return PAMO_EINVAL;
  }
  if (!(o->max_cost >= 0.0)) {
    set_error("max_cost must be >= 0 (+infinity = no cost target)");
    return PAMO_EINVAL;
  }
  if (o->check_input_intersections != 0 && o->check_input_intersections != 1) {
    set_error("check_input_intersections must be 0 or 1");
    return PAMO_EINVAL;
  }
  if (o->recompute_quadrics != 0 && o->recompute_quadrics != 1) {
    set_error("recompute_quadrics must be 0 or 1");
    return PAMO_EINVAL;
  }
  if (o->device_loop != 0 && o->device_loop != 1) {
    set_error("device_loop must be 0 or 1");
    return PAMO_EINVAL;
  }
  if (o->grid_blocks_per_sm < 0 || o->grid_blocks_per_sm > 32 || o->resort_percent < 0 ||
      o->resort_percent > 100) {
    set_error("grid_blocks_per_sm must be in 0..32 and resort_percent in 0..100");
    return PAMO_EINVAL;
  }
  return PAMO_OK;
}

// the context's stream (ordered after the caller's) and options
pamo_status new_ctx(const pamo_options* opt, cudaStream_t st, pamo_ctx** out) {
  pamo_options o;
  if (opt) o = *opt;
  else pamo_default_options(&o);
  PAMO_TRY(check_options(&o));
  pamo_ctx* c = new pamo_ctx();
  c->ust = st;
  cudaError_t e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(c->join_ev, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->st, c->join_ev, 0);
  if (e != cudaSuccess) {
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->st) cudaStreamDestroy(c->st);
    delete c;
    return cuda_fail(e, "context stream");
  }
  c->opt = o;
  if (o.record_rounds) {
    cudaEventCreate(&c->round_ev[0]);
    cudaEventCreate(&c->round_ev[1]);
  }
  c->sm_count = sm_count();
  c->grid = c->sm_count * (o.grid_blocks_per_sm > 0 ? o.grid_blocks_per_sm : 6);
  *out = c;
  return PAMO_OK;
}

// every buffer of a simplification of nV vertices and nF faces (sizes only
// shrink, so nothing is allocated later); the batch arrays when n_mesh > 1
pamo_status alloc_state(pamo_ctx* c, int64_t nV, int64_t nF) {
  cudaStream_t st = c->st;
  c->nV0 = c->nV = nV;
  c->nF0 = c->nF = nF;
  c->Emax = (3 * nF) / 2 + 2;
  const int64_t mx = std::max(nV, nF);
  const int M = c->n_mesh;
  pamo_status s = PAMO_OK;
#define A(ptr, n) if (s == PAMO_OK) s = alloc(&c->ptr, (size_t)(n), st)
  A(pos, nV); A(pos_s, nV); A(K, 10 * nV); A(K_s, 10 * nV); A(F, nF); A(F_s, nF);
  A(vf_off, nV + 1); A(vf_idx, 3 * nF); A(vf_nbr, 3 * nF); A(vcount, nV + 1);
  A(E, c->Emax); A(e_off, nV + 1); A(key, c->Emax); A(vbar, c->Emax); A(vkey, nV);
  A(win, c->Emax); A(wscan, c->Emax + 1); A(wlist, c->Emax); A(standing, c->Emax);
  A(undo, c->Emax); A(ftag, nF); A(qlist, nF); A(rlist, nF);
  A(fdead, nF); A(vdead, nV); A(vmap, nV + 1);
  A(dbuf, mx + 1); A(dbufF, nF + 1); A(flags, c->Emax); A(flags_next, c->Emax); A(dc, 1);
  A(E_prev, c->Emax); A(e_off_prev, nV + 1); A(cbits, c->Emax); A(cbits_prev, c->Emax);
  A(vbar_prev, c->Emax); A(link, c->Emax); A(link_prev, c->Emax); A(ivmap, nV);
  A(vsurv, nV); A(vdirty, nV); A(dlist, c->Emax); A(vgap, nV); A(vgap_tmp, nV);
  if (c->opt.proposal) {
    A(pX, 16 * c->Emax); A(pprob, c->Emax); A(pkeep, c->Emax);
  }
  if (c->opt.recompute_quadrics) A(qface, 10 * nF);
  A(scan_sums, scan_sums_count(std::max<int64_t>(c->Emax, mx + 1)));
  c->scan_span = scan_sums_count(mx + 1);
  A(scan_sums2, 3 * c->scan_span);
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
  if (M > 1) {
    A(vmesh, nV); A(vmesh_tmp, nV); A(voff_d, M + 1); A(foff_d, M + 1);
    A(mframe, 6 * (int64_t)M); A(mcost, 2 * (int64_t)M); A(mactive, M);
    A(mcount, 3 * (int64_t)M); A(mvbase, M); A(flags_old, c->Emax);
  }
#undef A
  if (s == PAMO_OK) {  // read by the proposal's features before the first check / commit
    cudaError_t e = cudaMemsetAsync(c->vgap, 0x7f, sizeof(uint32_t) * (size_t)nV, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->vsurv, 0, (size_t)nV, st);
    // per-vertex counts start at zero (each use leaves them zeroed)
    if (e == cudaSuccess) e = cudaMemsetAsync(c->vcount, 0, sizeof(int32_t) * (size_t)(nV + 1), st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemsetAsync");
  }
  c->bvh.n_mesh = M;
  c->bvh.vmesh = c->vmesh;
  c->bvh.mframe = c->mframe;
  c->bvh.vgap = c->vgap;
  if (s == PAMO_OK) s = bvh_alloc(c->bvh, (int)nF, st);
  if (s == PAMO_OK) {
    s = pinned_get((void**)&c->hc, sizeof(RoundCounters));
  }
  if (s == PAMO_OK && M > 1) {
    s = pinned_get((void**)&c->mcount_h, sizeof(int32_t) * 3 * (size_t)M);
  }
  return s;
}

// device counters at the start: sizes and the target edge cost
pamo_status init_counters(pamo_ctx* c) {
  std::memset(c->hc, 0, sizeof(RoundCounters));
  c->hc->nV = (int)c->nV;
  c->hc->nF = (int)c->nF;
  c->hc->last_committed = 1;
  // target edge cost as float bits (costs are keyed as floats, Section 5.1)
  c->hc->max_bits = 0x7f800000u;
  if (c->opt.max_cost < INFINITY) {
    const float f = (float)c->opt.max_cost;
    std::memcpy(&c->hc->max_bits, &f, 4);
  }
  PAMO_CUDA(cudaMemcpyAsync(c->dc, c->hc, sizeof(RoundCounters), cudaMemcpyHostToDevice, c->st));
  return PAMO_OK;
}

// options.check_input_intersections: Algorithm 3 over every face of the
// input (exact); a pair means the input breaks the method's precondition
pamo_status check_input(pamo_ctx* c, const float lo[3], const float hi[3]) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  PAMO_CUDA(cudaMemsetAsync(&dc->n_pairs, 0, sizeof(int), st));
  PAMO_CUDA(cudaMemsetAsync(c->bvh.flags.p, 0, sizeof(int32_t) * (size_t)(c->bvh.n_max + 2), st));
  PAMO_TRY(bvh_build(c->bvh, c->pos, c->F, nullptr, nullptr, (int)c->nF, lo, hi, false, c->grid, st));
  PAMO_TRY(bvh_check(c->bvh, c->pos, c->F, nullptr, nullptr, 1, nullptr, nullptr, 0, nullptr, dc,
                     nullptr, 0, (int)c->nF, st));
  int h[2] = {0, 0};
  PAMO_CUDA(cudaMemcpyAsync(h, &dc->n_pairs, sizeof(int), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaMemcpyAsync(h + 1, &dc->overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  PAMO_CUDA(cudaMemsetAsync(&dc->n_pairs, 0, sizeof(int), st));
  if (h[1]) {
    set_error("BVH traversal bound exceeded in the input check");
    return PAMO_EINTERNAL;
  }
  if (h[0]) {
    set_error("the input mesh intersects itself (" + std::to_string(h[0]) + " face pairs)");
    return PAMO_EINTERSECT;
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
  pamo_ctx* c = nullptr;
  PAMO_TRY(new_ctx(opt, st, &c));
  st = c->st;
  pamo_status s = alloc_state(c, nV, nF);
  if (s == PAMO_OK) s = load_mesh(d_V, nV, d_F, nF, c->pos, c->F, st);
  if (s == PAMO_OK) s = init_counters(c);
  if (s == PAMO_OK && c->opt.validate_input) s = validate_mesh(c);
  if (s == PAMO_OK && !c->opt.validate_input) s = build_vertex_faces(c);
  if (s == PAMO_OK) s = mesh_bbox(c->pos, nV, c->bb_lo, c->bb_hi, c->scan_tmp, st);
  if (s == PAMO_OK) {
    // s = 1 / (largest extent of the input box), the [0,1]^3 normalisation
    double ext = 0.0;
    for (int k = 0; k < 3; k++) ext = std::max(ext, (double)c->bb_hi[k] - (double)c->bb_lo[k]);
    c->scale = ext > 0.0 ? 1.0 / ext : 1.0;
    s = init_quadrics(c);
  }
  if (s == PAMO_OK && c->opt.check_input_intersections) s = check_input(c, c->bb_lo, c->bb_hi);
  if (s != PAMO_OK) {
    destroy_ctx(c);
    return s;
  }
  *out = c;
  return PAMO_OK;
}

// A batch: M meshes as one disjoint union.  h_voff / h_foff (host, M + 1
// entries) delimit each mesh's vertices and faces in the concatenated input;
// each mesh's faces index its own vertices from 0.
pamo_status create_batch(int M, const float* d_V, const int64_t* h_voff, const int32_t* d_F,
                         const int64_t* h_foff, const int64_t* h_targets,
                         const pamo_options* opt, cudaStream_t st, pamo_ctx** out) {
  *out = nullptr;
  if (M < 1 || !d_V || !d_F || !h_voff || !h_foff || !h_targets) {
    set_error("batch: need M >= 1, device arrays and host offsets and targets");
    return PAMO_EINVAL;
  }
  if (h_voff[0] != 0 || h_foff[0] != 0) {
    set_error("batch: offsets must start at 0");
    return PAMO_EINVAL;
  }
  for (int m = 0; m < M; m++) {
    const int64_t nv = h_voff[m + 1] - h_voff[m], nf = h_foff[m + 1] - h_foff[m];
    if (nv < 4 || nf < 4 || nf % 2 != 0 || h_targets[m] < 0) {
      set_error("batch: every mesh needs >= 4 vertices, an even face count >= 4 and a target >= 0");
      return PAMO_EINVAL;
    }
  }
  const int64_t nV = h_voff[M], nF = h_foff[M];
  if (nF >= (int64_t)1 << 30 || nV >= (int64_t)1 << 30) {
    set_error("batch: total sizes must stay below 2^30");
    return PAMO_EINVAL;
  }
  if (opt && (opt->exact_target || opt->proposal)) {
    set_error("batch: exact_target and the learned proposal are single-mesh options");
    return PAMO_EINVAL;
  }
  pamo_ctx* c = nullptr;
  PAMO_TRY(new_ctx(opt, st, &c));
  st = c->st;
  c->n_mesh = M;
  pamo_status s = alloc_state(c, nV, nF);
  if (s == PAMO_OK) {
    cudaError_t e = cudaMemcpyAsync(c->voff_d, h_voff, sizeof(int64_t) * (M + 1),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->foff_d, h_foff, sizeof(int64_t) * (M + 1), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync offsets");
  }
  if (s == PAMO_OK) s = init_counters(c);
  if (s == PAMO_OK)
    s = load_mesh_batch(d_V, nV, d_F, nF, c->voff_d, c->foff_d, M, c->pos, c->F, c->vmesh,
                        &c->dc->bad, st);
  if (s == PAMO_OK && c->opt.validate_input) s = validate_mesh(c);
  if (s == PAMO_OK && !c->opt.validate_input) s = build_vertex_faces(c);
  std::vector<float> lo(3 * (size_t)M), hi(3 * (size_t)M);
  if (s == PAMO_OK) s = buf_reserve(c->scan_tmp, sizeof(unsigned) * 6 * (size_t)M, st);
  if (s == PAMO_OK) s = mesh_bbox_batch(c->pos, c->voff_d, M, (unsigned*)c->scan_tmp.p, lo.data(),
                                        hi.data(), st);
  if (s == PAMO_OK) {
    // per mesh: the [0,1]^3 scale of Eq. 1 and the Morton frame of the LBVH
    std::vector<double> cost(2 * (size_t)M);
    std::vector<float> frame(6 * (size_t)M);
    for (int m = 0; m < M; m++) {
      double ext = 0.0;
      for (int k = 0; k < 3; k++)
        ext = std::max(ext, (double)hi[3 * m + k] - (double)lo[3 * m + k]);
      const double scale = ext > 0.0 ? 1.0 / ext : 1.0;
      cost[2 * m] = scale * scale;
      cost[2 * m + 1] = c->opt.w_e * scale;
      for (int k = 0; k < 3; k++) {
        const float e = hi[3 * m + k] - lo[3 * m + k];
        frame[6 * m + k] = lo[3 * m + k];
        frame[6 * m + 3 + k] = e > 0.f ? 1.0f / e : 0.0f;
      }
    }
    c->m_nV.resize(M); c->m_nF.resize(M); c->m_target.resize(M); c->m_nflags.assign(M, 0);
    c->m_hold.assign(M, 0); c->m_zero.assign(M, 0); c->m_status.assign(M, PAMO_OK);
    c->m_rounds.assign(M, 0); c->m_active.assign(M, 1);
    for (int m = 0; m < M; m++) {
      c->m_nV[m] = h_voff[m + 1] - h_voff[m];
      c->m_nF[m] = h_foff[m + 1] - h_foff[m];
      c->m_target[m] = h_targets[m];
      if (c->m_nF[m] <= c->m_target[m]) c->m_active[m] = 0;  // nothing to do
    }
    cudaError_t e = cudaMemcpyAsync(c->mcost, cost.data(), sizeof(double) * 2 * M,
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->mframe, frame.data(), sizeof(float) * 6 * M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->mactive, c->m_active.data(), M, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host sources are locals
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync batch tables");
  }
  if (s == PAMO_OK) s = init_quadrics(c);
  if (s == PAMO_OK && c->opt.check_input_intersections) {
    float lo0[3] = {0.f, 0.f, 0.f}, hi0[3] = {1.f, 1.f, 1.f};  // per-mesh frames are used
    s = check_input(c, lo0, hi0);
  }
  if (s != PAMO_OK) {
    destroy_ctx(c);
    return s;
  }
  *out = c;
  return PAMO_OK;
}

// ---- kernel-class accounting ------------------------------------------------
// Graph slots: 0 = round graph with a sorted BVH build, 1 = round graph with
// the carried leaf order, 2 = re-check graph.
thread_local int g_capture_slot = -1;  // slot being captured by this thread (-1 = eager)

}  // namespace

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
  if (!(c->opt.profile & (1 << cls))) return;
  if (g_capture_slot >= 0) {
    cudaEvent_t& e = c->gev[g_capture_slot][cls][0];
    if (!e) cudaEventCreate(&e);
    cudaEventRecordWithFlags(e, c->st, cudaEventRecordExternal);
  } else {
    cudaEvent_t e = pool_event(c);
    cudaEventRecord(e, c->st);
    c->kc_open[cls] = e;
  }
}

void kc_end(pamo_ctx* c, int cls, double bytes) {
  const long long n = launch_count() - c->kc_launch0[cls];
  if (g_capture_slot >= 0) {
    long long* t = g_capture_slot < 2 ? c->gA_launch[g_capture_slot] : c->gB_launch;
    t[cls] += n;
  } else {
    c->class_launches[cls] += n;
  }
  c->class_bytes[cls] += bytes;
  c->bytes_model += bytes;
  if (!(c->opt.profile & (1 << cls))) return;
  if (g_capture_slot >= 0) {
    cudaEvent_t& e = c->gev[g_capture_slot][cls][1];
    if (!e) cudaEventCreate(&e);
    cudaEventRecordWithFlags(e, c->st, cudaEventRecordExternal);
  } else if (c->kc_open[cls]) {
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

namespace {

// after a replay of graph slot g (stream synchronised)
void graph_resolve(pamo_ctx* c, int g) {
  c->gk_run += c->g_nodes[g];
  const long long* t = g < 2 ? c->gA_launch[g] : c->gB_launch;
  for (int cls = 0; cls < 8; cls++) {
    c->class_launches[cls] += t[cls];
    cudaEvent_t a = c->gev[g][cls][0], b = c->gev[g][cls][1];
    if (a && b) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, a, b) == cudaSuccess) c->class_ms[cls] += ms;
    }
  }
}

pamo_status sync_out(pamo_ctx* c) {
  PAMO_CUDA(cudaMemcpyAsync(c->hc, c->dc, sizeof(RoundCounters), cudaMemcpyDeviceToHost, c->st));
  if (c->n_mesh > 1)
    PAMO_CUDA(cudaMemcpyAsync(c->mcount_h, c->mcount, sizeof(int32_t) * 3 * c->n_mesh,
                              cudaMemcpyDeviceToHost, c->st));
  return PAMO_OK;
}

pamo_status sync_now(pamo_ctx* c) {
  PAMO_TRY(sync_out(c));
  PAMO_CUDA(cudaStreamSynchronize(c->st));
  return PAMO_OK;
}

// ---- the phases of a round (device sizes; capturable) ---------------------
pamo_status phase_begin(pamo_ctx* c) {
  kc_begin(c, PAMO_KC_ADJACENCY);
  // the round's counters start at zero; last round's edges and their costs
  // become the reuse source
  PAMO_TRY(save_prev(c));
  PAMO_TRY(build_vertex_faces(c, true));
  PAMO_TRY(build_edges(c));
  if (c->opt.recompute_quadrics) PAMO_TRY(recompute_quadrics(c));
  const double nV = (double)c->nV, nF = (double)c->nF, nE = 1.5 * nF;
  // previous edge data copied; F read; CSR written and read back; edges written
  kc_end(c, PAMO_KC_ADJACENCY, 2 * nE * 29 + 16 * nF + 2 * (4 * nV + 12 * nF) + 8 * nE + 4 * nV);
  return PAMO_OK;
}

pamo_status phase_cost(pamo_ctx* c) {
  const double nV = (double)c->nV, nF = (double)c->nF, nE = 1.5 * nF;
  kc_begin(c, PAMO_KC_COST);
  PAMO_TRY(edge_costs(c));
  // E, positions, quadrics, CSR and faces read once; keys and placements written
  kc_end(c, PAMO_KC_COST, nE * (8 + 8 + 16) + nV * (16 + 80 + 4) + nF * (16 + 12));
  return PAMO_OK;
}

pamo_status phase_select(pamo_ctx* c) {
  const double nV = (double)c->nV, nF = (double)c->nF, nE = 1.5 * nF;
  kc_begin(c, PAMO_KC_SELECT);
  PAMO_TRY(select_winners(c));
  // exact-target mode (a full run only: the per-round entry points have no N_t)
  if (c->opt.exact_target && c->in_run) PAMO_TRY(trim_winners(c));
  if (c->sched_on) PAMO_TRY(defer_scheduled(c));  // a given deferral schedule
  else if (c->opt.proposal) PAMO_TRY(propose(c));  // learned deferral of predicted rejects
  // edges+keys read twice, vkey written and read, CSR+faces read, flags scanned
  kc_end(c, PAMO_KC_SELECT, nE * (2 * 16 + 1 + 1 + 4 + 1 + 4) + nV * (8 + 8 + 4) + nF * (16 + 12));
  return PAMO_OK;
}

pamo_status phase_collapse(pamo_ctx* c) {
  const double nV = (double)c->nV, nF = (double)c->nF;
  kc_begin(c, PAMO_KC_COLLAPSE);
  PAMO_TRY(collapse_winners(c));
  // M_1 -> M_s copy, flag resets, and each winner's region (~12 faces)
  kc_end(c, PAMO_KC_COLLAPSE, 2 * (16 * nV + 80 * nV + 16 * nF) + nF * 5 + nV);
  return PAMO_OK;
}

double bvh_build_bytes(double nF, double nV) {
  // leaf keys, 4 sort passes (read+write 8 B/face, histogram), tree, refit
  return nF * (16 + 9) + nV * 16 + 4 * nF * (8 + 8 + 4) + nF * (4 + 32 + 8) + nF * (16 + 4 + 64 + 1);
}
double bvh_refit_bytes(double nF, double nV) { return nF * (16 + 4 + 64 + 1 + 4) + nV * 16; }
double query_bytes(double nF, double nV) { return nF * (64 + 16 + 1 + 4 + 1) + nV * 16; }

pamo_status phase_bvh(pamo_ctx* c, bool carry) {
  kc_begin(c, PAMO_KC_BVH);
  PAMO_TRY(bvh_build(c->bvh, c->pos_s, c->F_s, c->fdead, &c->dc->nF, 0, c->bb_lo, c->bb_hi, carry,
                     c->grid, c->st));
  kc_end(c, PAMO_KC_BVH, carry ? bvh_refit_bytes(c->nF, c->nV) : bvh_build_bytes(c->nF, c->nV));
  return PAMO_OK;
}

pamo_status phase_refit(pamo_ctx* c) {
  kc_begin(c, PAMO_KC_BVH);
  PAMO_TRY(bvh_refit(c->bvh, c->pos_s, c->F_s, c->fdead, &c->dc->nF, 0, c->grid, c->st));
  kc_end(c, PAMO_KC_BVH, bvh_refit_bytes(c->nF, c->nV));
  return PAMO_OK;
}

// one check iteration: split check, undo of the marked collapses, outcome
pamo_status phase_check(pamo_ctx* c) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  if (c->opt.check_mode == 3) return check_result(c);  // debug: no check
  kc_begin(c, PAMO_KC_QUERY);
  PAMO_TRY(bvh_check_split(c->bvh, c->pos_s, c->F_s, c->fdead, c->ftag, c->opt.check_mode == 1,
                           c->qlist, &dc->n_query, c->undo, dc, c->cand, c->cand_cap, dc->ncand,
                           &dc->nF, c->grid, st));
  kc_end(c, PAMO_KC_QUERY, query_bytes(c->nF, c->nV));
  kc_begin(c, 7);
  PAMO_TRY(undo_marked(c));  // skipped on the device if a bucket overflowed
  PAMO_TRY(check_result(c));
  kc_end(c, 7, 0.0);
  return PAMO_OK;
}

// a check iteration after an undo: the restored faces against the standing
// collapses' faces (no refit; see bvh_recheck_restored), undo, outcome
pamo_status phase_recheck(pamo_ctx* c) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  if (c->opt.check_mode == 3) return check_result(c);  // debug: no check
  if (c->opt.check_mode == 1) {  // all-faces mode re-checks everything
    PAMO_TRY(phase_refit(c));
    return phase_check(c);
  }
  kc_begin(c, PAMO_KC_QUERY);
  PAMO_TRY(bvh_recheck_restored(c->bvh, c->pos_s, c->F_s, c->fdead, c->ftag, c->rlist, c->undo,
                                dc, c->cand, c->cand_cap, dc->ncand, &dc->nF, st));
  kc_end(c, PAMO_KC_QUERY, 0.0);
  kc_begin(c, 7);
  PAMO_TRY(undo_marked(c));  // skipped on the device if a bucket overflowed
  PAMO_TRY(check_result(c));
  kc_end(c, 7, 0.0);
  return PAMO_OK;
}

pamo_status phase_commit(pamo_ctx* c) {
  RoundCounters* dc = c->dc;
  kc_begin(c, PAMO_KC_COMMIT);
  PAMO_TRY(commit_compact(c));
  if (c->opt.check_mode != 3)
    PAMO_TRY(bvh_compact_order(c->bvh, c->fdead, c->dbufF, &dc->goF, &dc->goFn, c->grid, c->st));
  PAMO_TRY(commit_sizes(c));
  // M_s read (positions, quadrics, faces, liveness), M_1 written, vertex map
  kc_end(c, PAMO_KC_COMMIT, (double)c->nV * (16 + 80 + 1 + 4) * 2 + (double)c->nF * (16 + 1 + 4) * 2);
  return PAMO_OK;
}

// eager fallback after a candidate overflow: the fused check of every
// standing collapse's faces on the refitted tree of the current mesh state
// (a whole re-check, so the restored faces waiting in rlist are covered),
// undo, outcome, gated commit
pamo_status fallback_check(pamo_ctx* c) {
  cudaStream_t st = c->st;
  RoundCounters* dc = c->dc;
  PAMO_CUDA(cudaMemsetAsync(&dc->n_pairs, 0, 2 * sizeof(int), st));
  PAMO_CUDA(cudaMemsetAsync(&dc->cand_overflow, 0, sizeof(int), st));
  if (c->opt.check_mode != 3) PAMO_TRY(phase_refit(c));
  kc_begin(c, PAMO_KC_QUERY);
  PAMO_TRY(bvh_check(c->bvh, c->pos_s, c->F_s, c->fdead, c->ftag, c->opt.check_mode == 1, c->qlist,
                     &dc->n_query, c->nF, c->undo, dc, nullptr, 0, (int)c->nF, st));
  kc_end(c, PAMO_KC_QUERY, query_bytes(c->nF, c->nV));
  kc_begin(c, 7);
  PAMO_TRY(undo_marked(c));
  PAMO_TRY(check_result(c));
  kc_end(c, 7, 0.0);
  return PAMO_OK;
}

// ---- graphs -----------------------------------------------------------------
template <typename Fn>
pamo_status capture(pamo_ctx* c, int slot, cudaGraphExec_t* exec, Fn fn) {
  cudaGraph_t graph = nullptr;
  PAMO_CUDA(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  g_capture_slot = slot;
  const long long l0 = launch_count();
  const double bytes0 = c->bytes_model;
  double cb0[8];
  for (int i = 0; i < 8; i++) cb0[i] = c->class_bytes[i];
  pamo_status s = fn();
  g_capture_slot = -1;
  c->g_nodes[slot] = launch_count() - l0;
  c->gk_captured += c->g_nodes[slot];
  // bytes are counted per replay, not per capture
  c->bytes_model = bytes0;
  for (int i = 0; i < 8; i++) c->class_bytes[i] = cb0[i];
  cudaError_t e = cudaStreamEndCapture(c->st, &graph);
  if (s != PAMO_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return PAMO_OK;
}

pamo_status round_body(pamo_ctx* c, bool carry) {
  PAMO_TRY(phase_begin(c));
  PAMO_TRY(phase_cost(c));
  PAMO_TRY(phase_select(c));
  PAMO_TRY(phase_collapse(c));
  if (c->opt.check_mode != 3) PAMO_TRY(phase_bvh(c, carry));
  PAMO_TRY(phase_check(c));
  PAMO_TRY(phase_commit(c));
  return sync_out(c);
}

pamo_status recheck_body(pamo_ctx* c) {
  PAMO_TRY(phase_recheck(c));
  PAMO_TRY(phase_commit(c));
  return sync_out(c);
}

// bytes of one replay, from the sizes at the start of the round
void account_bytes(pamo_ctx* c, int slot) {
  const double nV = (double)c->nV, nF = (double)c->nF, nE = 1.5 * nF;
  auto add = [c](int cls, double b) {
    c->class_bytes[cls] += b;
    c->bytes_model += b;
  };
  if (slot < 2) {
    add(PAMO_KC_ADJACENCY, 2 * nE * 29 + 16 * nF + 2 * (4 * nV + 12 * nF) + 8 * nE + 4 * nV);
    add(PAMO_KC_COST, nE * (8 + 8 + 16) + nV * (16 + 80 + 4) + nF * (16 + 12));
    add(PAMO_KC_SELECT, nE * (2 * 16 + 1 + 1 + 4 + 1 + 4) + nV * (8 + 8 + 4) + nF * (16 + 12));
    add(PAMO_KC_COLLAPSE, 2 * (16 * nV + 80 * nV + 16 * nF) + nF * 5 + nV);
    if (c->opt.check_mode != 3)
      add(PAMO_KC_BVH, slot == 1 ? bvh_refit_bytes(nF, nV) : bvh_build_bytes(nF, nV));
  } else {
    add(PAMO_KC_BVH, bvh_refit_bytes(nF, nV));
  }
  if (c->opt.check_mode != 3) add(PAMO_KC_QUERY, query_bytes(nF, nV));
  add(PAMO_KC_COMMIT, nV * (16 + 80 + 1 + 4) * 2 + nF * (16 + 1 + 4) * 2);
}

pamo_status check_device_errors(pamo_ctx* c) {
  if (c->hc->bad & 64) {
    set_error("edge count is not 3F/2: the mesh is not a closed oriented manifold");
    return PAMO_ENOTMANIFOLD;
  }
  if (c->hc->overflow) {
    set_error("BVH traversal or refit bound exceeded");
    return PAMO_EINTERNAL;
  }
  return PAMO_OK;
}

pamo_status finish_round_batch(pamo_ctx* c);

// host bookkeeping once a round is committed (hc holds the device state)
pamo_status finish_round(pamo_ctx* c) {
  if (c->n_mesh > 1) return finish_round_batch(c);
  cudaStream_t st = c->st;
  const RoundCounters& h = *c->hc;
  const int64_t nV_in = c->nV, nF_in = c->nF, nE_in = h.nE, nW = h.nW;
  const int64_t nflags_in = c->nflags, committed = h.committed, nund = h.nund;
  RoundRecord rec;
  if (c->opt.record_rounds && nW > 0) {
    std::vector<int32_t> wl(nW);
    std::vector<uint8_t> stand(nW);
    std::vector<int2> Eh(nE_in);
    PAMO_CUDA(cudaMemcpyAsync(wl.data(), c->wlist, sizeof(int32_t) * nW, cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaMemcpyAsync(stand.data(), c->standing, nW, cudaMemcpyDeviceToHost, st));
    PAMO_CUDA(cudaMemcpyAsync(Eh.data(), c->E, sizeof(int2) * nE_in, cudaMemcpyDeviceToHost, st));
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
  // invalid-edge flags for the next round (Sec. 5.3): after a commit the
  // device already holds the undone edges; otherwise merge on the host
  if (committed > 0) {
    c->hold = 0;
    c->zero_streak = 0;
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
    const int nf = (int)m.size();
    if (nf)
      PAMO_CUDA(cudaMemcpyAsync(c->flags, m.data(), sizeof(unsigned long long) * nf,
                                cudaMemcpyHostToDevice, st));
    PAMO_CUDA(cudaMemcpyAsync(&c->dc->nflags, &nf, sizeof(int), cudaMemcpyHostToDevice, st));
    PAMO_CUDA(cudaStreamSynchronize(st));
  }
  const int64_t eligible = (int64_t)h.eligible;
  const int64_t info[12] = {nV_in, nF_in, nE_in, (int64_t)h.link_rejects, (int64_t)h.flagged,
                            eligible, nW, committed, nund, h.undo_iters, h.pairs_total,
                            c->last_round_us};
  c->last_round_us = 0;
  if (c->opt.record_rounds) {
    std::memcpy(rec.info, info, sizeof(info));
    c->rec.push_back(std::move(rec));
  }
  c->class_flops[PAMO_KC_COST] += kCostFlopsEdge * h.n_dirty + kCostFlopsTri * (double)h.cost_tris;
  c->deferred_total += h.deferred;
  c->cost_edges_total += h.n_dirty;
  c->cost_f64_total += h.cost_f64;
  c->committed_total += committed;
  c->undone_total += nund;
  c->link_total += info[3];
  c->win_total += nW;
  c->undo_hist[std::min(h.undo_iters, 7)]++;
  c->undo_iters = h.undo_iters;
  c->last_pairs = h.pairs_total;
  c->rounds++;
  c->nW = nW;
  c->nE = nE_in;
  c->nV = h.nV;
  c->nF = h.nF;
  c->stage = 0;
  const bool stall_empty = (eligible == 0 && nflags_in == 0);
  if (stall_empty || c->zero_streak >= c->opt.stall_limit) {
    c->stalled = true;
    c->stall_empty = stall_empty;
  }
  return PAMO_OK;
}

// Batch bookkeeping after a committed round: every mesh follows the rules of
// a single simplification (Section 5.3 flags with their own tolerance count,
// stall, target), so each output equals that mesh simplified alone.  The
// device has the undone pairs of every mesh (flags_next) and last round's
// flags in the new numbering (flags_old); the per-mesh merge is done here.
pamo_status finish_round_batch(pamo_ctx* c) {
  cudaStream_t st = c->st;
  const RoundCounters& h = *c->hc;
  const int M = c->n_mesh;
  const int32_t* elig = c->mcount_h;
  const int32_t* com = elig + M;
  const int64_t nflags_in = c->nflags, nund = h.nund;
  std::vector<unsigned long long> old(nflags_in), nw(nund);
  if (nflags_in)
    PAMO_CUDA(cudaMemcpyAsync(old.data(), c->flags_old, sizeof(unsigned long long) * nflags_in,
                              cudaMemcpyDeviceToHost, st));
  if (nund)
    PAMO_CUDA(cudaMemcpyAsync(nw.data(), c->flags_next, sizeof(unsigned long long) * nund,
                              cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  // sizes and vertex bases of the committed union
  std::vector<int64_t> vbase(M + 1, 0);
  for (int m = 0; m < M; m++) {
    c->m_nV[m] -= com[m];
    c->m_nF[m] -= 2 * (int64_t)com[m];
    vbase[m + 1] = vbase[m] + c->m_nV[m];
  }
  auto mesh_of = [&](unsigned long long p) {
    const int64_t a = (int64_t)(p >> 32);
    return (int)(std::upper_bound(vbase.begin(), vbase.end(), a) - vbase.begin()) - 1;
  };
  std::vector<unsigned long long> next;
  next.reserve(nflags_in + nund);
  size_t io = 0, in = 0;
  bool active_changed = false;
  const bool cost_target = c->opt.max_cost < INFINITY;
  for (int m = 0; m < M; m++) {
    std::vector<unsigned long long> om, nm;  // this mesh's old (valid) and new entries
    for (; io < old.size() && (old[io] == ~0ull || mesh_of(old[io]) <= m); io++)
      if (old[io] != ~0ull && mesh_of(old[io]) == m) om.push_back(old[io]);
    for (; in < nw.size() && mesh_of(nw[in]) <= m; in++)
      if (mesh_of(nw[in]) == m) nm.push_back(nw[in]);
    if (!c->m_active[m]) continue;
    std::vector<unsigned long long> fm;
    if (com[m] > 0) {
      c->m_hold[m] = 0;
      c->m_zero[m] = 0;
      fm.swap(nm);
    } else {
      c->m_hold[m]++;
      c->m_zero[m]++;
      std::merge(om.begin(), om.end(), nm.begin(), nm.end(), std::back_inserter(fm));
      fm.erase(std::unique(fm.begin(), fm.end()), fm.end());
      if (c->m_hold[m] >= c->opt.tolerance) {
        fm.clear();
        c->m_hold[m] = 0;
      }
    }
    const bool stall_empty = elig[m] == 0 && c->m_nflags[m] == 0;
    c->m_rounds[m]++;
    if (stall_empty || c->m_zero[m] >= c->opt.stall_limit) {
      const bool cost_end = stall_empty && cost_target;
      c->m_status[m] = (c->m_nF[m] > c->m_target[m] && !cost_end) ? PAMO_ESTALL : PAMO_OK;
      c->m_active[m] = 0;
    } else if (c->m_nF[m] <= c->m_target[m]) {
      c->m_active[m] = 0;  // reached N_t
    }
    if (!c->m_active[m]) {
      active_changed = true;
      fm.clear();
    }
    c->m_nflags[m] = (int64_t)fm.size();
    next.insert(next.end(), fm.begin(), fm.end());
  }
  const int nf = (int)next.size();
  if (nf)
    PAMO_CUDA(cudaMemcpyAsync(c->flags, next.data(), sizeof(unsigned long long) * nf,
                              cudaMemcpyHostToDevice, st));
  PAMO_CUDA(cudaMemcpyAsync(&c->dc->nflags, &nf, sizeof(int), cudaMemcpyHostToDevice, st));
  if (active_changed)
    PAMO_CUDA(cudaMemcpyAsync(c->mactive, c->m_active.data(), M, cudaMemcpyHostToDevice, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  c->nflags = nf;
  // totals over the batch
  c->class_flops[PAMO_KC_COST] += kCostFlopsEdge * h.n_dirty + kCostFlopsTri * (double)h.cost_tris;
  c->cost_edges_total += h.n_dirty;
  c->cost_f64_total += h.cost_f64;
  c->committed_total += h.committed;
  c->undone_total += h.nund;
  c->link_total += (int64_t)h.link_rejects;
  c->win_total += h.nW;
  c->undo_hist[std::min(h.undo_iters, 7)]++;
  c->undo_iters = h.undo_iters;
  c->last_pairs = h.pairs_total;
  c->rounds++;
  c->nW = h.nW;
  c->nE = h.nE;
  c->nV = h.nV;
  c->nF = h.nF;
  c->stage = 0;
  bool any = false;
  for (int m = 0; m < M; m++) any |= c->m_active[m] != 0;
  if (!any) c->stalled = true;  // every mesh is done
  return PAMO_OK;
}

pamo_status graph_round(pamo_ctx* c);

// the rounds of a batch: until every mesh has reached its target or stopped
pamo_status run_rounds_device(pamo_ctx* c, int64_t target);
bool use_device_loop(const pamo_ctx* c);

pamo_status run_batch(pamo_ctx* c) {
  c->in_run = true;
  const int M = c->n_mesh;
  bool any = false;
  for (int m = 0; m < M; m++) any |= c->m_active[m] != 0;
  if (any && use_device_loop(c) && c->stage == 0 && c->rounds < c->opt.max_rounds) {
    pamo_status s = run_rounds_device(c, INT32_MAX);  // the target of every mesh is its own
    c->in_run = false;
    if (s != PAMO_OK) return s;
    c->status = PAMO_OK;
    for (int m = 0; m < M; m++)
      if (c->m_status[m] != PAMO_OK) c->status = PAMO_ESTALL;
    return PAMO_OK;
  }
  while (any) {
    if (c->rounds >= c->opt.max_rounds) {
      for (int m = 0; m < M; m++)
        if (c->m_active[m]) {
          c->m_active[m] = 0;
          c->m_status[m] = PAMO_ESTALL;
        }
      break;
    }
    pamo_status s = graph_round(c);
    if (s != PAMO_OK) {
      c->in_run = false;
      return s;
    }
    any = !c->stalled;
  }
  c->in_run = false;
  c->status = PAMO_OK;
  for (int m = 0; m < M; m++)
    if (c->m_status[m] != PAMO_OK) c->status = PAMO_ESTALL;
  return PAMO_OK;
}

bool use_carry(pamo_ctx* c) {
  // keep the carried leaf order while the face count stays above resort% of
  // the count at the last sort (Morton order only affects speed)
  const int64_t pct = c->opt.resort_percent > 0 ? c->opt.resort_percent : 25;
  return c->bvh.order_ok && 100 * c->nF > pct * (int64_t)c->bvh.n_sorted &&
         pct < 100 && c->opt.check_mode != 3;
}

void note_build(pamo_ctx* c, bool carry) {
  if (!carry && c->opt.check_mode != 3) {
    c->bvh.order_ok = true;
    c->bvh.n_sorted = (int)c->nF;
  }
}

// one round of Algorithm 1 through the captured graphs: one synchronisation
// unless the check found intersections (then one per undo iteration)
pamo_status graph_round(pamo_ctx* c) {
  cudaStream_t st = c->st;
  const bool carry = use_carry(c);
  const int slot = carry ? 1 : 0;
  if (!c->gA[slot]) PAMO_TRY(capture(c, slot, &c->gA[slot], [&] { return round_body(c, carry); }));
  note_build(c, carry);
  const bool timed = c->opt.record_rounds && c->round_ev[0];
  if (timed) PAMO_CUDA(cudaEventRecord(c->round_ev[0], st));
  PAMO_CUDA(cudaGraphLaunch(c->gA[slot], st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  account_bytes(c, slot);
  graph_resolve(c, slot);
  PAMO_TRY(check_device_errors(c));
  for (int64_t it = 0; !c->hc->clean; it++) {
    if (it > c->hc->nW + 2) {
      set_error("undo loop did not settle");
      return PAMO_EINTERNAL;
    }
    if (c->hc->cand_overflow) {
      PAMO_TRY(fallback_check(c));
      PAMO_TRY(phase_commit(c));
      PAMO_TRY(sync_now(c));
      kc_resolve(c);
    } else {
      if (!c->gB) PAMO_TRY(capture(c, 2, &c->gB, [&] { return recheck_body(c); }));
      PAMO_CUDA(cudaGraphLaunch(c->gB, st));
      PAMO_CUDA(cudaStreamSynchronize(st));
      account_bytes(c, 2);
      graph_resolve(c, 2);
    }
    PAMO_TRY(check_device_errors(c));
  }
  if (timed) {
    PAMO_CUDA(cudaEventRecord(c->round_ev[1], st));
    PAMO_CUDA(cudaEventSynchronize(c->round_ev[1]));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->round_ev[0], c->round_ev[1]);
    c->last_round_us = (int64_t)(ms * 1000.0f);
  }
  return finish_round(c);
}

// ---- eager per-round steps (the pamo_round_* entry points) ----------------
pamo_status round_cost(pamo_ctx* c) {
  if (c->stage != 0) {
    set_error("pamo_round_cost: previous round not committed");
    return PAMO_EINVAL;
  }
  PAMO_TRY(phase_begin(c));
  PAMO_TRY(phase_cost(c));
  PAMO_TRY(sync_now(c));
  kc_resolve(c);
  PAMO_TRY(check_device_errors(c));
  c->nE = c->hc->nE;
  c->stage = 1;
  return PAMO_OK;
}

pamo_status round_select(pamo_ctx* c) {
  if (c->stage != 1) {
    set_error("pamo_round_select: call pamo_round_cost first");
    return PAMO_EINVAL;
  }
  PAMO_TRY(phase_select(c));
  PAMO_TRY(sync_now(c));
  kc_resolve(c);
  c->nW = c->hc->nW;
  c->stage = 2;
  return PAMO_OK;
}

pamo_status round_collapse(pamo_ctx* c) {
  if (c->stage != 2) {
    set_error("pamo_round_collapse: call pamo_round_select first");
    return PAMO_EINVAL;
  }
  PAMO_TRY(phase_collapse(c));
  c->stage = 3;
  return PAMO_OK;
}

pamo_status round_check_undo(pamo_ctx* c) {
  if (c->stage != 3) {
    set_error("pamo_round_check_undo: call pamo_round_collapse first");
    return PAMO_EINVAL;
  }
  const bool carry = use_carry(c);
  if (c->opt.check_mode != 3) PAMO_TRY(phase_bvh(c, carry));
  note_build(c, carry);
  for (int64_t it = 0;; it++) {
    if (it > c->nW + 2) {
      set_error("undo loop did not settle");
      return PAMO_EINTERNAL;
    }
    PAMO_TRY(it == 0 ? phase_check(c) : phase_recheck(c));
    PAMO_TRY(sync_now(c));
    if (c->hc->cand_overflow) {
      PAMO_TRY(fallback_check(c));
      PAMO_TRY(sync_now(c));
    }
    kc_resolve(c);
    PAMO_TRY(check_device_errors(c));
    if (c->hc->clean) break;
  }
  c->undo_iters = c->hc->undo_iters;
  c->last_pairs = c->hc->pairs_total;
  c->stage = 4;
  return PAMO_OK;
}

pamo_status round_commit(pamo_ctx* c) {
  if (c->stage != 4) {
    set_error("pamo_round_commit: call pamo_round_check_undo first");
    return PAMO_EINVAL;
  }
  PAMO_TRY(phase_commit(c));
  PAMO_TRY(sync_now(c));
  kc_resolve(c);
  return finish_round(c);
}

pamo_status run_rounds(pamo_ctx* c, int64_t target);

pamo_status run(pamo_ctx* c, int64_t target) {
  c->in_run = true;
  pamo_status s = run_rounds(c, target);
  c->in_run = false;
  return s;
}

// ---- the device-side round loop (loop.cu) ----------------------------------
// Captures fn's launches on the context's stream into graph g after the nodes
// in deps; deps then holds the capture's last nodes.  kernels counts the
// launches captured.
template <typename Fn>
pamo_status capture_into(pamo_ctx* c, cudaGraph_t g, std::vector<cudaGraphNode_t>& deps,
                         long long* kernels, Fn fn) {
  PAMO_CUDA(cudaStreamBeginCaptureToGraph(c->st, g, deps.empty() ? nullptr : deps.data(), nullptr,
                                          deps.size(), cudaStreamCaptureModeThreadLocal));
  const long long l0 = launch_count();
  pamo_status s = fn();
  if (kernels) *kernels += launch_count() - l0;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(c->st, &cs, nullptr, nullptr, &d, nullptr, &nd);
  std::vector<cudaGraphNode_t> last;
  if (e == cudaSuccess && d) last.assign(d, d + nd);
  cudaGraph_t out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(c->st, &out);
  if (s != PAMO_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamGetCaptureInfo");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
  deps.swap(last);
  return PAMO_OK;
}

// A conditional node after deps; bodies receives its body graphs (size of
// them); deps then holds the node.
pamo_status add_conditional(cudaGraph_t g, std::vector<cudaGraphNode_t>& deps,
                            cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            unsigned size, cudaGraph_t* bodies) {
  cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = size;
  cudaGraphNode_t node = nullptr;
  PAMO_CUDA(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                             &p));
  for (unsigned i = 0; i < size; i++) bodies[i] = p.conditional.phGraph_out[i];
  deps.assign(1, node);
  return PAMO_OK;
}

// The whole run as one graph:
//   init -> WHILE(round) { begin, cost, select, collapse;
//                          IF(sort) sort build ELSE carried-order build;
//                          check; IF(overflow) fallback;
//                          WHILE(not clean) { re-check; IF(overflow) fallback };
//                          commit; flags; finish }
pamo_status build_loop_graph(pamo_ctx* c) {
  cudaGraph_t g = nullptr;
  PAMO_CUDA(cudaGraphCreate(&g, 0));
  // launch and byte accounting of the phases is per replay, not per capture
  const double bytes0 = c->bytes_model;
  double cb0[8];
  long long cl0[8];
  for (int i = 0; i < 8; i++) {
    cb0[i] = c->class_bytes[i];
    cl0[i] = c->class_launches[i];
  }
  const long long captured0 = launch_count();
  long long* kn = c->gL_nodes;
  for (int i = 0; i < 5; i++) kn[i] = 0;
  auto body = [&]() -> pamo_status {
    cudaGraphConditionalHandle h_round, h_sort, h_fb1, h_undo, h_fb2;
    PAMO_CUDA(cudaGraphConditionalHandleCreate(&h_round, g, 1, cudaGraphCondAssignDefault));
    PAMO_CUDA(cudaGraphConditionalHandleCreate(&h_sort, g, 0, 0));
    PAMO_CUDA(cudaGraphConditionalHandleCreate(&h_fb1, g, 0, 0));
    PAMO_CUDA(cudaGraphConditionalHandleCreate(&h_undo, g, 0, 0));
    PAMO_CUDA(cudaGraphConditionalHandleCreate(&h_fb2, g, 0, 0));
    std::vector<cudaGraphNode_t> top;
    PAMO_TRY(capture_into(c, g, top, nullptr, [&] { return loop_init(c, h_sort); }));
    cudaGraph_t round_g;
    PAMO_TRY(add_conditional(g, top, h_round, cudaGraphCondTypeWhile, 1, &round_g));
    std::vector<cudaGraphNode_t> d;
    PAMO_TRY(capture_into(c, round_g, d, &kn[0], [&]() -> pamo_status {
      PAMO_TRY(phase_begin(c));
      PAMO_TRY(phase_cost(c));
      PAMO_TRY(phase_select(c));
      return phase_collapse(c);
    }));
    cudaGraph_t build[2];
    PAMO_TRY(add_conditional(round_g, d, h_sort, cudaGraphCondTypeIf, 2, build));
    std::vector<cudaGraphNode_t> b0, b1;
    PAMO_TRY(capture_into(c, build[0], b0, &kn[1], [&] { return phase_bvh(c, false); }));
    PAMO_TRY(capture_into(c, build[1], b1, &kn[2], [&] { return phase_bvh(c, true); }));
    PAMO_TRY(capture_into(c, round_g, d, &kn[0], [&]() -> pamo_status {
      PAMO_TRY(phase_check(c));
      return loop_cond_fallback(c, h_fb1, 1);
    }));
    cudaGraph_t fb;
    PAMO_TRY(add_conditional(round_g, d, h_fb1, cudaGraphCondTypeIf, 1, &fb));
    std::vector<cudaGraphNode_t> f1;
    PAMO_TRY(capture_into(c, fb, f1, &kn[4], [&] { return fallback_check(c); }));
    PAMO_TRY(capture_into(c, round_g, d, &kn[0], [&] { return loop_cond_undo(c, h_undo); }));
    cudaGraph_t undo_g;
    PAMO_TRY(add_conditional(round_g, d, h_undo, cudaGraphCondTypeWhile, 1, &undo_g));
    std::vector<cudaGraphNode_t> u;
    PAMO_TRY(capture_into(c, undo_g, u, &kn[3], [&]() -> pamo_status {
      PAMO_TRY(phase_recheck(c));
      return loop_cond_fallback(c, h_fb2, 0);
    }));
    cudaGraph_t fb2;
    PAMO_TRY(add_conditional(undo_g, u, h_fb2, cudaGraphCondTypeIf, 1, &fb2));
    std::vector<cudaGraphNode_t> f2;
    PAMO_TRY(capture_into(c, fb2, f2, nullptr, [&] { return fallback_check(c); }));
    PAMO_TRY(capture_into(c, undo_g, u, &kn[3], [&] { return loop_cond_undo(c, h_undo); }));
    PAMO_TRY(capture_into(c, round_g, d, &kn[0], [&]() -> pamo_status {
      PAMO_TRY(phase_commit(c));
      return loop_finish(c, h_round, h_sort);
    }));
    PAMO_CUDA(cudaGraphInstantiate(&c->gL, g, 0));
    return PAMO_OK;
  };
  pamo_status s = body();
  cudaGraphDestroy(g);
  c->gk_captured += launch_count() - captured0;
  c->bytes_model = bytes0;
  for (int i = 0; i < 8; i++) {
    c->class_bytes[i] = cb0[i];
    c->class_launches[i] = cl0[i];
  }
  return s;
}

// The device loop (options.device_loop) runs plain simplifications and
// batches; per-round records, class timing and the all-faces / no-check debug
// modes keep the host loop.
bool use_device_loop(const pamo_ctx* c) {
  return c->opt.device_loop && !c->opt.record_rounds && !c->opt.profile &&
         c->opt.check_mode == 0;
}

pamo_status run_rounds_device(pamo_ctx* c, int64_t target) {
  cudaStream_t st = c->st;
  const int M = c->n_mesh;
  if (!c->loop) {
    PAMO_TRY(alloc(&c->loop, 1, st));
    PAMO_TRY(alloc(&c->flags_tmp, (size_t)c->Emax, st));
    PAMO_TRY(pinned_get((void**)&c->loop_h, sizeof(LoopState)));
    if (M > 1) {
      PAMO_TRY(alloc(&c->mstate, (size_t)M, st));
      PAMO_TRY(pinned_get((void**)&c->mstate_h, sizeof(MeshState) * (size_t)M));
    }
  }
  if (M > 1) {  // every mesh's state, as the host loop keeps it
    for (int m = 0; m < M; m++) {
      MeshState& ms = c->mstate_h[m];
      ms.nV = c->m_nV[m];
      ms.nF = c->m_nF[m];
      ms.target = c->m_target[m];
      ms.nflags = (int)c->m_nflags[m];
      ms.hold = c->m_hold[m];
      ms.zero = c->m_zero[m];
      ms.status = c->m_status[m];
      ms.rounds = c->m_rounds[m];
      ms.active = c->m_active[m];
      ms.mode = 0;
    }
    PAMO_CUDA(cudaMemcpyAsync(c->mstate, c->mstate_h, sizeof(MeshState) * M,
                              cudaMemcpyHostToDevice, st));
  }
  if (!c->gL) PAMO_TRY(build_loop_graph(c));
  LoopState& L = *c->loop_h;
  std::memset(&L, 0, sizeof(L));
  L.target = (int)std::min<int64_t>(target, INT32_MAX);
  L.max_rounds = c->opt.max_rounds;
  L.stall_limit = c->opt.stall_limit;
  L.tolerance = c->opt.tolerance;
  L.resort_pct = c->opt.resort_percent > 0 ? c->opt.resort_percent : 25;
  L.cost_target = c->opt.max_cost < INFINITY ? 1 : 0;
  L.rounds = (int)c->rounds;
  L.hold = c->hold;
  L.zero_streak = c->zero_streak;
  const bool carry = use_carry(c);
  note_build(c, carry);
  L.sort_first = carry ? 0 : 1;
  L.sorts = carry ? 0 : 1;
  L.order_ok = c->bvh.order_ok ? 1 : 0;
  L.n_sorted = c->bvh.n_sorted;
  PAMO_CUDA(cudaMemcpyAsync(c->loop, &L, sizeof(L), cudaMemcpyHostToDevice, st));
  PAMO_CUDA(cudaGraphLaunch(c->gL, st));
  PAMO_CUDA(cudaMemcpyAsync(&L, c->loop, sizeof(L), cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaMemcpyAsync(c->hc, c->dc, sizeof(RoundCounters), cudaMemcpyDeviceToHost, st));
  if (M > 1)
    PAMO_CUDA(cudaMemcpyAsync(c->mstate_h, c->mstate, sizeof(MeshState) * M,
                              cudaMemcpyDeviceToHost, st));
  PAMO_CUDA(cudaStreamSynchronize(st));
  if (M > 1) {
    for (int m = 0; m < M; m++) {
      const MeshState& ms = c->mstate_h[m];
      c->m_nV[m] = ms.nV;
      c->m_nF[m] = ms.nF;
      c->m_nflags[m] = ms.nflags;
      c->m_hold[m] = ms.hold;
      c->m_zero[m] = ms.zero;
      c->m_status[m] = ms.status;
      c->m_rounds[m] = ms.rounds;
      c->m_active[m] = (uint8_t)ms.active;
    }
  }
  const int64_t done = L.rounds - c->rounds;
  // kernels run: every round, its BVH build, its re-checks and fallbacks
  c->gk_run += done * c->gL_nodes[0] + L.sorts * c->gL_nodes[1] +
               (done - L.sorts) * c->gL_nodes[2] + L.rechecks * c->gL_nodes[3] +
               L.fallbacks * c->gL_nodes[4] + 1;
  c->rounds = L.rounds;
  c->hold = L.hold;
  c->zero_streak = L.zero_streak;
  c->bvh.order_ok = L.order_ok != 0;
  c->bvh.n_sorted = L.n_sorted;
  c->nflags = c->hc->nflags;
  c->nV = c->hc->nV;
  c->nF = c->hc->nF;
  c->nE = L.nE;
  c->nW = L.nW;
  c->undo_iters = L.undo_iters;
  c->last_pairs = L.pairs;
  c->committed_total += L.committed;
  c->undone_total += L.undone;
  c->link_total += L.link;
  c->win_total += L.winners;
  c->deferred_total += L.deferred;
  c->cost_edges_total += L.cost_edges;
  c->cost_f64_total += L.cost_f64;
  c->class_flops[PAMO_KC_COST] += kCostFlopsEdge * (double)L.cost_edges +
                                  kCostFlopsTri * (double)L.cost_tris;
  for (int i = 0; i < 8; i++) c->undo_hist[i] += (int32_t)L.undo_hist[i];
  c->stage = 0;
  if (L.error) {
    set_error(L.error == PAMO_ENOTMANIFOLD
                  ? "edge count is not 3F/2: the mesh is not a closed oriented manifold"
                  : "BVH traversal or refit bound exceeded, or the undo loop did not settle");
    return (pamo_status)L.error;
  }
  if (L.status == PAMO_ESTALL) {
    c->stalled = true;
    c->stall_empty = L.stall_empty != 0;
    c->status = PAMO_ESTALL;
  }
  return PAMO_OK;
}

pamo_status run_rounds(pamo_ctx* c, int64_t target) {
  {  // N_t on the device (exact-target trimming reads it); pageable source,
     // so the call returns once the value has been staged
    const int t = (int)std::min<int64_t>(target, INT32_MAX);
    PAMO_CUDA(cudaMemcpyAsync(&c->dc->target, &t, sizeof(int), cudaMemcpyHostToDevice, c->st));
  }
  if (use_device_loop(c) && c->nF > target && c->stage == 0 && !c->stalled &&
      c->rounds < c->opt.max_rounds)
    return run_rounds_device(c, target);
  while (c->nF > target) {
    if (c->rounds >= c->opt.max_rounds) {
      c->status = PAMO_ESTALL;
      break;
    }
    if (c->stage != 0) {
      set_error("a round is in progress (per-round entry points)");
      return PAMO_EINVAL;
    }
    PAMO_TRY(graph_round(c));
    if (c->stalled) {
      // with a target edge cost, running out of eligible edges is the normal end
      const bool cost_end = c->stall_empty && c->opt.max_cost < INFINITY;
      if (c->nF > target && !cost_end) c->status = PAMO_ESTALL;
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
  s->deferred = c->deferred_total;
  s->cost_edges = c->cost_edges_total;
  s->cost_f64 = c->cost_f64_total;
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
  o->exact_target = 0;
  o->max_cost = INFINITY;
  o->grid_blocks_per_sm = 0;
  o->resort_percent = 0;
  o->proposal = nullptr;
  o->proposal_threshold = 0.5f;
  o->recompute_quadrics = 0;
  o->device_loop = 0;
  o->check_input_intersections = 0;
}

const char* pamo_last_error(void) { return g_err.c_str(); }

pamo_status pamo_release_cached_memory(void) { return release_cached_memory(); }

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
  PAMO_TRY(enter(c));
  pamo_status s = round_cost(c);
  join(c);
  return s;
}

pamo_status pamo_round_select(pamo_ctx* c, int64_t* n_winners) {
  CTX_GUARD(c);
  PAMO_TRY(enter(c));
  pamo_status s = round_select(c);
  join(c);
  if (s == PAMO_OK && n_winners) *n_winners = c->nW;
  return s;
}

pamo_status pamo_round_collapse(pamo_ctx* c) {
  CTX_GUARD(c);
  PAMO_TRY(enter(c));
  pamo_status s = round_collapse(c);
  join(c);
  return s;
}

pamo_status pamo_round_check_undo(pamo_ctx* c, int32_t* undo_iters) {
  CTX_GUARD(c);
  PAMO_TRY(enter(c));
  pamo_status s = round_check_undo(c);
  join(c);
  if (s == PAMO_OK && undo_iters) *undo_iters = c->undo_iters;
  return s;
}

pamo_status pamo_round_commit(pamo_ctx* c, int64_t* nF_now) {
  CTX_GUARD(c);
  PAMO_TRY(enter(c));
  pamo_status s = round_commit(c);
  join(c);
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
  PAMO_TRY(enter(c));
  if (d_V && d_F) PAMO_TRY(store_mesh(c->pos, c->nV, c->F, c->nF, d_V, d_F, c->st));
  if (d_keys)
    PAMO_CUDA(cudaMemcpyAsync(d_keys, c->key, sizeof(uint64_t) * c->nE, cudaMemcpyDeviceToDevice,
                              c->st));
  if (d_edges)
    PAMO_CUDA(cudaMemcpyAsync(d_edges, c->E, sizeof(int2) * c->nE, cudaMemcpyDeviceToDevice, c->st));
  PAMO_CUDA(cudaStreamSynchronize(c->st));
  return join(c);
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

pamo_status pamo_ctx_winner_features(pamo_ctx* c, float* d_X) {
  CTX_GUARD(c);
  if (c->stage != 2 || !d_X) {
    set_error("pamo_ctx_winner_features: call after pamo_round_select, with an output");
    return PAMO_EINVAL;
  }
  PAMO_TRY(enter(c));
  PAMO_TRY(edge_features_list(c, c->wlist, &c->dc->nW, d_X, c->st));
  PAMO_CUDA(cudaStreamSynchronize(c->st));
  return join(c);
}

pamo_status pamo_ctx_winner_standing(pamo_ctx* c, uint8_t* d_out) {
  CTX_GUARD(c);
  if (c->stage != 4 || !d_out) {
    set_error("pamo_ctx_winner_standing: call after pamo_round_check_undo, with an output");
    return PAMO_EINVAL;
  }
  PAMO_TRY(enter(c));
  if (c->nW > 0)
    PAMO_CUDA(cudaMemcpyAsync(d_out, c->standing, (size_t)c->nW, cudaMemcpyDeviceToDevice, c->st));
  PAMO_CUDA(cudaStreamSynchronize(c->st));
  return join(c);
}

pamo_status pamo_ctx_set_deferrals(pamo_ctx* c, const int64_t* h_off, int64_t n_rounds,
                                   const int32_t* h_pairs) {
  CTX_GUARD(c);
  if (n_rounds < 0 || (n_rounds > 0 && (!h_off || (h_off[n_rounds] > 0 && !h_pairs)))) {
    set_error("pamo_ctx_set_deferrals: offsets (n_rounds + 1) and pairs required");
    return PAMO_EINVAL;
  }
  if (c->rounds != 0 || c->stage != 0 || c->n_mesh > 1 || c->opt.proposal) {
    set_error("pamo_ctx_set_deferrals: a single-mesh context without a learned proposal, "
              "before its first round");
    return PAMO_EINVAL;
  }
  std::vector<int64_t> off(h_off, h_off + n_rounds + 1);
  int64_t widest = 0;
  for (int64_t r = 0; r < n_rounds; r++) {
    if (off[r + 1] < off[r] || off[0] != 0) {
      set_error("pamo_ctx_set_deferrals: offsets must start at 0 and not decrease");
      return PAMO_EINVAL;
    }
    widest = std::max(widest, off[r + 1] - off[r]);
  }
  if (widest > c->Emax) {
    set_error("pamo_ctx_set_deferrals: more pairs in a round than the mesh has edges");
    return PAMO_EINVAL;
  }
  std::vector<unsigned long long> keys(n_rounds > 0 ? (size_t)off[n_rounds] : 0);
  for (size_t i = 0; i < keys.size(); i++) {
    const int32_t a = h_pairs[2 * i], b = h_pairs[2 * i + 1];
    if (a < 0 || b <= a) {
      set_error("pamo_ctx_set_deferrals: pairs must be (a, b) with 0 <= a < b");
      return PAMO_EINVAL;
    }
    keys[i] = ((unsigned long long)(unsigned)a << 32) | (unsigned)b;
  }
  for (int64_t r = 0; r < n_rounds; r++)
    std::sort(keys.begin() + off[r], keys.begin() + off[r + 1]);
  PAMO_TRY(enter(c));
  pamo_status s = PAMO_OK;
  if (!c->pkeep) s = alloc(&c->pkeep, (size_t)c->Emax, c->st);
  if (s == PAMO_OK && c->dsched) release(c->dsched, c->st);
  if (s == PAMO_OK && c->dsched_off) release(c->dsched_off, c->st);
  if (s == PAMO_OK) s = alloc(&c->dsched, std::max<size_t>(keys.size(), 1), c->st);
  if (s == PAMO_OK) s = alloc(&c->dsched_off, (size_t)n_rounds + 1, c->st);
  if (s == PAMO_OK) {
    cudaError_t e = cudaSuccess;
    if (!keys.empty())
      e = cudaMemcpyAsync(c->dsched, keys.data(), sizeof(unsigned long long) * keys.size(),
                          cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->dsched_off, off.data(), sizeof(int64_t) * off.size(),
                          cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);  // the host arrays are locals
    if (e != cudaSuccess) s = cuda_fail(e, "pamo_ctx_set_deferrals: upload");
  }
  if (s == PAMO_OK) {
    c->n_sched = (int)n_rounds;
    c->sched_on = true;
  }
  pamo_status j = join(c);
  return s != PAMO_OK ? s : j;
}

pamo_status pamo_ctx_rounds(const pamo_ctx* c, int64_t* rounds) {
  CTX_GUARD(c);
  if (rounds) *rounds = c->rounds;
  return (pamo_status)c->status;
}

pamo_status pamo_ctx_run(pamo_ctx* c, int64_t target, pamo_stats* stats) {
  CTX_GUARD(c);
  PAMO_TRY(enter(c));
  EventPair ev;
  PAMO_CUDA(ev.create());
  PAMO_CUDA(cudaEventRecord(ev.a, c->st));
  const long long l0 = launch_count() - c->gk_run + c->gk_captured;
  pamo_status s = run(c, target);
  cudaError_t e = cudaEventRecord(ev.b, c->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev.b);
  if (e != cudaSuccess) {
    join(c);
    return cuda_fail(e, "pamo_ctx_run: synchronisation");
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev.a, ev.b);
  kc_resolve(c);
  fill_stats(c, stats, ms);
  // kernels that ran: eager launches plus the kernel nodes of each replay
  if (stats) stats->launches = launch_count() - c->gk_captured + c->gk_run - l0;
  join(c);
  if (s != PAMO_OK) return s;
  return (pamo_status)c->status;
}

void pamo_ctx_destroy(pamo_ctx* c) {
  if (!c) return;
  join(c);
  destroy_ctx(c);
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
  EventPair ev;
  PAMO_CUDA(ev.create());
  PAMO_CUDA(cudaEventRecord(ev.a, st));
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  pamo_ctx* c = nullptr;
  const long long l0 = launch_count();
  pamo_status s = create(d_V, nV, d_F, nF, opt, st, &c);
  if (s == PAMO_OK) s = run(c, target);
  if (s == PAMO_OK) s = store_mesh(c->pos, c->nV, c->F, c->nF, d_Vout, d_Fout, c->st);
  if (s == PAMO_OK) s = join(c);
  float ms = 0.f;
  if (s == PAMO_OK) {  // the output copy's errors surface here
    cudaError_t e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) s = cuda_fail(e, "pamo_simplify: final synchronisation");
  }
  if (s == PAMO_OK) {
    cudaEventElapsedTime(&ms, e0, e1);
    *nV_out = c->nV;
    *nF_out = c->nF;
    kc_resolve(c);
    fill_stats(c, stats, ms);
    if (stats) stats->launches = launch_count() - c->gk_captured + c->gk_run - l0;
    s = (pamo_status)c->status;
  }
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
  if (s == PAMO_OK) {
    cudaError_t e = cudaMemsetAsync(dc, 0, sizeof(RoundCounters), st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemsetAsync");
  }
  // every face index is checked against [0, nV) before anything reads the mesh
  if (s == PAMO_OK) s = load_mesh_checked(d_V, nV, d_F, nF, pos, F, &dc->bad, st);
  float lo[3], hi[3];
  if (s == PAMO_OK) s = mesh_bbox(pos, nV, lo, hi, tmp, st);
  if (s == PAMO_OK) s = bvh_alloc(b, (int)nF, st);
  if (s == PAMO_OK)
    s = bvh_build(b, pos, F, nullptr, nullptr, (int)nF, lo, hi, false, default_grid(), st);
  if (s == PAMO_OK)
    s = bvh_check(b, pos, F, nullptr, nullptr, 1, nullptr, nullptr, 0, nullptr, dc, d_pairs, cap,
                  (int)nF, st);
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

pamo_status pamo_simplify_batch(int32_t n_meshes, const float* d_V, const int64_t* h_voff,
                                const int32_t* d_F, const int64_t* h_foff,
                                const int64_t* h_targets, const pamo_options* opt, void* stream,
                                float* d_Vout, int64_t* h_voff_out, int32_t* d_Fout,
                                int64_t* h_foff_out, int32_t* h_status, int32_t* h_rounds,
                                pamo_stats* stats) {
  if (!d_Vout || !d_Fout || !h_voff_out || !h_foff_out) {
    set_error("output arguments must not be NULL");
    return PAMO_EINVAL;
  }
  if (n_meshes == 1 && h_voff && h_foff && h_targets) {  // one mesh: the plain path
    if (h_voff[0] != 0 || h_foff[0] != 0) {
      set_error("batch: offsets must start at 0");
      return PAMO_EINVAL;
    }
    pamo_stats local;
    int64_t nvo = 0, nfo = 0;
    pamo_status s = pamo_simplify(d_V, h_voff[1], d_F, h_foff[1], h_targets[0], opt, stream,
                                  d_Vout, &nvo, d_Fout, &nfo, &local);
    if (s != PAMO_OK && s != PAMO_ESTALL) return s;
    h_voff_out[0] = 0;
    h_voff_out[1] = nvo;
    h_foff_out[0] = 0;
    h_foff_out[1] = nfo;
    if (h_status) h_status[0] = s;
    if (h_rounds) h_rounds[0] = local.rounds;
    if (stats) *stats = local;
    return s;
  }
  cudaStream_t st = (cudaStream_t)stream;
  EventPair ev;
  PAMO_CUDA(ev.create());
  PAMO_CUDA(cudaEventRecord(ev.a, st));
  cudaEvent_t e0 = ev.a, e1 = ev.b;
  pamo_ctx* c = nullptr;
  const long long l0 = launch_count();
  pamo_status s = create_batch(n_meshes, d_V, h_voff, d_F, h_foff, h_targets, opt, st, &c);
  if (s == PAMO_OK) s = run_batch(c);
  if (s == PAMO_OK) {
    const int M = c->n_mesh;
    std::vector<int32_t> vb(M);
    h_voff_out[0] = 0;
    h_foff_out[0] = 0;
    for (int m = 0; m < M; m++) {
      vb[m] = (int32_t)h_voff_out[m];
      h_voff_out[m + 1] = h_voff_out[m] + c->m_nV[m];
      h_foff_out[m + 1] = h_foff_out[m] + c->m_nF[m];
      if (h_status) h_status[m] = c->m_status[m];
      if (h_rounds) h_rounds[m] = c->m_rounds[m];
    }
    cudaError_t e = cudaMemcpyAsync(c->mvbase, vb.data(), sizeof(int32_t) * M,
                                    cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) s = cuda_fail(e, "cudaMemcpyAsync vertex bases");
  }
  if (s == PAMO_OK)
    s = store_mesh_batch(c->pos, c->nV, c->F, c->nF, c->vmesh, c->mvbase, d_Vout, d_Fout, c->st);
  if (s == PAMO_OK) s = join(c);
  if (s == PAMO_OK) {  // the output copy's errors surface here
    cudaError_t e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) s = cuda_fail(e, "pamo_simplify_batch: final synchronisation");
  }
  if (s == PAMO_OK) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    kc_resolve(c);
    fill_stats(c, stats, ms);
    if (stats) stats->launches = launch_count() - c->gk_captured + c->gk_run - l0;
    s = (pamo_status)c->status;
  }
  if (c) pamo_ctx_destroy(c);
  return s;
}

pamo_status pamo_autotune_batch(int32_t n_meshes, const float* d_V, const int64_t* h_voff,
                                const int32_t* d_F, const int64_t* h_foff,
                                const int64_t* h_targets, const pamo_options* base,
                                void* stream, pamo_options* best, double* h_ms,
                                int32_t* n_trials) {
  if (!best || n_meshes < 1 || !h_voff || !h_foff || !h_targets) {
    set_error("autotune: need the batch description and an output");
    return PAMO_EINVAL;
  }
  pamo_options b;
  if (base) b = *base;
  else pamo_default_options(&b);
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t nV = h_voff[n_meshes], nF = h_foff[n_meshes];
  float* dVo = nullptr;
  int32_t* dFo = nullptr;
  pamo_status s = alloc(&dVo, 3 * nV, st);
  if (s == PAMO_OK) s = alloc(&dFo, 3 * nF, st);
  std::vector<int64_t> vo(n_meshes + 1), fo(n_meshes + 1);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (s == PAMO_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
    set_error("autotune: cudaEventCreate");
    s = PAMO_ECUDA;
  }
  auto trial = [&](const pamo_options& o, double* ms) -> pamo_status {
    cudaEventRecord(e0, st);
    pamo_status r = pamo_simplify_batch(n_meshes, d_V, h_voff, d_F, h_foff, h_targets, &o, stream,
                                        dVo, vo.data(), dFo, fo.data(), nullptr, nullptr, nullptr);
    if (r != PAMO_OK && r != PAMO_ESTALL) return r;
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    *ms = t;
    return PAMO_OK;
  };
  int nt = 0;
  double best_ms = 1e300, t = 0.0;
  pamo_options cur = b;
  cur.grid_blocks_per_sm = 6;
  cur.resort_percent = 25;
  pamo_options chosen = cur;
  if (s == PAMO_OK) s = trial(cur, &t);  // warm-up (allocator pool, module load)
  static const int kResort[4] = {25, 50, 75, 100};
  for (int i = 0; i < 4 && s == PAMO_OK; i++) {
    cur.resort_percent = kResort[i];
    s = trial(cur, &t);
    if (s == PAMO_OK) {
      if (h_ms) h_ms[nt] = t;
      nt++;
      if (t < best_ms) {
        best_ms = t;
        chosen = cur;
      }
    }
  }
  static const int kGrid[2] = {4, 8};
  cur = chosen;
  for (int i = 0; i < 2 && s == PAMO_OK; i++) {
    cur.grid_blocks_per_sm = kGrid[i];
    s = trial(cur, &t);
    if (s == PAMO_OK) {
      if (h_ms) h_ms[nt] = t;
      nt++;
      if (t < best_ms) {
        best_ms = t;
        chosen = cur;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  release(dVo, st);
  release(dFo, st);
  cudaStreamSynchronize(st);
  if (s != PAMO_OK) return s;
  *best = chosen;
  if (n_trials) *n_trials = nt;
  return PAMO_OK;
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
