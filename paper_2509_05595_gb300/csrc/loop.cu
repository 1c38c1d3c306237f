// The rounds of Algorithm 1 as one device-side loop: a CUDA graph whose
// conditional WHILE node repeats the round (cost -> select -> collapse ->
// repeat{check; undo} -> commit), with the decisions the host otherwise makes
// between rounds taken by the small kernels below:
//   * after every check iteration: whether the candidate-overflow fallback
//     runs (an IF node) and whether another undo iteration follows (a nested
//     WHILE node), the iterations bounded by the winners + 2 (Section 5.3's
//     loop ends because M_1 is intersection-free; the bound guards the
//     device against a malformed state);
//   * after the commit: the invalid-edge flags of Section 5.3 (after a round
//     without a commit the undone pairs join the old flags, and after
//     `tolerance` such rounds they are cleared), the stall and target tests,
//     max_rounds, errors, the running totals, and whether the next round
//     re-sorts the LBVH leaves (an IF/ELSE node); for a batch, all of it per
//     mesh, the loop running while any mesh is unfinished.
// Each condition is written by one thread of one kernel with the graph's
// handle (cudaGraphSetConditional).
#include "common.cuh"

namespace pamo {

namespace {

// start of a launch of the loop graph: the first round's BVH build (sort or
// carried order), decided by the host like every round's
__global__ void k_loop_init(const LoopState* __restrict__ ls, cudaGraphConditionalHandle h_sort) {
  cudaGraphSetConditional(h_sort, ls->sort_first ? 1 : 0);
}

// after a check iteration: run the fused fallback check when a candidate
// bucket overflowed.  After a round's first check (first = 1) it also notes
// the round's starting flag count (nothing changes the flags before the
// commit) and starts the undo-iteration count.
__global__ void k_cond_fallback(const RoundCounters* __restrict__ dc, LoopState* __restrict__ ls,
                                cudaGraphConditionalHandle h, int first) {
  if (first) {
    ls->nflags_in = dc->nflags;
    ls->iter = 0;
  }
  const int on = dc->cand_overflow ? 1 : 0;
  ls->fallbacks += on;
  cudaGraphSetConditional(h, on);
}

// after a check iteration and its fallback: another undo iteration while the
// check was not clean
__global__ void k_cond_undo(const RoundCounters* __restrict__ dc, LoopState* __restrict__ ls,
                            cudaGraphConditionalHandle h) {
  int more = dc->clean ? 0 : 1;
  if (more && ++ls->iter > dc->nW + 2) {
    ls->error = PAMO_EINTERNAL;  // the undo loop did not settle
    more = 0;
  }
  ls->rechecks += more;
  cudaGraphSetConditional(h, more);
}

// invalid-edge flags after the commit (Section 5.3).  A committing round has
// already written its undone pairs as the flags (k_undone_pairs); a round
// without a commit merges them into the old flags here (both lists sorted and
// unique; one thread, such rounds are rare and their lists short).
__device__ void flags_merge(RoundCounters* __restrict__ dc, LoopState* __restrict__ ls,
                            unsigned long long* __restrict__ flags,
                            const unsigned long long* __restrict__ fresh,
                            unsigned long long* __restrict__ tmp) {
  if (dc->committed > 0) {
    ls->hold = 0;
    ls->zero_streak = 0;
    return;
  }
  ls->hold++;
  ls->zero_streak++;
  const int na = ls->nflags_in, nb = dc->nund;
  int i = 0, j = 0, n = 0;
  while (i < na || j < nb) {
    unsigned long long x;
    if (j >= nb || (i < na && flags[i] < fresh[j])) {
      x = flags[i++];
    } else if (i >= na || fresh[j] < flags[i]) {
      x = fresh[j++];
    } else {  // in both
      x = flags[i++];
      j++;
    }
    tmp[n++] = x;
  }
  if (ls->hold >= ls->tolerance) {
    n = 0;
    ls->hold = 0;
  }
  for (int k = 0; k < n; k++) flags[k] = tmp[k];
  dc->nflags = n;
}

// end of a round: totals, stop tests, the next round's re-sort decision, and
// the loop's conditions
__global__ void k_round_finish(RoundCounters* __restrict__ dc, LoopState* __restrict__ ls,
                               unsigned long long* __restrict__ flags,
                               const unsigned long long* __restrict__ fresh,
                               unsigned long long* __restrict__ tmp,
                               cudaGraphConditionalHandle h_round,
                               cudaGraphConditionalHandle h_sort) {
  flags_merge(dc, ls, flags, fresh, tmp);
  const int committed = dc->committed, nund = dc->nund;
  ls->committed += committed;
  ls->undone += nund;
  ls->link += (long long)dc->link_rejects;
  ls->winners += dc->nW;
  ls->cost_edges += dc->n_dirty;
  ls->cost_tris += (long long)dc->cost_tris;
  ls->cost_f64 += dc->cost_f64;
  ls->deferred += dc->deferred;
  ls->pairs = dc->pairs_total;
  ls->undo_hist[dc->undo_iters < 7 ? dc->undo_iters : 7]++;
  ls->undo_iters = dc->undo_iters;
  ls->nW = dc->nW;
  ls->nE = dc->nE;
  ls->rounds++;
  int stop = 0;
  if (dc->bad & 64) ls->error = PAMO_ENOTMANIFOLD;
  if (dc->overflow) ls->error = PAMO_EINTERNAL;
  const int nF = dc->nF;
  const bool stall_empty = dc->eligible == 0 && ls->nflags_in == 0;
  if (ls->error) {
    stop = 1;
  } else if (stall_empty || ls->zero_streak >= ls->stall_limit) {
    stop = 1;
    ls->stall_empty = stall_empty ? 1 : 0;
    // with a target edge cost, running out of eligible edges is the normal end
    const bool cost_end = stall_empty && ls->cost_target;
    ls->status = (nF > ls->target && !cost_end) ? PAMO_ESTALL : PAMO_OK;
  } else if (nF <= ls->target) {
    stop = 1;
  } else if (ls->rounds >= ls->max_rounds) {
    stop = 1;
    ls->status = PAMO_ESTALL;
  }
  // the next round keeps the carried leaf order while the face count stays
  // above resort_pct % of the count at the last sort
  int sort = 0;
  if (!stop) {
    const bool carry = ls->order_ok && 100LL * nF > (long long)ls->resort_pct * ls->n_sorted &&
                       ls->resort_pct < 100;
    if (!carry) {
      sort = 1;
      ls->order_ok = 1;
      ls->n_sorted = nF;
      ls->sorts++;
    }
  }
  cudaGraphSetConditional(h_sort, sort);
  cudaGraphSetConditional(h_round, stop ? 0 : 1);
}

// End of a round of a batch: every mesh keeps the rules of a single
// simplification (its own flags, tolerance count, stall, target and status;
// a finished mesh holds no key), so each output equals that mesh simplified
// alone.  One thread per mesh updates its state and the mode of its flags;
// then one thread merges last round's flags (remapped to the new numbering,
// ~0 where a vertex died) with this round's undone pairs, both sorted and
// grouped by mesh (vertex ranges follow the mesh order), keeping per the
// entry's mesh: 0 this round's only, 1 both, 2 and 3 none.
__global__ void __launch_bounds__(256) k_batch_finish(
    RoundCounters* __restrict__ dc, LoopState* __restrict__ ls, MeshState* __restrict__ ms, int M,
    const int32_t* __restrict__ mcount, uint8_t* __restrict__ mactive,
    const unsigned long long* __restrict__ old, const unsigned long long* __restrict__ fresh,
    unsigned long long* __restrict__ flags, const int32_t* __restrict__ vmesh,
    cudaGraphConditionalHandle h_round, cudaGraphConditionalHandle h_sort) {
  __shared__ int any_active;
  if (threadIdx.x == 0) any_active = 0;
  __syncthreads();
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    MeshState s = ms[m];
    const int elig = mcount[m], com = mcount[M + m];
    s.nV -= com;
    s.nF -= 2LL * com;
    int mode = 3;
    if (s.active) {
      if (com > 0) {
        s.hold = 0;
        s.zero = 0;
        mode = 0;
      } else {
        s.hold++;
        s.zero++;
        mode = 1;
        if (s.hold >= ls->tolerance) {
          mode = 2;
          s.hold = 0;
        }
      }
      const bool stall_empty = elig == 0 && s.nflags == 0;
      s.rounds++;
      if (stall_empty || s.zero >= ls->stall_limit) {
        const bool cost_end = stall_empty && ls->cost_target;
        s.status = (s.nF > s.target && !cost_end) ? PAMO_ESTALL : PAMO_OK;
        s.active = 0;
      } else if (s.nF <= s.target) {
        s.active = 0;  // reached N_t
      }
      if (!s.active) mode = 3;
    }
    s.mode = mode;
    s.nflags = 0;
    ms[m] = s;
    if (s.active) atomicOr(&any_active, 1);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const int na = ls->nflags_in, nb = dc->nund;
  int i = 0, j = 0, n = 0;
  for (;;) {
    while (i < na && old[i] == ~0ull) i++;
    if (i >= na && j >= nb) break;
    unsigned long long x;
    bool from_old;
    if (j >= nb || (i < na && old[i] < fresh[j])) {
      x = old[i++];
      from_old = true;
    } else if (i >= na || fresh[j] < old[i]) {
      x = fresh[j++];
      from_old = false;
    } else {  // in both
      x = old[i++];
      j++;
      from_old = false;
    }
    const int m = vmesh[(int)(x >> 32)];
    const int md = ms[m].mode;
    if (md == 1 || (md == 0 && !from_old)) {
      flags[n++] = x;
      ms[m].nflags++;
    }
  }
  dc->nflags = n;
  ls->committed += dc->committed;
  ls->undone += dc->nund;
  ls->link += (long long)dc->link_rejects;
  ls->winners += dc->nW;
  ls->cost_edges += dc->n_dirty;
  ls->cost_tris += (long long)dc->cost_tris;
  ls->cost_f64 += dc->cost_f64;
  ls->pairs = dc->pairs_total;
  ls->undo_hist[dc->undo_iters < 7 ? dc->undo_iters : 7]++;
  ls->undo_iters = dc->undo_iters;
  ls->nW = dc->nW;
  ls->nE = dc->nE;
  ls->rounds++;
  if (dc->bad & 64) ls->error = PAMO_ENOTMANIFOLD;
  if (dc->overflow) ls->error = PAMO_EINTERNAL;
  int stop = ls->error || !any_active;
  if (!stop && ls->rounds >= ls->max_rounds) {  // every unfinished mesh stops above N_t
    stop = 1;
    for (int m = 0; m < M; m++)
      if (ms[m].active) {
        ms[m].active = 0;
        ms[m].status = PAMO_ESTALL;
      }
  }
  for (int m = 0; m < M; m++) mactive[m] = (uint8_t)ms[m].active;
  int sort = 0;
  if (!stop) {
    const int nF = dc->nF;
    const bool carry = ls->order_ok && 100LL * nF > (long long)ls->resort_pct * ls->n_sorted &&
                       ls->resort_pct < 100;
    if (!carry) {
      sort = 1;
      ls->order_ok = 1;
      ls->n_sorted = nF;
      ls->sorts++;
    }
  }
  cudaGraphSetConditional(h_sort, sort);
  cudaGraphSetConditional(h_round, stop ? 0 : 1);
}

}  // namespace

pamo_status loop_init(pamo_ctx* c, cudaGraphConditionalHandle h_sort) {
  k_loop_init<<<1, 1, 0, c->st>>>(c->loop, h_sort); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status loop_cond_fallback(pamo_ctx* c, cudaGraphConditionalHandle h, int first) {
  k_cond_fallback<<<1, 1, 0, c->st>>>(c->dc, c->loop, h, first); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status loop_cond_undo(pamo_ctx* c, cudaGraphConditionalHandle h) {
  k_cond_undo<<<1, 1, 0, c->st>>>(c->dc, c->loop, h); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

pamo_status loop_finish(pamo_ctx* c, cudaGraphConditionalHandle h_round,
                        cudaGraphConditionalHandle h_sort) {
  if (c->n_mesh > 1) {
    k_batch_finish<<<1, 256, 0, c->st>>>(c->dc, c->loop, c->mstate, c->n_mesh, c->mcount,
                                         c->mactive, c->flags_old, c->flags_next, c->flags,
                                         c->vmesh, h_round, h_sort); note_launch();
    PAMO_CUDA(cudaGetLastError());
    return PAMO_OK;
  }
  k_round_finish<<<1, 1, 0, c->st>>>(c->dc, c->loop, c->flags, c->flags_next, c->flags_tmp,
                                     h_round, h_sort); note_launch();
  PAMO_CUDA(cudaGetLastError());
  return PAMO_OK;
}

}  // namespace pamo
