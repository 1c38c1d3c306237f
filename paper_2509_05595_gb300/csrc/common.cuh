// Internal declarations of the sm_103a simplifier (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pamo.h"

namespace pamo {

constexpr int kBlock = 256;
// Blocks of the kernels with long per-item work (edge costs, the exact pair
// test): small blocks spread a small round's items over every SM instead of
// packing them into a few 256-thread blocks, at the same occupancy.
constexpr int kItemBlock = 64;

// Tile sizes shared by the scans (scan.cu), the LBVH radix sort (bvh.cu) and
// the fixed scratch layout of the allocation-free check (noalloc.cu).
constexpr int kScanTile = kBlock * 8;   // items per block of a prefix scan
constexpr int kSortTile = kBlock * 16;  // keys per block of a radix-sort pass

// Algorithmic float64 flops of the edge cost (Eq. 1), for the roofline (a
// fused multiply-add counts 2, a division or a square root 1): per evaluated
// edge, the quadric sum, the 3x3 Cramer solve, the quadric at the placement,
// the edge length and the weighted sum (114); per produced triangle, the
// edge differences, the cross product and its length, the three squared
// edge lengths, the quotient and the running sum of 1 - C_ijk (45).
constexpr double kCostFlopsEdge = 114.0;
constexpr double kCostFlopsTri = 45.0;

// ----------------------------------------------------------------------------
// error plumbing: every host helper returns pamo_status; the message is kept
// per thread and surfaced by pamo_last_error().
// ----------------------------------------------------------------------------
void set_error(const std::string& msg);
// process-wide count of kernels launched by this library
void note_launch();
long long launch_count();
pamo_status cuda_fail(cudaError_t e, const char* what);

#define PAMO_CUDA(call)                                     \
  do {                                                      \
    cudaError_t e__ = (call);                               \
    if (e__ != cudaSuccess) return ::pamo::cuda_fail(e__, #call); \
  } while (0)

#define PAMO_TRY(call)                           \
  do {                                           \
    pamo_status s__ = (call);                    \
    if (s__ != PAMO_OK) return s__;              \
  } while (0)

// fixed grid of the standalone intersection check's kernels: 4 blocks per SM
int default_grid();
int sm_count();

// Grid of a latency-bound grid-stride kernel: as many blocks of kBlock threads
// as the SMs hold at once (one full wave), so that no block runs in a second,
// partial wave.  Evaluated once per kernel (static at the call site).
template <typename K>
int occ_grid(K kernel, int block = kBlock) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, block, 0) != cudaSuccess || b < 1)
    b = 1;
  return b * sm_count();
}

inline unsigned grid_for(int64_t n, int block = kBlock) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Device-resident state of a simplification: the mesh sizes (maintained on
// the device so that a whole round can be replayed as a CUDA graph) and the
// counters of the current round.  Mirrored to pinned host memory at each
// synchronisation.
struct RoundCounters {
  // ---- persistent
  int nV, nF, nE;           // current mesh M_1
  int nflags;               // entries of the invalid-edge flag list
  int have_prev;            // last round's edge costs can be reused
  int nV_edges;             // vertex count the edge offsets were built for
  int target;               // N_t of the running simplification
  unsigned max_bits;        // float bits of the target edge cost (0x7f800000 = off)
  int last_committed;       // collapses committed by the last round (1 at the start)
  int round_no;             // rounds started (k_save_prev counts them)
  // ---- zeroed at the start of every round (from link_rejects on)
  unsigned long long link_rejects, flagged, eligible;
  unsigned long long cost_tris;  // triangles produced, summed over evaluated edges
  int nW, n_pairs, n_undo, n_undone_total, overflow, bad, n_query, n_dirty;
  int ncand[3];
  int cand_overflow;        // a candidate bucket overflowed: undo waits for the fused check
  int nund, committed;      // undone / committed collapses (set by the commit)
  int clean;                // last check found no pair: the commit may run
  int ne_actual;            // edges written by the edge pass (must be 3F/2)
  int pairs_total, undo_iters;
  int go;                   // commit gate: 1 when the last check was clean
  int goV, goF, goW;        // gated sizes for the commit (0 when not committing)
  int goVn, goFn;           // gated sizes of the committed mesh
  int cost_f64;             // edges whose key came from the float64 skinny sum
  int deferred;             // edges deferred by the learned proposal
  int n_listed;             // eligible edges listed for the proposal
  // faces restored by undos this round (rlist): [rest_lo, rest_mid) are the
  // queries of the current re-check, rest_end the append position
  int rest_lo, rest_mid, rest_end;
};

#define PAMO_ROUND_ZERO_OFFSET offsetof(::pamo::RoundCounters, link_rejects)
static_assert((sizeof(RoundCounters) - PAMO_ROUND_ZERO_OFFSET) % 4 == 0 &&
                  (sizeof(RoundCounters) - PAMO_ROUND_ZERO_OFFSET) / 4 <= 256,
              "the round's counters are zeroed by one block, one word per thread");

// State of the device-side round loop (loop.cu): its inputs, the running
// Section 5.3 bookkeeping and the totals the host reads after the graph.
struct LoopState {
  // inputs
  int target, max_rounds, stall_limit, tolerance, resort_pct, cost_target, sort_first;
  // running state
  int rounds, hold, zero_streak, order_ok, n_sorted, nflags_in, iter;
  int status, error, stall_empty;
  int nW, nE, undo_iters;
  // totals since the loop started
  long long committed, undone, link, winners, cost_edges, cost_tris, cost_f64, deferred, pairs;
  long long sorts, rechecks, fallbacks;
  long long undo_hist[8];
};

// Per-mesh state of a batch in the device-side round loop: the sizes, the
// Section 5.3 bookkeeping and the outcome of every mesh.
struct MeshState {
  long long nV, nF, target;
  int nflags, hold, zero, status, rounds, active, mode;
};

// Element count of a launch: the device value when n_dev is set, else n_host.
__device__ __forceinline__ int dev_n(const int* n_dev, int n_host) {
  return n_dev ? *n_dev : n_host;
}

// Scratch buffer owned by a context, grown on demand (stream-ordered).
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};
pamo_status buf_reserve(Buf& b, size_t bytes, cudaStream_t st);
void buf_free(Buf& b, cudaStream_t st);

// Linear BVH over the faces of a mesh (Karras 2012).  Internal nodes only,
// 64 bytes each (both child boxes and links; leaves are encoded as ~face).
// vals/keys hold the leaf order (face ids) and Morton keys.
struct Bvh {
  int n_max = 0;                 // capacity the buffers were allocated for
  Buf nodes, parent, flags, keys, vals, keys2, vals2, hist, face_aux, sort_len, sums;
  Buf posn;  // [n_max+1] new leaf positions of a compaction
  // many meshes in one tree (a batch): the mesh id of each leaf (high key
  // word, sorted order) and each mesh's subtree root; vmesh maps a vertex to
  // its mesh and mframe holds each mesh's Morton frame (lo.xyz, 1/extent.xyz)
  int n_mesh = 1;
  Buf hkeys, hkeys2, mroot;
  const int32_t* vmesh = nullptr;
  const float* mframe = nullptr;
  uint32_t* vgap = nullptr;  // per-vertex clearance of non-adjacent overlapping pairs (may be null)
  // leaf order carried over rounds: valid when order_ok; re-sorted by Morton
  // code when the face count has fallen below resort_percent (default 25) of
  // the count at the last sort
  bool order_ok = false;
  int n_sorted = 0;
};

struct RoundRecord {
  int64_t info[12];
  std::vector<int32_t> win, com, und;
};

}  // namespace pamo

// The context (opaque to C callers).
struct pamo_ctx {
  // the context works on its own stream (graph capture needs a non-default
  // stream); it is ordered after the caller's stream at creation and the
  // caller's stream waits for it at the end of every entry point
  cudaStream_t st = nullptr;
  cudaStream_t ust = nullptr;          // the caller's stream
  cudaEvent_t join_ev = nullptr;
  pamo_options opt{};
  int64_t nV0 = 0, nF0 = 0, Emax = 0;
  int64_t nV = 0, nF = 0, nE = 0;     // current M_1 sizes
  int64_t nW = 0;                      // winners this round
  int undo_iters = 0;
  int64_t last_pairs = 0;              // intersecting pairs found this round
  bool stalled = false;
  bool stall_empty = false;            // stopped because nothing was eligible
  bool in_run = false;                 // inside pamo_simplify / pamo_ctx_run
  double scale = 1.0;                  // 1 / max bbox extent of the input
  float bb_lo[3], bb_hi[3];            // input bounding box (Morton frame)
  int stage = 0;                       // 0 idle, 1 costed, 2 selected, 3 collapsed, 4 checked
  int status = PAMO_OK;                // PAMO_ESTALL once stalled
  // --- M_1 (current mesh) and M_s (tentative mesh of this round)
  float4* pos = nullptr;   float4* pos_s = nullptr;   // [nV0]
  double* K = nullptr;     double* K_s = nullptr;     // [nV0][10]
  int4* F = nullptr;       int4* F_s = nullptr;       // [nF0]
  // --- adjacency of M_1: faces around each vertex, ascending face id
  int32_t* vf_off = nullptr;  // [nV0+1]
  int32_t* vf_idx = nullptr;  // [3 nF0]
  int32_t* vf_nbr = nullptr;  // [3 nF0] per vertex segment: its higher neighbours, ascending
  int32_t* vcount = nullptr;  // [nV0+1] scratch counts / cursors
  // --- edges of M_1 (sorted unique (a<b) pairs) and their keys
  int2* E = nullptr;          // [Emax]
  int32_t* e_off = nullptr;   // [nV0+1]
  // --- previous round's edge data, reused for edges whose inputs did not
  // change (cost is a pure function of the edge's two vertex rings)
  int2* E_prev = nullptr;              // [Emax]
  int32_t* e_off_prev = nullptr;       // [nV0+1]
  uint32_t* cbits = nullptr;           // [Emax] float bits of the cost (~0 = non-finite)
  uint32_t* cbits_prev = nullptr;      // [Emax]
  float4* vbar_prev = nullptr;         // [Emax]
  uint8_t* link = nullptr;             // [Emax] link condition holds
  uint8_t* link_prev = nullptr;        // [Emax]
  int32_t* ivmap = nullptr;            // [nV0] new vertex id -> previous id
  uint8_t* vsurv = nullptr;            // [nV0] survivor of a committed collapse
  uint8_t* vdirty = nullptr;           // [nV0] survivor or neighbour of one
  uint32_t* vgap = nullptr;            // [nV0] float bits: smallest distance to a
                                       // non-adjacent face with an overlapping box
                                       // in the last check (+inf: none)
  uint32_t* vgap_tmp = nullptr;        // [nV0] compaction scratch
  // learned proposal (when options.proposal is set)
  float* pX = nullptr;                 // [Emax][16] winner features
  float* pprob = nullptr;              // [Emax] predicted probability of an undo
  uint8_t* pkeep = nullptr;            // [Emax] winner not deferred
  int32_t* rlist = nullptr;            // [nF] faces restored by this round's undos
  // the device-side round loop (loop.cu): its state, the merge buffer of the
  // flags, and the instantiated graph with the kernels of each of its parts
  pamo::LoopState* loop = nullptr;     // device
  pamo::LoopState* loop_h = nullptr;   // pinned host mirror
  unsigned long long* flags_tmp = nullptr;
  pamo::MeshState* mstate = nullptr;   // [n_mesh] device (a batch)
  pamo::MeshState* mstate_h = nullptr; // pinned host mirror
  cudaGraphExec_t gL = nullptr;
  long long gL_nodes[5] = {0, 0, 0, 0, 0};  // round, sort build, carry build, recheck, fallback
  // deferral schedule (pamo_ctx_set_deferrals) on the device: keys
  // (a << 32 | b, sorted within a round) and n_sched + 1 round offsets
  unsigned long long* dsched = nullptr;
  int64_t* dsched_off = nullptr;
  int n_sched = 0;
  bool sched_on = false;
  int64_t deferred_total = 0;
  cudaEvent_t round_ev[2] = {nullptr, nullptr};  // device time of a round (records)
  int64_t last_round_us = 0;
  int64_t cost_edges_total = 0;        // dirty edges evaluated by k_edge_cost
  int64_t cost_f64_total = 0;          // of those, keys from the float64 skinny sum
  int32_t* dlist = nullptr;            // [Emax] edges whose cost is recomputed
  bool have_prev = false;
  unsigned long long* key = nullptr;   // [Emax]
  float4* vbar = nullptr;     // [Emax]
  unsigned long long* vkey = nullptr;  // [nV0]
  uint8_t* win = nullptr;     // [Emax] winner flag -> scan input
  int32_t* wscan = nullptr;   // [Emax+1]
  int32_t* wlist = nullptr;   // [Emax] winner edge ids (ascending)
  uint8_t* standing = nullptr;  // [Emax] per winner slot
  uint8_t* undo = nullptr;      // [Emax] per winner slot
  int32_t* ftag = nullptr;      // [nF0] winner slot that rewrote the face
  int32_t* qlist = nullptr;     // [nF0] faces changed this round (query list)
  double* qface = nullptr;      // [10 nF0] face-plane quadrics (recompute_quadrics)
  int2* cand[3] = {nullptr, nullptr, nullptr};  // candidate pairs by shared-vertex count
  int64_t cand_cap[3] = {0, 0, 0};
  int sm_count = 152;
  uint8_t* fdead = nullptr;     // [nF0]
  uint8_t* vdead = nullptr;     // [nV0]
  int32_t* vmap = nullptr;      // [nV0+1]
  int32_t* dbuf = nullptr;      // [max(nV0,nF0)+1] dead-before scan (vertices)
  int32_t* dbufF = nullptr;     // [nF0+1] dead-before scan of the faces
  // --- invalid-edge flags (sorted vertex pairs a<<32|b)
  unsigned long long* flags = nullptr;       // [Emax]
  unsigned long long* flags_next = nullptr;  // [Emax]
  int64_t nflags = 0;
  int hold = 0, zero_streak = 0;
  // --- batch (n_mesh > 1): the union of many meshes, each with its own
  // normalisation, target, flags and termination
  int n_mesh = 1;
  int32_t* vmesh = nullptr;            // [nV0] vertex -> mesh
  int32_t* vmesh_tmp = nullptr;        // [nV0] compaction scratch
  int64_t* voff_d = nullptr;           // [M+1] input vertex offsets
  int64_t* foff_d = nullptr;           // [M+1] input face offsets
  float* mframe = nullptr;             // [M][6] Morton frame (lo, 1/extent)
  double* mcost = nullptr;             // [M][2] s^2, w_e s of Eq. 1
  uint8_t* mactive = nullptr;          // [M] the mesh still simplifies
  int32_t* mcount = nullptr;           // [3M] eligible, committed, undone (per round)
  int32_t* mcount_h = nullptr;         // pinned mirror
  int32_t* mvbase = nullptr;           // [M] output vertex bases
  unsigned long long* flags_old = nullptr;  // [Emax] last flags, committed numbering
  std::vector<int64_t> m_nV, m_nF, m_target, m_nflags;
  std::vector<int> m_hold, m_zero, m_status, m_rounds;
  std::vector<uint8_t> m_active;
  // --- per-round counters
  pamo::RoundCounters* dc = nullptr;    // device
  pamo::RoundCounters* hc = nullptr;    // pinned host mirror
  // --- scratch
  pamo::Buf scan_tmp, quad_tmp;
  int32_t* scan_sums = nullptr;  // tile sums of the device-sized scans
  int32_t* scan_sums2 = nullptr; // three more tile-sum buffers (the commit's batched scans)
  int64_t scan_span = 0;         // words per tile-sum buffer in scan_sums2
  int grid = 608;                // fixed grid of the per-round kernels
  pamo::Bvh bvh;
  // CUDA graphs of a round (A: full round, B: re-check after an undo); [carry]
  cudaGraphExec_t gA[2] = {nullptr, nullptr};
  cudaGraphExec_t gB = nullptr;
  long long gA_launch[2][8] = {{0}}, gB_launch[8] = {0};
  cudaEvent_t gev[3][8][2] = {};  // per graph (A sort, A carry, B), class, begin/end
  long long g_nodes[3] = {0, 0, 0};  // kernels in each graph
  // kernels counted at capture (not run then) and kernels run by replays
  long long gk_captured = 0, gk_run = 0;
  // --- per-kernel-class accounting (pamo_stats.class_*)
  long long kc_launch0[8] = {0};
  cudaEvent_t kc_open[8] = {nullptr};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> kc_pending;
  std::vector<cudaEvent_t> ev_pool;
  double class_ms[8] = {0};
  long long class_launches[8] = {0};
  double class_bytes[8] = {0};
  double class_flops[8] = {0};
  // --- records
  std::vector<pamo::RoundRecord> rec;
  int64_t rounds = 0;
  int64_t committed_total = 0, undone_total = 0, link_total = 0, win_total = 0;
  int32_t undo_hist[8] = {0};
  double bytes_model = 0.0;
};

namespace pamo {

// kernel-class accounting (api.cu): launches between begin/end are charged to
// the class with the given algorithmic bytes; CUDA events time the span when
// the class is in options.profile.
void kc_begin(pamo_ctx* c, int cls);
void kc_end(pamo_ctx* c, int cls, double bytes);
void kc_resolve(pamo_ctx* c);

// scan.cu -------------------------------------------------------------------
// Exclusive prefix sum of n int32 (or uint8 flags) into out[0..n]; out[n] is
// the total.  Deterministic.  n is read from device memory; the caller gives
// the tile-sum buffer (scan_sums_count(n_max) words) and a fixed grid.
int64_t scan_sums_count(int64_t n);
pamo_status scan_dev_i32(const int32_t* in, const int* n_dev, int32_t* out, int32_t* sums, int grid,
                         cudaStream_t st);
pamo_status scan_dev_u8(const uint8_t* in, const int* n_dev, int32_t* out, int32_t* sums, int grid,
                        cudaStream_t st);
// Up to kMaxScanSegs independent byte scans in one set of three launches.
// Item j of a segment is in[j] (in[gather[j]] when gather is set), counted as
// itself or, with invert, as 1 for a zero byte; out[0..n] as above, n from
// the device; each segment has its own tile-sum buffer.
struct ScanSeg {
  const uint8_t* in;
  const int32_t* gather;
  const int* n;
  int32_t* out;
  int32_t* sums;
  int invert;
};
constexpr int kMaxScanSegs = 4;
pamo_status scan_dev_u8_multi(const ScanSeg* segs, int count, int grid, cudaStream_t st);

// mesh.cu -------------------------------------------------------------------
pamo_status mesh_bbox(const float4* pos, int64_t nV, float lo[3], float hi[3],
                      Buf& tmp, cudaStream_t st);
pamo_status mesh_bbox_into(const float4* pos, int64_t nV, unsigned* d_tmp, float lo[3],
                           float hi[3], cudaStream_t st);
pamo_status validate_mesh(pamo_ctx* c);
pamo_status build_vertex_faces(pamo_ctx* c, bool neighbours = false);
pamo_status build_edges(pamo_ctx* c);
pamo_status save_prev(pamo_ctx* c);
pamo_status init_quadrics(pamo_ctx* c);
pamo_status recompute_quadrics(pamo_ctx* c);
pamo_status commit_compact(pamo_ctx* c);
pamo_status commit_sizes(pamo_ctx* c);
pamo_status load_mesh(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                      float4* pos, int4* F, cudaStream_t st);
// load_mesh that also checks every face index against [0, nV): synchronises
// `st` once and returns PAMO_EINVAL before anything reads the mesh when an
// index is out of range (d_bad: one device int of scratch)
pamo_status load_mesh_checked(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                              float4* pos, int4* F, int* d_bad, cudaStream_t st);
pamo_status store_mesh(const float4* pos, int64_t nV, const int4* F, int64_t nF,
                       float* d_V, int32_t* d_F, cudaStream_t st);
// batches: the union of M meshes (vertex / face offsets on the device)
pamo_status load_mesh_batch(const float* d_V, int64_t nV, const int32_t* d_F, int64_t nF,
                            const int64_t* d_voff, const int64_t* d_foff, int M, float4* pos,
                            int4* F, int32_t* vmesh, int* d_bad, cudaStream_t st);
pamo_status mesh_bbox_batch(const float4* pos, const int64_t* d_voff, int M, unsigned* d_out,
                            float* lo, float* hi, cudaStream_t st);
pamo_status store_mesh_batch(const float4* pos, int64_t nV, const int4* F, int64_t nF,
                             const int32_t* vmesh, const int32_t* d_vbase, float* d_V,
                             int32_t* d_F, cudaStream_t st);

// cost.cu -------------------------------------------------------------------
pamo_status edge_costs(pamo_ctx* c);

// propose.cu / mlp.cu: the learned proposal
pamo_status propose(pamo_ctx* c);
// marks the winners named by the deferral schedule for this round as deferred
// kernels of the device-side round loop (loop.cu)
pamo_status loop_init(pamo_ctx* c, cudaGraphConditionalHandle h_sort);
pamo_status loop_cond_fallback(pamo_ctx* c, cudaGraphConditionalHandle h, int first);
pamo_status loop_cond_undo(pamo_ctx* c, cudaGraphConditionalHandle h);
pamo_status loop_finish(pamo_ctx* c, cudaGraphConditionalHandle h_round,
                        cudaGraphConditionalHandle h_sort);
pamo_status defer_scheduled(pamo_ctx* c);
pamo_status edge_features_list(pamo_ctx* c, const int32_t* list, const int* n_dev, float* X,
                               cudaStream_t st);
pamo_status mlp_forward_dev(const pamo_mlp* m, const float* X, const int* n_dev, float* prob,
                            int64_t n_max, cudaStream_t st);

// select.cu -----------------------------------------------------------------
pamo_status select_winners(pamo_ctx* c);
// exact-target mode: keep the ceil((nF - target) / 2) lowest-key winners
pamo_status trim_winners(pamo_ctx* c);
pamo_status collapse_winners(pamo_ctx* c);
pamo_status undo_marked(pamo_ctx* c);
pamo_status check_result(pamo_ctx* c);

// bvh.cu --------------------------------------------------------------------
pamo_status bvh_alloc(Bvh& b, int n_max, cudaStream_t st);
void bvh_bytes(int n, size_t* nodes, size_t* parent, size_t* flags, size_t* kv, size_t* hist,
               size_t* aux, int64_t* hist_words);
// Build the LBVH over faces [0, n) (n from n_dev, else n_host); dead faces
// (fdead, nullable) get empty boxes; Morton frame [lo, hi].  carry keeps the
// current leaf order (bvh_compact_order) and rebuilds only the hierarchy.
pamo_status bvh_build(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                      const int* n_dev, int n_host, const float lo[3], const float hi[3],
                      bool carry, int grid, cudaStream_t st);
pamo_status bvh_refit(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                      const int* n_dev, int n_host, int grid, cudaStream_t st);
// Fused check (host sizes): query live faces (all of them when query_all,
// else qlist[0..*qcount)) against the tree; intersecting pairs mark
// undo[ftag[f]] and undo[ftag[g]] (when tagged and undo is non-null), are
// counted in dc->n_pairs and, when pairs_out is non-null, written (f<g).
pamo_status bvh_check(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                      const int32_t* ftag, int query_all, const int32_t* qlist,
                      const int* qcount, int64_t nq_max, uint8_t* undo, RoundCounters* dc,
                      int32_t* pairs_out, int64_t cap, int n_host, cudaStream_t st);
// The same check in two passes (device sizes): traversal appends candidate
// pairs into three buckets (by shared-vertex count, capacities cap[]), then
// one thread per pair runs the exact test.  A bucket overflow sets
// dc->cand_overflow; the undo then waits and the caller reruns bvh_check.
pamo_status bvh_check_split(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                            const int32_t* ftag, int query_all, const int32_t* qlist,
                            const int* qcount, uint8_t* undo, RoundCounters* dc, int2* const cand[3],
                            const int64_t cap[3], int* ncand, const int* n_dev, int grid,
                            cudaStream_t st);
// A re-check after an undo (every check iteration after the first): the
// faces the last undo restored (rlist[dc->rest_lo, dc->rest_mid) once the
// window is advanced) against the faces of standing collapses, on the tree as
// it was refitted for the first iteration; same candidate buckets and exact
// pair test as bvh_check_split.
pamo_status bvh_recheck_restored(Bvh& b, const float4* pos, const int4* F, const uint8_t* fdead,
                                 const int32_t* ftag, const int32_t* rlist, uint8_t* undo,
                                 RoundCounters* dc, int2* const cand[3], const int64_t cap[3],
                                 int* ncand, const int* n_dev, cudaStream_t st);
// After a commit: keep the leaf order for the compacted faces (stable filter
// of the current order through fdead / dead_before); sizes from the device.
// b.posn must hold the exclusive scan of the live leaves (fdead[vals[i]] == 0,
// i < *n_old_dev), which the commit computes with its other scans.
pamo_status bvh_compact_order(Bvh& b, const uint8_t* fdead, const int32_t* dead_before,
                              const int* n_old_dev, const int* n_new_dev, int grid,
                              cudaStream_t st);
void bvh_free(Bvh& b, cudaStream_t st);
pamo_status tri_batch(const float* P, const int32_t* idx, int64_t n, uint8_t* out,
                      cudaStream_t st);
pamo_status orient3d_batch(const float* P, int64_t n, int8_t* out, cudaStream_t st);
pamo_status orient2d_batch(const float* P, int64_t n, int8_t* out, cudaStream_t st);

}  // namespace pamo
