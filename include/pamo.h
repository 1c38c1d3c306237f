/*
 * pamo.h -- C ABI of the GB300 (sm_103a) parallel intersection-free
 * edge-collapse simplifier.
 *
 * The operation is the simplification stage of PaMO (arXiv 2509.05595),
 * Algorithm 1 ("ParallelSimplification") with the edge cost of Eq. 1, the
 * independent-region selection and link condition of Section 5.1, the
 * self-intersection check of Section 5.2 / Algorithm 3 / supplementary
 * Section 3, and the undo loop and invalid-edge flags of Section 5.3.
 *
 * Conventions shared by every entry point
 *   - Array arguments named d_* are DEVICE pointers (CUDA global memory on the
 *     current device); h_* are HOST pointers.  The caller owns every array it
 *     passes; the library never frees or retains caller memory beyond a call,
 *     except the input mesh a context copies at creation.
 *   - Vertices: float32 [nV][3], row-major, x y z.  Faces: int32 [nF][3],
 *     corner indices into the vertex array, counter-clockwise seen from
 *     outside.  The input mesh must be closed, oriented, edge- and
 *     vertex-manifold and free of self-intersections (the problem statement of
 *     Section 3 and Algorithm 1's input); validation of the topology is done
 *     when pamo_options.validate_input is set.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it; calls that return counts to host
 *     memory synchronise that stream before returning.
 *   - Internal scratch comes from the library's stream-ordered memory pool and
 *     goes back to it before the call returns (or in pamo_ctx_destroy for a
 *     context); the pool keeps that memory for later calls until
 *     pamo_release_cached_memory().  Work runs on a stream of the library's
 *     own, ordered after `stream` on entry and joined back into it on exit.
 *   - Errors are reported by return code; nothing aborts.  pamo_last_error()
 *     returns a thread-local message for the last failing call.
 *   - Indices are int32: nF < 2^31 and the edge count (3 nF / 2) < 2^31.
 */
#ifndef PAMO_H
#define PAMO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PAMO_OK = 0,
  PAMO_EINVAL = 1,       /* bad argument or input mesh (message says which) */
  PAMO_ENOMEM = 2,       /* device allocation failed */
  PAMO_ECUDA = 3,        /* a CUDA runtime call failed */
  PAMO_ESTALL = 4,       /* stopped before the target; output is valid */
  PAMO_ETIMEOUT = 5,     /* a device-side bounded wait ran out */
  PAMO_ENOTMANIFOLD = 6, /* input is not a closed oriented manifold */
  PAMO_EINTERNAL = 7,    /* an internal capacity or consistency check failed */
  PAMO_EINTERSECT = 8    /* options.check_input_intersections: the input
                            mesh intersects itself (the method requires an
                            intersection-free input, Section 5) */
} pamo_status;

/* Options.  pamo_default_options() fills the paper's defaults. */
typedef struct {
  double w_e;              /* Eq. 1 length weight, default 0.001 (Sec. 5.1) */
  double w_s;              /* Eq. 1 skinny weight, default 0.005 (Sec. 5.1) */
  int32_t tolerance;       /* flag tolerance in rounds, default 4 (Sec. 5.3) */
  int32_t max_rounds;      /* default 100000; reaching it returns PAMO_ESTALL */
  int32_t stall_limit;     /* consecutive rounds without a committed collapse
                              before PAMO_ESTALL, default 12 */
  int32_t validate_input;  /* 1 = check closed/oriented/manifold/finite, default 1 */
  int32_t check_mode;      /* 0 = check faces changed this round against all
                              faces (default; equivalent to Algorithm 3 on
                              every face because the previous mesh is
                              intersection-free), 1 = every face against every
                              face through the BVH, 3 = no check (debug only:
                              output may self-intersect) */
  int32_t record_rounds;   /* 1 = keep per-round counters and collapse sets for
                              pamo_ctx_round_info / pamo_ctx_round_pairs */
  int32_t profile;         /* bit mask of PAMO_KC_* kernel classes to time with
                              CUDA events (0 = none; timing adds event records) */
  int32_t exact_target;    /* 1 = stop at exactly the target face count where
                              collapses allow it: a round whose winners would
                              remove more faces than |F| - N_t collapses only
                              the ceil((|F| - N_t) / 2) winners with the
                              lowest keys. 0 (default) collapses every winner,
                              as Algorithm 1 does, so |F| may end below N_t */
  double max_cost;         /* target edge cost (Section 5.1 names it as the
                              other termination criterion): an edge whose
                              float cost exceeds it is not eligible, and the
                              run ends with PAMO_OK once no edge is eligible
                              and no flag is pending, even above N_t. Must be
                              >= 0; default +infinity (off) */
  /* Speed-only knobs (the results are identical for every value; chosen by
   * pamo_autotune_batch or left at 0 for the defaults): */
  int32_t grid_blocks_per_sm; /* blocks per SM of the bandwidth-bound
                              grid-stride kernels (0 = 6; 1..32) */
  int32_t resort_percent;  /* the LBVH keeps last round's compacted leaf order
                              until the face count falls below this percent of
                              the count at the last Morton sort (0 = 25;
                              1..100, 100 = sort every round) */
  /* Learned proposal (no counterpart in the paper): a trained pamo_mlp (see
   * below) that predicts, from 16 features of a selected winner, that the
   * intersection check would undo its collapse; such winners are deferred
   * (not collapsed this round; winners are independent, so the others are
   * unaffected), unless the previous round committed nothing.  Every
   * committed collapse still passes the exact check.  NULL = off (default);
   * single-mesh calls only. */
  const struct pamo_mlp* proposal;
  float proposal_threshold; /* defer when the predicted probability exceeds it */
  int32_t check_input_intersections; /* 1 = run the exact self-intersection
                              check (Algorithm 3 over every face) on the input
                              first and refuse a self-intersecting mesh with
                              PAMO_EINTERSECT; 0 (default) trusts the caller */
  int32_t recompute_quadrics; /* 1 = every round starts from the face-plane
                              quadrics of the current mesh (summed in ascending
                              face order) instead of carrying K_a + K_b through
                              collapses (0, the default, standard QEM memory);
                              Eq. 1 cites QEM without fixing this */
  int32_t device_loop;        /* 1 = run all rounds of pamo_simplify /
                              pamo_ctx_run / pamo_simplify_batch as ONE CUDA
                              graph launch: conditional graph nodes repeat the
                              round and the undo iterations, and device kernels
                              keep the Section 5.3 bookkeeping, so the host
                              does not wake between rounds.  Same results.  0
                              (default): one graph launch per round from the
                              host, measured faster on a GB300.  Ignored with
                              record_rounds, profile or check_mode != 0 */
} pamo_options;

/* Kernel classes reported in pamo_stats (index = bit of pamo_options.profile). */
enum {
  PAMO_KC_ADJACENCY = 0, /* vertex->face lists and the canonical edge list */
  PAMO_KC_COST = 1,      /* edge costs, link condition, keys (Eq. 1) */
  PAMO_KC_SELECT = 2,    /* propagation and independent regions (Sec. 5.1) */
  PAMO_KC_COLLAPSE = 3,  /* M_s copy, collapses and undos */
  PAMO_KC_BVH = 4,       /* Morton keys, radix sort, hierarchy, refit */
  PAMO_KC_QUERY = 5,     /* BVH traversal + exact narrow phase (Alg. 3) */
  PAMO_KC_COMMIT = 6,    /* stable compaction and flag list */
  PAMO_KC_COUNT = 8
};

/* Statistics of one simplification (Section 7 reports time, rounds and the
 * undo-iteration histogram of Table 'worst'). */
typedef struct {
  int32_t rounds;
  int32_t undo_iters_hist[8];  /* rounds with 0,1,..,7+ undo iterations */
  int64_t committed, undone, link_rejects, winners;
  int64_t nV_out, nF_out;
  double ms_total;             /* wall time on the stream, CUDA events */
  double bytes_model;          /* algorithmic bytes moved (sum over rounds) */
  int64_t launches;            /* kernels launched by the call */
  /* per kernel class (PAMO_KC_*): event-timed milliseconds (only classes in
   * options.profile), launches, and algorithmic bytes (compulsory reads and
   * writes of each launch's inputs and outputs, summed) */
  double class_ms[8];
  int64_t class_launches[8];
  double class_bytes[8];
  /* algorithmic float64 operations per class (edge cost only: per evaluated
   * edge 114 + 32 per produced triangle, counting +,-,*,/,sqrt as 1 and a
   * fused multiply-add as 2) */
  double class_flops[8];
  int64_t deferred;            /* edges deferred by the learned proposal */
  int64_t cost_edges;          /* edges whose Eq. 1 cost was evaluated (dirty edges) */
  int64_t cost_f64;            /* of those, edges whose key took the float64 skinny sum
                                  (the float-float bound did not decide the float key) */
} pamo_stats;

typedef struct pamo_ctx pamo_ctx;

/* Fill *o with the defaults listed above. */
void pamo_default_options(pamo_options* o);

/* Simplify until the face count is <= target_faces (Algorithm 1, P: while
 * |F(M_1)| > N_t).  Every round collapses all winners, so the result can end
 * below the target.
 *   d_V [nV][3] float32, d_F [nF][3] int32: input mesh (device, read only).
 *   d_Vout >= nV*3 floats, d_Fout >= nF*3 ints: output capacity (device).
 *   *nV_out, *nF_out: output sizes (host).  stats may be NULL.
 * Returns PAMO_OK, or PAMO_ESTALL with a valid (manifold, intersection-free)
 * output larger than the target, or an error with outputs untouched. */
pamo_status pamo_simplify(const float* d_V, int64_t nV, const int32_t* d_F,
                          int64_t nF, int64_t target_faces,
                          const pamo_options* opt, void* stream, float* d_Vout,
                          int64_t* nV_out, int32_t* d_Fout, int64_t* nF_out,
                          pamo_stats* stats);

/* pamo_simplify with HOST arrays: copies the mesh to the device, simplifies,
 * copies the result back (h_Vout >= nV*3, h_Fout >= nF*3).  Synchronous. */
pamo_status pamo_simplify_host(const float* h_V, int64_t nV, const int32_t* h_F,
                               int64_t nF, int64_t target_faces,
                               const pamo_options* opt, void* stream,
                               float* h_Vout, int64_t* nV_out, int32_t* h_Fout,
                               int64_t* nF_out, pamo_stats* stats);

/* Simplify a batch of n_meshes closed manifold meshes in one pass (no
 * counterpart in the paper, which simplifies one mesh at a time): every
 * round of Algorithm 1 runs once over the disjoint union of all meshes, and
 * each mesh keeps its own [0,1]^3 normalisation (Section 4 start), target,
 * invalid-edge flags and tolerance count (Section 5.3) and termination, so
 * the output of every mesh is bit-identical to pamo_simplify on that mesh.
 *   d_V      device, [h_voff[n], 3] float32: the meshes' vertices, concatenated
 *   h_voff   host, n + 1 int64 vertex offsets (h_voff[0] = 0)
 *   d_F      device, [h_foff[n], 3] int32: the meshes' faces, concatenated;
 *            each mesh's faces index its own vertices from 0
 *   h_foff   host, n + 1 int64 face offsets (h_foff[0] = 0)
 *   h_targets host, n target face counts (>= 0)
 * Outputs: d_Vout / d_Fout (device, capacity of the inputs) hold the results
 * in the same layout, with offsets in h_voff_out / h_foff_out (host, n + 1);
 * h_status (host, n, may be NULL) gets PAMO_OK or PAMO_ESTALL per mesh and
 * h_rounds (host, n, may be NULL) the rounds each mesh took.  Returns
 * PAMO_ESTALL if any mesh stalled (all outputs still valid); PAMO_EINVAL for
 * bad sizes, offsets, an index outside its mesh, or options.exact_target;
 * PAMO_ENOTMANIFOLD as pamo_simplify.  Every mesh needs >= 4 vertices and an
 * even face count >= 4; totals below 2^30.  Synchronous on return. */
pamo_status pamo_simplify_batch(int32_t n_meshes, const float* d_V, const int64_t* h_voff,
                                const int32_t* d_F, const int64_t* h_foff,
                                const int64_t* h_targets, const pamo_options* opt, void* stream,
                                float* d_Vout, int64_t* h_voff_out, int32_t* d_Fout,
                                int64_t* h_foff_out, int32_t* h_status, int32_t* h_rounds,
                                pamo_stats* stats);

/* ---- the learned proposal's network (no counterpart in the paper) ----
 * A per-edge MLP 16 -> 64 -> 64 -> 1 (ReLU, ReLU, logistic): BF16 weights
 * (a BF16 copy of FP32 master weights), FP32 accumulation.  Parameters, flat:
 * W1 [16][64] at 0, b1 [64] at 1024, W2 [64][64] at 1088, b2 [64] at 5184,
 * W3 [64] at 5248, b3 at 5312 (W[i][j] maps input i to output j).  Inputs are
 * the 16 edge features of pamo_ctx_winner_features, row-major float32. */
#define PAMO_MLP_IN 16
#define PAMO_MLP_HIDDEN 64
#define PAMO_MLP_PARAMS 5313
typedef struct pamo_mlp pamo_mlp;

/* New network with all parameters zero (device memory, about 120 KB). */
pamo_status pamo_mlp_create(pamo_mlp** out);
void pamo_mlp_destroy(pamo_mlp* m);
/* Set the FP32 master parameters (host, PAMO_MLP_PARAMS floats); refreshes
 * the BF16 copy and resets the Adam state. */
pamo_status pamo_mlp_set_params(pamo_mlp* m, const float* h_params);
/* Standardise the inputs before the first layer: x' = (x - mu) / sd per
 * feature (host, 16 floats each, sd > 0; FP32).  Default mu = 0, sd = 1. */
pamo_status pamo_mlp_set_input_norm(pamo_mlp* m, const float* h_mu, const float* h_sd);
/* Fit that standardisation to training data: mu and sd are the mean and the
 * population standard deviation of each feature over the n rows of d_X
 * (device, n x 16 float32), computed on the device in float64 in a fixed
 * order (deterministic); an sd below 1e-6 is taken as 1.  Synchronises
 * `stream`. */
pamo_status pamo_mlp_fit_input_norm(pamo_mlp* m, const float* d_X, int64_t n, void* stream);
/* Read the master parameters and/or the BF16 copy (host, may be NULL). */
pamo_status pamo_mlp_get_params(const pamo_mlp* m, float* h_params, uint16_t* h_bf16);
/* Probabilities (device, n floats) for n feature rows (device, n x 16). */
pamo_status pamo_mlp_forward(const pamo_mlp* m, const float* d_X, int64_t n, float* d_prob,
                             void* stream);
/* Gradient of the mean weighted binary cross-entropy
 *   -(pos_weight y log p + (1 - y) log(1 - p))
 * over n samples (d_X n x 16, d_y n labels in {0, 1}, device) with respect to
 * the parameters, evaluated with the BF16 weights; kept in the model (see
 * pamo_mlp_get_grad); *h_loss (host, may be NULL) gets the loss.
 * Deterministic (fixed reduction order). */
pamo_status pamo_mlp_grad(pamo_mlp* m, const float* d_X, const float* d_y, int64_t n,
                          float pos_weight, void* stream, float* h_loss);
pamo_status pamo_mlp_get_grad(const pamo_mlp* m, float* h_grad);
/* One Adam step (Kingma & Ba 2015) with the last gradient. */
pamo_status pamo_mlp_adam_step(pamo_mlp* m, float lr, float beta1, float beta2, float eps,
                               void* stream);

/* Autotuner of the speed-only knobs for a batch (no counterpart in the
 * paper): simplifies the given batch (arguments as pamo_simplify_batch) with
 * a sequence of candidate settings -- coordinate descent over resort_percent
 * in {25, 50, 75, 100}, then grid_blocks_per_sm in {4, 6, 8} -- timing each
 * run with CUDA events, and writes the fastest into *best (a copy of *base
 * with the two knobs set).  h_ms (host, may be NULL, capacity 8) receives
 * the time of every trial and *n_trials their number.  Every trial produces
 * the same meshes.  Synchronous; allocates only what pamo_simplify_batch
 * allocates plus the trial outputs. */
pamo_status pamo_autotune_batch(int32_t n_meshes, const float* d_V, const int64_t* h_voff,
                                const int32_t* d_F, const int64_t* h_foff,
                                const int64_t* h_targets, const pamo_options* base,
                                void* stream, pamo_options* best, double* h_ms,
                                int32_t* n_trials);

/* ---- per-round entry points (one round = one iteration of Algorithm 1's
 * while loop) over a context that owns the evolving mesh ---- */

/* Copy the input mesh (device) into a new context; computes vertex quadrics.
 * Returns PAMO_EINVAL / PAMO_ENOTMANIFOLD for bad input. */
pamo_status pamo_ctx_create(const float* d_V, int64_t nV, const int32_t* d_F,
                            int64_t nF, const pamo_options* opt, void* stream,
                            pamo_ctx** out);

/* Edge costs and keys of the current mesh (Eq. 1; Alg. 1 first loop). */
pamo_status pamo_round_cost(pamo_ctx* ctx);

/* Cost propagation and independent-region selection (Sec. 5.1; Alg. 1
 * second loop and the collapse condition).  *n_winners (host) receives the
 * number of selected collapses. */
pamo_status pamo_round_select(pamo_ctx* ctx, int64_t* n_winners);

/* Collapse every selected edge into the tentative mesh M_s (Alg. 1
 * CollapseEdge). */
pamo_status pamo_round_collapse(pamo_ctx* ctx);

/* repeat { IntersectionCheck(M_s); UndoCollapse } until clean (Alg. 1,
 * Sec. 5.2-5.3).  *undo_iters (host, may be NULL) receives the number of undo
 * iterations performed. */
pamo_status pamo_round_check_undo(pamo_ctx* ctx, int32_t* undo_iters);

/* Commit M_s as the next M_1: stable compaction of live vertices and faces,
 * invalid-edge flags for the next round (Sec. 5.3).  *nF_now (host, may be
 * NULL) receives the new face count. */
pamo_status pamo_round_commit(pamo_ctx* ctx, int64_t* nF_now);

/* Current mesh sizes (host). */
pamo_status pamo_ctx_sizes(const pamo_ctx* ctx, int64_t* nV, int64_t* nF,
                           int64_t* nE);

/* Copy the current mesh out (device arrays of capacity >= current sizes).
 * d_keys (nullable, nE uint64) receives the last computed edge keys
 * (cost bits << 32 | edge id, ~0 = ineligible); d_edges (nullable, nE x 2
 * int32) the edge endpoints (sorted unique (min,max) pairs). */
pamo_status pamo_ctx_export(pamo_ctx* ctx, float* d_V, int32_t* d_F,
                            uint64_t* d_keys, int32_t* d_edges);

/* Per-round record (requires options.record_rounds).  out[12] receives
 * nV nF nE link_rejects flagged eligible winners committed undone undo_iters
 * pairs_found of round r, and the round's device time in microseconds (its
 * graph replays, CUDA events; 0 for rounds run by the per-round entry
 * points). */
pamo_status pamo_ctx_round_info(const pamo_ctx* ctx, int64_t r, int64_t* out);

/* Vertex pairs (in round r's input numbering) of kind 0 = winners,
 * 1 = committed, 2 = undone.  h_out (host, nullable) receives up to cap pairs;
 * *n receives the total. */
pamo_status pamo_ctx_round_pairs(const pamo_ctx* ctx, int64_t r, int32_t kind,
                                 int32_t* h_out, int64_t cap, int64_t* n);

/* Training data of the learned proposal (no counterpart in the paper).
 * After pamo_round_select: the 16 features of every winner of this round, in
 * winner order (d_X: device, n_winners x 16 float32; see pamo_mlp).  After
 * pamo_round_check_undo: 1 for each winner whose collapse stands, 0 for an
 * undone one (d_out: device, n_winners bytes). */
pamo_status pamo_ctx_winner_features(pamo_ctx* ctx, float* d_X);
pamo_status pamo_ctx_winner_standing(pamo_ctx* ctx, uint8_t* d_out);

/* A deferral schedule (no counterpart in the paper; the bound on what the
 * learned proposal can save).  In round r of the context (0 = its first
 * round) every winner whose vertex pair (a, b), a < b, in that round's input
 * numbering, is listed in h_pairs[2*h_off[r] .. 2*h_off[r+1]) is not collapsed
 * and counts as undone (an invalid edge of the next round, Section 5.3),
 * exactly like a predicted reject.  Given the undone pairs of every round of a
 * plain run (pamo_ctx_round_pairs, kind 2), the run repeats that plain run's
 * output, round by round, without any undo iteration: what a perfect
 * predictor of the intersection check would save.
 *   h_off: host int64 [n_rounds + 1], ascending from 0; h_pairs: host int32
 *   pairs [h_off[n_rounds]][2] (copied).  Rounds beyond n_rounds defer nothing.
 *   Call before the context's first round, on a single-mesh context without a
 *   learned proposal; otherwise PAMO_EINVAL. */
pamo_status pamo_ctx_set_deferrals(pamo_ctx* ctx, const int64_t* h_off, int64_t n_rounds,
                                   const int32_t* h_pairs);

/* Number of recorded rounds and the run status so far (PAMO_OK / ESTALL). */
pamo_status pamo_ctx_rounds(const pamo_ctx* ctx, int64_t* rounds);

/* Run rounds until |F| <= target (the loop of pamo_simplify on a context). */
pamo_status pamo_ctx_run(pamo_ctx* ctx, int64_t target_faces, pamo_stats* stats);

void pamo_ctx_destroy(pamo_ctx* ctx);

/* ---- the intersection check on its own (Algorithm 3) ---- */

/* All intersecting face pairs of a mesh (LBVH broad phase, exact narrow
 * phase with the shared-vertex cases of supplementary Section 3).
 * *n_pairs (host) receives the count; d_pairs (nullable, device int32
 * [cap][2]) receives up to cap pairs (f < g), in no particular order.
 * Every face index must lie in [0, nV): the call checks this first and
 * returns PAMO_EINVAL, before anything reads the mesh, when one does not.
 * Positions must be finite.  Synchronises `stream` before it returns. */
pamo_status pamo_check_self_intersections(const float* d_V, int64_t nV,
                                          const int32_t* d_F, int64_t nF,
                                          void* stream, int64_t* n_pairs,
                                          int32_t* d_pairs, int64_t cap);

/* pamo_check_self_intersections without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc while they run -- e.g. a service whose device memory
 * is reserved and budgeted by another component, or a latency-bound loop that
 * must not block on the allocator.  Arguments, outputs and the result are
 * those of pamo_check_self_intersections (d_V/d_F device mesh, *n_pairs host,
 * d_pairs device [cap][2], caller-owned).
 *   - All scratch lives in one fixed device array inside the library (about
 *     4.9 MiB); every GPU that loads the library holds it until the process
 *     exits.  Limit: nF <= 32768 and nV <= 32768; larger meshes return
 *     PAMO_EINVAL with a message.
 *   - Face indices outside [0, nV) return PAMO_EINVAL before the mesh is
 *     read, as in pamo_check_self_intersections.
 *   - The first call on each device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.
 *   - Every call reuses the same array: calls that overlap on the GPU (on
 *     different streams, or from different threads) race and must be
 *     serialised by the caller.  The call synchronises `stream` before it
 *     returns.  It calls no cudaMalloc, cudaFree or allocating routine. */
pamo_status pamo_check_self_intersections_noalloc(const float* d_V, int64_t nV,
                                                  const int32_t* d_F, int64_t nF,
                                                  void* stream, int64_t* n_pairs,
                                                  int32_t* d_pairs, int64_t cap);

/* The triangle-pair predicate on a batch (device arrays):
 * d_P [n][18] float32 (T's corners then C's), d_idx [n][6] int32 vertex
 * indices (equal indices = shared vertices), d_out [n] uint8 (1 = intersect).
 * Stream-ordered; does not synchronise. */
pamo_status pamo_tri_intersect_batch(const float* d_P, const int32_t* d_idx,
                                     int64_t n, uint8_t* d_out, void* stream);

/* Exact orientation signs on a batch (device arrays, stream-ordered):
 * orient3d: d_P [n][12] -> d_out [n] in {-1,0,1}, the sign of
 * det[a-d; b-d; c-d]; orient2d: d_P [n][6] -> sign of (b-a) x (c-a). */
pamo_status pamo_orient3d_batch(const float* d_P, int64_t n, int8_t* d_out,
                                void* stream);
pamo_status pamo_orient2d_batch(const float* d_P, int64_t n, int8_t* d_out,
                                void* stream);

/* Measured float64 throughput of the current device (measurement support for
 * the roofline of the edge cost, whose float64 arithmetic includes divisions
 * and square roots that the hardware runs as instruction sequences).  Runs a
 * few short probe kernels (about 0.1 s) on `stream` and synchronises it.
 * h_rates (host, 3 doubles) receives fused multiply-adds per second,
 * divisions per second and square roots per second over the whole GPU
 * (divisions and roots timed beyond an identical loop without them). */
pamo_status pamo_measure_fp64(void* stream, double* h_rates);

/* Verification support for the skinny term of Eq. 1 (Sec. 5.1): the edge-cost
 * kernel evaluates each produced triangle's 1 - C_ijk in float-float
 * arithmetic and keeps a key only when an error bound proves it equal to the
 * float64 evaluation's.  For n triangles, d_tri (device, n x 9 float32:
 * corners P0 P1 P2, P0 the placement) gives d_t64 (device, n float64) = 1 -
 * C_ijk as the kernel evaluates it in float64 (corners in the given order)
 * and d_tff (device, n x 2 float32) = the float-float pair (high, low), NaN
 * high part outside the certified range.  Asynchronous on `stream`.
 * PAMO_EINVAL for n < 0 or a null array with n > 0. */
pamo_status pamo_skinny_terms(const float* d_tri, int64_t n, double* d_t64, float* d_tff,
                              void* stream);

/* Thread-local message of the last failing call ("" if none). */
const char* pamo_last_error(void);

/* Memory kept between calls.  Device buffers come from a stream-ordered pool
 * owned by the library (one per device, created on first use) that keeps the
 * memory freed by a finished call for the next one instead of returning it to
 * the CUDA driver, and the small pinned host mirrors of finished contexts are kept
 * for reuse, so back-to-back calls do not map, zero and unmap their working
 * set each time.  The library therefore holds, after a call returns, up to
 * the largest working set it has used on each device (roughly 0.8 KB per
 * input face).  This call returns everything that no live context uses to
 * the CUDA driver (device pools trimmed, cached pinned blocks freed).  It does not
 * synchronise any stream; call it when no simplification is running. */
pamo_status pamo_release_cached_memory(void);

#ifdef __cplusplus
}
#endif

#endif /* PAMO_H */
