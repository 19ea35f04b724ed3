/*
 * vj.h -- C ABI of the B300 vector epsilon-join library (libvj.so).
 *
 * The operation (Def. 1 of "Fast Approximate Vector Joins via Offline-Online
 * Co-Design", arXiv 2603.16360): given data vectors X and query vectors Q in
 * R^d, a distance dist(.,.) and a threshold eps, return for every query q the
 * data vectors x with dist(x, q) < eps (strict).  The approximate join walks a
 * merged proximity graph built over X U Q (Sec. 4.3, "merged index"), with soft
 * work sharing between nearby queries (Sec. 4.2, Alg. 8) and the OOD-adaptive
 * hybrid expansion (Sec. 4.4, Alg. 6-7).  The exact join is the nested-loop
 * join of Sec. 3.2.
 *
 * Naming: the paper calls the query set X and the data set Y; this ABI calls
 * the data set X and the query set Q.  Merged node ids: data 0..nx-1, queries
 * nx..nx+nq-1.
 *
 * Conventions for every call:
 *  - Return value: VJ_OK or an error code; on error vj_last_error() returns a
 *    thread-local, NUL-terminated message that stays valid until the next call
 *    on the same thread.  No call exits, traps or throws across the ABI.
 *  - Ownership: input buffers stay owned by the caller and are not retained
 *    (vj_build copies them into device memory).  vj_index / vj_result objects
 *    are owned by the library until the matching *_free call.
 *  - Device: every call uses the CUDA device current on the calling thread at
 *    vj_build time; all work runs on the index's stream (vj_set_stream).
 *  - Threads: an index may be used by one thread at a time.
 */
#ifndef VJ_H
#define VJ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VJ_OK = 0,
    VJ_ERR_ARG = 1,     /* invalid argument (null pointer, size, mode) */
    VJ_ERR_OOM = 2,     /* device or host allocation failed */
    VJ_ERR_CUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    VJ_ERR_TIMEOUT = 4, /* a bounded device wait gave up (see vj_last_error) */
    VJ_ERR_STATE = 5    /* capacity exceeded or object in the wrong state */
} vj_status;

typedef enum {
    VJ_L2 = 0,    /* dist = sqrt(sum (x_i - q_i)^2) */
    VJ_COSINE = 1 /* dist = 1 - <x,q> / (|x| |q|) */
} vj_metric;

/* cfg.work_sharing of Tab. cfg (Sec. 4.1).  Under the merged index, SOFT also
 * seeds the query node itself (S = {entry, q} U C[parent]); SELF is the
 * paper's default merged mode (S = {entry, q}).  HARD (HWS: the parent's result
 * row as seeds) runs on separate indexes only (vj_params.separate); a join of
 * a merged index with HARD returns VJ_ERR_ARG. */
enum { VJ_WS_NONE = 0, VJ_WS_HARD = 1, VJ_WS_SOFT = 2, VJ_WS_SELF = 3 };

enum { VJ_PREC_FP32 = 0, VJ_PREC_BF16 = 1, VJ_PREC_FP8 = 2 };

/* Build and join parameters (Tab. cfg plus build knobs). */
typedef struct {
    int degree;           /* graph out-degree R (1..32), default 32 */
    int knn_k;            /* kNN candidates per node for the build, R <= K <= 112; default 64 */
    int greedy_beam;      /* cfg.greedy_beam_size, default 256 (Alg. 4) */
    int conv_threshold;   /* cfg.conv_threshold, default 10 (Alg. 5) */
    int hybrid_beam;      /* cfg.hybrid_beam_size, default 256 (Alg. 7) */
    int work_sharing;     /* VJ_WS_*, default VJ_WS_SOFT (MI+SWS) */
    int adapt_hybrid;     /* cfg.adapt_hybrid (Alg. 6), default 1 */
    int force_hybrid;     /* cfg.force_hybrid (Alg. 6), default 0 */
    int precision;        /* VJ_PREC_* of the kNN build's distance tiles: BF16 (default) sweeps on the
                             tensor cores, FP32 on the SIMT units; candidates are re-ranked with exact
                             keys and certified either way, so the lists are the same.  FP8 is
                             accepted only by the scan (the join-time field scan), not by the
                             build (VJ_ERR_ARG). */
    int learned;          /* joins: 1 = plan every query with the attached predictor
                             (vj_attach_predictor) in place of Alg. 6's rule; default 0 */
    int route_bruteforce; /* reserved, must be 0 */
    int input_on_device;  /* 1: X and Q passed to vj_build are device pointers */
    uint64_t seed;        /* reserved for randomised steps; recorded only */
    int gather;           /* joins: VJ_PREC_* of the traversal's vector gathers.  BF16 reads the BF16
                             copy of the vectors (half the bytes) when every coordinate is exactly a
                             BF16 value, so every key equals the FP32 one; otherwise, and by default
                             (FP32), the FP32 rows.  A join-time field. */
    int hybrid_seed_best; /* joins: 1 = a hybrid expansion whose greedy phase found no in-range point
                             starts from the closest visited data node (the paper's Alg. 7 as
                             written starts nowhere and returns nothing); default 0 */
    int nnmap;            /* build: 1 = an NN-Map index (the paper's closing design, "NN-Map"):
                             the data set's own graph G_X (kNN among data only, pruned over data
                             rows only) and, per query, its witness (nearest data vector, ties by
                             id), the witness's FP64 distance and an OOD bit (the d1/d2 > 1.5 rule
                             with N1 = the query's R nearest data vectors and d2 = the mean length
                             of the G_X edges from N1 to data outside N1; no such edge: not OOD).
                             vj_join on it has no greedy phase: a query whose witness distance is
                             >= eps has an empty row and computes nothing; the others run the
                             expansion of Alg. 7 on G_X from the witness (BFS; hybrid when
                             force_hybrid, or adapt_hybrid and the OOD bit), with no work
                             sharing.  steps counts distance evaluations (the stored witness
                             distance costs none); default 0 */
    int separate;         /* build: 1 = separate (per-set) indexes (Sec. 3.2): the data graph G_Y
                             over the data rows and the query graph over the query rows (each
                             row's kNN list ranks its own set only), the entry s_Y nearest the
                             data centroid, and the MST over the query graph plus a star edge
                             (s_Y, q) per query.  vj_join on it runs Alg. 1 with Alg. 4-5's
                             best-first greedy search on G_Y (queue trimmed to greedy_beam after
                             each expansion, stopped by an in-range front or conv_threshold
                             checks without a smaller front key) from S = {s_Y} (INLJ:
                             work_sharing NONE or SELF), {s_Y, C[parent]} (SOFT) or {s_Y} plus
                             the parent's result row (HARD); with sharing, queries run parents
                             first.  adapt_hybrid does not apply (the rule reads the merged
                             graph); force_hybrid does.  Exclusive with nnmap; default 0 */
    int scan;             /* joins: VJ_PREC_* of the brute-force scan's tiles (vj_join_exact, routed
                             queries): BF16 (default; FP32 selects it too, there is no FP32 tile
                             path) or FP8 (E4M3 operands, a power-of-two scale per data row and one
                             for the scanned query rows, FP32 accumulation).  Either way a pair is
                             a candidate when its tile value is within a rounding bound of eps, and
                             every candidate is re-decided from the FP32 vectors (FP64 near eps), so
                             the result is the same; the precision changes the candidate count.
                             A join-time field */
} vj_params;

/* Per-call counters and device timings of a join. */
typedef struct {
    int64_t dist_computations; /* "steps" of Sec. 5.3: distance evaluations */
    int64_t expansions;        /* nodes popped in the expansion phase */
    int64_t adj_rows_read;     /* adjacency rows read (probe + expansions + OOD) */
    int64_t hybrid_queries;    /* queries that ran the hybrid expansion */
    int64_t rechecks;          /* FP64 re-evaluations near eps or near ties */
    int64_t spill_queries;     /* queries whose visited set left shared memory */
    double ms_traverse;        /* device time of the traversal kernel */
    double ms_csr;             /* device time of the final CSR assembly */
    double ms_total;           /* device time of the whole join */
    int64_t bytes_algorithmic; /* vector + adjacency bytes the traversal must read */
    int64_t kernel_launches;   /* kernels this call launched */
    double ms_scan;            /* device time of the tensor-core brute-force scan (exact join / routed queries) */
    int64_t scan_candidates;   /* pairs the scan passed to the exact re-check */
    double ms_prologue;        /* device time of the learned prologue (features + predictor + plan) */
    int64_t sws_restarts;      /* soft-sharing queries re-run in the parent-ordered second pass
                                  (hybrid queries, and queries whose result the cached seed changes) */
    double ms_route;           /* device time of the routed queries' rows (scan, exact re-check and
                                  their CSR); ms_scan is the scan kernel alone */
    double ms_sws[3];          /* soft sharing: device time of the speculative pass, the parallel
                                  decision pass and the parent-ordered commit pass (of the last
                                  traversal attempt; the three add up to ms_traverse) */
} vj_stats;

/* CSR result of a join.  ids are data ids (0..nx-1), ascending within each
 * query row; dists are the pair distances.  steps/cache/hybrid are per-query
 * (query index order): distance evaluations, the soft cache C[q] of Alg. 8
 * (closest visited data node, -1 if none) and the expansion the query ran:
 * 0 BFS, 1 hybrid (the CheckHybrid outcome), 2 routed to the brute-force
 * scan, 3 none (a plan of -1).
 * When on_device is 1 every array is a device pointer; otherwise every array
 * is page-locked host memory from the library's block cache.  Either way the
 * result is released with vj_result_free. */
typedef struct {
    int64_t nq;
    int64_t nnz;
    int64_t *offsets; /* [nq + 1] */
    int32_t *ids;     /* [nnz] */
    float *dists;     /* [nnz] */
    int32_t *steps;   /* [nq] */
    int32_t *cache;   /* [nq] */
    uint8_t *hybrid;  /* [nq] */
    int on_device;
    vj_stats stats;
} vj_result;

typedef struct vj_index vj_index;

/* Fill *p with the defaults listed above. */
void vj_default_params(vj_params *p);

/* Offline merged-index build (Sec. 4.3; the paper's index is NSG, a black
 * box; this library builds an exact kNN graph of X U Q, RNG-prunes it to R
 * (App. C rule), adds reverse edges, picks the entry nearest the centroid,
 * stores data-edge lengths and the MST order over queries of Alg. 2).
 *   X: nx*d row-major float32, Q: nq*d row-major float32 (host pointers, or
 *   device pointers when p->input_on_device).  nx >= 1, nq >= 1, 1 <= d <= 4096,
 *   nx + nq < 2^31.  p may be NULL (defaults).
 * Errors: VJ_ERR_ARG, VJ_ERR_OOM, VJ_ERR_CUDA.  *out is NULL on error. */
vj_status vj_build(const float *X, int64_t nx, const float *Q, int64_t nq, int d,
                   vj_metric metric, const vj_params *p, vj_index **out);

/* Run all further work of this index on `stream` (a cudaStream_t; NULL =
 * the legacy default stream). */
vj_status vj_set_stream(vj_index *ix, void *stream);

/* Replace the join-time fields (greedy_beam, conv_threshold, hybrid_beam,
 * work_sharing, adapt_hybrid, force_hybrid, learned, gather,
 * hybrid_seed_best) used by later joins. */
vj_status vj_set_join_params(vj_index *ix, const vj_params *p);

/* Per-query plan used by later joins in place of Alg. 6's CheckHybrid rule
 * (a predictor's output; the paper has the rule only).  Host arrays of nq
 * entries, copied; either may be NULL (NULL for both clears the plan):
 *   route[q] != 0: after its greedy phase (seeds + probe of N(q), so soft
 *     work sharing still hands C[q] to its children) the query's row is its
 *     exact nested-loop-join row, computed by the tensor-core brute-force scan
 *     with exact re-check; hybrid flag 2 in the result.
 *   beam[q] > 0: hybrid expansion with hybrid_beam_size = beam[q];
 *   beam[q] == 0: the BFS expansion;
 *   beam[q] == -1: no expansion phase: the row is the probe's in-range data
 *     points (hybrid flag 3 in the result).  An expansion budget of zero,
 *     not in the paper (a knob for the learned predictor).
 * Errors: VJ_ERR_ARG (beam outside [-1, 2^20]). */
vj_status vj_set_plan(vj_index *ix, const uint8_t *route, const int32_t *beam);

/* ---- Learned route / budget predictor (not in the paper, which decides with
 * the d1/d2 > 1.5 rule of Sec. 4.4 only; that rule stays the default).
 * A 3-layer MLP din -> h1 -> h2 -> 2 (ReLU): output 0 regresses
 * log2(budget + 2), output 1 is the route logit.  Loss = mean squared error on
 * output 0 + binary cross-entropy with logits on output 1, averaged over rows.
 * Parameters: one flat FP32 array W1[h1][din] b1 W2[h2][h1] b2 W3[2][h2] b3.
 * Inputs are standardised per feature with the training rows' mean / std. */
typedef struct vj_mlp vj_mlp;
vj_status vj_mlp_create(int din, int h1, int h2, uint64_t seed, vj_mlp **out); /* He-uniform init */
int64_t vj_mlp_num_params(const vj_mlp *m);
/* host buffers: flat [num_params], mu/sd [din] (mu/sd may be NULL) */
vj_status vj_mlp_get_params(const vj_mlp *m, float *flat, float *mu, float *sd);
/* mu and sd both NULL: no standardisation */
vj_status vj_mlp_set_params(vj_mlp *m, const float *flat, const float *mu, const float *sd);
/* Mean loss and its gradient (flat, host) over n host rows x [n][din] with
 * targets t_reg [n], t_cls [n] (0/1); rows used as given (no standardisation). */
vj_status vj_mlp_loss_grad(vj_mlp *m, const float *x, const float *t_reg, const float *t_cls, int64_t n,
                           double *loss, float *grad);
/* Adam (beta 0.9 / 0.999, eps 1e-8) over seeded shuffled mini-batches;
 * sets the standardisation from x first.  final_loss: last epoch's mean. */
vj_status vj_mlp_train(vj_mlp *m, const float *x, const float *t_reg, const float *t_cls, int64_t n, int epochs,
                       int batch, float lr, uint64_t seed, double *final_loss);
/* outputs [n][2] (host) for host rows x [n][din], standardised */
vj_status vj_mlp_predict(vj_mlp *m, const float *x, int64_t n, float *out);
void vj_mlp_free(vj_mlp *m);

/* Predictor features of every query at threshold eps, host [nq][7 + d]:
 * d1/eps, d2/eps, d1/d2 (Sec. 4.4), dist(q, entry)/eps, dist to the nearest
 * data neighbour/eps, #data neighbours/R, #data neighbours within eps/R,
 * then the d coordinates of q. */
vj_status vj_features(vj_index *ix, float eps, float *out);

/* Use predictor m (din = 7 + d; NULL detaches) for joins with
 * params.learned = 1: a prologue computes the features, runs m and routes
 * a query to the brute-force scan when sigmoid(output 1) > route_threshold,
 * else reads the budget b = 2^output0 - 2: b < -1/2 no expansion phase (plan
 * -1), b < 4 the BFS expansion, else the hybrid queue size b capped at
 * beam_cap (a cap below 4: BFS).  Output 0 therefore regresses
 * log2(budget + 2) with budget -1 (none), 0 (BFS) or a queue size.  The index
 * keeps the pointer; m must outlive it or be detached. */
vj_status vj_attach_predictor(vj_index *ix, vj_mlp *m, float route_threshold, int beam_cap);

/* Outputs [nq][2] (host) of the attached predictor on the features at eps,
 * computed exactly as the learned prologue of a join computes them (on the
 * tensor cores with BF16 inputs and weights when h1 is a multiple of 64 and
 * h2 a multiple of 16, both at most 256; FP32 otherwise).  No paper
 * counterpart (the paper has only the d1/d2 rule, Sec. 4.4).  VJ_ERR_STATE
 * when no predictor is attached. */
vj_status vj_predictor_outputs(vj_index *ix, float eps, float *out);

/* ---- Training the predictor inside the library (no paper counterpart: the
 * paper's route is the d1/d2 rule of Sec. 4.4).  The training queries are
 * rows of the index's own query set, which the caller keeps apart from the
 * queries it evaluates on (a held-out set built into the same merged index).
 * Labels, per training query q at threshold eps:
 *   - the exact row of q (tensor-core scan with the exact re-check, Sec. 3.2);
 *   - for each ladder budget in order (-1 no expansion, 0 BFS, > 0 hybrid
 *     queue size) one join of every query planned with that budget, giving
 *     q's row recall against its exact row and q's cost (its distance
 *     evaluations); a join that fails (a hybrid search outgrowing its visited
 *     set) ends the ladder, the first must succeed;
 *   - budget = the first ladder budget whose recall reaches query_recall,
 *     else the last budget that ran;
 *   - route = 1 when q's cost at its budget is at least scan_row_cost; then,
 *     while the training queries' pooled recall (pairs found / exact pairs)
 *     is below pooled_recall, the query with the most missed pairs per unit of
 *     extra cost, missed / (scan_row_cost - cost), ties by smaller query
 *     index, is routed too.
 * scan_row_cost is the cost of one brute-force row in distance evaluations;
 * <= 0 measures it (scan time per training query over the BFS join's time
 * per distance evaluation).  The index's plan is cleared and its join
 * parameters restored afterwards. */
typedef struct {
    int n_ladder;        /* 1..8 entries of ladder used, in order of increasing cost */
    int ladder[8];       /* default -1, 0, 8 */
    float query_recall;  /* default 0.95 */
    float pooled_recall; /* default 0.955 */
    float scan_row_cost; /* default 0 (measured) */
    int h1, h2;          /* hidden widths, default 256, 256 */
    int epochs, batch;   /* default 30, 256 */
    float lr;            /* default 1e-3 */
    uint64_t seed;       /* weight init and batch shuffle, default 7 */
} vj_train_params;

typedef struct {
    int64_t n;              /* training queries */
    int64_t routed;         /* route labels set */
    int64_t per_budget[8];  /* budget labels per ladder entry */
    int ladder_run;         /* ladder entries whose join completed */
    double scan_row_cost;   /* the cost the route labels used */
    double final_loss;      /* vj_train_predictor: last epoch's mean loss */
    double ms_labels;       /* host wall time of the labels (joins included) */
    double ms_train;        /* host wall time of features + training */
} vj_train_report;

void vj_default_train_params(vj_train_params *tp);

/* The labels above for the n training queries rows[] (query indices, host):
 * budget[n] (int32) and route[n] (uint8, 0/1), host buffers.  rep may be NULL.
 * Errors: VJ_ERR_ARG (bad rows or parameters), and those of vj_join. */
vj_status vj_predictor_labels(vj_index *ix, float eps, const int32_t *rows, int64_t n,
                              const vj_train_params *tp, int32_t *budget, uint8_t *route,
                              vj_train_report *rep);

/* Labels as above, features of the training queries (vj_features), then a
 * new predictor din = 7 + d -> h1 -> h2 -> 2 trained with vj_mlp_train on
 * targets log2(budget + 2) and route.  *out receives it (free with
 * vj_mlp_free; attach with vj_attach_predictor).  rep may be NULL. */
vj_status vj_train_predictor(vj_index *ix, float eps, const int32_t *rows, int64_t n,
                             const vj_train_params *tp, vj_mlp **out, vj_train_report *rep);

/* Approximate join (Alg. 1 on the merged index) at threshold eps > 0.
 * budget > 0 overrides hybrid_beam for this call.  The result lives in host
 * memory (the device->host copy is part of the call).
 * Errors: VJ_ERR_ARG, VJ_ERR_OOM, VJ_ERR_CUDA, VJ_ERR_TIMEOUT (a work-sharing
 * dependency wait ran out; the index stays usable).
 * Threads: calls on one index must not overlap; joins of different indexes may
 * run at the same time from different host threads. */
vj_status vj_join(vj_index *ix, float eps, int budget, vj_result **out);

/* As vj_join, but the result arrays stay in device memory (on_device = 1). */
vj_status vj_join_device(vj_index *ix, float eps, int budget, vj_result **out);

/* n independent joins, instance i = vj_join(ixs[i], eps[i], 0) (Def. 1 for
 * each pair of sets; the scalability study of Sec. 5 runs many instances of
 * very different sizes).  The traversal passes of all instances run fused,
 * one launch per pass over up to 64 instances of one kernel class (indexes
 * whose padded dimensions fall in the same class share a launch); each
 * result equals what vj_join gives for that instance alone.
 *   ixs [n]: distinct built indexes (an index listed twice -> VJ_ERR_ARG).  A
 *   predictor attached to several of them is shared safely (its inference is
 *   serialised).  The call uses each index's stream; the fused passes run on
 *   the largest index's stream with one traversal workspace from the
 *   library's cache.
 *   eps [n] (host): per-instance thresholds, each > 0.
 *   outs [n] (host): receives n host results, each freed by vj_result_free.
 *   In each result's stats, ms_traverse is the time of the fused passes
 *   (shared by all instances) and ms_sws is zero.
 * All or nothing: on any failure every outs[i] is NULL and vj_last_error
 * names the first failing instance.  n = 0 is a no-op. */
vj_status vj_join_batch(vj_index **ixs, const float *eps, int n, vj_result **outs);

/* Query-data switching (the paper's large-threshold discussion, App. E):
 * the join X |><| Q equals Q |><| X transposed, so for large eps the roles may
 * be swapped.  ix must be built with them swapped (vj_build(Q, nq, X, nx,
 * ...): the original queries as the index's data).  The call runs Alg. 1 on
 * it (the original data vectors as queries) and transposes the pair list
 * back: one row per original query (the index's data row), ids the original
 * data ids (the index's query indices) ascending, dists the pair distances.
 * Host result with nq = the index's nx; steps and hybrid are 0 and cache -1
 * (the swapped join's per-query outputs describe the other set); stats are
 * the swapped join's.  Errors: as vj_join. */
vj_status vj_join_switched(vj_index *ix, float eps, vj_result **out);

/* Exact nested-loop join (Sec. 3.2) of the index's X and Q on the GPU, host
 * result.  Pairs whose FP32 distance lies within the FP32 rounding bound of
 * eps are re-decided in FP64. */
vj_status vj_join_exact(vj_index *ix, float eps, vj_result **out);

/* Exact join for callers that cannot allocate device memory (the paper has no
 * counterpart: this is a deployment variant of vj_join_exact).  Callers that
 * live inside a fixed, pre-carved device-memory budget, or that cannot afford
 * cudaMalloc/cudaFree (allocator locks, device-wide synchronization), pass
 * every buffer themselves; the call allocates nothing.
 *   X [nx*d], Q [nq*d]: device pointers, row-major float32 (no index needed).
 *   offsets [nq+1] (device, int64): CSR row offsets, always written in full.
 *   ids [cap] (device, int32), dists [cap] (device, float32): pairs in
 *   ascending data id per query; pairs beyond cap are not written.
 *   nnz (host): total number of pairs.  stream: a cudaStream_t or NULL.
 * Scratch is a fixed 4 MiB device array inside the library, which limits nq
 * to 1,048,576 (larger nq -> VJ_ERR_ARG).  A GPU holds the array, until the
 * process exits, from the moment the library's device code is loaded on it.
 * Under CUDA's lazy module loading (the default) that is the first call into
 * the library on that device, so a first call of this entry point can take
 * those 4 MiB implicitly: make one warm-up call (or any other vj call) before
 * entering a budgeted phase, or set CUDA_MODULE_LOADING=EAGER.  All calls
 * share the array: calls that overlap on the GPU race and give wrong results.
 * The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) and should come before any stream capture on that
 * device.  Every call copies nnz to the host and waits for `stream` to finish
 * before it returns.  Returns VJ_ERR_STATE when nnz > cap.
 * Decisions: FP32 keys, re-decided in FP64 within the FP32 rounding bound
 * of eps (same rule as vj_join_exact). */
vj_status vj_join_exact_noalloc(const float *X, int64_t nx, const float *Q, int64_t nq, int d,
                                vj_metric metric, float eps, int64_t *offsets, int32_t *ids,
                                float *dists, int64_t cap, int64_t *nnz, void *stream);

/* Traversal tuning (no paper counterpart: the paper's join is single-threaded
 * CPU code).  The GPU traversal gathers each vector row with a group of
 * `lanes` threads holding `slots` 16-byte pieces each (a row of up to
 * lanes * slots * 4 floats) and keeps `inflight` rows in flight per group; it
 * runs as a persistent grid of `blocks` blocks, and the probe of N(q) streams
 * rows through a ring of `probe_ring` stages per warp, each row as 16-byte
 * copies issued by every lane or, with `probe_bulk`, as one bulk copy of the
 * whole row by the copy engine.  Every setting computes
 * the same join (in-range decisions near eps are re-decided in FP64; only
 * the FP32 summation order of a key changes), so tuning changes time only.
 *
 * vj_autotune times joins of the index at eps (the index's current join
 * parameters and plan) under each candidate setting: the default class (the
 * smallest that holds the row) and the next two larger ones, each with the
 * full and half persistent grid, and, on a merged index, shallower probe
 * rings and the bulk-copy probe for the default class.  Each setting runs one
 * untimed join and then
 * `reps` (1..10) timed ones; its time is the median device time of the whole
 * join (vj_stats.ms_total).  A setting counts only when its joins give the
 * same pair count and distance evaluations as the default setting.  The
 * fastest is kept on the index for later joins (vj_join, vj_join_batch) and
 * the report lists every setting tried.  The index's previous setting is
 * restored on error. */
#define VJ_TUNE_MAX 16
typedef struct {
    int n;                      /* settings tried (the first is the default) */
    int lanes[VJ_TUNE_MAX];     /* threads per gathered row */
    int slots[VJ_TUNE_MAX];     /* 16-byte pieces per thread */
    int inflight[VJ_TUNE_MAX];  /* rows in flight per group */
    int blocks[VJ_TUNE_MAX];    /* persistent blocks of the traversal */
    int probe_ring[VJ_TUNE_MAX];/* probe ring stages per warp (0: no probe kernel) */
    int probe_bulk[VJ_TUNE_MAX];/* 1: the probe copies each row in one bulk copy */
    double ms[VJ_TUNE_MAX];     /* median device time of the join */
    int valid[VJ_TUNE_MAX];     /* 1: same pairs and evaluations as the default */
    int chosen;                 /* index of the setting kept on the index */
} vj_tune_report;
vj_status vj_autotune(vj_index *ix, float eps, int reps, vj_tune_report *report);

/* Set the traversal setting directly (for instance the one vj_autotune chose
 * on another index of the same row width).  lanes = 0 selects the default
 * class (slots and inflight are then ignored); otherwise (lanes, slots,
 * inflight) must name a class whose rows hold d floats, else VJ_ERR_ARG.
 * blocks = 0 and probe_ring = 0 select the defaults; probe_ring is 2..8;
 * probe_bulk is 0 (16-byte copies, the default) or 1. */
vj_status vj_set_tuning(vj_index *ix, int lanes, int slots, int inflight, int blocks, int probe_ring,
                        int probe_bulk);

/* Bounded dependency wait of soft work sharing (for tests of its failure
 * path; no paper counterpart).  max_polls > 0 limits the polls of a query's
 * wait for its MST parent's cache before the join gives up with
 * VJ_ERR_TIMEOUT (0 restores the default of 2^24 polls with back-off, about
 * seconds).  hold_q >= 0 makes that query never publish its cache, so its
 * children's waits run out (-1: none).  The index stays usable after a
 * timeout. */
vj_status vj_set_wait_test(vj_index *ix, long long max_polls, int64_t hold_q);

/* Copy the built graph to host buffers (any may be NULL):
 *   adj [(nx+nq) * R] int32 (-1 padded), entry (1 value),
 *   parent [nq] (MST parent query index, -1 = entry), order [nq]
 *   (processing order), depth [nq] (MST depth, entry = 0). */
vj_status vj_export_graph(const vj_index *ix, int32_t *adj, int32_t *entry, int32_t *parent,
                          int32_t *order, int32_t *depth);

/* Copy the exact kNN lists computed by the build: ids [(nx+nq) * K] and
 * dists [(nx+nq) * K] (ascending by (dist, id)). */
vj_status vj_export_knn(const vj_index *ix, int32_t *ids, float *dists);

/* The NN-Map outputs of an index built with nnmap = 1 (any pointer may be
 * NULL): witness [nq] int32 data ids, wdist [nq] FP64 distances, ood [nq].
 * VJ_ERR_STATE for an index built without nnmap. */
vj_status vj_export_nnmap(const vj_index *ix, int32_t *witness, double *wdist, uint8_t *ood);

/* Shape of an index: any pointer may be NULL. */
vj_status vj_index_info(const vj_index *ix, int64_t *nx, int64_t *nq, int *d, int *degree,
                        int *knn_k, int *max_depth);

/* How the offline build went (any pointer may be NULL): knn_tensor_cores = 1
 * when the kNN candidates came from the BF16 tensor-core sweep (0: the FP32
 * SIMT sweep); knn_uncertified = rows whose candidates could not be
 * certified and were scanned exactly; ms_build = device time of vj_build,
 * ms_knn = the part spent on the exact kNN lists. */
vj_status vj_build_info(const vj_index *ix, int *knn_tensor_cores, int64_t *knn_uncertified, double *ms_build,
                        double *ms_knn);

/* Release a result (its arrays go back to the library's caches). */
void vj_result_free(vj_result *r);
/* Release an index.  Joins borrow their traversal workspace (GBs: visited
 * lists and bitmaps per resident warp) from a process-wide cache, one per join
 * running at once; freeing the last live index empties that cache. */
void vj_free(vj_index *ix);
const char *vj_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VJ_H */
