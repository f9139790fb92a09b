/*
 * apsp.h -- C ABI of the GB300 warm-start all-pairs-shortest-path library.
 *
 * The library keeps the APSP matrix D of a dense weighted graph (directed or
 * undirected, non-negative weights) resident in device memory and keeps it
 * exact while the graph changes by one node or one edge at a time, following
 * "Solving the all pairs shortest path problem after minor update of a large
 * dense graph" (arXiv 2412.15122):
 *
 *   - adding a node: Corollary 1, Corollary 2 and Theorem 3 (Section 3.1);
 *   - removing a node: the need_update_list of Section 3.2 (Theorem 4 /
 *     Corollary 3), the Cost of Eq. (equ:cost_defi) and the warm/cold choice of
 *     Algorithm 5;
 *   - changing an edge weight: the result Algorithm 6 defines (the APSP
 *     matrix of the graph with the new weight), computed by direct exact
 *     formulas for decreases and by affected-pair detection plus restricted
 *     re-relaxation for increases;
 *   - cold recomputation: blocked min-plus Floyd-Warshall.
 *
 * Conventions shared by every call:
 *   - Node ids are stable slot indices in [0, capacity).  At init slots
 *     0..n-1 are live.  A removed node leaves a dead slot; a new node takes the
 *     lowest dead slot, else the next never-used slot.
 *   - Matrices passed in or out are dense row-major with a leading dimension
 *     given in elements.  W[i][j] is the weight of edge i -> j.
 *   - Element type is int32 (APSP_I32) or float (APSP_F32), chosen at init.
 *     A missing edge / unreachable pair is APSP_INF_I32 (int32) or +infinity
 *     (float).  Int32 inputs >= APSP_INF_I32 are read as missing.  Weights must
 *     be >= 0 (Section 1: w maps edges to non-negative reals), else
 *     APSP_E_NEGATIVE; NaN is APSP_E_ARG.  Int32 callers must keep every finite
 *     shortest-path length below APSP_INF_I32; longer sums saturate to it.
 *   - Host buffers are owned by the caller and only read (or written) during
 *     the call.  All device memory is owned by the library and freed by
 *     apsp_destroy.
 *   - Every call on one handle is ordered on the handle's CUDA stream and
 *     returns once the work is enqueued; calls that return data to the host
 *     (apsp_query*, apsp_copy_*, apsp_last_stats, apsp_sync) wait for it.
 *     A handle must not be used from two host threads at once; different
 *     handles may be used concurrently.
 *   - Errors are status codes, never exceptions.  A failure detected by a
 *     kernel (for example a bounded wait that timed out, or invalid weights
 *     passed as device pointers) is recorded on the device and returned by
 *     the next call that waits for the stream.
 */
#ifndef APSP_H
#define APSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct apsp_graph apsp_graph;

typedef enum { APSP_I32 = 0, APSP_F32 = 1 } apsp_dtype;

/* init flags */
enum {
    APSP_DIRECTED = 0u,
    APSP_UNDIRECTED = 1u,     /* W must be symmetric; every update keeps D symmetric */
    APSP_D_GIVEN = 4u,        /* D_or_null holds the APSP matrix of W (trusted, not recomputed) */
    APSP_DEVICE_INPUT = 8u,   /* W / D_or_null are device pointers */
    APSP_MINIMAX = 16u        /* minimax (bottleneck) distances, see below */
};
/* APSP_MINIMAX: the variant of the paper's Discussion in which a path's value
 * is its largest edge weight and D[i][j] is the least such value over all
 * paths i -> j (Floyd-Warshall, insertion, Corollary 3's list and the
 * re-relaxation all run with max in place of +; max and min are exact, so
 * int32 and fp32 results are both exact).  Removals and edge increases wait
 * for the device once to read the list's size and choose warm or cold
 * (APSP_DISPATCH_DELTA / ALWAYS_*; the cost model is not used).  Path
 * queries, batches, serving and list modes other than Corollary 3 return
 * APSP_E_UNSUPPORTED for such a graph. */

typedef enum {
    APSP_OK = 0,
    APSP_E_ARG = 1,          /* bad argument (null pointer, bad size, NaN, u == v, ...) */
    APSP_E_NODE = 2,         /* node id out of range or not live */
    APSP_E_NEGATIVE = 3,     /* a negative weight */
    APSP_E_CAPACITY = 4,     /* no free slot for a new node */
    APSP_E_NOMEM = 5,        /* device or pinned host allocation failed */
    APSP_E_CUDA = 6,         /* a CUDA runtime error */
    APSP_E_TIMEOUT = 7,      /* a bounded device-side wait gave up; D may be stale */
    APSP_E_BUSY = 8,         /* resource in use */
    APSP_E_UNSUPPORTED = 9   /* configuration not supported by this build */
} apsp_status;

#define APSP_INF_I32 0x3FFFFFFF
/* Largest capacity: one row of D plus per-row scratch must fit the 227 KB of
 * shared memory of one CTA. */
#define APSP_MAX_CAPACITY 18432

/* What the last update did (apsp_last_stats). */
typedef enum {
    APSP_OP_NONE = 0, APSP_OP_INIT = 1, APSP_OP_ADD = 2, APSP_OP_REMOVE = 3,
    APSP_OP_DECREASE = 4, APSP_OP_INCREASE = 5, APSP_OP_SAME = 6, APSP_OP_RECOMPUTE = 7
} apsp_op;

typedef enum {
    APSP_PATH_NONE = 0,      /* no D work (weight unchanged) */
    APSP_PATH_SWEEP = 1,     /* O(n^2) (or smaller) relaxation sweep, no affected set */
    APSP_PATH_TRIVIAL = 2,   /* detection found no affected pair (e.g. non-tight edge) */
    APSP_PATH_WARM = 3,      /* affected pairs re-relaxed */
    APSP_PATH_COLD = 4       /* full blocked Floyd-Warshall */
} apsp_path;

/* warm/cold dispatch for node removal and edge increase */
typedef enum {
    APSP_DISPATCH_DELTA = 0,        /* Algorithm 5's rule: cold iff Cost > delta */
    APSP_DISPATCH_ALWAYS_WARM = 1,
    APSP_DISPATCH_ALWAYS_COLD = 2,
    APSP_DISPATCH_MODEL = 3         /* learned cost model (apsp_set_model); falls back to DELTA without one */
} apsp_dispatch;

typedef struct {
    int32_t op;               /* apsp_op */
    int32_t path;             /* apsp_path */
    int32_t node;             /* node added / removed, or edge source */
    int32_t node2;            /* edge target, else -1 */
    int32_t n_live;           /* live nodes after the update */
    int32_t affected_rows;    /* non-empty items of need_update_list (Section 3.2) */
    int64_t affected_pairs;   /* pairs re-relaxed */
    int32_t sweep_rows;       /* rows touched by a relaxation sweep */
    int32_t passes;           /* re-relaxation passes until no pair changed */
    int32_t overflow;         /* 1 if the affected set exceeded the scratch capacity (forces cold) */
    int32_t cold_reason;      /* 0 warm, 1 Cost rule, 2 model, 3 forced, 4 overflow */
    float cost;               /* Cost = affected_rows / (N - 1), Eq. (equ:cost_defi) */
    float model_warm;         /* model's predicted log2 microseconds, warm / cold (0 if unused) */
    float model_cold;
    int64_t pairs_rechecked;  /* pair evaluations in re-relaxation passes after the first */
    float warm_pass1_us;      /* device time of the first re-relaxation pass */
    float warm_total_us;      /* device time of the whole warm repair */
    /* Algorithm 12's need_update_list (measured only after apsp_set_exact_list
     * on; -1 otherwise or when the affected set overflowed): listed pairs whose
     * distance grew, the rows holding them, and its Cost (rows / (N - 1)). */
    int64_t grown_pairs;
    int32_t grown_rows;
    float grown_cost;
    /* Node insertion (Section 3.1): rows of D and of D transposed that the
     * reductions of Corollaries 1 and 2 read.  Only rows t with
     * w(p, t) <= min_t' w(p, t') + max_j D[t0][j] (t0 the argmin) can attain
     * a minimum of Corollary 1, and likewise for Corollary 2; when that bound
     * leaves at most span / 8 of them only those are read, else every row is
     * (reported as -1).  0 for other updates. */
    int32_t reduce_rows;
} apsp_stats;

typedef struct {
    int32_t n_live, n_slots, capacity, ld;  /* n_slots = 1 + highest slot ever used */
    int32_t dtype;                          /* apsp_dtype */
    uint32_t flags;
    int64_t device_bytes;                   /* device memory held by the handle */
} apsp_info;

/* ----- lifecycle ------------------------------------------------------- */

/* Create a graph of n live nodes (slots 0..n-1) with room for `capacity`
 * slots (n <= capacity <= APSP_MAX_CAPACITY).  W: n x n, row-major, leading
 * dimension n, host memory unless APSP_DEVICE_INPUT; its diagonal is ignored
 * (read as 0).  D is computed by blocked Floyd-Warshall on the device, or
 * taken from D_or_null when APSP_D_GIVEN is set.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream); every later call on the
 * handle runs on it.  On success *g owns its device memory until
 * apsp_destroy. */
apsp_status apsp_init(apsp_graph **g, const void *W, int32_t n, int32_t capacity,
                      apsp_dtype dtype, uint32_t flags, const void *D_or_null,
                      void *cuda_stream);
apsp_status apsp_destroy(apsp_graph *g);

/* Optional: route the library's device allocations through a caller's
 * allocator (for example a framework's caching allocator).  Affects handles
 * created afterwards.  Pass NULLs to restore cudaMalloc / cudaFree. */
typedef void *(*apsp_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*apsp_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
apsp_status apsp_set_allocator(apsp_alloc_fn alloc, apsp_free_fn free_fn, void *ctx);

/* ----- updates (Sections 3.1-3.3) ---------------------------------------- */

/* Add a node p (Section 3.1; Corollaries 1, 2, Theorem 3).  in_w[t] is the
 * weight of edge t -> p and out_w[t] of p -> t, both arrays of `capacity`
 * elements indexed by slot, host memory; entries at dead slots and at p are
 * ignored.  Undirected graphs: in_w may be NULL or must equal out_w.  The
 * new node's slot is written to *new_id. */
apsp_status apsp_add_node(apsp_graph *g, const void *in_w, const void *out_w, int32_t *new_id);
/* Same with in_w / out_w in device memory (read on the stream). */
apsp_status apsp_add_node_device(apsp_graph *g, const void *in_w, const void *out_w, int32_t *new_id);

/* Remove node v (Section 3.2, Algorithm 5): detect the need_update_list,
 * compute Cost, then re-relax the listed pairs (warm) or recompute D by
 * Floyd-Warshall (cold), as the dispatch mode decides on the device. */
apsp_status apsp_remove_node(apsp_graph *g, int32_t v);

/* Set the weight of edge u -> v (and v -> u for undirected graphs) to *w
 * (host pointer to one element of the graph's dtype; APSP_INF_I32 / +inf
 * deletes the edge).  The result is the APSP matrix of the modified graph,
 * the quantity Algorithm 6 (Section 3.3) computes. */
apsp_status apsp_update_edge(apsp_graph *g, int32_t u, int32_t v, const void *w);

/* Recompute D from the current weights by blocked Floyd-Warshall (the cold
 * path, also used as the comparison baseline). */
apsp_status apsp_recompute(apsp_graph *g);

/* ----- queries ------------------------------------------------------------ */

/* Distance u -> v into *dist_out (host, one element of the dtype).  Waits. */
apsp_status apsp_query(apsp_graph *g, int32_t u, int32_t v, void *dist_out);
/* count distances: pairs uv[2*i], uv[2*i+1] (host int32), results into out
 * (host, count elements).  Waits. */
apsp_status apsp_query_batch(apsp_graph *g, const int32_t *uv, int32_t count, void *out);

/* ----- path queries (Section 4) -----------------------------------------
 * Algorithm 7 (warm-start shortest path): from the resident APSP matrix, the
 * candidate list of the pair -- u, every live node t with not
 * D[u][v] < D[u][t] + D[t][v] (in increasing slot order), then v; by Theorem
 * al_correct it holds every shortest u -> v path -- and Dijkstra on the small
 * graph of the weights among the candidates.  Ties: the next settled node is
 * the one of least distance and lowest candidate index; a predecessor changes
 * only on a strict improvement.  The float candidate test keeps t within a
 * relative slack of 2^-8 (extra candidates only enlarge the small graph).
 * Result: the slots of one shortest path u, ..., v; [u] when u == v; empty
 * (length 0) when v is unreachable.  All buffers are host memory owned by the
 * caller; the calls wait for the GPU.  Errors: APSP_E_NODE for a dead or
 * out-of-range id; APSP_E_ARG for bad sizes / null pointers, or if the small
 * graph does not reach v (possible only when an APSP_D_GIVEN matrix was not
 * the APSP matrix of W). */

/* count queries: pairs uv[2*q], uv[2*q+1].  lens[q] receives the number of
 * nodes of path q and paths[q*stride ..] its first min(lens[q], stride)
 * slots (a longer path is cut; lens[q] still gives its full length). */
apsp_status apsp_query_paths(apsp_graph *g, const int32_t *uv, int32_t count, int32_t *paths, int32_t stride,
                             int32_t *lens);
/* One query: path[0 .. min(*len, cap)) as above. */
apsp_status apsp_query_path(apsp_graph *g, int32_t u, int32_t v, int32_t *path, int32_t cap, int32_t *len);
/* Algorithm 8 (warm-start "all shortest paths") on Algorithm 7's small graph:
 * Algorithm 7's path first, then for each candidate t other than u and v (in
 * candidate order) the tree path u -> t of the forward Dijkstra joined to the
 * tree path t -> v of a Dijkstra from v on the reversed small graph, unless
 * already listed or not loop-free (a zero-weight cycle can make the join a
 * walk).  Every listed path is a shortest path; the list need not hold all
 * of them.  Path p is nodes[offsets[p] .. offsets[p + 1]); *n_paths and
 * *n_nodes receive the counts.  With nodes or offsets NULL only the counts
 * are returned; if paths_cap < *n_paths or nodes_cap < *n_nodes nothing is
 * written and APSP_E_ARG is returned (offsets needs paths_cap + 1 entries). */
apsp_status apsp_query_all_paths(apsp_graph *g, int32_t u, int32_t v, int32_t *nodes, int64_t nodes_cap,
                                 int64_t *offsets, int32_t paths_cap, int32_t *n_paths, int64_t *n_nodes);

/* Next hops (the hot-path plan's optional next-hop output), derived from the
 * resident D and W when asked for rather than carried through every update:
 * for each of the `count` live rows i = rows[r] (host int32),
 * out[r * ld_out + j] (host, ld_out >= n_slots) receives for j < n_slots the
 * lowest live slot t != i with W[i][t] + D[t][j] == D[i][j] (fp32: within the
 * 2^-8 tightness slack) -- the first hop of a shortest walk i -> t ~> j --,
 * i for j == i and -1 where j is dead or unreachable.  With positive weights
 * following next hops from i reaches j along a shortest path; zero-weight
 * cycles can make them loop (use apsp_query_path for paths then).  Cost per
 * row: the row's tight out-edges times n_slots reads of D.  APSP_E_NODE for a
 * dead or out-of-range row; APSP_E_UNSUPPORTED for APSP_MINIMAX graphs.
 * Waits. */
apsp_status apsp_next_hops(apsp_graph *g, const int32_t *rows, int32_t count, int32_t *out, int64_t ld_out);

/* Copy the n_slots x n_slots top-left block of D (or W) to dst with leading
 * dimension ld_dst (elements); dst is device memory if dst_on_device, else
 * host.  Dead slots read as missing.  Waits. */
apsp_status apsp_copy_D(apsp_graph *g, void *dst, int64_t ld_dst, int32_t dst_on_device);
apsp_status apsp_copy_W(apsp_graph *g, void *dst, int64_t ld_dst, int32_t dst_on_device);
/* alive[s] = 1 for a live slot s, 0 otherwise; `capacity` bytes, host. */
apsp_status apsp_copy_alive(apsp_graph *g, uint8_t *alive);

apsp_status apsp_info_get(apsp_graph *g, apsp_info *info);
/* Statistics of the last update.  Waits. */
apsp_status apsp_last_stats(apsp_graph *g, apsp_stats *stats);
/* Wait for all work on the handle's stream; returns any deferred device error. */
apsp_status apsp_sync(apsp_graph *g);

/* The list of (i, j) pairs that the last update re-relaxed or handed to the
 * cold path: for a removal of k, the need_update_list of Section 3.2 (every
 * pair of live i, j other than k with D[i][k] + D[k][j] == D[i][j], Corollary
 * 3), for a tight edge increase the pairs whose every shortest path may use
 * the edge; filtered as apsp_set_list_mode chose.  ij receives 2 * *count
 * int32 (i, j, i, j, ...) in no particular order; *count = 0 after any other
 * update.  With ij NULL only *count is written; cap (pairs) below *count
 * gives APSP_E_ARG; a list that overflowed the scratch gives
 * APSP_E_CAPACITY.  Host memory; waits. */
apsp_status apsp_copy_last_list(apsp_graph *g, int32_t *ij, int64_t cap, int64_t *count);

/* ----- dispatch ----------------------------------------------------------- */

/* Choose how removals and edge increases pick warm or cold (default:
 * APSP_DISPATCH_DELTA with delta = 1.0, i.e. cold only when the affected set
 * overflows the scratch capacity). */
apsp_status apsp_set_dispatch(apsp_graph *g, apsp_dispatch mode, double delta);

/* Algorithm 12 (Theorem theo_algo12): the need_update_list of a removal is
 * the set of Corollary 3's pairs whose distance actually grows (k needed by
 * every shortest path), and likewise for an edge increase with the old edge.
 * With `on`, each removal / increase also counts that list after its repair
 * (one extra kernel over the listed pairs, comparing each final distance with
 * its old tight sum) and apsp_last_stats reports grown_pairs / grown_rows /
 * grown_cost.  int32: exact; fp32: "grew" beyond the 2^-8 tightness slack.
 * The result of every update is the same either way. */
apsp_status apsp_set_exact_list(apsp_graph *g, int32_t on);

/* Which pairs removals and edge increases re-relax (the result of every
 * update is the same in every mode; affected_pairs / affected_rows and Cost
 * count the chosen list):
 *   APSP_LIST_COROLLARY3   Section 3.2's need_update_list: every pair with
 *                          D[i][k] + D[k][j] == D[i][j] (the default);
 *   APSP_LIST_DIRECT_EDGE  minus the pairs whose direct edge is itself a
 *                          shortest path (W[i][j] == D[i][j]): that edge avoids
 *                          the removed node, and an increased edge's weight is
 *                          already the new one, so they keep their distance;
 *   APSP_LIST_ALGORITHM12  Algorithm 12: each listed pair keeps its place only
 *                          if Dijkstra on Algorithm 7's small graph without the
 *                          removed node (for an increase: with the edge's new
 *                          weight) does not reach j within its old distance --
 *                          by Theorem theo_algo12 exactly the pairs whose
 *                          distance grows.  Pairs whose small graph has more
 *                          than 126 candidates stay listed (always safe).
 * On this library's pair-parallel repair neither filter pays for itself on
 * the workloads measured (n = 16384 undirected Euclidean updates): the
 * direct-edge test drops 3 % of the pairs, and Algorithm 12's test, which
 * cuts the list to under a tenth, costs about 20x the re-relaxation it
 * spares.  They serve comparisons with the paper's Algorithm 11 / 12. */
typedef enum { APSP_LIST_COROLLARY3 = 0, APSP_LIST_DIRECT_EDGE = 1, APSP_LIST_ALGORITHM12 = 2 } apsp_list_mode;
apsp_status apsp_set_list_mode(apsp_graph *g, apsp_list_mode mode);

/* ----- learned warm/cold cost model ---------------------------------------
 * Algorithm 5 chooses between re-running the affected rows and recomputing
 * everything with a threshold delta on Cost (Definition of Cost, Section
 * 3.2).  APSP_DISPATCH_MODEL replaces the threshold with a small regression
 * model evaluated on the device at the decision point: a multilayer
 * perceptron 6 -> 64 -> 64 -> 2 with ReLU hidden layers (fp32) that predicts
 * log2(microseconds) of the warm and of the cold path; the smaller wins.
 *
 * Features of an update (computed on the device from detection counters):
 *   0 update type (0 add, 1/3 removal, 2/3 decrease, 1 increase)
 *   1 log2(N), N = live nodes before the update
 *   2 relative weight change (w_new - w_old) / w_old (0 for node updates)
 *   3 affected pairs / N^2
 *   4 Cost = rows with an affected pair / (N - 1)
 *   5 rows with an affected pair / N
 * Parameter block (APSP_MODEL_NPARAM floats, this order): mu[6], sd[6]
 * (features are standardised as (f - mu) / sd), W1[64][6], b1[64],
 * W2[64][64], b2[64], W3[2][64], b3[2]; output o = W3 relu(W2 relu(W1 x +
 * b1) + b2) + b3.  The trainable part starts at W1 (APSP_MODEL_NTRAIN floats).
 *
 * The training entry points are stateless and run on the current CUDA
 * device; all buffers are host memory owned by the caller.  Labels Y are
 * n x 2 (warm, cold) log2 microseconds; a NaN label is missing and
 * contributes nothing.  Loss = (1/n) sum over samples and outputs of
 * (o - y)^2 over present labels. */
#define APSP_MODEL_NPARAM 4750
#define APSP_MODEL_NTRAIN 4738

/* Install model parameters (host, APSP_MODEL_NPARAM floats) on the handle;
 * used by APSP_DISPATCH_MODEL.  params == NULL removes the model. */
apsp_status apsp_set_model(apsp_graph *g, const float *params);
/* Loss and its gradient with respect to the trainable parameters over all n
 * samples (X: n x 6 raw features, row-major; grad: APSP_MODEL_NTRAIN floats
 * in parameter order).  Hand-written forward / backward kernels. */
apsp_status apsp_model_loss_grad(const float *params, const float *X, const float *Y, int32_t n, float *loss,
                                 float *grad);
/* Outputs (n x 2) of the model for n raw feature rows. */
apsp_status apsp_model_predict(const float *params, const float *X, int32_t n, float *out);
/* Trains a model from scratch: standardisation from X, He-initialised
 * weights from `seed` (SplitMix64), mini-batch Adam (beta 0.9 / 0.999) with
 * learning rate lr for `epochs` passes over a per-epoch shuffle.  Writes
 * APSP_MODEL_NPARAM floats to params_out and the final full-data loss. */
apsp_status apsp_model_train(const float *X, const float *Y, int32_t n, int32_t epochs, int32_t batch, float lr,
                             uint64_t seed, float *params_out, float *final_loss);

/* ----- batched execution: many graphs, one persistent launch --------------
 * A batch applies ordered update sequences to several independent graphs
 * with ONE persistent kernel: CTAs take graphs from a device queue and each
 * applies its graph's updates in order (add: Corollaries 1-2 and Theorem 3;
 * removal and edge increase: Corollary 3's test, starting upper bounds and
 * re-relaxation to the fixed point; edge decrease: the exact closed form).
 * Results are the same exact matrices as the one-call-per-update path.
 * Graphs must be directed, of one dtype, with capacity <= APSP_BATCH_MAX_SLOTS.
 * Items of one graph are applied in their order in `items`; items of
 * different graphs are independent.  The call validates every item first
 * (nothing changes on an error), waits for each graph's pending work, and
 * returns when the batch is done.  new_ids (count entries, may be NULL)
 * receives the slot of each ADD and -1 for the other items. */
#define APSP_BATCH_MAX_SLOTS 8192
typedef enum { APSP_BATCH_ADD = 0, APSP_BATCH_REMOVE = 1, APSP_BATCH_EDGE = 2 } apsp_batch_op;
typedef struct {
    int32_t graph;            /* index into the graphs array of the call */
    int32_t op;               /* apsp_batch_op */
    int32_t u, v;             /* REMOVE: node u; EDGE: edge (u, v) */
    const void *in_w;         /* ADD: host, `capacity` weights w(t -> new) (see apsp_add_node) */
    const void *out_w;        /* ADD: host, `capacity` weights w(new -> t) */
    double w;                 /* EDGE: new weight; missing (INF_I32 / +inf or larger) deletes the edge */
} apsp_batch_item;
typedef struct apsp_batch apsp_batch;
/* An executor with its own stream (cuda_stream, or a new one when NULL) and
 * device buffers that grow as needed. */
apsp_status apsp_batch_create(apsp_batch **b, void *cuda_stream);
apsp_status apsp_batch_run(apsp_batch *b, apsp_graph *const *graphs, int32_t n_graphs, const apsp_batch_item *items,
                           int32_t count, int32_t *new_ids);
apsp_status apsp_batch_destroy(apsp_batch *b);
/* Each launch is one CUDA graph (upload, persistent kernel, status
 * read-back), captured once per dtype and CTA width on the executor and then
 * replayed with updated parameters.  The CTA width (128, 256 or 512 threads)
 * is chosen by a process-wide autotuner per dtype and size bucket
 * (ceil(log2) of the batch's widest span): each width runs two batches of at
 * least 2^20 span^2 of work, then the one with the least device time per
 * span^2 is kept.  Widths never change results.  threads = 0 restores the
 * autotuner; 128 / 256 / 512 fixes the width for this executor. */
apsp_status apsp_batch_set_width(apsp_batch *b, int32_t threads);
typedef struct {
    int64_t launches;         /* batches launched */
    int64_t graph_captures;   /* CUDA graphs captured */
    int64_t graph_replays;    /* launches that replayed a captured graph */
    int32_t last_width;       /* CTA width of the last launch */
    int32_t fixed_width;      /* 0 when the autotuner chooses */
} apsp_batch_info;
apsp_status apsp_batch_info_get(apsp_batch *b, apsp_batch_info *info);
/* The autotuner's settled width for batches whose widest span is max_span (0
 * while it is still measuring). */
apsp_status apsp_batch_tuned_width(apsp_dtype dtype, int32_t max_span, int32_t *threads);

/* ----- serving loop ---------------------------------------------------------
 * Replays a trace of timed requests against resident graphs in real time
 * through an online server (apsp_server_*, below): each request is submitted
 * at its arrival time and served with the server's continuous batching.  Per
 * graph, requests take effect in arrival order, so every graph ends exactly
 * as if its requests had been applied alone.  Requests must be sorted by
 * arrival time; admit_s / done_s are seconds after the start of the call. */
#define APSP_BATCH_QUERY 3    /* request op besides apsp_batch_op: distance u -> v */
typedef struct {
    apsp_batch_item item;     /* ADD / REMOVE / EDGE, or APSP_BATCH_QUERY with (u, v) */
    double arrival_s;         /* seconds after the start of apsp_serve */
} apsp_request;
typedef struct {
    double admit_s;           /* seconds after the start: taken into a wave */
    double done_s;            /* seconds after the start: result visible on the host */
    double dist;              /* QUERY: the distance (missing: INF_I32 or +inf) */
    int32_t status;           /* apsp_status of the request */
    int32_t wave;             /* wave that served it */
    int32_t new_id;           /* ADD: the new node's slot, else -1 */
    int32_t pad_;
} apsp_request_result;
typedef struct {
    double hbm_budget_bytes;  /* bytes of graph state (W, D, D^T) in work at once; 0 = unlimited
                                 (a single graph larger than the budget still runs alone) */
    int32_t small_max_slots;  /* graphs of capacity <= this use the batched kernel (0: none) */
    int32_t max_wave_requests;/* 0 = unlimited */
} apsp_serve_config;
apsp_status apsp_serve(apsp_graph *const *graphs, int32_t n_graphs, const apsp_request *reqs, int32_t count,
                       const apsp_serve_config *cfg, apsp_request_result *results);

/* ----- online server --------------------------------------------------------
 * A server owns a worker thread that applies requests to resident graphs as
 * they arrive, with continuous batching: every graph has a FIFO of requests;
 * whenever a graph has no work on the GPU it takes the requests queued for it
 * (up to and including its first query, so a query sees exactly the updates
 * submitted before it for that graph) and they go to the GPU at once -- small
 * graphs (capacity <= cfg.small_max_slots) together in one persistent batched
 * launch, the others one call per update on their own streams.  A graph whose
 * work completes is served again at once, whatever the other graphs are
 * doing, so small graphs are not held back by a large graph's repair.  A graph
 * is admitted only while the graph state on the GPU stays within
 * cfg.hbm_budget_bytes (a graph larger than the budget still runs alone).
 * Per graph, requests take effect in submission order: every graph ends as if
 * its requests had been applied alone.  Results report the time the request
 * went to the GPU (admit_s) and the time its completion was observed (done_s)
 * in seconds on the server's clock (apsp_server_clock), `wave` = the dispatch
 * round that took it.  While a server lives, the served graphs must not be
 * used by any other call.  submit / poll / wait / clock may be called from
 * any host thread. */
typedef struct apsp_server apsp_server;
/* Graphs of one dtype, not APSP_MINIMAX.  cfg is copied. */
apsp_status apsp_server_create(apsp_server **s, apsp_graph *const *graphs, int32_t n_graphs,
                               const apsp_serve_config *cfg);
/* Queues one request (an apsp_batch_item whose graph indexes the server's
 * graphs; op APSP_BATCH_ADD / REMOVE / EDGE or APSP_BATCH_QUERY with (u, v)).
 * The weight vectors of an ADD are copied, so the caller's buffers may be
 * reused at once.  *ticket identifies the request (0, 1, 2, ... in
 * submission order).  An invalid request completes with its error status. */
apsp_status apsp_server_submit(apsp_server *s, const apsp_batch_item *item, int64_t *ticket);
/* Non-blocking: *done = 1 and *res filled once the request has completed. */
apsp_status apsp_server_poll(apsp_server *s, int64_t ticket, apsp_request_result *res, int32_t *done);
/* Waits up to timeout_s seconds for the request; APSP_E_BUSY if it has not
 * completed by then. */
apsp_status apsp_server_wait(apsp_server *s, int64_t ticket, double timeout_s, apsp_request_result *res);
/* Seconds since the server was created (the clock of admit_s / done_s). */
double apsp_server_clock(apsp_server *s);
/* Completes every submitted request, then stops the worker and frees the
 * server (the graphs stay valid). */
apsp_status apsp_server_destroy(apsp_server *s);

/* ----- instrumentation ---------------------------------------------------- */

/* Number of kernels this handle has launched so far, counting the kernels an
 * edge increase's graph ran (its detection and repair run only when the edge
 * was tight).  Waits for the handle's stream; -1 for a null handle. */
int64_t apsp_launch_count(apsp_graph *g);
/* When on, every kernel launch is bracketed by CUDA events on the handle's
 * stream and its time is accumulated per kernel name. */
apsp_status apsp_profile_enable(apsp_graph *g, int32_t on);
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} apsp_profile_entry;
/* Waits, then copies up to cap entries; *count = number of distinct kernels. */
apsp_status apsp_profile_read(apsp_graph *g, apsp_profile_entry *out, int32_t cap, int32_t *count);
apsp_status apsp_profile_reset(apsp_graph *g);

/* Measurement probes (instrumentation; the paper has no counterpart): the
 * ceilings that the cold solver and the first re-relaxation pass are reported
 * against.
 *
 * Measures, on the current CUDA device, how many min-plus steps min(a + b, c)
 * of the given dtype the CUDA cores issue per second when every thread keeps
 * an 8 x 8 register tile of them (the inner loop of the cold Floyd-Warshall)
 * and touches no memory: the ceiling against which the cold path's n^3 steps
 * are reported.  Takes a few milliseconds; waits for the device. */
apsp_status apsp_probe_addmin_rate(apsp_dtype dtype, double *pair_ops_per_s);
/* Measures the L2 read bandwidth of the current CUDA device (GB/s): 16-byte
 * coalesced loads from a warm buffer of a quarter of L2, 8 in flight per
 * thread.  The ceiling of the first re-relaxation pass, whose reads are
 * served by L2.  Takes a few milliseconds; waits for the device. */
apsp_status apsp_probe_l2_read_gbs(double *gbs);
/* Failure-detection self-test (no paper counterpart): launches two CTAs
 * cooperatively that meet at the same bounded grid barrier the repair kernel
 * uses.  With lose_cta set, one CTA leaves without arriving, so the other's
 * wait ends only by its 2-second limit; *status_out is then APSP_E_TIMEOUT
 * (else APSP_OK) and the device stays usable.  Nothing faults, traps or hangs.
 * Uses the legacy default stream and waits. */
apsp_status apsp_selftest_barrier_timeout(int32_t lose_cta, int32_t *status_out);

/* ----- insertion without allocation ---------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they add a node (a request handler that
 * must not block on cudaMalloc, which synchronises the device; a framework
 * that owns all device memory through its own pool; a fixed memory budget).
 *
 * Adds node p to a caller-owned APSP matrix D in place and gives the matrix
 * apsp_add_node gives: D (device, 16-byte aligned, leading dimension ld
 * elements, a multiple of 4 and >= n_slots) holds on entry the APSP matrix of
 * the live slots among the first n_slots; on return it also holds row and
 * column p.  Only entries whose row and column are both live and not p are
 * read: row and column p, the rows and columns of dead slots and the padding
 * beyond n_slots may hold anything (int32 values >= APSP_INF_I32 read as
 * missing).  Row p is written over all n_slots columns (missing at dead
 * slots) and column p at live rows; no other entry of a dead slot changes.
 * alive (device, n_slots int32: 1 = live, p must be 0 and is not changed),
 * in_w / out_w (device, n_slots weights t -> p and p -> t) are only read.
 * n_slots must be a multiple of 4 in [4, APSP_NOALLOC_MAX_SLOTS]
 * (APSP_E_CAPACITY above the maximum, APSP_E_ARG otherwise); negative or NaN
 * weights are read as missing edges.
 *
 * Scratch lives in one fixed library-owned device array of
 * 4 * APSP_NOALLOC_MAX_SLOTS * 4 bytes (256 KiB) that every GPU loading the
 * library holds until the process exits; the call allocates nothing and does
 * not wait for the GPU.  Each call looks up the array's device address on the
 * current device; the first call on a device (or the first after its context
 * was reset) loads the library's device code, so make it before any CUDA
 * stream capture.  All calls share the array (each re-initialises it): calls
 * whose work overlaps on the GPU race and must be serialised by the caller. */
#define APSP_NOALLOC_MAX_SLOTS 16384
apsp_status apsp_add_node_noalloc(void *D, int64_t ld, int32_t n_slots, const int32_t *alive,
                                  apsp_dtype dtype, const void *in_w, const void *out_w,
                                  int32_t p, void *cuda_stream);

const char *apsp_status_string(apsp_status s);
/* The CUDA runtime error code behind this thread's last APSP_E_CUDA or
 * APSP_E_NOMEM (0 if none); *name (may be NULL) receives its name. */
int32_t apsp_last_cuda_error(const char **name);
/* Library version, e.g. "0.1.0". */
const char *apsp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* APSP_H */
