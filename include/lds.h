/*
 * liblds - top-k locally densest subgraphs (LDS, edge density) and locally
 * triangle-densest subgraphs (LTDS) on one NVIDIA GB300 (sm_103a), following
 * arXiv 2504.10937, "Finding Locally Densest Subgraphs: Convex Programming with
 * Edge and Triangle Density".
 *
 * Conventions for every entry point
 *   - Vertex ids are int32 in [0, n), n <= 2^31 - 2.  The graph is simple and
 *     undirected; input pairs may repeat, appear in either orientation or be
 *     self-loops: repeats and self-loops are dropped at ingest (Sec. 3).
 *   - "Canonical edge order" is the list of distinct pairs (u, v), u < v,
 *     sorted by (u, v).  "Triangle order" lists every triangle {a < b < c}
 *     sorted by (a, b, c).  Every per-edge / per-triangle array in and out of
 *     the library uses these orders and original vertex ids.
 *   - Buffers are host or device memory as the lds_mem argument says; the
 *     caller owns every buffer it passes, and the library keeps no pointer to
 *     them after the call returns.
 *   - Calls enqueue work on the graph's stream (set at creation, NULL = the
 *     legacy default stream) and return when results are visible to the
 *     caller.  A handle must not be used from two threads at once; different
 *     handles are independent.
 *   - No call throws.  Each returns an lds_status; on failure lds_last_error()
 *     gives a thread-local message and output buffers are unspecified.
 *   - There is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns LDS_ECUDA.
 */
#ifndef LDS_H
#define LDS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LDS_OK = 0,
    LDS_EINVAL = 1,     /* bad argument: id out of range, null pointer, size  */
    LDS_ENOMEM = 2,     /* device or host allocation failed                   */
    LDS_ECUDA = 3,      /* CUDA runtime error or no device                    */
    LDS_ETIMEOUT = 4,   /* a bounded device loop hit its iteration cap        */
    LDS_EOVERFLOW = 5,  /* a value does not fit the integer range used        */
    LDS_EBUSY = 6       /* request refused: over the memory budget            */
} lds_status;

typedef enum { LDS_EDGE = 0, LDS_TRIANGLE = 1 } lds_density;

/* Arithmetic of the Frank-Wolfe iterations (Alg. 1 / Alg. 6).
 *   LDS_EXACT: integer form.  With D_i = (i+1)(i+2), W = D_i alpha and
 *              R = D_i r are integers (3 D_i for triangles); bit-exact.
 *   LDS_FP32:  loads carried in binary32 by r <- (1-gamma) r + gamma c (the sum
 *              of Alg. 1's alpha update over a vertex's edges); the weights are
 *              rebuilt exactly from the choices made.
 *   LDS_FP64:  Alg. 1 / Alg. 6 literally in binary64: one alpha per ordered
 *              pair (vertex-triangle pair), r summed per vertex in ascending
 *              neighbour (triangle) order.  The plain reference path.        */
typedef enum { LDS_EXACT = 0, LDS_FP64 = 1, LDS_FP32 = 2 } lds_precision;

typedef enum { LDS_MEM_HOST = 0, LDS_MEM_DEVICE = 1 } lds_mem;

typedef struct lds_graph lds_graph;

typedef struct {
    int32_t n;                 /* vertices                                    */
    int64_t m;                 /* distinct undirected edges                   */
    int64_t input_pairs;       /* pairs passed to lds_create_graph            */
    int64_t self_loops;        /* of which self-loops (dropped)               */
    int64_t duplicates;        /* of which repeats of an earlier pair         */
    int32_t max_degree;
    int32_t isolated;          /* vertices without an edge                    */
    int64_t triangles;         /* |T| once listed (lds_list_triangles), else -1 */
} lds_graph_info_t;

/* Library version string. */
const char* lds_version(void);

/* Thread-local message of the last failing call on this thread. */
const char* lds_last_error(void);

/* Number of CUDA devices visible (0 when none); never fails. */
int32_t lds_device_count(void);

/* Graph ingest (Sec. 3: G = (V, E) simple and undirected).
 *   n          number of vertices
 *   m          number of input pairs (src[i], dst[i])
 *   src, dst   int32[m] in host or device memory per `where`; copied
 *   stream     cudaStream_t for all work on this graph (NULL: default stream)
 *   out        receives the new handle; free with lds_free
 * Builds the canonical edge list and a symmetric CSR on the device.
 * Errors: LDS_EINVAL (n < 0, m < 0, null pointers, id outside [0, n)),
 *         LDS_ENOMEM, LDS_ECUDA. */
lds_status lds_create_graph(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            lds_mem where, void* stream, lds_graph** out);

/* Releases every device buffer of the handle (NULL is ignored). */
void lds_free(lds_graph* g);

lds_status lds_graph_info(const lds_graph* g, lds_graph_info_t* info);

/* Canonical edges: u[e] < v[e], int32[m] each, sorted by (u, v). */
lds_status lds_get_edges(const lds_graph* g, int32_t* u, int32_t* v, lds_mem where);

/* Triangle listing (the set T of Eq. 3 / Eq. 4, needed by Alg. 6 and Alg. 7).
 * Lists T once and keeps it on the device with the handle; writes |T|.
 * Errors: LDS_ENOMEM when T does not fit, LDS_ECUDA. */
lds_status lds_list_triangles(lds_graph* g, int64_t* count);

/* Copies T (after lds_list_triangles) as int32[3 |T|] rows (a, b, c), a < b < c,
 * in triangle order. */
lds_status lds_get_triangles(lds_graph* g, int32_t* tri, lds_mem where);

/* Core numbers (Def. 6) or tr-core numbers (Def. 11) of every vertex: int64[n].
 * LDS_TRIANGLE lists triangles first if needed. */
lds_status lds_core_numbers(lds_graph* g, lds_density d, int64_t* core, lds_mem where);

/* Compact numbers phi(u) (Def. 4; tr-compact for LDS_TRIANGLE, Def. 10) of every
 * vertex, exactly, as reduced fractions num[u] / den[u] (int64[n] each; den >= 1,
 * phi = 0 for a vertex in no edge / triangle).  By Thm. 1 and Thm. 4 they are the
 * optimal loads r* of the convex program; here they come from the
 * density-friendly decomposition (Sec. 4.2), one maximum flow of Alg. 8's
 * network per split: at the mean ratio rho of a vertex set F (patterns inside the
 * settled levels above plus F and touching F, over |F|), the largest minimum-cut
 * source side is {u in F : phi(u) >= rho}, which is all of F exactly when F is
 * one level.  Same answer as lds_topk's exact settle.  Errors: LDS_EINVAL,
 * LDS_ENOMEM, LDS_ECUDA, LDS_EOVERFLOW (more than 2^31 - 1 patterns in one
 * sub-problem). */
lds_status lds_compact_numbers(lds_graph* g, lds_density d, int64_t* num, int64_t* den, lds_mem where);

/* Results of lds_fw; every pointer may be NULL to skip that output.        */
typedef struct {
    double*  r;        /* [n] loads r_u after `iters` iterations: EXACT gives R_u / D
                          rounded once, FP32 the binary32 value, FP64 the binary64 value */
    int64_t* R;        /* [n] exact scaled loads of the returned weights: R_u = D r_u   */
    int64_t* W;        /* [m] D alpha_{u,v} per canonical edge (edge density), or
                          [3 |T|] D alpha_{w,t} per triangle row (triangle density)     */
    uint8_t* last;     /* [m] alpha_hat_{u,v} of the last iteration (1: u received), or
                          [|T|] column (0, 1, 2) of the triangle's receiving vertex     */
    int64_t  D;        /* out: denominator, (N+1)(N+2) (edges) or 3(N+1)(N+2)           */
} lds_fw_result;

/* Frank-Wolfe for CP(G) (Eq. 2, Alg. 1) or for the triangle program (Eq. 4,
 * Alg. 6) from the initial point alpha = 1/2 (1/3), `iters` iterations.
 * Ties: an edge (u, v), u < v, goes to u only when r_u < r_v (Alg. 1), so ties
 * go to the larger id; a triangle goes to its lowest-load vertex, ties to the
 * larger id (appendix, proof of Thm. 4).
 *   where   memory kind of every output pointer in `out`
 * Errors: LDS_EINVAL (iters < 0, iters > 60000, bad precision),
 *         LDS_EOVERFLOW (scaled loads exceed int64), LDS_ENOMEM, LDS_ECUDA. */
lds_status lds_fw(lds_graph* g, lds_density d, int32_t iters, lds_precision p, lds_mem where,
                  lds_fw_result* out);

/* Times of the most recent lds_fw call on this handle, measured with CUDA events
 * on the handle's stream (pass times only while lds_set_pass_profiling is on).
 *   fw_ms          all iterations, from the first pass to the last fold
 *   pass_us        average duration of the per-iteration pass kernel
 *   pass_launches  number of pass launches timed
 *   pass_bytes     algorithmic bytes one pass must move (the roofline numerator):
 *                  every stored slot's column word, the per-chunk row index and
 *                  bit-plane word, and one load (key) read per vertex
 *   pass_kernel    name of the pass kernel used (static string)
 * Any pointer may be NULL. */
/* The current Frank-Wolfe state of the handle (left by lds_fw, lds_fw_batch or
 * the first round of lds_topk) copied out as lds_fw does: r, R, W in original
 * ids and canonical order (`last` must be NULL unless the state kept it).
 * Errors: LDS_EINVAL when the handle holds no state. */
lds_status lds_fw_state(lds_graph* g, lds_mem where, lds_fw_result* out);

/* Edge-density Frank-Wolfe (Alg. 1) of `iters` iterations on `count` distinct
 * graphs.  Every graph whose non-isolated vertices fit in shared memory
 * (at most 24,576, and max degree x D_iters below 2^32; EXACT or FP32) runs
 * in one persistent launch: one CTA per SM takes graphs from a queue, largest
 * first, and runs all iterations of a graph with its loads and counts on chip.
 * The others run as lds_fw does.  Each handle is left with exactly the state
 * lds_fw(g, LDS_EDGE, iters, p, ...) would leave (same iterates, ties and
 * rounding), and the next lds_topk on it with the same iterations and
 * arithmetic takes that state for its first round instead of recomputing it.
 *   onchip   receives how many graphs ran on chip (may be NULL)
 * Errors: LDS_EINVAL (NULL or repeated graph, bad iters or precision),
 * LDS_ENOMEM, LDS_ECUDA. */
lds_status lds_fw_batch(int32_t count, lds_graph** graphs, int32_t iters, lds_precision p, int32_t* onchip);

/* Threads per graph (32 x warps per graph) that lds_fw_batch's persistent launch
 * uses for graphs of `nact` active vertices: graphs are grouped by size bucket
 * (the bit length of nact), each bucket launched with shared memory for its
 * largest graph and as many CTAs per SM as fit.  lds_batch_autotune times 128,
 * 256, 512 and 1024 threads per graph on its batch, per bucket, and keeps the
 * fastest for the rest of the process; untuned buckets use 1024.  Never fails. */
int32_t lds_fw_batch_threads(int32_t nact);

lds_status lds_fw_last_timing(const lds_graph* g, double* fw_ms, double* pass_us,
                              int64_t* pass_launches, int64_t* pass_bytes, const char** pass_kernel);

/* Stable groups of the last lds_fw run on this handle (Alg. 2; Def. 5 for edge
 * density, Def. 12 for triangle density) with the bounds of Lemma 4 / Lemma 8.
 * Vertices are sorted by exact load descending, ties by id ascending; candidate
 * groups end at the cut points (positions j whose prefix density beats every
 * longer prefix); each candidate is checked on a modified feasible solution and
 * merged with the next one when it fails.  Every output is a host array:
 *   order      [n]  vertices in sorted order (original ids)
 *   ngroups         number of accepted groups; group k covers positions
 *                   [group_end[k-1], group_end[k]) (group_end[-1] = 0); positions
 *                   after the last group form the unaccepted remainder
 *   group_end  [n]  exclusive end positions
 *   lo_num, hi_num [n]  lo_num[k] / D <= phi(u) <= hi_num[k] / D for u in group k
 *   D               common denominator ((N+1)(N+2), or 3(N+1)(N+2) for triangles)
 *   ncuts, cuts [n] number and 1-based positions of the cut points
 * Any output pointer may be NULL.  Errors: LDS_EINVAL (no lds_fw run yet),
 * LDS_EOVERFLOW (loads beyond the 64-bit sort key), LDS_ENOMEM, LDS_ECUDA. */
lds_status lds_extract_sg(lds_graph* g, int32_t* order, int32_t* ngroups, int64_t* group_end, int64_t* lo_num,
                          int64_t* hi_num, int64_t* D, int32_t* ncuts, int64_t* cuts);

/* Pruning (Alg. 3) of this graph with the given bounds on the compact numbers.
 * Pruning rule 1 (Cor. 1) removes every vertex x with an edge (x, y) such that
 * ub(x) < lb(y); Pruning rule 2 (Lemma 5, Lemma 6) then removes vertices whose
 * core number (tr-core number for LDS_TRIANGLE) in the remaining graph is below
 * lb, until none is left.
 *   ub_num, ub_den, lb_num, lb_den  host int64[n]: bounds num / den (den > 0)
 *   status  host uint8[n] output: 0 kept, 1 removed by rule 1, 2 by rule 2
 * Errors: LDS_EINVAL, LDS_ENOMEM, LDS_ECUDA. */
lds_status lds_prune(lds_graph* g, lds_density d, const int64_t* ub_num, const int64_t* ub_den,
                     const int64_t* lb_num, const int64_t* lb_den, uint8_t* status);

/* Maximum flow of the pattern network of Alg. 8: a source, one node per
 * pattern, one node per vertex, a sink; arcs source -> pattern (capacity q),
 * pattern -> each of its vertices (q), vertex -> sink (p), i.e. rho = p / q
 * scaled by q.  GPU push-relabel.
 *   nv, np            vertices and patterns
 *   pat_ptr[np + 1], pat_idx[pat_ptr[np]]  host arrays: pattern j lists vertices
 *                     pat_idx[pat_ptr[j] .. pat_ptr[j+1]) (indices in [0, nv),
 *                     distinct within a pattern; pat_ptr[0] = 0)
 *   flow              output: maximum flow value
 *   source_side[nv]   output (may be NULL): 1 for vertices on the largest source
 *                     side of a minimum cut (those that cannot reach the sink in
 *                     the final residual network; Lemma 9's cut)
 * Errors: LDS_EINVAL, LDS_ETIMEOUT (iteration bound), LDS_EOVERFLOW (np q above
 * 2^62), LDS_ENOMEM, LDS_ECUDA. */
lds_status lds_pattern_max_flow(int32_t nv, int32_t np, const int64_t* pat_ptr, const int32_t* pat_idx, int64_t p,
                                int64_t q, int64_t* flow, uint8_t* source_side);

/* Result of lds_topk, owned by the library until lds_result_free. */
typedef struct {
    int32_t  count;         /* number of sets (<= k)                                    */
    int64_t* dens_num;      /* [count] density of set i = dens_num[i] / dens_den[i],     */
    int64_t* dens_den;      /*         as a reduced fraction                              */
    int64_t* offsets;       /* [count + 1] set i is vertices[offsets[i] .. offsets[i+1])  */
    int32_t* vertices;      /* original ids, ascending within each set                   */
} lds_result;

/* Counters and phase times of the most recent lds_topk on this thread. */
typedef struct {
    int64_t fw_rounds;          /* Frank-Wolfe runs (first round + refinements)      */
    int64_t fw_edge_updates;    /* sum over runs of |E'| (|T'|) x iterations         */
    int64_t certified;          /* components that passed IsLDS / IsLTDS             */
    int64_t failed;             /* self-densest components that failed it            */
    int64_t refined;            /* refinement rounds on G[C]                         */
    int64_t exact_settled;      /* components settled by exact compact numbers       */
    int64_t skipped_by_bound;   /* groups skipped since ub < k-th density            */
    int64_t flows;              /* maximum-flow runs in verification                 */
    int64_t denser_neighbour;   /* candidates rejected by a denser neighbour         */
    double ms_total, ms_fw, ms_extract, ms_prune, ms_verify;
} lds_topk_stats_t;

/* Top-k locally densest subgraphs (Problem 1; LDScvx, Alg. 5) for LDS_EDGE, or
 * top-k locally triangle-densest subgraphs (Problem 2; LTDScvx, Sec. 6) for
 * LDS_TRIANGLE.  The answer is the k sets of largest density among all LDSs
 * (LTDSs) of positive density, densest first, ties by smallest member id; every
 * returned set is certified by IsDensest and IsLDS / IsLTDS (max-flow), and the
 * search continues until no unexamined vertex can belong to a denser one, so
 * the answer does not depend on `iters` or the arithmetic.
 *   iters   Frank-Wolfe iterations per round (refinements may use up to 8x)
 *   p       arithmetic of the iterations (lds_precision)
 *   out     receives the result; free with lds_result_free
 * Errors: LDS_EINVAL, LDS_ENOMEM, LDS_ETIMEOUT, LDS_EOVERFLOW, LDS_ECUDA. */
lds_status lds_topk(lds_graph* g, int32_t k, lds_density d, int32_t iters, lds_precision p, lds_result** out);

/* Verification network of IsLDS / IsLTDS (the Sec. 7 ablation).  All three
 * certify the same sets; they differ in the size of the flow network.
 *   LDS_VERIFY_BOUNDS  Alg. 4 / Alg. 7: U grows from S over vertices with
 *                      lb <= rho <= ub; a neighbour with lb > rho rejects S
 *                      at once, edges to denser outside vertices become loops
 *                      (the default);
 *   LDS_VERIFY_CORE    IsLDS-core / IsLTDS-core: U grows over every vertex
 *                      with ub >= rho; no lower-bound test, no loops;
 *   LDS_VERIFY_WHOLE   IsLTDS-bs (the LTDSflow baseline), and its edge
 *                      analogue: the network holds every vertex of G. */
typedef enum { LDS_VERIFY_BOUNDS = 0, LDS_VERIFY_CORE = 1, LDS_VERIFY_WHOLE = 2 } lds_verify;

/* Per-call options of lds_topk_ex; a NULL pointer means every default. */
typedef struct {
    lds_precision prec;             /* FW arithmetic (default LDS_EXACT)                     */
    void*         cuda_stream;      /* cudaStream_t for this call; NULL: the graph's stream   */
    int32_t       include_zero_density; /* 1: LDSs of density 0 (isolated vertices; for LTDS
                                       triangle-free connected sets) count as results (Def. 3
                                       makes them LDSs); default 0 drops them                  */
    lds_verify    verify;           /* verification network (default LDS_VERIFY_BOUNDS)      */
} lds_options;

/* lds_topk with per-call options (Problem 1 / Problem 2 as lds_topk states).
 * With a stream other than the graph's, the call first waits for the graph's
 * stream, runs every kernel on the given one and waits for it before returning;
 * the graph keeps its own stream afterwards.
 * Errors: as lds_topk; LDS_EINVAL for an unknown precision or verify value. */
lds_status lds_topk_ex(lds_graph* g, int32_t k, lds_density d, int32_t iters, const lds_options* opt,
                       lds_result** out);

void lds_result_free(lds_result* r);

lds_status lds_topk_last_stats(lds_topk_stats_t* stats);

/* ---- Many queries at once: batches and the serving loop.
 * Neither has a counterpart in the paper, which defines one query at a time;
 * both run the queries of lds_topk unchanged (same kernels, same answers) and
 * only decide when each one runs.  Worker threads, each with its own
 * non-blocking CUDA stream, take queries from a FIFO queue; a query starts
 * when its graph handle is idle (queries on one handle run one after another)
 * and its estimated device footprint fits in what is left of the memory
 * budget; among those the oldest starts first.  Queries on different handles
 * overlap on the device.  While a query runs, its handle works on the
 * worker's stream; the handle's own stream is synchronised before and given
 * back after.  The caller must not use a handle while one of its queries is
 * queued or running. */
typedef struct {
    lds_graph*    g;        /* graph handle (owned by the caller)          */
    int32_t       k;        /* number of sets wanted (>= 1)                 */
    lds_density   d;        /* LDS_EDGE (LDS) or LDS_TRIANGLE (LTDS)        */
    int32_t       iters;    /* Frank-Wolfe iterations per round (>= 1)      */
    lds_precision p;        /* arithmetic of the iterations                 */
} lds_query;

typedef struct lds_server lds_server;

/* Per-request timing of the serving loop. */
typedef struct {
    double  queue_ms;          /* submit -> start                             */
    double  run_ms;            /* start -> end                                */
    int64_t footprint_bytes;   /* the estimate the admission used             */
    lds_topk_stats_t stats;    /* the query's counters                        */
} lds_request_info;

/* Starts `workers` worker threads on the current device with a device-memory
 * budget of `budget_bytes` for the queries in flight.  A query's footprint is
 * estimated as 96 B per edge and per vertex plus 64 B per triangle for LTDS
 * (16 per edge stands in for |T| while the triangles are not listed yet).
 * Errors: LDS_EINVAL, LDS_ECUDA. */
lds_status lds_server_create(int64_t budget_bytes, int32_t workers, lds_server** out);

/* Queues one query and returns its ticket at once.  LDS_EBUSY when the query's
 * footprint alone exceeds the budget; LDS_EINVAL on a bad query. */
lds_status lds_server_submit(lds_server* s, const lds_query* q, int64_t* ticket);

/* *done = 1 once the query has finished (successfully or not). */
lds_status lds_server_poll(lds_server* s, int64_t ticket, int32_t* done);

/* Blocks until the query has finished, then hands over its result (free with
 * lds_result_free) and, if info is not NULL, its timing.  Returns the query's
 * own status; the ticket is retired either way. */
lds_status lds_server_wait(lds_server* s, int64_t ticket, lds_result** out, lds_request_info* info);

/* Runs every queued query to the end, stops the workers and frees what was
 * not collected. */
void lds_server_destroy(lds_server* s);

/* Runs `count` queries with `workers` worker threads (0: the count chosen by
 * lds_batch_autotune) and no memory budget.  The first rounds of edge-density
 * queries whose graph appears once in the batch run together first, in
 * lds_fw_batch's persistent launch.  results[i] / status[i] belong to
 * queries[i]; the return value is the first failure, or LDS_OK. */
lds_status lds_topk_batch(int32_t count, const lds_query* queries, int32_t workers, lds_result** results,
                          lds_status* status);

/* Tuning for a batch.  First the launch shape of the on-chip Frank-Wolfe: for
 * the batch's edge queries, every size bucket is timed with 128, 256, 512 and
 * 1024 threads per graph (see lds_fw_batch_threads).  Then the worker count:
 * the first min(count, 64) queries are timed with 1, 2, 4, 8 and 16 workers and
 * the fastest is kept.  Both choices are cached (per vertex-count bucket, and
 * per bucket of log2 of the mean edge count) for the rest of the process. */
lds_status lds_batch_autotune(int32_t count, const lds_query* queries, int32_t* workers);

/* The admission rule itself, for tests: index of the request the serving loop
 * would start next among nq queued ones (oldest first) given their footprints,
 * whether each one's graph is busy, and the free budget; -1 if none fits. */
int32_t lds_debug_pick_next(int32_t nq, const int64_t* bytes, const uint8_t* graph_busy, int64_t free_bytes);

/* Edge-density kernel choice for LDS_EXACT / LDS_FP32 (process-wide):
 *   0  automatic: a graph whose active vertices fit in shared memory (at
 *      most 24,576, every scaled load below 2^32) and with few edges (at most
 *      49,152) runs on one thread-block
 *      cluster of 8 CTAs, each holding every load word and 1/8 of the edges,
 *      the counts reduced and the new loads broadcast through distributed
 *      shared memory; otherwise the degree-oriented pass (each edge once, stored at its
 *      lower-degree endpoint, hot loads in shared memory) with 32-bit load
 *      words when every scaled load fits 32 bits, else with 64-bit keys
 *      (load, id), else variant 1.  With 32-bit words the pass counts only
 *      the receipts of the stored targets; the vertex update adds each row
 *      endpoint's receipts as the popcount of its row's bits in the
 *      iteration's choice plane, and many iterations (pass, grid barrier,
 *      update, grid barrier) run in one cooperative launch;
 *   1  the symmetric-CSR pass (each edge twice, once from each endpoint);
 *   2  the degree-oriented pass with 64-bit keys;
 *   3  as 0 with 32-bit words, both endpoints' receipts counted inside the
 *      pass, one pass launch and one update launch per iteration;
 *   4  as 0 with 32-bit words, one pass launch and one update launch per
 *      iteration;
 *   5  as 0 without the cluster form (the cooperative launch for every size);
 *   6  as 0 with the cluster form for every graph that fits, whatever its
 *      edge count.
 * All compute the same iterates.  Errors: LDS_EINVAL. */
lds_status lds_set_fw_variant(int32_t variant);

/* Maximum-flow form for the verification networks (process-wide):
 *   0  automatic: the vertex-node form (2) for every network;
 *   1  pattern-node form: Alg. 8's network with a node per pattern of three
 *      members (one- and two-member patterns contracted), asynchronous
 *      push-relabel with periodic global relabels;
 *   2  vertex-node form: no pattern nodes; a push moves part of a pattern's
 *      share from one member to another, in phases of one global relabel and
 *      one downhill sweep, all in one cooperative launch.
 * Both return the same maximum flow and the same largest minimum-cut source
 * side.  Errors: LDS_EINVAL. */
lds_status lds_set_flow_variant(int32_t variant);

/* ExtractSG walk (Alg. 2's merge loop) for lds_extract_sg and lds_topk
 * (process-wide):
 *   0  automatic: graphs of at most 65,536 vertices run every single-candidate
 *      check at once and then the whole walk in one CTA; larger graphs run the
 *      walk on the host, single checks in growing batches, and each chain of
 *      merged candidates on the device in one launch (running extremes of X
 *      and S, chunk maxima of Z, chunk minima of S recomputed where they
 *      changed);
 *   1  the large-graph walk at every size.
 * Both give the same groups and bounds.  Errors: LDS_EINVAL. */
lds_status lds_set_extract_variant(int32_t variant);

/* Number of CUDA kernels this library has launched since it was loaded
 * (process-wide counter; never fails). */
int64_t lds_launch_count(void);

/* When on != 0, lds_fw records a CUDA event pair around every pass launch so
 * that lds_fw_last_timing can report the pass kernel's average duration. */
void lds_set_pass_profiling(int32_t on);

/* Largest vertex count lds_fw_exact_noalloc accepts. */
#define LDS_NOALLOC_MAX_VERTICES (1 << 20)

/* The exact edge-density Frank-Wolfe iteration without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory themselves - a host framework that owns the whole
 * device heap, a latency-critical loop that cannot take the implicit
 * synchronisation of cudaMalloc / cudaFree, or a process whose memory budget is
 * fixed at start-up.  It computes the same R and W as lds_fw(..., LDS_EDGE,
 * iters, LDS_EXACT, ...), in one thread per edge.
 *   n        vertices, 0 <= n <= LDS_NOALLOC_MAX_VERTICES (else LDS_EINVAL)
 *   m, u, v  device int32[m] edges with 0 <= u[e] < v[e] < n, no repeats
 *            (canonical edges as lds_get_edges returns them); else LDS_EINVAL
 *   iters    0 <= iters <= 60000
 *   R        device int64[n], output: scaled loads R_x = (iters+1)(iters+2) r_x
 *   W        device int64[m], output: (iters+1)(iters+2) alpha_{u,v} per edge
 *   stream   cudaStream_t for all work (NULL: default stream); the call returns
 *            after the stream has finished it
 * Edges that repeat, or are not sorted by (u, v), are refused with LDS_EINVAL.
 * Scratch: a fixed device array of LDS_NOALLOC_MAX_VERTICES + 64 int32 words,
 * held by every GPU that loads the library until the process exits; the call
 * makes no cudaMalloc / cudaFree or other allocating call.  The first call on
 * each device looks up the array's device address while that device is
 * current; make that first call before any stream capture.  The address is
 * kept per device ordinal for the rest of the process: it assumes the
 * device's primary context stays alive (no cudaDeviceReset, no other context
 * made current on that ordinal between calls).  Every call on a
 * device shares the array (each clears what it uses first), so calls that
 * overlap on the GPU race: do not issue them concurrently. */
lds_status lds_fw_exact_noalloc(int32_t n, int64_t m, const int32_t* u, const int32_t* v, int32_t iters,
                                int64_t* R, int64_t* W, void* stream);

/* Test hook: make the k-th device allocation from now fail with LDS_ENOMEM
 * (k <= 0 disables).  Host-side fault injection; no GPU fault involved. */
void lds_debug_fail_alloc_after(int32_t k);

#ifdef __cplusplus
}
#endif

#endif /* LDS_H */
