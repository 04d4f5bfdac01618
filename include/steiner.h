/*
 * steiner.h — C ABI of the GB300 Voronoi-cell 2-approximation Steiner tree
 * library (arXiv 2205.14503, "Towards Distributed 2-Approximation Steiner
 * Minimal Trees in Billion-edge Graphs").
 *
 * Problem (paper, Section "Introduction" and Table "preliminaries_notation"):
 * an undirected graph G(V, E, d) with positive integer edge distances
 * d : E -> Z+ \ {0} and a seed set S; the library returns a Steiner tree
 * G_S whose total distance D(G_S) = sum of its edge distances is within
 * 2(1 - 1/l) of the minimum (Section "Parallel Steiner Tree Algorithm").
 *
 * The method (Algorithm 2): (1) Voronoi cells of all seeds — every vertex
 * gets its nearest seed, distance and predecessor; (2) per pair of adjacent
 * cells the minimum bridge d1(s,u) + d(u,v) + d1(v,t); (3) an MST of that
 * seed graph; (4-7) the bridges of the MST pairs plus predecessor paths
 * back to the seeds, and their total distance.
 *
 * Tie rules (fixed so every result is exact and reproducible):
 *   - seeds are ranked by ascending vertex id;
 *   - a vertex equidistant from several seeds joins the smallest-id seed;
 *   - pred(v) is the smallest-id neighbour u in v's cell with
 *     d1(u) + d(u,v) = d1(v);
 *   - per cell pair the bridge is the minimum (bridge distance, arc id),
 *     the arc being the CSR arc leaving the endpoint in the smaller-rank cell;
 *   - the seed-graph MST is the unique MST under the order
 *     (bridge distance, rank a, rank b).
 *
 * Graph format: symmetric CSR with uint32 row offsets (n_arcs < 2^32),
 * int32 neighbour ids sorted strictly ascending per row, no self-loops,
 * uint32 weights >= 1, and both arcs of an edge carrying the same weight.
 *
 * Pointers: arrays named "host" must be host memory; arrays documented as
 * "host or device" may be either (the library asks the CUDA runtime).
 * Unless stated otherwise the library copies what it needs and never keeps
 * a caller pointer after the call returns.
 *
 * Threading: calls on one graph handle are serialised by the library; the
 * serving calls (submit/poll) may be made from any thread.
 *
 * Errors: every int-returning call returns STEINER_OK (0), STEINER_PENDING
 * (1, poll only) or one of the negative codes below.
 */
#ifndef STEINER_H
#define STEINER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STEINER_OK             0
#define STEINER_PENDING        1   /* steiner_poll: not finished yet */
#define STEINER_EINVAL        -1   /* malformed CSR, weight 0, bad seed list, bad handle */
#define STEINER_ENOMEM        -2   /* device or host allocation failed, or a size limit */
#define STEINER_EOVERFLOW     -3   /* a seed distance or bridge sum reached 2^32 - 1 */
#define STEINER_EDISCONNECTED -4   /* seeds lie in several components: result is a forest */
#define STEINER_ETIMEOUT      -5   /* a device loop or barrier hit its iteration cap */
#define STEINER_EBUSY         -6   /* serving admission refused (budget or queue full) */
#define STEINER_ECUDA         -7   /* CUDA runtime error (message: steiner_last_error) */

typedef struct steiner_graph *steiner_graph_t;     /* opaque; owns the device copy */

/* One tree edge: u < v, w = d(u, v). */
typedef struct { uint32_t u, v, w; } steiner_edge_t;

/*
 * A query result.  edges (n_edges entries, ascending by (u, v)) is
 * allocated by the library and released with steiner_result_free.
 * total = D(G_S) (Algorithm 2 Step 7).  status repeats the return code of
 * the call that filled it; edges are valid for STEINER_OK and
 * STEINER_EDISCONNECTED (spanning forest), empty otherwise.
 */
typedef struct {
    steiner_edge_t *edges;
    uint32_t n_edges;
    uint64_t total;
    int32_t status;
} steiner_result_t;

/* One edge of the distance graph G'_1 (Algorithm 2 Step 2). */
typedef struct {
    uint32_t ra, rb;      /* seed ranks, ra < rb */
    uint64_t b;           /* d'_1 = d1(s,u) + d(u,v) + d1(v,t) */
    uint32_t arc;         /* CSR arc u -> v, u in the cell of rank ra */
    uint32_t in_mst;      /* 1 if the pair is an edge of the MST G'_2 */
} steiner_pair_t;

/* Per-query counters (tracing; the paper's per-phase breakdown, Fig. 3). */
typedef struct {
    uint64_t relax_attempts;     /* arcs scanned by the Voronoi phase */
    uint64_t relax_improved;     /* label improvements */
    uint32_t iterations;         /* frontier iterations */
    uint32_t phases;             /* threshold advances (near/far splits) */
    uint64_t n_pairs;            /* |E'_1| */
    uint32_t n_tree_edges;       /* |E_S| */
    uint32_t gpu_launches;       /* kernels this query launched */
    /* device time per phase (CUDA events on the library's stream, ms):
     * init = labels and seeds, voronoi = the near/far SSSP kernel alone,
     * bridges = pred + bridge scan and pair compaction, mst = Boruvka,
     * tree = expansion, sort and total */
    float ms_init, ms_voronoi, ms_bridges, ms_mst, ms_tree;
} steiner_stats_t;

/*
 * steiner_load_graph — copy a CSR graph to device `device` and validate it
 * on the device (symmetry, sorted rows, no self-loops, weights >= 1).
 *   row_ptr  host, n + 1 entries, row_ptr[0] = 0, row_ptr[n] = n_arcs
 *   col      host, n_arcs neighbour ids
 *   w        host, n_arcs weights
 * On success *out receives a handle; the caller keeps ownership of the
 * arrays.  On a skewed degree distribution the device copy numbers the
 * vertices by descending degree (ties by id) for cache locality; every
 * result (tree edges, pair arcs, cell/dist/pred) is still in the caller's
 * vertex ids and arc indices, and the tie rules use the caller's order.
 * The environment variable STEINER_RELABEL=0 or 1, read here, forces this
 * internal order off or on; STEINER_DELTA=<n> sets the initial band width
 * (default 32 x mean weight / mean degree; "delta" below changes it later).
 * With STEINER_TRACE set, each single query prints its Voronoi loop's exit
 * reason and its first iterations' frontier sizes to stderr.
 * Errors: STEINER_EINVAL (malformed graph or n_arcs >= 2^32),
 * STEINER_ENOMEM, STEINER_ECUDA.  Cites: Table "preliminaries_notation"
 * (positive integer distances); Section "Evaluation" (symmetric arcs).
 */
int steiner_load_graph(const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                       uint32_t n, uint64_t n_arcs, int device, steiner_graph_t *out);

/* Release the graph, its device memory and any serving state. */
void steiner_free_graph(steiner_graph_t g);

/*
 * steiner_query — Algorithm 2 end to end for one seed set.
 *   seeds  host, k distinct vertex ids in any order (k >= 1)
 *   out    receives the tree (see steiner_result_t)
 * k = 1 gives an empty tree with total 0.  Returns the status (also stored
 * in out->status).  Errors: STEINER_EINVAL (k = 0, id out of range,
 * duplicate), STEINER_EOVERFLOW, STEINER_EDISCONNECTED (forest returned),
 * STEINER_ETIMEOUT, STEINER_ENOMEM (k too large for the pair table:
 * k (k - 1) / 2 > 2^28), STEINER_ECUDA.
 */
int steiner_query(steiner_graph_t g, const int32_t *seeds, uint32_t k, steiner_result_t *out);

/*
 * steiner_query_detail — as steiner_query, and also returns the distance
 * graph G'_1 with its MST flags (Algorithm 2 Steps 2-3) and counters.
 *   pairs    receives a library-allocated array of *n_pairs entries in
 *            ascending (ra, rb) order (free with steiner_pairs_free); may be
 *            NULL to skip
 *   stats    optional counters (may be NULL)
 */
int steiner_query_detail(steiner_graph_t g, const int32_t *seeds, uint32_t k,
                         steiner_result_t *out, steiner_pair_t **pairs, uint64_t *n_pairs,
                         steiner_stats_t *stats);

/*
 * steiner_voronoi — Algorithm 2 Step 1 only (Voronoi cells, Algorithm 4's
 * fixed point), exported per vertex.  Outputs (host or device, n entries
 * each, any may be NULL):
 *   cell  seed vertex id of the vertex's cell, -1 if no seed reaches it
 *   dist  d1(src(v), v), 0xFFFFFFFF if unreached
 *   pred  predecessor on a shortest path from src(v); pred(s) = s; -1 if
 *         unreached
 * Errors as steiner_query (STEINER_EOVERFLOW when a reachable distance
 * does not fit below 2^32 - 1).
 */
int steiner_voronoi(steiner_graph_t g, const int32_t *seeds, uint32_t k,
                    int32_t *cell, uint32_t *dist, int32_t *pred);

/*
 * steiner_query_batch — q independent queries over the resident graph in
 * one batched run (per-query label arrays, shared CSR reads).
 *   seeds  host, q pointers to host seed lists
 *   ks     host, q sizes
 *   outs   host, q results (each as steiner_query)
 * Returns STEINER_OK if every query finished with STEINER_OK, else the
 * first non-OK status; each outs[i].status holds the query's own status.
 */
int steiner_query_batch(steiner_graph_t g, const int32_t *const *seeds, const uint32_t *ks,
                        uint32_t q, steiner_result_t *outs);

/*
 * Serving (continuous batching).  steiner_serve_start allocates up to
 * `slots` concurrent query slots within `budget_bytes` of per-query device
 * state and starts the device loop; steiner_submit enqueues a query
 * (seeds copied; non-blocking) and returns a ticket; steiner_poll returns
 * STEINER_PENDING until the result is ready, then fills *out once and
 * returns the query's status.  Polling a ticket that was never issued, or
 * whose result was already returned, gives STEINER_EINVAL and leaves *out
 * untouched.  steiner_submit returns STEINER_EBUSY if the queue is full.
 * steiner_submit and steiner_poll may be called from any thread while the
 * loop runs.  steiner_serve_stop joins the loop's worker thread and frees
 * the serving state (results not yet polled are dropped): it must not run
 * concurrently with steiner_submit or steiner_poll on the same handle.
 */
int steiner_serve_start(steiner_graph_t g, uint32_t slots, uint64_t budget_bytes);
int steiner_submit(steiner_graph_t g, const int32_t *seeds, uint32_t k, uint64_t *ticket);
int steiner_poll(steiner_graph_t g, uint64_t ticket, steiner_result_t *out);
int steiner_serve_stop(steiner_graph_t g);

/*
 * Tuning parameters of a graph handle (used by the autotuner):
 *   "delta"        near/far band width of the Voronoi phase (>= 1)
 *   "sssp_blocks"  blocks of the persistent Voronoi kernel (0 = every
 *                  co-resident block; at most "sssp_max_blocks")
 *   "local_rounds" local relaxation rounds per frontier iteration
 *                  (0 = off): each warp keeps relaxing the vertices it
 *                  just queued, a hop per round, before the grid barrier
 *   "batch_delta"  band width of the multi-query engine (0 = w_max / 8 when
 *                  "delta" is at most the largest weight w_max, else "delta")
 *   "batch_pull"   1 (default): a query's first heavy-arc pass in the
 *                  multi-query engine runs in the pull form (each vertex
 *                  unsettled in that query reads its own heavy arcs and the
 *                  labels at their other ends); 0: it pushes the heavy arcs
 *                  of the band's vertices
 *   "batch_tails"  1 (default): the tails (MST, expansion, sorted edges) of
 *                  the queries that finish together run as one launch per
 *                  step for all of them; 0: one query at a time
 *   "batch_yield_div"  a serving launch returns to the host (to retire and
 *                  admit) once 1/batch_yield_div of its in-flight queries
 *                  converged (1..64, default 1: whole waves), or earlier
 *                  when a request waits and a slot is free
 *   "max_iters"    frontier iteration cap (STEINER_ETIMEOUT beyond it)
 *   "dense"        1 (default): where splits scan the labels and no local
 *                  rounds run, a large frontier is kept as a bitmap (one bit
 *                  per vertex) that the next iteration reads in vertex
 *                  order, and so is the list of a band's vertices; 0: queues
 *   "far_scan"     how a band split finds the vertices left for later
 *                  bands: -1 (default) chooses, 0 keeps a pile of them
 *                  (one stamp exchange and queue slot per improvement),
 *                  1 scans every label at the split instead
 *   "pull"         form of a band's heavy-arc pass (with the far scan):
 *                  1 (default) chooses per band the form that reads fewer
 *                  arcs, 0 pushes the heavy arcs of the band's vertices,
 *                  2 pulls: every vertex still at or above the threshold
 *                  reads its own heavy arcs and takes the best proposal
 *                  from the settled vertices at their other ends
 *   "tail"         1 (default): after a heavy-arc pass in the pull form the
 *                  rest of the Voronoi phase runs as one unbounded band (a
 *                  frontier Bellman-Ford over whole rows); 0 keeps the bands
 *   "label_bits"   width of the Voronoi labels: 0 (default) chooses per
 *                  query, 32 or 64 force it.  A 32-bit label holds
 *                  (distance << b) | rank with b the bits of the largest
 *                  seed rank; a query whose distances do not fit runs again
 *                  with 64-bit labels, so results never depend on the width
 * steiner_get_param also reads "sssp_max_blocks", "sm_count",
 * "heavy_chunks", "label_bits_last" (the width the last query ended with),
 * "narrow_reruns" (queries rerun with 64-bit labels), "pull_passes_last"
 * (heavy-arc passes of the last query run in the pull form),
 * "tail_iteration_last" (the iteration its unbounded tail began at, 0 for
 * none) and the multi-query
 * engine's tracing counters
 * ("batch_ms_sssp", "batch_ms_scan", "batch_ms_tail", "batch_ms_admit" in
 * microseconds, "batch_launches", "batch_iterations", "batch_items",
 * "batch_pairs", "batch_t0".."batch_t4" in nanoseconds, "batch_admitted"
 * (queries admitted into slots), "batch_admitted_busy" (of those, the
 * ones admitted while other slots were still on the device) and
 * "batch_tail_batches" (retirements whose tails ran batched),
 * "batch_pull_sweeps" (pull-form passes the engine ran) and
 * "batch_narrow_reruns" (queries answered by the single-query path because
 * a distance outgrew the engine's 32-bit labels); "batch_reset" clears the
 * timers).  It returns -1 for an unknown key.
 */
int steiner_set_param(steiner_graph_t g, const char *key, int64_t value);
int64_t steiner_get_param(steiner_graph_t g, const char *key);

/*
 * steiner_voronoi_noalloc — the Voronoi cells of steiner_voronoi for callers
 * that cannot allocate device memory (a framework that owns every device
 * allocation through its own pool, or code that must not grow its device
 * footprint after start-up).  This call allocates nothing: no cudaMalloc,
 * no cudaFree, no allocating library routine.  Its working memory is one
 * fixed array of device memory inside the library (24 MiB + 256 bytes),
 * present on every GPU that loads the library until the process exits.
 * The paper has no counterpart to this entry point.
 *   row_ptr, col, w  device, the CSR of the graph in the steiner_load_graph
 *                    format (row offsets and neighbour ids are range-checked;
 *                    sortedness and symmetry are not re-validated)
 *   n, n_arcs        sizes; n <= STEINER_NOALLOC_MAX_VERTICES
 *   seeds            device, k distinct seed ids in ASCENDING order
 *   cell, dist, pred device outputs, n entries each (may be NULL), same
 *                    meaning as in steiner_voronoi
 *   stream           a cudaStream_t (NULL = the legacy default stream); the
 *                    call returns after the stream has finished the work
 * The first call on a device looks up the array's device address and the
 * launch size (cudaGetSymbolAddress with that device current); make that
 * first call before any stream capture.  Every call reuses the same array,
 * so calls that overlap on the GPU (other streams or host threads) race:
 * serialise them.  Errors: STEINER_ENOMEM if n exceeds the limit (nothing
 * is launched), STEINER_EINVAL (bad sizes, unsorted or out-of-range seeds,
 * row offsets that do not run from 0 to n_arcs without decreasing,
 * out-of-range neighbour ids; the outputs are then left untouched),
 * STEINER_EOVERFLOW, STEINER_ETIMEOUT, STEINER_ECUDA (after these three the
 * outputs' contents are undefined).
 */
#define STEINER_NOALLOC_MAX_VERTICES 1048576u
int steiner_voronoi_noalloc(const uint32_t *row_ptr, const int32_t *col, const uint32_t *w,
                            uint32_t n, uint64_t n_arcs, const int32_t *seeds, uint32_t k,
                            int32_t *cell, uint32_t *dist, int32_t *pred, void *stream);

/* Release library-allocated outputs. */
void steiner_result_free(steiner_result_t *r);
void steiner_pairs_free(steiner_pair_t *pairs);

/* Text of the last error on this thread (static storage). */
const char *steiner_last_error(void);

/* Library version string. */
const char *steiner_version(void);

#ifdef __cplusplus
}
#endif

#endif /* STEINER_H */
