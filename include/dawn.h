/*
 * dawn.h -- C ABI of the B300 (sm_103a) implementation of DAWN's hot path.
 *
 * DAWN (Feng et al., ICS '24) computes exact unweighted shortest-path lengths
 * as a level-synchronous Boolean vector-matrix product over (OR, AND): the
 * frontier vector alpha is multiplied by the adjacency matrix, the product is
 * masked by the set of vertices already reached, and every newly reached
 * vertex gets dist = step (Sec. 3.2 Eq. 2-4 and Alg. 1 "BOVM"; Sec. 3.3
 * Eq. 5-7 and Alg. 3 "SOVM").  A single source runs until a step reaches no
 * new vertex (Sec. 3.1, stop condition 2); all-pairs runs it from every
 * source (Sec. 3.3, the APSP cost T < 2 S_wcc E_wcc).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status: DAWN_OK (0) or a DAWN_E_* code below.
 *    No exception and no CUDA error crosses the ABI.  dawn_last_error()
 *    gives a human-readable message for the calling thread's last failure.
 *  - Graphs are CSR, int32: row_ptr[n+1] (row_ptr[0] = 0, non-decreasing,
 *    row_ptr[n] = m) and col_idx[m] with 0 <= col_idx[j] < n.  Arc i -> c
 *    exists when c is listed in row i (the paper's A[i][c] = 1).  Duplicate
 *    arcs and self-loops are tolerated and do not change any result.
 *    m < 2^31.
 *  - Distances: dist[v] = number of arcs on a shortest src -> v path
 *    (Thm 1), dist[src] = 0, dist[v] = -1 when no path exists.  The paper
 *    writes 0 for "unset"; this ABI reserves 0 for the source and uses -1.
 *    The result is unique, so every call is bit-exact and deterministic.
 *  - Pointers marked "host or device" may point to pageable host memory,
 *    pinned host memory or device memory of the current device; the
 *    library inspects them with cudaPointerGetAttributes.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that produce results synchronize `stream` before they return, so caller
 *    buffers are only borrowed for the duration of the call.
 *  - A graph handle owns one set of device work buffers: calls on the same
 *    handle must not run concurrently (from several host threads); calls on
 *    different handles may.
 *  - Every device-side wait (the grid barrier between levels, the serving
 *    loop's polls) is bounded; on expiry the call returns DAWN_E_TIMEOUT and
 *    the device stays usable.
 */
#ifndef DAWN_H
#define DAWN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define DAWN_API __attribute__((visibility("default")))
#else
#define DAWN_API
#endif

/* ------------------------------------------------------------ status codes */
#define DAWN_OK          0
#define DAWN_E_INVALID   1 /* malformed CSR, source out of range, bad k / flags / sizes */
#define DAWN_E_NOMEM     2 /* device allocation failed, or a request can never fit the budget */
#define DAWN_E_OVERFLOW  3 /* an int16 distance block would need a level above 32767 */
#define DAWN_E_TIMEOUT   4 /* a bounded device wait expired */
#define DAWN_E_CUDA      5 /* a CUDA runtime call failed (see dawn_last_error) */
#define DAWN_E_STATE     6 /* unknown request id, or a call made in the wrong state */

/* ------------------------------------------------------------- graph flags */
#define DAWN_DIRECTED    0u /* general digraph: the in-adjacency (CSC) is built on the device */
#define DAWN_SYMMETRIC   1u /* every arc has its reverse (the arc multiset equals its reverse): the CSR is
                               its own CSC; checked at upload, DAWN_E_INVALID naming a witness otherwise */

/* --------------------------------------------------------- traversal modes */
#define DAWN_MODE_AUTO   0 /* per level: SOVM push or BOVM pull, chosen from frontier counters */
#define DAWN_MODE_PUSH   1 /* SOVM only (Alg. 3): expand the frontier's CSR rows */
#define DAWN_MODE_PULL   2 /* BOVM only (Alg. 1): unreached vertices test their in-neighbours */

/* ------------------------------------------------------ dist block layouts */
#define DAWN_SOURCE_MAJOR 0 /* dist_block[s * n + v] */
#define DAWN_VERTEX_MAJOR 1 /* dist_block[v * k + s] */

/* ----------------------------------------------------------- request state */
#define DAWN_REQ_PENDING 0 /* admitted to the queue, not yet on the device */
#define DAWN_REQ_RUNNING 1 /* some of its sources occupy bit lanes on the device */
#define DAWN_REQ_DONE    2 /* every distance row is in the caller's buffer */
#define DAWN_REQ_FAILED  3 /* the request ended with an error (see dawn_serve_poll's return) */

/* Where one source's level loop runs (dawn_sssp_opts.engine). */
#define DAWN_ENGINE_AUTO    0 /* CLUSTER for low-degree graphs (m < 8n) whose visited bitmap fits the
                                 cluster's shared memory, in AUTO or PUSH mode without a trace; else GRID */
#define DAWN_ENGINE_GRID    1 /* one persistent cooperative grid over every SM, grid barrier per level */
#define DAWN_ENGINE_CLUSTER 2 /* one thread-block cluster (16 CTAs, or 8): visited bitmap in distributed
                                 shared memory, frontier lists in shared memory, cluster barrier per
                                 level; SOVM push only (Alg. 3); DAWN_E_INVALID when the bitmap does not
                                 fit (n above about 24 M) or with DAWN_MODE_PULL or a trace */

/* Per-graph server step (dawn_serve_create_ex). */
#define DAWN_SERVE_AUTO     0 /* FRONTIER when the average out-degree m / n is below 8, else DENSE */
#define DAWN_SERVE_DENSE    1 /* every iteration pulls every vertex (bit-lane Alg. 1 over the CSC) */
#define DAWN_SERVE_FRONTIER 2 /* every iteration pushes only the last iteration's arrivals (bit-lane Alg. 3 over the CSR) */

typedef struct dawn_graph* dawn_graph_t;
typedef struct dawn_server* dawn_server_t;

/*
 * Copy a CSR graph to the current device and prepare it for traversal.
 * Defines the adjacency A of Sec. 3.1 (Table 1: "CSR" / "CSC").
 *   row_ptr  host or device, int32[n+1]; col_idx host or device, int32[m].
 *   n >= 1, 0 <= m < 2^31, flags = DAWN_DIRECTED or DAWN_SYMMETRIC.
 * The library validates the CSR on the device (DAWN_E_INVALID with the first
 * offending index in dawn_last_error).  With DAWN_SYMMETRIC it checks, in one
 * O(n + m) device pass over two 64-bit hash sums, that the arc multiset equals
 * its reverse (every arc (u, v) appears as often as (v, u); self-loops are
 * their own reverse), and returns DAWN_E_INVALID naming an arc without a
 * matching reverse (or, on rows of more than 4,096 arcs, the vertex) when it
 * does not: such a graph must be uploaded as DAWN_DIRECTED.  It builds the
 * in-adjacency for directed
 * graphs, a copy of the in-adjacency with each row ordered by the neighbours'
 * out-degree (largest first) and the first two entries of each such row, and
 * allocates the per-graph work buffers: about 4m + 45n bytes beyond the CSR
 * for a symmetric graph, 8m + 49n for a directed one.  For a symmetric graph
 * it also finds the connected components, so that a search stops as soon as
 * the source's component is reached.  Host memory: 8n bytes (copies of
 * row_ptr and of the component sizes).  The caller keeps ownership of its
 * arrays; *out owns the device copy until dawn_graph_free.  Synchronizes
 * `stream`.
 */
DAWN_API int dawn_graph_upload(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t m,
                               uint32_t flags, void* stream, dawn_graph_t* out);

/* Release every device buffer of g.  g may be NULL.  Not to be called while a
 * call on g is in flight or while a server created over g exists. */
DAWN_API int dawn_graph_free(dawn_graph_t g);

/* n, m and flags of an uploaded graph (any pointer may be NULL). */
DAWN_API int dawn_graph_info(dawn_graph_t g, int32_t* n, int64_t* m, uint32_t* flags);

/*
 * Single-source shortest paths (Alg. 3 SOVM and Alg. 1 BOVM, Sec. 3.2-3.3).
 *   src   0 <= src < n, else DAWN_E_INVALID.
 *   dist  host or device, int32[n], written in full.
 * Runs the level loop from src until a step reaches no vertex (on a
 * symmetric graph: until every vertex of src's connected component has its
 * distance, which skips that empty step), in one persistent cooperative
 * kernel on `stream`, then synchronizes `stream`.
 * DAWN_MODE_AUTO is used; see dawn_sssp_ex for the other modes.
 */
DAWN_API int dawn_sssp(dawn_graph_t g, int32_t src, int32_t* dist, void* stream);

typedef struct {
    int32_t mode;          /* DAWN_MODE_*; 0 = AUTO */
    int32_t alpha;         /* push -> pull when m_f * alpha > m_u; 0 = tuned or 15 */
    int32_t beta;          /* pull -> push when n_f * beta < n and n_f shrank; 0 = tuned or 18 */
    int32_t blocks_per_sm; /* CTAs per SM of the persistent grid; 0 = occupancy-derived */
    int64_t spin_limit;    /* grid-barrier spin budget in SM clock cycles; 0 = default (~2 s) */
    int64_t* trace;        /* device memory or NULL: one record of 4 int64 per grid barrier,
                              {kind, step, count, globaltimer ns}; kind 0 = kernel entry,
                              1 = init done, 2 = push level, 3 = pull level over the bitmap,
                              4 = bitmap-to-queue conversion, 5 = pull level over the lists of
                              candidates a previous pull left unreached; count = vertices the
                              level reached (entries queued for kind 4); records past trace_cap
                              are dropped */
    int32_t trace_cap;     /* records that fit in trace */
    int32_t pull_serial;   /* in-neighbours a lane tests on its own in a pull level before
                              the warp takes the rest of the row; 0 = tuned or 8 */
    int32_t engine;        /* DAWN_ENGINE_*; 0 = AUTO */
    int32_t reserved;      /* 0 */
} dawn_sssp_opts;

typedef struct {
    int32_t levels;        /* eccentricity of src: the last step that reached a vertex */
    int32_t push_steps;    /* levels run as SOVM push */
    int32_t pull_steps;    /* levels run as BOVM pull */
    int32_t reserved;
    int64_t reached;       /* vertices with dist >= 0 (src included) */
    int64_t edges;         /* E_r: sum of out-degrees of the reached vertices, the
                              SOVM cost T = E_wcc(i) of Sec. 3.3 */
} dawn_sssp_stats;

/* dawn_sssp with options (opts may be NULL) and per-call statistics (stats may be NULL). */
DAWN_API int dawn_sssp_ex(dawn_graph_t g, int32_t src, int32_t* dist, const dawn_sssp_opts* opts,
                          dawn_sssp_stats* stats, void* stream);

/*
 * Stream-ordered dawn_sssp_ex: enqueue the level loop and return without
 * synchronizing, so that many sources (and the caller's own work and events)
 * can be queued back to back.
 *   dist_dev   device memory, int32[n] (DAWN_E_INVALID otherwise).
 *   stats_dev  device memory or NULL; receives this call's dawn_sssp_stats.
 * A device-side failure (DAWN_E_TIMEOUT) is sticky: later calls on g do no
 * work until dawn_graph_sync reports and clears it.
 */
DAWN_API int dawn_sssp_async(dawn_graph_t g, int32_t src, int32_t* dist_dev, const dawn_sssp_opts* opts,
                             dawn_sssp_stats* stats_dev, void* stream);

/*
 * Shortest-path tree (Fact 1 / Thm 1: a vertex first reached at level d has
 * an in-neighbour at level d - 1 on a shortest path).  Runs the level loop of
 * dawn_sssp (DAWN_MODE_AUTO), then one pass over the in-adjacency:
 *   parent[v] = min { u : (u, v) is an arc and dist[u] = dist[v] - 1 }
 * for dist[v] > 0, and -1 for the source and for unreached vertices.  Several
 * predecessors can qualify; the smallest id is the tie-break that makes the
 * tree unique.  Following parent from any reached v visits dist[v] arcs and
 * ends at src.
 *   dist, parent  host or device int32[n], caller-owned (written; synchronous).
 * Cost: the level loop plus a read of every in-arc of every reached vertex.
 */
DAWN_API int dawn_sssp_tree(dawn_graph_t g, int32_t src, int32_t* dist, int32_t* parent, void* stream);

/* Stream-ordered dawn_sssp_tree (no synchronization): dist_dev and parent_dev
 * are device int32[n]; errors of the device wait are reported by
 * dawn_graph_sync. */
DAWN_API int dawn_sssp_tree_async(dawn_graph_t g, int32_t src, int32_t* dist_dev, int32_t* parent_dev,
                                  void* stream);

/*
 * k single-source searches in one call (APSP by repetition, Sec. 3.3): row i
 * of dist (k x n int32, source-major) receives the distances from
 * sources[i], exactly as dawn_sssp_ex would (same options).  With host
 * dist the rows are staged in two device buffers and each row's copy to the
 * host overlaps the next source's level loop on a second stream; pinned host
 * memory is needed for that overlap.  Device dist is written in place.
 *   sources  host or device int32[k], each in [0, n) (DAWN_E_INVALID otherwise).
 *   stats    host or device dawn_sssp_stats[k], or NULL.
 * Synchronous: returns when every row is in dist (or on the first error).
 */
DAWN_API int dawn_sssp_many(dawn_graph_t g, const int32_t* sources, int32_t k, int32_t* dist,
                            dawn_sssp_stats* stats, const dawn_sssp_opts* opts, void* stream);

/*
 * Diagnostic (no counterpart in the paper): this GPU's L2 read bandwidth in
 * GB/s, the denominator for kernels whose working set stays in L2.  A device
 * buffer of `bytes` (>= 1 MiB; pick one that fits in L2) is read `passes`
 * times with 16-byte loads by every SM after one untimed pass; *gbs receives
 * bytes * passes / time.  Synchronizes `stream`.
 */
DAWN_API int dawn_l2_read_gbs(int64_t bytes, int32_t passes, double* gbs, void* stream);

/*
 * Weighted extension.  Sec. 5 names (min, +) operations on weighted graphs as
 * the way DAWN is to be extended; these calls run the SOVM rounds of Alg. 3
 * with (min, +) in place of (OR, AND).
 *
 * Attach arc weights to g: weights[j] belongs to arc j of the col_idx array
 * given to dawn_graph_upload (same order).
 *   weights  host or device, int32[m], every entry >= 0; DAWN_E_INVALID with
 *            the first negative index in dawn_last_error otherwise (g then
 *            has no weights until a valid set is given).
 * Replaces earlier weights.  The first call allocates the weighted path's
 * buffers (about 12m + 33n bytes: the weights, a copy of the arcs with their
 * weights interleaved, {head, weight} per arc, which the rounds read with one
 * 8-byte load, and the round queues); dawn_graph_free releases them.
 * Synchronizes `stream`.
 */
DAWN_API int dawn_graph_set_weights(dawn_graph_t g, const int32_t* weights, void* stream);

typedef struct {
    int32_t rounds;        /* rounds that lowered some distance (at most n - 1) */
    int32_t reserved;
    int64_t reached;       /* vertices with dist >= 0 (src included) */
    int64_t relaxations;   /* arcs offered a distance: the out-degrees of every frontier, summed */
    int64_t improvements;  /* offers that lowered a distance */
} dawn_wsssp_stats;

/*
 * Weighted single-source shortest paths: dist[v] = the least total weight of
 * a directed path src -> v, -1 when there is none, 0 at src.  Round r offers
 * d(u) + w(u, v) from every vertex u whose distance fell in round r - 1 to
 * each out-neighbour v (an atomic minimum); the vertices whose distance fell
 * form the next frontier; the loop stops on a round that lowers nothing.
 * The result is unique; the rounds and counts can vary from run to run
 * (values lowered during a round are offered at once).
 *   src    0 <= src < n.
 *   dist   host or device, int64[n], written in full.
 *   stats  host or device, or NULL.
 * DAWN_E_INVALID when g has no weights.  Synchronous.
 */
DAWN_API int dawn_wsssp(dawn_graph_t g, int32_t src, int64_t* dist, dawn_wsssp_stats* stats, void* stream);

/* Stream-ordered dawn_wsssp: dist_dev device int64[n], stats_dev device or
 * NULL; a device-side failure is reported by dawn_graph_sync. */
DAWN_API int dawn_wsssp_async(dawn_graph_t g, int32_t src, int64_t* dist_dev, dawn_wsssp_stats* stats_dev,
                              void* stream);

/* Synchronize `stream` and return (then clear) the sticky device status of g:
 * DAWN_OK, DAWN_E_TIMEOUT or DAWN_E_OVERFLOW. */
DAWN_API int dawn_graph_sync(dawn_graph_t g, void* stream);

/*
 * Allocation-free single source (the paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc, e.g. a process whose
 * framework allocator has already reserved the device memory it is allowed
 * to use, or a latency-critical request path whose policy forbids device
 * allocation after start-up).  It runs the same persistent level loop as
 * dawn_sssp in SOVM push mode (Alg. 3) on a CSR the caller keeps on the
 * device; no graph handle is needed.
 *   row_ptr, col_idx  device memory, int32[n+1] / int32[m]; checked on the
 *                     device before the traversal (DAWN_E_INVALID if bad).
 *   n, m              1 <= n <= 1,048,576 and 0 <= m <= 33,554,432, else
 *                     DAWN_E_INVALID.
 *   src               0 <= src < n.
 *   dist              device memory, int32[n], written in full.
 * The work buffers (control block, visited bitmap, two frontier queues)
 * live in one file-scope device array of about 27 MB that every GPU which
 * loads this library holds until the process exits.  The call allocates
 * nothing: no cudaMalloc, cudaFree, pinned host buffer or library routine
 * that allocates.  The first call on a device looks up the array's device
 * address and the kernel's occupancy (once per device); make that first call
 * before any stream capture.  Every call uses the same array and leaves its
 * contents behind (the call clears what must start at zero), so calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must
 * be serialized by the caller.  Synchronizes `stream`.
 */
DAWN_API int dawn_sssp_noalloc(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t m,
                               int32_t src, int32_t* dist, void* stream);

/*
 * Autotuner (the paper fixes one block size and has no tuner; Sec. 4.1).
 * Times short trials of dawn_sssp on `sample` (up to 16 sources) for a grid
 * of push/pull switch thresholds (alpha, beta) and per-lane pull lengths,
 * and of dawn_msbfs for 64 / 128 / 256 lanes (the sample repeated to 1024
 * sources), then stores the fastest settings in g: later calls whose options
 * leave these fields at 0 use them.  Results are bit-identical whatever the
 * settings; only time changes.  sample: host or device int32[k], k >= 1.
 * out (nullable) receives the choice and the times measured with it.
 * Synchronizes `stream`.
 */
typedef struct {
    int32_t alpha;
    int32_t beta;
    int32_t pull_serial;
    int32_t lanes;
    double sssp_us;            /* mean device time per source with the chosen settings */
    double msbfs_sources_per_s;
} dawn_tuning;

DAWN_API int dawn_autotune(dawn_graph_t g, const int32_t* sample, int32_t k, dawn_tuning* out, void* stream);

/* Store settings in g as dawn_autotune does (e.g. read back from a cache);
 * fields at 0 keep the built-in defaults. */
DAWN_API int dawn_set_tuning(dawn_graph_t g, const dawn_tuning* t);

/*
 * Multi-source (APSP-style) batch: SSSP from each of k sources (Sec. 3.3,
 * APSP as repeated SSSP), advanced together as bit lanes: 64 * W sources per
 * pass share each vertex's W uint64 visited words, and one level does
 * new[v] = (OR over in-neighbours u of visited[u]) AND NOT visited[v].
 *   sources     host or device, int32[k], each in [0, n); repeats allowed.
 *   k           >= 1.
 *   dist_block  host or device or NULL; int16 (dist_bytes = 2) or int32
 *               (dist_bytes = 4); k x n in `layout` order.  NULL keeps each
 *               pass's block in a device scratch buffer only (the reductions
 *               are still produced).
 *   ecc, dsum, reached  host or device or NULL, int32[k] / int64[k] / int32[k]:
 *               largest finite distance (epsilon(i) of Table 1; 0 for an
 *               isolated source), sum of finite distances, count of reached
 *               vertices (src included).
 * DAWN_E_OVERFLOW when dist_bytes = 2 and some level exceeds 32767 (the
 * block is then incomplete; nothing wraps).  Synchronizes `stream`.
 */
DAWN_API int dawn_msbfs(dawn_graph_t g, const int32_t* sources, int32_t k, void* dist_block,
                        int dist_bytes, int layout, int32_t* ecc, int64_t* dsum, void* stream);

/* Kernels of the batched level loop (dawn_msbfs_opts.kernel, also read by
 * dawn_centrality).  Both give identical results.
 *   DAWN_MSBFS_SLICED     in-arc rows cut into warp tasks by in-degree (one
 *                         vertex per lane for short rows, row pieces for long
 *                         ones); level 1 pushed from the sources; each level
 *                         only ORs visited words and keeps its new bits, so
 *                         each distance row is written once, whole, after the
 *                         pass's last level.  Up to 32767 levels; harmonic
 *                         centrality up to 15 (DAWN_E_INVALID past that when
 *                         asked for by name).
 *   DAWN_MSBFS_PER_LEVEL  distances written level by level as bits appear;
 *                         any number of levels.
 * 0 picks SLICED, and PER_LEVEL for a graph on which a run has needed more
 * levels than SLICED holds (for harmonic centrality: more than 15). */
#define DAWN_MSBFS_SLICED 1
#define DAWN_MSBFS_PER_LEVEL 2

typedef struct {
    int32_t lanes;         /* sources per pass: 64, 128 or 256; 0 = tuned, else by k */
    int32_t trace_cap;     /* records that fit in trace */
    int64_t spin_limit;    /* as in dawn_sssp_opts */
    int64_t* trace;        /* device memory or NULL: one record of 4 int64 per level,
                              {pass, level, lanes that reached a vertex in the level,
                              globaltimer ns} */
    int32_t kernel;        /* 0, DAWN_MSBFS_SLICED or DAWN_MSBFS_PER_LEVEL */
    int32_t reserved;      /* 0 */
} dawn_msbfs_opts;

/* dawn_msbfs with the reached counts and options (reached, opts may be NULL). */
DAWN_API int dawn_msbfs_ex(dawn_graph_t g, const int32_t* sources, int32_t k, void* dist_block,
                           int dist_bytes, int layout, int32_t* ecc, int64_t* dsum, int32_t* reached,
                           const dawn_msbfs_opts* opts, void* stream);

/* Whole-run figures of dawn_centrality over the listed sources. */
typedef struct {
    int32_t diameter;    /* largest finite distance from a listed source (max ecc); the graph's
                            diameter when every vertex is listed */
    int32_t radius;      /* smallest ecc among listed sources that reach another vertex; -1 if none */
    int64_t pairs;       /* ordered pairs (s, v), v != s, v reached from a listed s */
    int64_t dist_total;  /* sum of their distances */
} dawn_apsp_summary;

/*
 * Centrality from the batched level loop (Sec. 3.3's APSP, one bit lane per
 * source, no distance rows written).  Per listed source s, all optional
 * (NULL = not wanted; host or device memory, k entries each):
 *   ecc[s]       largest finite distance (0 for an isolated source)
 *   dsum[s]      sum of finite distances
 *   reached[s]   vertices reached, s included
 *   closeness[s] (reached - 1) / dsum, 0 when nothing else is reached
 *   harmonic[s]  sum over reached v != s of 1 / d(s, v), computed as the sum
 *                over distances d = 1, 2, ... of (vertices at distance d) / d
 *                in ascending d, in IEEE double: the same value on any grid
 *   summary      host struct (may be NULL): diameter, radius, pairs, total.
 * The integer figures are exact.  opts: as dawn_msbfs_ex (lanes, spin_limit).
 */
DAWN_API int dawn_centrality(dawn_graph_t g, const int32_t* sources, int32_t k, int32_t* ecc, int64_t* dsum,
                             int32_t* reached, double* closeness, double* harmonic, dawn_apsp_summary* summary,
                             const dawn_msbfs_opts* opts, void* stream);

/*
 * Continuous-batching server over several resident graphs (APSP-style
 * batching of Sec. 3.3 applied to a request stream; the paper has no
 * serving layer).  Requests name a graph and k sources; each source becomes
 * one bit lane of that graph, admitted as lanes free up, so requests that
 * arrive while others run share the device.  One persistent kernel advances
 * every occupied lane one level per iteration (bit-lane Alg. 1 pull); a
 * lane's distance is (iteration - its start iteration), so a request's
 * result is identical alone and in any mix.  A host thread owned by the
 * server admits requests and collects completions; while work is queued the
 * server's kernel occupies every SM (other kernels wait), and it exits
 * after about 2 ms without work.  A request of at most 4 sources on a graph
 * served in AUTO mode that arrives while the server is idle (nothing queued
 * or on the device) runs instead as single-source searches, each on the
 * engine dawn_sssp would pick (on a low-degree graph, thread-block clusters
 * side by side), on a stream of the server's, with the same rows as in the
 * loop; the server then uses that graph's single-source work buffers too, so
 * no other call may use the handle while the server is live.
 *   graphs          ngraphs handles (borrowed; must outlive the server).
 *   mem_budget_bytes  device bytes for the distance blocks of admitted
 *                   requests whose dist_out is host memory (k * n * dist_bytes
 *                   each, held from admission until the block is copied out);
 *                   a request waits in the queue until its block fits; 0 =
 *                   1 GiB.  Requests with device dist_out write in place.
 *   max_lanes       lanes per graph batch: 64, 128 or 256.
 */
DAWN_API int dawn_serve_create(const dawn_graph_t* graphs, int ngraphs, size_t mem_budget_bytes,
                               int max_lanes, dawn_server_t* out);

/*
 * dawn_serve_create with the step chosen per graph.  modes: ngraphs values
 * DAWN_SERVE_AUTO / _DENSE / _FRONTIER (host memory, read during the call), or
 * NULL for all AUTO.  Both steps give identical distances.  DENSE keeps two
 * n * max_lanes / 8-byte visited arrays per graph and reads all of them every
 * iteration.  FRONTIER keeps per vertex its visited words and two frontier
 * words per lane word (3 * n * max_lanes / 8 bytes) and two lists of
 * n * max_lanes / 64 uint32 keys; an iteration touches only the out-arcs of
 * the vertices reached in the previous one, plus one clearing pass over the
 * visited words in iterations that admit lanes to that graph.  FRONTIER
 * needs n * max_lanes / 64 < 2^32 (AUTO falls back to DENSE above it).
 * DAWN_E_INVALID on a bad mode.
 */
DAWN_API int dawn_serve_create_ex(const dawn_graph_t* graphs, int ngraphs, size_t mem_budget_bytes,
                                  int max_lanes, const int32_t* modes, dawn_server_t* out);

/*
 * Enqueue a request (non-blocking).  dist_out: host or device, k x n
 * source-major, int16 (dist_bytes = 2) or int32 (4); caller-owned, borrowed
 * until dawn_serve_poll reports DAWN_REQ_DONE or DAWN_REQ_FAILED.
 * *req_id identifies the request.  DAWN_E_NOMEM when the request alone can
 * never fit mem_budget_bytes.
 */
DAWN_API int dawn_serve_submit(dawn_server_t s, int graph_idx, const int32_t* sources, int32_t k,
                               int dist_bytes, void* dist_out, uint64_t* req_id);

/* State of a request (DAWN_REQ_*).  Returns the request's error code once it
 * has failed (e.g. DAWN_E_OVERFLOW), DAWN_E_STATE for an unknown id. */
DAWN_API int dawn_serve_poll(dawn_server_t s, uint64_t req_id, int* state);

/* Host clock (seconds, steady clock) at which the request was submitted and
 * at which it became DONE or FAILED (0 while open): its latency is the
 * difference.  DAWN_E_STATE for an unknown id. */
DAWN_API int dawn_serve_times(dawn_server_t s, uint64_t req_id, double* submit_s, double* done_s);

/* Block until every submitted request is done or failed (timeout_ms < 0:
 * no limit).  DAWN_E_TIMEOUT if the time ran out first. */
DAWN_API int dawn_serve_drain(dawn_server_t s, int64_t timeout_ms);

/* Drain, stop the server thread and free its buffers. */
DAWN_API int dawn_serve_destroy(dawn_server_t s);

/* Message of the calling thread's last failed call ("" if none). */
DAWN_API const char* dawn_last_error(void);

/* Library version, (major << 16) | minor. */
DAWN_API int dawn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DAWN_H */
