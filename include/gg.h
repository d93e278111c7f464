/*
 * gg.h -- C ABI of the B300 frontier single-source-shortest-path library.
 *
 * The library implements the native-graph decomposition of "Essentials of
 * Parallel Graph Analytics" (Osama, Porumbescu, Owens, 2022):
 *
 *   graph      a CSR graph (Sec. IV-A, Listing 1) -- row offsets, column
 *              indices and uint32 edge weights -- plus its transpose (CSC)
 *              for pull traversals (Sec. III-C, "Push vs. Pull" box);
 *   frontier   the active vertex set, held both as a sparse vertex queue
 *              and as a dense bitmap (Sec. III-B, Sec. IV-B, Listing 2);
 *   operator   neighbors_expand, the advance that relaxes every out-edge of
 *              the frontier with an atomic minimum, fused with a filter that
 *              deduplicates and compacts the improved vertices into the next
 *              frontier (Sec. IV-C, Listing 3);
 *   loop       repeat while the frontier is non-empty (the convergence
 *              condition of Listing 4), either bulk-synchronously (the
 *              execution::par policy) or asynchronously over a work queue
 *              (the execution::par_nosync policy, Sec. III-A and the
 *              "Timing Model and Parallelism" box).
 *
 * Numeric contract (the paper's Listing 4 with uint32 in place of float):
 *   dist[v] = min over directed paths source ~> v of the sum of the uint32
 *   edge weights; dist[source] = 0; GG_INF (0xFFFFFFFF) marks an unreachable
 *   vertex.  Results are exact integers, identical for every policy,
 *   direction and load-balance mode.  Weights may be zero; self-loops and
 *   multi-edges are allowed (the lightest parallel edge wins).  A finite
 *   distance of 2^32 - 1 or more cannot be represented: the run then reports
 *   GG_ERR_OVERFLOW from gg_graph_check (the stored value saturates at
 *   0xFFFFFFFE).
 *
 * Conventions:
 *   - Every call returns a gg_status; no C++ exception crosses the ABI.
 *     gg_last_error() gives a thread-local message for the last failure.
 *   - Device work is stream-ordered on the cudaStream_t passed in (0 = the
 *     legacy default stream).  Results are valid once that stream reaches
 *     the point after the call.  Device-side failures (overflow, iteration
 *     cap, watchdog timeout) are recorded in the graph handle and returned
 *     by gg_graph_check(), which synchronises the stream.
 *   - Pointers documented as "device" must be device (or managed) memory of
 *     the current CUDA device; "host" pointers are ordinary host memory.
 *   - One graph handle runs one SSSP at a time.  Calls on the same handle
 *     from different streams are ordered by the library (each call waits for
 *     the previous one on that handle).
 */
#ifndef GG_H
#define GG_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GG_INF 0xFFFFFFFFu
#define GG_ABI_VERSION 4

typedef struct gg_graph* gg_graph_t;

typedef enum {
    GG_OK = 0,
    GG_ERR_INVALID_ARG = 1,   /* bad pointer, size, index or CSR structure        */
    GG_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed               */
    GG_ERR_CUDA = 3,          /* a CUDA runtime call failed (see gg_last_error)   */
    GG_ERR_TIMEOUT = 4,       /* a bounded device wait gave up (watchdog)         */
    GG_ERR_BUSY = 5,          /* resource in use / admission refused              */
    GG_ERR_NOT_READY = 6,     /* asynchronous result not available yet            */
    GG_ERR_OVERFLOW = 7,      /* a finite distance did not fit below GG_INF       */
    GG_ERR_INTERNAL = 8,      /* iteration cap exceeded or internal invariant     */
    GG_ERR_NOT_SUPPORTED = 9  /* option combination not available                 */
} gg_status;

/* gg_graph_create_csr flags */
#define GG_DEVICE_PTRS 0x1u   /* row_offsets/col_indices/weights are device pointers */
#define GG_SYMMETRIC   0x2u   /* caller asserts the graph is symmetric: the CSR is
                                 its own transpose, so pull reuses it (no CSC built) */
#define GG_NO_VALIDATE 0x4u   /* skip the structural checks (offsets, col < n)     */
#define GG_NO_PACK     0x8u   /* keep 8-byte {col, weight} edges even when the
                                 4-byte packed form (col << wbits | weight) fits  */
#define GG_FLOAT_WEIGHTS 0x10u /* weights are IEEE-754 binary32 bit patterns, as the
                                 paper's float weights (Listing 1, Listing 4): each
                                 must be finite and >= +0.0 (-0.0, negatives, inf
                                 and NaN are rejected unless GG_NO_VALIDATE).
                                 gg_sssp / gg_sssp_ex then write binary32 distance
                                 bit patterns: dist[src] = +0.0, each relaxation
                                 computes the round-to-nearest float sum
                                 dist[u] + w, unreached = FLT_MAX (0x7F7FFFFF, the
                                 paper's initial value), and a sum that rounds to
                                 +inf never improves a distance.  Near-far buckets
                                 are not used (delta is ignored).  Batched,
                                 multi-graph and server calls return
                                 GG_ERR_NOT_SUPPORTED for such a graph. */

/* Execution policy: the paper's execution::par / execution::par_nosync
 * (Sec. III-A; Listing 3 and the "Timing Model and Parallelism" box). */
typedef enum {
    GG_POLICY_BSP_GRAPH = 0,        /* bulk-synchronous supersteps in a CUDA graph whose
                                       conditional WHILE node tests frontier size != 0 */
    GG_POLICY_ASYNC_PERSISTENT = 1, /* one persistent kernel over a device work queue,
                                       no barriers, device-side termination detection */
    GG_POLICY_BSP_HOST = 2,         /* the same supersteps launched one by one from the
                                       host (for comparison and per-kernel timing)   */
    GG_POLICY_BSP_PERSISTENT = 3    /* the same supersteps in one cooperative launch,
                                       separated by a bounded grid barrier (no launch
                                       per superstep: for high-diameter graphs)      */
} gg_policy;

/* Traversal direction (Sec. III-C): push over CSR, pull over CSC. */
typedef enum { GG_DIR_AUTO = 0, GG_DIR_PUSH = 1, GG_DIR_PULL = 2 } gg_direction;

/* Load balancing of the push advance (Sec. IV-C: "data parallelism and load
 * balancing"). */
typedef enum {
    GG_LB_AUTO = 0,        /* library choice: warp streaming, with warp-local rounds on  */
                           /* graphs of mean degree < 8                                 */
    GG_LB_MERGE_PATH = 1,  /* equal edge ranges per CTA over the frontier's degree scan  */
    GG_LB_BINS = 2,        /* thread / warp / CTA per vertex by degree thresholds        */
    GG_LB_WARP = 3,        /* equal edge ranges per warp, streamed 32 edges at a time,   */
                           /* with no CTA barriers (push only; pull uses merge-path)     */
    GG_LB_LOCAL = 4        /* warp streaming, then up to 16 warp-local rounds per        */
                           /* superstep: the near vertices a warp improves are expanded  */
                           /* by that warp at once (rows of <= 32 edges), the rest goes  */
                           /* to the next frontier (BSP graph and host policies; for     */
                           /* high-diameter graphs: several hops per superstep)          */
} gg_lb_mode;

typedef struct {
    uint32_t iterations;       /* supersteps run (BSP) or 0 (async)                   */
    uint32_t pull_iterations;  /* of which pull                                        */
    uint64_t edges_scanned;    /* edges relaxed, summed over supersteps / queue pops    */
    uint64_t frontier_total;   /* sum of frontier sizes (vertex activations)          */
    uint32_t max_frontier;     /* largest frontier                                     */
    uint32_t device_status;    /* gg_status recorded on the device                     */
} gg_stats;

typedef struct {
    uint32_t struct_size;      /* sizeof(gg_options); set by gg_options_default        */
    gg_policy policy;
    gg_direction direction;
    gg_lb_mode lb_mode;
    uint32_t warp_threshold;   /* LB_BINS: degree >= this -> warp per vertex (0 = auto)  */
    uint32_t cta_threshold;    /* LB_BINS: degree >= this -> CTA per vertex (0 = auto)   */
    uint32_t pull_alpha;       /* AUTO direction: go pull when frontier edges > m/alpha
                                  (0 = 4)                                               */
    uint32_t pull_beta;        /* AUTO direction: back to push when frontier vertices <
                                  (vertices with in-edges)/beta (0 = 24)                */
    uint32_t max_iterations;   /* BSP superstep cap (0 = n + 2)                          */
    uint64_t watchdog_ns;      /* give up and report GG_ERR_TIMEOUT after this long
                                  (0 = 10 s for ASYNC, 60 s for the BSP policies)      */
    gg_stats* stats;           /* host; if not NULL the call synchronises the stream
                                  and fills it                                          */
    uint32_t* trace;           /* device u32[trace_cap*4] or NULL.  BSP: per superstep
                                  (frontier size, frontier edges, kind 0 push / 1 pull
                                  / 2 near-far split / 3 heavy-edge push / 4 heavy-edge
                                  pull / 5 heavy-edge pull that ends the buckets and
                                  writes the plain push's first frontier, next
                                  frontier size).  ASYNC: per
                                  near-far split (split number, new threshold, far-pile
                                  size, microseconds since the kernel started)         */
    uint32_t trace_cap;
    uint32_t delta;            /* near-far bucket width: vertices improved to a distance
                                  below the current threshold stay in the frontier, the
                                  rest wait in a far pile until the frontier empties and
                                  the threshold rises by delta (0 = the graph's default,
                                  GG_DELTA_NONE = plain frontier loop, no buckets)       */
    uint32_t light_heavy;      /* GG_LH_AUTO: with buckets, the BSP graph and host policies
                                  relax heavy edges (weight >= delta) once per settled
                                  vertex (Meyer-Sanders delta-stepping): near supersteps
                                  relax only light edges, and a heavy superstep runs
                                  when the near frontier empties (on symmetric graphs,
                                  by pull into the unsettled vertices when that scans
                                  fewer edges).  Once the unsettled vertices hold fewer
                                  than m/8 heavy edges the threshold becomes infinite
                                  and the rest of the run is plain push supersteps
                                  over all edges.  Push direction,
                                  integer weights, and delta <= the largest weight.  The
                                  first such run builds a copy of the edges with each
                                  row's light edges first (4 or 8 bytes per edge, kept
                                  by the handle; rebuilt when delta changes).
                                  GG_LH_OFF: every expansion relaxes all edges.
                                  Distances are the same either way.                     */
} gg_options;

#define GG_DELTA_NONE 0xFFFFFFFFu
#define GG_LH_AUTO 0u
#define GG_LH_OFF 1u
#define GG_LH_ROUNDS 2u   /* batched calls: light-first rounds without buckets (the
                             label-correcting schedule); single source: as GG_LH_AUTO */

/* ---- graph (Sec. IV-A, Listing 1) ------------------------------------- */

/* Builds a graph handle from a CSR.
 *   n            vertices, 1 <= n < 2^32 - 1
 *   m            directed edges, m < 2^32 (offsets are uint32)
 *   row_offsets  u32[n+1], row_offsets[0] = 0, non-decreasing, row_offsets[n] = m
 *   col_indices  u32[m], each < n
 *   weights      u32[m]
 *   flags        GG_DEVICE_PTRS | GG_SYMMETRIC | GG_NO_VALIDATE | GG_NO_PACK
 *   stream       stream for the upload and preprocessing; the call returns after
 *                they are complete (it synchronises the stream)
 *   out          receives the handle
 * The handle owns a device copy (edges re-encoded as interleaved {col, weight}
 * pairs, or packed into one u32 (col << wbits) | weight when the bits of n-1
 * and of the largest weight fit in 32, plus the transpose unless
 * GG_SYMMETRIC); the caller's arrays may be freed after the call.  Errors: GG_ERR_INVALID_ARG for a null pointer, n or m
 * out of range, or (unless GG_NO_VALIDATE) a CSR whose offsets are not
 * monotone from 0 to m or whose column index is >= n; GG_ERR_OUT_OF_MEMORY;
 * GG_ERR_CUDA.  On error *out is set to NULL. */
gg_status gg_graph_create_csr(uint32_t n, uint64_t m, const uint32_t* row_offsets,
                              const uint32_t* col_indices, const uint32_t* weights,
                              uint32_t flags, cudaStream_t stream, gg_graph_t* out);

/* Frees the handle and its device memory (synchronises its last stream).
 * Handles and their workspaces allocate from a stream-ordered pool per device
 * that keeps up to 8 GiB of freed memory mapped for later handles (no device
 * synchronisation or re-mapping per handle); that memory is released when the
 * process exits. */
gg_status gg_graph_destroy(gg_graph_t g);

/* n, m and the device bytes held by the handle. */
gg_status gg_graph_info(gg_graph_t g, uint32_t* n, uint64_t* m, uint64_t* device_bytes);

/* Synchronises the stream of the handle's last call and returns the device
 * status of that call: GG_OK, GG_ERR_OVERFLOW, GG_ERR_INTERNAL (superstep cap)
 * or GG_ERR_TIMEOUT (async watchdog).  Clears the recorded status. */
gg_status gg_graph_check(gg_graph_t g);

/* ---- SSSP (Sec. IV-D, Listing 4) ---------------------------------------- */

/* Fills opt with the defaults: BSP graph policy, push direction (a pull
 * superstep sweeps every edge of the transpose; on the measured SSSP
 * workloads push-only was faster), merge-path load balancing, the graph's
 * default near-far bucket width. */
void gg_options_default(gg_options* opt);

/* Single-source shortest paths from src.
 *   dist_out  device u32[n], caller-owned; receives the distances.
 * Asynchronous on `stream`.  The first call on a handle allocates its
 * workspace (frontier queues, bitmaps: about 12n + 3n/8 bytes) and builds the
 * CUDA graph.  Errors: GG_ERR_INVALID_ARG (null handle or dist_out, src >= n),
 * GG_ERR_OUT_OF_MEMORY, GG_ERR_CUDA. */
gg_status gg_sssp(gg_graph_t g, uint32_t src, uint32_t* dist_out, cudaStream_t stream);

/* As gg_sssp with explicit options (opt may be NULL for the defaults). */
gg_status gg_sssp_ex(gg_graph_t g, uint32_t src, uint32_t* dist_out, const gg_options* opt,
                     cudaStream_t stream);

/* Breadth-first search: a second vertex program on the same operators,
 * frontiers and loop.  Sec. III-C makes the operator's work a user program
 * applied to each {source, destination, edge}; here that program counts every
 * edge as 1, so depth_out[v] = the fewest edges on a path src -> v (u32;
 * depth_out[src] = 0; unreachable = 0xFFFFFFFF), whatever the graph's weights
 * (u32 or binary32).
 *   depth_out  device u32[n], caller-owned; valid once `stream` completes
 * gg_bfs_ex honours the same options as gg_sssp_ex (policy, direction,
 * load balance, stats, trace, watchdog); delta is ignored.  Errors as
 * gg_sssp_ex. */
gg_status gg_bfs(gg_graph_t g, uint32_t src, uint32_t* depth_out, cudaStream_t stream);
gg_status gg_bfs_ex(gg_graph_t g, uint32_t src, uint32_t* depth_out, const gg_options* opt, cudaStream_t stream);

/* ---- an edge-frontier program: the shortest-path DAG and predecessors ---- */

/* Sec. III-C lets a frontier hold edges and the operator apply the user's
 * program to each {source, destination, edge}.  This program runs two
 * operators over the graph and a distance vector from src:
 *   advance + filter  every out-edge (u, v, w) of every reached vertex u is
 *                     tested and joins the output edge frontier when it is
 *                     tight, dist[u] + w == dist[v] (exact 64-bit sum): the
 *                     edges that lie on some shortest path from src;
 *   edge operator     over that edge frontier, parent[v] = min(parent[v], u).
 *   src          < n; dist: device u32[n], the distances from src (for
 *                example gg_sssp's output; GG_INF = unreached)
 *   parent_out   device u32[n], caller-owned: parent[src] = src; for every
 *                other reached vertex the smallest u with a tight edge
 *                (u, v) (GG_INF if dist admits none); GG_INF for unreached
 *                vertices.  With zero-weight edges the parent map may hold
 *                cycles among vertices of equal distance.
 *   tight_out    device u32[tight_cap] or NULL: receives up to tight_cap
 *                tight edges as positions in the CSR (edge ids), in no
 *                particular order
 *   tight_count  host, optional: the number of tight edges (may exceed
 *                tight_cap)
 * Synchronous on `stream` (orders after the handle's last call).  The edge
 * frontier takes up to 8 bytes per edge of temporary device memory (4 when
 * tight_cap >= m).  Integer-weight graphs only (GG_ERR_NOT_SUPPORTED for
 * GG_FLOAT_WEIGHTS).  Errors: GG_ERR_INVALID_ARG (NULLs, src >= n,
 * tight_cap > 0 with tight_out NULL), GG_ERR_OUT_OF_MEMORY, GG_ERR_CUDA. */
gg_status gg_sssp_tree(gg_graph_t g, uint32_t src, const uint32_t* dist, uint32_t* parent_out,
                       uint32_t* tight_out, uint64_t tight_cap, uint64_t* tight_count, cudaStream_t stream);

/* ---- autotuning ----------------------------------------------------------- */

/* Picks the fastest single-source options for this graph (Sec. IV-C leaves
 * load balancing and the operator's execution choices to the implementation):
 * coordinate descent over the loop policy (CUDA graph or persistent), the
 * bucket width (on graphs with a light/heavy width: widths giving 1.5 to 4.5
 * light edges per vertex; otherwise the near-far width from 1/8 to 8 times
 * the default; and no buckets), push-only vs push/pull switching thresholds, and
 * warp streaming with or without warp-local rounds vs merge-path vs degree
 * bins with their thresholds.  Every candidate runs
 * gg_sssp_ex from each sample source on `stream` and is timed with CUDA
 * events (median of 3); candidates that report a device error are skipped.
 *   srcs          host u32[nsrc], each < n
 *   dist_scratch  device u32[n] the runs write into
 *   best          receives the winning options (stats/trace pointers NULL)
 *   best_ms       optional: its time per source in milliseconds
 * Synchronous; takes roughly 50 runs per sample source. */
gg_status gg_autotune(gg_graph_t g, const uint32_t* srcs, uint32_t nsrc, uint32_t* dist_scratch,
                      gg_options* best, float* best_ms, cudaStream_t stream);

/* Picks the fastest batched options for this graph and these sources: the
 * schedule (GG_LH_AUTO normalised buckets or GG_LH_ROUNDS) and the
 * light/heavy width (delta: 1.5 to 4.5 light edges per vertex, or
 * GG_DELTA_NONE).  Each candidate runs gg_sssp_batch_ex over all k sources on
 * `stream`, timed with CUDA events (median of 3); candidates that report a
 * device error are skipped.
 *   srcs          host u32[k], each < n
 *   dist_scratch  device u32[n*k] the runs write into
 *   best          receives the winning options (stats/trace pointers NULL)
 *   best_ms       optional: its time per batched call in milliseconds
 * Synchronous; about 45 batched calls. */
gg_status gg_autotune_batch(gg_graph_t g, const uint32_t* srcs, uint32_t k, uint32_t* dist_scratch,
                            gg_options* best, float* best_ms, cudaStream_t stream);

/* ---- batched multi-source SSSP ------------------------------------------ */

/* k independent single-source runs of the same frontier loop (Listing 4)
 * fused into one bulk-synchronous loop: the frontier holds vertices with a
 * 64-bit mask of the sources whose distance there just improved, so one read
 * of an edge serves every such source.  Sources are processed in groups of
 * 64 (one fused loop per group).
 *   srcs      host u32[k], each < n (duplicates allowed)
 *   k         >= 1
 *   dist_out  device u32[n*k], caller-owned, vertex-major:
 *             dist_out[v*k + s] = distance from srcs[s] to v (GG_INF if none)
 * Asynchronous on `stream` (the source list is copied before the call
 * returns).  Push traversal only.  The first call allocates the handle's
 * batch workspace (about 60n bytes).  Errors: GG_ERR_INVALID_ARG (null
 * pointers, k == 0, a source >= n), GG_ERR_OUT_OF_MEMORY, GG_ERR_CUDA;
 * device status (overflow, superstep cap) via gg_graph_check. */
gg_status gg_sssp_batch(gg_graph_t g, const uint32_t* srcs, uint32_t k, uint32_t* dist_out,
                        cudaStream_t stream);

/* As gg_sssp_batch with options: max_iterations, stats (summed over the
 * 64-source groups; setting stats synchronises the stream), trace (first
 * 64-source group only: per superstep kind | 16 once bucketing has ended
 * (kind 0 light or plain push, 1 split, 2 heavy push, 3 mask clear before
 * the tail, 4 heavy pull, 5 heavy pull that ends the buckets and writes the
 * tail's first frontier), entries, edges, next frontier size), delta,
 * light_heavy and the policy GG_POLICY_BSP_HOST (supersteps launched one by
 * one from the host, synchronising after each; every other policy runs the
 * CUDA-graph loop);
 * direction and load-balance fields are ignored.
 *
 * On graphs with a light/heavy width (mean degree >= 8, integer weights),
 * unless light_heavy is GG_LH_OFF or delta is GG_DELTA_NONE or exceeds the
 * largest weight, the sources run light-first rounds over the light-first
 * edge copy that the single-source loop uses (built on first use), with
 * width delta (0 = the graph's width): light supersteps relax only the light
 * edges (weight < width) of their (vertex, sources) entries, every improving
 * pair is also recorded in an R mask, and when the light frontier empties one
 * heavy superstep relaxes the heavy edges of the R pairs.
 *   GG_LH_AUTO (default): normalised buckets.  Each source's distances are
 *     shifted by sh[s] = max o - o_s, o_s its distance from the graph's
 *     highest-degree vertex (computed once per handle by a single-source run,
 *     kept by the handle); one shared threshold over the shifted distances
 *     moves in steps of the width, pairs at or above it wait parked, and
 *     each pair's heavy edges are relaxed once, when its bucket settles
 *     (delta-stepping per source with the buckets of all sources aligned).
 *     Once the pairs not yet settled hold fewer than 1/8 of the heavy edges,
 *     the rest is plain push over all edges.
 *   GG_LH_ROUNDS: the same rounds without buckets (label-correcting: a
 *     pair's heavy edges are relaxed once per epoch in which it improved).
 * Otherwise delta 0 or GG_DELTA_NONE runs the plain frontier loop, and
 * another delta parks (vertex, source) pairs at or above the threshold in
 * per-vertex far masks (near-far buckets).  Distances are the same in every
 * mode. */
gg_status gg_sssp_batch_ex(gg_graph_t g, const uint32_t* srcs, uint32_t k, uint32_t* dist_out,
                           const gg_options* opt, cudaStream_t stream);

/* ---- many graphs in one launch sequence --------------------------------- */

/* One single-source query per (graphs[i], srcs[i]) pair, all advanced
 * together: every superstep is one kernel over the union of the queries'
 * frontiers, balanced by edges across the GPU whatever the graphs' sizes
 * (graphs may repeat; each query has its own distance array).
 *   graphs     host array of count handles on the current device
 *   srcs       host u32[count], srcs[i] < n of graphs[i]
 *   dist_outs  host array of count device pointers, dist_outs[i] u32[n_i]
 * Asynchronous on `stream`; the arrays are read before the call returns.
 * The library keeps one engine per device for these calls (allocated or
 * grown on demand); calls are ordered among themselves.  Push traversal with
 * each graph's default near-far bucket width; at most 1024 queries per call.
 * Errors: GG_ERR_INVALID_ARG, GG_ERR_OUT_OF_MEMORY, GG_ERR_CUDA. */
gg_status gg_sssp_multi(const gg_graph_t* graphs, const uint32_t* srcs, uint32_t count,
                        uint32_t* const* dist_outs, cudaStream_t stream);

/* As gg_sssp_multi with an explicit near-far bucket width for every query
 * (0 = each graph's default, GG_DELTA_NONE = plain frontier loop).  Each query
 * keeps its own threshold and far pile; a query whose near frontier empties
 * splits its pile during the next shared superstep. */
gg_status gg_sssp_multi_ex(const gg_graph_t* graphs, const uint32_t* srcs, uint32_t count,
                           uint32_t* const* dist_outs, uint32_t delta, cudaStream_t stream);

/* ---- single source over a 1D vertex partition (one part per rank) -------- */

/* Sec. III-D and Table I place the graph on several processors by a
 * partition of its vertices (random partitioning being the simplest).  Each
 * rank (one process per GPU) holds a part: the out-edges of the vertices it
 * owns, with global column ids, and those vertices' distances.  One
 * superstep is
 *   gg_part_advance   relax the part's frontier: updates to owned vertices
 *                     are applied at once (atomicMin; a vertex whose distance
 *                     dropped joins the next frontier once), updates to other
 *                     ranks' vertices are written to send_pairs, grouped by
 *                     destination rank;
 *   (the caller exchanges the groups between ranks: a collective)
 *   gg_part_apply     relax the received pairs the same way and close the
 *                     superstep.
 * The run ends when every rank's next frontier is empty (the caller reduces
 * next_size over the ranks).  The fixed point is the one of the one-GPU loop.
 * Parts are independent handles: no call waits on another rank. */
typedef struct gg_part* gg_part_t;

/* route: host u32[n_global], route[v] = (owner rank << 24) | (index of v
 * among its owner's vertices, in the owner's row order); nranks <= 256,
 * n_local <= 2^24.  row_offsets: host u32[n_local + 1] over the owned
 * vertices in local order; cols (global ids < n_global), weights: host
 * u32[m_local].  Uploads and synchronises `stream`.  Errors:
 * GG_ERR_INVALID_ARG (NULLs, ranks out of range, offsets not monotone from
 * 0, a column >= n_global, a route to a rank >= nranks, a local index
 * >= n_local, or a route that gives this rank other than n_local vertices),
 * GG_ERR_CUDA. */
gg_status gg_part_create(uint32_t n_global, uint32_t rank, uint32_t nranks, uint32_t n_local, const uint32_t* route,
                         const uint32_t* row_offsets, const uint32_t* cols, const uint32_t* weights,
                         cudaStream_t stream, gg_part_t* out);
gg_status gg_part_destroy(gg_part_t p);
/* n_local and the part's edge count (the most remote updates one superstep can emit). */
gg_status gg_part_info(gg_part_t p, uint32_t* n_local, uint64_t* m_local);
/* dist := GG_INF on the part; the source's owner seeds dist = 0 and its
 * frontier.  Every rank calls it with the same src_global. */
gg_status gg_part_begin(gg_part_t p, uint32_t src_global, cudaStream_t stream);
/* send_pairs: device u32[2 * cap]; receives (index on the destination rank,
 * distance) pairs, destination d's from offset sum(send_counts[0..d)) on.
 * send_counts: host u64[nranks] (this rank's own entry is 0).  Synchronous.
 * GG_ERR_INVALID_ARG when the pairs exceed cap (cap = m_local always
 * suffices). */
gg_status gg_part_advance(gg_part_t p, cudaStream_t stream, uint32_t* send_pairs, uint64_t cap,
                          uint64_t* send_counts);
/* recv_pairs: device u32[2 * count], pairs addressed to this rank (local
 * index, distance).  Closes the superstep; next_size (host) receives this
 * rank's next frontier size.  Synchronous.  GG_ERR_OVERFLOW when a finite
 * distance did not fit below GG_INF. */
gg_status gg_part_apply(gg_part_t p, const uint32_t* recv_pairs, uint64_t count, cudaStream_t stream,
                        uint32_t* next_size);
/* The part's distances (device u32[n_local], local order). */
gg_status gg_part_distances(gg_part_t p, uint32_t* dist_out, cudaStream_t stream);

/* ---- query server (continuous batching) --------------------------------- */

typedef struct gg_server* gg_server_t;

typedef struct {
    uint32_t struct_size;            /* sizeof(gg_server_config)                          */
    uint32_t max_slots;              /* queries in flight at once (0 = 64)                */
    uint32_t max_graph_vertices;     /* largest graph that may be queried (required)      */
    uint32_t supersteps_per_launch;  /* supersteps between admission rounds (0 = 8)       */
    uint64_t max_vertices_in_flight; /* budget: sum of n over in-flight queries
                                        (0 = max_slots * max_graph_vertices), capped by
                                        the free HBM at creation                          */
    uint64_t hbm_reserve_bytes;      /* HBM the server leaves free (default 1 GiB)        */
    uint32_t delta;                  /* near-far bucket width per query (0 = each graph's
                                        default, GG_DELTA_NONE = plain frontier loop)     */
    uint32_t reserved;
} gg_server_config;

typedef struct {
    uint64_t submitted, completed;
    uint64_t launches;               /* superstep-graph launches by the worker            */
    uint64_t vertex_budget;          /* in-flight vertex budget of the last admission round */
    uint32_t queued, running, max_running;
    uint32_t reserved;
    double p50_us, p99_us, mean_us, max_us;   /* submit -> completion latency           */
} gg_server_stats;

void gg_server_config_default(gg_server_config* cfg);

/* Creates a server on the current device: one worker thread with its own
 * stream runs a loop of {admit queued queries into free slots while the
 * in-flight vertex budget allows; advance every in-flight query by up to
 * supersteps_per_launch supersteps in one CUDA-graph launch; retire the
 * queries whose frontier emptied}.  Queries arriving while others run join
 * the running union frontier at the next admission round.  The engine's
 * capacity is sized from the free HBM at creation (16 bytes of frontier state
 * per vertex, plus per slot three bitmaps and two far piles of
 * max_graph_vertices entries); GG_ERR_OUT_OF_MEMORY if even one graph does
 * not fit.  Admission then follows the free HBM live: at every admission
 * round the budget in force is min(capacity, vertices in flight +
 * (free HBM - hbm_reserve_bytes) / 32), so when other allocations leave
 * less than the reserve free, queued queries wait (in-flight ones finish)
 * until memory is released.  max_slots <= 1024.
 * Queries on graphs with a light/heavy width (mean degree >= 8, integer
 * weights), when cfg.delta is 0, do not take slots: they are coalesced per
 * graph, up to 64 queued sources of one graph at a time (round robin over the
 * graphs), into one batched call (gg_sssp_batch_ex on the server's second
 * stream, overlapping the slot launches) whose matrix columns are then copied
 * to the queries' arrays.  A batch starts when the free HBM above the reserve
 * holds its n x k distance matrix. */
gg_status gg_server_create(const gg_server_config* cfg, gg_server_t* out);

/* Queues the query (graph g, source src) whose distances go to dist_out
 * (device u32[n], caller-owned, untouched by anyone else until the query
 * completes).  g must stay alive until then.  Returns a ticket.  Errors:
 * GG_ERR_INVALID_ARG (NULLs, src >= n, graph larger than
 * max_graph_vertices), GG_ERR_BUSY after destroy began. */
gg_status gg_server_submit(gg_server_t s, gg_graph_t g, uint32_t src, uint32_t* dist_out, uint64_t* ticket);

/* GG_ERR_NOT_READY while the query is queued or running.  When it is done:
 * returns GG_OK, sets *result to the query's own status (GG_OK or
 * GG_ERR_OVERFLOW) and forgets the ticket. */
gg_status gg_server_poll(gg_server_t s, uint64_t ticket, gg_status* result);

/* As poll, blocking up to timeout_ms (GG_ERR_NOT_READY on timeout). */
gg_status gg_server_wait(gg_server_t s, uint64_t ticket, uint32_t timeout_ms, gg_status* result);

/* Counters and latency percentiles over the queries completed so far. */
gg_status gg_server_get_stats(gg_server_t s, gg_server_stats* out);
/* Forgets the latency samples and counters (queries in flight stay). */
gg_status gg_server_reset_stats(gg_server_t s);

/* Finishes every queued and in-flight query, then frees the server. */
gg_status gg_server_destroy(gg_server_t s);

/* ---- SSSP without any device allocation ---------------------------------- */

/* Largest vertex count gg_sssp_noalloc accepts. */
#define GG_NOALLOC_MAX_VERTICES (1u << 20)

/* The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory: for example code whose GPU memory is
 * already owned by another allocator (a framework's caching allocator that has
 * reserved most of the device, where a fresh cudaMalloc fails or fragments
 * the pool), or a latency-sensitive loop that cannot afford the implicit
 * device-wide synchronisation of cudaFree.
 *
 * Computes the same distances as gg_sssp, reading the caller's CSR in place:
 *   n            vertices, 1 <= n <= GG_NOALLOC_MAX_VERTICES; larger n returns
 *                GG_ERR_INVALID_ARG (use gg_graph_create_csr + gg_sssp)
 *   m            edges, m < 2^32 - 1
 *   row_offsets  device u32[n+1]; col_indices, weights: device u32[m]
 *                (checked on the device: offsets monotone from 0 to m,
 *                columns < n; a bad CSR returns GG_ERR_INVALID_ARG)
 *   src          < n
 *   dist_out     device u32[n], caller-owned
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its working
 * memory is one fixed array of about 24.3 MiB compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 * All calls share that array and it keeps the last call's contents: each
 * call resets what must start at zero, and calls whose GPU work overlaps (on
 * different streams or host threads) race on it, so the caller must order
 * them.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * outside any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset on a device the kept address is stale, so
 * gg_sssp_noalloc must not be called on that device after a reset.  The call synchronises `stream` and returns
 * when dist_out is complete (push supersteps launched from the host).
 * Returns GG_ERR_OVERFLOW when a finite distance does not fit below GG_INF. */
gg_status gg_sssp_noalloc(uint32_t n, uint64_t m, const uint32_t* row_offsets,
                          const uint32_t* col_indices, const uint32_t* weights, uint32_t src,
                          uint32_t* dist_out, cudaStream_t stream);

/* ---- errors ------------------------------------------------------------- */

const char* gg_status_string(gg_status s);
/* Thread-local message describing the last failed call on this thread. */
const char* gg_last_error(void);
/* GG_ABI_VERSION of the loaded library. */
uint32_t gg_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GG_H */
