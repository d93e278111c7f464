/*
 * oracle.c -- CPU oracle for single-source shortest paths (test
 * infrastructure only).
 *
 * This file is the correctness reference for the CUDA frontier SSSP library.
 * It shares no code with that library: it is plain, slow, obviously correct
 * C.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it; the product path never does.
 *
 * What the method computes (the paper's parallel SSSP example, Listing 4,
 * with the expand operator of Listing 3): starting from dist[source] = 0 and
 * every other distance at "infinity", the frontier loop relaxes every
 * out-edge of every active vertex with an atomic minimum and re-activates
 * every vertex whose distance strictly decreased, until no vertex is active.
 * With non-negative weights this label-correcting loop stops exactly at the
 * least fixed point of  d[v] = min(d[v], d[u] + w(u,v)),  i.e. at the true
 * shortest-path distances
 *
 *     dist[v] = min over directed paths source ~> v of the sum of weights,
 *
 * whatever order the relaxations run in.  So the oracle is that definition,
 * computed by textbook algorithms:
 *
 *   oracle_dijkstra       binary-heap Dijkstra with lazy deletion (the
 *                         reference the GPU path is compared to);
 *   oracle_floyd_warshall all-pairs min-plus closure (brute force, small n);
 *   oracle_bellman_ford   rounds of relaxing every edge until nothing changes
 *                         (a different algorithm for cross-checks);
 *   oracle_bfs_hops       queue BFS hop counts (the unit-weight special case);
 *   oracle_check          the invariants that characterise shortest-path
 *                         distances for positive weights;
 *   oracle_sp_tree        the edge-frontier program: the tight edges
 *                         (dist[u] + w == dist[v], the edges on some shortest
 *                         path) and, per vertex, the smallest tight
 *                         predecessor.
 *
 * The paper's own listing keeps float weights and distances, initialised to
 * the largest float (Listings 1 and 4).  That variant is here too:
 *
 *   oracle_dijkstra_f32     the same Dijkstra over IEEE binary32: each
 *                           relaxation is the single-precision sum d[u] + w
 *                           (round to nearest) and unreached is FLT_MAX;
 *   oracle_bellman_ford_f32 Bellman-Ford rounds with the same float sums.
 *
 * Because w >= 0 makes  x -> fl(x + w)  non-decreasing and never below x,
 * both reach the least fixed point of d[v] = min(d[v], fl(d[u] + w)) from
 * d[src] = +0, d[else] = FLT_MAX, which is  min(FLT_MAX, the smallest
 * left-to-right rounded sum over the paths src ~> v).
 *
 * Types: vertex ids, CSR offsets and weights are uint32.  Distances are
 * accumulated in uint64, so the oracle cannot overflow, and stored as uint32
 * with 0xFFFFFFFF meaning unreachable.  A finite distance >= 0xFFFFFFFF
 * cannot be represented: the functions return ORACLE_ERR_RANGE for it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <time.h>
#include <float.h>

#define OR_EXPORT __attribute__((visibility("default")))
#define OR_INF32 0xFFFFFFFFu
#define OR_INF64 0xFFFFFFFFFFFFFFFFull

enum {
    ORACLE_OK = 0,
    ORACLE_ERR_ARG = 1,
    ORACLE_ERR_RANGE = 2,
    ORACLE_ERR_NOMEM = 3,
};

/* ------------------------------------------------------------------------- */
/* Binary min-heap of (distance, vertex), lazy deletion.                     */
/* ------------------------------------------------------------------------- */

typedef struct { uint64_t d; uint32_t v; } heap_item;

typedef struct {
    heap_item* a;
    uint64_t size, cap;
} heap_t;

static int heap_push(heap_t* h, uint64_t d, uint32_t v) {
    if (h->size == h->cap) {
        uint64_t nc = h->cap ? h->cap * 2 : 1024;
        heap_item* na = (heap_item*)realloc(h->a, nc * sizeof(heap_item));
        if (!na) return -1;
        h->a = na; h->cap = nc;
    }
    uint64_t i = h->size++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h->a[p].d <= d) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].d = d; h->a[i].v = v;
    return 0;
}

static heap_item heap_pop(heap_t* h) {
    heap_item top = h->a[0];
    heap_item last = h->a[--h->size];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, s = i;
        uint64_t sd = last.d;
        if (l < h->size && h->a[l].d < sd) { s = l; sd = h->a[l].d; }
        if (r < h->size && h->a[r].d < sd) { s = r; }
        if (s == i) break;
        h->a[i] = h->a[s];
        i = s;
    }
    if (h->size) h->a[i] = last;
    return top;
}

/* Dijkstra (CLRS ch. 24.3) from `src` over the CSR (row_offsets[n+1],
 * cols[m], weights[m]).  Writes dist[n] (uint32, 0xFFFFFFFF = unreachable).
 * If edges_scanned is not NULL it receives the number of edge relaxations
 * performed (each settled vertex scans its out-edges once). */
OR_EXPORT int oracle_dijkstra(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                              const uint32_t* weights, uint32_t src, uint32_t* dist,
                              uint64_t* edges_scanned) {
    if (src >= n || !row_offsets || !dist) return ORACLE_ERR_ARG;
    uint64_t* d = (uint64_t*)malloc(sizeof(uint64_t) * n);
    unsigned char* done = (unsigned char*)calloc(n, 1);
    heap_t h = {0, 0, 0};
    if (!d || !done) { free(d); free(done); return ORACLE_ERR_NOMEM; }
    for (uint32_t v = 0; v < n; ++v) d[v] = OR_INF64;
    d[src] = 0;
    if (heap_push(&h, 0, src)) { free(d); free(done); return ORACLE_ERR_NOMEM; }
    uint64_t scanned = 0;
    while (h.size) {
        heap_item it = heap_pop(&h);
        uint32_t u = it.v;
        if (done[u] || it.d != d[u]) continue;      /* stale entry */
        done[u] = 1;
        for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            uint32_t v = cols[e];
            uint64_t nd = d[u] + (uint64_t)weights[e];
            ++scanned;
            if (nd < d[v]) {
                d[v] = nd;
                if (heap_push(&h, nd, v)) { free(h.a); free(d); free(done); return ORACLE_ERR_NOMEM; }
            }
        }
    }
    int rc = ORACLE_OK;
    for (uint32_t v = 0; v < n; ++v) {
        if (d[v] == OR_INF64) dist[v] = OR_INF32;
        else if (d[v] >= OR_INF32) { dist[v] = OR_INF32; rc = ORACLE_ERR_RANGE; }
        else dist[v] = (uint32_t)d[v];
    }
    if (edges_scanned) *edges_scanned = scanned;
    free(h.a); free(d); free(done);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Floyd-Warshall: D[i*n + j] = shortest i ~> j distance (uint64, INF64 =    */
/* unreachable).  Brute force for small graphs (n <= a few hundred).         */
/* ------------------------------------------------------------------------- */
OR_EXPORT int oracle_floyd_warshall(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                                    const uint32_t* weights, uint64_t* D) {
    if (!D || n > 4096) return ORACLE_ERR_ARG;
    for (uint64_t i = 0; i < (uint64_t)n * n; ++i) D[i] = OR_INF64;
    for (uint32_t i = 0; i < n; ++i) D[(uint64_t)i * n + i] = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            uint64_t* cell = &D[(uint64_t)u * n + cols[e]];
            if (weights[e] < *cell) *cell = weights[e];
        }
    for (uint32_t k = 0; k < n; ++k)
        for (uint32_t i = 0; i < n; ++i) {
            uint64_t dik = D[(uint64_t)i * n + k];
            if (dik == OR_INF64) continue;
            for (uint32_t j = 0; j < n; ++j) {
                uint64_t dkj = D[(uint64_t)k * n + j];
                if (dkj == OR_INF64) continue;
                if (dik + dkj < D[(uint64_t)i * n + j]) D[(uint64_t)i * n + j] = dik + dkj;
            }
        }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Bellman-Ford by rounds: every round relaxes every edge of the graph, in   */
/* CSR order, from the distances at the start of the round; stop when a     */
/* round changes nothing.  At most n-1 productive rounds.                    */
/* ------------------------------------------------------------------------- */
OR_EXPORT int oracle_bellman_ford(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                                  const uint32_t* weights, uint32_t src, uint32_t* dist,
                                  uint32_t* rounds_out) {
    if (src >= n) return ORACLE_ERR_ARG;
    uint64_t* d = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint64_t* nd = (uint64_t*)malloc(sizeof(uint64_t) * n);
    if (!d || !nd) { free(d); free(nd); return ORACLE_ERR_NOMEM; }
    for (uint32_t v = 0; v < n; ++v) d[v] = OR_INF64;
    d[src] = 0;
    uint32_t rounds = 0;
    for (;;) {
        memcpy(nd, d, sizeof(uint64_t) * n);
        int changed = 0;
        for (uint32_t u = 0; u < n; ++u) {
            if (d[u] == OR_INF64) continue;
            for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
                uint64_t c = d[u] + weights[e];
                if (c < nd[cols[e]]) { nd[cols[e]] = c; changed = 1; }
            }
        }
        uint64_t* t = d; d = nd; nd = t;
        if (!changed) break;
        ++rounds;
    }
    int rc = ORACLE_OK;
    for (uint32_t v = 0; v < n; ++v) {
        if (d[v] == OR_INF64) dist[v] = OR_INF32;
        else if (d[v] >= OR_INF32) { dist[v] = OR_INF32; rc = ORACLE_ERR_RANGE; }
        else dist[v] = (uint32_t)d[v];
    }
    if (rounds_out) *rounds_out = rounds;
    free(d); free(nd);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* IEEE binary32 variant (the paper's float weights).  Weights and output   */
/* distances are passed as their bit patterns (uint32); every weight must   */
/* be a finite float >= +0.0.  Arithmetic is plain C float: one rounded     */
/* single-precision addition per relaxation.                                */
/* ------------------------------------------------------------------------- */

static float f32_of(uint32_t bits) { float f; memcpy(&f, &bits, 4); return f; }
static uint32_t bits_of(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

static int f32_weights_ok(uint32_t n, const uint32_t* row_offsets, const uint32_t* weights) {
    for (uint32_t e = 0; e < row_offsets[n]; ++e) {
        float w = f32_of(weights[e]);
        if (!(w >= 0.0f) || w > FLT_MAX || (weights[e] >> 31)) return 0;   /* NaN, negative, -0, inf */
    }
    return 1;
}

/* Binary min-heap of (float distance, vertex), lazy deletion. */
typedef struct { float d; uint32_t v; } fheap_item;
typedef struct { fheap_item* a; uint64_t size, cap; } fheap_t;

static int fheap_push(fheap_t* h, float d, uint32_t v) {
    if (h->size == h->cap) {
        uint64_t nc = h->cap ? h->cap * 2 : 1024;
        fheap_item* na = (fheap_item*)realloc(h->a, nc * sizeof(fheap_item));
        if (!na) return -1;
        h->a = na; h->cap = nc;
    }
    uint64_t i = h->size++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h->a[p].d <= d) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].d = d; h->a[i].v = v;
    return 0;
}

static fheap_item fheap_pop(fheap_t* h) {
    fheap_item top = h->a[0];
    fheap_item last = h->a[--h->size];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, s = i;
        float sd = last.d;
        if (l < h->size && h->a[l].d < sd) { s = l; sd = h->a[l].d; }
        if (r < h->size && h->a[r].d < sd) { s = r; }
        if (s == i) break;
        h->a[i] = h->a[s];
        i = s;
    }
    if (h->size) h->a[i] = last;
    return top;
}

/* Dijkstra over binary32: dist_bits[v] = bits of min(FLT_MAX, smallest
 * rounded path sum); an edge relaxation that rounds to +inf improves nothing. */
OR_EXPORT int oracle_dijkstra_f32(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                                  const uint32_t* weight_bits, uint32_t src, uint32_t* dist_bits) {
    if (src >= n || !row_offsets || !dist_bits) return ORACLE_ERR_ARG;
    if (!f32_weights_ok(n, row_offsets, weight_bits)) return ORACLE_ERR_ARG;
    float* d = (float*)malloc(sizeof(float) * n);
    unsigned char* done = (unsigned char*)calloc(n, 1);
    fheap_t h = {0, 0, 0};
    if (!d || !done) { free(d); free(done); return ORACLE_ERR_NOMEM; }
    for (uint32_t v = 0; v < n; ++v) d[v] = FLT_MAX;
    d[src] = 0.0f;
    if (fheap_push(&h, 0.0f, src)) { free(d); free(done); return ORACLE_ERR_NOMEM; }
    while (h.size) {
        fheap_item it = fheap_pop(&h);
        uint32_t u = it.v;
        if (done[u] || it.d != d[u]) continue;      /* stale entry */
        done[u] = 1;
        for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            uint32_t v = cols[e];
            volatile float nd = d[u] + f32_of(weight_bits[e]);   /* one rounded float addition */
            if (nd < d[v]) {
                d[v] = nd;
                if (fheap_push(&h, nd, v)) { free(h.a); free(d); free(done); return ORACLE_ERR_NOMEM; }
            }
        }
    }
    for (uint32_t v = 0; v < n; ++v) dist_bits[v] = bits_of(d[v]);
    free(h.a); free(d); free(done);
    return ORACLE_OK;
}

/* Bellman-Ford rounds over binary32 (a second algorithm for the same fixed point). */
OR_EXPORT int oracle_bellman_ford_f32(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                                      const uint32_t* weight_bits, uint32_t src, uint32_t* dist_bits,
                                      uint32_t* rounds_out) {
    if (src >= n) return ORACLE_ERR_ARG;
    if (!f32_weights_ok(n, row_offsets, weight_bits)) return ORACLE_ERR_ARG;
    float* d = (float*)malloc(sizeof(float) * n);
    float* nd = (float*)malloc(sizeof(float) * n);
    if (!d || !nd) { free(d); free(nd); return ORACLE_ERR_NOMEM; }
    for (uint32_t v = 0; v < n; ++v) d[v] = FLT_MAX;
    d[src] = 0.0f;
    uint32_t rounds = 0;
    for (;;) {
        memcpy(nd, d, sizeof(float) * n);
        int changed = 0;
        for (uint32_t u = 0; u < n; ++u) {
            if (d[u] == FLT_MAX) continue;   /* never reached: relaxes nothing */
            for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
                volatile float c = d[u] + f32_of(weight_bits[e]);
                if (c < nd[cols[e]]) { nd[cols[e]] = c; changed = 1; }
            }
        }
        float* t = d; d = nd; nd = t;
        if (!changed) break;
        ++rounds;
    }
    for (uint32_t v = 0; v < n; ++v) dist_bits[v] = bits_of(d[v]);
    if (rounds_out) *rounds_out = rounds;
    free(d); free(nd);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* BFS hop counts (CLRS ch. 22.2); 0xFFFFFFFF = unreachable.                 */
/* ------------------------------------------------------------------------- */
OR_EXPORT int oracle_bfs_hops(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                              uint32_t src, uint32_t* hops) {
    if (src >= n) return ORACLE_ERR_ARG;
    uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * n);
    if (!q) return ORACLE_ERR_NOMEM;
    for (uint32_t v = 0; v < n; ++v) hops[v] = OR_INF32;
    uint32_t head = 0, tail = 0;
    hops[src] = 0;
    q[tail++] = src;
    while (head < tail) {
        uint32_t u = q[head++];
        for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            uint32_t v = cols[e];
            if (hops[v] == OR_INF32) { hops[v] = hops[u] + 1; q[tail++] = v; }
        }
    }
    free(q);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Invariant check of a candidate distance array.                            */
/*   1: dist[src] != 0                                                       */
/*   2: some edge (u,v) with finite dist[u] has dist[v] > dist[u] + w        */
/*   3: some reachable v != src has no tight in-edge (dist[u] + w == dist[v])*/
/*   4: finite/infinite pattern differs from weight-blind reachability       */
/* For strictly positive weights, 1-4 passing means dist is exactly the      */
/* shortest-path distance vector (feasibility gives dist <= true, a chain of */
/* tight edges back to src gives dist >= true).                              */
/* bad_vertex receives the first offending vertex (or edge source for 2).    */
/* ------------------------------------------------------------------------- */
OR_EXPORT int oracle_check(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                           const uint32_t* weights, uint32_t src, const uint32_t* dist,
                           uint32_t* bad_vertex) {
    if (src >= n) return -1;
    if (dist[src] != 0) { if (bad_vertex) *bad_vertex = src; return 1; }
    unsigned char* tight = (unsigned char*)calloc(n, 1);
    uint32_t* hops = (uint32_t*)malloc(sizeof(uint32_t) * n);
    if (!tight || !hops) { free(tight); free(hops); return -2; }
    int rc = 0;
    tight[src] = 1;
    for (uint32_t u = 0; u < n && !rc; ++u) {
        if (dist[u] == OR_INF32) continue;
        for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            uint32_t v = cols[e];
            uint64_t c = (uint64_t)dist[u] + weights[e];
            if ((uint64_t)dist[v] > c) { rc = 2; if (bad_vertex) *bad_vertex = u; break; }
            if ((uint64_t)dist[v] == c) tight[v] = 1;
        }
    }
    if (!rc) {
        for (uint32_t v = 0; v < n; ++v)
            if (dist[v] != OR_INF32 && !tight[v]) { rc = 3; if (bad_vertex) *bad_vertex = v; break; }
    }
    if (!rc) {
        oracle_bfs_hops(n, row_offsets, cols, src, hops);
        for (uint32_t v = 0; v < n; ++v)
            if ((hops[v] == OR_INF32) != (dist[v] == OR_INF32)) { rc = 4; if (bad_vertex) *bad_vertex = v; break; }
    }
    free(tight); free(hops);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Shortest-path DAG from a distance vector (the edge-frontier program of    */
/* Sec. III-C: an operator over the frontier of tight edges).  An edge       */
/* (u, v, w) with dist[u] finite is tight when dist[u] + w == dist[v],        */
/* summed in uint64; tight[e] = 1 for those edges, 0 otherwise.  parent[src] */
/* = src; every other vertex gets the smallest u over its tight in-edges, or */
/* OR_INF32 when it has none (every unreached vertex).                       */
/* ------------------------------------------------------------------------- */
OR_EXPORT int oracle_sp_tree(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                             const uint32_t* weights, uint32_t src, const uint32_t* dist,
                             uint32_t* parent, unsigned char* tight) {
    if (src >= n) return ORACLE_ERR_ARG;
    for (uint32_t v = 0; v < n; ++v) parent[v] = OR_INF32;
    parent[src] = src;
    for (uint32_t u = 0; u < n; ++u) {
        for (uint32_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {
            const uint32_t v = cols[e];
            const int t = dist[u] != OR_INF32 && (uint64_t)dist[u] + weights[e] == (uint64_t)dist[v];
            tight[e] = (unsigned char)t;
            if (t && v != src && u < parent[v]) parent[v] = u;
        }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* Many independent Dijkstra runs spread over host threads: out row s holds  */
/* the distances from srcs[s] (out[s*n + v]).  Used to time the CPU baseline */
/* of batched queries; each thread runs the same oracle_dijkstra.            */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint32_t n; const uint32_t *ro, *cols, *w;
    const uint32_t* srcs; uint32_t k; uint32_t* out;
    uint32_t next; pthread_mutex_t mu; int rc;
} many_ctx;

static void* many_worker(void* arg) {
    many_ctx* c = (many_ctx*)arg;
    for (;;) {
        pthread_mutex_lock(&c->mu);
        uint32_t s = c->next++;
        pthread_mutex_unlock(&c->mu);
        if (s >= c->k) break;
        int rc = oracle_dijkstra(c->n, c->ro, c->cols, c->w, c->srcs[s], c->out + (uint64_t)s * c->n, NULL);
        if (rc) { pthread_mutex_lock(&c->mu); c->rc = rc; pthread_mutex_unlock(&c->mu); }
    }
    return NULL;
}

OR_EXPORT int oracle_dijkstra_many(uint32_t n, const uint32_t* row_offsets, const uint32_t* cols,
                                   const uint32_t* weights, const uint32_t* srcs, uint32_t k,
                                   uint32_t* out, uint32_t threads) {
    if (threads == 0) threads = 1;
    many_ctx c = {n, row_offsets, cols, weights, srcs, k, out, 0, PTHREAD_MUTEX_INITIALIZER, 0};
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
    if (!th) return ORACLE_ERR_NOMEM;
    for (uint32_t t = 0; t < threads; ++t) pthread_create(&th[t], NULL, many_worker, &c);
    for (uint32_t t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    return c.rc;
}
