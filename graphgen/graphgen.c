/*
 * graphgen.c -- seeded synthetic graph generators (host C, OpenMP).
 *
 * This module only builds inputs: CSR graphs and their uint32 edge weights.
 * It holds none of the shortest-path arithmetic, so both the CPU oracle and
 * the CUDA library can be fed from it without sharing any method code.
 *
 * Graph shapes (the workloads of the frontier SSSP hot path):
 *   - 2D 4-neighbour undirected grid, side x side, vertex id = y*side + x.
 *   - RMAT (Chakrabarti et al. 2004) with quadrant probabilities a, b, c,
 *     d = 1-a-b-c, symmetrised, self-loops and duplicate edges removed, with
 *     a seeded vertex relabelling (Fisher-Yates permutation).
 *
 * Weights: one weight per unordered vertex pair, shared by both directions:
 *     w(u, v) = 1 + H(seed, min(u,v), max(u,v)) mod W
 * where H is built from splitmix64 (Steele, Lea, Flood, OOPSLA 2014).
 *
 * Every random number comes from splitmix64 applied to a counter, so the
 * output is a pure function of the parameters, independent of the number of
 * OpenMP threads.
 *
 * Rows of the CSR are sorted by destination id.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GGEN_EXPORT __attribute__((visibility("default")))

/* splitmix64 output function: the increment-then-mix step of the published
 * generator, applied to an arbitrary 64-bit counter value. */
static inline uint64_t sm64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

GGEN_EXPORT uint64_t ggen_splitmix64(uint64_t x) { return sm64(x); }

/* Weight of the unordered pair {u, v} in [1, W]. */
static inline uint32_t pair_weight(uint64_t seed, uint32_t u, uint32_t v, uint32_t W) {
    uint32_t a = u < v ? u : v, b = u < v ? v : u;
    uint64_t h = sm64(sm64(seed ^ 0xA5A5A5A55A5A5A5AULL) ^ (((uint64_t)a << 32) | b));
    return 1u + (uint32_t)(h % (uint64_t)W);
}

GGEN_EXPORT uint32_t ggen_pair_weight(uint64_t seed, uint32_t u, uint32_t v, uint32_t W) {
    return pair_weight(seed, u, v, W);
}

/* ------------------------------------------------------------------------- */
/* Grid                                                                      */
/* ------------------------------------------------------------------------- */

GGEN_EXPORT uint64_t ggen_grid_num_edges(uint32_t side) {
    if (side < 2) return 0;
    return 4ULL * side * (side - 1);
}

/* Fills row_offsets[n+1], cols[m], weights[m] for the side x side grid.
 * W == 0 means every weight is 1 (unit grid); otherwise pair weights in
 * [1, W].  const_w != 0 overrides: every weight equals const_w. */
GGEN_EXPORT int ggen_grid(uint32_t side, uint32_t W, uint32_t const_w, uint64_t seed,
                          uint32_t* row_offsets, uint32_t* cols, uint32_t* weights) {
    if (side == 0) return -1;
    const uint64_t n = (uint64_t)side * side;
    /* Rows are filled in parallel; the first edge index of row y follows
     * from the closed-form edge count of rows 0..y-1. */
    #pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < (int64_t)side; ++y) {
        /* edges before row y: sum of degrees of rows 0..y-1 */
        uint64_t before = 0;
        if (side >= 2) {
            /* per row: horizontal 2*(side-1); vertical: side per neighbouring row */
            uint64_t horiz = 2ULL * (side - 1);
            uint64_t rows_above = (uint64_t)y;
            /* vertical edges of rows 0..y-1: row 0 has side down-edges (if side>1),
             * rows 1..y-1 have 2*side each, capped by last row (not reached here) */
            uint64_t vert = 0;
            if (rows_above > 0) {
                vert = (uint64_t)side; /* row 0 */
                if (rows_above > 1) vert += 2ULL * side * (rows_above - 1);
            }
            before = horiz * rows_above + vert;
        }
        uint64_t e = before;
        for (uint32_t x = 0; x < side; ++x) {
            uint32_t v = (uint32_t)y * side + x;
            row_offsets[v] = (uint32_t)e;
            uint32_t nb[4]; int k = 0;
            if (y > 0) nb[k++] = v - side;
            if (x > 0) nb[k++] = v - 1;
            if (x + 1 < side) nb[k++] = v + 1;
            if ((uint32_t)y + 1 < side) nb[k++] = v + side;
            for (int i = 0; i < k; ++i) {
                cols[e] = nb[i];
                uint32_t w;
                if (const_w) w = const_w;
                else if (W == 0) w = 1;
                else w = pair_weight(seed, v, nb[i], W);
                weights[e] = w;
                ++e;
            }
        }
    }
    row_offsets[n] = (uint32_t)ggen_grid_num_edges(side);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Parallel LSD radix sort of 64-bit keys (used to symmetrise and dedup).    */
/* ------------------------------------------------------------------------- */

#define RBITS 16
#define RSIZE (1u << RBITS)

static void radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint64_t count, int key_bits) {
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)RSIZE * nthreads);
    uint64_t* src = keys;
    uint64_t* dst = tmp;
    int passes = (key_bits + RBITS - 1) / RBITS;
    for (int p = 0; p < passes; ++p) {
        int shift = p * RBITS;
        memset(hist, 0, sizeof(uint64_t) * (size_t)RSIZE * nthreads);
        #pragma omp parallel num_threads(nthreads)
        {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            uint64_t lo = count * t / nthreads, hi = count * (t + 1) / nthreads;
            uint64_t* h = hist + (size_t)t * RSIZE;
            for (uint64_t i = lo; i < hi; ++i) h[(src[i] >> shift) & (RSIZE - 1)]++;
            #pragma omp barrier
            #pragma omp single
            {
                uint64_t run = 0;
                for (uint32_t d = 0; d < RSIZE; ++d)
                    for (int tt = 0; tt < nthreads; ++tt) {
                        uint64_t c = hist[(size_t)tt * RSIZE + d];
                        hist[(size_t)tt * RSIZE + d] = run;
                        run += c;
                    }
            }
            for (uint64_t i = lo; i < hi; ++i) {
                uint64_t k = src[i];
                dst[h[(k >> shift) & (RSIZE - 1)]++] = k;
            }
        }
        uint64_t* s = src; src = dst; dst = s;
    }
    if (src != keys) memcpy(keys, src, sizeof(uint64_t) * count);
    free(hist);
}

/* ------------------------------------------------------------------------- */
/* RMAT                                                                      */
/* ------------------------------------------------------------------------- */

typedef struct {
    uint32_t n;
    uint64_t m;
    uint32_t* row_offsets;
    uint32_t* cols;
    uint32_t* weights;
} ggen_csr;

GGEN_EXPORT void ggen_csr_free(ggen_csr* g) {
    if (!g) return;
    free(g->row_offsets); free(g->cols); free(g->weights); free(g);
}

GGEN_EXPORT uint32_t ggen_csr_n(const ggen_csr* g) { return g->n; }
GGEN_EXPORT uint64_t ggen_csr_m(const ggen_csr* g) { return g->m; }

/* Copies the CSR into caller arrays of sizes n+1, m, m. */
GGEN_EXPORT void ggen_csr_export(const ggen_csr* g, uint32_t* ro, uint32_t* cols, uint32_t* w) {
    memcpy(ro, g->row_offsets, sizeof(uint32_t) * ((size_t)g->n + 1));
    memcpy(cols, g->cols, sizeof(uint32_t) * g->m);
    memcpy(w, g->weights, sizeof(uint32_t) * g->m);
}

/* Seeded Fisher-Yates permutation of 0..n-1. */
static void fisher_yates(uint32_t* perm, uint32_t n, uint64_t seed) {
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    uint64_t base = sm64(seed ^ 0x5EEDF00DULL);
    for (uint32_t i = n - 1; i > 0; --i) {
        uint64_t r = sm64(base + i);
        uint32_t j = (uint32_t)(r % ((uint64_t)i + 1));
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* RMAT graph with 2^scale vertices and edge_factor * 2^scale edge draws.
 * a, b, c are quadrant probabilities (d = 1 - a - b - c).  Each draw walks
 * `scale` levels; level l picks the quadrant from a 32-bit uniform taken
 * from splitmix64(counter) (two levels per 64-bit output).  The endpoints
 * are relabelled by a seeded permutation, self-loops are dropped, both
 * directions are inserted, duplicates removed, rows sorted.  Weights are
 * pair weights in [1, W] with seed `wseed`. */
GGEN_EXPORT ggen_csr* ggen_rmat(uint32_t scale, uint32_t edge_factor, double a, double b, double c,
                                uint64_t seed, uint32_t W, uint64_t wseed) {
    if (scale == 0 || scale > 30 || W == 0) return NULL;
    const uint32_t n = 1u << scale;
    const uint64_t draws = (uint64_t)edge_factor << scale;
    const uint64_t ta = (uint64_t)(a * 4294967296.0);
    const uint64_t tab = (uint64_t)((a + b) * 4294967296.0);
    const uint64_t tabc = (uint64_t)((a + b + c) * 4294967296.0);
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * 2 * draws);
    if (!perm || !keys) { free(perm); free(keys); return NULL; }
    fisher_yates(perm, n, seed);
    const uint64_t base = sm64(seed);
    const uint32_t words_per_edge = (scale + 1) / 2;
    uint64_t kept = 0;
    #pragma omp parallel
    {
        #pragma omp for schedule(static) reduction(+:kept)
        for (int64_t i = 0; i < (int64_t)draws; ++i) {
            uint32_t u = 0, v = 0;
            uint64_t ctr = base + (uint64_t)i * words_per_edge;
            uint64_t r = 0;
            for (uint32_t l = 0; l < scale; ++l) {
                uint32_t p;
                if ((l & 1) == 0) { r = sm64(ctr + (l >> 1)); p = (uint32_t)r; }
                else p = (uint32_t)(r >> 32);
                uint32_t bu, bv;
                if (p < ta) { bu = 0; bv = 0; }
                else if (p < tab) { bu = 0; bv = 1; }
                else if (p < tabc) { bu = 1; bv = 0; }
                else { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            u = perm[u]; v = perm[v];
            if (u == v) {
                keys[2 * i] = ~0ULL; keys[2 * i + 1] = ~0ULL;   /* dropped below */
            } else {
                keys[2 * i] = ((uint64_t)u << scale) | v;
                keys[2 * i + 1] = ((uint64_t)v << scale) | u;
                kept += 2;
            }
        }
    }
    free(perm);
    /* compact out the self-loop markers */
    uint64_t cnt = 0;
    for (uint64_t i = 0; i < 2 * draws; ++i) if (keys[i] != ~0ULL) keys[cnt++] = keys[i];
    (void)kept;
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (cnt ? cnt : 1));
    if (!tmp) { free(keys); return NULL; }
    radix_sort_u64(keys, tmp, cnt, 2 * (int)scale);
    free(tmp);
    uint64_t m = 0;
    for (uint64_t i = 0; i < cnt; ++i)
        if (m == 0 || keys[i] != keys[m - 1]) keys[m++] = keys[i];
    ggen_csr* g = (ggen_csr*)calloc(1, sizeof(ggen_csr));
    g->n = n; g->m = m;
    g->row_offsets = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
    g->cols = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    g->weights = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    const uint64_t vmask = ((uint64_t)1 << scale) - 1;
    for (uint64_t i = 0; i < m; ++i) g->row_offsets[(keys[i] >> scale) + 1]++;
    for (uint32_t v = 0; v < n; ++v) g->row_offsets[v + 1] += g->row_offsets[v];
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)m; ++i) {
        uint32_t u = (uint32_t)(keys[i] >> scale), v = (uint32_t)(keys[i] & vmask);
        g->cols[i] = v;
        g->weights[i] = pair_weight(wseed, u, v, W);
    }
    free(keys);
    return g;
}
