/*
 * Seeded synthetic graph generators (input side only).
 *
 * This file builds the unweighted test graphs on which both the CPU oracle and
 * the CUDA path are run.  It holds none of the shortest-path arithmetic: it only
 * draws random graphs and writes them as CSR (row_ptr int32[n+1], col_idx
 * int32[m], every row sorted ascending, no duplicate arcs, no self-loops).
 *
 * Graph classes stand in for the paper's evaluation graphs (Sec. 4.1: 66
 * SuiteSparse / Gunrock graphs, small-world and high-diameter road-like):
 *   - directed Erdos-Renyi with Poisson(lambda) out-degrees,
 *   - RMAT (Graph500-style recursive matrix, a/b/c/d quadrant probabilities,
 *     no noise), vertex ids randomly permuted, optionally symmetrised,
 *   - 2-D 4-neighbour lattice with independent bond deletion.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood, 2014), both written from their published
 * definitions.  Uniform doubles take the top 53 bits; a uniform integer in
 * [0, k) is the high half of a 32x32-bit product (bias below 2^-32 * k).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;
    int64_t m;
    int32_t* row_ptr;
    int32_t* col_idx;
} gg_csr;

/* ---------------------------------------------------------------- PRNG -- */

typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t splitmix64_next(uint64_t* x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void rng_seed(gg_rng* r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(gg_rng* r) {
    uint64_t* s = r->s;
    const uint64_t result = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

static inline double rng_uniform(gg_rng* r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

static inline uint32_t rng_below(gg_rng* r, uint32_t k) {
    return (uint32_t)(((rng_next(r) >> 32) * (uint64_t)k) >> 32);
}

/* Exported so that tests can pin the generator to the published test vectors. */
uint64_t gg_splitmix64_first(uint64_t seed) {
    uint64_t x = seed;
    return splitmix64_next(&x);
}

void gg_xoshiro_stream(uint64_t seed, int64_t count, uint64_t* out) {
    gg_rng r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < count; ++i) out[i] = rng_next(&r);
}

/* ------------------------------------------------------- CSR assembly -- */

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Insertion sort for short rows, qsort for long ones. */
static void sort_row(int32_t* a, int64_t len) {
    if (len < 32) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t v = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > v) { a[j + 1] = a[j]; --j; }
            a[j + 1] = v;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Build a CSR from an arc list (src[i] -> dst[i]); self-loops are dropped,
 * each row is sorted and duplicate arcs are removed.  Consumes src/dst.
 */
static gg_csr* csr_from_arcs(int32_t n, int64_t na, int32_t* src, int32_t* dst) {
    gg_csr* g = (gg_csr*)calloc(1, sizeof(gg_csr));
    if (!g) return NULL;
    g->n = n;
    int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!cnt) { free(g); return NULL; }
    for (int64_t i = 0; i < na; ++i)
        if (src[i] != dst[i]) cnt[src[i] + 1]++;
    for (int32_t v = 0; v < n; ++v) cnt[v + 1] += cnt[v];
    int64_t tot = cnt[n];
    int32_t* col = (int32_t*)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
    int64_t* pos = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!col || !pos) { free(col); free(pos); free(cnt); free(g); return NULL; }
    memcpy(pos, cnt, ((size_t)n + 1) * sizeof(int64_t));
    for (int64_t i = 0; i < na; ++i)
        if (src[i] != dst[i]) col[pos[src[i]]++] = dst[i];
    free(pos);
    /* sort + dedup each row (rows are independent: in parallel), then
     * compact the rows in order */
    int32_t* rp = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    int64_t* keep = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!rp || !keep) { free(rp); free(keep); free(col); free(cnt); free(g); return NULL; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int32_t v = 0; v < n; ++v) {
        int64_t b = cnt[v], e = cnt[v + 1];
        sort_row(col + b, e - b);
        int64_t w = b;
        for (int64_t i = b; i < e; ++i) {
            if (w > b && col[w - 1] == col[i]) continue;
            col[w++] = col[i];
        }
        keep[v] = w - b;
    }
    int64_t w = 0;
    rp[0] = 0;
    for (int32_t v = 0; v < n; ++v) {
        const int64_t b = cnt[v], k = keep[v];
        if (w != b) memmove(col + w, col + b, (size_t)k * sizeof(int32_t));
        w += k;
        rp[v + 1] = (int32_t)w;
    }
    free(keep);
    free(cnt);
    g->m = w;
    g->row_ptr = rp;
    g->col_idx = (int32_t*)realloc(col, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
    if (!g->col_idx) g->col_idx = col;
    return g;
}

/* ------------------------------------------------------- generators -- */

/*
 * Directed Erdos-Renyi: for every u, k_u ~ Poisson(lambda) drawn by Knuth's
 * product-of-uniforms method, then k_u targets uniform in [0, n).
 * Self-loops dropped, duplicates removed, rows sorted.
 */
gg_csr* gg_er(int32_t n, double lambda, uint64_t seed) {
    if (n <= 0 || lambda < 0) return NULL;
    gg_rng r;
    rng_seed(&r, seed);
    const double L = exp(-lambda);
    int64_t cap = (int64_t)n * (int64_t)(lambda + 8) + 64, na = 0;
    int32_t* src = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    if (!src || !dst) { free(src); free(dst); return NULL; }
    for (int32_t u = 0; u < n; ++u) {
        int k = 0;
        double p = 1.0;
        do { ++k; p *= rng_uniform(&r); } while (p > L);
        k -= 1;
        for (int t = 0; t < k; ++t) {
            if (na == cap) {
                cap *= 2;
                int32_t* s2 = (int32_t*)realloc(src, (size_t)cap * sizeof(int32_t));
                int32_t* d2 = (int32_t*)realloc(dst, (size_t)cap * sizeof(int32_t));
                if (!s2 || !d2) { free(s2 ? s2 : src); free(d2 ? d2 : dst); return NULL; }
                src = s2; dst = d2;
            }
            src[na] = u;
            dst[na] = (int32_t)rng_below(&r, (uint32_t)n);
            ++na;
        }
    }
    gg_csr* g = csr_from_arcs(n, na, src, dst);
    free(src);
    free(dst);
    return g;
}

/*
 * RMAT (Chakrabarti, Zhan & Faloutsos 2004; Graph500 parameters): edge_factor
 * * 2^scale samples; each sample descends `scale` levels, choosing quadrant
 * (0,0),(0,1),(1,0),(1,1) with probabilities a, b, c, 1-a-b-c (most
 * significant bit first).  Vertex ids are relabelled by a Fisher-Yates
 * permutation drawn from the same stream after all samples.  With
 * `symmetrise`, every sample (u,v) contributes both arcs u->v and v->u.
 * Self-loops dropped, duplicates removed, rows sorted.
 */
gg_csr* gg_rmat(int scale, int edge_factor, double a, double b, double c,
                uint64_t seed, int symmetrise) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return NULL;
    const int32_t n = (int32_t)1 << scale;
    const int64_t ns = (int64_t)edge_factor * (int64_t)n;
    const int64_t na = symmetrise ? 2 * ns : ns;
    gg_rng r;
    rng_seed(&r, seed);
    int32_t* src = (int32_t*)malloc((size_t)na * sizeof(int32_t));
    int32_t* dst = (int32_t*)malloc((size_t)na * sizeof(int32_t));
    int32_t* perm = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!src || !dst || !perm) { free(src); free(dst); free(perm); return NULL; }
    const double ab = a + b, abc = a + b + c;
    for (int64_t e = 0; e < ns; ++e) {
        uint32_t u = 0, v = 0;
        for (int lvl = 0; lvl < scale; ++lvl) {
            double x = rng_uniform(&r);
            uint32_t ub, vb;
            if (x < a)        { ub = 0; vb = 0; }
            else if (x < ab)  { ub = 0; vb = 1; }
            else if (x < abc) { ub = 1; vb = 0; }
            else              { ub = 1; vb = 1; }
            u = (u << 1) | ub;
            v = (v << 1) | vb;
        }
        src[e] = (int32_t)u;
        dst[e] = (int32_t)v;
    }
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = n - 1; i > 0; --i) {
        int32_t j = (int32_t)rng_below(&r, (uint32_t)i + 1);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (int64_t e = 0; e < ns; ++e) {
        src[e] = perm[src[e]];
        dst[e] = perm[dst[e]];
    }
    if (symmetrise) {
        for (int64_t e = 0; e < ns; ++e) {
            src[ns + e] = dst[e];
            dst[ns + e] = src[e];
        }
    }
    free(perm);
    gg_csr* g = csr_from_arcs(n, na, src, dst);
    free(src);
    free(dst);
    return g;
}

/*
 * rows x cols 4-neighbour lattice, vertex id = r * cols + c.  Bonds are visited
 * in row-major vertex order, right bond then down bond; each is deleted with
 * probability p_delete (one uniform draw per bond, kept iff draw >= p_delete).
 * A kept bond contributes both arcs.  Rows are emitted sorted (up, left,
 * right, down).
 */
gg_csr* gg_lattice(int32_t rows, int32_t cols, double p_delete, uint64_t seed) {
    if (rows <= 0 || cols <= 0) return NULL;
    int64_t nn = (int64_t)rows * cols;
    if (nn > 0x7fffffffLL) return NULL;
    const int32_t n = (int32_t)nn;
    gg_rng r;
    rng_seed(&r, seed);
    uint8_t* bond = (uint8_t*)calloc((size_t)n, 1); /* bit0: right kept, bit1: down kept */
    if (!bond) return NULL;
    for (int32_t y = 0; y < rows; ++y)
        for (int32_t x = 0; x < cols; ++x) {
            int32_t id = y * cols + x;
            if (x + 1 < cols && rng_uniform(&r) >= p_delete) bond[id] |= 1;
            if (y + 1 < rows && rng_uniform(&r) >= p_delete) bond[id] |= 2;
        }
    gg_csr* g = (gg_csr*)calloc(1, sizeof(gg_csr));
    int32_t* rp = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!g || !rp) { free(g); free(rp); free(bond); return NULL; }
    int64_t m = 0;
    rp[0] = 0;
    for (int32_t id = 0; id < n; ++id) {
        int32_t y = id / cols, x = id % cols;
        int d = 0;
        if (y > 0 && (bond[id - cols] & 2)) ++d;
        if (x > 0 && (bond[id - 1] & 1)) ++d;
        if (bond[id] & 1) ++d;
        if (bond[id] & 2) ++d;
        m += d;
        rp[id + 1] = (int32_t)m;
    }
    int32_t* col = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!col) { free(g); free(rp); free(bond); return NULL; }
    int64_t w = 0;
    for (int32_t id = 0; id < n; ++id) {
        int32_t y = id / cols, x = id % cols;
        if (y > 0 && (bond[id - cols] & 2)) col[w++] = id - cols;
        if (x > 0 && (bond[id - 1] & 1)) col[w++] = id - 1;
        if (bond[id] & 1) col[w++] = id + 1;
        if (bond[id] & 2) col[w++] = id + cols;
    }
    free(bond);
    g->n = n;
    g->m = m;
    g->row_ptr = rp;
    g->col_idx = col;
    return g;
}

/*
 * Draw k distinct vertices uniformly from those with out-degree >= 1
 * (Graph500 root convention).  Returns the number drawn (< k only when fewer
 * than k such vertices exist).
 */
int32_t gg_sample_sources(const int32_t* row_ptr, int32_t n, int32_t k, uint64_t seed,
                          int32_t* out) {
    int32_t avail = 0;
    for (int32_t v = 0; v < n; ++v) avail += row_ptr[v + 1] > row_ptr[v];
    if (k > avail) k = avail;
    uint8_t* taken = (uint8_t*)calloc((size_t)n, 1);
    if (!taken) return -1;
    gg_rng r;
    rng_seed(&r, seed);
    int32_t got = 0;
    while (got < k) {
        int32_t v = (int32_t)rng_below(&r, (uint32_t)n);
        if (taken[v] || row_ptr[v + 1] == row_ptr[v]) continue;
        taken[v] = 1;
        out[got++] = v;
    }
    free(taken);
    return got;
}

/* Draw k vertices uniformly from [0, n) (repeats allowed). */
void gg_uniform_vertices(int32_t n, int32_t k, uint64_t seed, int32_t* out) {
    gg_rng r;
    rng_seed(&r, seed);
    for (int32_t i = 0; i < k; ++i) out[i] = (int32_t)rng_below(&r, (uint32_t)n);
}

/*
 * Arc weights for the weighted extension: w = lo + h mod (hi - lo + 1), h the
 * splitmix64 output of seed mixed with the arc's endpoints.  With symmetric
 * set the endpoints are taken as an unordered pair, so both arcs of an
 * undirected edge carry the same weight; repeated arcs get the same weight.
 */
void gg_arc_weights(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int32_t lo, int32_t hi,
                    uint64_t seed, int symmetric, int32_t* out) {
    const uint64_t span = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
    for (int32_t u = 0; u < n; ++u) {
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            uint32_t a = (uint32_t)u, b = (uint32_t)col_idx[j];
            if (symmetric && b < a) { uint32_t t = a; a = b; b = t; }
            uint64_t x = seed ^ (((uint64_t)a << 32) | (uint64_t)b);
            out[j] = (int32_t)((int64_t)lo + (int64_t)(splitmix64_next(&x) % span));
        }
    }
}

int32_t gg_n(const gg_csr* g) { return g->n; }
int64_t gg_m(const gg_csr* g) { return g->m; }

void gg_copy(const gg_csr* g, int32_t* row_ptr, int32_t* col_idx) {
    memcpy(row_ptr, g->row_ptr, ((size_t)g->n + 1) * sizeof(int32_t));
    if (g->m > 0) memcpy(col_idx, g->col_idx, (size_t)g->m * sizeof(int32_t));
}

void gg_free(gg_csr* g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col_idx);
    free(g);
}
