/*
 * CPU ORACLE for DAWN (Feng et al., "DAWN: Matrix Operation-Optimized Algorithm
 * for Shortest Paths Problem on Unweighted Graphs", ICS '24).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path calls this file; only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark do.  It
 * shares no code, header or table with the CUDA library.  It is plain,
 * single-threaded and deliberately slow: every loop follows the paper's
 * algorithm in its own order, with dense Boolean vectors where the paper has
 * them.
 *
 * Conventions (readings of the paper, see the design notes):
 *   - dist[v] = -1 means "no path"; dist[src] = 0.  The paper uses 0 for
 *     "unset", which collides with the source's own distance (Thm 1 requires
 *     i != j), so the source is pre-marked reached with distance 0.
 *   - step counts from 1: the first expansion stamps distance 1.
 *   - the outer loop runs while step < n, as printed, and ends early on the
 *     first step that reaches no new vertex (Sec. 3.1, stop condition 2).
 *
 * Functions and the passages they follow:
 *   oracle_sssp_sovm     Alg. 3 (SOVM), Eq. 5-7: push over CSR rows of alpha.
 *   oracle_sssp_bovm     Alg. 1 (BOVM), Eq. 2-4: pull over CSC columns with
 *                        the first-hit exit; merge of alpha and beta after
 *                        the whole vertex loop.
 *   oracle_bfs_queue     Alg. 2 (General BFS), FIFO queue.
 *   oracle_apsp_floyd    brute force on the unit-weight digraph (Floyd-Warshall),
 *                        small n only.
 *   oracle_apsp_powers   Thm 1 read literally: d(i,j) = the first k with
 *                        (A^k)_{ij} != 0, i != j, with Boolean matrix powers
 *                        (Lemma 1); small n only.
 *   oracle_certificate   O(n+m) check that a distance vector is the exact
 *                        unweighted distance from src (Thm 1 with Fact 1).
 *   oracle_wcc           weakly connected component labels (union-find).
 *   oracle_parents       shortest-path tree from exact distances (Fact 1 /
 *                        Thm 1: a vertex at level d > 0 is entered from one at
 *                        level d - 1), smallest-id tie-break.
 *   oracle_centrality    closeness, harmonic centrality and whole-run
 *                        diameter / radius from the SOVM distances of each
 *                        listed source (Sec. 3.3's APSP, Table 1's epsilon).
 *   oracle_msbfs         APSP as SOVM from each listed source (Sec. 3.3,
 *                        "APSP repeats the SSSP per source"), plus per-source
 *                        eccentricity (largest finite distance, Table 1's
 *                        epsilon(i)), distance sum and reached count. *
 * The weighted extension (Sec. 5 names (min, +) operations on weighted graphs
 * as future work; the readings are in the design notes): non-negative int32
 * arc weights, int64 distances, -1 = no path.
 *   oracle_wsssp_minplus  the SOVM iteration of Alg. 3 over the (min, +)
 *                        semiring: each round every frontier vertex i (its
 *                        distance changed in the previous round) offers
 *                        d(i) + w(i, c) to every out-neighbour c, with d(i)
 *                        as it was at the start of the round; the minimum
 *                        is kept; the vertices whose distance fell form the
 *                        next frontier; stop on a round that changes nothing.
 *   oracle_dijkstra      textbook Dijkstra with a binary heap (a different
 *                        algorithm for the same distances: a pin).
 *   oracle_wcertificate  O(n + m) exactness check of a weighted distance
 *                        vector: d(src) = 0; no arc from a reached vertex
 *                        can lower its head; every reached vertex is reached
 *                        from src along arcs with d(u) + w = d(v).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * Alg. 3, Sparse Optimized Boolean Vector-Matrix Operation.
 * alpha: the vertices whose distance was set in the previous step (dense bool).
 * beta:  the vertices whose distance is set in this step (dense bool).
 * For each alpha[i], every CSR arc i->c with c unset gets beta[c] = 1 and
 * dist[c] = step; then alpha takes beta and beta is cleared.
 *
 * edge_visits (nullable) counts every arc examined; Sec. 3.3 gives its value
 * as the sum of out-degrees over the reached vertices.  levels (nullable)
 * receives the number of steps that found at least one vertex.
 * Returns 0, or -1 on allocation failure / bad source.
 */
int oracle_sssp_sovm(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                     int32_t src, int32_t* dist, int64_t* edge_visits, int32_t* levels) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    uint8_t* alpha = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* beta = (uint8_t*)calloc((size_t)n, 1);
    if (!alpha || !beta) { free(alpha); free(beta); return -1; }
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    dist[src] = 0;
    alpha[src] = 1;
    int64_t visits = 0;
    int32_t found_levels = 0;
    int32_t step = 0;
    while (step < n) {
        step += 1;
        int converged = 1;
        for (int32_t i = 0; i < n; ++i) {
            if (!alpha[i]) continue;
            int32_t start = row_ptr[i], end = row_ptr[i + 1];
            for (int32_t j = start; j < end; ++j) {
                int32_t c = col_idx[j];
                visits += 1;
                if (dist[c] == -1) {
                    beta[c] = 1;
                    dist[c] = step;
                    converged = 0;
                }
            }
        }
        /* alpha <- beta, beta <- 0 ("reset the vector by swap") */
        uint8_t* t = alpha;
        alpha = beta;
        beta = t;
        memset(beta, 0, (size_t)n);
        if (converged) break;
        found_levels = step;
    }
    free(alpha);
    free(beta);
    if (edge_visits) *edge_visits = visits;
    if (levels) *levels = found_levels;
    return 0;
}

/*
 * Alg. 1, Boolean Vector-Matrix Operation, on the CSC (in-adjacency) of the
 * graph: csc_ptr[i]..csc_ptr[i+1] lists the in-neighbours of i.
 * alpha: every vertex reached so far (dense bool).  For each i not in alpha,
 * the compressed inner product of Eq. 4 is evaluated over i's in-neighbours
 * and stops at the first in-neighbour in alpha; then beta[i] = 1 and
 * dist[i] = step.  alpha <- alpha OR beta and beta <- 0 happen after the whole
 * i loop, so that every test in a step sees the vertex set of the step start.
 */
int oracle_sssp_bovm(int32_t n, const int32_t* csc_ptr, const int32_t* csc_row,
                     int32_t src, int32_t* dist, int32_t* levels) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    uint8_t* alpha = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* beta = (uint8_t*)calloc((size_t)n, 1);
    if (!alpha || !beta) { free(alpha); free(beta); return -1; }
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    dist[src] = 0;
    alpha[src] = 1;
    int32_t found_levels = 0;
    int32_t step = 0;
    while (step < n) {
        step += 1;
        int converged = 1;
        for (int32_t i = 0; i < n; ++i) {
            if (alpha[i]) continue;
            int32_t start = csc_ptr[i], end = csc_ptr[i + 1];
            for (int32_t j = start; j < end; ++j) {
                int32_t r = csc_row[j];
                if (alpha[r] && r != i) {
                    beta[i] = 1;
                    dist[i] = step;
                    converged = 0;
                    break;
                }
            }
        }
        for (int32_t i = 0; i < n; ++i) {
            alpha[i] = (uint8_t)(alpha[i] | beta[i]);
            beta[i] = 0;
        }
        if (converged) break;
        found_levels = step;
    }
    free(alpha);
    free(beta);
    if (levels) *levels = found_levels;
    return 0;
}

/* Alg. 2, General BFS, with a FIFO queue; a popped vertex i stamps
 * dist[i] + 1 on every unset out-neighbour and enqueues it. */
int oracle_bfs_queue(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                     int32_t src, int32_t* dist) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    int32_t* q = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!q) return -1;
    for (int32_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t head = 0, tail = 0;
    dist[src] = 0;
    q[tail++] = src;
    while (head < tail) {
        int32_t i = q[head++];
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
            int32_t c = col_idx[j];
            if (dist[c] == -1) {
                dist[c] = dist[i] + 1;
                q[tail++] = c;
            }
        }
    }
    free(q);
    return 0;
}

/* Floyd-Warshall on the unit-weight digraph; d is n*n row-major, -1 = no path. */
int oracle_apsp_floyd(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* d) {
    if (n <= 0 || n > 4096) return -1;
    const int32_t INF = 0x3fffffff;
    for (int64_t x = 0; x < (int64_t)n * n; ++x) d[x] = INF;
    for (int32_t i = 0; i < n; ++i) {
        d[(int64_t)i * n + i] = 0;
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
            int32_t c = col_idx[j];
            if (c != i) d[(int64_t)i * n + c] = 1;
        }
    }
    for (int32_t k = 0; k < n; ++k)
        for (int32_t i = 0; i < n; ++i) {
            int32_t dik = d[(int64_t)i * n + k];
            if (dik == INF) continue;
            for (int32_t j = 0; j < n; ++j) {
                int32_t via = dik + d[(int64_t)k * n + j];
                if (d[(int64_t)k * n + j] != INF && via < d[(int64_t)i * n + j])
                    d[(int64_t)i * n + j] = via;
            }
        }
    for (int64_t x = 0; x < (int64_t)n * n; ++x)
        if (d[x] == INF) d[x] = -1;
    return 0;
}

/*
 * Thm 1 with Lemma 1: with P_k = Boolean A^k, d(i,j) for i != j is the first
 * k in 1..n-1 with P_k[i][j] = 1; d(i,i) = 0; never set = -1.
 * P_{k+1}[i][j] = OR_l P_k[i][l] AND A[l][j].  O(n^4) worst case: small n only.
 */
int oracle_apsp_powers(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* d) {
    if (n <= 0 || n > 512) return -1;
    size_t nn = (size_t)n * n;
    uint8_t* A = (uint8_t*)calloc(nn, 1);
    uint8_t* P = (uint8_t*)calloc(nn, 1);
    uint8_t* Q = (uint8_t*)calloc(nn, 1);
    if (!A || !P || !Q) { free(A); free(P); free(Q); return -1; }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) A[(size_t)i * n + col_idx[j]] = 1;
    for (size_t x = 0; x < nn; ++x) d[x] = -1;
    for (int32_t i = 0; i < n; ++i) d[(size_t)i * n + i] = 0;
    memcpy(P, A, nn); /* P = A^1 */
    for (int32_t k = 1; k < n; ++k) {
        int any_new = 0;
        for (int32_t i = 0; i < n; ++i)
            for (int32_t j = 0; j < n; ++j)
                if (i != j && P[(size_t)i * n + j] && d[(size_t)i * n + j] == -1) {
                    d[(size_t)i * n + j] = k;
                    any_new = 1;
                }
        (void)any_new;
        /* Q = P * A over (OR, AND) */
        memset(Q, 0, nn);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t l = 0; l < n; ++l) {
                if (!P[(size_t)i * n + l]) continue;
                const uint8_t* arow = A + (size_t)l * n;
                uint8_t* qrow = Q + (size_t)i * n;
                for (int32_t j = 0; j < n; ++j) qrow[j] |= arow[j];
            }
        uint8_t* t = P; P = Q; Q = t;
    }
    free(A); free(P); free(Q);
    return 0;
}

/*
 * Certificate that dist is the exact unweighted distance vector from src.
 * Returns 0 when all hold, otherwise the number of the first failed item:
 *   1  dist[src] != 0, or some v != src has dist 0, or some dist < -1
 *   2  an arc (u,v) with dist[u] >= 0 has dist[v] == -1 or dist[v] > dist[u]+1
 *   3  some v with dist[v] > 0 has no in-neighbour u with dist[u] == dist[v]-1
 * Items 1-3 together characterise the distance vector: item 2 closes the
 * reached set under out-arcs and bounds dist above by the true distance;
 * item 3 exhibits a path of length dist[v] from src, bounding it below.
 * `bad` (nullable) receives the offending vertex.
 */
int oracle_certificate(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                       int32_t src, const int32_t* dist, int32_t* bad) {
    if (bad) *bad = -1;
    if (src < 0 || src >= n || dist[src] != 0) { if (bad) *bad = src; return 1; }
    for (int32_t v = 0; v < n; ++v)
        if (dist[v] < -1 || (dist[v] == 0 && v != src)) { if (bad) *bad = v; return 1; }
    uint8_t* supported = (uint8_t*)calloc((size_t)n, 1);
    if (!supported) return -1;
    for (int32_t u = 0; u < n; ++u) {
        if (dist[u] < 0) continue;
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            int32_t v = col_idx[j];
            if (dist[v] == -1 || dist[v] > dist[u] + 1) {
                free(supported);
                if (bad) *bad = v;
                return 2;
            }
            if (dist[v] == dist[u] + 1) supported[v] = 1;
        }
    }
    for (int32_t v = 0; v < n; ++v)
        if (dist[v] > 0 && !supported[v]) {
            free(supported);
            if (bad) *bad = v;
            return 3;
        }
    free(supported);
    return 0;
}

static int32_t uf_find(int32_t* p, int32_t x) {
    while (p[x] != x) {
        p[x] = p[p[x]];
        x = p[x];
    }
    return x;
}

/* Weakly connected components: label[v] = smallest vertex id of v's WCC. */
int oracle_wcc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, int32_t* label) {
    int32_t* p = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!p) return -1;
    for (int32_t v = 0; v < n; ++v) p[v] = v;
    for (int32_t u = 0; u < n; ++u)
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            int32_t a = uf_find(p, u), b = uf_find(p, col_idx[j]);
            if (a == b) continue;
            if (a < b) p[b] = a; else p[a] = b;
        }
    for (int32_t v = 0; v < n; ++v) label[v] = uf_find(p, v);
    free(p);
    return 0;
}

/*
 * APSP-style batch: SOVM from each of the k sources.  dist_block (nullable) is
 * k x n source-major int32.  ecc[s] = largest finite distance from sources[s]
 * (0 for an isolated source), dsum[s] = sum of finite distances, reached[s] =
 * number of vertices with a finite distance (the source included).
 */
int oracle_msbfs(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                 const int32_t* sources, int32_t k, int32_t* dist_block,
                 int32_t* ecc, int64_t* dsum, int32_t* reached) {
    int32_t* dist = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!dist) return -1;
    for (int32_t s = 0; s < k; ++s) {
        if (oracle_sssp_sovm(n, row_ptr, col_idx, sources[s], dist, NULL, NULL) != 0) {
            free(dist);
            return -1;
        }
        int32_t e = 0, r = 0;
        int64_t sum = 0;
        for (int32_t v = 0; v < n; ++v) {
            if (dist[v] < 0) continue;
            r += 1;
            sum += dist[v];
            if (dist[v] > e) e = dist[v];
        }
        if (ecc) ecc[s] = e;
        if (dsum) dsum[s] = sum;
        if (reached) reached[s] = r;
        if (dist_block) memcpy(dist_block + (size_t)s * n, dist, (size_t)n * sizeof(int32_t));
    }
    free(dist);
    return 0;
}

/*
 * Shortest-path tree (Fact 1 / Thm 1).  Given the exact distances from a
 * source, a vertex v at distance d > 0 is entered on some shortest path from
 * every u with an arc u->v and dist[u] = d - 1.  parent[v] is the smallest
 * such u (the tie-break that makes the tree unique); -1 for the source and
 * for unreached vertices.  Every CSR arc is examined, in CSR order.
 */
int oracle_parents(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                   const int32_t* dist, int32_t* parent) {
    if (n < 0) return -1;
    for (int32_t v = 0; v < n; ++v) parent[v] = -1;
    for (int32_t u = 0; u < n; ++u) {
        if (dist[u] < 0) continue;
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            const int32_t v = col_idx[j];
            if (dist[v] == dist[u] + 1 && (parent[v] < 0 || u < parent[v])) parent[v] = u;
        }
    }
    return 0;
}

/*
 * Centrality of each listed source from its SOVM distances (Alg. 3 per
 * source, Sec. 3.3).  With c_d = number of vertices at distance d:
 *   ecc = largest d with c_d > 0 (0 if none), dsum = sum of d * c_d,
 *   reached = 1 + sum of c_d, closeness = (reached - 1) / dsum (0 when
 *   nothing else is reached), harmonic = sum over d = 1, 2, ... of c_d / d,
 *   added in ascending d in double precision.
 * summary (nullable) = {largest ecc, smallest ecc over the sources that reach
 * another vertex (-1 if none), sum of (reached - 1), sum of dsum}.
 * Any output pointer may be NULL.  Returns 0, or -1 on bad input.
 */
int oracle_centrality(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                      const int32_t* sources, int32_t k, int32_t* ecc, int64_t* dsum, int32_t* reached,
                      double* closeness, double* harmonic, int64_t* summary) {
    int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t* count = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!dist || !count) { free(dist); free(count); return -1; }
    int64_t big = 0, small = -1, pairs = 0, total = 0;
    for (int32_t i = 0; i < k; ++i) {
        if (oracle_sssp_sovm(n, row_ptr, col_idx, sources[i], dist, NULL, NULL) != 0) {
            free(dist); free(count);
            return -1;
        }
        for (int32_t d = 0; d < n; ++d) count[d] = 0;
        for (int32_t v = 0; v < n; ++v)
            if (dist[v] > 0) count[dist[v]] += 1;
        int32_t e = 0;
        int64_t sum = 0, r = 1;
        double h = 0.0;
        for (int32_t d = 1; d < n; ++d) {
            if (count[d] == 0) continue;
            e = d;
            sum += (int64_t)d * count[d];
            r += count[d];
            h += (double)count[d] / (double)d;
        }
        if (ecc) ecc[i] = e;
        if (dsum) dsum[i] = sum;
        if (reached) reached[i] = (int32_t)r;
        if (closeness) closeness[i] = r > 1 ? (double)(r - 1) / (double)sum : 0.0;
        if (harmonic) harmonic[i] = h;
        if (e > big) big = e;
        if (r > 1 && (small < 0 || e < small)) small = e;
        pairs += r - 1;
        total += sum;
    }
    if (summary) {
        summary[0] = big;
        summary[1] = small;
        summary[2] = pairs;
        summary[3] = total;
    }
    free(dist);
    free(count);
    return 0;
}


/* ------------------------------------------------------------------------
 * Weighted extension: (min, +) in place of (OR, AND).
 * ---------------------------------------------------------------------- */

#define ORACLE_INF INT64_MAX

/*
 * The SOVM loop of Alg. 3 with (min, +): alpha = vertices whose distance
 * changed in the previous round; each round every alpha[i] offers
 * dprev[i] + w to each out-neighbour, dprev being the distances at the start
 * of the round, and the smaller value is kept; beta collects the vertices
 * whose distance fell.  A round that lowers nothing ends the loop.  With
 * non-negative weights at most n - 1 rounds change something; a further one
 * is reported as an error (-2).  rounds (nullable) receives the number of
 * rounds that changed a distance; relax (nullable) the arcs offered.
 */
int oracle_wsssp_minplus(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* w,
                         int32_t src, int64_t* dist, int32_t* rounds, int64_t* relax) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    for (int32_t v = 0; v < n; ++v)
        for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j)
            if (w[j] < 0) return -1;
    int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    int64_t* dprev = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    uint8_t* alpha = (uint8_t*)calloc((size_t)n, 1);
    uint8_t* beta = (uint8_t*)calloc((size_t)n, 1);
    if (!d || !dprev || !alpha || !beta) {
        free(d); free(dprev); free(alpha); free(beta);
        return -1;
    }
    for (int32_t v = 0; v < n; ++v) d[v] = ORACLE_INF;
    d[src] = 0;
    alpha[src] = 1;
    int32_t r = 0;
    int64_t offered = 0;
    int rc = 0;
    while (1) {
        memcpy(dprev, d, sizeof(int64_t) * (size_t)n);
        int changed = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (!alpha[i]) continue;
            for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
                const int32_t c = col_idx[j];
                const int64_t nd = dprev[i] + (int64_t)w[j];
                offered += 1;
                if (nd < d[c]) {
                    d[c] = nd;
                    beta[c] = 1;
                    changed = 1;
                }
            }
        }
        if (!changed) break;
        r += 1;
        if (r > n - 1) { rc = -2; break; }
        uint8_t* t = alpha;
        alpha = beta;
        beta = t;
        memset(beta, 0, (size_t)n);
    }
    for (int32_t v = 0; v < n; ++v) dist[v] = d[v] == ORACLE_INF ? -1 : d[v];
    if (rounds) *rounds = r;
    if (relax) *relax = offered;
    free(d); free(dprev); free(alpha); free(beta);
    return rc;
}

/* Textbook Dijkstra: binary min-heap of (distance, vertex) with lazy deletion. */
typedef struct { int64_t key; int32_t v; } oracle_heap_item;

static void heap_push(oracle_heap_item* h, int64_t* size, int64_t key, int32_t v) {
    int64_t i = (*size)++;
    h[i].key = key;
    h[i].v = v;
    while (i > 0) {
        const int64_t p = (i - 1) / 2;
        if (h[p].key <= h[i].key) break;
        oracle_heap_item t = h[p]; h[p] = h[i]; h[i] = t;
        i = p;
    }
}

static oracle_heap_item heap_pop(oracle_heap_item* h, int64_t* size) {
    oracle_heap_item top = h[0];
    h[0] = h[--(*size)];
    int64_t i = 0;
    while (1) {
        const int64_t l = 2 * i + 1, r = l + 1;
        int64_t m = i;
        if (l < *size && h[l].key < h[m].key) m = l;
        if (r < *size && h[r].key < h[m].key) m = r;
        if (m == i) break;
        oracle_heap_item t = h[m]; h[m] = h[i]; h[i] = t;
        i = m;
    }
    return top;
}

int oracle_dijkstra(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* w,
                    int32_t src, int64_t* dist) {
    if (n <= 0 || src < 0 || src >= n) return -1;
    const int64_t m = row_ptr[n];
    oracle_heap_item* h = (oracle_heap_item*)malloc(sizeof(oracle_heap_item) * (size_t)(m + 1));
    uint8_t* done = (uint8_t*)calloc((size_t)n, 1);
    if (!h || !done) { free(h); free(done); return -1; }
    for (int32_t v = 0; v < n; ++v) dist[v] = ORACLE_INF;
    dist[src] = 0;
    int64_t size = 0;
    heap_push(h, &size, 0, src);
    while (size > 0) {
        const oracle_heap_item it = heap_pop(h, &size);
        if (done[it.v]) continue;
        done[it.v] = 1;
        for (int32_t j = row_ptr[it.v]; j < row_ptr[it.v + 1]; ++j) {
            const int32_t c = col_idx[j];
            const int64_t nd = it.key + (int64_t)w[j];
            if (nd < dist[c]) {
                dist[c] = nd;
                heap_push(h, &size, nd, c);
            }
        }
    }
    for (int32_t v = 0; v < n; ++v)
        if (dist[v] == ORACLE_INF) dist[v] = -1;
    free(h);
    free(done);
    return 0;
}

/*
 * Exactness certificate for non-negative weights.  Returns 1 when
 *   (1) dist[src] = 0 and every entry is >= -1;
 *   (2) for every arc u -> v with dist[u] >= 0: dist[v] >= 0 and
 *       dist[v] <= dist[u] + w (no arc can lower v);
 *   (3) every v with dist[v] >= 0 is reached from src along tight arcs
 *       (dist[u] + w = dist[v]), found by a graph search over them.
 * (3) gives a path of weight dist[v], so dist[v] >= the true distance; (2)
 * along a shortest path gives dist[v] <= it, and closes the reached set
 * under out-arcs.  Zero weights need the search in (3): vertices that only
 * support each other through zero-weight arcs are not reached from src.
 * Returns 0 otherwise, with *bad the first offending vertex.
 */
int oracle_wcertificate(int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const int32_t* w,
                        int32_t src, const int64_t* dist, int32_t* bad) {
    *bad = -1;
    if (n <= 0 || src < 0 || src >= n) return 0;
    if (dist[src] != 0) { *bad = src; return 0; }
    for (int32_t v = 0; v < n; ++v)
        if (dist[v] < -1) { *bad = v; return 0; }
    for (int32_t u = 0; u < n; ++u) {
        if (dist[u] < 0) continue;
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            const int32_t v = col_idx[j];
            if (dist[v] < 0 || dist[v] > dist[u] + (int64_t)w[j]) { *bad = v; return 0; }
        }
    }
    uint8_t* seen = (uint8_t*)calloc((size_t)n, 1);
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!seen || !stack) { free(seen); free(stack); return 0; }
    int64_t top = 0;
    stack[top++] = src;
    seen[src] = 1;
    while (top > 0) {
        const int32_t u = stack[--top];
        for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            const int32_t v = col_idx[j];
            if (!seen[v] && dist[v] == dist[u] + (int64_t)w[j]) {
                seen[v] = 1;
                stack[top++] = v;
            }
        }
    }
    int ok = 1;
    for (int32_t v = 0; v < n && ok; ++v)
        if (dist[v] >= 0 && !seen[v]) { *bad = v; ok = 0; }
    free(seen);
    free(stack);
    return ok;
}
