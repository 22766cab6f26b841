/*
 * bb_oracle.c - the CPU oracle for balanced butterfly counting.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may call, link or
 * load this file; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg do. It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper, Section "Problem Definition"):
 *   Def. 1  a butterfly is a 4-cycle u_i - v_i - u_j - v_j (a 2x2 biclique);
 *   Def. 2  it is balanced when it holds an even number of negative edges,
 *           i.e. the product of its four edge signs is +1.
 *   balanced = number of balanced butterflies, total = number of butterflies.
 *
 * How (plain, slow, no degree priority): a butterfly is fixed by one pair of
 * vertices {s1, s2} on one side S plus a pair {m1, m2} of their common
 * neighbours. Its sign product is [s(s1,m1) s(s2,m1)] * [s(s1,m2) s(s2,m2)],
 * so it is balanced exactly when both common neighbours have the same
 * product. With P = #common neighbours of product +1 and N = #of product -1,
 * the pair {s1,s2} holds C(P+N,2) butterflies of which C(P,2)+C(N,2) are
 * balanced. The oracle enumerates, for every s1, each s2 > s1 reachable in
 * two hops, tallies P and N, and adds those binomials. Sums are kept in
 * unsigned 128-bit integers and reported as int64 (error if they overflow).
 *
 * Per-edge counts (the paper's edge-level extension, eBBFC) are taken from
 * the definition: for each edge, every butterfly through it is enumerated
 * by its other U vertex and its other V vertex and tested with Def. 2.
 *
 * Per-vertex counts follow Algorithm 3 (vBBFC, Section "Extensions"): for a
 * vertex x, walk x - v - w for every v in N(x) and w in N(v) with w != x
 * (reading: the paper's listing has no w != x test, but the wedge x-v-x is
 * not part of any butterfly), bucket each wedge by whether its two signs are
 * equal, and add C(B1[w],2) + C(B2[w],2).
 *
 * BB-Base (Algorithm 1, Section "Baseline Approach") is kept as a second,
 * independent enumeration: degree priority (Def. 4), per start u the lists
 * H(w) of middle vertices, and an explicit sign-product test on every pair.
 *
 * Threads only split the outer loop over start vertices; each thread owns
 * its counters and results are summed as exact integers, so the answer does
 * not depend on the thread count.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_EOVERFLOW = -3 };

/* C(n,2) */
static inline u128 c2(uint64_t n) { return n < 2 ? 0 : ((u128)n * (u128)(n - 1)) / 2; }

/* ------------------------------------------------------------ graph view */
/* Both adjacency directions of the input, ids local to each side, each list
 * sorted by id ascending, with the edge sign next to each neighbour. */
typedef struct {
    int64_t n[2];          /* n[0] = |U|, n[1] = |V| */
    int64_t *off[2];       /* off[side][x] .. off[side][x+1] */
    int32_t *nbr[2];       /* neighbour id on the other side */
    int8_t *sgn[2];        /* sign of that edge */
} view_t;

static void view_free(view_t *g) {
    for (int s = 0; s < 2; s++) { free(g->off[s]); free(g->nbr[s]); free(g->sgn[s]); }
}

/* validates the CSR and builds both directions; rows must hold distinct
 * ids (E is a set, Section "Problem Definition") */
static int view_build(int64_t nU, int64_t nV, const int64_t *rowptr, const int32_t *col,
                      const int8_t *sign, view_t *g) {
    memset(g, 0, sizeof(*g));
    if (nU < 0 || nV < 0 || !rowptr) return OR_EINVAL;
    int64_t nE = rowptr[nU];
    if (rowptr[0] != 0 || nE < 0) return OR_EINVAL;
    g->n[0] = nU; g->n[1] = nV;
    g->off[0] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nU + 1));
    g->off[1] = (int64_t *)calloc((size_t)nV + 1, sizeof(int64_t));
    for (int s = 0; s < 2; s++) {
        g->nbr[s] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nE ? nE : 1));
        g->sgn[s] = (int8_t *)malloc((size_t)(nE ? nE : 1));
    }
    if (!g->off[0] || !g->off[1] || !g->nbr[0] || !g->nbr[1] || !g->sgn[0] || !g->sgn[1]) {
        view_free(g); return OR_ENOMEM;
    }
    /* U side: copy the rows, then sort each row by id with a bottom-up
     * merge sort through a scratch buffer (input rows may be unsorted) */
    for (int64_t u = 0; u <= nU; u++) g->off[0][u] = rowptr[u];
    for (int64_t u = 0; u < nU; u++) {
        if (rowptr[u + 1] < rowptr[u]) { view_free(g); return OR_EINVAL; }
    }
    for (int64_t e = 0; e < nE; e++) {
        if (col[e] < 0 || col[e] >= nV || (sign[e] != 1 && sign[e] != -1)) { view_free(g); return OR_EINVAL; }
        g->nbr[0][e] = col[e];
        g->sgn[0][e] = sign[e];
    }
    int32_t *tn = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nE ? nE : 1));
    int8_t *ts = (int8_t *)malloc((size_t)(nE ? nE : 1));
    if (!tn || !ts) { free(tn); free(ts); view_free(g); return OR_ENOMEM; }
    for (int64_t u = 0; u < nU; u++) {
        int64_t a = rowptr[u], b = rowptr[u + 1];
        /* bottom-up merge sort of nbr[0][a..b) carrying signs */
        for (int64_t w = 1; w < b - a; w *= 2) {
            for (int64_t lo = a; lo < b; lo += 2 * w) {
                int64_t mid = lo + w < b ? lo + w : b, hi = lo + 2 * w < b ? lo + 2 * w : b;
                int64_t i = lo, j = mid, k = lo;
                while (i < mid && j < hi) {
                    if (g->nbr[0][i] <= g->nbr[0][j]) { tn[k] = g->nbr[0][i]; ts[k++] = g->sgn[0][i++]; }
                    else { tn[k] = g->nbr[0][j]; ts[k++] = g->sgn[0][j++]; }
                }
                while (i < mid) { tn[k] = g->nbr[0][i]; ts[k++] = g->sgn[0][i++]; }
                while (j < hi) { tn[k] = g->nbr[0][j]; ts[k++] = g->sgn[0][j++]; }
                for (k = lo; k < hi; k++) { g->nbr[0][k] = tn[k]; g->sgn[0][k] = ts[k]; }
            }
        }
        for (int64_t e = a + 1; e < b; e++)
            if (g->nbr[0][e] == g->nbr[0][e - 1]) { free(tn); free(ts); view_free(g); return OR_EINVAL; }
    }
    free(tn); free(ts);
    /* V side: counting sort by v; scanning u in increasing order keeps each
     * V row sorted by u */
    for (int64_t e = 0; e < nE; e++) g->off[1][g->nbr[0][e] + 1]++;
    for (int64_t v = 0; v < nV; v++) g->off[1][v + 1] += g->off[1][v];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nV ? nV : 1));
    if (!cur) { view_free(g); return OR_ENOMEM; }
    for (int64_t v = 0; v < nV; v++) cur[v] = g->off[1][v];
    for (int64_t u = 0; u < nU; u++)
        for (int64_t e = g->off[0][u]; e < g->off[0][u + 1]; e++) {
            int64_t p = cur[g->nbr[0][e]]++;
            g->nbr[1][p] = (int32_t)u;
            g->sgn[1][p] = g->sgn[0][e];
        }
    free(cur);
    return OR_OK;
}

/* ------------------------------------------------ pair-enumeration count */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0   /* tests build planted-mistake variants with 1..7 */
#endif

typedef struct {
    const view_t *g;
    int S;                       /* endpoint side */
    const int64_t *starts;       /* list of s1 to process (NULL = all) */
    int64_t nstarts;
    int64_t next;                /* shared work cursor */
    pthread_mutex_t mu;
    u128 bal, tot;
    uint64_t steps;
} count_job_t;

static void *count_worker(void *arg) {
    count_job_t *J = (count_job_t *)arg;
    const view_t *g = J->g;
    int S = J->S, M = 1 - S;
    int64_t nS = g->n[S];
    uint32_t *P = (uint32_t *)calloc((size_t)(nS ? nS : 1), sizeof(uint32_t));
    uint32_t *N = (uint32_t *)calloc((size_t)(nS ? nS : 1), sizeof(uint32_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nS ? nS : 1));
    u128 bal = 0, tot = 0;
    uint64_t steps = 0;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i0 = J->next, i1 = i0 + 64 < J->nstarts ? i0 + 64 : J->nstarts;
        J->next = i1;
        pthread_mutex_unlock(&J->mu);
        if (i0 >= J->nstarts) break;
        for (int64_t i = i0; i < i1; i++) {
            int64_t s1 = J->starts ? J->starts[i] : i;
            int64_t nt = 0;
            for (int64_t e = g->off[S][s1]; e < g->off[S][s1 + 1]; e++) {
                int32_t m = g->nbr[S][e];
                int8_t a = g->sgn[S][e];
                /* N(m) is sorted by id: walk down from its end while s2 > s1 */
                for (int64_t f = g->off[M][m + 1] - 1; f >= g->off[M][m]; f--) {
                    int32_t s2 = g->nbr[M][f];
#if ORACLE_MUTANT == 3
                    if (s2 < s1) break;           /* planted: keeps s2 == s1 */
#else
                    if (s2 <= s1) break;
#endif
                    steps++;
                    if (P[s2] == 0 && N[s2] == 0) touched[nt++] = s2;
#if ORACLE_MUTANT == 2
                    if (a == 1) P[s2]++;          /* planted: ignores the second sign */
#else
                    if (a * g->sgn[M][f] == 1) P[s2]++;
#endif
                    else N[s2]++;
                }
            }
            for (int64_t t = 0; t < nt; t++) {
                int32_t s2 = touched[t];
#if ORACLE_MUTANT == 1
                bal += c2(P[s2]);                 /* planted: drops the C(N,2) term */
#elif ORACLE_MUTANT == 4
                bal += c2(P[s2]) + c2(N[s2]) + (P[s2] > 0 && N[s2] > 0 ? 1 : 0); /* planted: off by one */
#else
                bal += c2(P[s2]) + c2(N[s2]);
#endif
#if ORACLE_MUTANT == 5
                tot += c2(P[s2]) + c2(N[s2]);     /* planted: total counts balanced only */
#else
                tot += c2((uint64_t)P[s2] + N[s2]);
#endif
                P[s2] = 0; N[s2] = 0;
            }
        }
    }
    free(P); free(N); free(touched);
    pthread_mutex_lock(&J->mu);
    J->bal += bal; J->tot += tot; J->steps += steps;
    pthread_mutex_unlock(&J->mu);
    return NULL;
}

static int run_threads(void *(*fn)(void *), void *job, int threads) {
    if (threads < 1) threads = 1;
    if (threads == 1) { fn(job); return OR_OK; }
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    if (!th) return OR_ENOMEM;
    int started = 0;
    for (int t = 0; t < threads; t++)
        if (pthread_create(&th[t], NULL, fn, job) == 0) started++; else break;
    for (int t = 0; t < started; t++) pthread_join(th[t], NULL);
    free(th);
    if (started == 0) fn(job);
    return OR_OK;
}

static int store_i64(u128 x, int64_t *out) {
    if (x > (u128)INT64_MAX) return OR_EOVERFLOW;
    *out = (int64_t)x;
    return OR_OK;
}

/* wedges walked when side S holds the endpoints: sum over the other side of C(deg,2) */
static u128 pair_steps(const view_t *g, int S) {
    int M = 1 - S;
    u128 s = 0;
    for (int64_t m = 0; m < g->n[M]; m++) s += c2((uint64_t)(g->off[M][m + 1] - g->off[M][m]));
    return s;
}

/* Full count. side: 0 = endpoints in U, 1 = endpoints in V, -1 = the side
 * with fewer two-hop steps. */
int oracle_count(int64_t nU, int64_t nV, const int64_t *rowptr, const int32_t *col,
                 const int8_t *sign, int side, int threads, int64_t *balanced, int64_t *total) {
    view_t g;
    int rc = view_build(nU, nV, rowptr, col, sign, &g);
    if (rc) return rc;
    int S = side;
    if (S < 0) S = pair_steps(&g, 1) <= pair_steps(&g, 0) ? 1 : 0;
    count_job_t J;
    memset(&J, 0, sizeof(J));
    J.g = &g; J.S = S; J.nstarts = g.n[S];
    pthread_mutex_init(&J.mu, NULL);
    rc = run_threads(count_worker, &J, threads);
    pthread_mutex_destroy(&J.mu);
    view_free(&g);
    if (rc) return rc;
    if ((rc = store_i64(J.bal, balanced))) return rc;
    return store_i64(J.tot, total);
}

/* Partial count over a list of s1 on side `side` (0/1): the contribution of
 * the pairs {s1, s2 > s1}. Also reports the two-hop steps it walked and the
 * steps the full count would walk. Used for the timed CPU baseline on a
 * bounded sample. */
int oracle_count_sample(int64_t nU, int64_t nV, const int64_t *rowptr, const int32_t *col,
                        const int8_t *sign, int side, const int64_t *starts, int64_t nstarts,
                        int threads, int64_t *balanced, int64_t *total, int64_t *steps,
                        int64_t *full_steps) {
    view_t g;
    int rc = view_build(nU, nV, rowptr, col, sign, &g);
    if (rc) return rc;
    int S = side < 0 ? (pair_steps(&g, 1) <= pair_steps(&g, 0) ? 1 : 0) : side;
    for (int64_t i = 0; i < nstarts; i++)
        if (starts[i] < 0 || starts[i] >= g.n[S]) { view_free(&g); return OR_EINVAL; }
    count_job_t J;
    memset(&J, 0, sizeof(J));
    J.g = &g; J.S = S; J.starts = starts; J.nstarts = nstarts;
    pthread_mutex_init(&J.mu, NULL);
    rc = run_threads(count_worker, &J, threads);
    pthread_mutex_destroy(&J.mu);
    u128 fs = pair_steps(&g, S);
    view_free(&g);
    if (rc) return rc;
    if ((rc = store_i64(J.bal, balanced))) return rc;
    if ((rc = store_i64(J.tot, total))) return rc;
    if ((rc = store_i64(J.steps, steps))) return rc;
    return store_i64(fs, full_steps);
}

/* --------------------------------------------- per-vertex (Algorithm 3) */
typedef struct {
    const view_t *g;
    const int64_t *gids;   /* vertices to evaluate, gid = u or nU + v */
    int64_t n;
    int64_t *out;
    int64_t next;
    pthread_mutex_t mu;
    int err;
} pv_job_t;

static void *pv_worker(void *arg) {
    pv_job_t *J = (pv_job_t *)arg;
    const view_t *g = J->g;
    int64_t nmax = g->n[0] > g->n[1] ? g->n[0] : g->n[1];
    uint32_t *H1 = (uint32_t *)calloc((size_t)(nmax ? nmax : 1), sizeof(uint32_t));
    uint32_t *H2 = (uint32_t *)calloc((size_t)(nmax ? nmax : 1), sizeof(uint32_t));
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax ? nmax : 1));
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (i >= J->n) break;
        int64_t x = J->gids[i];
        int S = x < g->n[0] ? 0 : 1, M = 1 - S;
        if (S == 1) x -= g->n[0];
        int64_t nt = 0;
        for (int64_t e = g->off[S][x]; e < g->off[S][x + 1]; e++) {
            int32_t v = g->nbr[S][e];
            int8_t a = g->sgn[S][e];
            for (int64_t f = g->off[M][v]; f < g->off[M][v + 1]; f++) {
                int32_t w = g->nbr[M][f];
                if (w == x) continue;
                if (H1[w] == 0 && H2[w] == 0) touched[nt++] = w;
                if (a == g->sgn[M][f]) H1[w]++; else H2[w]++;
            }
        }
        u128 b = 0;
        for (int64_t t = 0; t < nt; t++) {
            int32_t w = touched[t];
            b += c2(H1[w]) + c2(H2[w]);
            H1[w] = 0; H2[w] = 0;
        }
        if (b > (u128)INT64_MAX) { J->err = OR_EOVERFLOW; b = 0; }
        J->out[i] = (int64_t)b;
    }
    free(H1); free(H2); free(touched);
    return NULL;
}

/* Balanced butterflies containing each listed vertex (gid: u for U, nU+v
 * for V). gids == NULL means every vertex in gid order; out has n entries. */
int oracle_per_vertex(int64_t nU, int64_t nV, const int64_t *rowptr, const int32_t *col,
                      const int8_t *sign, const int64_t *gids, int64_t n, int threads,
                      int64_t *out) {
    view_t g;
    int rc = view_build(nU, nV, rowptr, col, sign, &g);
    if (rc) return rc;
    int64_t *all = NULL;
    if (!gids) {
        n = nU + nV;
        all = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
        if (!all) { view_free(&g); return OR_ENOMEM; }
        for (int64_t i = 0; i < n; i++) all[i] = i;
        gids = all;
    }
    for (int64_t i = 0; i < n; i++)
        if (gids[i] < 0 || gids[i] >= nU + nV) { free(all); view_free(&g); return OR_EINVAL; }
    pv_job_t J;
    memset(&J, 0, sizeof(J));
    J.g = &g; J.gids = gids; J.n = n; J.out = out;
    pthread_mutex_init(&J.mu, NULL);
    rc = run_threads(pv_worker, &J, threads);
    pthread_mutex_destroy(&J.mu);
    free(all);
    view_free(&g);
    return rc ? rc : J.err;
}

/* ----------------------------------------------------------- per edge */
/* Balanced butterflies containing one edge (the quantity of the paper's
 * edge-level extension, eBBFC, Section "Extensions"), from the definition:
 * for edge (u1, v1) every butterfly through it is fixed by a second U vertex
 * u2 in N(v1) \ {u1} and a second V vertex v2 in N(u1) ∩ N(u2) \ {v1}; it is
 * balanced when s(u1,v1) s(u1,v2) s(u2,v1) s(u2,v2) = +1 (Def. 2). N(u1) is
 * marked with its signs in a dense array over V, then every two-hop path
 * v1 - u2 - v2 is tested against the marks. */
typedef struct {
    const view_t *g;
    const int64_t *rowptr;
    const int32_t *col;
    const int8_t *sign;
    const int64_t *edges;  /* edge ids (positions in the input CSR) */
    int64_t n;
    int64_t *out;
    int64_t next;
    pthread_mutex_t mu;
    int err;
} pe_job_t;

static void *pe_worker(void *arg) {
    pe_job_t *J = (pe_job_t *)arg;
    const view_t *g = J->g;
    const int64_t nU = g->n[0];
    int8_t *mark = (int8_t *)calloc((size_t)(g->n[1] ? g->n[1] : 1), 1);
    if (!mark) { J->err = OR_ENOMEM; return NULL; }
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (i >= J->n) break;
        const int64_t e = J->edges[i];
        /* the row of edge e: last u with rowptr[u] <= e */
        int64_t lo = 0, hi = nU;
        while (hi - lo > 1) {
            int64_t m = (lo + hi) / 2;
            if (J->rowptr[m] <= e) lo = m; else hi = m;
        }
        const int64_t u1 = lo;
        const int32_t v1 = J->col[e];
        const int s11 = J->sign[e];
        for (int64_t f = g->off[0][u1]; f < g->off[0][u1 + 1]; f++) mark[g->nbr[0][f]] = g->sgn[0][f];
        u128 b = 0;
        for (int64_t f = g->off[1][v1]; f < g->off[1][v1 + 1]; f++) {
            const int32_t u2 = g->nbr[1][f];
#if ORACLE_MUTANT != 6
            if (u2 == u1) continue;
#endif
            const int s21 = g->sgn[1][f];
            for (int64_t h = g->off[0][u2]; h < g->off[0][u2 + 1]; h++) {
                const int32_t v2 = g->nbr[0][h];
                if (v2 == v1 || mark[v2] == 0) continue;
                const int s12 = mark[v2], s22 = g->sgn[0][h];
#if ORACLE_MUTANT == 7
                if (s11 * s12 * s21 == 1) b++;
#else
                if (s11 * s12 * s21 * s22 == 1) b++;
#endif
            }
        }
        for (int64_t f = g->off[0][u1]; f < g->off[0][u1 + 1]; f++) mark[g->nbr[0][f]] = 0;
        if (b > (u128)INT64_MAX) { J->err = OR_EOVERFLOW; b = 0; }
        J->out[i] = (int64_t)b;
    }
    free(mark);
    return NULL;
}

/* Balanced butterflies containing each listed edge (positions in the input
 * CSR); edges == NULL means every edge in input order; out has n entries. */
int oracle_per_edge(int64_t nU, int64_t nV, const int64_t *rowptr, const int32_t *col,
                    const int8_t *sign, const int64_t *edges, int64_t n, int threads,
                    int64_t *out) {
    view_t g;
    int rc = view_build(nU, nV, rowptr, col, sign, &g);
    if (rc) return rc;
    const int64_t nE = rowptr[nU];
    int64_t *all = NULL;
    if (!edges) {
        n = nE;
        all = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
        if (!all) { view_free(&g); return OR_ENOMEM; }
        for (int64_t i = 0; i < n; i++) all[i] = i;
        edges = all;
    }
    for (int64_t i = 0; i < n; i++)
        if (edges[i] < 0 || edges[i] >= nE) { free(all); view_free(&g); return OR_EINVAL; }
    pe_job_t J;
    memset(&J, 0, sizeof(J));
    J.g = &g; J.rowptr = rowptr; J.col = col; J.sign = sign;
    J.edges = edges; J.n = n; J.out = out;
    pthread_mutex_init(&J.mu, NULL);
    rc = run_threads(pe_worker, &J, threads);
    pthread_mutex_destroy(&J.mu);
    free(all);
    view_free(&g);
    return rc ? rc : J.err;
}

/* ------------------------------------------------ BB-Base (Algorithm 1) */
/* Degree priority (Def. 4): p(a) > p(b) iff deg(a) > deg(b), or equal
 * degrees and id(a) > id(b); ids are compared in one namespace with
 * gid = u for U and |U| + v for V (the paper does not fix it; any strict
 * total order gives the same count). */
int oracle_bb_base(int64_t nU, int64_t nV, const int64_t *rowptr, const int32_t *col,
                   const int8_t *sign, int64_t *balanced, int64_t *total) {
    view_t g;
    int rc = view_build(nU, nV, rowptr, col, sign, &g);
    if (rc) return rc;
    int64_t n = nU + nV;
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t *hcnt = (int64_t *)calloc((size_t)(n ? n : 1), sizeof(int64_t));
    int64_t *hoff = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg || !hcnt || !hoff) { free(deg); free(hcnt); free(hoff); view_free(&g); return OR_ENOMEM; }
    for (int64_t x = 0; x < n; x++) {
        int S = x < nU ? 0 : 1;
        int64_t l = S ? x - nU : x;
        deg[x] = g.off[S][l + 1] - g.off[S][l];
    }
#define PRI_LT(a, b) (deg[a] < deg[b] || (deg[a] == deg[b] && (a) < (b)))
    /* H(w) holds (middle gid, sign(u,v), sign(v,w)) triples for one start u */
    int64_t hcap = 1024, hn = 0;
    int64_t *hw = (int64_t *)malloc(sizeof(int64_t) * (size_t)hcap);
    int64_t *hv = (int64_t *)malloc(sizeof(int64_t) * (size_t)hcap);
    int8_t *hs1 = (int8_t *)malloc((size_t)hcap);
    int8_t *hs2 = (int8_t *)malloc((size_t)hcap);
    int64_t *order = NULL;
    u128 bal = 0, tot = 0;
    for (int64_t u = 0; u < n && hw; u++) {
        int S = u < nU ? 0 : 1, M = 1 - S;
        int64_t ul = S ? u - nU : u;
        hn = 0;
        for (int64_t e = g.off[S][ul]; e < g.off[S][ul + 1]; e++) {
            int64_t vl = g.nbr[S][e], v = M ? nU + vl : vl;
            if (!PRI_LT(v, u)) continue;
            for (int64_t f = g.off[M][vl]; f < g.off[M][vl + 1]; f++) {
                int64_t wl = g.nbr[M][f], w = S ? nU + wl : wl;
                if (!PRI_LT(w, u)) continue;
                if (hn == hcap) {
                    hcap *= 2;
                    hw = (int64_t *)realloc(hw, sizeof(int64_t) * (size_t)hcap);
                    hv = (int64_t *)realloc(hv, sizeof(int64_t) * (size_t)hcap);
                    hs1 = (int8_t *)realloc(hs1, (size_t)hcap);
                    hs2 = (int8_t *)realloc(hs2, (size_t)hcap);
                    if (!hw || !hv || !hs1 || !hs2) { rc = OR_ENOMEM; goto done; }
                }
                hw[hn] = w; hv[hn] = v; hs1[hn] = g.sgn[S][e]; hs2[hn] = g.sgn[M][f]; hn++;
            }
        }
        /* group the wedges by end vertex w: count per w, give each w a
         * block in order of first appearance, place indices, reset */
        free(order);
        order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(hn ? hn : 1));
        if (!order) { rc = OR_ENOMEM; goto done; }
        for (int64_t i = 0; i < hn; i++) hcnt[hw[i]]++;
        {
            int64_t pos = 0;
            for (int64_t i = 0; i < hn; i++) {
                int64_t w = hw[i];
                if (hcnt[w] > 0) { hoff[w] = pos; pos += hcnt[w]; hcnt[w] = -1; }
            }
        }
        for (int64_t i = 0; i < hn; i++) order[hoff[hw[i]]++] = i;
        for (int64_t i = 0; i < hn; i++) { hcnt[hw[i]] = 0; hoff[hw[i]] = 0; }
        /* every pair of wedges in one H(w) group closes one butterfly
         * u - v1 - w - v2; test its four signs explicitly */
        for (int64_t a = 0; a < hn;) {
            int64_t w = hw[order[a]], b = a;
            while (b < hn && hw[order[b]] == w) b++;
            for (int64_t i = a; i < b; i++)
                for (int64_t j = i + 1; j < b; j++) {
                    int64_t x = order[i], y = order[j];
                    int prod = hs1[x] * hs2[x] * hs1[y] * hs2[y];
                    tot += 1;
                    if (prod == 1) bal += 1;
                }
            a = b;
        }
    }
done:
#undef PRI_LT
    free(order); free(hw); free(hv); free(hs1); free(hs2);
    free(deg); free(hcnt); free(hoff);
    view_free(&g);
    if (rc) return rc;
    if ((rc = store_i64(bal, balanced))) return rc;
    return store_i64(tot, total);
}

/* Every butterfly by brute force over all vertex 4-tuples on a dense sign
 * matrix (|U|, |V| small): definition 1-2 written out directly. */
int oracle_brute(int64_t nU, int64_t nV, const int64_t *rowptr, const int32_t *col,
                 const int8_t *sign, int64_t *balanced, int64_t *total, int64_t *per_vertex) {
    if (nU < 0 || nV < 0 || nU > 4096 || nV > 4096) return OR_EINVAL;
    int8_t *A = (int8_t *)calloc((size_t)(nU * nV > 0 ? nU * nV : 1), 1);
    if (!A) return OR_ENOMEM;
    for (int64_t u = 0; u < nU; u++)
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++) {
            if (col[e] < 0 || col[e] >= nV || (sign[e] != 1 && sign[e] != -1) || A[u * nV + col[e]]) {
                free(A); return OR_EINVAL;
            }
            A[u * nV + col[e]] = sign[e];
        }
    if (per_vertex) memset(per_vertex, 0, sizeof(int64_t) * (size_t)(nU + nV));
    u128 bal = 0, tot = 0;
    for (int64_t u1 = 0; u1 < nU; u1++)
        for (int64_t u2 = u1 + 1; u2 < nU; u2++)
            for (int64_t v1 = 0; v1 < nV; v1++) {
                int a1 = A[u1 * nV + v1], a2 = A[u2 * nV + v1];
                if (!a1 || !a2) continue;
                for (int64_t v2 = v1 + 1; v2 < nV; v2++) {
                    int b1 = A[u1 * nV + v2], b2 = A[u2 * nV + v2];
                    if (!b1 || !b2) continue;
                    tot++;
                    if (a1 * a2 * b1 * b2 == 1) {
                        bal++;
                        if (per_vertex) {
                            per_vertex[u1]++; per_vertex[u2]++;
                            per_vertex[nU + v1]++; per_vertex[nU + v2]++;
                        }
                    }
                }
            }
    free(A);
    int rc;
    if ((rc = store_i64(bal, balanced))) return rc;
    return store_i64(tot, total);
}
