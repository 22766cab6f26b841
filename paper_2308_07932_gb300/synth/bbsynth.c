/*
 * bbsynth.c - seeded synthetic signed bipartite graph generators.
 *
 * This file produces INPUTS only. It holds none of the counting arithmetic;
 * both the CPU oracle tests and the CUDA path read graphs made here.
 *
 * Determinism across machines (x86-64 here, aarch64 on the GPU hosts):
 *   - the only random source is xoshiro256** (Blackman & Vigna, 2018) seeded
 *     through splitmix64 (Steele, Lea & Flood, 2014), one stream per purpose;
 *   - no libm transcendental is called: bb_log/bb_exp below are written with
 *     + - * / only, and the file is compiled with -ffp-contract=off, so every
 *     double operation is a single IEEE-754 rounding on both machines;
 *   - Bernoulli and alias decisions compare 53-bit integers against integer
 *     thresholds.
 *
 * Output graphs are U-side CSR: rowptr int64[nU+1], col int32[nE] strictly
 * increasing within each row (distinct edges), sign int8[nE] in {+1,-1}.
 * Buffers are malloc'd here and released with synth_free().
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int64_t nU, nV, nE;
    int64_t *rowptr;
    int32_t *col;
    int8_t *sign;
} synth_graph;

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } xo_t;

static uint64_t splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void xo_seed(xo_t *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ull);
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
    if ((r->s[0] | r->s[1] | r->s[2] | r->s[3]) == 0) r->s[0] = 1;
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return result;
}

/* 53-bit integer in [0, 2^53) */
static inline uint64_t xo_u53(xo_t *r) { return xo_next(r) >> 11; }
/* double in [0,1) with 53 random bits (exact conversion) */
static inline double xo_unif(xo_t *r) { return (double)xo_u53(r) * (1.0 / 9007199254740992.0); }

/* unbiased integer in [0, n), Lemire's multiply-shift with rejection */
static inline uint64_t xo_below(xo_t *r, uint64_t n) {
    __uint128_t m = (__uint128_t)xo_next(r) * n;
    uint64_t l = (uint64_t)m;
    if (l < n) {
        uint64_t t = (0 - n) % n;
        while (l < t) { m = (__uint128_t)xo_next(r) * n; l = (uint64_t)m; }
    }
    return (uint64_t)(m >> 64);
}

/* probability p in [0,1] -> threshold on a 53-bit draw */
static inline uint64_t p_threshold(double p) {
    if (p <= 0) return 0;
    if (p >= 1) return (uint64_t)1 << 53;
    return (uint64_t)(p * 9007199254740992.0);
}

/* ------------------------------------------- portable log / exp (own code) */
/* natural log for x > 0: x = m * 2^e with m in [sqrt(1/2), sqrt(2)),
 * log m = 2 atanh(z), z = (m-1)/(m+1), summed as an odd power series. */
static double bb_log(double x) {
    static const double LN2 = 0.69314718055994530942;
    int e = 0;
    double m = x;
    while (m >= 1.4142135623730951) { m *= 0.5; e++; }
    while (m < 0.70710678118654752) { m *= 2.0; e--; }
    double z = (m - 1.0) / (m + 1.0);
    double z2 = z * z, term = z, sum = 0.0;
    for (int k = 1; k < 60; k += 2) { sum += term / (double)k; term *= z2; }
    return 2.0 * sum + (double)e * LN2;
}

/* exp via range reduction y = k ln2 + r, |r| <= ln2/2, Taylor series */
static double bb_exp(double y) {
    static const double LN2 = 0.69314718055994530942;
    if (y > 700) y = 700;
    if (y < -700) return 0.0;
    double kf = y / LN2;
    long k = (long)(kf < 0 ? kf - 0.5 : kf + 0.5);
    double r = y - (double)k * LN2;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 30; i++) { term *= r / (double)i; sum += term; }
    while (k > 0) { sum *= 2.0; k--; }
    while (k < 0) { sum *= 0.5; k++; }
    return sum;
}

/* ------------------------------------------------------------ utilities */
static void radix_sort_u64(uint64_t *a, uint64_t *tmp, int64_t n, uint64_t maxkey) {
    int bits = 0;
    while (bits < 64 && (maxkey >> bits) != 0) bits++;
    uint64_t *src = a, *dst = tmp;
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 65536);
    for (int shift = 0; shift < bits; shift += 16) {
        memset(cnt, 0, sizeof(int64_t) * 65536);
        for (int64_t i = 0; i < n; i++) cnt[(src[i] >> shift) & 0xFFFF]++;
        int64_t s = 0;
        for (int d = 0; d < 65536; d++) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (int64_t i = 0; i < n; i++) dst[cnt[(src[i] >> shift) & 0xFFFF]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(uint64_t) * (size_t)n);
    free(cnt);
}

/* sorted unique pair keys (u*nV+v) -> CSR, signs drawn per edge in order */
static int keys_to_graph(uint64_t *keys, int64_t nk, int64_t nU, int64_t nV,
                         xo_t *rs, uint64_t pos_thr, synth_graph *out) {
    int64_t m = 0;
    for (int64_t i = 0; i < nk; i++)
        if (i == 0 || keys[i] != keys[i - 1]) keys[m++] = keys[i];
    out->nU = nU; out->nV = nV; out->nE = m;
    out->rowptr = (int64_t *)calloc((size_t)nU + 1, sizeof(int64_t));
    out->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    out->sign = (int8_t *)malloc((size_t)(m ? m : 1));
    if (!out->rowptr || !out->col || !out->sign) return -1;
    for (int64_t i = 0; i < m; i++) {
        int64_t u = (int64_t)(keys[i] / (uint64_t)nV);
        out->rowptr[u + 1]++;
        out->col[i] = (int32_t)(keys[i] % (uint64_t)nV);
        out->sign[i] = (int8_t)(xo_u53(rs) < pos_thr ? 1 : -1);
    }
    for (int64_t u = 0; u < nU; u++) out->rowptr[u + 1] += out->rowptr[u];
    return 0;
}

void synth_free(synth_graph *g) {
    if (!g) return;
    free(g->rowptr); free(g->col); free(g->sign);
    g->rowptr = NULL; g->col = NULL; g->sign = NULL;
}

/* ---------------------------------------------- uniform (Floyd sampling) */
/* m distinct (u,v) pairs drawn uniformly without replacement from nU x nV
 * (Floyd's algorithm, one draw per pair), sign +1 with probability p_pos. */
int synth_uniform(uint64_t seed, int64_t nU, int64_t nV, int64_t m, double p_pos,
                  synth_graph *out) {
    memset(out, 0, sizeof(*out));
    if (nU <= 0 || nV <= 0 || m < 0) return -2;
    uint64_t N = (uint64_t)nU * (uint64_t)nV;
    if ((uint64_t)m > N) return -2;
    xo_t re, rs;
    xo_seed(&re, seed, 1);
    xo_seed(&rs, seed, 2);
    uint64_t cap = 16;
    while (cap < 2 * (uint64_t)m + 16) cap <<= 1;
    uint64_t *set = (uint64_t *)malloc(sizeof(uint64_t) * cap);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m ? m : 1));
    if (!set || !keys || !tmp) return -1;
    for (uint64_t i = 0; i < cap; i++) set[i] = ~0ull;
    int64_t k = 0;
    for (uint64_t j = N - (uint64_t)m; j < N; j++) {
        uint64_t t = xo_below(&re, j + 1);
        /* insert t, or j if t already present */
        for (int pass = 0; pass < 2; pass++) {
            uint64_t key = pass == 0 ? t : j;
            uint64_t h = (key * 0x9E3779B97F4A7C15ull) & (cap - 1);
            int found = 0;
            while (set[h] != ~0ull) {
                if (set[h] == key) { found = 1; break; }
                h = (h + 1) & (cap - 1);
            }
            if (!found) { set[h] = key; keys[k++] = key; break; }
        }
    }
    free(set);
    radix_sort_u64(keys, tmp, k, N);
    int rc = keys_to_graph(keys, k, nU, nV, &rs, p_threshold(p_pos), out);
    free(keys); free(tmp);
    return rc;
}

/* ------------------------------------------------------------- Chung-Lu */
typedef struct { uint64_t *thr; int32_t *alias; int64_t n; } alias_t;

/* Vose's alias method over non-negative weights w[0..n) */
static int alias_build(const double *w, int64_t n, alias_t *a) {
    a->n = n;
    a->thr = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    a->alias = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!a->thr || !a->alias || !p || !small || !large) return -1;
    double tot = 0;
    for (int64_t i = 0; i < n; i++) tot += w[i];
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; i++) {
        p[i] = w[i] * (double)n / tot;
        if (p[i] < 1.0) small[ns++] = (int32_t)i; else large[nl++] = (int32_t)i;
    }
    while (ns > 0 && nl > 0) {
        int32_t s = small[--ns], l = large[--nl];
        a->thr[s] = p_threshold(p[s]);
        a->alias[s] = l;
        p[l] = (p[l] + p[s]) - 1.0;
        if (p[l] < 1.0) small[ns++] = l; else large[nl++] = l;
    }
    while (nl > 0) { int32_t l = large[--nl]; a->thr[l] = (uint64_t)1 << 53; a->alias[l] = l; }
    while (ns > 0) { int32_t s = small[--ns]; a->thr[s] = (uint64_t)1 << 53; a->alias[s] = s; }
    free(p); free(small); free(large);
    return 0;
}

static inline int64_t alias_draw(const alias_t *a, xo_t *r) {
    int64_t i = (int64_t)xo_below(r, (uint64_t)a->n);
    return xo_u53(r) < a->thr[i] ? i : a->alias[i];
}

static void alias_free(alias_t *a) { free(a->thr); free(a->alias); }

/* expected degrees: Pareto(x_min = 1) weights with density ~ x^-alpha,
 * scaled so they sum to m_draw, then clipped at cap_deg */
static double *pareto_degrees(xo_t *r, int64_t n, double alpha, int64_t m_draw, double cap_deg) {
    double *w = (double *)malloc(sizeof(double) * (size_t)n);
    if (!w) return NULL;
    double inv = -1.0 / (alpha - 1.0), tot = 0;
    for (int64_t i = 0; i < n; i++) {
        double one_minus_u = 1.0 - xo_unif(r); /* in (0,1] */
        w[i] = bb_exp(inv * bb_log(one_minus_u));
        tot += w[i];
    }
    double scale = (double)m_draw / tot;
    for (int64_t i = 0; i < n; i++) {
        double d = w[i] * scale;
        w[i] = d > cap_deg ? cap_deg : d;
    }
    return w;
}

/* Chung-Lu bipartite graph: m_draw endpoint pairs, u drawn with probability
 * proportional to its expected degree on U and v likewise on V, duplicates
 * removed; sign +1 with probability p_pos. */
int synth_chung_lu(uint64_t seed, int64_t nU, int64_t nV, int64_t m_draw,
                   double alphaU, double alphaV, double cap_deg, double p_pos,
                   synth_graph *out) {
    memset(out, 0, sizeof(*out));
    if (nU <= 0 || nV <= 0 || m_draw < 0 || alphaU <= 1 || alphaV <= 1) return -2;
    if (nU >= 0x7FFFFFFF || nV >= 0x7FFFFFFF) return -2;
    xo_t rwu, rwv, rp, rs;
    xo_seed(&rwu, seed, 11);
    xo_seed(&rwv, seed, 12);
    xo_seed(&rp, seed, 13);
    xo_seed(&rs, seed, 14);
    double capU = cap_deg < (double)nV ? cap_deg : (double)nV;
    double capV = cap_deg < (double)nU ? cap_deg : (double)nU;
    double *dU = pareto_degrees(&rwu, nU, alphaU, m_draw, capU);
    double *dV = pareto_degrees(&rwv, nV, alphaV, m_draw, capV);
    if (!dU || !dV) return -1;
    alias_t aU, aV;
    if (alias_build(dU, nU, &aU) || alias_build(dV, nV, &aV)) return -1;
    free(dU); free(dV);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m_draw ? m_draw : 1));
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(m_draw ? m_draw : 1));
    if (!keys || !tmp) return -1;
    for (int64_t i = 0; i < m_draw; i++) {
        int64_t u = alias_draw(&aU, &rp);
        int64_t v = alias_draw(&aV, &rp);
        keys[i] = (uint64_t)u * (uint64_t)nV + (uint64_t)v;
    }
    alias_free(&aU); alias_free(&aV);
    radix_sort_u64(keys, tmp, m_draw, (uint64_t)nU * (uint64_t)nV);
    free(tmp);
    int rc = keys_to_graph(keys, m_draw, nU, nV, &rs, p_threshold(p_pos), out);
    free(keys);
    return rc;
}

/* ----------------------------------------------------------- vote-like */
/* Every (u,v) present independently with probability p_edge. U is split
 * into n_blocks contiguous blocks; each (v, block) draws a stance (+1 with
 * probability p_stance); an edge copies its block's stance with probability
 * agree, else draws its own sign (+1 with probability p_stance). */
int synth_vote(uint64_t seed, int64_t nU, int64_t nV, double p_edge, int64_t n_blocks,
               double p_stance, double agree, synth_graph *out) {
    memset(out, 0, sizeof(*out));
    if (nU <= 0 || nV <= 0 || n_blocks <= 0 || n_blocks > nU) return -2;
    xo_t re, rt, rs;
    xo_seed(&re, seed, 21);
    xo_seed(&rt, seed, 22);
    xo_seed(&rs, seed, 23);
    uint64_t te = p_threshold(p_edge), tst = p_threshold(p_stance), tag = p_threshold(agree);
    int8_t *stance = (int8_t *)malloc((size_t)(nV * n_blocks));
    if (!stance) return -1;
    for (int64_t v = 0; v < nV; v++)
        for (int64_t b = 0; b < n_blocks; b++)
            stance[v * n_blocks + b] = (int8_t)(xo_u53(&rt) < tst ? 1 : -1);
    int64_t cap = (int64_t)((double)nU * (double)nV * p_edge * 1.1) + 1024;
    out->nU = nU; out->nV = nV;
    out->rowptr = (int64_t *)calloc((size_t)nU + 1, sizeof(int64_t));
    out->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    out->sign = (int8_t *)malloc((size_t)cap);
    if (!out->rowptr || !out->col || !out->sign) return -1;
    int64_t m = 0;
    for (int64_t u = 0; u < nU; u++) {
        int64_t b = u * n_blocks / nU;
        for (int64_t v = 0; v < nV; v++) {
            if (xo_u53(&re) >= te) continue;
            if (m == cap) {
                cap = cap * 2;
                out->col = (int32_t *)realloc(out->col, sizeof(int32_t) * (size_t)cap);
                out->sign = (int8_t *)realloc(out->sign, (size_t)cap);
                if (!out->col || !out->sign) return -1;
            }
            out->col[m] = (int32_t)v;
            if (xo_u53(&rs) < tag) out->sign[m] = stance[v * n_blocks + b];
            else out->sign[m] = (int8_t)(xo_u53(&rs) < tst ? 1 : -1);
            m++;
        }
        out->rowptr[u + 1] = m;
    }
    out->nE = m;
    free(stance);
    return 0;
}

/* -------------------------------------------- parameter draws for mixes */
/* one log-uniform draw in [lo, hi] from stream `stream` of `seed` */
double synth_log_uniform(uint64_t seed, uint64_t stream, double lo, double hi) {
    xo_t r;
    xo_seed(&r, seed, stream);
    double a = bb_log(lo), b = bb_log(hi);
    return bb_exp(a + (b - a) * xo_unif(&r));
}

/* one uniform draw in [lo, hi) from stream `stream` of `seed` */
double synth_uniform_real(uint64_t seed, uint64_t stream, double lo, double hi) {
    xo_t r;
    xo_seed(&r, seed, stream);
    return lo + (hi - lo) * xo_unif(&r);
}

/* n uniform integers in [0, bound) (e.g. edge indices to flip) */
void synth_uniform_ints(uint64_t seed, uint64_t stream, int64_t n, int64_t bound, int64_t *out) {
    xo_t r;
    xo_seed(&r, seed, stream);
    for (int64_t i = 0; i < n; i++) out[i] = (int64_t)xo_below(&r, (uint64_t)bound);
}

/* n exponential inter-arrival gaps with rate lambda (seconds) */
void synth_exponential(uint64_t seed, uint64_t stream, int64_t n, double lambda, double *out) {
    xo_t r;
    xo_seed(&r, seed, stream);
    for (int64_t i = 0; i < n; i++) out[i] = -bb_log(1.0 - xo_unif(&r)) / lambda;
}
