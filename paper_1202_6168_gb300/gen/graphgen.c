/*
 * graphgen.c - seeded synthetic directed graphs shaped like the web-graph
 * prefixes the paper evaluates on (Sec. 3, Table 1: power-law out-degrees,
 * a few percent dangling nodes, strong locality of links).
 *
 * This file holds input generation only: no step of the D-iteration method.
 * Both the CPU oracle and the CUDA path consume its output (a CSR of
 * out-edges), and neither shares any other code.
 *
 * Recipe, for every source node j (all draws come from a per-node
 * xoshiro256** stream seeded by SplitMix64 from (seed, j), so the graph is
 * reproducible and rows can be generated in parallel):
 *   - j is dangling (no out-edge) with probability p_dangling;
 *   - otherwise k ~ Zipf(zipf_exp) on [1, zipf_max] and
 *     outdeg_j = clamp(round(k * mean_deg / E[k]), 1, N-1), so the mean over
 *     non-dangling nodes is mean_deg before deduplication;
 *   - each edge target is uniform in [j-window, j+window] mod N with
 *     probability p_local; otherwise it is perm(r) with r drawn from the
 *     continuous law of density proportional to (x+1)^-rank_exp on [0, N),
 *     by inverse CDF, floored; perm is a seeded random permutation;
 *   - self-loops are dropped and duplicate targets merged (a row left empty
 *     makes j dangling); each row is sorted by target.
 *
 * Determinism across machines: only integer arithmetic and correctly
 * rounded IEEE +, -, *, / are used (no libm transcendental call; the
 * power function below is a short series evaluated in a fixed order), and
 * the build passes -ffp-contract=off so no FMA contraction changes a
 * rounding. x86-64 and aarch64 therefore produce the same bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------- random numbers (SplitMix64, xoshiro256**) ---------------- */

static inline uint64_t sm64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

typedef struct { uint64_t s[4]; } rng_t;

static inline uint64_t rotl64(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

static inline uint64_t rng_u64(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* stream id `stream` of master seed `seed` */
static void rng_init(rng_t *r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed;
    uint64_t a = sm64_next(&x);
    x = a ^ (stream * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL);
    for (int i = 0; i < 4; ++i) r->s[i] = sm64_next(&x);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_unif(rng_t *r) { return (double)(rng_u64(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, n), n >= 1 (multiply-shift) */
static inline uint64_t rng_below(rng_t *r, uint64_t n) {
    return (uint64_t)(((__uint128_t)rng_u64(r) * (__uint128_t)n) >> 64);
}

/* ---------------- deterministic elementary functions ---------------- */

static const double LN2 = 0.69314718055994530942;

/* natural log for finite x > 0: x = m 2^e with m in [1/sqrt2, sqrt2),
 * ln m = 2 atanh((m-1)/(m+1)) summed as an odd power series. */
static double det_log(double x) {
    int e;
    double m = frexp(x, &e);           /* exact */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double z = (m - 1.0) / (m + 1.0);
    double z2 = z * z, term = z, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) { sum += term / (double)k; term *= z2; }
    return 2.0 * sum + (double)e * LN2;
}

/* exp by reduction y = n ln2 + t, |t| <= ln2/2, and a Taylor series in t */
static double det_exp(double y) {
    double n = floor(y / LN2 + 0.5);
    double t = y - n * LN2;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 24; ++k) { term = term * t / (double)k; sum += term; }
    return ldexp(sum, (int)n);          /* exact scaling */
}

static double det_pow(double a, double b) { return det_exp(b * det_log(a)); }

/* ---------------- generator context ---------------- */

typedef struct {
    int64_t n;
    double mean_deg;
    int64_t window;
    double p_local, p_dangling, zipf_exp, rank_exp;
    int zipf_max;
    uint64_t seed;
    double *zipf_cdf;      /* [zipf_max+1], cdf[k] = P(K <= k) */
    double zipf_mean;
    double rank_c;         /* (N+1)^(1-rank_exp) - 1 */
    double rank_q;         /* 1 - rank_exp */
    int32_t *perm;         /* [n] */
    int64_t max_deg;
} dg_ctx;

#define STREAM_PERM 0xFFFFFFFFFFFF0001ULL

void dg_free(dg_ctx *c) {
    if (!c) return;
    free(c->zipf_cdf);
    free(c->perm);
    free(c);
}

dg_ctx *dg_new(int64_t n, double mean_deg, int64_t window, double p_local, double p_dangling,
               double zipf_exp, int zipf_max, double rank_exp, uint64_t seed) {
    if (n < 1 || n > 2147483647LL || zipf_max < 1 || mean_deg <= 0.0 || window < 0) return NULL;
    if (!(rank_exp > 0.0 && rank_exp < 1.0)) return NULL;
    dg_ctx *c = (dg_ctx *)calloc(1, sizeof(dg_ctx));
    if (!c) return NULL;
    c->n = n; c->mean_deg = mean_deg; c->window = window; c->p_local = p_local;
    c->p_dangling = p_dangling; c->zipf_exp = zipf_exp; c->zipf_max = zipf_max;
    c->rank_exp = rank_exp; c->seed = seed;
    c->zipf_cdf = (double *)malloc(sizeof(double) * (size_t)(zipf_max + 1));
    c->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!c->zipf_cdf || !c->perm) { dg_free(c); return NULL; }

    /* Zipf table: weights k^-s, cumulative in increasing k */
    double tot = 0.0, mom = 0.0;
    c->zipf_cdf[0] = 0.0;
    for (int k = 1; k <= zipf_max; ++k) {
        double w = det_pow((double)k, -zipf_exp);
        tot += w;
        mom += (double)k * w;
        c->zipf_cdf[k] = tot;
    }
    for (int k = 1; k <= zipf_max; ++k) c->zipf_cdf[k] /= tot;
    c->zipf_cdf[zipf_max] = 2.0;        /* guard: every u < 1 finds a k */
    c->zipf_mean = mom / tot;

    c->rank_q = 1.0 - rank_exp;
    c->rank_c = det_pow((double)n + 1.0, c->rank_q) - 1.0;

    /* seeded Fisher-Yates permutation */
    for (int64_t i = 0; i < n; ++i) c->perm[i] = (int32_t)i;
    rng_t r;
    rng_init(&r, seed, STREAM_PERM);
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)rng_below(&r, (uint64_t)(i + 1));
        int32_t t = c->perm[i]; c->perm[i] = c->perm[j]; c->perm[j] = t;
    }

    double dmax = floor((double)zipf_max * mean_deg / c->zipf_mean + 0.5);
    c->max_deg = (int64_t)dmax;
    if (c->max_deg > n - 1) c->max_deg = n - 1;
    if (c->max_deg < 1) c->max_deg = 1;
    return c;
}

double dg_zipf_mean(const dg_ctx *c) { return c->zipf_mean; }
int64_t dg_max_degree(const dg_ctx *c) { return c->max_deg; }

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_i32(int32_t *v, int64_t len) {
    if (len <= 24) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t x = v[i];
            int64_t j = i - 1;
            while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; --j; }
            v[j + 1] = x;
        }
    } else {
        qsort(v, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/* raw targets of row j into buf (capacity >= max_deg); returns the count
 * after self-loop removal and deduplication (sorted ascending). */
static int64_t gen_row(const dg_ctx *c, int64_t j, int32_t *buf) {
    rng_t r;
    rng_init(&r, c->seed, (uint64_t)j);
    const int64_t n = c->n;
    if (n < 2) return 0;
    if (rng_unif(&r) < c->p_dangling) return 0;
    /* Zipf draw by binary search: smallest k with cdf[k] > u */
    double u = rng_unif(&r);
    int lo = 1, hi = c->zipf_max;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (c->zipf_cdf[mid] > u) hi = mid; else lo = mid + 1;
    }
    double dk = floor((double)lo * c->mean_deg / c->zipf_mean + 0.5);
    int64_t deg = (int64_t)dk;
    if (deg < 1) deg = 1;
    if (deg > n - 1) deg = n - 1;

    int64_t m = 0;
    for (int64_t e = 0; e < deg; ++e) {
        int64_t t;
        double sel = rng_unif(&r);
        if (sel < c->p_local) {
            int64_t off = (int64_t)rng_below(&r, (uint64_t)(2 * c->window + 1)) - c->window;
            t = (j + off) % n;
            if (t < 0) t += n;
        } else {
            double v = rng_unif(&r);
            double y = 1.0 + v * c->rank_c;           /* (x+1)^q = 1 + v c */
            /* x = y^(1/q) - 1; for q = 0.1 this is y^10 by repeated squaring */
            double x;
            if (c->rank_q == 0.1) {
                double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
                x = y8 * y2 - 1.0;
            } else {
                x = det_pow(y, 1.0 / c->rank_q) - 1.0;
            }
            int64_t rr = (int64_t)floor(x);
            if (rr < 0) rr = 0;
            if (rr > n - 1) rr = n - 1;
            t = c->perm[rr];
        }
        if (t == j) continue;                         /* self-loop */
        buf[m++] = (int32_t)t;
    }
    sort_i32(buf, m);
    int64_t u_cnt = 0;
    for (int64_t i = 0; i < m; ++i)
        if (u_cnt == 0 || buf[i] != buf[u_cnt - 1]) buf[u_cnt++] = buf[i];
    return u_cnt;
}

/* pass 1: row_ptr[n+1]; returns nnz, or -1 on allocation failure */
int64_t dg_row_ptr(const dg_ctx *c, int64_t *row_ptr) {
    const int64_t n = c->n;
    int failed = 0;
    #pragma omp parallel
    {
        int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(c->max_deg + 1));
        if (!buf) {
            #pragma omp atomic write
            failed = 1;
        } else {
            #pragma omp for schedule(dynamic, 4096)
            for (int64_t j = 0; j < n; ++j) row_ptr[j + 1] = gen_row(c, j, buf);
            free(buf);
        }
    }
    if (failed) return -1;
    row_ptr[0] = 0;
    for (int64_t j = 0; j < n; ++j) row_ptr[j + 1] += row_ptr[j];
    return row_ptr[n];
}

/* pass 2: col[row_ptr[n]] given the row_ptr of pass 1; returns 0 or -1 */
int dg_fill(const dg_ctx *c, const int64_t *row_ptr, int32_t *col) {
    const int64_t n = c->n;
    int failed = 0;
    #pragma omp parallel
    {
        int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(c->max_deg + 1));
        if (!buf) {
            #pragma omp atomic write
            failed = 1;
        } else {
            #pragma omp for schedule(dynamic, 4096)
            for (int64_t j = 0; j < n; ++j) {
                int64_t m = gen_row(c, j, buf);
                if (m != row_ptr[j + 1] - row_ptr[j]) {
                    #pragma omp atomic write
                    failed = 1;
                } else {
                    memcpy(col + row_ptr[j], buf, sizeof(int32_t) * (size_t)m);
                }
            }
            free(buf);
        }
    }
    return failed ? -1 : 0;
}

/* 64-bit FNV-1a over the CSR arrays, for recording graph identity */
uint64_t dg_hash(int64_t n, const int64_t *row_ptr, const int32_t *col) {
    uint64_t h = 0xCBF29CE484222325ULL;
    const unsigned char *p = (const unsigned char *)row_ptr;
    for (int64_t i = 0; i < (n + 1) * 8; ++i) { h ^= p[i]; h *= 0x100000001B3ULL; }
    p = (const unsigned char *)col;
    for (int64_t i = 0; i < row_ptr[n] * 4; ++i) { h ^= p[i]; h *= 0x100000001B3ULL; }
    return h;
}

/* deterministic helpers exposed for tests of the generator itself */
double dg_det_pow(double a, double b) { return det_pow(a, b); }
double dg_det_log(double a) { return det_log(a); }
double dg_det_exp(double a) { return det_exp(a); }
