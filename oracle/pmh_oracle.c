/*
 * ProbMinHash oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 restatement of the ProbMinHash paper
 * (Ertl, "ProbMinHash -- A Class of Locality-Sensitive Hash Algorithms for
 * the (Probability) Jaccard Similarity", arXiv 1911.00675).  It exists so
 * that the CUDA library can be checked against something written directly
 * from the paper.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline / reference arm may load it.  The product path never does, and
 * this file shares no code, header, table or constant generator with the
 * CUDA library.
 *
 * Contents (each function cites the paper passage it follows):
 *   - the counter-based random stream (replaces the paper's Wyrand PRNG,
 *     Sec. Experiments; distributions as in Eq. def_hash_jp)
 *   - Algorithm "Maintenance of stop limit" (track_max), binary max tree
 *   - Algorithm "Lazy generation of random permutation elements"
 *   - Algorithms ProbMinHash1, 2, 3, 4, 1a, 3a exactly in the paper's step
 *     order, with the tie-break reading documented below
 *   - brute force: Eq. def_new_exp + Eq. signature_def without early stop
 *   - P-MinHash (Algorithm P-MinHash), statistics only
 *   - exact probability Jaccard similarity J_P (definition, Sec. Incorporating
 *     Weights), the estimator of Eq. jaccard_estimator
 *   - a near-tie scan used to exempt components whose two best candidates are
 *     closer than a relative gap (GPU and host log1p may differ in the last ulp)
 *   - Algorithm "Reduction to a b-bit signature" (Sec. Introduction / related
 *     work on b-bit minwise hashing) and the collision-corrected estimate
 *   - the binary-weight specialisations of ProbMinHash3, 3a and 4 (Sec.
 *     Conventional Jaccard Similarity): uniform variates, gamma_i = i
 *   - the rejection sampler for Exp(lambda;0,1) of Sec. Truncated Exponential
 *     Sampling (Algorithm "Fast generation of random values from
 *     Exp(lambda;0,1)") as an alternative to inversion for ProbMinHash3/3a/4
 *
 * Readings of the paper taken here:
 *   - Ties: components keep the lexicographic minimum of (value, element id);
 *     the stop test is strict (stop when a point is > q_max), so an equal
 *     value with a smaller id is still examined.  The paper's "<" / ">=" make
 *     ties order dependent; ties have probability ~0.
 *   - Labels are 0-based internally (paper: 1..m).
 *   - Uniform integers use a multiply-high without rejection.
 *   - Truncated exponentials use inverse-transform sampling by default, the
 *     direct method the paper gives before its rejection sampler (Sec.
 *     Truncated Exponential Sampling).  With the rejection sampler (flag
 *     OR_TE_REJECTION) point i's first uniform is its value word; the
 *     rejection loop's uniforms sit at fixed stream words 2^40 + 256 (i-1) + j
 *     (attempt t uses j = 2t for x and 2t+1 for y), so consumption stays
 *     independent of order and precision; after 64 rejected attempts
 *     (probability below 2^-190) inversion of the value word is used.  The
 *     last test of the loop compares with expm1(lambda (1 - x)), the paper's
 *     exp(lambda (1 - x)) - 1.
 *   - Fixed FP64 evaluation order t = b*c, s = a + t, x = w_inv * s; compile
 *     with -ffp-contract=off so no FMA contraction changes the rounding.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_ERR_INVALID_ARG = 1, OR_ERR_BAD_WEIGHT = 2, OR_ERR_ITER_LIMIT = 3, OR_ERR_NO_MEMORY = 5 };
enum { OR_V1 = 0, OR_V1A = 1, OR_V2 = 2, OR_V3 = 3, OR_V3A = 4, OR_V4 = 5,
       /* binary-weight specialisations (Sec. Conventional Jaccard Similarity) */
       OR_V3U = 6, OR_V3AU = 7, OR_V4U = 8 };
static int is_unweighted(int variant) { return variant == OR_V3U || variant == OR_V3AU || variant == OR_V4U; }
enum { OR_TE_REJECTION = 1 };   /* option flag: Exp(lambda;0,1) by the paper's rejection sampler */

/* ------------------------------------------------------------------------ */
/* Random stream.  SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output j of
 * a generator seeded with `key` is mix(key + (j+1)*phi), phi = 2^64/golden
 * ratio, mix = the SplitMix64 finalizer.  Counter-addressable, so the value
 * word and label word of point i sit at fixed positions 2i-2 and 2i-1 and no
 * early stop or execution order shifts later draws. */
static const uint64_t PHI64 = 0x9E3779B97F4A7C15ULL;

uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* "PRNG with seed d" (Algorithm ProbMinHash1): the element's key. */
uint64_t or_key(uint64_t id, uint64_t seed) { return or_mix64(id ^ or_mix64(seed)); }

uint64_t or_word(uint64_t key, uint64_t j) { return or_mix64(key + (j + 1) * PHI64); }

/* U in [0,1) with 53 random bits. */
double or_unif(uint64_t w) { return (double)(w >> 11) * 0x1p-53; }

/* Exp(1) by inversion: -log(1-U); U < 1 keeps it finite. */
double or_exp1(uint64_t w) { return -log1p(-or_unif(w)); }

/* Exp(lambda; 0, 1) by inversion of F(x) = (1-e^{-lambda x})/(1-e^{-lambda}):
 * x = -log1p(U * expm1(-lambda)) / lambda.  c = expm1(-lambda), inv = 1/lambda. */
double or_texp(uint64_t w, double c, double inv_lambda)
{
    double a = or_unif(w) * c;
    double l = log1p(a);
    return -l * inv_lambda;
}

/* Uniform integer in {0..r-1}: floor(w * r / 2^64). */
uint32_t or_uint(uint64_t w, uint32_t r) { return (uint32_t)(((unsigned __int128)w * r) >> 64); }

/* ------------------------------------------------------------------------ */
/* Per-m constants (Sec. ProbMinHash2/3/4).  Computed here from libm, with no
 * shared generator. */
typedef struct {
    uint32_t m;
    double lambda3, c3, inv3;  /* ProbMinHash3: lambda = log(1 + 1/(m-1)) */
    double *beta;              /* ProbMinHash2: beta_i = m/(m-i+1), i = 1..m */
    double *gamma;             /* ProbMinHash4: gamma_i, i = 0..m-1 */
    double *dgamma;            /* gamma_i - gamma_{i-1}, i = 1..m-1 */
    double *c4, *inv4;         /* expm1(-lambda_i), 1/lambda_i, i = 1..m-1 */
    double delta;              /* 1/lambda_1 */
    int unweighted;            /* binary weights: uniform variates, gamma_i = i */
    int te_rej;                /* Exp(lambda;0,1) by the rejection sampler */
    /* rejection sampler constants per rate lambda_i, i = 1..m-1 (ProbMinHash3 uses i = 1):
     * c1 = (e^lambda - 1)/lambda, c2 = log(2/(1+e^-lambda))/lambda, c3 = (1-e^-lambda)/lambda */
    double *rl, *rc1, *rc2, *rc3;
} or_consts;

static void consts_free(or_consts *c)
{
    free(c->beta); free(c->gamma); free(c->dgamma); free(c->c4); free(c->inv4);
    free(c->rl); free(c->rc1); free(c->rc2); free(c->rc3);
}

static void rej_consts(double lambda, double *c1, double *c2, double *c3)
{
    *c1 = expm1(lambda) / lambda;
    *c2 = log(2.0 / (1.0 + exp(-lambda))) / lambda;
    *c3 = -expm1(-lambda) / lambda;
}

static int consts_init(or_consts *c, uint32_t m)
{
    memset(c, 0, sizeof(*c));
    c->m = m;
    c->beta = (double *)calloc(m + 1, sizeof(double));
    c->gamma = (double *)calloc(m + 1, sizeof(double));
    c->dgamma = (double *)calloc(m + 1, sizeof(double));
    c->c4 = (double *)calloc(m + 1, sizeof(double));
    c->inv4 = (double *)calloc(m + 1, sizeof(double));
    c->rl = (double *)calloc(m + 1, sizeof(double));
    c->rc1 = (double *)calloc(m + 1, sizeof(double));
    c->rc2 = (double *)calloc(m + 1, sizeof(double));
    c->rc3 = (double *)calloc(m + 1, sizeof(double));
    if (!c->beta || !c->gamma || !c->dgamma || !c->c4 || !c->inv4 || !c->rl || !c->rc1 || !c->rc2 || !c->rc3) {
        consts_free(c);
        return OR_ERR_NO_MEMORY;
    }
    for (uint32_t i = 1; i <= m; i++) c->beta[i] = (double)m / (double)(m - i + 1);
    if (m >= 2) {
        c->lambda3 = log1p(1.0 / (double)(m - 1));
        c->c3 = expm1(-c->lambda3);
        c->inv3 = 1.0 / c->lambda3;
        double lambda1 = c->lambda3; /* lambda_1 = log(1 + 1/(m-1)) */
        c->gamma[0] = 0.0;
        for (uint32_t i = 1; i < m; i++) {
            double li = log1p(1.0 / (double)(m - i));
            c->c4[i] = expm1(-li);
            c->inv4[i] = 1.0 / li;
            c->gamma[i] = log1p((double)i / (double)(m - i)) / lambda1;
            c->dgamma[i] = c->gamma[i] - c->gamma[i - 1];
            c->rl[i] = li;
            rej_consts(li, &c->rc1[i], &c->rc2[i], &c->rc3[i]);
        }
        c->delta = 1.0 / lambda1;
    }
    return OR_OK;
}

/* Exposed for tests (closed forms of the tables). */
int or_tables(uint32_t m, double *beta, double *gamma, double *dgamma, double *lambda_i, double *scalars)
{
    or_consts c;
    if (m < 2) return OR_ERR_INVALID_ARG;
    if (consts_init(&c, m)) return OR_ERR_NO_MEMORY;
    for (uint32_t i = 0; i <= m; i++) {
        if (beta) beta[i] = c.beta[i];
        if (gamma) gamma[i] = c.gamma[i];
        if (dgamma) dgamma[i] = c.dgamma[i];
        if (lambda_i) lambda_i[i] = (i >= 1 && i < m) ? log1p(1.0 / (double)(m - i)) : 0.0;
    }
    if (scalars) { scalars[0] = c.lambda3; scalars[1] = c.c3; scalars[2] = c.inv3; scalars[3] = c.delta; }
    consts_free(&c);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm "Fast generation of random values from Exp(lambda;0,1)" (Sec.
 * Truncated Exponential Sampling).  Under the density e^{-lambda x} on [0,1)
 * the region splits into the rectangle A1 = [0,1) x [0, e^{-lambda}) and the
 * rest A2.  A draw x = c1 U (c1 = |A1 u A2| / |A1|) below 1 falls in A1 and is
 * returned as it is.  Otherwise a point of A2 is drawn by rejection, in the
 * rescaled coordinate y~ = (y - e^{-lambda}) / (1 - e^{-lambda}): x uniform on
 * [0,1) is accepted at once below c2 (the part of the rectangle
 * [0,1) x [0, 1/2) under the density); else y~ is uniform on [0, 1/2), a point
 * above the anti-diagonal is reflected through (1/2, 1/2), and the point is
 * accepted below the tangent at 0, below the tangent at 1, or below the density
 * itself.  Returns x; *attempts (optional) the number of rejection attempts. */
#define TE_REJ_MAX 64
static uint64_t te_aux_word(uint64_t key, uint64_t i, uint32_t j)
{
    return or_word(key, (1ULL << 40) + ((i - 1) << 8) + j);
}

static double texp_rejection(uint64_t key, uint64_t i, uint64_t vw, double lambda, double c1, double c2, double c3,
                             int *attempts)
{
    if (attempts) *attempts = 0;
    double x = c1 * or_unif(vw);
    if (x < 1.0) return x;                                   /* A1 */
    for (uint32_t t = 0; t < TE_REJ_MAX; t++) {
        if (attempts) *attempts = (int)t + 1;
        x = or_unif(te_aux_word(key, i, 2 * t));
        if (x < c2) return x;                                /* entirely below the density */
        double y = 0.5 * or_unif(te_aux_word(key, i, 2 * t + 1));
        if (y > 1.0 - x) { x = 1.0 - x; y = 1.0 - y; }       /* reflection through (1/2, 1/2) */
        if (x <= c3 * (1.0 - y)) return x;                   /* below the tangent at 0 */
        if (y * c1 <= 1.0 - x) return x;                     /* below the tangent at 1 */
        if (y * c1 * lambda <= expm1(lambda * (1.0 - x))) return x;   /* below the density */
    }
    return or_texp(vw, expm1(-lambda), 1.0 / lambda);
}

/* Exposed for tests: one variate of the rejection sampler for rate lambda
 * (point i of the element with key `key`, value word vw). */
double or_texp_rej(uint64_t key, uint64_t i, uint64_t vw, double lambda, int *attempts)
{
    double c1, c2, c3;
    rej_consts(lambda, &c1, &c2, &c3);
    return texp_rejection(key, i, vw, lambda, c1, c2, c3, attempts);
}

/* Exposed for tests: the sampler's constants for rate lambda. */
void or_rej_consts(double lambda, double *out3)
{
    rej_consts(lambda, &out3[0], &out3[1], &out3[2]);
}

/* ------------------------------------------------------------------------ */
/* Point values x_i(d), Sec. Sequence Generation.  For the correlated variants
 * the i-th point is a direct function of i; for the uncorrelated ones it is
 * the running sum of the paper's recursion. */

/* ProbMinHash3: x_i = w_inv * ((i-1) + Exp(lambda;0,1)).  With binary weights
 * (Sec. Conventional Jaccard Similarity) every element has the same interval
 * boundaries, only the order of points matters, and Exp(lambda;0,1) is
 * replaced by Uniform([0,1)). */
static double pmh3_point(const or_consts *c, uint64_t key, double w_inv, uint64_t i)
{
    uint64_t vw = or_word(key, 2 * i - 2);
    double te;
    if (c->unweighted) te = or_unif(vw);
    else if (c->te_rej) te = texp_rejection(key, i, vw, c->rl[1], c->rc1[1], c->rc2[1], c->rc3[1], NULL);
    else te = or_texp(vw, c->c3, c->inv3);
    double s = (double)(i - 1) + te;
    return w_inv * s;
}

/* ProbMinHash4: x_i = w_inv * (gamma_{i-1} + (gamma_i-gamma_{i-1}) * Exp(lambda_i;0,1)), i < m;
 * x_m = w_inv * (gamma_{m-1} + delta * Exp(1)). */
static double pmh4_point(const or_consts *c, uint64_t key, double w_inv, uint64_t i)
{
    uint64_t vw = or_word(key, 2 * i - 2);
    double s;
    if (c->unweighted) {
        /* binary weights: gamma_i = i, and both truncated exponentials and the last
         * point's delta * Exp(1) become Uniform([0,1)) (Sec. Conventional Jaccard Similarity) */
        s = (double)(i - 1) + or_unif(vw);
    } else if (i < c->m) {
        double te = c->te_rej ? texp_rejection(key, i, vw, c->rl[i], c->rc1[i], c->rc2[i], c->rc3[i], NULL)
                              : or_texp(vw, c->c4[i], c->inv4[i]);
        double t = c->dgamma[i] * te;
        s = c->gamma[i - 1] + t;
    } else {
        double t = c->delta * or_exp1(vw);
        s = c->gamma[c->m - 1] + t;
    }
    return w_inv * s;
}

/* Lower bound of point i of ProbMinHash4: w_inv * gamma_{i-1} (gamma_{i-1} = i-1 with binary weights). */
static double pmh4_lower(const or_consts *c, double w_inv, uint64_t i)
{
    return c->unweighted ? w_inv * (double)(i - 1) : w_inv * c->gamma[i - 1];
}

/* ------------------------------------------------------------------------ */
/* Algorithm "Maintenance of stop limit" (Sec. Stop Limit Update): the array
 * q[1..2m-1] holds the m leaves and their m-1 parents; q[2m-1] is q_max.
 * 1-based exactly as printed; index 0 unused. */
typedef struct {
    uint32_t m;
    double *q;      /* size 2m */
    uint64_t *z;    /* size m+1 */
} or_sig;

static int sig_init(or_sig *s, uint32_t m)
{
    s->m = m;
    s->q = (double *)malloc(sizeof(double) * (2 * (size_t)m + 1));
    s->z = (uint64_t *)calloc((size_t)m + 1, sizeof(uint64_t));
    if (!s->q || !s->z) { free(s->q); free(s->z); return OR_ERR_NO_MEMORY; }
    for (size_t i = 0; i <= 2 * (size_t)m; i++) s->q[i] = INFINITY;
    return OR_OK;
}

static void sig_free(or_sig *s) { free(s->q); free(s->z); }

static double sig_qmax(const or_sig *s) { return s->q[2 * (size_t)s->m - 1]; }

static void track_max(or_sig *s, double h, uint64_t k)
{
    const uint64_t m = s->m;
    double *q = s->q;
    while (h < q[k]) {
        q[k] = h;
        uint64_t i = m + (k + 1) / 2;       /* index of parent */
        if (i >= 2 * m) break;
        uint64_t j = ((k - 1) ^ 1) + 1;     /* index of sibling */
        if (q[j] >= q[i]) break;
        if (h < q[j]) h = q[j];
        k = i;
    }
}

/* Exposed for tests: apply a sequence of (value, leaf) updates and return the
 * root after each one. */
int or_track_max_run(uint32_t m, const double *h, const uint32_t *k0, int64_t cnt, double *root_out)
{
    or_sig s;
    if (m < 1) return OR_ERR_INVALID_ARG;
    if (sig_init(&s, m)) return OR_ERR_NO_MEMORY;
    for (int64_t t = 0; t < cnt; t++) {
        track_max(&s, h[t], (uint64_t)k0[t] + 1);
        root_out[t] = sig_qmax(&s);
    }
    sig_free(&s);
    return OR_OK;
}

/* Offer point h of element d to component k (0-based).  Lexicographic
 * (value, id) minimum; the tree only moves when the value drops. */
static void sig_offer(or_sig *s, double h, uint64_t d, uint32_t k0)
{
    uint64_t k = (uint64_t)k0 + 1;
    double qk = s->q[k];
    if (h < qk || (h == qk && d < s->z[k])) {
        s->z[k] = d;
        if (h < qk) track_max(s, h, k);
    }
}

/* Exposed for tests: apply offers (value, id, 0-based component) in order and
 * return the final (q, z); pins the lexicographic (value, id) tie rule. */
int or_offer_run(uint32_t m, const double *h, const uint64_t *ids, const uint32_t *k0, int64_t cnt, double *q_out,
                 uint64_t *z_out)
{
    or_sig s;
    if (m < 1) return OR_ERR_INVALID_ARG;
    if (sig_init(&s, m)) return OR_ERR_NO_MEMORY;
    for (int64_t t = 0; t < cnt; t++) sig_offer(&s, h[t], ids[t], k0[t]);
    for (uint32_t k = 0; k < m; k++) { q_out[k] = s.q[k + 1]; z_out[k] = s.z[k + 1]; }
    sig_free(&s);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Algorithm "Lazy generation of random permutation elements" (Sec.
 * ProbMinHash2): arrays g (values) and v (versions), counter c. */
typedef struct {
    uint32_t m, i;
    uint64_t c;
    uint32_t *g;
    uint64_t *v;
} or_perm;

static int perm_init(or_perm *p, uint32_t m)
{
    p->m = m; p->i = 0; p->c = 0;
    p->g = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)m + 1));
    p->v = (uint64_t *)calloc((size_t)m + 1, sizeof(uint64_t));
    if (!p->g || !p->v) { free(p->g); free(p->v); return OR_ERR_NO_MEMORY; }
    return OR_OK;
}
static void perm_free(or_perm *p) { free(p->g); free(p->v); }
static void perm_reset(or_perm *p) { p->i = 0; p->c++; }

/* Returns a 0-based label.  The uniform draw in {0..m-i} uses the label word. */
static uint32_t perm_next(or_perm *p, uint64_t label_word)
{
    p->i++;
    uint32_t i = p->i;
    uint32_t j = i + or_uint(label_word, p->m - i + 1);
    uint32_t k = (p->v[j] == p->c) ? p->g[j] : j;
    p->g[j] = (p->v[i] == p->c) ? p->g[i] : i;
    p->v[j] = p->c;
    return k - 1;
}

/* Exposed for tests: the first `steps` labels of the lazy permutation of an
 * element with key `key` (label word of step i = stream word 2i-1). */
int or_perm_labels(uint32_t m, uint64_t key, uint32_t steps, uint32_t *out)
{
    or_perm p;
    if (m < 1 || steps > m) return OR_ERR_INVALID_ARG;
    if (perm_init(&p, m)) return OR_ERR_NO_MEMORY;
    perm_reset(&p);
    for (uint32_t i = 1; i <= steps; i++) out[i - 1] = perm_next(&p, or_word(key, 2 * (uint64_t)i - 1));
    perm_free(&p);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t elements;     /* elements with w > 0 */
    uint64_t points;       /* point values generated */
    uint64_t updates;      /* component (value) decreases */
    uint64_t buffer_max;   /* ProbMinHash1a/3a: elements in the buffer after pass 1 */
    uint64_t passes;       /* ProbMinHash1a/3a: buffer passes */
} or_stats;

/* Iteration cap for sampling with replacement (Sec. Experiments): all labels
 * appear among the first mu*m*log(m) points except with probability below
 * m^(1-mu).  The cap is far beyond that for every m. */
static uint64_t point_cap(uint32_t m) { return (uint64_t)(64.0 * m * log((double)m + 1.0)) + 4096; }

static int check_weight(double w)
{
    if (isnan(w) || w < 0.0 || isinf(w)) return OR_ERR_BAD_WEIGHT;
    if (w > 0.0 && !isfinite(1.0 / w)) return OR_ERR_BAD_WEIGHT;
    return OR_OK;
}

/* Algorithm ProbMinHash1. */
static int run_pmh1(or_sig *s, const uint64_t *ids, const double *w, int64_t n, uint64_t seed, or_stats *st)
{
    const uint32_t m = s->m;
    const uint64_t cap = point_cap(m);
    for (int64_t e = 0; e < n; e++) {
        if (!(w[e] > 0.0)) continue;
        st->elements++;
        const uint64_t d = ids[e];
        const double w_inv = 1.0 / w[e];
        const uint64_t key = or_key(d, seed);
        uint64_t i = 1;
        double h = w_inv * or_exp1(or_word(key, 0));
        st->points++;
        while (h <= sig_qmax(s)) {
            uint32_t k = or_uint(or_word(key, 2 * i - 1), m);
            double before = s->q[k + 1];
            sig_offer(s, h, d, k);
            if (s->q[k + 1] < before) st->updates++;
            if (h > sig_qmax(s)) break;
            i++;
            if (i > cap) return OR_ERR_ITER_LIMIT;
            double t = w_inv * or_exp1(or_word(key, 2 * i - 2));
            h = h + t;
            st->points++;
        }
    }
    return OR_OK;
}

/* Algorithm ProbMinHash2 (with the lazy permutation). */
static int run_pmh2(or_sig *s, const or_consts *c, const uint64_t *ids, const double *w, int64_t n, uint64_t seed,
                    or_stats *st)
{
    const uint32_t m = s->m;
    or_perm p;
    if (perm_init(&p, m)) return OR_ERR_NO_MEMORY;
    for (int64_t e = 0; e < n; e++) {
        if (!(w[e] > 0.0)) continue;
        st->elements++;
        const uint64_t d = ids[e];
        const double w_inv = 1.0 / w[e];
        const uint64_t key = or_key(d, seed);
        perm_reset(&p);
        uint64_t i = 1;
        double h = w_inv * (c->beta[1] * or_exp1(or_word(key, 0)));
        st->points++;
        while (h <= sig_qmax(s)) {
            uint32_t k = perm_next(&p, or_word(key, 2 * i - 1));
            double before = s->q[k + 1];
            sig_offer(s, h, d, k);
            if (s->q[k + 1] < before) st->updates++;
            if (h > sig_qmax(s)) break;
            if (i == m) break; /* the sequence has m points (sampling without replacement) */
            i++;
            double t = w_inv * (c->beta[i] * or_exp1(or_word(key, 2 * i - 2)));
            h = h + t;
            st->points++;
        }
    }
    perm_free(&p);
    return OR_OK;
}

/* Algorithm ProbMinHash3 (requires m >= 2). */
static int run_pmh3(or_sig *s, const or_consts *c, const uint64_t *ids, const double *w, int64_t n, uint64_t seed,
                    or_stats *st)
{
    const uint32_t m = s->m;
    const uint64_t cap = point_cap(m);
    for (int64_t e = 0; e < n; e++) {
        if (!(w[e] > 0.0)) continue;
        st->elements++;
        const uint64_t d = ids[e];
        const double w_inv = 1.0 / w[e];
        const uint64_t key = or_key(d, seed);
        double h = pmh3_point(c, key, w_inv, 1);
        uint64_t i = 1;
        st->points++;
        while (h <= sig_qmax(s)) {
            uint32_t k = or_uint(or_word(key, 2 * i - 1), m);
            double before = s->q[k + 1];
            sig_offer(s, h, d, k);
            if (s->q[k + 1] < before) st->updates++;
            i++;
            if (i > cap) return OR_ERR_ITER_LIMIT;
            h = w_inv * (double)(i - 1);
            if (h > sig_qmax(s)) break;
            h = pmh3_point(c, key, w_inv, i);
            st->points++;
        }
    }
    return OR_OK;
}

/* Algorithm ProbMinHash4 (requires m >= 2). */
static int run_pmh4(or_sig *s, const or_consts *c, const uint64_t *ids, const double *w, int64_t n, uint64_t seed,
                    or_stats *st)
{
    const uint32_t m = s->m;
    or_perm p;
    if (perm_init(&p, m)) return OR_ERR_NO_MEMORY;
    for (int64_t e = 0; e < n; e++) {
        if (!(w[e] > 0.0)) continue;
        st->elements++;
        const uint64_t d = ids[e];
        const double w_inv = 1.0 / w[e];
        const uint64_t key = or_key(d, seed);
        perm_reset(&p);
        double h = pmh4_point(c, key, w_inv, 1);
        uint64_t i = 1;
        st->points++;
        while (h <= sig_qmax(s)) {
            uint32_t k = perm_next(&p, or_word(key, 2 * i - 1));
            double before = s->q[k + 1];
            sig_offer(s, h, d, k);
            if (s->q[k + 1] < before) st->updates++;
            i++;
            if (pmh4_lower(c, w_inv, i) > sig_qmax(s)) break;
            if (i < m) {
                h = pmh4_point(c, key, w_inv, i);
                st->points++;
            } else {
                h = pmh4_point(c, key, w_inv, m);
                st->points++;
                if (h <= sig_qmax(s)) {
                    k = perm_next(&p, or_word(key, 2 * (uint64_t)m - 1));
                    before = s->q[k + 1];
                    sig_offer(s, h, d, k);
                    if (s->q[k + 1] < before) st->updates++;
                }
                break;
            }
        }
    }
    perm_free(&p);
    return OR_OK;
}

/* Algorithm ProbMinHash1a: interleaved processing with a buffer holding
 * (element, w_inv, point index, current point). */
typedef struct { uint64_t d, key; double w_inv, h; uint64_t i; } buf1_t;

static int run_pmh1a(or_sig *s, const uint64_t *ids, const double *w, int64_t n, uint64_t seed, or_stats *st)
{
    const uint32_t m = s->m;
    const uint64_t cap = point_cap(m);
    buf1_t *b = (buf1_t *)malloc(sizeof(buf1_t) * (size_t)(n > 0 ? n : 1));
    if (!b) return OR_ERR_NO_MEMORY;
    int64_t cnt = 0;
    for (int64_t e = 0; e < n; e++) {
        if (!(w[e] > 0.0)) continue;
        st->elements++;
        const uint64_t d = ids[e];
        const double w_inv = 1.0 / w[e];
        const uint64_t key = or_key(d, seed);
        double h = w_inv * or_exp1(or_word(key, 0));
        st->points++;
        if (h > sig_qmax(s)) continue;
        uint32_t k = or_uint(or_word(key, 1), m);
        double before = s->q[k + 1];
        sig_offer(s, h, d, k);
        if (s->q[k + 1] < before) st->updates++;
        if (h > sig_qmax(s)) continue;
        b[cnt].d = d; b[cnt].key = key; b[cnt].w_inv = w_inv; b[cnt].h = h; b[cnt].i = 1;
        cnt++;
    }
    st->buffer_max = (uint64_t)cnt;
    while (cnt > 0) {
        st->passes++;
        int64_t cnt2 = 0;
        for (int64_t j = 0; j < cnt; j++) {
            buf1_t x = b[j];
            if (x.h > sig_qmax(s)) continue;
            x.i++;
            if (x.i > cap) { free(b); return OR_ERR_ITER_LIMIT; }
            double t = x.w_inv * or_exp1(or_word(x.key, 2 * x.i - 2));
            x.h = x.h + t;
            st->points++;
            if (x.h > sig_qmax(s)) continue;
            uint32_t k = or_uint(or_word(x.key, 2 * x.i - 1), m);
            double before = s->q[k + 1];
            sig_offer(s, x.h, x.d, k);
            if (s->q[k + 1] < before) st->updates++;
            if (x.h > sig_qmax(s)) continue;
            b[cnt2++] = x;
        }
        cnt = cnt2;
    }
    free(b);
    return OR_OK;
}

/* Algorithm ProbMinHash3a: interleaved processing; pass i generates point i
 * of every buffered element. */
typedef struct { uint64_t d, key; double w_inv; } buf3_t;

static int run_pmh3a(or_sig *s, const or_consts *c, const uint64_t *ids, const double *w, int64_t n, uint64_t seed,
                     or_stats *st)
{
    const uint32_t m = s->m;
    const uint64_t cap = point_cap(m);
    buf3_t *b = (buf3_t *)malloc(sizeof(buf3_t) * (size_t)(n > 0 ? n : 1));
    if (!b) return OR_ERR_NO_MEMORY;
    int64_t cnt = 0;
    for (int64_t e = 0; e < n; e++) {
        if (!(w[e] > 0.0)) continue;
        st->elements++;
        const uint64_t d = ids[e];
        const double w_inv = 1.0 / w[e];
        const uint64_t key = or_key(d, seed);
        double h = pmh3_point(c, key, w_inv, 1);
        st->points++;
        if (h > sig_qmax(s)) continue;
        uint32_t k = or_uint(or_word(key, 1), m);
        double before = s->q[k + 1];
        sig_offer(s, h, d, k);
        if (s->q[k + 1] < before) st->updates++;
        if (w_inv > sig_qmax(s)) continue;   /* lower bound of point 2: w_inv * 1 */
        b[cnt].d = d; b[cnt].key = key; b[cnt].w_inv = w_inv;
        cnt++;
    }
    st->buffer_max = (uint64_t)cnt;
    uint64_t i = 2;
    while (cnt > 0) {
        if (i > cap) { free(b); return OR_ERR_ITER_LIMIT; }
        st->passes++;
        int64_t cnt2 = 0;
        for (int64_t j = 0; j < cnt; j++) {
            buf3_t x = b[j];
            double h = x.w_inv * (double)(i - 1);
            if (h > sig_qmax(s)) continue;
            h = pmh3_point(c, x.key, x.w_inv, i);
            st->points++;
            if (h > sig_qmax(s)) continue;
            uint32_t k = or_uint(or_word(x.key, 2 * i - 1), m);
            double before = s->q[k + 1];
            sig_offer(s, h, x.d, k);
            if (s->q[k + 1] < before) st->updates++;
            if (x.w_inv * (double)i > sig_qmax(s)) continue;
            b[cnt2++] = x;
        }
        cnt = cnt2;
        i++;
    }
    free(b);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Generates, for one element, every point needed for its hash values h_k(d)
 * (Eq. def_new_exp): with replacement until every label has appeared, without
 * replacement all m points.  Calls emit(k, value) for the first occurrence of
 * each label only, and stops early once points exceed `bound` (bound = +inf
 * gives the complete definition).  Returns the number of points generated or
 * -1 on the iteration cap. */
typedef struct {
    double *h;        /* per label: h_k(d) of the current element (or +inf) */
    uint8_t *seen;
    uint32_t *touched;
    uint32_t ntouched;
} elem_scratch;

static int64_t element_hashes(int variant, const or_consts *c, or_perm *p, uint64_t key, double w_inv, double bound,
                              elem_scratch *es)
{
    const uint32_t m = c->m;
    const uint64_t cap = point_cap(m);
    uint32_t covered = 0;
    int64_t pts = 0;
    es->ntouched = 0;
    int fam = (variant == OR_V1 || variant == OR_V1A) ? 1 : (variant == OR_V2) ? 2
            : (variant == OR_V3 || variant == OR_V3A || variant == OR_V3U || variant == OR_V3AU) ? 3 : 4;
    if (fam == 2 || fam == 4) perm_reset(p);
    double h = 0.0;
    for (uint64_t i = 1;; i++) {
        if (fam == 1 || fam == 3) { if (i > cap) return -1; }
        else if (i > m) break;
        /* lower bounds (correlated) or the running value (uncorrelated) */
        if (fam == 3 && i >= 2 && w_inv * (double)(i - 1) > bound) break;
        if (fam == 4 && i >= 2 && pmh4_lower(c, w_inv, i) > bound) break;
        if (fam == 1) h = h + w_inv * or_exp1(or_word(key, 2 * i - 2));
        else if (fam == 2) h = h + w_inv * (c->beta[i] * or_exp1(or_word(key, 2 * i - 2)));
        else if (fam == 3) h = pmh3_point(c, key, w_inv, i);
        else h = pmh4_point(c, key, w_inv, i);
        pts++;
        if ((fam == 1 || fam == 2) && h > bound) break;
        uint64_t lw = or_word(key, 2 * i - 1);
        uint32_t k = (fam == 1 || fam == 3) ? or_uint(lw, m) : perm_next(p, lw);
        if (h > bound) continue;   /* correlated: later points may still be below */
        if (!es->seen[k]) {
            es->seen[k] = 1;
            es->touched[es->ntouched++] = k;
            es->h[k] = h;
            covered++;
            if (covered == m) break;
        }
    }
    return pts;
}

static void scratch_clear(elem_scratch *es)
{
    for (uint32_t t = 0; t < es->ntouched; t++) { es->seen[es->touched[t]] = 0; es->h[es->touched[t]] = INFINITY; }
    es->ntouched = 0;
}

static int scratch_init(elem_scratch *es, uint32_t m)
{
    es->h = (double *)malloc(sizeof(double) * m);
    es->seen = (uint8_t *)calloc(m, 1);
    es->touched = (uint32_t *)malloc(sizeof(uint32_t) * m);
    es->ntouched = 0;
    if (!es->h || !es->seen || !es->touched) { free(es->h); free(es->seen); free(es->touched); return OR_ERR_NO_MEMORY; }
    for (uint32_t k = 0; k < m; k++) es->h[k] = INFINITY;
    return OR_OK;
}
static void scratch_free(elem_scratch *es) { free(es->h); free(es->seen); free(es->touched); }

/* Brute force: per element all hash values h_k(d) (Eq. def_new_exp), then the
 * per-component lexicographic argmin (Eq. signature_def); no stop limit. */
static int run_brute(int variant, or_sig *s, const or_consts *c, const uint64_t *ids, const double *w, int64_t n,
                     uint64_t seed, or_stats *st)
{
    const uint32_t m = s->m;
    or_perm p;
    elem_scratch es;
    if (perm_init(&p, m)) return OR_ERR_NO_MEMORY;
    if (scratch_init(&es, m)) { perm_free(&p); return OR_ERR_NO_MEMORY; }
    int rc = OR_OK;
    for (int64_t e = 0; e < n && rc == OR_OK; e++) {
        if (!(w[e] > 0.0)) continue;
        st->elements++;
        const double w_inv = 1.0 / w[e];
        int64_t pts = element_hashes(variant, c, &p, or_key(ids[e], seed), w_inv, INFINITY, &es);
        if (pts < 0) { rc = OR_ERR_ITER_LIMIT; break; }
        st->points += (uint64_t)pts;
        for (uint32_t t = 0; t < es.ntouched; t++) {
            uint32_t k = es.touched[t];
            double h = es.h[k];
            if (h < s->q[k + 1] || (h == s->q[k + 1] && ids[e] < s->z[k + 1])) {
                s->q[k + 1] = h;
                s->z[k + 1] = ids[e];
            }
        }
        scratch_clear(&es);
    }
    scratch_free(&es);
    perm_free(&p);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Public entry: signature of one weighted set.
 * mode 0: the paper's algorithm for `variant`; mode 1: brute force.
 * Outputs q[m] (component minima, +inf if empty) and z[m] (ids, 0 if empty). */
int or_sketch_opt(int variant, int mode, int flags, const uint64_t *ids, const double *w, int64_t n, uint32_t m,
                  uint64_t seed, double *q_out, uint64_t *z_out, uint64_t *stats_out)
{
    if (m < 1 || n < 0 || variant < 0 || variant > 8 || mode < 0 || mode > 1) return OR_ERR_INVALID_ARG;
    if ((variant == OR_V3 || variant == OR_V3A || variant == OR_V4) && m < 2) return OR_ERR_INVALID_ARG;
    for (int64_t e = 0; e < n; e++) if (check_weight(w[e])) return OR_ERR_BAD_WEIGHT;
    or_consts c;
    or_sig s;
    or_stats st;
    memset(&st, 0, sizeof(st));
    if (consts_init(&c, m)) return OR_ERR_NO_MEMORY;
    c.te_rej = (flags & OR_TE_REJECTION) != 0;
    if (sig_init(&s, m)) { consts_free(&c); return OR_ERR_NO_MEMORY; }
    /* binary weights: every element with w > 0 counts with weight 1 */
    const double *wu = w;
    double *ones = NULL;
    if (is_unweighted(variant)) {
        c.unweighted = 1;
        ones = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (!ones) { sig_free(&s); consts_free(&c); return OR_ERR_NO_MEMORY; }
        for (int64_t e = 0; e < n; e++) ones[e] = w[e] > 0.0 ? 1.0 : 0.0;
        wu = ones;
    }
    int rc;
    if (mode == 1) rc = run_brute(variant, &s, &c, ids, wu, n, seed, &st);
    else switch (variant) {
        case OR_V1: rc = run_pmh1(&s, ids, w, n, seed, &st); break;
        case OR_V1A: rc = run_pmh1a(&s, ids, w, n, seed, &st); break;
        case OR_V2: rc = run_pmh2(&s, &c, ids, w, n, seed, &st); break;
        case OR_V3: case OR_V3U: rc = run_pmh3(&s, &c, ids, wu, n, seed, &st); break;
        case OR_V3A: case OR_V3AU: rc = run_pmh3a(&s, &c, ids, wu, n, seed, &st); break;
        default: rc = run_pmh4(&s, &c, ids, wu, n, seed, &st); break;
    }
    free(ones);
    if (rc == OR_OK) {
        for (uint32_t k = 0; k < m; k++) {
            q_out[k] = s.q[k + 1];
            z_out[k] = isinf(s.q[k + 1]) ? 0 : s.z[k + 1];
        }
    }
    if (stats_out) {
        stats_out[0] = st.elements; stats_out[1] = st.points; stats_out[2] = st.updates;
        stats_out[3] = st.buffer_max; stats_out[4] = st.passes;
    }
    sig_free(&s);
    consts_free(&c);
    return rc;
}

int or_sketch(int variant, int mode, const uint64_t *ids, const double *w, int64_t n, uint32_t m, uint64_t seed,
              double *q_out, uint64_t *z_out, uint64_t *stats_out)
{
    return or_sketch_opt(variant, mode, 0, ids, w, n, m, seed, q_out, z_out, stats_out);
}

/* Signatures of a CSR batch of sets (offsets[num_sets+1]), one after another;
 * status[s] receives each set's code.  Single-threaded. */
int or_sketch_batch(int variant, const uint64_t *ids, const double *w, const int64_t *offsets, int64_t num_sets,
                    uint32_t m, uint64_t seed, double *q_out, uint64_t *z_out, int32_t *status)
{
    int first = OR_OK;
    for (int64_t t = 0; t < num_sets; t++) {
        int64_t b = offsets[t], e = offsets[t + 1];
        int rc = or_sketch(variant, 0, ids + b, w + b, e - b, m, seed, q_out ? q_out + (size_t)t * m : NULL,
                           z_out + (size_t)t * m, NULL);
        if (rc == OR_ERR_BAD_WEIGHT || rc == OR_ERR_ITER_LIMIT) {
            for (uint32_t k = 0; k < m; k++) { z_out[(size_t)t * m + k] = 0; if (q_out) q_out[(size_t)t * m + k] = INFINITY; }
        }
        if (status) status[t] = rc;
        if (rc && !first) first = rc;
        if (rc == OR_ERR_INVALID_ARG || rc == OR_ERR_NO_MEMORY) return rc;
    }
    return first;
}

/* ------------------------------------------------------------------------ */
/* Near-tie scan.  For every component, the runner-up hash value over elements
 * other than the winner, considering all points up to bound = q_max*(1+rel)
 * (every candidate that can be within rel of any component minimum).
 * flags[k] = 1 when runner-up - q_k < rel * q_k.  Returns the number flagged,
 * or a negative error code.  Also verifies that the scan's minimum equals the
 * given signature (returns -100 if not). */
int64_t or_near_ties_opt(int variant, int opt, const uint64_t *ids, const double *w, int64_t n, uint32_t m,
                         uint64_t seed, const double *q, const uint64_t *z, double rel, uint8_t *flags,
                         double *runner_up);

int64_t or_near_ties(int variant, const uint64_t *ids, const double *w, int64_t n, uint32_t m, uint64_t seed,
                     const double *q, const uint64_t *z, double rel, uint8_t *flags, double *runner_up)
{
    return or_near_ties_opt(variant, 0, ids, w, n, m, seed, q, z, rel, flags, runner_up);
}

int64_t or_near_ties_opt(int variant, int opt, const uint64_t *ids, const double *w, int64_t n, uint32_t m,
                         uint64_t seed, const double *q, const uint64_t *z, double rel, uint8_t *flags,
                         double *runner_up)
{
    if ((variant == OR_V3 || variant == OR_V3A || variant == OR_V4) && m < 2) return -OR_ERR_INVALID_ARG;
    const int unw = is_unweighted(variant);
    double qmax = 0.0;
    for (uint32_t k = 0; k < m; k++) if (q[k] > qmax) qmax = q[k];
    double bound = qmax * (1.0 + rel);
    or_consts c;
    or_perm p;
    elem_scratch es;
    if (consts_init(&c, m)) return -OR_ERR_NO_MEMORY;
    c.unweighted = unw;
    c.te_rej = (opt & OR_TE_REJECTION) != 0;
    if (perm_init(&p, m)) { consts_free(&c); return -OR_ERR_NO_MEMORY; }
    if (scratch_init(&es, m)) { perm_free(&p); consts_free(&c); return -OR_ERR_NO_MEMORY; }
    double *b1 = (double *)malloc(sizeof(double) * m), *b2 = (double *)malloc(sizeof(double) * m);
    uint64_t *id1 = (uint64_t *)malloc(sizeof(uint64_t) * m);
    int64_t rc = 0;
    if (!b1 || !b2 || !id1) rc = -OR_ERR_NO_MEMORY;
    for (uint32_t k = 0; rc == 0 && k < m; k++) { b1[k] = INFINITY; b2[k] = INFINITY; id1[k] = 0; }
    for (int64_t e = 0; rc == 0 && e < n; e++) {
        if (!(w[e] > 0.0)) continue;
        const double w_inv = unw ? 1.0 : 1.0 / w[e];
        int64_t pts = element_hashes(variant, &c, &p, or_key(ids[e], seed), w_inv, bound, &es);
        if (pts < 0) { rc = -OR_ERR_ITER_LIMIT; break; }
        for (uint32_t t = 0; t < es.ntouched; t++) {
            uint32_t k = es.touched[t];
            double h = es.h[k];
            if (h < b1[k] || (h == b1[k] && ids[e] < id1[k])) { b2[k] = b1[k]; b1[k] = h; id1[k] = ids[e]; }
            else if (h < b2[k]) b2[k] = h;
        }
        scratch_clear(&es);
    }
    int64_t flagged = 0;
    for (uint32_t k = 0; rc == 0 && k < m; k++) {
        if (n > 0 && (b1[k] != q[k] || id1[k] != z[k])) { rc = -100; break; }
        int f = isfinite(b2[k]) && (b2[k] - b1[k] < rel * b1[k]);
        if (flags) flags[k] = (uint8_t)f;
        if (runner_up) runner_up[k] = b2[k];
        flagged += f;
    }
    free(b1); free(b2); free(id1);
    scratch_free(&es);
    perm_free(&p);
    consts_free(&c);
    return rc ? rc : flagged;
}

/* ------------------------------------------------------------------------ */
/* Algorithm P-MinHash: m independent values w_inv * Exp(1) per element,
 * component k drawn from stream word k-1.  Statistics only. */
int or_pminhash(const uint64_t *ids, const double *w, int64_t n, uint32_t m, uint64_t seed, double *q_out,
                uint64_t *z_out)
{
    if (m < 1 || n < 0) return OR_ERR_INVALID_ARG;
    for (uint32_t k = 0; k < m; k++) { q_out[k] = INFINITY; z_out[k] = 0; }
    for (int64_t e = 0; e < n; e++) {
        if (check_weight(w[e])) return OR_ERR_BAD_WEIGHT;
        if (!(w[e] > 0.0)) continue;
        const double w_inv = 1.0 / w[e];
        const uint64_t key = or_key(ids[e], seed);
        for (uint32_t k = 0; k < m; k++) {
            double h = w_inv * or_exp1(or_word(key, k));
            if (h < q_out[k] || (h == q_out[k] && ids[e] < z_out[k])) { q_out[k] = h; z_out[k] = ids[e]; }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Probability Jaccard similarity from its definition:
 *   J_P = sum_{d} 1 / sum_{d'} max(w_A(d')/w_A(d), w_B(d')/w_B(d)),
 * where d runs over elements with w_A(d) > 0 and w_B(d) > 0 (the definition's
 * ratios are undefined otherwise and those terms are zero), d' over the union.
 * Inputs are two weighted sets with distinct ids each; O(u^2). */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

double or_jp(const uint64_t *ida, const double *wa, int64_t na, const uint64_t *idb, const double *wb, int64_t nb)
{
    int64_t u = na + nb;
    uint64_t *all = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(u > 0 ? u : 1));
    if (!all) return NAN;
    memcpy(all, ida, sizeof(uint64_t) * (size_t)na);
    memcpy(all + na, idb, sizeof(uint64_t) * (size_t)nb);
    qsort(all, (size_t)u, sizeof(uint64_t), cmp_u64);
    int64_t nu = 0;
    for (int64_t t = 0; t < u; t++) if (nu == 0 || all[nu - 1] != all[t]) all[nu++] = all[t];
    double *A = (double *)calloc((size_t)(nu > 0 ? nu : 1), sizeof(double));
    double *B = (double *)calloc((size_t)(nu > 0 ? nu : 1), sizeof(double));
    if (!A || !B) { free(all); free(A); free(B); return NAN; }
    for (int64_t t = 0; t < na; t++) {
        uint64_t *p = (uint64_t *)bsearch(&ida[t], all, (size_t)nu, sizeof(uint64_t), cmp_u64);
        A[p - all] = wa[t];
    }
    for (int64_t t = 0; t < nb; t++) {
        uint64_t *p = (uint64_t *)bsearch(&idb[t], all, (size_t)nu, sizeof(uint64_t), cmp_u64);
        B[p - all] = wb[t];
    }
    double jp = 0.0;
    for (int64_t d = 0; d < nu; d++) {
        if (!(A[d] > 0.0 && B[d] > 0.0)) continue;
        double den = 0.0;
        for (int64_t e = 0; e < nu; e++) {
            double ra = A[e] / A[d], rb = B[e] / B[d];
            den += ra > rb ? ra : rb;
        }
        jp += 1.0 / den;
    }
    free(all); free(A); free(B);
    return jp;
}

/* Eq. jaccard_estimator numerator: number of equal components. */
uint32_t or_count_equal(const uint64_t *za, const uint64_t *zb, uint32_t m)
{
    uint32_t c = 0;
    for (uint32_t k = 0; k < m; k++) c += (za[k] == zb[k]);
    return c;
}

/* All-pairs equal-component counts over num signatures (row-major num x m):
 * out[a*num + b] for every ordered pair (diagonal = m). */
int or_count_allpairs(const uint64_t *sig, int64_t num, uint32_t m, uint32_t *out)
{
    for (int64_t a = 0; a < num; a++)
        for (int64_t b = 0; b < num; b++)
            out[a * num + b] = or_count_equal(sig + (size_t)a * m, sig + (size_t)b * m, m);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Reduction to a b-bit signature (Algorithm "Reduction to a b-bit
 * signature"): component k (0-based here) becomes the least significant b
 * bits of a hash of the pair (z_k, k).  The hash: SplitMix64's finalizer of
 * z_k XOR a per-index key, the key being output k+1 of SplitMix64 seeded with
 * mix(seed) -- so the index enters every component's hash (the paper stresses
 * that it must, to keep collisions of different elements uncorrelated across
 * components).  b in {1, 2, 4, ..., 64}. */
uint64_t or_bbit_code(uint64_t z, uint32_t k, uint32_t b, uint64_t seed)
{
    const uint64_t key = or_mix64(or_mix64(seed) + ((uint64_t)k + 1) * PHI64);
    const uint64_t h = or_mix64(z ^ key);
    return b >= 64 ? h : (h & ((1ull << b) - 1));
}

int or_bbit_reduce(const uint64_t *sig, int64_t num, uint32_t m, uint32_t b, uint64_t seed, uint64_t *codes)
{
    if (b == 0 || b > 64 || (b & (b - 1))) return OR_ERR_INVALID_ARG;
    for (int64_t a = 0; a < num; a++)
        for (uint32_t k = 0; k < m; k++) codes[a * m + k] = or_bbit_code(sig[a * m + k], k, b, seed);
    return OR_OK;
}

/* Estimate from b-bit codes: equal codes come from equal components
 * (probability J) or from a collision of two different elements' codes
 * (probability 2^-b otherwise), so E[count/m] = J + (1 - J) 2^-b and
 * (count/m - 2^-b) / (1 - 2^-b) is unbiased for J. */
double or_bbit_estimate(uint32_t count, uint32_t m, uint32_t b)
{
    const double r = b >= 64 ? 0.0 : ldexp(1.0, -(int)b);
    return ((double)count / (double)m - r) / (1.0 - r);
}
