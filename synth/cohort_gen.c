/*
 * Seeded synthetic mutation cohorts.
 *
 * This module only draws inputs: binary gene x sample mutation matrices shaped
 * like the somatic-mutation cohorts of the paper's experiments (§IV-B: very
 * sparse rows, a few frequent genes and a long tail of rare ones, §III-A), packed
 * in the layout the
 * solver library and the oracle both accept.  It contains none of the method's
 * arithmetic (no covers, no scores, no search).
 *
 * Output layout (gene-major, one row per gene):
 *   row g = [ Wt tumor words | Wn normal words ],  Wt = ceil(Nt/64), Wn = ceil(Nn/64)
 *   sample s of a block is bit (s % 64) of word (s / 64), least significant bit
 *   first; bits past Nt (resp. Nn) are zero.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018) seeded through
 * splitmix64 (Steele, Lea & Flood; the seeding routine Blackman & Vigna give).
 * A Bernoulli(p) draw takes the top 53 bits u and answers u < floor(p * 2^53).
 * Normal variates use the Box-Muller transform (cosine branch only).
 * Bounded integers use Lemire's multiply-and-reject method, so they are exactly
 * uniform.
 *
 * Draw order (fixed, so the cohorts are reproducible):
 *   1. per-gene tumor rates, in generation order;
 *   2. per-sample burden multipliers (law 2 only): tumors, then normals;
 *   3. the bits: gene-major, for each gene its tumors then its normals;
 *   4. the planted combinations: genes, then coverage fraction, then tumors;
 *   5. a uniform random permutation of the gene order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} mhgen_rng;

static uint64_t sm64_next(uint64_t *x)
{
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(mhgen_rng *r, uint64_t seed)
{
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = sm64_next(&x);
}

static uint64_t rng_next(mhgen_rng *r)
{
    uint64_t *s = r->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

static uint64_t rng_u53(mhgen_rng *r) { return rng_next(r) >> 11; }

/* uniform double in [0, 1) */
static double rng_unit(mhgen_rng *r) { return (double)rng_u53(r) * 0x1.0p-53; }

/* Bernoulli(p): top 53 bits below floor(p * 2^53). */
static int rng_bernoulli(mhgen_rng *r, double p)
{
    if (p <= 0.0) { (void)rng_u53(r); return 0; }
    if (p >= 1.0) { (void)rng_u53(r); return 1; }
    const uint64_t thresh = (uint64_t)(p * 0x1.0p53);
    return rng_u53(r) < thresh;
}

/* uniform integer in [0, n), n >= 1 (Lemire 2019, with rejection). */
static uint64_t rng_below(mhgen_rng *r, uint64_t n)
{
    unsigned __int128 m = (unsigned __int128)rng_next(r) * n;
    uint64_t lo = (uint64_t)m;
    if (lo < n) {
        const uint64_t t = (0 - n) % n;
        while (lo < t) {
            m = (unsigned __int128)rng_next(r) * n;
            lo = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* standard normal, Box-Muller cosine branch */
static double rng_normal(mhgen_rng *r)
{
    const double u1 = ((double)rng_u53(r) + 1.0) * 0x1.0p-53; /* (0, 1] */
    const double u2 = rng_unit(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}

/* ------------------------------------------------------------------------ */

enum { MHGEN_LAW_LOGNORMAL = 0, MHGEN_LAW_POWER_TOP = 1, MHGEN_LAW_POWER_BURDEN = 2 };

typedef struct {
    int32_t G, Nt, Nn;
    int32_t law;
    /* law 0: p = clip(exp(ln_mu + ln_sigma * z), p_lo, p_hi) */
    double ln_mu, ln_sigma, p_lo, p_hi;
    /* law 1: n_top genes at U[top_lo, top_hi], the rest min(p_cap, c * r^-beta)
     *        with c bisected so that the mean rate over all genes is mean_rate.
     * law 2: every gene min(p_cap, c * r^-beta), c bisected to mean_rate, and a
     *        per-sample burden exp(burden_sigma * z - burden_sigma^2 / 2). */
    int32_t n_top;
    double top_lo, top_hi, beta, p_cap, mean_rate, burden_sigma;
    double normal_ratio;     /* normal rate = normal_ratio * tumor rate */
    int32_t n_plant, plant_h; /* planted combinations and their size */
    double f_lo, f_hi;        /* planted tumor fraction ~ U[f_lo, f_hi] */
    uint64_t seed;
} mhgen_params;

static int cmp_double(const void *a, const void *b)
{
    const double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double power_mean(const mhgen_params *p, double c, int first_rank, int count)
{
    double s = 0.0;
    for (int i = 0; i < count; ++i) {
        double v = c * pow((double)(first_rank + i), -p->beta);
        s += v < p->p_cap ? v : p->p_cap;
    }
    return s;
}

/* c such that sum of min(cap, c r^-beta) over the ranks equals target_sum */
static double bisect_c(const mhgen_params *p, int first_rank, int count, double target_sum)
{
    double lo = 0.0, hi = 1.0;
    while (power_mean(p, hi, first_rank, count) < target_sum && hi < 1e12) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (power_mean(p, mid, first_rank, count) < target_sum) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static void set_bit(uint64_t *row, int s) { row[s >> 6] |= 1ULL << (s & 63); }

/*
 * Fills bitmaps[G * (Wt + Wn)] and, if planted != NULL, planted[n_plant * plant_h]
 * with the planted genes in final (permuted) row indices.  Returns 0, or -1 on a
 * bad parameter or allocation failure.
 */
int mhgen_generate(const mhgen_params *p, uint64_t *bitmaps, int32_t *planted)
{
    const int G = p->G, Nt = p->Nt, Nn = p->Nn;
    if (G < 0 || Nt < 0 || Nn < 0 || !bitmaps) return -1;
    const int Wt = (Nt + 63) / 64, Wn = (Nn + 63) / 64, W = Wt + Wn;
    mhgen_rng rng;
    rng_seed(&rng, p->seed);
    memset(bitmaps, 0, sizeof(uint64_t) * (size_t)G * (size_t)W);
    if (G == 0) return 0;

    double *rate = (double *)malloc(sizeof(double) * (size_t)G);
    double *btum = (double *)malloc(sizeof(double) * (size_t)(Nt > 0 ? Nt : 1));
    double *bnor = (double *)malloc(sizeof(double) * (size_t)(Nn > 0 ? Nn : 1));
    uint64_t *tmp = (uint64_t *)calloc((size_t)G * (size_t)W, sizeof(uint64_t));
    int *pool = (int *)malloc(sizeof(int) * (size_t)(G > Nt ? G : (Nt > 0 ? Nt : 1)));
    double *sorted = (double *)malloc(sizeof(double) * (size_t)G);
    int ok = rate && btum && bnor && tmp && pool && sorted;
    if (!ok) goto done;

    /* 1. tumor rates */
    if (p->law == MHGEN_LAW_LOGNORMAL) {
        for (int g = 0; g < G; ++g) {
            double v = exp(p->ln_mu + p->ln_sigma * rng_normal(&rng));
            rate[g] = v < p->p_lo ? p->p_lo : (v > p->p_hi ? p->p_hi : v);
        }
    } else if (p->law == MHGEN_LAW_POWER_TOP) {
        const int nt = p->n_top < G ? p->n_top : G;
        double top_sum = 0.0;
        for (int g = 0; g < nt; ++g) {
            rate[g] = p->top_lo + (p->top_hi - p->top_lo) * rng_unit(&rng);
            top_sum += rate[g];
        }
        double rest = p->mean_rate * G - top_sum;
        if (rest < 0) rest = 0;
        const double c = bisect_c(p, nt + 1, G - nt, rest);
        for (int g = nt; g < G; ++g) {
            double v = c * pow((double)(g + 1), -p->beta);
            rate[g] = v < p->p_cap ? v : p->p_cap;
        }
    } else if (p->law == MHGEN_LAW_POWER_BURDEN) {
        const double c = bisect_c(p, 1, G, p->mean_rate * G);
        for (int g = 0; g < G; ++g) {
            double v = c * pow((double)(g + 1), -p->beta);
            rate[g] = v < p->p_cap ? v : p->p_cap;
        }
    } else {
        ok = 0;
        goto done;
    }

    /* 2. sample burdens */
    for (int s = 0; s < Nt; ++s) btum[s] = 1.0;
    for (int s = 0; s < Nn; ++s) bnor[s] = 1.0;
    if (p->law == MHGEN_LAW_POWER_BURDEN) {
        const double sg = p->burden_sigma, shift = 0.5 * sg * sg;
        for (int s = 0; s < Nt; ++s) btum[s] = exp(sg * rng_normal(&rng) - shift);
        for (int s = 0; s < Nn; ++s) bnor[s] = exp(sg * rng_normal(&rng) - shift);
    }

    /* 3. bits, gene-major: tumors then normals */
    for (int g = 0; g < G; ++g) {
        uint64_t *row = tmp + (size_t)g * W;
        for (int s = 0; s < Nt; ++s)
            if (rng_bernoulli(&rng, rate[g] * btum[s])) set_bit(row, s);
        for (int s = 0; s < Nn; ++s)
            if (rng_bernoulli(&rng, p->normal_ratio * rate[g] * bnor[s])) set_bit(row + Wt, s);
    }

    /* 4. planting: distinct genes with a rate strictly below the median */
    int *used_genes = NULL;
    if (p->n_plant > 0 && p->plant_h > 0 && Nt > 0) {
        memcpy(sorted, rate, sizeof(double) * (size_t)G);
        qsort(sorted, (size_t)G, sizeof(double), cmp_double);
        const double median = sorted[(G - 1) / 2];
        int n_elig = 0;
        for (int g = 0; g < G; ++g)
            if (rate[g] < median) pool[n_elig++] = g;
        if (n_elig < p->n_plant * p->plant_h) { ok = 0; goto done; }
        used_genes = (int *)malloc(sizeof(int) * (size_t)(p->n_plant * p->plant_h));
        int *tum = (int *)malloc(sizeof(int) * (size_t)Nt);
        if (!used_genes || !tum) { free(tum); ok = 0; goto done; }
        for (int c = 0; c < p->n_plant; ++c) {
            for (int j = 0; j < p->plant_h; ++j) {
                const int k = (int)rng_below(&rng, (uint64_t)n_elig);
                used_genes[c * p->plant_h + j] = pool[k];
                pool[k] = pool[--n_elig];
            }
            const double f = p->f_lo + (p->f_hi - p->f_lo) * rng_unit(&rng);
            int m = (int)floor(f * Nt + 0.5);
            if (m > Nt) m = Nt;
            for (int s = 0; s < Nt; ++s) tum[s] = s;
            for (int i = 0; i < m; ++i) { /* partial Fisher-Yates */
                const int k = i + (int)rng_below(&rng, (uint64_t)(Nt - i));
                const int t = tum[i]; tum[i] = tum[k]; tum[k] = t;
            }
            for (int j = 0; j < p->plant_h; ++j) {
                uint64_t *row = tmp + (size_t)used_genes[c * p->plant_h + j] * W;
                for (int i = 0; i < m; ++i) set_bit(row, tum[i]);
            }
        }
        free(tum);
    }

    /* 5. permute the gene order: final row i = generated row src[i] */
    for (int g = 0; g < G; ++g) pool[g] = g;
    for (int i = G - 1; i > 0; --i) {
        const int k = (int)rng_below(&rng, (uint64_t)(i + 1));
        const int t = pool[i]; pool[i] = pool[k]; pool[k] = t;
    }
    for (int i = 0; i < G; ++i)
        memcpy(bitmaps + (size_t)i * W, tmp + (size_t)pool[i] * W, sizeof(uint64_t) * (size_t)W);
    if (planted && used_genes) {
        /* inverse map: generated gene -> final row */
        int *inv = (int *)malloc(sizeof(int) * (size_t)G);
        if (!inv) { ok = 0; goto done; }
        for (int i = 0; i < G; ++i) inv[pool[i]] = i;
        for (int i = 0; i < p->n_plant * p->plant_h; ++i) planted[i] = inv[used_genes[i]];
        free(inv);
    }
    free(used_genes);

done:
    free(rate);
    free(btum);
    free(bnor);
    free(tmp);
    free(pool);
    free(sorted);
    return ok ? 0 : -1;
}

/* Cohort shape of a batch member: G, Nt, Nn uniform on the inclusive ranges,
 * drawn from the cohort's own seed (before mhgen_generate reseeds it). */
void mhgen_draw_shape(uint64_t seed, int32_t g_lo, int32_t g_hi, int32_t t_lo, int32_t t_hi,
                      int32_t n_lo, int32_t n_hi, int32_t *G, int32_t *Nt, int32_t *Nn)
{
    mhgen_rng rng;
    rng_seed(&rng, seed ^ 0x5851f42d4c957f2dULL);
    *G = g_lo + (int32_t)rng_below(&rng, (uint64_t)(g_hi - g_lo + 1));
    *Nt = t_lo + (int32_t)rng_below(&rng, (uint64_t)(t_hi - t_lo + 1));
    *Nn = n_lo + (int32_t)rng_below(&rng, (uint64_t)(n_hi - n_lo + 1));
}

/* Request trace: exponential inter-arrival gaps with the given mean, and a
 * categorical draw of h over (h_values[i], h_weights[i]). */
void mhgen_trace(uint64_t seed, int32_t n, double mean_gap, int32_t n_cat, const int32_t *h_values,
                 const double *h_weights, double *gaps, int32_t *hs)
{
    mhgen_rng rng;
    rng_seed(&rng, seed);
    double tot = 0.0;
    for (int i = 0; i < n_cat; ++i) tot += h_weights[i];
    for (int i = 0; i < n; ++i) {
        const double u = ((double)rng_u53(&rng) + 1.0) * 0x1.0p-53;
        gaps[i] = -log(u) * mean_gap;
        double v = rng_unit(&rng) * tot;
        int k = 0;
        while (k < n_cat - 1 && v >= h_weights[k]) { v -= h_weights[k]; ++k; }
        hs[i] = h_values[k];
    }
}

/* The raw generator stream, for the published-value pins of the RNG itself. */
void mhgen_stream(uint64_t seed, int32_t n, uint64_t *out)
{
    mhgen_rng rng;
    rng_seed(&rng, seed);
    for (int i = 0; i < n; ++i) out[i] = rng_next(&rng);
}
