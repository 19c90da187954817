/*
 * Oracle for the multi-hit greedy weighted set cover (WSC) with P-DFS.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's CPU
 * baseline may load this code.  It is a plain, slow, single-threaded CPU restatement
 * of what the paper's method computes; it shares nothing with the CUDA library.
 *
 * Input layout (same as the library's boundary): gene-major rows,
 *   row g = [Wt tumor words | Wn normal words], Wt = ceil(Nt/64), Wn = ceil(Nn/64),
 *   sample s of a block = bit (s % 64) of word (s / 64), LSB first, padding zero.
 *
 * Two solvers, both returning the ordered list Gamma of selected h-gene
 * combinations (original gene indices, ascending inside a tuple) with their
 * tumor-covered (TP) and normal-covered (FP) counts:
 *
 * oracle_bruteforce -- the definition.  Algorithm 1 (greedy set cover) whose
 *   step "argmax F" is evaluated by enumerating every h-subset of genes in
 *   lexicographic order of original index, with no pruning and no sharing of
 *   partial intersections:
 *     cover C(gamma) = samples where all genes of gamma are mutated   (Eq. 1)
 *     TP = |C(gamma) restricted to still-uncovered tumors U|
 *     FP = |C(gamma) restricted to normals|
 *     F = (alpha TP + (Nn - FP)) / (Nt + Nn)                          (§II-B)
 *   alpha = a_num / a_den, and the integer score
 *     S = a_num * TP + a_den * (Nn - FP) = F * a_den * (Nt + Nn)
 *   orders candidates exactly like F within a round.  A combination with TP = 0
 *   is not a candidate.  Ties keep the first combination met, i.e. the
 *   lexicographically smallest tuple of original indices (the strict ">" of
 *   Algorithm 2's maximum search).  The covered tumors are removed from U
 *   (DelCols, Algorithm 1), and the loop ends when U is empty (the "while C is
 *   a strict subset of T" test) or when no combination has TP > 0.
 *
 * oracle_pdfs -- P-DFS (§III-D, Algorithm 2, Fig. 5) as the paper describes it:
 *   genes are first reordered from most sparse to least sparse (§III-C: ascending
 *   tumor mutation count, ties by original index); nested loops
 *   g_1 < g_2 < ... < g_h over that order, level l ranging over
 *   (g_{l-1}, G - h + l] (1-based), keep the running intersection
 *   y_l = y_{l-1} AND x_{g_l} over the uncovered tumors (y_0 = U) and backtrack
 *   as soon as y_l is empty (at any depth, §III-D); a leaf with y_h != 0 is
 *   scored and compared with the running best.  Because enumeration order is
 *   no longer the original order, equal scores are resolved explicitly by the
 *   smallest ascending tuple of original indices, so both solvers return the
 *   same Gamma.  Per round and per depth l it counts
 *     visited[l] = depth-l nodes whose y_l was computed,
 *     pruned[l]  = those with y_l = 0,
 *   so scored leaves = visited[h] - pruned[h].  With prune = 0 every node is
 *   expanded (the exhaustive baseline, where visited[l] = C(G-h+l, l)).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_H 9

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOMEM = 3, ORACLE_ECAP = 8 };

static int popcount64(uint64_t x)
{
    /* plain bit loop: obviously correct, no intrinsics */
    int c = 0;
    while (x) {
        x &= x - 1;
        ++c;
    }
    return c;
}

static int popcount_words(const uint64_t *w, int n)
{
    int c = 0;
    for (int i = 0; i < n; ++i) c += popcount64(w[i]);
    return c;
}

static int any_words(const uint64_t *w, int n)
{
    for (int i = 0; i < n; ++i)
        if (w[i]) return 1;
    return 0;
}

static void full_mask(uint64_t *w, int nwords, int nbits)
{
    for (int i = 0; i < nwords; ++i) {
        const int lo = i * 64;
        const int rem = nbits - lo;
        w[i] = rem >= 64 ? ~0ULL : (rem <= 0 ? 0ULL : ((1ULL << rem) - 1ULL));
    }
}

static int check_args(const uint64_t *bm, int G, int Nt, int Nn, int h, int64_t a_num, int64_t a_den)
{
    if (G < 0 || Nt < 0 || Nn < 0 || h < 1 || h > ORACLE_MAX_H) return ORACLE_EINVAL;
    if (a_num < 0 || a_den <= 0 || a_num > 0x7fffffff || a_den > 0x7fffffff) return ORACLE_EINVAL;
    if (G > 0 && !bm) return ORACLE_EINVAL;
    return ORACLE_OK;
}

/* lexicographic compare of two ascending tuples of length h */
static int tuple_less(const int32_t *a, const int32_t *b, int h)
{
    for (int i = 0; i < h; ++i) {
        if (a[i] != b[i]) return a[i] < b[i];
    }
    return 0;
}

static void sort_tuple(int32_t *t, int h)
{
    for (int i = 1; i < h; ++i) {
        int32_t v = t[i];
        int j = i - 1;
        while (j >= 0 && t[j] > v) {
            t[j + 1] = t[j];
            --j;
        }
        t[j + 1] = v;
    }
}

/* ------------------------------------------------------------------------ */
/* Brute force: the definition.                                              */

int oracle_bruteforce(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, int32_t h,
                      int64_t a_num, int64_t a_den, int32_t max_rounds, int32_t cap,
                      int32_t *genes, int32_t *tp, int32_t *fp, int32_t *k_out)
{
    int rc = check_args(bm, G, Nt, Nn, h, a_num, a_den);
    if (rc) return rc;
    const int Wt = (Nt + 63) / 64, Wn = (Nn + 63) / 64, W = Wt + Wn;
    uint64_t *U = calloc((size_t)Wt + 1, sizeof(uint64_t));
    uint64_t *y = calloc((size_t)Wt + 1, sizeof(uint64_t));
    uint64_t *n = calloc((size_t)Wn + 1, sizeof(uint64_t));
    uint64_t *ybest = calloc((size_t)Wt + 1, sizeof(uint64_t));
    if (!U || !y || !n || !ybest) {
        free(U); free(y); free(n); free(ybest);
        return ORACLE_ENOMEM;
    }
    full_mask(U, Wt, Nt);
    int k = 0;
    rc = ORACLE_OK;
    for (int round = 0; max_rounds < 0 || round < max_rounds; ++round) {
        if (!any_words(U, Wt)) break; /* C = T: every tumor covered */
        if (G < h) break;
        int32_t c[ORACLE_MAX_H], best[ORACLE_MAX_H];
        for (int i = 0; i < h; ++i) c[i] = i; /* first h-subset in lex order */
        int have = 0;
        int64_t best_s = 0;
        int best_tp = 0, best_fp = 0;
        for (;;) {
            /* cover of c over the uncovered tumors and over the normals */
            memcpy(y, U, sizeof(uint64_t) * (size_t)Wt);
            full_mask(n, Wn, Nn);
            for (int i = 0; i < h; ++i) {
                const uint64_t *row = bm + (size_t)c[i] * W;
                for (int w = 0; w < Wt; ++w) y[w] &= row[w];
                for (int w = 0; w < Wn; ++w) n[w] &= row[Wt + w];
            }
            const int TP = popcount_words(y, Wt);
            if (TP > 0) {
                const int FP = popcount_words(n, Wn);
                const int64_t S = a_num * (int64_t)TP + a_den * (int64_t)(Nn - FP);
                if (!have || S > best_s) {
                    have = 1;
                    best_s = S;
                    best_tp = TP;
                    best_fp = FP;
                    memcpy(best, c, sizeof(int32_t) * (size_t)h);
                    memcpy(ybest, y, sizeof(uint64_t) * (size_t)Wt);
                }
            }
            /* next h-subset in lexicographic order */
            int i = h - 1;
            while (i >= 0 && c[i] == G - h + i) --i;
            if (i < 0) break;
            ++c[i];
            for (int j = i + 1; j < h; ++j) c[j] = c[j - 1] + 1;
        }
        if (!have) break; /* no combination covers an uncovered tumor */
        if (k >= cap) { rc = ORACLE_ECAP; break; }
        memcpy(genes + (size_t)k * h, best, sizeof(int32_t) * (size_t)h);
        tp[k] = best_tp;
        fp[k] = best_fp;
        ++k;
        for (int w = 0; w < Wt; ++w) U[w] &= ~ybest[w]; /* DelCols on the tumors */
    }
    *k_out = k;
    free(U); free(y); free(n); free(ybest);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* P-DFS.                                                                    */

typedef struct {
    const uint64_t *bm;
    int G, Nt, Nn, h, Wt, Wn, W, prune;
    int64_t a_num, a_den;
    const int32_t *order; /* order[i] = original index of the i-th gene in search order */
    uint64_t *ystack;     /* (h+1) x Wt : y_0 = U, y_1 .. y_h */
    uint64_t *nstack;     /* (h+1) x Wn */
    int32_t path[ORACLE_MAX_H];
    uint64_t *visited, *pruned; /* h counters of this round */
    int have;
    int64_t best_s;
    int best_tp, best_fp;
    int32_t best[ORACLE_MAX_H]; /* ascending original indices */
} pdfs_state;

static void pdfs_level(pdfs_state *st, int level /* 1-based */, int first /* 0-based */)
{
    const int h = st->h, Wt = st->Wt, Wn = st->Wn;
    const int last = st->G - h + level - 1; /* 0-based inclusive bound */
    const uint64_t *yp = st->ystack + (size_t)(level - 1) * Wt;
    const uint64_t *np = st->nstack + (size_t)(level - 1) * Wn;
    uint64_t *yc = st->ystack + (size_t)level * Wt;
    uint64_t *nc = st->nstack + (size_t)level * Wn;
    for (int g = first; g <= last; ++g) {
        const uint64_t *row = st->bm + (size_t)st->order[g] * st->W;
        for (int w = 0; w < Wt; ++w) yc[w] = yp[w] & row[w];
        for (int w = 0; w < Wn; ++w) nc[w] = np[w] & row[Wt + w];
        st->path[level - 1] = g;
        st->visited[level - 1] += 1;
        const int empty = !any_words(yc, Wt);
        if (empty) {
            st->pruned[level - 1] += 1;
            if (st->prune) continue; /* backtrack: the whole subtree is empty */
        }
        if (level < h) {
            pdfs_level(st, level + 1, g + 1);
            continue;
        }
        if (empty) continue; /* TP = 0: not a candidate */
        const int TP = popcount_words(yc, Wt);
        const int FP = popcount_words(nc, Wn);
        const int64_t S = st->a_num * (int64_t)TP + st->a_den * (int64_t)(st->Nn - FP);
        if (st->have && S < st->best_s) continue;
        int32_t t[ORACLE_MAX_H];
        for (int i = 0; i < h; ++i) t[i] = st->order[st->path[i]];
        sort_tuple(t, h);
        if (!st->have || S > st->best_s || tuple_less(t, st->best, h)) {
            st->have = 1;
            st->best_s = S;
            st->best_tp = TP;
            st->best_fp = FP;
            memcpy(st->best, t, sizeof(int32_t) * (size_t)h);
        }
    }
}

/* order genes from most sparse to least sparse: ascending tumor popcount, ties by index */
static const uint64_t *g_sort_bm;
static int g_sort_W, g_sort_Wt;
static int cmp_sparsity(const void *pa, const void *pb)
{
    const int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    const int ca = popcount_words(g_sort_bm + (size_t)a * g_sort_W, g_sort_Wt);
    const int cb = popcount_words(g_sort_bm + (size_t)b * g_sort_W, g_sort_Wt);
    if (ca != cb) return ca < cb ? -1 : 1;
    return (a > b) - (a < b);
}

int oracle_sparsity_order(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, int32_t *order)
{
    if (G < 0 || Nt < 0 || Nn < 0 || (G > 0 && !bm)) return ORACLE_EINVAL;
    for (int i = 0; i < G; ++i) order[i] = i;
    g_sort_bm = bm;
    g_sort_Wt = (Nt + 63) / 64;
    g_sort_W = g_sort_Wt + (Nn + 63) / 64;
    qsort(order, (size_t)G, sizeof(int32_t), cmp_sparsity);
    return ORACLE_OK;
}

/*
 * visited / pruned: (max rounds actually run) x h counters, row r = round r.
 * Both arrays must hold cap_rounds * h entries; rounds_out receives the number
 * of P-DFS rounds run (k, or k + 1 when the last round found no candidate).
 */
int oracle_pdfs(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, int32_t h,
                int64_t a_num, int64_t a_den, int32_t prune, int32_t sort, int32_t max_rounds,
                int32_t cap, int32_t *genes, int32_t *tp, int32_t *fp, int32_t *k_out,
                int32_t cap_rounds, uint64_t *visited, uint64_t *pruned, int32_t *rounds_out)
{
    int rc = check_args(bm, G, Nt, Nn, h, a_num, a_den);
    if (rc) return rc;
    pdfs_state st;
    memset(&st, 0, sizeof st);
    st.bm = bm;
    st.G = G; st.Nt = Nt; st.Nn = Nn; st.h = h;
    st.Wt = (Nt + 63) / 64; st.Wn = (Nn + 63) / 64; st.W = st.Wt + st.Wn;
    st.prune = prune;
    st.a_num = a_num; st.a_den = a_den;
    int32_t *order = malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    st.ystack = calloc((size_t)(h + 1) * (size_t)st.Wt + 1, sizeof(uint64_t));
    st.nstack = calloc((size_t)(h + 1) * (size_t)st.Wn + 1, sizeof(uint64_t));
    uint64_t *ybest = calloc((size_t)st.Wt + 1, sizeof(uint64_t));
    if (!order || !st.ystack || !st.nstack || !ybest) {
        free(order); free(st.ystack); free(st.nstack); free(ybest);
        return ORACLE_ENOMEM;
    }
    if (sort) {
        oracle_sparsity_order(bm, G, Nt, Nn, order);
    } else {
        for (int i = 0; i < G; ++i) order[i] = i;
    }
    st.order = order;
    uint64_t *U = st.ystack; /* y_0 */
    full_mask(U, st.Wt, Nt);
    full_mask(st.nstack, st.Wn, Nn); /* n_0 = all normals */
    int k = 0, rounds = 0;
    rc = ORACLE_OK;
    for (int round = 0; max_rounds < 0 || round < max_rounds; ++round) {
        if (!any_words(U, st.Wt)) break;
        if (rounds >= cap_rounds) { rc = ORACLE_ECAP; break; }
        st.visited = visited + (size_t)rounds * h;
        st.pruned = pruned + (size_t)rounds * h;
        memset(st.visited, 0, sizeof(uint64_t) * (size_t)h);
        memset(st.pruned, 0, sizeof(uint64_t) * (size_t)h);
        ++rounds;
        st.have = 0;
        if (G >= h) pdfs_level(&st, 1, 0);
        if (!st.have) break;
        if (k >= cap) { rc = ORACLE_ECAP; break; }
        memcpy(genes + (size_t)k * h, st.best, sizeof(int32_t) * (size_t)h);
        tp[k] = st.best_tp;
        fp[k] = st.best_fp;
        ++k;
        /* DelCols: clear the tumors covered by the chosen combination */
        full_mask(ybest, st.Wt, Nt);
        for (int i = 0; i < h; ++i) {
            const uint64_t *row = bm + (size_t)st.best[i] * st.W;
            for (int w = 0; w < st.Wt; ++w) ybest[w] &= row[w];
        }
        for (int w = 0; w < st.Wt; ++w) U[w] &= ~ybest[w];
    }
    *k_out = k;
    *rounds_out = rounds;
    free(order); free(st.ystack); free(st.nstack); free(ybest);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Point evaluation: TP / FP of given combinations against an uncovered mask, */
/* for checking sampled outputs of solves too large to enumerate.            */

int oracle_cover_counts(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, int32_t h,
                        const uint64_t *U, int32_t n_combos, const int32_t *genes,
                        int32_t *tp, int32_t *fp)
{
    if (G < 0 || Nt < 0 || Nn < 0 || h < 1 || h > ORACLE_MAX_H) return ORACLE_EINVAL;
    const int Wt = (Nt + 63) / 64, Wn = (Nn + 63) / 64, W = Wt + Wn;
    uint64_t *y = calloc((size_t)Wt + 1, sizeof(uint64_t));
    uint64_t *n = calloc((size_t)Wn + 1, sizeof(uint64_t));
    if (!y || !n) { free(y); free(n); return ORACLE_ENOMEM; }
    for (int c = 0; c < n_combos; ++c) {
        memcpy(y, U, sizeof(uint64_t) * (size_t)Wt);
        full_mask(n, Wn, Nn);
        for (int i = 0; i < h; ++i) {
            const int32_t g = genes[(size_t)c * h + i];
            if (g < 0 || g >= G) { free(y); free(n); return ORACLE_EINVAL; }
            const uint64_t *row = bm + (size_t)g * W;
            for (int w = 0; w < Wt; ++w) y[w] &= row[w];
            for (int w = 0; w < Wn; ++w) n[w] &= row[Wt + w];
        }
        tp[c] = popcount_words(y, Wt);
        fp[c] = popcount_words(n, Wn);
    }
    free(y); free(n);
    return ORACLE_OK;
}
