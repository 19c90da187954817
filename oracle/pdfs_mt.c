/*
 * Threaded CPU P-DFS for the multi-hit greedy weighted set cover.
 *
 * TEST INFRASTRUCTURE ONLY, like oracle.c: only tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code; the CUDA library never does,
 * and the two share nothing.  It is a second CPU implementation of the same
 * search, checked against oracle_pdfs and oracle_bruteforce by the CPU tests:
 *
 *   - the paper's parallel scheme run on the host's cores (§III-E): the depth-1
 *     subtrees of a round are the units of work, handed out one at a time by an
 *     atomic counter (the master's chunked dispatch), each worker thread runs
 *     Algorithm 2 below the genes it draws, and the per-worker best candidates
 *     and counters are reduced at the end of the round;
 *   - a shard option that searches only the depth-1 genes g (search order) with
 *     g % nshards == shard, so that several processes can split one round and
 *     merge their results (largest key, summed counters) before every one of
 *     them applies the same DelCols -- the per-round exchange of a multi-process
 *     solve;
 *   - a score-bound mode (an addition; the paper states no branch and bound,
 *     §II-B): a non-empty prefix with tumor intersection y can only lead to
 *     leaves with TP <= |y| and FP >= 0, so their scores are at most
 *     a_num * |y| + a_den * Nn (Eq. 1 and the score of §II-B).  When that bound
 *     is below the best score already found in the round (strictly: an equal
 *     score could still win on the tuple order), the prefix's subtree is cut.
 *     The selections are unchanged; the counters then depend on the order in
 *     which the threads found their candidates and are reported as they came.
 *
 * Same input layout, readings and outputs as oracle_pdfs (see oracle.c): genes
 * searched in the sparsity order of §III-C, loop bounds (g_{l-1}, G - h + l]
 * (1-based), pruning of empty tumor intersections with the uncovered tumors at
 * every depth, TP = 0 leaves not candidates, scores S = a_num TP + a_den (Nn - FP),
 * ties to the lexicographically smallest tuple of original indices.
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MT_MAX_H 9
#define MT_MAX_THREADS 256

enum { MT_OK = 0, MT_EINVAL = 1, MT_ENOMEM = 3, MT_ECAP = 8 };
enum { MT_PRUNE_OFF = 0, MT_PRUNE_PAPER = 1, MT_PRUNE_BOUND = 2 };

typedef struct {
    const uint64_t *bm;
    int G, Nt, Nn, h, Wt, Wn, W, prune;
    int64_t a_num, a_den;
    const int32_t *order; /* search position -> original index */
    const uint64_t *U;    /* uncovered tumors */
    int shard, nshards;
    atomic_int next;      /* next depth-1 unit to hand out */
    atomic_llong best_known; /* largest score found so far in the round (bound mode), -1: none */
} mt_round_ctx;

typedef struct {
    mt_round_ctx *rc;
    uint64_t *ystack, *nstack;
    int32_t path[MT_MAX_H];
    uint64_t visited[MT_MAX_H], pruned[MT_MAX_H], cut[MT_MAX_H];
    int have;
    int64_t best_s;
    int best_tp, best_fp;
    int32_t best[MT_MAX_H];
} mt_worker;

static int mt_popcount_words(const uint64_t *w, int n)
{
    int c = 0;
    for (int i = 0; i < n; ++i) c += __builtin_popcountll(w[i]);
    return c;
}

static int mt_tuple_less(const int32_t *a, const int32_t *b, int h)
{
    for (int i = 0; i < h; ++i)
        if (a[i] != b[i]) return a[i] < b[i];
    return 0;
}

static void mt_sort_tuple(int32_t *t, int h)
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

static void mt_publish(mt_round_ctx *rc, int64_t s)
{
    long long cur = atomic_load(&rc->best_known);
    while (s > cur && !atomic_compare_exchange_weak(&rc->best_known, &cur, (long long)s)) {
    }
}

/* Algorithm 2 below a node of depth level - 1 whose intersections sit in the
 * worker's stacks at index level - 1; children g in [first, G - h + level - 1]. */
static void mt_level(mt_worker *wk, int level, int first)
{
    mt_round_ctx *rc = wk->rc;
    const int h = rc->h, Wt = rc->Wt, Wn = rc->Wn;
    const int last = rc->G - h + level - 1;
    const uint64_t *yp = wk->ystack + (size_t)(level - 1) * Wt;
    const uint64_t *np = wk->nstack + (size_t)(level - 1) * Wn;
    uint64_t *yc = wk->ystack + (size_t)level * Wt;
    uint64_t *nc = wk->nstack + (size_t)level * Wn;
    for (int g = first; g <= last; ++g) {
        if (level == 1 && g != first) break; /* depth 1: one unit (one gene) per call */
        const uint64_t *row = rc->bm + (size_t)rc->order[g] * rc->W;
        uint64_t any = 0;
        for (int w = 0; w < Wt; ++w) {
            yc[w] = yp[w] & row[w];
            any |= yc[w];
        }
        for (int w = 0; w < Wn; ++w) nc[w] = np[w] & row[Wt + w];
        wk->path[level - 1] = g;
        wk->visited[level - 1] += 1;
        if (!any) {
            wk->pruned[level - 1] += 1;
            if (rc->prune != MT_PRUNE_OFF) continue;
        }
        if (level < h) {
            if (rc->prune == MT_PRUNE_BOUND) {
                const int ky = mt_popcount_words(yc, Wt);
                const int64_t ub = rc->a_num * (int64_t)ky + rc->a_den * (int64_t)rc->Nn;
                if (ub < (int64_t)atomic_load(&rc->best_known)) {
                    wk->cut[level - 1] += 1;
                    continue;
                }
            }
            mt_level(wk, level + 1, g + 1);
            continue;
        }
        if (!any) continue; /* TP = 0: not a candidate */
        const int ky = mt_popcount_words(yc, Wt);
        const int FP = mt_popcount_words(nc, Wn);
        const int64_t S = rc->a_num * (int64_t)ky + rc->a_den * (int64_t)(rc->Nn - FP);
        if (wk->have && S < wk->best_s) continue;
        int32_t t[MT_MAX_H];
        for (int i = 0; i < h; ++i) t[i] = rc->order[wk->path[i]];
        mt_sort_tuple(t, h);
        if (!wk->have || S > wk->best_s || mt_tuple_less(t, wk->best, h)) {
            wk->have = 1;
            wk->best_s = S;
            wk->best_tp = ky;
            wk->best_fp = FP;
            memcpy(wk->best, t, sizeof(int32_t) * (size_t)h);
            if (rc->prune == MT_PRUNE_BOUND) mt_publish(rc, S);
        }
    }
}

static void *mt_worker_main(void *arg)
{
    mt_worker *wk = (mt_worker *)arg;
    mt_round_ctx *rc = wk->rc;
    const int last1 = rc->G - rc->h; /* 0-based bound of depth 1 */
    for (;;) {
        /* unit u -> the u-th depth-1 gene of this shard */
        const int u = atomic_fetch_add(&rc->next, 1);
        const long long g = (long long)u * rc->nshards + rc->shard;
        if (g > last1) break;
        mt_level(wk, 1, (int)g);
    }
    return NULL;
}

/*
 * One greedy round's search (step F of Algorithm 1) over the uncovered tumors U,
 * restricted to shard `shard` of `nshards` (depth-1 genes g with
 * g % nshards == shard, search order), on `nthreads` threads.  order: the search
 * order (search position -> original index).  Outputs: *have = 1 and the best
 * candidate (score, ascending original tuple, TP, FP) if one exists in the shard;
 * visited / pruned / cut: h counters each (cut: subtrees cut by the score bound).
 */
int pdfs_mt_round(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, int32_t h, int64_t a_num,
                  int64_t a_den, int32_t prune, const int32_t *order, const uint64_t *U, int32_t nthreads,
                  int32_t shard, int32_t nshards, int32_t *have, int64_t *score, int32_t *tuple, int32_t *tp,
                  int32_t *fp, uint64_t *visited, uint64_t *pruned, uint64_t *cut)
{
    if (G < 0 || Nt < 0 || Nn < 0 || h < 1 || h > MT_MAX_H || a_num < 0 || a_den <= 0) return MT_EINVAL;
    if (prune < MT_PRUNE_OFF || prune > MT_PRUNE_BOUND) return MT_EINVAL;
    if (nshards < 1 || shard < 0 || shard >= nshards) return MT_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > MT_MAX_THREADS) nthreads = MT_MAX_THREADS;
    mt_round_ctx rc;
    memset(&rc, 0, sizeof rc);
    rc.bm = bm;
    rc.G = G; rc.Nt = Nt; rc.Nn = Nn; rc.h = h;
    rc.Wt = (Nt + 63) / 64; rc.Wn = (Nn + 63) / 64; rc.W = rc.Wt + rc.Wn;
    rc.prune = prune;
    rc.a_num = a_num; rc.a_den = a_den;
    rc.order = order;
    rc.U = U;
    rc.shard = shard; rc.nshards = nshards;
    atomic_init(&rc.next, 0);
    atomic_init(&rc.best_known, -1);
    mt_worker *wk = calloc((size_t)nthreads, sizeof(mt_worker));
    pthread_t *th = calloc((size_t)nthreads, sizeof(pthread_t));
    int rcode = (wk && th) ? MT_OK : MT_ENOMEM;
    for (int i = 0; rcode == MT_OK && i < nthreads; ++i) {
        wk[i].rc = &rc;
        wk[i].ystack = calloc((size_t)(h + 1) * (size_t)rc.Wt + 1, sizeof(uint64_t));
        wk[i].nstack = calloc((size_t)(h + 1) * (size_t)rc.Wn + 1, sizeof(uint64_t));
        if (!wk[i].ystack || !wk[i].nstack) { rcode = MT_ENOMEM; break; }
        memcpy(wk[i].ystack, U, sizeof(uint64_t) * (size_t)rc.Wt); /* y_0 = U */
        for (int w = 0; w < rc.Wn; ++w) {                           /* n_0 = all normals */
            const int rem = Nn - 64 * w;
            wk[i].nstack[w] = rem >= 64 ? ~0ULL : ((1ULL << rem) - 1ULL);
        }
    }
    int started = 0;
    if (rcode == MT_OK && G >= h) {
        for (int i = 1; i < nthreads; ++i) {
            if (pthread_create(&th[i], NULL, mt_worker_main, &wk[i]) != 0) break;
            ++started;
        }
        mt_worker_main(&wk[0]);
        for (int i = 1; i <= started; ++i) pthread_join(th[i], NULL);
    }
    *have = 0;
    memset(visited, 0, sizeof(uint64_t) * (size_t)h);
    memset(pruned, 0, sizeof(uint64_t) * (size_t)h);
    memset(cut, 0, sizeof(uint64_t) * (size_t)h);
    for (int i = 0; rcode == MT_OK && i < nthreads; ++i) {
        for (int l = 0; l < h; ++l) {
            visited[l] += wk[i].visited[l];
            pruned[l] += wk[i].pruned[l];
            cut[l] += wk[i].cut[l];
        }
        if (!wk[i].have) continue;
        if (!*have || wk[i].best_s > *score ||
            (wk[i].best_s == *score && mt_tuple_less(wk[i].best, tuple, h))) {
            *have = 1;
            *score = wk[i].best_s;
            *tp = wk[i].best_tp;
            *fp = wk[i].best_fp;
            memcpy(tuple, wk[i].best, sizeof(int32_t) * (size_t)h);
        }
    }
    for (int i = 0; wk && i < nthreads; ++i) {
        free(wk[i].ystack);
        free(wk[i].nstack);
    }
    free(wk);
    free(th);
    return rcode;
}

/* DelCols of Algorithm 1: clear from U the tumors that carry every gene of tuple. */
int pdfs_mt_delcols(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, int32_t h, const int32_t *tuple,
                    uint64_t *U)
{
    if (G < 0 || Nt < 0 || Nn < 0 || h < 1 || h > MT_MAX_H) return MT_EINVAL;
    const int Wt = (Nt + 63) / 64, W = Wt + (Nn + 63) / 64;
    for (int w = 0; w < Wt; ++w) {
        uint64_t y = U[w];
        for (int i = 0; i < h; ++i) {
            if (tuple[i] < 0 || tuple[i] >= G) return MT_EINVAL;
            y &= bm[(size_t)tuple[i] * W + w];
        }
        U[w] &= ~y;
    }
    return MT_OK;
}

static const uint64_t *mt_sort_bm;
static int mt_sort_W, mt_sort_Wt;
static int mt_cmp_sparsity(const void *pa, const void *pb)
{
    const int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    const int ca = mt_popcount_words(mt_sort_bm + (size_t)a * mt_sort_W, mt_sort_Wt);
    const int cb = mt_popcount_words(mt_sort_bm + (size_t)b * mt_sort_W, mt_sort_Wt);
    if (ca != cb) return ca < cb ? -1 : 1;
    return (a > b) - (a < b);
}

/*
 * The whole greedy loop (Algorithm 1) with every round searched by pdfs_mt_round
 * on one shard (nshards = 1).  Outputs as oracle_pdfs, plus cut (per round, per
 * depth).  Not thread-safe (the sort uses file-scope state).
 */
int pdfs_mt_solve(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, int32_t h, int64_t a_num,
                  int64_t a_den, int32_t prune, int32_t max_rounds, int32_t nthreads, int32_t cap, int32_t *genes,
                  int32_t *tp, int32_t *fp, int32_t *k_out, int32_t cap_rounds, uint64_t *visited,
                  uint64_t *pruned, uint64_t *cut, int32_t *rounds_out)
{
    if (G < 0 || Nt < 0 || Nn < 0 || h < 1 || h > MT_MAX_H || a_num < 0 || a_den <= 0) return MT_EINVAL;
    const int Wt = (Nt + 63) / 64;
    int32_t *order = malloc(sizeof(int32_t) * (size_t)(G > 0 ? G : 1));
    uint64_t *U = calloc((size_t)Wt + 1, sizeof(uint64_t));
    if (!order || !U) { free(order); free(U); return MT_ENOMEM; }
    for (int i = 0; i < G; ++i) order[i] = i;
    mt_sort_bm = bm;
    mt_sort_Wt = Wt;
    mt_sort_W = Wt + (Nn + 63) / 64;
    qsort(order, (size_t)G, sizeof(int32_t), mt_cmp_sparsity);
    for (int w = 0; w < Wt; ++w) {
        const int rem = Nt - 64 * w;
        U[w] = rem >= 64 ? ~0ULL : ((1ULL << rem) - 1ULL);
    }
    int k = 0, rounds = 0, rc = MT_OK;
    for (int round = 0; max_rounds < 0 || round < max_rounds; ++round) {
        int any = 0;
        for (int w = 0; w < Wt; ++w) any |= U[w] != 0;
        if (!any) break;
        if (rounds >= cap_rounds) { rc = MT_ECAP; break; }
        int32_t have = 0, t[MT_MAX_H], btp = 0, bfp = 0;
        int64_t S = 0;
        rc = pdfs_mt_round(bm, G, Nt, Nn, h, a_num, a_den, prune, order, U, nthreads, 0, 1, &have, &S, t, &btp,
                           &bfp, visited + (size_t)rounds * h, pruned + (size_t)rounds * h,
                           cut + (size_t)rounds * h);
        if (rc) break;
        ++rounds;
        if (!have) break;
        if (k >= cap) { rc = MT_ECAP; break; }
        memcpy(genes + (size_t)k * h, t, sizeof(int32_t) * (size_t)h);
        tp[k] = btp;
        fp[k] = bfp;
        ++k;
        pdfs_mt_delcols(bm, G, Nt, Nn, h, t, U);
    }
    *k_out = k;
    *rounds_out = rounds;
    free(order);
    free(U);
    return rc;
}
