/*
 * mh.h -- C ABI of the GB300 multi-hit weighted-set-cover library (libmh).
 *
 * The library finds multi-hit gene combinations with the greedy weighted set
 * cover of Dash et al. as used by the paper (Algorithm 1), whose argmax step is
 * evaluated by Pruned Depth-First Search (P-DFS, §III-D, Algorithm 2) over
 * bit-packed gene x sample mutation bitmaps.  All arithmetic is exact integer
 * arithmetic; every step of a solve runs in the library's own CUDA kernels.
 *
 * Conventions shared by every entry point
 *   - Status: every call returns MH_OK (0) or one of the MH_E* codes below; a
 *     readable message for the calling thread is available from mh_last_error().
 *     No entry point exits, traps or aborts the process.
 *   - Bitmap layout ("packed rows"): gene-major, one row per gene,
 *       row g = [Wt tumor words | Wn normal words],  Wt = ceil(Nt/64), Wn = ceil(Nn/64),
 *     as uint64_t; sample s of a block is bit (s % 64) of word (s / 64), least
 *     significant bit first; bits at and past Nt (resp. Nn) must be zero.
 *     Bit x[g][s] = 1 means sample s carries a mutation in gene g (§II-B).
 *   - Gene indices in results are the caller's row indices ("original" indices),
 *     ascending inside each combination.
 *   - Limits: 1 <= G <= 65535, 0 <= Nt <= 2048, 0 <= Nn <= 2048, 1 <= h <= 9.
 *   - Streams: a handle runs all its work on one CUDA stream (the legacy default
 *     stream unless one is given).  Handles are not thread-safe; distinct handles
 *     may be used from distinct threads.
 */
#ifndef MH_H
#define MH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MH_API __attribute__((visibility("default")))
#else
#define MH_API
#endif

/* status codes */
#define MH_OK 0
#define MH_EINVAL 1   /* bad argument: sizes out of range, h outside [1, 9], den <= 0, non-zero padding bits */
#define MH_ENOMEM 2   /* a host or device allocation failed, or the frontier budget was exceeded */
#define MH_ECUDA 3    /* a CUDA runtime call failed (the message names it) */
#define MH_ETIMEOUT 4 /* a bounded device-side wait expired; the kernel returned early */
#define MH_EAGAIN 5   /* the result is not ready yet (served mode) */
#define MH_EREJECT 6  /* a request does not fit the server's memory budget */
#define MH_ECANCELED 7 /* a served request was cancelled (mh_cancel) */

#define MH_MAX_H 9

typedef struct mh_handle mh_handle;

/* alpha = num / den of the weight function F (§II-B; the paper's usual 0.1 is {1, 10}).
 * Requires 0 <= num and 0 < den, both below 2^31. */
typedef struct {
    int32_t num;
    int32_t den;
} mh_rational;

/* Pruning mode of the search.
 *   MH_PRUNE_PAPER: cut every prefix whose tumor intersection with the still
 *                   uncovered tumors is empty, at every depth (§III-D).
 *   MH_PRUNE_OFF:   exhaustive enumeration of every h-subset (the paper's
 *                   BOUND=OFF baseline); the result is identical, the counters
 *                   are the closed forms C(G-h+l, l).
 *   MH_PRUNE_BOUND: paper pruning plus a score bound, an addition (the paper uses
 *                   no branch and bound, §II-B): a non-empty prefix with tumor
 *                   intersection y can only lead to leaves scoring at most
 *                   alpha.num * |y| + alpha.den * Nn (TP <= |y|, FP >= 0 in the
 *                   score of §II-B), so it is cut when that bound is below the
 *                   score of a candidate already found in the round (strictly:
 *                   an equal score could still win on the tuple order).  The
 *                   selections are those of MH_PRUNE_PAPER; visited / pruned
 *                   count the nodes the bounded search computed and cut counts
 *                   the prefixes it cut, both depending on when candidates were
 *                   found (not reproducible from run to run). */
#define MH_PRUNE_PAPER 0
#define MH_PRUNE_OFF 1
#define MH_PRUNE_BOUND 2

/* Execution of a solve.
 *   MH_MODE_PERSISTENT: one cooperative kernel runs every round, its phases
 *                       separated by grid barriers (default; falls back to
 *                       MH_MODE_LAUNCHES where cooperative launch is unavailable).
 *   MH_MODE_LAUNCHES:   one kernel launch per phase of every round. */
#define MH_MODE_PERSISTENT 0
#define MH_MODE_LAUNCHES 1

/* Options of a solve; zero-initialise and set what you need. */
typedef struct {
    int32_t h;            /* hits per combination, 1..9 */
    mh_rational alpha;    /* weight of true positives */
    int32_t prune;        /* MH_PRUNE_PAPER (default 0), MH_PRUNE_OFF or MH_PRUNE_BOUND */
    int32_t max_rounds;   /* stop after this many greedy rounds; <= 0 means no limit */
    int32_t time_kernels; /* non-zero: time every kernel launch with CUDA events */
    int32_t mode;         /* MH_MODE_PERSISTENT (default 0) or MH_MODE_LAUNCHES */
} mh_solve_opts;

/* Result of a solve, allocated by the library; release with mh_result_free.
 * Round r of the greedy loop searched the tree once; visited[r*h + l-1] counts the
 * depth-l nodes whose intersection was computed, pruned[r*h + l-1] those found
 * empty (scored leaves = visited - pruned at l = h).  rounds = k, or k + 1 when
 * the last round found no combination covering an uncovered tumor. */
typedef struct {
    int32_t h;
    int32_t k;           /* number of selected combinations */
    int32_t rounds;      /* greedy rounds searched */
    int32_t *genes;      /* k*h original gene indices, ascending per combination */
    int32_t *tp;         /* k: uncovered tumors covered when selected */
    int32_t *fp;         /* k: normals covered */
    uint64_t *visited;   /* rounds*h */
    uint64_t *pruned;    /* rounds*h */
    double solve_ms;     /* wall time of the solve measured with CUDA events on the handle's stream */
    double leaf_ms;      /* summed duration of the leaf phase (see level1_ms) */
    int64_t leaf_launches;   /* leaf-kernel launches in this solve */
    int64_t kernel_launches; /* all kernel launches of this solve */
    uint64_t leaf_words;     /* 64-bit sample-major column words read by the leaf kernel */
    uint64_t leaf_prefixes;  /* prefixes (depth h-1 nodes) the leaf kernel expanded */
    uint64_t leaf_scored;    /* leaves whose TP / FP the leaf kernel evaluated exactly */
    uint64_t leaf_alu_ops;   /* 32-bit integer operations of the leaf kernel's tests and scores */
    uint64_t leaf_dense;     /* prefixes the leaf kernel took on its row (dense) path */
    double level1_ms;        /* summed durations of the depth-1, frontier-expansion and */
    double expand_ms;        /* end-of-round phases: CUDA events around each kernel with */
    double finalize_ms;      /* time_kernels (launch mode), the device clock (persistent mode) */
    int32_t mode;            /* the mode that ran (MH_MODE_*) */
    uint64_t diag[8];        /* diagnostics, [expansion, leaf]: summed warp cycles, summed per-round
                                longest warp cycles, warp count (indices 0-1, 2-3, 4-5); a batched
                                result's diag[6] is 1 if every launch numbered its blocks SM-major,
                                diag[7] is 1 if its first launch ran from a captured CUDA graph */
    double kernel_ms;        /* persistent mode: the solve kernel's own duration (CUDA events around
                                each cooperative launch, summed over relaunches); launch mode with
                                time_kernels: the four phase times summed; else 0 */
    uint64_t *cut;           /* rounds*h: MH_PRUNE_BOUND, the depth-l prefixes cut by the score bound
                                (cut[r*h + l-1]); zero in the other modes */
} mh_result;

/* Create a handle for one cohort from packed rows in HOST memory.
 * bitmaps: G * (Wt + Wn) uint64_t words (see layout above); copied, the caller
 * keeps ownership.  The library sorts genes from most to least sparse (§III-C,
 * ascending tumor mutation count, ties by row index), uploads the sorted rows and
 * a sample-major copy of the tumor bits, and owns that device memory until
 * mh_destroy.  Errors: MH_EINVAL (NULL pointers, sizes out of range, padding bits
 * set), MH_ENOMEM, MH_ECUDA.  On error *out is set to NULL. */
MH_API int mh_create(const uint64_t *bitmaps, int32_t G, int32_t Nt, int32_t Nn, mh_handle **out);

/* Same as mh_create, with the packed rows in DEVICE memory (e.g. a torch tensor's
 * data pointer) and the CUDA stream (a cudaStream_t, or NULL for the legacy
 * default stream) that the handle will use.  The rows are read once, during this
 * call; the caller keeps ownership. */
MH_API int mh_create_device(const uint64_t *d_bitmaps, int32_t G, int32_t Nt, int32_t Nn, void *stream,
                            mh_handle **out);

/* Select the CUDA stream (cudaStream_t or NULL) used by later calls on the handle. */
MH_API int mh_set_stream(mh_handle *handle, void *stream);

/* Run the greedy loop (Algorithm 1) to completion: every round evaluates
 * argmax_gamma F(gamma) by P-DFS on the device, appends the winner and clears the
 * tumors it covers, until every tumor is covered or no h-combination covers an
 * uncovered tumor.  Scores are compared as the integers
 *   S = alpha.num * TP + alpha.den * (Nn - FP)
 * (F scaled by alpha.den * (Nt + Nn)); equal scores go to the lexicographically
 * smallest tuple of original indices.  Synchronous: returns when the result is on
 * the host.  Each call starts from "no tumor covered".  *out receives a result to
 * release with mh_result_free.  Errors: MH_EINVAL, MH_ENOMEM, MH_ECUDA,
 * MH_ETIMEOUT. */
MH_API int mh_solve(mh_handle *handle, int32_t h, mh_rational alpha, mh_result **out);

/* mh_solve with options (pruning mode, round limit, kernel timing). */
MH_API int mh_solve_ex(mh_handle *handle, const mh_solve_opts *opts, mh_result **out);

MH_API void mh_result_free(mh_result *result);
MH_API void mh_destroy(mh_handle *handle);

/* Message of the last error on the calling thread ("" if none). */
MH_API const char *mh_last_error(void);

/* Diagnostic (no counterpart in the paper): checks the bounded device-side wait
 * that every barrier of the persistent kernels uses.  One block enters a barrier
 * that no other block reaches; the wait gives up after its bound (about two to
 * five seconds), records the timeout and returns, and the CUDA context stays
 * usable.  *status receives MH_ETIMEOUT when the wait ended by its bound (the
 * expected outcome).  Returns MH_OK when the check ran, MH_EINVAL (NULL status)
 * or MH_ECUDA otherwise. */
MH_API int mh_check_bounded_wait(int32_t *status);

/* Batched solve: n cohorts (distinct handles, one device) with their options are
 * solved by cooperative launches of one persistent kernel.  The co-resident grid
 * is split into teams of blocks, team i running the greedy loop of cohort i
 * (Algorithm 1 with P-DFS) at its own pace; each time a cohort finishes, the
 * launch ends at the others' next round boundary and the unfinished cohorts
 * share the whole grid again (one launch per finished cohort at most).  The paper
 * runs one cohort at a time; this is the GB300 batching of independent problems.
 * Teams own whole SMs when the split allows it (blocks in multiples of the blocks
 * one SM holds).  blocks: n block counts (each >= 1, summing to at most the
 * co-resident grid of the three-blocks-per-SM build; kept fixed), or NULL to let
 * the autotuner choose the kernel build (one block of 16 warps, or three or four
 * blocks of 8 warps, per SM) and the
 * split: blocks ~ work^gamma with the per-cohort work estimated from the tumors'
 * mutation counts (the gene sets of size h-1, or of size h, that share a tumor);
 * build, model and gamma are picked by timing each candidate once per batch shape
 * and cached in the file
 * named by MH_AUTOTUNE_CACHE (default ~/.cache/mh_autotune.txt; MH_AUTOTUNE=0
 * disables tuning).  Work runs on the first handle's stream; the call is
 * synchronous.  On a stream other than the legacy default one, the start of the
 * batch (every cohort's round state and the first launch) is captured as a CUDA
 * graph and replayed when the same cohorts are solved again (diag[7]).  out: n result pointers, each as from mh_solve_ex (solve_ms is the
 * batch's time).  Errors: MH_EINVAL, MH_ENOMEM, MH_ECUDA, MH_ETIMEOUT; on error no
 * result is returned. */
MH_API int mh_solve_batch(mh_handle *const *handles, const mh_solve_opts *opts, int32_t n, const int32_t *blocks,
                          mh_result **out);

/* ---- Served runtime: continuous batching of solves ------------------------
 * A server owns a scheduler thread.  Submitted requests (a cohort in host
 * memory, h, alpha) wait in arrival order until a slot and device memory are
 * free: admission packs the cohort and uploads it (copies only, while a launch
 * may be running) when its estimated footprint (store, workspace and, for h >= 3,
 * the search frontiers estimated from the gene sets sharing a tumor) fits the
 * memory budget.  A launch ends at a round boundary when a request finishes or an
 * admitted one is ready, so new requests join at the next round of the others
 * (continuous batching) and every cohort stays resident on the device between its
 * rounds.  Small requests run batched (a team of whole SMs each, the batched
 * kernel); while any is active, "large" requests (see large_slots) pause at
 * their round boundary, and the large requests run when no small one is active
 * (a lone one on the single-cohort kernel, several batched).  Results are those of
 * mh_solve (MH_MODE_PERSISTENT); a served result's solve_ms is the request's
 * latency from submission to completion. */
typedef struct mh_server mh_server;
typedef struct {
    int64_t hbm_budget_bytes; /* device memory for active requests; <= 0: 80% of the free memory */
    int32_t slots;            /* requests solved concurrently; <= 0: 8 */
    int32_t large_slots;      /* "large" requests (more than 4e6 (h-1)-gene sets sharing a tumor)
                                 admitted at a time, run batched together; <= 0: 2.  Large
                                 requests start in arrival order; smaller ones queued behind a
                                 waiting large one may start first (backfill) */
    int32_t large_wait_ms;    /* an admitted large request paused longer than this (while small
                                 ones run) joins the next launch with them; <= 0: 250 */
} mh_server_opts;

/* Starts a server on the current device.  opts may be NULL (defaults).
 * Errors: MH_ECUDA (no cooperative launch), MH_ENOMEM. */
MH_API int mh_server_create(const mh_server_opts *opts, mh_server **out);

/* Queues a request; the packed rows (HOST memory, layout above) are copied, so the
 * caller may free them on return.  Non-blocking.  *ticket identifies the request.
 * Errors: MH_EINVAL.  A request larger than the whole budget later completes
 * with MH_EREJECT. */
MH_API int mh_submit(mh_server *server, const uint64_t *bitmaps, int32_t G, int32_t Nt, int32_t Nn, int32_t h,
                     mh_rational alpha, uint64_t *ticket);

/* Result of a finished request (the ticket is then released): MH_OK with *out set,
 * MH_EAGAIN while it is queued or running, or the request's own error. */
MH_API int mh_poll(mh_server *server, uint64_t ticket, mh_result **out);

/* As mh_poll, waiting up to timeout_ms (< 0: without limit); MH_EAGAIN on timeout. */
MH_API int mh_wait(mh_server *server, uint64_t ticket, int32_t timeout_ms, mh_result **out);

/* Cancels a request: a queued one completes at once with MH_ECANCELED; an admitted
 * one is retired at its next round boundary (the running launch is asked to end
 * there) and completes with MH_ECANCELED; a finished one keeps its result.  The
 * ticket stays valid until mh_poll / mh_wait returns its status.  Errors:
 * MH_EINVAL (unknown ticket). */
MH_API int mh_cancel(mh_server *server, uint64_t ticket);

/* Diagnostic (no counterpart in the paper): host-side fault injection for tests of
 * the error paths.  spec: "alloc_fail=N" -- the N-th next device allocation of the
 * library fails (MH_ENOMEM); "timeout_after=N" -- the N-th next persistent solve
 * reports MH_ETIMEOUT as if a bounded device wait had expired (after its kernel has
 * run normally); "none" or NULL clears both.  The environment variable MH_FAULT
 * takes the same specs and is read at the first allocation or solve.  Nothing is
 * injected on the device.  Errors: MH_EINVAL (unknown spec). */
MH_API int mh_set_fault(const char *spec);

/* Launches made so far, queued and active requests, device bytes reserved. */
MH_API int mh_server_stats(mh_server *server, int64_t *launches, int32_t *queued, int32_t *active,
                           int64_t *bytes_in_use);

/* Finishes every submitted request, then stops the server; results not taken are freed. */
MH_API void mh_server_destroy(mh_server *server);

/* Greedy solve that allocates nothing (the paper has no counterpart: this is a
 * deployment variant of mh_solve).  For callers that cannot call cudaMalloc --
 * code running while another component owns all device memory through its own
 * pool, plug-ins handed fixed buffers by a host framework, or latency-critical
 * streams that must not see allocator traffic -- every piece of scratch lives
 * in one file-scope __device__ array of about 30 MB that every GPU loading this
 * library keeps until the process exits.  It returns the same selections as
 * mh_solve(h, alpha) with MH_PRUNE_PAPER.
 *   d_bitmaps : DEVICE pointer to packed rows (layout above), caller-owned, read only.
 *   d_genes   : DEVICE int32 buffer of capacity*h entries (original indices, ascending per row).
 *   d_tp, d_fp: DEVICE int32 buffers of capacity entries.
 *   capacity  : rows available in the outputs; must be >= Nt (each selection covers >= 1 tumor).
 *   k_out     : HOST pointer receiving the number of selections; rounds_out (HOST, may be NULL)
 *               receives the number of greedy rounds searched.
 *   stream    : cudaStream_t (NULL = legacy default stream); the call is synchronous.
 * Limits: G <= 8192, Nt <= 1024, Nn <= 1024, 1 <= h <= 4, and at most 2^17
 * prefixes per intermediate depth of the search; larger inputs return MH_EINVAL,
 * a larger frontier MH_ENOMEM, each with a message naming the limit.  Every call
 * looks up the array's device address on the current device (cudaGetSymbolAddress,
 * so calls may span a device reset); the first call on a device also loads the
 * library's device code there, so make it before any CUDA stream capture.  All calls share the array and
 * each leaves its contents behind (every call clears what must start at zero):
 * calls whose GPU work overlaps, on different streams or host threads, race on
 * it and must be serialised by the caller.  No cudaMalloc, cudaFree or
 * allocating library routine is called. */
MH_API int mh_solve_noalloc(const uint64_t *d_bitmaps, int32_t G, int32_t Nt, int32_t Nn, int32_t h,
                            mh_rational alpha, void *stream, int32_t *d_genes, int32_t *d_tp, int32_t *d_fp,
                            int32_t capacity, int32_t *k_out, int32_t *rounds_out);

/* Diagnostic (no counterpart in the paper): measured integer throughput of the
 * current GPU, the denominator of the search kernels' integer roofline.  One
 * kernel keeps every SM busy with one 32-bit operation in independent chains:
 * op 0 = LOP3 (three-input logic), 1 = POPC, 2 = IADD.  *ops_per_s receives the
 * thread operations retired per second (best of three timed launches after one
 * warm-up, CUDA events on the legacy default stream); *kernel_ms (may be NULL)
 * the duration of that launch.  Allocates a small output buffer with cudaMalloc.
 * Errors: MH_EINVAL (bad op or NULL ops_per_s), MH_ECUDA. */
MH_API int mh_int_peak(int32_t op, double *ops_per_s, double *kernel_ms);

/* Diagnostic (no counterpart in the paper): the time of one dependent load served
 * by L2 on the current GPU, the unit of the persistent solve's per-round latency
 * chain.  One thread follows a chain of loads (L1 bypassed) through a 4 MB buffer,
 * one 128-byte line per load, twice; *ns_per_load receives the second pass's
 * device-clock time per load.  Allocates 4 MB with cudaMalloc.  Errors: MH_EINVAL
 * (NULL), MH_ECUDA. */
MH_API int mh_l2_latency(double *ns_per_load);

/* ---- Split search: one solve divided over processes --------------------------
 * The paper runs each greedy round's search over many workers by handing out the
 * lambda units of the search (§III-E) and reducing their best candidates; here a
 * process (a rank, e.g. one per GPU) searches the depth-1 genes g of its shard
 * (g % nshards == shard, in the sparsity order of §III-C) and the caller merges
 * the shards' results between rounds.  Per round, every rank calls
 * mh_shard_search, exchanges its mh_round_best with the others (an all-gather of
 * a few hundred bytes), merges them -- the winner is the candidate with the
 * largest score, ties to the smallest ascending tuple of original indices
 * (§III-D); the counters are summed (modulo 2^64) -- and calls mh_shard_commit
 * with the same merged value, which applies the winner (DelCols, Algorithm 1)
 * identically on every rank.  The selections and summed counters equal those of
 * mh_solve_ex in MH_MODE_LAUNCHES.  Runs the one-kernel-per-phase path on the
 * handle's stream; each call is synchronous.  A handle serves one split search
 * at a time and no other solve meanwhile. */
typedef struct mh_shard mh_shard;
typedef struct {
    int32_t done;               /* search: 1 if the solve has ended (nothing was searched) */
    int32_t have;               /* 1 if there is a candidate (search: in this shard; commit: a winner) */
    int64_t score;              /* S = alpha.num * TP + alpha.den * (Nn - FP) of the candidate */
    int32_t genes[MH_MAX_H];    /* its original gene indices, ascending (the first h are used) */
    uint64_t visited[MH_MAX_H]; /* the round's counters per depth: this shard's share from search; */
    uint64_t pruned[MH_MAX_H];  /* the sums over all shards for commit */
} mh_round_best;

/* Starts the split search of one solve on handle H: opts as for mh_solve_ex (prune
 * MH_PRUNE_PAPER or MH_PRUNE_OFF; mode is ignored), shard in [0, nshards).
 * Errors: MH_EINVAL, MH_ENOMEM, MH_ECUDA. */
MH_API int mh_shard_begin(mh_handle *H, const mh_solve_opts *opts, int32_t shard, int32_t nshards, mh_shard **out);

/* Searches the current round on this shard (growing a frontier and rerunning the
 * round when one overflows).  *out: have / score / genes of the shard's best
 * candidate and its share of the round's counters; done = 1 once the solve has
 * ended.  Errors: MH_ENOMEM, MH_ECUDA, MH_ETIMEOUT. */
MH_API int mh_shard_search(mh_shard *X, mh_round_best *out);

/* Applies the merged round (the winner, or have = 0 to end the solve, and the
 * summed counters) and advances to the next round; *done (may be NULL) becomes 1
 * when the solve has ended.  Every shard must commit the same merged value. */
MH_API int mh_shard_commit(mh_shard *X, const mh_round_best *merged, int32_t *done);

/* The solve's result so far (selections, merged counters), as from mh_solve_ex. */
MH_API int mh_shard_result(mh_shard *X, mh_result **out);

MH_API void mh_shard_free(mh_shard *X);

/* ---- Coverage evaluation (§IV-D, Tables III and IV) ----------------------------
 * The paper freezes the combinations learned on a training split and measures
 * their coverage on a held-out split: a sample is covered when it carries every
 * gene of at least one combination (the coverage of Eq. 1).  TC / NC: covered
 * tumor / normal samples; TT / NT: all of them; sensitivity = TC / TT,
 * specificity = 1 - NC / NT (0 when the total is 0). */
typedef struct {
    int32_t tc, tt, nc, nt;
    double sensitivity, specificity;
} mh_coverage;

/* Coverage of k combinations (HOST array genes of k*h original gene indices of the
 * handle's cohort) on the handle's samples, computed on the device.  The optional
 * HOST buffers tumor_covered (Wt words) and normal_covered (Wn words) receive the
 * covered samples as bit masks (layout of the packed rows).  Errors: MH_EINVAL (NULL
 * out, h outside [1, 9], an index outside [0, G)), MH_ENOMEM, MH_ECUDA. */
MH_API int mh_evaluate(mh_handle *H, const int32_t *genes, int32_t k, int32_t h, mh_coverage *out,
                       uint64_t *tumor_covered, uint64_t *normal_covered);

/* Cohort dimensions of a handle (any pointer may be NULL). */
MH_API int mh_handle_info(const mh_handle *handle, int32_t *G, int32_t *Nt, int32_t *Nn,
                          int64_t *device_bytes);

#ifdef __cplusplus
}
#endif

#endif /* MH_H */
