// Internal definitions shared by the host runtime and the kernels of libmh.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace mh {

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned short u16;

constexpr int kMaxH = 9;
constexpr int kMaxWords = 32;      // per-block row words: Nt, Nn <= 2048
constexpr int kMaxSamples = 2048;  // Nt <= 2048
constexpr int kMaxGenes = 65535;   // gene indices are 16-bit in prefixes and keys
constexpr int kWarpsPerBlock = 8;
constexpr int kMaxWarpsPerBlock = 32;
constexpr int kErrTimeout = 4;     // same value as MH_ETIMEOUT
constexpr int kThreads = kWarpsPerBlock * 32;
constexpr int kCountStride = 16;   // u32 slots per counter array (>= kMaxH + 1)
// Frontier appends are spread over kShards counters, each in its own 128-byte
// line, so that thousands of warps do not serialise on one atomic: depth l,
// shard i counts the records of region i of the depth-l frontier
// (counts[(l * kShards + i) * kShardStride]).
constexpr int kShards = 32;
constexpr int kShardStride = 32;
constexpr int kCountWords = kMaxH * kShards * kShardStride;
__host__ __device__ constexpr int shard_slot(int level, int shard) { return (level * kShards + shard) * kShardStride; }

struct Rec;

// Device view of one cohort, genes in search order (most sparse first, §III-C).
struct Cohort {
    int G, Nt, Nn;
    int Wt, Wn;     // words holding Nt / Nn bits
    int WTp, WNp;   // row strides in words (even: 16-byte aligned rows)
    int GW;         // words of one sample-major column over the G sorted genes (even)
    const u64 *T;   // G x WTp   tumor rows, gene-major
    const u64 *N;   // G x WNp   normal rows, gene-major
    const u64 *CT;  // Nt x GW   tumor bits, sample-major: bit g of column s = T[g] bit s
    const u64 *CN;  // Nn x GW   normal bits, sample-major
    const u16 *orig;  // G: search position -> original row index
    const u32 *inv;   // G: original row index -> search position
    // Nt x (GW + 1) running counts of CT: CC[s][w] = set bits of column s in words
    // below w (CC[s][GW]: genes mutated in sample s).  nullptr: single-sample
    // subtrees are searched like any other (no closed-form counts).
    const u16 *CC;
    // Genes of each tumor sample, ascending search positions: sample s's list is
    // SL[SO[s] .. SO[s + 1]) (the set bits of column s of CT, listed).
    const u16 *SL;
    const u32 *SO;
    // The same genes as original row indices, ascending: SLo[SO[s] .. SO[s + 1]).
    const u16 *SLo;
    // G static depth-1 records, one per gene in search order, built at create time
    // over ALL tumors: ky / kn = the gene's tumor / normal mutation counts, the
    // samples listed when few (see Rec).  A round filters the listed tumors by U.
    // nullptr: depth-1 records are built from the rows.
    const Rec *GR;
    // G static tumor signatures: OR of 1 << (s & 63) over the tumors of each gene.
    const u64 *GS;
    // The rows again in the caller's (original) gene order, G x WTp and G x WNp: a
    // key's genes read without the search-position lookup.  nullptr: use inv.
    const u64 *TO, *NO;
};

// Best candidate of a search, compared as (score desc, original tuple asc).
// s = S + 1 (0 = no candidate); t0..t2 pack the ascending original indices,
// 16 bits each, first index in the high bits of t0 (so the tuple's
// lexicographic order is the numeric order of (t0, t1, t2)).
struct Key {
    u64 s, t0, t1, t2;
};

// A prefix of the search tree (genes g_1 < ... < g_l in search order),
// 16 bits per gene: gene i in word i / 4 at bits 16 * (i % 4).
struct Prefix {
    u64 w0, w1;
};

// A node of the search frontier: the prefix and the samples of its
// intersections, listed when few (ky <= kListT and kn <= kListN: "sparse"),
// otherwise only counted ("dense": consumers rebuild them from the rows).
constexpr int kListT = 20;  // tumor samples listed per sparse node
constexpr int kListN = 12;  // normal samples listed per sparse node
struct __align__(16) Rec {
    Prefix p;
    u16 ky, kn;                  // |y| (uncovered tumors) and |n| (normals), saturated at 0xffff
    u16 ids[kListT + kListN];    // tumor sample indices, then normal sample indices
    u32 pad[3];
};
static_assert(sizeof(Rec) == 96, "frontier records are 96 bytes");

// Device build of a cohort's store (mh_store.cu): the uploaded rows and the
// sparsity permutation in, every piece of the store out.
struct StoreBuild {
    Cohort c;          // sizes: G, Nt, Nn, Wt, Wn, WTp, WNp, GW
    const u64 *bm;     // the packed rows as given, G x (Wt + Wn)
    const u32 *order;  // search position -> original row index
    const u32 *SO;     // each tumor's offset into SL / SLo (Nt + 1)
    u64 *T, *N, *TO, *NO, *CT, *CN, *CTo;  // CTo: sample-major copy of TO (scratch)
    u16 *CC, *SL, *SLo, *orig;
    u32 *inv;
    Rec *GR;
    u64 *GS;
};

// Per-solve device state.
struct Solve {
    int h;
    int prune;          // 0 = paper (cut empty intersections), 1 = off
    u64 a_num, a_den;
    u64 *U;             // WTp words: uncovered tumors
    int *state;         // kStateWords ints: k selected, done, error, overflow, round, round limit
    int *res;           // per round: h original indices, TP, FP
    u64 *cnt;           // per round, per level: visited, pruned
    Key *slots;         // per-block best candidates of the current round (persistent solve:
                        // two arrays of nslots, by round parity)
    int nslots;
    u64 *work;          // leaf-kernel work counters, see kWork*
    Key *cand;          // kCandidates best keys of the previous round (for the next threshold)
    u64 *best_hint;     // best score (s field) known to exist in the round, for skipping hopeless
                        // scoring (persistent solve: two words, by round parity)
    // Per tumor sample s (Nt entries), computed once per solve by the persistent
    // kernels: champ[s] = the best key, valued with TP = 1, over the h-subsets of
    // the genes of s; champ_ok[s] = 1 once known (champ[s].s = 0: fewer than h
    // genes), 0 if its search exceeded its budget.  nullptr: not computed.
    Key *champ;
    int *champ_ok;
    // Per tumor sample s (Nt x 2h entries): ssum[s * 2h + l - 1] = A_l(s), the
    // number of in-bound depth-l nodes (prefixes whose genes are all mutated in s,
    // each within its depth's loop bound), and ssum[s * 2h + h + l - 1] = V_l(s),
    // the children the depth-(l-1) ones among them have (their loop ranges summed).
    // Summed over the uncovered tumors they give a round's counters up to a
    // correction from the nodes shared by two or more uncovered tumors (see
    // mh_kernels.cu).  nullptr: the counters are counted node by node.
    u64 *ssum;
    // Incremental rounds: gk[g] = uncovered tumors carrying gene g (G entries);
    // cov = the tumors the previous round's winner covered (WTp words).
    u32 *gk;
    u64 *cov;
    u64 *run;  // 2 (kMaxH + 1) words: running totals of the counter corrections (see mh_kernels.cu)
    u64 *cut;  // score-bound mode: per round, per depth, the prefixes cut by the bound (nullptr: none)
    // Split search (one kernel per phase only): this solve searches the depth-1
    // genes g (search order) with g % nshards == shard; xbest[0] receives the
    // shard's best key of a round, xbest[1] holds the winner merged over all shards.
    int shard, nshards;
    Key *xbest;
};

constexpr int kCandidates = 32;
constexpr int kStateWords = 8;

// Leaf-kernel work counters (Solve::work).
enum {
    kWorkColWords = 0,   // 64-bit sample-major column words read in sibling tests
    kWorkPrefixes = 1,   // depth-(h-1) prefixes expanded by the leaf kernel
    kWorkScored = 2,     // leaves whose TP / FP were evaluated exactly
    kWorkAluOps = 3,     // 32-bit integer operations of those steps (see mh_kernels.cu)
    kWorkDense = 4,      // prefixes taken by the dense (row) path
    kWorkPhaseNs = 5,    // persistent solve: ns spent in depth 1, depths 2..h-1, leaves, end of round (4 slots)
    kWorkWarpSum = 9,    // diagnostics, [expand, leaf]: summed warp cycles of the phase,
    kWorkWarpMax = 11,   //   the longest warp of the current round,
    kWorkWarpMaxSum = 13,//   the longest warps summed over rounds,
    kWorkWarpN = 15,     //   warp count
    kWorkWarpMaxOdd = 17,//   the longest warp of the current round when it is odd (persistent solve)
    kWorkCount = 20
};

// Frontier buffers (depth l at index l): kShards regions of cap[l] records each.
// Incremental rounds keep, per record slot of every depth: sig = the OR of
// 1 << (s & 63) over the record's tumor samples (0: no longer shared by two
// uncovered tumors, ~0: samples not listed), and for the leaf parents (depth h-1)
// lb = the best key among the record's leaves with TP >= 2 and lc = the sum of
// TP - 1 over them.  nullptr where not allocated.
struct Frontiers {
    Rec *F[kMaxH];
    u32 cap[kMaxH];
    u64 *sig[kMaxH];
    Key *lb[kMaxH];
    u64 *lc[kMaxH];
};
// Device bytes of one frontier record slot with its incremental-round data.
constexpr size_t kSlotBytes = sizeof(Rec) + 2 * sizeof(u64) + sizeof(Key);

// Grid-wide barrier state of the persistent solve (zeroed before each launch):
// arrived counts the blocks' arrivals over the launch's barriers; flag is raised by
// a block that found the batch's yield request set when it arrived.
struct GridSync {
    unsigned arrived;
    int flag;
    unsigned pad[2];
};

// The persistent solve keeps the frontier counters (kCountWords) twice, by round
// parity: round r appends into counts + (r & 1) * kCountWords.
constexpr int kCountSets = 2;

// Launchers (mh_kernels.cu).
void launch_transpose(const Cohort &c, const u64 *rows, int row_stride, int samples, u64 *cols, cudaStream_t st);
cudaError_t launch_store_build(const StoreBuild &b, cudaStream_t st);
// Rounds run on the device: every kernel reads the round index and the done /
// overflow flags from Solve::state, so the host can enqueue many rounds ahead.
// counts: kCountWords u32 (see shard_slot); cap values are per shard.
// sets: frontier counter sets (and slot arrays, threshold words) to clear: 1 for the
// one-kernel-per-phase path, kCountSets for a persistent solve.
void launch_solve_init(const Cohort &c, const Solve &s, int counter_rounds, int max_rounds, u32 *counts, int sets,
                       cudaStream_t st);
void launch_level1(const Cohort &c, const Solve &s, const Frontiers &f, u32 *counts, cudaStream_t st);
void launch_expand(const Cohort &c, const Solve &s, int level, const Frontiers &f, u32 *counts, int grid,
                   cudaStream_t st);
void launch_leaf(const Cohort &c, const Solve &s, const Frontiers &f, u32 *counts, int grid, cudaStream_t st);
void launch_finalize(const Cohort &c, const Solve &s, u32 *counts, cudaStream_t st);
// Split search: step 1 reduces the round's blocks to the shard's best key (xbest[0]),
// step 2 applies the merged winner xbest[1] (DelCols, selection, next round).
void launch_finalize_split(const Cohort &c, const Solve &s, u32 *counts, int step, cudaStream_t st);
// Coverage masks of k combinations (k x h original indices, device): tcov (WTp
// words) and ncov (WNp words), zeroed by the caller.
void launch_coverage(const Cohort &c, const int *genes, int k, int h, u64 *tcov, u64 *ncov, cudaStream_t st);

// Persistent solve: all rounds in one cooperative launch of `grid` blocks
// (persistent_grid(): one block per SM for the default build, the co-resident
// maximum of the four-blocks-per-SM build with `large`; 0 if it cannot be
// determined).
// It returns when the solve is done, a frontier overflowed (state) or a grid
// barrier timed out (state error = kErrTimeout).
int persistent_grid(int num_sms, bool large);
// The batched kernel comes in three builds: one block of 16 warps per SM (the most
// registers per thread), or 3 or 4 co-resident blocks of 8 warps per SM (more warps);
// batch_grid / batch_blocks_per_sm take the build (its blocks per SM).
int batch_grid(int num_sms, int build);
int batch_blocks_per_sm(int build);
constexpr int kBatchBuilds[3] = {1, 3, 4};

// One cohort of a batched solve: its device state and its share of the grid
// (blocks [first_block, first_block + nblocks)).
struct BatchItem {
    Cohort c;
    Solve s;
    Frontiers f;
    GridSync *gsync;
    u32 *counts;
    int first_block, nblocks;
};
// Block numbering of a batched launch.  Teams are ranges of "SM-major" block
// numbers: the blocks resident on one SM get consecutive numbers, so a team whose
// range is a multiple of the blocks per SM owns whole SMs (its L1 and shared memory
// are not shared with another cohort).  tab: kBatchTabInts device ints owned by the
// caller (reset by the launcher); sync: a GridSync for the launch's start.
constexpr int kMaxSmid = 1024;
constexpr int kBatchTabInts = 2 * kMaxSmid + 2;
struct BatchMap {
    int *tab;
    GridSync *sync;
    int per_sm, num_sms;
    int build;  // 3 or 4 blocks per SM
};
// Runs the cohorts of d_items (device array of n items) in one cooperative launch
// of the whole batch grid (per_sm x num_sms blocks; blocks beyond the items' ranges
// return at once).  With d_yield (a zeroed int in device or mapped host memory),
// the launch ends as soon as one cohort finishes or overflows a frontier: every
// other team stops at its next round boundary.
cudaError_t launch_solve_batch(const BatchItem *d_items, int n, int *d_yield, const BatchMap &map, cudaStream_t st);
// yield: as for launch_solve_batch (the server runs a lone request this way), or NULL.
cudaError_t launch_solve_persistent(const Cohort &c, const Solve &s, const Frontiers &f, GridSync *gsync,
                                    u32 *counts, int grid, bool large, cudaStream_t st, int *yield = nullptr);
int level1_grid(const Cohort &c);
// One block waiting at a barrier that no other block reaches (the bounded wait's
// timeout path); state: kStateWords zeroed ints.
cudaError_t launch_barrier_probe(GridSync *g, int *state, cudaStream_t st);

// Message returned by mh_last_error() on the calling thread.
void set_error_text(const char *text);

}  // namespace mh
