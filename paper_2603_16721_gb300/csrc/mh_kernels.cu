// Kernels of libmh: one greedy round of the weighted set cover (Algorithm 1)
// whose argmax step is a level-by-level P-DFS (§III-D, Algorithm 2).
//
// Search order and notation: genes are in search order (most sparse first,
// §III-C); a depth-l node is a prefix g_1 < ... < g_l, its tumor intersection
// y_l = U & x_{g_1} & ... & x_{g_l} (U = still uncovered tumors) and its normal
// intersection n_l = x^N_{g_1} & ... & x^N_{g_l}.  The children of a depth-(l-1)
// node are g_l in (g_{l-1}, G - h + l] (1-based), exactly the loop bounds of
// Algorithm 2.  A child is cut ("pruned") when y_l is empty.
//
// Sibling test.  All children of one prefix share y_{l-1}; child g is non-empty
// iff some sample s in y_{l-1} has bit g set in the sample-major copy CT of the
// tumor bits.  So the non-empty children of a prefix are the set bits of
//     OR over s in y_{l-1} of CT[s]      restricted to the child range,
// which one lane evaluates 64 siblings at a time.  This is the same emptiness
// test as AND-ing y_{l-1} with every sibling row, bit-sliced over the siblings.
//
// Leaf scores.  For a sparse prefix (few samples in y_{l-1} and n_{l-1}) the same
// column words, summed in bit-sliced counters (one 64-bit plane per bit of the
// count), give TP(g) = |y_{l-1} & x_g| and FP(g) = |n_{l-1} & x^N_g| for 64
// siblings at once, so a leaf is scored without touching its rows.  Prefixes
// with many samples take a row path: popcounts over the non-zero words only.
//
// Work distribution.  A warp takes 32 prefixes at a time from a per-depth atomic
// counter (the analogue of the paper's chunked lambda dispatch, §III-E).  Each
// lane first lists the samples of one prefix; then the (prefix, column word)
// items of the batch's sparse prefixes are spread over the 32 lanes, so
// neighbouring lanes read neighbouring column words; dense prefixes are taken by
// the whole warp, one at a time.
#include "mh.h"
#include "mh_internal.h"

namespace mh {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBatch = 32;       // prefixes taken per warp
constexpr int kPlanesT = 5;      // bit planes for counts <= 20
constexpr int kPlanesN = 4;      // bit planes for counts <= 12

// The blocks that work on one cohort: this block's rank among them and their
// number (the whole grid for a single solve; a share of it in a batch).
struct Team {
    int rank, size;
};
__device__ __forceinline__ Team grid_team() { return Team{(int)blockIdx.x, (int)gridDim.x}; }

// Where a phase of one round takes its inputs and leaves its results.  One kernel
// per phase: depth-1 records from the frontier, bests merged into s.slots, the
// threshold in s.best_hint.  Persistent solve: depth-1 nodes built from the gene
// rows and the block's copy of U (Ush), bests stored into the round's slot array,
// the round's threshold word, diagnostics by round parity.
// fm: counters by per-sample sums and incremental rounds (see "Counting by
// per-sample sums" and "Incremental rounds" below): only nodes shared by two or
// more uncovered tumors are built and searched; build: the expansion builds the
// kept frontiers of round 0 and adds no counters (the evaluation that follows
// counts every kept node).
struct RoundIO {
    const u64 *Ush;
    Key *slots;
    bool overwrite;
    u64 *hint;
    int par;
    bool fm;
    bool build;
};
__device__ __forceinline__ RoundIO launch_io(const Solve &s)
{
    return RoundIO{nullptr, s.slots, false, s.best_hint, 0, false, false};
}

__device__ __forceinline__ int prefix_gene(const Prefix &p, int i)
{
    const u64 w = i < 4 ? p.w0 : p.w1;
    return (int)((w >> (16 * (i & 3))) & 0xffffull);
}

__device__ __forceinline__ Prefix prefix_with(Prefix p, int i, int g)
{
    if (i < 4) p.w0 |= (u64)g << (16 * i);
    else p.w1 |= (u64)g << (16 * (i - 4));
    return p;
}

__device__ __forceinline__ bool key_better(const Key &a, const Key &b)
{
    if (a.s != b.s) return a.s > b.s;
    if (a.t0 != b.t0) return a.t0 < b.t0;
    if (a.t1 != b.t1) return a.t1 < b.t1;
    return a.t2 < b.t2;
}

__device__ __forceinline__ Key key_empty()
{
    Key k;
    k.s = k.t0 = k.t1 = k.t2 = 0;
    return k;
}

__device__ __forceinline__ void key_put(Key &k, int pos, int v)
{
    const u64 x = (u64)v << (16 * (3 - (pos & 3)));
    if (pos < 4) k.t0 |= x;
    else if (pos < 8) k.t1 |= x;
    else k.t2 |= x;
}

__device__ __forceinline__ int key_get(const Key &k, int pos)
{
    const u64 w = pos < 4 ? k.t0 : (pos < 8 ? k.t1 : k.t2);
    return (int)((w >> (16 * (3 - (pos & 3)))) & 0xffffull);
}

// Key of a leaf: the prefix's original indices (ascending, po[0..L)) with o inserted.
__device__ __forceinline__ Key leaf_key(u64 s1, const int *po, int L, int o)
{
    Key k;
    k.s = s1;
    k.t0 = k.t1 = k.t2 = 0;
    int pos = 0;
    bool placed = false;
    for (int q = 0; q < L; ++q) {
        const int v = po[q];
        if (!placed && o < v) {
            key_put(k, pos++, o);
            placed = true;
        }
        key_put(k, pos++, v);
    }
    if (!placed) key_put(k, pos, o);
    return k;
}

// The warp's largest key: the largest score by two 32-bit warp reductions, then,
// only when several lanes hold it, the smallest tuple among them, 32 bits at a
// time; the winning lane's key is broadcast.
__device__ __forceinline__ unsigned lanes_min_part(unsigned cand, u64 v, int lane)
{
    const bool in = (cand >> lane) & 1u;
    const unsigned hi = __reduce_min_sync(kFull, in ? (unsigned)(v >> 32) : ~0u);
    cand &= __ballot_sync(kFull, in && (unsigned)(v >> 32) == hi);
    if (__popc(cand) == 1) return cand;
    const bool in2 = (cand >> lane) & 1u;
    const unsigned lo = __reduce_min_sync(kFull, in2 ? (unsigned)v : ~0u);
    return cand & __ballot_sync(kFull, in2 && (unsigned)v == lo);
}
__device__ __forceinline__ Key warp_max_key(Key k)
{
    const int lane = threadIdx.x & 31;
    const unsigned hi = __reduce_max_sync(kFull, (unsigned)(k.s >> 32));
    const bool top = (unsigned)(k.s >> 32) == hi;
    const unsigned lo = __reduce_max_sync(kFull, top ? (unsigned)k.s : 0u);
    unsigned cand = __ballot_sync(kFull, top && (unsigned)k.s == lo);
    if (__popc(cand) > 1) cand = lanes_min_part(cand, k.t0, lane);
    if (__popc(cand) > 1) cand = lanes_min_part(cand, k.t1, lane);
    if (__popc(cand) > 1) cand = lanes_min_part(cand, k.t2, lane);
    const int src = __ffs(cand) - 1;  // equal keys: any of them
    Key o;
    o.s = __shfl_sync(kFull, k.s, src);
    o.t0 = __shfl_sync(kFull, k.t0, src);
    o.t1 = __shfl_sync(kFull, k.t1, src);
    o.t2 = __shfl_sync(kFull, k.t2, src);
    return o;
}

__device__ __forceinline__ u64 warp_sum_u64(u64 v)
{
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}

__device__ __forceinline__ u64 warp_max_u64(u64 v)
{
    for (int off = 16; off; off >>= 1) {
        const u64 o = __shfl_xor_sync(kFull, v, off);
        v = o > v ? o : v;
    }
    return v;
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(kFull, v, off);
        if (lane >= off) v += o;
    }
    return v;
}

// Block-wide best key -> slots[rank]: stored (overwrite), or merged with what an
// earlier launch of the same round left there.  All threads of the block must call it.
// The warps' best keys on their way to a block maximum (one array for every phase:
// each use ends at a block barrier before the next begins).
__device__ __forceinline__ Key *warp_keys()
{
    __shared__ Key w[kMaxWarpsPerBlock];
    return w;
}
__device__ void block_commit_best(Key best, Key *slots, int rank, bool overwrite)
{
    Key *wbest = warp_keys();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    best = warp_max_key(best);
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (warp == 0) {
        Key k = lane < (int)(blockDim.x >> 5) ? wbest[lane] : key_empty();
        k = warp_max_key(k);
        if (lane == 0 && overwrite) {
            slots[rank] = k;
        } else if (lane == 0 && k.s != 0) {
            const Key old = slots[rank];
            if (key_better(k, old)) slots[rank] = k;
        }
    }
}

__device__ __forceinline__ u64 range_word(int wi, int lo, int hi)
{
    u64 m = ~0ull;
    if (wi == (lo >> 6)) m &= ~0ull << (lo & 63);
    if (wi == (hi >> 6)) m &= ~0ull >> (63 - (hi & 63));
    return m;
}

// Adds the 64 one-bit values of x to the bit-sliced counters p[0..P).
template <int P>
__device__ __forceinline__ void planes_add(u64 (&p)[P], u64 x, int used)
{
#pragma unroll
    for (int i = 0; i < P; ++i) {
        if (i < used) {
            const u64 c = p[i] & x;
            p[i] ^= x;
            x = c;
        }
    }
}

template <int P>
__device__ __forceinline__ int planes_get(const u64 (&p)[P], int b, int used)
{
    int v = 0;
#pragma unroll
    for (int i = 0; i < P; ++i)
        if (i < used) v |= (int)((p[i] >> b) & 1ull) << i;
    return v;
}

__device__ __forceinline__ int bit_length(int v) { return 32 - __clz(v); }

__device__ __forceinline__ bool is_dense(int ky, int kn) { return ky > kListT || kn > kListN; }

__device__ __forceinline__ u16 sat16(int v) { return (u16)(v < 0xffff ? v : 0xffff); }

// Round state (Solve::state): a kernel of a round does nothing once the solve is
// done or a frontier of the round has overflowed.
enum { kStK = 0, kStDone = 1, kStError = 2, kStOverflow = 3, kStRound = 4, kStMaxRounds = 5, kStYield = 6 };

__device__ __forceinline__ bool halted(const Solve &s) { return s.state[kStDone] | s.state[kStOverflow]; }

// Sharded frontier of one depth as a consumer sees it: lane i reads the record
// count of shard i; the exclusive prefix sums map a record index to its shard.
// Returns the number of records, or -1 if a shard overflowed its region (then
// the round must be rerun with a larger frontier).
__device__ __forceinline__ long long front_open(const u32 *counts, int level, u32 cap_s, int *soff, int lane)
{
    const u32 n = __ldcg(&counts[shard_slot(level, lane)]);
    if (__any_sync(kFull, n > cap_s)) return -1;
    const int incl = warp_incl_scan((int)n, lane);
    soff[lane] = incl - (int)n;
    if (lane == 31) soff[32] = incl;
    __syncwarp();
    return __shfl_sync(kFull, incl, 31);
}

// Address of record i of a sharded frontier (soff from front_open).
__device__ __forceinline__ const Rec *front_rec(const Rec *F, u32 cap_s, const int *soff, u32 i)
{
    int lo = 0, hi = kShards - 1;  // last shard with soff <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((u32)soff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return F + (size_t)lo * cap_s + (i - (u32)soff[lo]);
}

// The shard a warp appends to: neighbouring warps use different counters.
__device__ __forceinline__ int my_shard(const Team &t)
{
    return (int)((t.rank * (blockDim.x >> 5) + (threadIdx.x >> 5)) % kShards);
}

// Block-wide accumulation of counters: warps add into shared memory, then one
// global atomic per counter and block (not per warp) at the end of a phase.
// 8, 9: depth-1 visited / pruned of a persistent round; from kAccDeep: visited and
// surviving nodes of every depth counted in closed form (single-sample subtrees)
constexpr int kAccDeep = 10;
constexpr int kAccN = kAccDeep + 2 * (kMaxH + 1);
__device__ __forceinline__ void acc_begin(u64 *acc)
{
    if (threadIdx.x < kAccN) acc[threadIdx.x] = 0;
    __syncthreads();
}
__device__ __forceinline__ void acc_add(u64 *acc, int i, u64 v)
{
    if (v) atomicAdd(&acc[i], v);
}

// Closed-form counters of the block (depths 1 .. h) into the round's counters.
// Every thread of the block calls it after the block's last update of acc.
__device__ __forceinline__ void acc_flush_deep(const Solve &s, int round, const u64 *acc)
{
    const int e = (int)threadIdx.x - 32;
    if (e >= 1 && e <= s.h) {
        const u64 v = acc[kAccDeep + 2 * e], a = acc[kAccDeep + 2 * e + 1];
        if (v) {
            atomicAdd(s.cnt + ((size_t)round * s.h + (e - 1)) * 2, v);
            if (v - a) atomicAdd(s.cnt + ((size_t)round * s.h + (e - 1)) * 2 + 1, v - a);
        }
    }
}

__device__ __forceinline__ void copy_rec(Rec *dst, const Rec *src)
{
    const uint4 *a = reinterpret_cast<const uint4 *>(src);
    uint4 *b = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(Rec) / 16); ++i) b[i] = a[i];
}

// Frontier record from global memory, read through L2 only (records are
// rewritten every round; a persistent kernel must not see stale L1 lines).
__device__ __forceinline__ void load_rec(Rec *dst, const Rec *src)
{
    const uint4 *a = reinterpret_cast<const uint4 *>(src);
    uint4 *b = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(Rec) / 16); ++i) b[i] = __ldcg(a + i);
}

// ---------------------------------------------------------------------------
// Single-sample subtrees.  Below a node whose tumor intersection is one sample
// smp, every node's intersection is {smp} or empty, so the tree there is fixed by
// the genes of smp after the node's last gene g: with b_1 < b_2 < ... those genes,
// a depth-(d+k) descendant survives iff its last k genes are k of the b's, each
// within its depth's bound hi(e) = G - h + e - 1 (0-based, inclusive).  Its
// counters -- visited and pruned per depth, exactly those of Algorithm 2's loops
// over this subtree -- follow from one pass over the bits of column smp, and none
// of its leaves scores above a_num + a_den * Nn (TP = 1).  So when a candidate of
// the round is known to score more than that, the subtree is counted in closed
// form instead of being searched.

// Which single-sample subtrees a phase may count in closed form:
//   2: all of them -- a candidate of the round is known to score above
//      a_num * 1 + a_den * Nn (thr, as S + 1), which no TP = 1 leaf reaches;
//   1: those of the samples whose champion is known (Solve::champ): the
//      champions stand for every TP = 1 leaf (see phase_champions);
//   0: none.  Paper pruning only (with pruning off the empty nodes have children too).
__device__ __forceinline__ int single_sample_mode(const Cohort &c, const Solve &s, u64 thr)
{
    if (s.prune != 0 || c.CC == nullptr) return 0;
    if (s.a_num + s.a_den * (u64)c.Nn + 1ull < thr) return 2;
    return s.champ ? 1 : 0;
}

// champ_ok is written once per solve, before the grid barrier that precedes its
// first read, so plain (L1-cached) loads see the final values.
__device__ __forceinline__ bool single_sample_closed(int mode, const int *champ_ok, int smp)
{
    return mode == 2 || (mode == 1 && champ_ok[smp] != 0);
}

// Position in sample smp's gene list of its first gene after g.
__device__ __forceinline__ int single_sample_rank(const Cohort &c, int g, int smp)
{
    const int w = g >> 6, bt = g & 63;
    const u64 upto = bt == 63 ? ~0ull : ((2ull << bt) - 1ull);
    return (int)__ldg(c.CC + (size_t)smp * (c.GW + 1) + w) + __popcll(__ldg(c.CT + (size_t)smp * c.GW + w) & upto);
}

// Counters of the subtree below a depth-d node (d <= h - 2) with y = {smp} and last
// gene g, added to the block's per-depth sums deep[2e] (visited) and deep[2e + 1]
// (surviving) for e = d+1 .. h.  f_k(b) = number of surviving depth-(d+k) nodes
// whose last gene is b: f_1(b) = [b <= hi(d+1)], f_k(b) = [b <= hi(d+k)] * (sum of
// f_{k-1} over the earlier genes); each such node has hi(d+k+1) - b children.
// genes: the n genes of smp after g, ascending; G: the cohort's gene count.
__device__ __noinline__ void single_sample_subtree(const u16 *genes, int n, int G, int h, int d, int g, u64 *deep)
{
    const int K = h - d;            // levels below the node, 2 .. kMaxH - 1
    const int hi0 = G - h + d - 1;  // hi(d + k) = hi0 + k
    u64 S[kMaxH], av[kMaxH], vi[kMaxH];
#pragma unroll
    for (int k = 0; k < kMaxH; ++k) S[k] = av[k] = vi[k] = 0;
    vi[1] = (u64)(hi0 + 1 - g);
    for (int i = 0; i < n; ++i) {
        const int b = (int)__ldg(genes + i);
        // descending k: f_k reads the sum of f_{k-1} before this gene's update
#pragma unroll
        for (int k = kMaxH - 1; k >= 1; --k) {
            if (k > K || b > hi0 + k) continue;
            const u64 f = k == 1 ? 1ull : S[k - 1];
            av[k] += f;
            if (k < K) {
                vi[k + 1] += f * (u64)(hi0 + k + 1 - b);
                S[k] += f;
            }
        }
    }
#pragma unroll
    for (int k = 1; k < kMaxH; ++k) {
        if (k > K) break;
        if (vi[k]) atomicAdd(&deep[2 * (d + k)], vi[k]);
        if (av[k]) atomicAdd(&deep[2 * (d + k) + 1], av[k]);
    }
}

// The same recurrence for a compile-time number of levels K = h - d (2 or 3: the
// subtrees of depth-1 and depth-2 nodes for h <= 5), with every sum in registers.
template <int K>
__device__ __noinline__ void single_sample_subtree_k(const u16 *genes, int n, int G, int h, int d, int g, u64 *deep)
{
    const int hi0 = G - h + d - 1;
    u64 S[K + 1], av[K + 1], vi[K + 1];
#pragma unroll
    for (int k = 0; k <= K; ++k) S[k] = av[k] = vi[k] = 0;
    vi[1] = (u64)(hi0 + 1 - g);
    for (int i = 0; i < n; ++i) {
        const int b = (int)__ldg(genes + i);
#pragma unroll
        for (int k = K; k >= 1; --k) {
            if (b > hi0 + k) continue;
            const u64 f = k == 1 ? 1ull : S[k - 1];
            av[k] += f;
            if (k < K) {
                vi[k + 1] += f * (u64)(hi0 + k + 1 - b);
                S[k] += f;
            }
        }
    }
#pragma unroll
    for (int k = 1; k <= K; ++k) {
        if (vi[k]) atomicAdd(&deep[2 * (d + k)], vi[k]);
        if (av[k]) atomicAdd(&deep[2 * (d + k) + 1], av[k]);
    }
}

// Closed-form counters of the subtree below a depth-d node (d < h) with y = {smp}
// and last gene g: the leaves of a leaf parent into vis_h / alive_h, a deeper
// subtree into deep.
__device__ __forceinline__ void single_sample_count(const Cohort &c, int h, int d, int g, int smp, u64 &vis_h,
                                                    u64 &alive_h, u64 *deep)
{
    const int r = single_sample_rank(c, g, smp);
    const int m = (int)__ldg(c.CC + (size_t)smp * (c.GW + 1) + c.GW);
    if (d == h - 1) {
        vis_h += (u64)(c.G - 1 - g);
        alive_h += (u64)(m - r);
    } else {
        const u16 *genes = c.SL + __ldg(c.SO + smp) + r;
        if (h - d == 2) single_sample_subtree_k<2>(genes, m - r, c.G, h, d, g, deep);
        else if (h - d == 3) single_sample_subtree_k<3>(genes, m - r, c.G, h, d, g, deep);
        else single_sample_subtree(genes, m - r, c.G, h, d, g, deep);
    }
}

// Per-warp scratch: one batch of frontier records and their child ranges.
struct Batch {
    Rec r[kBatch];
    int lo[kBatch], hi[kBatch];     // child range (0-based, inclusive); lo > hi when empty
    int off[kBatch + 1];            // exclusive prefix sum of the sparse records' column words
    int soff[kShards + 1];          // input frontier: exclusive prefix sums of the shard counts
    u64 ys[kMaxWords];              // dense path: y_{l-1} and n_{l-1} words; expansion: staged
    u64 ns[kMaxWords];              // child masks and their (record, word) of one item per lane
    int cx[33];                     // expansion: exclusive prefix sum of the lanes' child counts
    u16 po[kBatch][kMaxH - 1];      // leaves: ascending original indices of each record's prefix
    Key rb[kBatch];                 // incremental rounds: per leaf parent, its best leaf (TP >= 2)
    u64 rc[kBatch];                 //   and the sum of TP - 1 over those leaves (rb[j].s holds
                                    //   the packed best while a listed record's items merge)
};

// Depth-1 node of gene g (search order) built from its rows and U: y_1 = U & x_g,
// n_1 = x^N_g, their sizes and, when few, their samples.  Returns |y_1| > 0.
__device__ __forceinline__ bool gene_record(const Cohort &c, const u64 *Ush, int g, Rec &r)
{
    if (c.GR) {
        // the gene's static record lists its tumors (all of them) and normals when
        // few: y_1's samples are the listed tumors still in U
        const uint4 *a = reinterpret_cast<const uint4 *>(c.GR + g);
        uint4 *d = reinterpret_cast<uint4 *>(&r);
#pragma unroll
        for (int i = 0; i < (int)(sizeof(Rec) / 16); ++i) d[i] = __ldg(a + i);
        if (!is_dense(r.ky, r.kn)) {
            int k = 0;
            for (int q = 0; q < (int)r.ky; ++q) {
                const int smp = r.ids[q];
                if ((Ush[smp >> 6] >> (smp & 63)) & 1ull) r.ids[k++] = (u16)smp;
            }
            r.ky = (u16)k;
            return k > 0;
        }
    }
    const u64 *trow = c.T + (size_t)g * c.WTp;
    const u64 *nrow = c.N + (size_t)g * c.WNp;
    int ky = 0, kn = 0;
    for (int w = 0; w < c.Wt; ++w) ky += __popcll(trow[w] & Ush[w]);
    for (int w = 0; w < c.Wn; ++w) kn += __popcll(nrow[w]);
    r.p.w0 = (u64)g;
    r.p.w1 = 0;
    r.ky = sat16(ky);
    r.kn = sat16(kn);
    if (!is_dense(ky, kn)) {
        int k = 0;
        for (int w = 0; w < c.Wt; ++w)
            for (u64 y = trow[w] & Ush[w]; y; y &= y - 1) r.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
        k = kListT;
        for (int w = 0; w < c.Wn; ++w)
            for (u64 y = nrow[w]; y; y &= y - 1) r.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
    }
    return ky > 0;
}

// Work assignment of a phase.  The phase's records are cut into batches of R <= 32
// records, R = ceil(records / warps) capped at 32 so that every warp gets work even
// when records are few: batch B holds records B % nw + (B / nw * R + j) * nw,
// j = 0..R-1, for nw warps.  Warp gw first takes the batches gw, gw + nw, ... of
// the first three quarters of the rounds (static, no atomics); the last quarter is
// handed out by kDispensers counters (warp gw draws from counter gw % kDispensers),
// so warps that finish early take over the batches of slow ones.
constexpr int kDispensers = 4;
#ifndef MH_SMALL_WARPS
#define MH_SMALL_WARPS 16
#endif
constexpr int kSmallWarps = MH_SMALL_WARPS;  // warps per block of the one-block-per-SM persistent build
struct Dispenser {
    u32 nw, gw, it, it_static, R;
    u32 *ctr;
    __device__ Dispenser(u32 nw_, u32 gw_, u32 count, u32 *ctrs) : nw(nw_), gw(gw_), it(0)
    {
        const u64 per_warp = ((u64)count + nw - 1) / nw;
        R = per_warp < (u64)kBatch ? (u32)(per_warp ? per_warp : 1) : (u32)kBatch;
        const u64 iters = ((u64)count + (u64)R * nw - 1) / ((u64)R * nw);
        it_static = (u32)(iters - iters / 4);
        ctr = ctrs + (gw % kDispensers) * kShardStride;
    }
    // First record of the warp's next batch, or >= the record count when the phase is done.
    __device__ u64 next(int lane)
    {
        u64 B;
        if (it < it_static) {
            B = (u64)it * nw + gw;
            ++it;
        } else {
            u32 d = 0;
            if (lane == 0) d = atomicAdd(ctr, 1u);
            d = __shfl_sync(kFull, d, 0);
            B = (u64)it_static * nw + (gw % kDispensers) + (u64)d * kDispensers;
        }
        return (B % nw) + (B / nw) * R * nw;
    }
};

// The dispenser counters of phase p (p = level - 2 for an expansion, h - 2 for
// the leaves) in the unused depth-0 slots of a counter set.
__device__ __forceinline__ u32 *dispenser_counters(u32 *counts, int p)
{
    return counts + shard_slot(0, kDispensers * p);
}

// Depth-1 counters of the nodes built by gene_record.
struct Depth1 {
    u64 visited = 0, pruned = 0;
};

// Lane j < R takes record first + j*stride (if < count) into the warp scratch with
// its child range [last gene + 1, hi_bound]; counts its children as visited.
// With io.Ush the records are the depth-1 nodes of genes 0 .. count-1, built from
// the rows (empty ones are counted as pruned and have no children, unless
// all_children).  With `single` (single_sample_mode), a listed record whose tumor
// intersection is one sample is counted in closed form and left with no children
// to search: a leaf parent (L = h - 1) adds its surviving leaves to alive_cf, a
// shallower record adds its whole subtree to deep.  Returns the number of column
// words of the batch's sparse records (those with samples, or all of them with
// `all_children`) and the bit mask of dense records.
__device__ __forceinline__ int batch_prepare(const Cohort &c, const RoundIO &io, Depth1 &d1, const Rec *Fin,
                                             u32 cap_s, u64 first, u64 stride, int R, u32 count, int L, int hi_bound,
                                             bool all_children, Batch &b, int lane, unsigned &dense_mask,
                                             u64 &visited, int h, int single, const int *champ_ok, u64 &alive_cf,
                                             u64 *deep, const u16 *orig = nullptr, bool fm = false,
                                             u64 cut_thr = 0, u64 a_num = 0, u64 nn_term = 0, u64 *cutn = nullptr)
{
    const u64 i = first + (u64)lane * stride;
    bool valid = lane < R && i < count;
    int lo = 1, hi = 0, ky = 0, kn = 0;
    if (valid && io.Ush) {
        const bool nonempty = gene_record(c, io.Ush, (int)i, b.r[lane]);
        ++d1.visited;
        d1.pruned += nonempty ? 0 : 1;
        valid = nonempty || all_children;
    } else if (valid) {
        load_rec(&b.r[lane], front_rec(Fin, cap_s, b.soff, (u32)i));
    }
    if (valid && fm) {
        // counting by per-sample sums: a node shared by fewer than two uncovered
        // tumors is accounted for by those sums (nothing to search below it); a
        // shared one adds (|y| - 1) x (its children) to the depth's correction
        lo = prefix_gene(b.r[lane].p, L - 1) + 1;
        hi = hi_bound;
        ky = b.r[lane].ky;
        kn = b.r[lane].kn;
        if (ky < 2) hi = lo - 1;
        else if (hi >= lo) visited += (u64)(ky - 1) * (u64)(hi - lo + 1);
        if (orig && hi >= lo) {  // ascending original indices of the prefix genes (leaf keys)
            for (int q = 0; q < L; ++q) {
                const u16 v = orig[prefix_gene(b.r[lane].p, q)];
                int k = q - 1;
                while (k >= 0 && b.po[lane][k] > v) {
                    b.po[lane][k + 1] = b.po[lane][k];
                    --k;
                }
                b.po[lane][k + 1] = v;
            }
        }
    } else if (valid) {
        lo = prefix_gene(b.r[lane].p, L - 1) + 1;
        hi = hi_bound;
        ky = b.r[lane].ky;
        kn = b.r[lane].kn;
        if (cutn && hi >= lo && ky > 0 && a_num * (u64)ky + nn_term < cut_thr) {
            // score bound: every leaf below scores at most a_num |y| + a_den Nn, below
            // a candidate already known, so the prefix is cut (nothing below is visited)
            hi = lo - 1;
            ++*cutn;
        } else if (single && ky == 1 && !is_dense(ky, kn) && hi >= lo &&
            single_sample_closed(single, champ_ok, b.r[lane].ids[0])) {
            single_sample_count(c, h, L, lo - 1, b.r[lane].ids[0], visited, alive_cf, deep);
            hi = lo - 1;  // nothing left to search below this record
        } else if (hi >= lo) {
            visited += (u64)(hi - lo + 1);
        }
        if (orig && hi >= lo) {  // ascending original indices of the prefix genes (leaf keys)
            for (int q = 0; q < L; ++q) {
                const u16 v = orig[prefix_gene(b.r[lane].p, q)];
                int k = q - 1;
                while (k >= 0 && b.po[lane][k] > v) {
                    b.po[lane][k + 1] = b.po[lane][k];
                    --k;
                }
                b.po[lane][k + 1] = v;
            }
        }
    }
    b.lo[lane] = lo;
    b.hi[lane] = hi;
    const bool live = valid && hi >= lo;
    const bool dense = live && is_dense(ky, kn);
    dense_mask = __ballot_sync(kFull, dense);
    const int nw = (live && !dense && (ky > 0 || all_children)) ? (hi >> 6) - (lo >> 6) + 1 : 0;
    const int incl = warp_incl_scan(nw, lane);
    b.off[lane] = incl - nw;
    if (lane == 31) b.off[kBatch] = incl;
    __syncwarp();
    return __shfl_sync(kFull, incl, 31);
}

// Dense path: lane w forms word w of y_{l-1} / n_{l-1} into the warp scratch.
__device__ __forceinline__ void dense_setup(const Cohort &c, const Solve &s, const Prefix &p, int L, Batch &b,
                                            unsigned &by, unsigned &bn, int lane)
{
    u64 y = 0, n = 0;
    if (lane < c.Wt) {
        y = __ldcg(&s.U[lane]);
        for (int i = 0; i < L; ++i) y &= c.T[(size_t)prefix_gene(p, i) * c.WTp + lane];
    }
    if (lane < c.Wn) {
        n = ~0ull;
        for (int i = 0; i < L; ++i) n &= c.N[(size_t)prefix_gene(p, i) * c.WNp + lane];
    }
    b.ys[lane] = y;
    b.ns[lane] = n;
    by = __ballot_sync(kFull, y != 0);
    bn = __ballot_sync(kFull, n != 0);
    __syncwarp();
}

// Sibling masks of the items t0, t0+32, ... (kIlp of them) of a batch: the
// column loads of all of them are issued together.  j is the lane's running
// record index (items are visited in increasing order).
constexpr int kIlp = 4;
__device__ __forceinline__ void sibling_items(const Cohort &c, const Batch &b, int t0, int total, int &j,
                                              int (&jj)[kIlp], int (&wi)[kIlp], int (&ky)[kIlp], u64 (&m)[kIlp],
                                              u64 (&rw)[kIlp])
{
    int kmax = 0;
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
        const int t = t0 + 32 * u;
        ky[u] = 0;
        wi[u] = 0;
        rw[u] = 0;
        m[u] = 0;
        if (t < total) {
            while (t >= b.off[j + 1]) ++j;
            wi[u] = (b.lo[j] >> 6) + (t - b.off[j]);
            ky[u] = b.r[j].ky;
            rw[u] = range_word(wi[u], b.lo[j], b.hi[j]);
        }
        jj[u] = j;
        kmax = ky[u] > kmax ? ky[u] : kmax;
    }
    // two samples of every item per step: all their loads are in flight together
    for (int q = 0; q < kmax; q += 2) {
        u64 x0[kIlp], x1[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            x0[u] = q < ky[u] ? __ldg(c.CT + (size_t)b.r[jj[u]].ids[q] * c.GW + wi[u]) : 0ull;
            x1[u] = q + 1 < ky[u] ? __ldg(c.CT + (size_t)b.r[jj[u]].ids[q + 1] * c.GW + wi[u]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) m[u] |= x0[u] | x1[u];
    }
#pragma unroll
    for (int u = 0; u < kIlp; ++u) m[u] &= rw[u];
}

// The same sibling test counting how many samples have each sibling: m = the
// siblings of at least one sample (non-empty children), m2 = of at least two
// (children shared by two or more uncovered tumors); with SUM, sum[u] = the
// number of (sample, sibling) pairs in the range word (the children's sizes
// summed).
template <bool SUM>
__device__ __forceinline__ void sibling_items2(const Cohort &c, const Batch &b, int t0, int total, int &j,
                                               int (&jj)[kIlp], int (&wi)[kIlp], int (&ky)[kIlp], u64 (&m)[kIlp],
                                               u64 (&m2)[kIlp], int (&sum)[kIlp])
{
    int kmax = 0;
    u64 rw[kIlp];
#pragma unroll
    for (int u = 0; u < kIlp; ++u) {
        const int t = t0 + 32 * u;
        ky[u] = 0;
        wi[u] = 0;
        rw[u] = 0;
        m[u] = 0;
        m2[u] = 0;
        sum[u] = 0;
        if (t < total) {
            while (t >= b.off[j + 1]) ++j;
            wi[u] = (b.lo[j] >> 6) + (t - b.off[j]);
            ky[u] = b.r[j].ky;
            rw[u] = range_word(wi[u], b.lo[j], b.hi[j]);
        }
        jj[u] = j;
        kmax = ky[u] > kmax ? ky[u] : kmax;
    }
    for (int q = 0; q < kmax; q += 2) {
        u64 x0[kIlp], x1[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            x0[u] = q < ky[u] ? __ldg(c.CT + (size_t)b.r[jj[u]].ids[q] * c.GW + wi[u]) : 0ull;
            x1[u] = q + 1 < ky[u] ? __ldg(c.CT + (size_t)b.r[jj[u]].ids[q + 1] * c.GW + wi[u]) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const u64 a = x0[u] & rw[u], e = x1[u] & rw[u];
            m2[u] |= (m[u] & (a | e)) | (a & e);
            m[u] |= a | e;
            if (SUM) sum[u] += __popcll(a) + __popcll(e);
        }
    }
}

// Reserves n consecutive slots of the warp's shard for each lane with one atomic
// per warp; returns the lane's first slot within the shard.
__device__ __forceinline__ u32 warp_reserve(int n, u32 *shard_count, int lane)
{
    const int incl = warp_incl_scan(n, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    u32 base = 0;
    if (total && lane == 0) base = atomicAdd(shard_count, (u32)total);
    base = __shfl_sync(kFull, base, 0);
    return base + (u32)(incl - n);
}

// Child record of a sparse parent: its samples are the parent's samples whose
// column word wi has bit bt set.  child_tumors fills the prefix and the tumor
// samples, child_normals the normal samples (not needed when the child is
// counted in closed form).
__device__ __forceinline__ void child_tumors(const Cohort &c, const Rec &parent, int L, int wi, int bt, Rec &out)
{
    out.p = prefix_with(parent.p, L, wi * 64 + bt);
    int ky = 0;
    for (int q = 0; q < parent.ky; ++q) {
        const int sm = parent.ids[q];
        if ((c.CT[(size_t)sm * c.GW + wi] >> bt) & 1ull) out.ids[ky++] = (u16)sm;
    }
    out.ky = (u16)ky;
}

__device__ __forceinline__ void child_normals(const Cohort &c, const Rec &parent, int wi, int bt, Rec &out)
{
    int kn = 0;
    for (int q = 0; q < parent.kn; ++q) {
        const int sm = parent.ids[kListT + q];
        if ((c.CN[(size_t)sm * c.GW + wi] >> bt) & 1ull) out.ids[kListT + kn++] = (u16)sm;
    }
    out.kn = (u16)kn;
}

// Child record of a dense parent (its y / n words in the warp scratch): samples
// from the rows of the child gene g, listed if few.
__device__ __forceinline__ void child_from_rows(const Cohort &c, const Batch &b, unsigned by, unsigned bn,
                                                const Prefix &parent, int L, int g, Rec &out)
{
    out.p = prefix_with(parent, L, g);
    const u64 *trow = c.T + (size_t)g * c.WTp;
    const u64 *nrow = c.N + (size_t)g * c.WNp;
    int ky = 0, kn = 0;
    for (unsigned bits = by; bits; bits &= bits - 1) ky += __popcll(b.ys[__ffs(bits) - 1] & trow[__ffs(bits) - 1]);
    for (unsigned bits = bn; bits; bits &= bits - 1) kn += __popcll(b.ns[__ffs(bits) - 1] & nrow[__ffs(bits) - 1]);
    if (!is_dense(ky, kn)) {
        int k = 0;
        for (unsigned bits = by; bits; bits &= bits - 1) {
            const int w = __ffs(bits) - 1;
            for (u64 y = b.ys[w] & trow[w]; y; y &= y - 1) out.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
        }
        k = kListT;
        for (unsigned bits = bn; bits; bits &= bits - 1) {
            const int w = __ffs(bits) - 1;
            for (u64 y = b.ns[w] & nrow[w]; y; y &= y - 1) out.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
        }
    }
    out.ky = sat16(ky);
    out.kn = sat16(kn);
}

// Scores the non-empty leaves m of sparse record j of the batch at column word
// wi: TP / FP from bit-sliced sums of the record's sample columns.  Returns the
// number scored.
__device__ __forceinline__ int score_item(const Cohort &c, const Solve &s, const Batch &b, int j, int wi, u64 m,
                                          int L, u64 thr, Key &best)
{
    const Rec &r = b.r[j];
    const int ky = r.ky, kn = r.kn;
    const int pt = bit_length(ky), pn = kn ? bit_length(kn) : 0;
    u64 tpl[kPlanesT] = {0, 0, 0, 0, 0};
    u64 fpl[kPlanesN] = {0, 0, 0, 0};
    // four column loads in flight at a time (a zero word leaves the planes as they are)
    for (int q = 0; q < ky; q += 4) {
        u64 x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = q + k < ky ? __ldg(c.CT + (size_t)r.ids[q + k] * c.GW + wi) : 0ull;
#pragma unroll
        for (int k = 0; k < 4; ++k) planes_add(tpl, x[k], pt);
    }
    for (int q = 0; q < kn; q += 4) {
        u64 x[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            x[k] = q + k < kn ? __ldg(c.CN + (size_t)r.ids[kListT + q + k] * c.GW + wi) : 0ull;
#pragma unroll
        for (int k = 0; k < 4; ++k) planes_add(fpl, x[k], pn);
    }
    int n = 0;
    while (m) {
        const int bt = __ffsll((long long)m) - 1;
        m &= m - 1;
        const int tp = planes_get(tpl, bt, pt);
        const int fp = planes_get(fpl, bt, pn);
        const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
        ++n;
        if (s1 < best.s || s1 < thr) continue;
        int po[kMaxH - 1];
#pragma unroll
        for (int q = 0; q < kMaxH - 1; ++q) po[q] = q < L ? b.po[j][q] : 0;
        const Key k = leaf_key(s1, po, L, c.orig[wi * 64 + bt]);
        if (key_better(k, best)) best = k;
    }
    return n;
}

// ---------------------------------------------------------------------------
// Phases of one greedy round.  Each is written for the whole grid of the kernel
// that runs it (blockIdx / gridDim): the one-kernel-per-phase path wraps each in
// its own kernel; the persistent solve kernel runs them back to back with a grid
// barrier in between.  Data that changes during a solve (U, frontier records,
// counters, slots) is read with L2-only loads so that a persistent kernel never
// sees a stale L1 line written by another SM.

// Re-scores the previous round's best candidates against the current U (one warp
// per key, lane w on word w).  A key still covering an uncovered tumor is a
// candidate of this round, so the largest value is a lower bound on this round's
// best: the leaf phase need not score what cannot reach it.
__device__ void rescore_candidates(const Cohort &c, const Solve &s, const Team &t)
{
    const int lane = threadIdx.x & 31;
    const int h = s.h;
    u64 hint = 0;
    for (int i = t.rank * (blockDim.x >> 5) + (threadIdx.x >> 5); i < kCandidates;
         i += t.size * (blockDim.x >> 5)) {
        Key k;
        k.s = __ldcg(&s.cand[i].s);
        if (k.s == 0) continue;
        k.t0 = __ldcg(&s.cand[i].t0);
        k.t1 = __ldcg(&s.cand[i].t1);
        k.t2 = __ldcg(&s.cand[i].t2);
        u64 y = 0, n = 0;
        if (lane < c.Wt) y = __ldcg(&s.U[lane]);
        if (lane < c.Wn) n = ~0ull;
        for (int q = 0; q < h; ++q) {
            const int g = (int)c.inv[key_get(k, q)];
            if (lane < c.Wt) y &= c.T[(size_t)g * c.WTp + lane];
            if (lane < c.Wn) n &= c.N[(size_t)g * c.WNp + lane];
        }
        int tp = __popcll(y), fp = __popcll(n);
        for (int off = 16; off; off >>= 1) {
            tp += __shfl_xor_sync(kFull, tp, off);
            fp += __shfl_xor_sync(kFull, fp, off);
        }
        if (tp == 0) continue;
        const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
        hint = s1 > hint ? s1 : hint;
    }
    if (lane == 0 && hint) atomicMax(s.best_hint, hint);
}

// Depth 1: y_1(g) = U & x_g for g in [0, G-h] (0-based).  For h = 1 these are
// the leaves and are scored here (the block's best goes to its slot); otherwise
// the non-empty ones (all of them with pruning off) become depth-1 records.
// Every thread of the block must call it.
__device__ void phase_level1(const Cohort &c, const Solve &s, int round, const Frontiers &f, u32 *counts,
                             const Team &t, const RoundIO &io)
{
    __shared__ u64 acc[kAccN];
    const int lane = threadIdx.x & 31;
    const int h = s.h;
    acc_begin(acc);
    if (h > 1 && !io.Ush) rescore_candidates(c, s, t);
    const int last = c.G - h;  // 0-based inclusive bound of depth 1
    u32 *my_count = counts + shard_slot(1, my_shard(t));
    Rec *out = f.F[1] + (size_t)my_shard(t) * f.cap[1];
    Key best = key_empty();
    for (int base = t.rank * blockDim.x; base < c.G; base += t.size * blockDim.x) {
        const int g = base + threadIdx.x;
        const bool in = g <= last && (s.nshards <= 1 || g % s.nshards == s.shard);  // split search: my genes
        int ky = 0;
        if (in) {
            const u64 *row = c.T + (size_t)g * c.WTp;
            for (int w = 0; w < c.Wt; ++w) ky += __popcll(row[w] & __ldcg(&s.U[w]));
        }
        const bool nonempty = ky > 0;
        const unsigned bin = __ballot_sync(kFull, in), bne = __ballot_sync(kFull, nonempty);
        if (lane == 0) {
            acc_add(acc, 0, (u64)__popc(bin));
            acc_add(acc, 1, (u64)__popc(bin & ~bne));
        }
        if (h == 1) {
            if (nonempty) {
                int fp = 0;
                const u64 *nrow = c.N + (size_t)g * c.WNp;
                for (int w = 0; w < c.Wn; ++w) fp += __popcll(nrow[w]);
                Key k = key_empty();
                k.s = s.a_num * (u64)ky + s.a_den * (u64)(c.Nn - fp) + 1;
                key_put(k, 0, c.orig[g]);
                if (key_better(k, best)) best = k;
            }
            continue;
        }
        const bool keep = s.prune == MH_PRUNE_OFF ? in : nonempty;
        const u32 pos = warp_reserve(keep ? 1 : 0, my_count, lane);
        if (!keep || pos >= f.cap[1]) continue;
        Rec r;
        r.p.w0 = (u64)g;
        r.p.w1 = 0;
        r.pad[0] = r.pad[1] = r.pad[2] = 0;
        const u64 *trow = c.T + (size_t)g * c.WTp;
        const u64 *nrow = c.N + (size_t)g * c.WNp;
        int kn = 0;
        for (int w = 0; w < c.Wn; ++w) kn += __popcll(nrow[w]);
        if (!is_dense(ky, kn)) {
            int k = 0;
            for (int w = 0; w < c.Wt; ++w)
                for (u64 y = trow[w] & __ldcg(&s.U[w]); y; y &= y - 1)
                    r.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
            k = kListT;
            for (int w = 0; w < c.Wn; ++w)
                for (u64 y = nrow[w]; y; y &= y - 1) r.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
        }
        r.ky = sat16(ky);
        r.kn = sat16(kn);
        copy_rec(&out[pos], &r);
    }
    if (h == 1) block_commit_best(best, io.slots, t.rank, io.overwrite);
    __syncthreads();
    if (threadIdx.x < 2 && acc[threadIdx.x])
        atomicAdd(s.cnt + ((size_t)round * h) * 2 + threadIdx.x, acc[threadIdx.x]);
}

// Per-warp cycle statistics of a phase (k = 0 expand, 1 leaf), for diagnostics,
// into the block accumulator slots 5 (sum), 6 (max), 7 (count).
__device__ __forceinline__ u64 *warp_cycle_slots()
{
    __shared__ u64 w[kMaxWarpsPerBlock];
    return w;
}
__device__ __forceinline__ void warp_cycles(u64 *acc, long long t0, int lane)
{
    (void)acc;
    if (lane == 0) warp_cycle_slots()[threadIdx.x >> 5] = (u64)(clock64() - t0);
}

__device__ __forceinline__ void warp_cycles_flush(const Solve &s, const u64 *acc, int k, int par)
{
    // after a block barrier: every warp's cycles of the phase are in its slot
    (void)acc;
    const int nw = (int)(blockDim.x >> 5);
    if (threadIdx.x == 5 || threadIdx.x == 6) {
        const u64 *w = warp_cycle_slots();
        u64 sum = 0, mx = 0;
        for (int i = 0; i < nw; ++i) {
            sum += w[i];
            mx = w[i] > mx ? w[i] : mx;
        }
        if (threadIdx.x == 5) atomicAdd(s.work + kWorkWarpSum + k, sum);
        else atomicMax(s.work + (par ? kWorkWarpMaxOdd : kWorkWarpMax) + k, mx);
    }
    if (threadIdx.x == 7) atomicAdd(s.work + kWorkWarpN + k, (u64)nw);
}

// Depths 2 .. h-1: the non-empty children (all children with pruning off) of
// every depth-(level-1) record become depth-level records.  Every thread of the
// block must call it; returns false (for every thread) if the input frontier
// overflowed.
__device__ bool phase_expand(const Cohort &c, const Solve &s, int round, int level, const Frontiers &f, u32 *counts,
                             Batch &b, const Team &t, const RoundIO &io_in)
{
    __shared__ u64 acc[kAccN];
    __shared__ int overflow;
    const long long t0 = clock64();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = level - 1;
    RoundIO io = io_in;
    const bool fm = io.fm;
    if (level != 2) io.Ush = nullptr;  // depth-1 nodes are built only as the parents of depth 2
    if (threadIdx.x == 0) overflow = 0;
    acc_begin(acc);
    const long long n_in = io.Ush ? (long long)(c.G - s.h + 1) : front_open(counts, level - 1, f.cap[level - 1], b.soff, lane);
    if (n_in < 0 && lane == 0) overflow = 1;
    __syncthreads();
    if (overflow) return false;
    const u32 count = (u32)n_in;
    Depth1 d1;
    const Rec *Fin = f.F[level - 1];
    const u32 cap_in = f.cap[level - 1];
    const u32 cap = f.cap[level];
    u32 *my_count = counts + shard_slot(level, my_shard(t));
    Rec *Fout = f.F[level] + (size_t)my_shard(t) * cap;
    const int hi_bound = c.G - s.h + level - 1;  // 0-based inclusive bound of this depth
    const bool all_children = s.prune == MH_PRUNE_OFF;
    u64 cutn = 0;  // prefixes cut by the score bound
    const u64 nw = (u64)t.size * (blockDim.x >> 5), gw = (u64)t.rank * (blockDim.x >> 5) + warp;
    u64 visited = 0, alive = 0;
    u64 leaf_vis = 0, leaf_alive = 0;  // closed-form leaves of single-sample children (level = h - 1)
    u64 *deep = acc + kAccDeep;
    const int h = s.h;
    Dispenser disp((u32)nw, (u32)gw, count, dispenser_counters(counts, level - 2));
    for (u64 first = disp.next(lane); first < count; first = disp.next(lane)) {
        unsigned dense;
        // the best score known to exist in the round decides whether single-sample
        // subtrees may be counted in closed form
        // (with champions known, every sample whose champion is known qualifies: no
        // threshold needed)
        int single = 1;
        u64 thr = 0;
        if (!(s.champ && s.prune == MH_PRUNE_PAPER && c.CC)) {
            if (lane == 0) thr = *(volatile u64 *)io.hint;
            thr = __shfl_sync(kFull, thr, 0);
            single = single_sample_mode(c, s, thr);
        }
        u64 alive_cf = 0;
        if (fm) single = 0;
        const bool bound = s.prune == MH_PRUNE_BOUND;
        const int total = batch_prepare(c, io, d1, Fin, cap_in, first, nw, (int)disp.R, count, L, hi_bound, all_children, b,
                                        lane, dense, visited, h, single, s.champ_ok, alive_cf, deep, nullptr, fm,
                                        thr, s.a_num, s.a_den * (u64)c.Nn + 1, bound ? &cutn : nullptr);
        // sparse records: (record, column word) items spread over the lanes
        int j = 0;
        for (int tb = 0; tb < total; tb += 32 * kIlp) {
            int jj[kIlp], wi[kIlp], ky[kIlp];
            u64 m[kIlp], rw[kIlp];
            if (fm) {
                // children shared by two or more uncovered tumors only
                u64 m1[kIlp];
                int sum[kIlp];
                sibling_items2<false>(c, b, tb + lane, total, j, jj, wi, ky, m1, m, sum);
            } else {
                sibling_items(c, b, tb + lane, total, j, jj, wi, ky, m, rw);
#pragma unroll
                for (int u = 0; u < kIlp; ++u) {
                    alive += (u64)__popcll(m[u]);
                    if (all_children) m[u] = rw[u];
                }
            }
            // spread the children of each item round over all lanes: lane i builds
            // children i, i+32, ... of the warp, whichever lane's item they came from
#pragma unroll
            for (int u = 0; u < kIlp; ++u) {
                const int n = __popcll(m[u]);
                const int incl = warp_incl_scan(n, lane);
                const int tot = __shfl_sync(kFull, incl, 31);
                if (tot == 0) continue;
                b.ys[lane] = m[u];
                b.ns[lane] = ((u64)(u32)jj[u] << 32) | (u32)wi[u];
                b.cx[lane] = incl - n;
                if (lane == 31) b.cx[32] = incl;
                __syncwarp();
                for (int k0 = 0; k0 < tot; k0 += 32) {
                    const int k = k0 + lane;
                    Rec child;
                    bool emit = false;
                    if (k < tot) {
                        int lo = 0, hi = 31;  // source lane: last with cx <= k
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (b.cx[mid] <= k) lo = mid; else hi = mid - 1;
                        }
                        u64 x = b.ys[lo];
                        for (int r = k - b.cx[lo]; r > 0; --r) x &= x - 1;
                        const u64 jw = b.ns[lo];
                        const int g = (int)(u32)jw * 64 + __ffsll((long long)x) - 1;
                        const Rec &parent = b.r[(int)(jw >> 32)];
                        child.pad[0] = child.pad[1] = child.pad[2] = 0;
                        child_tumors(c, parent, L, (int)(u32)jw, g & 63, child);
                        emit = true;
                        if (fm) alive += (u64)(child.ky - 1);  // the depth's correction
                        // a child of a listed parent is listed: one sample -> closed form
                        if (single && child.ky == 1 && single_sample_closed(single, s.champ_ok, child.ids[0])) {
                            single_sample_count(c, h, level, g, child.ids[0], leaf_vis, leaf_alive, deep);
                            emit = false;
                        } else {
                            child_normals(c, parent, (int)(u32)jw, g & 63, child);
                        }
                    }
                    const u32 pos = warp_reserve(emit ? 1 : 0, my_count, lane);
                    if (emit && pos < cap) copy_rec(&Fout[pos], &child);
                }
                __syncwarp();
            }
        }
        // dense records: the whole warp, one child gene per lane, tested on the rows
        // (y_{l-1} & x_g, the running intersection of Algorithm 2)
        while (dense) {
            const int jd = __ffs(dense) - 1;
            dense &= dense - 1;
            const Prefix p = b.r[jd].p;
            const int lo = b.lo[jd], hi = b.hi[jd];
            unsigned by, bn;
            dense_setup(c, s, p, L, b, by, bn, lane);
            for (int gb = lo; gb <= hi; gb += 32) {
                const int g = gb + lane;
                int kyc = 0, smp = 0;
                if (g <= hi) {
                    const u64 *trow = c.T + (size_t)g * c.WTp;
                    for (unsigned bits = by; bits; bits &= bits - 1) {
                        const int w = __ffs(bits) - 1;
                        const u64 yw = b.ys[w] & trow[w];
                        if (yw) smp = w * 64 + __ffsll((long long)yw) - 1;
                        kyc += __popcll(yw);
                    }
                }
                bool closed = false;
                if (fm) {
                    closed = kyc < 2;  // single-sample children: in the per-sample sums
                    if (!closed) alive += (u64)(kyc - 1);
                } else {
                    alive += (u64)(kyc > 0);
                    if (single && kyc == 1 && g <= hi && single_sample_closed(single, s.champ_ok, smp)) {
                        single_sample_count(c, h, level, g, smp, leaf_vis, leaf_alive, deep);
                        closed = true;
                    }
                }
                const bool emit = g <= hi && (all_children || kyc > 0) && !closed;
                const u32 pos = warp_reserve(emit ? 1 : 0, my_count, lane);
                if (emit && pos < cap) {
                    Rec child;
                    child.pad[0] = child.pad[1] = child.pad[2] = 0;
                    child_from_rows(c, b, by, bn, p, L, g, child);
                    copy_rec(&Fout[pos], &child);
                }
            }
            __syncwarp();
        }
    }
    visited = warp_sum_u64(visited);
    alive = warp_sum_u64(alive);
    leaf_vis = warp_sum_u64(leaf_vis);
    leaf_alive = warp_sum_u64(leaf_alive);
    cutn = warp_sum_u64(cutn);
    if (lane == 0 && cutn && s.cut) atomicAdd(s.cut + (size_t)round * h + (L - 1), cutn);
    d1.visited = warp_sum_u64(d1.visited);
    d1.pruned = warp_sum_u64(d1.pruned);
    if (lane == 0) {
        // fm: the depth's corrections (visited, surviving), finished at the end of the round
        acc_add(acc, 0, visited);
        acc_add(acc, 1, fm ? alive : visited - alive);
        acc_add(acc, 8, d1.visited);
        acc_add(acc, 9, d1.pruned);
        acc_add(deep, 2 * h, leaf_vis);
        acc_add(deep, 2 * h + 1, leaf_alive);
    }
    warp_cycles(acc, t0, lane);
    __syncthreads();
    if (!io.build) {
        if (threadIdx.x < 2 && acc[threadIdx.x])
            atomicAdd(s.cnt + ((size_t)round * s.h + (level - 1)) * 2 + threadIdx.x, acc[threadIdx.x]);
        if (threadIdx.x >= 8 && threadIdx.x < 10 && acc[threadIdx.x])
            atomicAdd(s.cnt + ((size_t)round * s.h) * 2 + (threadIdx.x - 8), acc[threadIdx.x]);
        acc_flush_deep(s, round, acc);
    }
    warp_cycles_flush(s, acc, 0, io.par);
    return true;
}

// Depth h (leaves): every non-empty leaf is a candidate with score
// S = a_num * TP + a_den * (Nn - FP); the best (score desc, original tuple asc)
// goes to the block's slot.  A record whose bound a_num * |y| + a_den * Nn is
// below the best score known to exist cannot hold the round's winner, so its
// leaves are tested (and counted) but not scored.  Every thread of the block
// must call it; returns false (for every thread) if the input frontier overflowed.
__device__ bool phase_leaf(const Cohort &c, const Solve &s, int round, const Frontiers &f, u32 *counts, Batch &b,
                           const Team &t, const RoundIO &io_in)
{
    __shared__ u64 acc[kAccN];
    __shared__ int overflow;
    const long long t0 = clock64();
    Key best = key_empty();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int h = s.h, L = h - 1;
    // the champions of the uncovered tumors (a share of them per block) are
    // candidates of the round and stand for its TP = 1 leaves
    if (s.champ && io_in.Ush) {
        for (int smp = t.rank * (int)blockDim.x + (int)threadIdx.x; smp < c.Nt; smp += t.size * (int)blockDim.x) {
            if (!((io_in.Ush[smp >> 6] >> (smp & 63)) & 1ull) || !__ldcg(s.champ_ok + smp)) continue;
            Key k;
            k.s = __ldcg(&s.champ[smp].s);
            k.t0 = __ldcg(&s.champ[smp].t0);
            k.t1 = __ldcg(&s.champ[smp].t1);
            k.t2 = __ldcg(&s.champ[smp].t2);
            if (k.s && key_better(k, best)) best = k;
        }
    }
    RoundIO io = io_in;
    if (h != 2) io.Ush = nullptr;  // depth-1 nodes are built only as the parents of the leaves of h = 2
    if (threadIdx.x == 0) overflow = 0;
    acc_begin(acc);
    const long long n_in = io.Ush ? (long long)(c.G - 1) : front_open(counts, h - 1, f.cap[h - 1], b.soff, lane);
    if (n_in < 0 && lane == 0) overflow = 1;
    __syncthreads();
    if (overflow) return false;
    const u32 count = (u32)n_in;
    Depth1 d1;
    const Rec *Fin = f.F[h - 1];
    const u32 cap_in = f.cap[h - 1];
    u64 visited = 0, alive = 0, words = 0, prefixes = 0, scored = 0, dense_n = 0, cutn = 0;
    const u64 nn_term = s.a_den * (u64)c.Nn + 1;
    const u64 nw = (u64)t.size * (blockDim.x >> 5), gw = (u64)t.rank * (blockDim.x >> 5) + warp;
    Dispenser disp((u32)nw, (u32)gw, count, dispenser_counters(counts, h - 2));
    for (u64 first = disp.next(lane); first < count; first = disp.next(lane)) {
        unsigned dense;
        // only candidates at least as good as the best score known to exist can win
        u64 thr = 0;
        if (lane == 0) thr = *(volatile u64 *)io.hint;
        thr = warp_max_u64(thr > best.s ? thr : best.s);
        u64 alive_cf = 0;
        // (with pruning off, the empty depth-1 nodes built here still have leaves)
        const int total = batch_prepare(c, io, d1, Fin, cap_in, first, nw, (int)disp.R, count, L, c.G - 1,
                                        io.Ush != nullptr && s.prune == MH_PRUNE_OFF, b, lane, dense, visited, h,
                                        single_sample_mode(c, s, thr), s.champ_ok, alive_cf, acc + kAccDeep,
                                        c.orig, false, thr, s.a_num, nn_term,
                                        s.prune == MH_PRUNE_BOUND ? &cutn : nullptr);
        alive += alive_cf;
        prefixes += (u64)(lane < (int)disp.R && first + (u64)lane * nw < count);
        int j = 0;
        for (int tb = 0; tb < total; tb += 32 * kIlp) {
            int jj[kIlp], wi[kIlp], ky[kIlp];
            u64 m[kIlp], rw[kIlp];
            sibling_items(c, b, tb + lane, total, j, jj, wi, ky, m, rw);
#pragma unroll
            for (int u = 0; u < kIlp; ++u) {
                alive += (u64)__popcll(m[u]);
                words += (u64)ky[u];
                if (m[u] && s.a_num * (u64)ky[u] + nn_term >= thr) {
                    scored += (u64)score_item(c, s, b, jj[u], wi[u], m[u], L, thr, best);
                    words += (u64)(ky[u] + b.r[jj[u]].kn);
                }
            }
        }
        // dense records: the whole warp, one leaf gene per lane, tested and scored
        // on the rows (popcounts over the prefix's non-zero words only)
        while (dense) {
            const int jd = __ffs(dense) - 1;
            dense &= dense - 1;
            const Prefix p = b.r[jd].p;
            const int lo = b.lo[jd], hi = b.hi[jd];
            const int ky = b.r[jd].ky;
            unsigned by, bn;
            dense_setup(c, s, p, L, b, by, bn, lane);
            if (lane == 0) ++dense_n;
            int po[kMaxH - 1];
#pragma unroll
            for (int q = 0; q < kMaxH - 1; ++q) po[q] = q < L ? b.po[jd][q] : 0;
            const bool score = s.a_num * (u64)ky + nn_term >= thr;
            const int nzy = __popc(by);
            for (int gb = lo; gb <= hi; gb += 32) {
                const int g = gb + lane;
                if (g > hi) break;
                const u64 *trow = c.T + (size_t)g * c.WTp;
                int tp = 0;
                for (unsigned bits = by; bits; bits &= bits - 1) {
                    const int w = __ffs(bits) - 1;
                    tp += __popcll(b.ys[w] & trow[w]);
                }
                words += (u64)nzy;
                if (tp == 0) continue;
                ++alive;
                if (!score) continue;
                const u64 *nrow = c.N + (size_t)g * c.WNp;
                int fp = 0;
                for (unsigned bits = bn; bits; bits &= bits - 1) {
                    const int w = __ffs(bits) - 1;
                    fp += __popcll(b.ns[w] & nrow[w]);
                }
                const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
                ++scored;
                if (s1 < best.s || s1 < thr) continue;
                const Key k = leaf_key(s1, po, L, c.orig[g]);
                if (key_better(k, best)) best = k;
            }
            __syncwarp();
        }
        // publish the warp's best score so that other warps can skip hopeless records
        const u64 wbest = warp_max_u64(best.s);
        if (lane == 0 && wbest > thr) atomicMax(io.hint, wbest);
    }
    visited = warp_sum_u64(visited);
    alive = warp_sum_u64(alive);
    cutn = warp_sum_u64(cutn);
    if (lane == 0 && cutn && s.cut) atomicAdd(s.cut + (size_t)round * h + (L - 1), cutn);
    words = warp_sum_u64(words);
    prefixes = warp_sum_u64(prefixes);
    scored = warp_sum_u64(scored);
    d1.visited = warp_sum_u64(d1.visited);
    d1.pruned = warp_sum_u64(d1.pruned);
    if (lane == 0) {
        acc_add(acc, 0, visited);
        acc_add(acc, 1, visited - alive);
        acc_add(acc, 2, words);
        acc_add(acc, 3, prefixes);
        acc_add(acc, 4, scored);
        acc_add(acc, 8, d1.visited);
        acc_add(acc, 9, d1.pruned);
    }
    warp_cycles(acc, t0, lane);
    // dense records counted through the block's slot 7 is taken: use an atomic per warp (rare)
    if (lane == 0 && dense_n) atomicAdd(s.work + kWorkDense, dense_n);
    __syncthreads();
    if (threadIdx.x < 2 && acc[threadIdx.x])
        atomicAdd(s.cnt + ((size_t)round * h + (h - 1)) * 2 + threadIdx.x, acc[threadIdx.x]);
    if (threadIdx.x == 2 && acc[2]) atomicAdd(s.work + kWorkColWords, acc[2]);
    if (threadIdx.x == 3 && acc[3]) atomicAdd(s.work + kWorkPrefixes, acc[3]);
    if (threadIdx.x == 4 && acc[4]) atomicAdd(s.work + kWorkScored, acc[4]);
    if (threadIdx.x >= 8 && threadIdx.x < 10 && acc[threadIdx.x])
        atomicAdd(s.cnt + ((size_t)round * h) * 2 + (threadIdx.x - 8), acc[threadIdx.x]);
    acc_flush_deep(s, round, acc);
    warp_cycles_flush(s, acc, 1, io.par);
    block_commit_best(best, io.slots, t.rank, io.overwrite);
    return true;
}

// End of a round, by one block: reduce the per-block bests, record the winner
// with its TP / FP, clear the tumors it covers (DelCols), keep the best other
// candidates for the next round's threshold, reset the frontier counters and
// advance the round; raise the done flag when nothing was found, every tumor is
// covered or the round limit is reached.  Every thread of the block must call it.
// step (split search only): 1 = stop after the reduction, writing the shard's best
// key to xbest[0]; 2 = skip the reduction and apply the merged winner xbest[1].
__device__ void phase_finalize(const Cohort &c, const Solve &s, u32 *counts, int nslots, int step = 0)
{
    __shared__ Key wbest[kMaxWarpsPerBlock];
    __shared__ int gs[kMaxH], os[kMaxH];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int h = s.h;
    Key best = key_empty();
    if (step == 2) nslots = 0;
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        Key k;
        k.s = __ldcg(&s.slots[i].s);
        k.t0 = __ldcg(&s.slots[i].t0);
        k.t1 = __ldcg(&s.slots[i].t1);
        k.t2 = __ldcg(&s.slots[i].t2);
        if (key_better(k, best)) best = k;
        s.slots[i] = key_empty();
    }
    // the best kCandidates of the warps' lane bests become next round's candidates
    Key mine = best;
    const int per_warp = (kCandidates + nwarps - 1) / nwarps;
    for (int r = 0; r < per_warp; ++r) {
        const Key m = warp_max_key(mine);
        const int idx = warp * per_warp + r;
        if (lane == 0 && idx < kCandidates) s.cand[idx] = m;
        if (m.s != 0 && mine.s == m.s && mine.t0 == m.t0 && mine.t1 == m.t1 && mine.t2 == m.t2) mine = key_empty();
        if (r == 0 && lane == 0) wbest[warp] = m;
    }
    if (step != 2)
        for (int i = threadIdx.x; i < kMaxH * kShards; i += blockDim.x) counts[i * kShardStride] = 0;
    __syncthreads();
    if (warp == 0) {
        best = lane < nwarps ? wbest[lane] : key_empty();
        best = warp_max_key(best);
        if (step == 1 && lane == 0) s.xbest[0] = best;  // the shard's best; the round goes on
        if (step == 2) {
            best.s = __ldcg(&s.xbest[1].s);
            best.t0 = __ldcg(&s.xbest[1].t0);
            best.t1 = __ldcg(&s.xbest[1].t1);
            best.t2 = __ldcg(&s.xbest[1].t2);
        }
        const int round = *(volatile int *)&s.state[kStRound];
        const bool last_round = round + 1 >= *(volatile int *)&s.state[kStMaxRounds];
        if (step == 1) best = key_empty();  // nothing is applied in step 1
        if (lane == 0 && step != 1) {
            *(volatile u64 *)s.best_hint = 0;
            s.state[kStRound] = round + 1;
        }
        if (lane < 2 && step != 1) {  // diagnostics: the round's longest warps
            s.work[kWorkWarpMaxSum + lane] += __ldcg(&s.work[kWorkWarpMax + lane]);
            s.work[kWorkWarpMax + lane] = 0;
        }
        if (step == 1) {
        } else if (best.s == 0) {
            if (lane == 0) s.state[kStDone] = 1;
        } else {
            if (lane < h) {
                const int o = key_get(best, lane);
                os[lane] = o;
                gs[lane] = (int)c.inv[o];
            }
            __syncwarp();
            u64 y = 0, n = 0, u = 0;
            if (lane < c.Wt) {
                u = __ldcg(&s.U[lane]);
                y = u;
                for (int i = 0; i < h; ++i) y &= c.T[(size_t)gs[i] * c.WTp + lane];
            }
            if (lane < c.Wn) {
                n = ~0ull;
                for (int i = 0; i < h; ++i) n &= c.N[(size_t)gs[i] * c.WNp + lane];
            }
            int tp = __popcll(y), fp = __popcll(n);
            for (int off = 16; off; off >>= 1) {
                tp += __shfl_xor_sync(kFull, tp, off);
                fp += __shfl_xor_sync(kFull, fp, off);
            }
            if (lane < c.Wt) {
                u &= ~y;
                s.U[lane] = u;
            }
            const unsigned left = __ballot_sync(kFull, u != 0);
            if (lane == 0) {
                const int k = *(volatile int *)&s.state[kStK];
                int *r = s.res + (size_t)k * (h + 2);
                for (int i = 0; i < h; ++i) r[i] = os[i];
                r[h] = tp;
                r[h + 1] = fp;
                s.state[kStK] = k + 1;
                if (!left || last_round) s.state[kStDone] = 1;
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// One kernel per phase.

__global__ void k_transpose(int G, const u64 *rows, int row_stride, int samples, int GW, u64 *cols)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)samples * GW;
    if (t >= total) return;
    const int s = (int)(t / GW), wi = (int)(t % GW);
    const int sw = s >> 6, sb = s & 63;
    u64 word = 0;
    for (int b = 0; b < 64; ++b) {
        const int g = wi * 64 + b;
        if (g < G) word |= ((rows[(size_t)g * row_stride + sw] >> sb) & 1ull) << b;
    }
    cols[t] = word;
}

__global__ void k_solve_init(Cohort c, Solve s, int max_rounds)
{
    const int w = threadIdx.x;
    if (w < c.WTp) {
        const int rem = c.Nt - 64 * w;
        s.U[w] = rem >= 64 ? ~0ull : (rem <= 0 ? 0ull : ((1ull << rem) - 1ull));
    }
    if (w < kStateWords) s.state[w] = w == kStMaxRounds ? max_rounds : 0;
}

__global__ void __launch_bounds__(kThreads) k_level1(const __grid_constant__ Cohort c, const __grid_constant__ Solve s,
                                                     const __grid_constant__ Frontiers f, u32 *counts)
{
    if (halted(s)) return;
    phase_level1(c, s, s.state[kStRound], f, counts, grid_team(), launch_io(s));
}

__global__ void __launch_bounds__(kThreads, 4) k_expand(const __grid_constant__ Cohort c, const __grid_constant__ Solve s,
                                                        int level, const __grid_constant__ Frontiers f, u32 *counts)
{
    __shared__ Batch scratch[kWarpsPerBlock];
    if (halted(s)) return;
    if (!phase_expand(c, s, s.state[kStRound], level, f, counts, scratch[threadIdx.x >> 5], grid_team(),
                      launch_io(s)) &&
        threadIdx.x == 0)
        s.state[kStOverflow] = 1;
}

__global__ void __launch_bounds__(kThreads, 3) k_leaf(const __grid_constant__ Cohort c, const __grid_constant__ Solve s,
                                                      const __grid_constant__ Frontiers f, u32 *counts)
{
    __shared__ Batch scratch[kWarpsPerBlock];
    if (halted(s)) return;
    if (!phase_leaf(c, s, s.state[kStRound], f, counts, scratch[threadIdx.x >> 5], grid_team(), launch_io(s)) &&
        threadIdx.x == 0)
        s.state[kStOverflow] = 1;
}

__global__ void __launch_bounds__(kThreads) k_finalize(const __grid_constant__ Cohort c, const __grid_constant__ Solve s,
                                                       u32 *counts)
{
    if (halted(s)) return;
    phase_finalize(c, s, counts, s.nslots);
}

__global__ void __launch_bounds__(kThreads) k_finalize_split(const __grid_constant__ Cohort c,
                                                             const __grid_constant__ Solve s, u32 *counts, int step)
{
    if (halted(s)) return;
    phase_finalize(c, s, counts, s.nslots, step);
}

// ---------------------------------------------------------------------------
// Persistent solve: every round of the greedy loop in one cooperative launch.

// Grid barrier with a bounded wait: a block that waits longer than about two
// seconds records a timeout in the state and returns false instead of hanging.
// One atomic per block: arrivals count up across the barriers of a launch (the
// word starts at zero), so barrier k ends when the count reaches (k + 1) * nblocks,
// and a block learns k from the count it found.  With `sample`, a block that finds
// *sample set raises g->flag before it arrives; after the barrier every block reads
// the same flag (the OR of what the blocks found), so they take the same decision.
// Arrival with release and acquire semantics at GPU scope (the block's writes,
// ordered before thread 0 by the block barrier, become visible to the blocks that
// see the arrival), and the waiters' acquiring load.
__device__ __forceinline__ unsigned arrive_acq_rel(unsigned *p)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
    return old;
}
__device__ __forceinline__ unsigned load_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool grid_sync(GridSync *g, int *state, int nblocks, const int *sample = nullptr)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        if (sample && *(volatile const int *)sample) *(volatile int *)&g->flag = 1;
        const unsigned old = arrive_acq_rel(&g->arrived);
        const unsigned target = (old / (unsigned)nblocks + 1u) * (unsigned)nblocks;
        // the last block to arrive goes on at once; the others wait for the count
        unsigned long long spins = 0;
        while (old + 1u != target && (int)(load_acquire(&g->arrived) - target) < 0) {
            __nanosleep(32);
            if (++spins > (1ull << 25)) {
                atomicExch(&state[kStError], kErrTimeout);
                ok = 0;
                break;
            }
        }
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Re-scores keys[0 .. kCandidates) against U (the block's copy): the largest S + 1
// of a key that still covers an uncovered tumor is a candidate score of the round,
// a lower bound on its best; merged into *hint.  A warp takes 32 / lpk keys at a
// time, lpk lanes each (one lane per row word), and issues the loads of all their
// rows together.
__device__ void block_rescore(const Cohort &c, const Solve &s, const Key *keys, const u64 *Ush, u64 *hint)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int h = s.h;
    int lpk = 1;
    while (lpk < c.Wt || lpk < c.Wn || lpk < h) lpk <<= 1;
    const int kpp = 32 / lpk, sub = lane / lpk, w = lane % lpk, lead = lane - w;
    u64 best = 0;
    for (int base = warp * kpp; base < kCandidates; base += nwarps * kpp) {
        const int i = base + sub;
        const Key k = i < kCandidates ? keys[i] : key_empty();
        const bool live = k.s != 0;
        const int gq = (live && w < h) ? (int)c.inv[key_get(k, w)] : 0;
        u64 y = (live && w < c.Wt) ? Ush[w] : 0ull;
        u64 n = (live && w < c.Wn) ? ~0ull : 0ull;
#pragma unroll
        for (int q = 0; q < kMaxH; ++q) {
            if (q >= h) break;
            const int g = __shfl_sync(kFull, gq, lead + q);
            if (live && w < c.Wt) y &= c.T[(size_t)g * c.WTp + w];
            if (live && w < c.Wn) n &= c.N[(size_t)g * c.WNp + w];
        }
        int tp = __popcll(y), fp = __popcll(n);
        for (int off = lpk >> 1; off; off >>= 1) {
            tp += __shfl_xor_sync(kFull, tp, off);
            fp += __shfl_xor_sync(kFull, fp, off);
        }
        if (live && tp > 0) {
            const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
            best = s1 > best ? s1 : best;
        }
    }
    best = warp_max_u64(best);
    if (lane == 0 && best) atomicMax(hint, best);
}

// Per-sample champions, computed once per solve before its first round.  For a
// tumor sample s every h-subset of its genes is a leaf whose tumor intersection
// holds s; valued with TP = 1 it scores a_num + a_den * (Nn - FP).  champ[s] is the
// largest key among them (least FP, then the smallest tuple of original indices).
// In any round with s uncovered, the h-subsets of s's genes that no other
// uncovered tumor carries are exactly the leaves of s's single-sample subtrees
// and score their TP = 1 value; the others are leaves of the multi-sample part of
// the tree (TP >= 2) and score at least that value there.  Hence the round's best
// key is the larger of the best multi-sample leaf and the best champion of an
// uncovered tumor, and single-sample subtrees need no scoring: this is the same
// argmax, evaluated without visiting the TP = 1 leaves one by one.
//
// Search: one warp per sample over the subsets in lexicographic order of original
// indices (each sample's genes listed ascending by original index), the last gene
// spread over the lanes; the first subset with FP = 0 is the champion.  A sample
// whose search passes kChampBudget subsets is left unknown (champ_ok = 0): its
// single-sample subtrees are then searched and scored like the rest.
constexpr int kChampBudget = 1 << 15;

__device__ void phase_champions(const Cohort &c, const Solve &s, const Team &t, Batch &b)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int h = s.h;
    for (int smp = t.rank * nwarps + warp; smp < c.Nt; smp += t.size * nwarps) {
        const u32 off = __ldg(c.SO + smp);
        const int m = (int)(__ldg(c.SO + smp + 1) - off);
        const u16 *go = c.SLo + off;
        Key best = key_empty();
        int ok = 1;
        if (m >= h) {
            int idx[kMaxH];  // positions of the prefix genes 0 .. h-2 (the same in every lane)
            for (int q = 0; q < h - 1; ++q) idx[q] = q;
            int best_fp = 0x7fffffff, best_j = 0, evaluated = 0;
            int best_idx[kMaxH];
            for (int q = 0; q < kMaxH; ++q) best_idx[q] = 0;
            for (;;) {
                // normal intersection of the prefix, word `lane`
                u64 pn = 0;
                if (lane < c.Wn) {
                    pn = ~0ull;
                    for (int q = 0; q < h - 1; ++q) pn &= c.N[(size_t)c.inv[go[idx[q]]] * c.WNp + lane];
                }
                b.ns[lane] = pn;
                __syncwarp();
                bool zero = false;
                for (int j0 = idx[h - 2] + 1; j0 < m; j0 += 32) {
                    const int j = j0 + lane;
                    unsigned v = 0xffffffffu;  // (FP, lane): least FP, then the first in order
                    if (j < m) {
                        const u64 *nrow = c.N + (size_t)c.inv[go[j]] * c.WNp;
                        int fp = 0;
                        for (int w = 0; w < c.Wn; ++w) fp += __popcll(b.ns[w] & nrow[w]);
                        v = ((unsigned)fp << 5) | (unsigned)lane;
                    }
                    const unsigned mv = __reduce_min_sync(kFull, v);
                    evaluated += m - j0 < 32 ? m - j0 : 32;
                    if ((int)(mv >> 5) < best_fp) {
                        best_fp = (int)(mv >> 5);
                        best_j = j0 + (int)(mv & 31u);
                        for (int q = 0; q < h - 1; ++q) best_idx[q] = idx[q];
                    }
                    if (best_fp == 0) {
                        zero = true;
                        break;
                    }
                }
                __syncwarp();
                if (zero) break;
                if (evaluated > kChampBudget) {
                    ok = 0;
                    break;
                }
                // next prefix in lexicographic order (position q is at most m - h + q)
                int q = h - 2;
                while (q >= 0 && idx[q] == m - h + q) --q;
                if (q < 0) break;
                ++idx[q];
                for (int r = q + 1; r < h - 1; ++r) idx[r] = idx[r - 1] + 1;
            }
            if (ok) {
                best.s = s.a_num + s.a_den * (u64)(c.Nn - best_fp) + 1;
                for (int q = 0; q < h - 1; ++q) key_put(best, q, go[best_idx[q]]);
                key_put(best, h - 1, go[best_j]);
            }
        }
        if (lane == 0) {
            s.champ[smp] = best;
            s.champ_ok[smp] = ok;
        }
        __syncwarp();
    }
}

// First round of a solve: no candidate of an earlier round bounds the round's best
// score yet.  Every uncovered tumor is covered by the combination of its h last
// genes in search order (its most frequently mutated ones); the best of their
// scores is a lower bound on the round's best, merged into *hint, so that the
// first round can already skip what cannot win.
__device__ void block_seed(const Cohort &c, const Solve &s, const Team &t, const u64 *Ush, u64 *hint)
{
    const int h = s.h;
    u64 best = 0;
    for (int smp = t.rank * (int)blockDim.x + (int)threadIdx.x; smp < c.Nt; smp += t.size * (int)blockDim.x) {
        if (!((Ush[smp >> 6] >> (smp & 63)) & 1ull)) continue;
        const u64 *col = c.CT + (size_t)smp * c.GW;
        int gs[kMaxH];
        int n = 0;
        for (int w = (c.G - 1) >> 6; w >= 0 && n < h; --w) {
            u64 x = __ldg(col + w);
            while (x && n < h) {
                const int bt = 63 - __clzll((long long)x);
                gs[n++] = w * 64 + bt;
                x &= ~(1ull << bt);
            }
        }
        if (n < h) continue;
        int tp = 0, fp = 0;
        for (int w = 0; w < c.Wt; ++w) {
            u64 y = Ush[w];
            for (int q = 0; q < h; ++q) y &= c.T[(size_t)gs[q] * c.WTp + w];
            tp += __popcll(y);
        }
        for (int w = 0; w < c.Wn; ++w) {
            u64 y = ~0ull;
            for (int q = 0; q < h; ++q) y &= c.N[(size_t)gs[q] * c.WNp + w];
            fp += __popcll(y);
        }
        const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
        best = s1 > best ? s1 : best;
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0 && best) atomicMax(hint, best);
}

// ---------------------------------------------------------------------------
// Counting by per-sample sums.  A depth-l node (an in-bound prefix P) survives iff
// some uncovered tumor carries all its genes.  Summing over the uncovered tumors s
// the number A_l(s) of in-bound depth-l prefixes made of s's genes counts every
// surviving node |y_l(P)| times, so
//   alive[l]   = sum_{s in U} A_l(s) - sum_{P at depth l, |y_l(P)| >= 2} (|y_l(P)| - 1),
// and since a depth-l node is visited once per surviving parent, one per gene of
// the parent's loop range (last(P), hi(l)],
//   visited[l] = sum_{s in U} V_l(s) - sum_{P at depth l-1, |y(P)| >= 2} (|y(P)| - 1) (hi(l) - last(P)),
// with V_l(s) those ranges summed over the in-bound depth-(l-1) prefixes of s's
// genes.  A_l and V_l depend only on s's genes and the loop bounds, so they are
// computed once per solve; the corrections come from the nodes that two or more
// uncovered tumors share, the only nodes this mode builds and searches (with the
// per-sample champions standing for every TP = 1 leaf).  The counters are those
// of Algorithm 2's loops exactly (as u64, i.e. modulo 2^64 like the counters
// themselves), and no node of a single uncovered tumor is ever visited.

// A_l(s) and V_l(s) of every tumor s from its genes b_1 < b_2 < ... (search
// positions): with f_k(b) the in-bound k-prefixes of s's genes ending at b,
// f_1(b) = [b <= hi(1)], f_k(b) = [b <= hi(k)] * sum_{b' < b} f_{k-1}(b'),
// A_k = sum_b f_k(b) and V_{k+1} = sum_b f_k(b) (hi(k+1) - b).
__device__ __noinline__ void phase_sample_sums(const Cohort &c, const Solve &s, const Team &t)
{
    const int h = s.h;
    const int hi0 = c.G - h - 1;  // hi(k) = hi0 + k (0-based, inclusive)
    for (int smp = t.rank * (int)blockDim.x + (int)threadIdx.x; smp < c.Nt; smp += t.size * (int)blockDim.x) {
        const u32 off = __ldg(c.SO + smp);
        const int m = (int)(__ldg(c.SO + smp + 1) - off);
        u64 S[kMaxH + 1], A[kMaxH + 1], V[kMaxH + 1];
#pragma unroll
        for (int k = 0; k <= kMaxH; ++k) S[k] = A[k] = V[k] = 0;
        for (int i = 0; i < m; ++i) {
            const int b = (int)__ldg(c.SL + off + i);
            // descending k: f_k reads the sum of f_{k-1} over the earlier genes
#pragma unroll
            for (int k = kMaxH; k >= 1; --k) {
                if (k > h || b > hi0 + k) continue;
                const u64 f = k == 1 ? 1ull : S[k - 1];
                A[k] += f;
                S[k] += f;
                if (k < h) V[k + 1] += f * (u64)(hi0 + k + 1 - b);
            }
        }
        u64 *out = s.ssum + (size_t)smp * 2 * h;
#pragma unroll
        for (int k = 1; k <= kMaxH; ++k) {
            if (k > h) break;
            out[k - 1] = A[k];
            out[h + k - 1] = V[k];
        }
    }
}

// tot[0 .. 2h) = the per-sample sums over all tumors.
__device__ void block_sample_totals(const Cohort &c, const Solve &s, u64 *tot)
{
    const int h2 = 2 * s.h, lane = threadIdx.x & 31;
    if (threadIdx.x < 2 * kMaxH) tot[threadIdx.x] = 0;
    __syncthreads();
    for (int k = 0; k < h2; ++k) {
        u64 v = 0;
        for (int smp = threadIdx.x; smp < c.Nt; smp += blockDim.x)
            v += __ldcg(s.ssum + (size_t)smp * h2 + k);
        v = warp_sum_u64(v);
        if (lane == 0 && v) atomicAdd(&tot[k], v);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Incremental rounds.  U only shrinks from one round to the next, so the nodes
// that two or more uncovered tumors share in a later round are among those of
// round 0, and a node's tumor intersection -- its size, its children's TP and its
// leaves' scores -- changes only if it holds a tumor that the previous winner
// covered.  With counting by per-sample sums, round 0 builds the shared
// ("multi-sample") nodes of every depth below the leaves and keeps them for the
// whole solve, and evaluates every leaf parent once, caching its best leaf key
// among its leaves with TP >= 2 and the sum of TP - 1 over them.  A later round
// scans the kept nodes, brings up to date only those holding a newly covered
// tumor (re-evaluating the leaf parents among them), reads everything else from
// the caches, and ends after one grid barrier.  The argmax and every counter are
// those of a full search of the round.

__device__ __forceinline__ bool in_mask(const u64 *m, int smp) { return (m[smp >> 6] >> (smp & 63)) & 1ull; }

// Signature of a record's tumor samples: OR of 1 << (s & 63) (~0 when not listed).
__device__ __forceinline__ u64 sample_sig(const Rec &r)
{
    if (is_dense(r.ky, r.kn)) return ~0ull;
    u64 g = 0;
    for (int q = 0; q < (int)r.ky; ++q) g |= 1ull << (r.ids[q] & 63);
    return g;
}

// Slot (shard * cap + offset) of record i of a sharded frontier (soff from front_open).
__device__ __forceinline__ u32 front_slot(u32 cap_s, const int *soff, u32 i)
{
    int lo = 0, hi = kShards - 1;  // last shard with soff <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((u32)soff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    return (u32)lo * cap_s + (i - (u32)soff[lo]);
}

// Uncovered tumors carrying gene g: its static record's listed tumors in U, or
// the popcount of its row and U.
__device__ __forceinline__ u32 gene_uncovered(const Cohort &c, const u64 *Ush, int g)
{
    const Rec &sr = c.GR[g];
    const int ky = (int)__ldg(&sr.ky);
    if (ky <= kListT) {
        u32 k = 0;
        for (int q = 0; q < ky; ++q) k += (u32)in_mask(Ush, (int)__ldg(&sr.ids[q]));
        return k;
    }
    const u64 *trow = c.T + (size_t)g * c.WTp;
    u32 k = 0;
    for (int w = 0; w < c.Wt; ++w) k += (u32)__popcll(__ldg(trow + w) & Ush[w]);
    return k;
}

// Brings a kept record of depth L up to date with U; returns true if its tumor
// intersection changed (always with force).  Listed samples: the covered ones are
// dropped.  Unlisted: the intersection is recounted from the rows, and listed
// once it is small enough.
__device__ bool refresh_record(const Cohort &c, const u64 *Ush, const u64 *Csh, int L, Rec &r, bool force)
{
    if (!is_dense(r.ky, r.kn)) {
        int k = 0;
        for (int q = 0; q < (int)r.ky; ++q) {
            const int smp = r.ids[q];
            if (in_mask(Ush, smp)) r.ids[k++] = (u16)smp;
        }
        const bool changed = k != (int)r.ky;
        r.ky = (u16)k;
        return changed || force;
    }
    const u64 *rows[kMaxH - 1];
#pragma unroll
    for (int i = 0; i < kMaxH - 1; ++i) rows[i] = i < L ? c.T + (size_t)prefix_gene(r.p, i) * c.WTp : nullptr;
    if (!force) {
        // unchanged unless the prefix rows meet a covered tumor (few words of Csh are non-zero)
        bool hit = false;
        for (int w = 0; w < c.Wt && !hit; ++w) {
            u64 y = Csh[w];
            if (!y) continue;
#pragma unroll
            for (int i = 0; i < kMaxH - 1; ++i)
                if (i < L) y &= __ldg(rows[i] + w);
            hit = y != 0;
        }
        if (!hit) return false;
    }
    // recount over U, four words (and their rows) in flight at a time
    int ky = 0;
    for (int w0 = 0; w0 < c.Wt; w0 += 4) {
        u64 y[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) y[k] = w0 + k < c.Wt ? Ush[w0 + k] : 0ull;
#pragma unroll
        for (int i = 0; i < kMaxH - 1; ++i) {
            if (i >= L) break;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (w0 + k < c.Wt) y[k] &= __ldg(rows[i] + w0 + k);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) ky += __popcll(y[k]);
    }
    r.ky = sat16(ky);
    if (!is_dense(ky, r.kn)) {
        int k = 0;
        for (int w = 0; w < c.Wt; ++w) {
            u64 y = Ush[w];
            for (int i = 0; i < L && y; ++i) y &= __ldg(c.T + (size_t)prefix_gene(r.p, i) * c.WTp + w);
            for (; y; y &= y - 1) r.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
        }
        k = kListT;
        for (int w = 0; w < c.Wn; ++w) {
            u64 n = ~0ull;
            for (int i = 0; i < L; ++i) n &= __ldg(c.N + (size_t)prefix_gene(r.p, i) * c.WNp + w);
            for (; n; n &= n - 1) r.ids[k++] = (u16)(w * 64 + __ffsll((long long)n) - 1);
        }
    }
    return true;
}

// One (record j, column word wi) item of a leaf parent: the record's tumor
// columns, eight loads in flight at a time, give the non-empty children m, the
// children of two or more tumors m2, the children's summed sizes (corr = that sum
// minus |m|, the item's share of sum(TP - 1) over its TP >= 2 leaves) and
// bit-sliced TP counts; the normal columns, read only when m2 is non-empty, give
// FP; the children in m2 are scored into best.
constexpr int kEvalLoads = 8;
// The leaves of one prefix, packed: (score + 1) << 16 | (0xffff - o), o the leaf
// gene's original index.  Inserting a smaller o into the same sorted prefix gives
// the lexicographically smaller tuple, so among the leaves of one prefix the larger
// packed value is the larger key (scores below 2^44, genes below 2^16).
__device__ __forceinline__ u64 pack_leaf(u64 s1, int o) { return (s1 << 16) | (u64)(0xffff - o); }
__device__ __forceinline__ Key unpack_leaf(u64 p, const int *po, int L)
{
    return leaf_key(p >> 16, po, L, 0xffff - (int)(p & 0xffffull));
}
__device__ __forceinline__ void leaf_item_eval(const Cohort &c, const Solve &s, const Rec &r, int wi, u64 rw, u64 &corr,
                                               u64 &pbest)
{
    const int ky = r.ky, kn = r.kn;
    const int pt = bit_length(ky), pn = kn ? bit_length(kn) : 0;
    u64 tpl[kPlanesT] = {0, 0, 0, 0, 0};
    u64 m = 0, m2 = 0;
    int sum = 0;
    for (int q = 0; q < ky; q += kEvalLoads) {
        u64 x[kEvalLoads];
#pragma unroll
        for (int k = 0; k < kEvalLoads; ++k)
            x[k] = q + k < ky ? __ldg(c.CT + (size_t)r.ids[q + k] * c.GW + wi) & rw : 0ull;
#pragma unroll
        for (int k = 0; k < kEvalLoads; ++k) {
            m2 |= m & x[k];
            m |= x[k];
            sum += __popcll(x[k]);
            planes_add(tpl, x[k], pt);
        }
    }
    corr = (u64)(sum - __popcll(m));
    if (!m2) return;
    u64 fpl[kPlanesN] = {0, 0, 0, 0};
    for (int q = 0; q < kn; q += kEvalLoads) {
        u64 x[kEvalLoads];
#pragma unroll
        for (int k = 0; k < kEvalLoads; ++k)
            x[k] = q + k < kn ? __ldg(c.CN + (size_t)r.ids[kListT + q + k] * c.GW + wi) : 0ull;
#pragma unroll
        for (int k = 0; k < kEvalLoads; ++k) planes_add(fpl, x[k], pn);
    }
    while (m2) {
        const int bt = __ffsll((long long)m2) - 1;
        m2 &= m2 - 1;
        const int tp = planes_get(tpl, bt, pt);
        const int fp = planes_get(fpl, bt, pn);
        const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
        if (s1 < (pbest >> 16)) continue;
        const u64 pk = pack_leaf(s1, c.orig[wi * 64 + bt]);
        pbest = pk > pbest ? pk : pbest;
    }
}

// Original indices of a kept record's prefix genes, ascending, in the record's
// spare bytes (prefixes of up to kPadGenes genes).
constexpr int kPadGenes = 6;
__device__ __forceinline__ u16 *pad_po(Rec &r) { return reinterpret_cast<u16 *>(r.pad); }
// The ascending original indices of a leaf parent's L prefix genes.
__device__ __forceinline__ void record_po(const Cohort &c, Rec &r, int L, int *po)
{
#pragma unroll
    for (int q = 0; q < kMaxH - 1; ++q) po[q] = 0;
    if (L <= kPadGenes) {
        for (int q = 0; q < L; ++q) po[q] = pad_po(r)[q];
        return;
    }
    for (int q = 0; q < L; ++q) {
        const int v = c.orig[prefix_gene(r.p, q)];
        int k = q - 1;
        while (k >= 0 && po[k] > v) {
            po[k + 1] = po[k];
            --k;
        }
        po[k + 1] = v;
    }
}

// Merges the per-lane keys of one item step into the records' best keys: items of
// a step sit on the lanes in record order, so a segmented warp maximum leaves each
// record's best on its first lane, which merges it into rb.
__device__ __forceinline__ void merge_item_keys(Batch &b, int jr, u64 p, u64 corr, int lane)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const u64 po = __shfl_down_sync(kFull, p, off);
        const u64 co = __shfl_down_sync(kFull, corr, off);
        const int jo = __shfl_down_sync(kFull, jr, off);
        if (lane + off < 32 && jo == jr) {
            p = po > p ? po : p;
            corr += co;
        }
    }
    const int jp = __shfl_up_sync(kFull, jr, 1);
    if (jr >= 0 && (lane == 0 || jp != jr)) {
        b.rc[jr] += corr;
        if (p > b.rb[jr].s) b.rb[jr].s = p;
    }
    __syncwarp();
}

// Evaluates the leaf parents b.r[j] (depth L = h - 1) of the lanes with `live`:
// b.rb[j] = the best key among the record's leaves with TP >= 2 (empty if none),
// b.rc[j] = the sum of TP - 1 over them.  TP = 1 leaves are left to the
// champions.  The (record, column word) items are spread over the lanes as in the
// leaf phase; unlisted records take the row path, the whole warp per record.
__device__ void leaf_parents_eval(const Cohort &c, const Solve &s, Batch &b, bool live, int L, int lane)
{
    int lo = 1, hi = 0, ky = 0, kn = 0;
    b.rb[lane] = key_empty();
    b.rc[lane] = 0;
    if (live) {
        Rec &r = b.r[lane];
        lo = prefix_gene(r.p, L - 1) + 1;
        hi = c.G - 1;
        ky = r.ky;
        kn = r.kn;
        if (L <= kPadGenes) {  // ascending original indices of the prefix (leaf keys)
            for (int q = 0; q < L; ++q) b.po[lane][q] = pad_po(r)[q];
        } else {
            for (int q = 0; q < L; ++q) {
                const u16 v = c.orig[prefix_gene(r.p, q)];
                int k = q - 1;
                while (k >= 0 && b.po[lane][k] > v) {
                    b.po[lane][k + 1] = b.po[lane][k];
                    --k;
                }
                b.po[lane][k + 1] = v;
            }
        }
    }
    b.lo[lane] = lo;
    b.hi[lane] = hi;
    const bool any = live && hi >= lo;
    const bool dense = any && is_dense(ky, kn);
    unsigned dmask = __ballot_sync(kFull, dense);
    const int nw = (any && !dense) ? (hi >> 6) - (lo >> 6) + 1 : 0;
    const int incl = warp_incl_scan(nw, lane);
    b.off[lane] = incl - nw;
    if (lane == 31) b.off[kBatch] = incl;
    __syncwarp();
    const int total = __shfl_sync(kFull, incl, 31);
    int j = 0;
    for (int tb = 0; tb < total; tb += 32) {
        const int t = tb + lane;
        const bool valid = t < total;
        u64 ib = 0, corr = 0;
        if (valid) {
            while (t >= b.off[j + 1]) ++j;
            const int wi = (b.lo[j] >> 6) + (t - b.off[j]);
            leaf_item_eval(c, s, b.r[j], wi, range_word(wi, b.lo[j], b.hi[j]), corr, ib);
        }
        merge_item_keys(b, valid ? j : -1, ib, corr, lane);
    }
    if (live && !dense && b.rb[lane].s != 0) {  // the packed best of each listed record as its key
        int po[kMaxH - 1];
#pragma unroll
        for (int q = 0; q < kMaxH - 1; ++q) po[q] = q < L ? b.po[lane][q] : 0;
        b.rb[lane] = unpack_leaf(b.rb[lane].s, po, L);
    }
    __syncwarp();
    // unlisted records: the whole warp, one leaf gene per lane, on the rows
    while (dmask) {
        const int jd = __ffs(dmask) - 1;
        dmask &= dmask - 1;
        const Prefix p = b.r[jd].p;
        const int dlo = b.lo[jd], dhi = b.hi[jd];
        unsigned by, bn;
        dense_setup(c, s, p, L, b, by, bn, lane);
        int po[kMaxH - 1];
#pragma unroll
        for (int q = 0; q < kMaxH - 1; ++q) po[q] = q < L ? b.po[jd][q] : 0;
        Key best = key_empty();
        u64 corr = 0;
        for (int g = dlo + lane; g <= dhi; g += 32) {
            const u64 *trow = c.T + (size_t)g * c.WTp;
            int tp = 0;
            for (unsigned bits = by; bits; bits &= bits - 1) {
                const int w = __ffs(bits) - 1;
                tp += __popcll(b.ys[w] & trow[w]);
            }
            if (tp < 2) continue;
            corr += (u64)(tp - 1);
            const u64 *nrow = c.N + (size_t)g * c.WNp;
            int fp = 0;
            for (unsigned bits = bn; bits; bits &= bits - 1) {
                const int w = __ffs(bits) - 1;
                fp += __popcll(b.ns[w] & nrow[w]);
            }
            const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
            if (s1 < best.s) continue;
            const Key k = leaf_key(s1, po, L, c.orig[g]);
            if (key_better(k, best)) best = k;
        }
        best = warp_max_key(best);
        corr = warp_sum_u64(corr);
        if (lane == 0) {
            b.rb[jd] = best;
            b.rc[jd] = corr;
        }
        __syncwarp();
    }
}

// Round 0 of an incremental solve with h = 2: the depth-1 nodes that two or more
// uncovered tumors share (the leaf parents) into the depth-1 frontier.  Every
// thread of the block must call it.
__device__ void phase_build1(const Cohort &c, const Solve &s, const Frontiers &f, u32 *counts, Batch &b,
                             const Team &t, const u64 *Ush)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int n = c.G - s.h + 1;  // depth-1 nodes
    u32 *my_count = counts + shard_slot(1, my_shard(t));
    Rec *out = f.F[1] + (size_t)my_shard(t) * f.cap[1];
    for (int base = (t.rank * nwarps + warp) * 32; base < n; base += t.size * nwarps * 32) {
        const int g = base + lane;
        bool keep = false;
        if (g < n) keep = gene_record(c, Ush, g, b.r[lane]) && b.r[lane].ky >= 2;
        const u32 pos = warp_reserve(keep ? 1 : 0, my_count, lane);
        if (keep && pos < f.cap[1]) {
            b.r[lane].pad[0] = b.r[lane].pad[1] = b.r[lane].pad[2] = 0;
            copy_rec(&out[pos], &b.r[lane]);
        }
    }
}

// One incremental round, or with force the evaluation that follows round 0's
// build, by every block of the team.  Depth 1: in round 0 the block counts its
// share of the genes; later, each gene of a tumor covered since the previous
// round loses one uncovered tumor.  Kept records: the block scans its share of
// every depth (record i to block i mod B, then to warp (i / B) mod W, so that
// records appended together spread out), brings up to date those holding a
// covered tumor (their signature meets the covered tumors'), re-evaluates the leaf
// parents among them, and takes the others' best keys from the caches.  After
// round 0 each warp keeps its live records in an on-chip list (built once they
// fit) and reads from L2 only the records a covered tumor touches; changed leaf
// parents are evaluated by the whole block through a queue of tasks.  What it
// adds to the round's counter slots are CHANGES of the running totals (in round
// 0, the corrections themselves), which the end of the round accumulates: depth
// 1's surviving count; (k - 1)(hi(2) - g) over the genes shared by k >= 2
// uncovered tumors; for a kept node of depth l >= 2 with k >= 2 tumors, k - 1 to
// depth l and (k - 1)(hi(l+1) - last) to depth l + 1; the leaf parents' sums of
// TP - 1 to depth h; and the per-sample sums of the tumors the last winner
// covered.  The block's best key (leaf caches, and the champions of its uncovered
// tumors, which stand for the TP = 1 leaves) goes to its slot.  Every thread of
// the block must call it; returns false (for every thread) if round 0 overflowed
// a frontier.
constexpr int kScanIlp = 4;  // records whose signature and cached score a lane loads at once
// changed leaf parents a block spreads over its warps per round (one-block-per-SM
// builds; the smaller blocks keep their shared memory for occupancy)
constexpr int kEvalQueue = 64;
// soffs / nrec / tab_ok: the kept frontiers' shard offsets and sizes, read once per
// launch (after round 0's build) into the block's shared memory.
struct FrontTab {
    int soff[kMaxH][kShards + 1];
    long long n[kMaxH];
    int ok;
    // per warp: its list of live kept records (built in a round after round 0, when
    // they fit) and, per depth, where the depth's entries start and how many there are
    signed char lok[kMaxWarpsPerBlock];
    short lbase[kMaxWarpsPerBlock][kMaxH];
    short lcnt[kMaxWarpsPerBlock][kMaxH];
};
// Entries of a warp's list of live kept records (one-block-per-SM builds).  After
// round 0 a record that no longer holds two uncovered tumors can never hold them
// again (U only shrinks): DelCols has emptied it for good, and the list drops it.
// The list keeps each live record's slot, sample signature and cached best score
// on chip, so a round reads only the records that a covered tumor touches.
constexpr int kList = 160;
template <int kLWarps>
struct LiveLists {
    u32 slot[kLWarps][kList];
    u64 sig[kLWarps][kList];
    u64 ls[kLWarps][kList];
    u16 dq[kLWarps][kList];  // a round's touched entries, by position
};
template <int kQueue, int kLWarps>
__device__ bool phase_update(const Cohort &c, const Solve &s, int round, const Frontiers &f, const u32 *counts,
                             Batch &b, const Team &t, const RoundIO &io, const u64 *Csh, bool force, FrontTab &ft)
{
    __shared__ u64 acc[kAccN];
    __shared__ int overflow;
    __shared__ int qn;  // the block's queue of changed leaf parents
    __shared__ Rec qrec[kQueue > 0 ? kQueue : 1];
    __shared__ u32 qslot[kQueue > 0 ? kQueue : 1];
    __shared__ u64 qlco[kQueue > 0 ? kQueue : 1];
    __shared__ short qidx[kQueue > 0 ? kQueue : 1];  // list entry of a queued record (-1: none)
    __shared__ signed char qwarp[kQueue > 0 ? kQueue : 1];
    __shared__ int qlo[kQueue > 0 ? kQueue : 1], qtasks[kQueue > 0 ? kQueue : 1];  // first leaf gene, tasks
    __shared__ u64 qbest[kQueue > 0 ? kQueue : 1];
    __shared__ u32 qcorr[kQueue > 0 ? kQueue : 1];  // a record's sum of TP - 1 stays below 2^27
    // a queued leaf parent's first leaf gene and tasks of 32 column words (set when it is queued)
    auto queue_tasks = [&](int q, const Rec &r, int L) {
        const int lo = prefix_gene(r.p, L - 1) + 1;
        qlo[q] = lo;
        qtasks[q] = (((c.G - 1) >> 6) - (lo >> 6) + 1 + 31) >> 5;
        qbest[q] = 0;
        qcorr[q] = 0;
    };
    __shared__ LiveLists<(kLWarps > 0 ? kLWarps : 1)> lv;
    const long long t0 = clock64();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int h = s.h;
    const u64 *Ush = io.Ush;
    const int qcap = kQueue < 32 * nwarps ? kQueue : 32 * nwarps;
    // each tumor's offset into the per-sample gene lists, on chip (one-block-per-SM builds)
    __shared__ u32 so_sh[kLWarps > 0 ? kMaxWords * 64 + 1 : 1];
    // the changes of the depths' corrections: per warp, summed over the warps at the
    // end (one-block-per-SM builds), else block-wide in acc
    __shared__ u64 wdeep[kLWarps > 0 ? kLWarps : 1][2 * kMaxH + 2];
    u64 *deep = acc + kAccDeep;
    if (kLWarps > 0)
        for (int i = lane; i < 2 * kMaxH + 2; i += 32) wdeep[warp][i] = 0;
    auto deep_add = [&](int i, u64 v) {
        if (kLWarps > 0) wdeep[warp][i] += v;
        else acc_add(deep, i, v);
    };
    if (threadIdx.x == 0) {
        overflow = 0;
        qn = 0;
    }
    if (kLWarps > 0 && (force || !ft.ok))  // once per launch, published by acc_begin's barrier
        for (int i = (int)threadIdx.x; i <= c.Nt; i += (int)blockDim.x) so_sh[i] = __ldg(c.SO + i);
    acc_begin(acc);
    u64 csig = 0;
    for (int w = 0; w < c.Wt; ++w) csig |= Csh[w];
    Key best = key_empty();
    // After round 0 the block's last warp takes the champions and depth 1 while the
    // others scan the kept records, so that their chains of loads overlap; the lead
    // block (rank 0), which ends the round with more work than the others, scans no
    // records then.
    const int gwarp = nwarps - 1;
    const bool side = force || warp == gwarp;
    const int sstride = force ? (int)blockDim.x : 32, sbase = force ? (int)threadIdx.x : lane;
    for (int smp = t.rank * sstride + sbase; side && smp < c.Nt; smp += t.size * sstride) {
        if (!in_mask(Ush, smp)) continue;
        Key k;  // the four words in one round trip
        k.s = __ldcg(&s.champ[smp].s);
        k.t0 = __ldcg(&s.champ[smp].t0);
        k.t1 = __ldcg(&s.champ[smp].t1);
        k.t2 = __ldcg(&s.champ[smp].t2);
        if (k.s != 0 && key_better(k, best)) best = k;
    }
    // the lead's idle warps: the previous round's longest warps join the diagnostics
    if (t.rank == 0 && !side) {
        if (warp == 0 && lane < 2 && round > 0) {
            const int mx = (((round - 1) & 1) ? kWorkWarpMaxOdd : kWorkWarpMax) + lane;
            s.work[kWorkWarpMaxSum + lane] += __ldcg(&s.work[mx]);
            s.work[mx] = 0;
        }
    }
    // depth 1
    if (side) {
        const int last1 = c.G - h, hi2 = c.G - h + 1;
        u64 alive1 = 0, corrv = 0, sv = 0;
        if (force) {  // the genes of a contiguous share, one per thread
            const int g0 = (int)((long long)c.G * t.rank / t.size), g1 = (int)((long long)c.G * (t.rank + 1) / t.size);
            for (int g = g0 + (int)threadIdx.x; g < g1; g += (int)blockDim.x) {
                const u32 k = gene_uncovered(c, Ush, g);
                s.gk[g] = k;
                if (g <= last1) {
                    alive1 += (u64)(k >= 1);
                    if (k >= 2) corrv += (u64)(k - 1) * (u64)(hi2 - g);
                }
            }
        } else {
            // each gene of a covered tumor loses one uncovered tumor, and the tumor's
            // per-sample sums of depths 2..h leave the totals: they join the running
            // totals that the end of the round subtracts (lane k < h - 1: the visited
            // sum of depth k + 2, lane h - 1 + k: its surviving sum)
            const int h2 = 2 * h;
            const bool sl = lane < 2 * (h - 1);
            const int sd = lane < h - 1 ? lane + 2 : lane - (h - 1) + 2;
            const int sidx = lane < h - 1 ? h + sd - 1 : sd - 1;
            for (int smp = t.rank; smp < c.Nt; smp += t.size) {
                if (!in_mask(Csh, smp)) continue;
                if (sl) sv += __ldcg(s.ssum + (size_t)smp * h2 + sidx);
                const u32 off = kLWarps > 0 ? so_sh[smp] : __ldg(c.SO + smp);
                const int m = (int)((kLWarps > 0 ? so_sh[smp + 1] : __ldg(c.SO + smp + 1)) - off);
                for (int q = lane; q < m; q += 32) {
                    const int g = (int)__ldg(c.SL + off + q);
                    const u32 old = atomicSub(s.gk + g, 1u);
                    if (g <= last1) {
                        if (old == 1) alive1 -= 1ull;
                        if (old >= 2) corrv -= (u64)(hi2 - g);
                    }
                }
            }
        }
        alive1 = warp_sum_u64(alive1);
        corrv = warp_sum_u64(corrv);
        if (lane == 0) {
            deep_add(3, alive1);
            deep_add(4, corrv);
        }
        __syncwarp();
        if (sv) deep_add(lane < h - 1 ? 2 * (lane + 2) : 2 * (lane - (h - 1) + 2) + 1, sv);
    }
    // kept records: depth 1 (h = 2) or 2 .. h-1; the deepest are the leaf parents
    if (force || !ft.ok) {  // their sizes and shard offsets, once per launch
        for (int l = h == 2 ? 1 : 2; l <= h - 1; ++l) {
            if (warp == 0) {
                const long long nl = front_open(counts, l, f.cap[l], b.soff, lane);
                if (nl < 0 && lane == 0) overflow = 1;
                for (int i = lane; i <= kShards; i += 32) ft.soff[l][i] = b.soff[i];
                if (lane == 0) ft.n[l] = nl;
            }
        }
        __syncthreads();
        if (overflow) return false;
        if (threadIdx.x == 0) ft.ok = 1;
    }
    // after round 0 a warp whose live records fit its list scans the list only; a warp
    // builds its list in the first round after round 0 in which they fit
    const bool use_list = kLWarps > 0 && !force && ft.lok[warp] == 1;
    const bool build_list = kLWarps > 0 && !force && ft.lok[warp] == 0;
    int lfill = 0;
    bool lfit = true;
    for (int l = h == 2 ? 1 : 2; l <= h - 1; ++l) {
        const long long n_in = ft.n[l];
        if (build_list && lane == 0) ft.lbase[warp][l] = (short)lfill;
        const int *soff = ft.soff[l];
        const bool leafp = l == h - 1;
        const int hiN = c.G - h + l;  // hi(l + 1), 0-based
        u64 dA = 0, dV = 0, dL = 0;
        // scanners: every block and warp in round 0; later all warps but the last of
        // every block but the lead
        const bool split = !force && t.size > 1 && nwarps > 1;
        const u64 B = split ? (u64)(t.size - 1) : (u64)t.size, W = split ? (u64)(nwarps - 1) : (u64)nwarps;
        const u64 rk = split ? (u64)(t.rank - 1) : (u64)t.rank;
        const u64 n = (n_in < 0 || (split && (t.rank == 0 || warp == gwarp))) ? 0ull : (u64)n_in;
        if (use_list) {
            // this warp's live records: drop the dead ones, pick out those a covered tumor
            // touches, and take the best cached leaf of the others
            u32 *Lslot = lv.slot[warp] + ft.lbase[warp][l];
            u64 *Lsig = lv.sig[warp] + ft.lbase[warp][l], *Lls = lv.ls[warp] + ft.lbase[warp][l];
            u16 *dq = lv.dq[warp];
            const int cnt = ft.lcnt[warp][l];
            int wpos = 0, nd = 0;
            u64 lmax = 0;
            for (int j0 = 0; j0 < cnt; j0 += 32) {
                const int j = j0 + lane;
                u32 sl = 0;
                u64 sg = 0, lsv = 0;
                if (j < cnt) {
                    sl = Lslot[j];
                    sg = Lsig[j];
                    lsv = Lls[j];
                }
                const bool keep = sg != 0;
                const unsigned km = __ballot_sync(kFull, keep);
                __syncwarp();
                const int pos = wpos + __popc(km & ((1u << lane) - 1u));
                if (keep) {
                    Lslot[pos] = sl;
                    Lsig[pos] = sg;
                    Lls[pos] = lsv;
                }
                wpos += __popc(km);
                const bool dirty = keep && (sg & csig) != 0;
                const unsigned dm = __ballot_sync(kFull, dirty);
                if (dirty) dq[nd + __popc(dm & ((1u << lane) - 1u))] = (u16)pos;
                nd += __popc(dm);
                if (keep && !dirty && lsv > lmax) lmax = lsv;
            }
            __syncwarp();
            if (lane == 0) ft.lcnt[warp][l] = (short)wpos;
            // the untouched records' best cached leaves: a lane's first record with the
            // warp's largest cached score is read now and merged after the touched
            // records (their loads overlap); further ties, rare, after that
            const u64 wmax = leafp ? warp_max_u64(lmax) : 0ull;
            int hitj = -1;
            bool more = false;
            Key kc = key_empty();
            if (wmax != 0) {  // warp-uniform (the lanes' bests differ)
                const bool want = wmax >= best.s;
                for (int j0 = 0; j0 < wpos; j0 += 32) {
                    const int j = j0 + lane;
                    if (want && j < wpos && Lls[j] == wmax && (Lsig[j] & csig) == 0) {
                        if (hitj < 0) hitj = j;
                        else more = true;
                    }
                }
                if (hitj >= 0) {
                    const u32 sl = Lslot[hitj];
                    kc.s = wmax;
                    kc.t0 = __ldcg(&f.lb[l][sl].t0);
                    kc.t1 = __ldcg(&f.lb[l][sl].t1);
                    kc.t2 = __ldcg(&f.lb[l][sl].t2);
                }
                if (__any_sync(kFull, more)) {  // before any touched record changes its entry
                    for (int j0 = 0; j0 < wpos; j0 += 32) {
                        const int j = j0 + lane;
                        if (j < wpos && j != hitj && Lls[j] == wmax && (Lsig[j] & csig) == 0) {
                            const u32 sl = Lslot[j];
                            Key k2;
                            k2.s = wmax;
                            k2.t0 = __ldcg(&f.lb[l][sl].t0);
                            k2.t1 = __ldcg(&f.lb[l][sl].t1);
                            k2.t2 = __ldcg(&f.lb[l][sl].t2);
                            if (key_better(k2, best)) best = k2;
                        }
                    }
                }
            }
            for (int d0 = 0; d0 < nd; d0 += 32) {  // the touched ones, one per lane
                const bool act = d0 + lane < nd;
                const int pos = act ? (int)dq[d0 + lane] : 0;
                const u32 sl = act ? Lslot[pos] : 0u;
                Rec &r = b.r[lane];
                bool changed = false;
                int kyn = 0;
                u64 lco = 0;
                if (act) {
                    load_rec(&r, f.F[l] + sl);
                    if (leafp) lco = __ldcg(f.lc[l] + sl);
                    const int kyo = (int)r.ky;
                    changed = refresh_record(c, Ush, Csh, l, r, false);
                    kyn = r.ky;
                    if (changed) {
                        const u64 nsg = kyn >= 2 ? sample_sig(r) : 0ull;
                        f.sig[l][sl] = nsg;
                        Lsig[pos] = nsg;
                        copy_rec(f.F[l] + sl, &r);
                        if (l >= 2) {
                            const u64 fo = kyo >= 2 ? (u64)(kyo - 1) : 0ull, fn = kyn >= 2 ? (u64)(kyn - 1) : 0ull;
                            dA += fn - fo;
                            dV += (fn - fo) * (u64)(hiN - prefix_gene(r.p, l - 1));
                        }
                    } else if (leafp) {  // nothing covered in it after all: its cached best stands
                        const u64 lsv = Lls[pos];
                        if (lsv != 0 && lsv >= best.s) {
                            Key kc;
                            kc.s = lsv;
                            kc.t0 = __ldcg(&f.lb[l][sl].t0);
                            kc.t1 = __ldcg(&f.lb[l][sl].t1);
                            kc.t2 = __ldcg(&f.lb[l][sl].t2);
                            if (key_better(kc, best)) best = kc;
                        }
                    }
                }
                const bool eval = leafp && changed && kyn >= 2;
                if (leafp && changed && kyn < 2) {
                    f.lb[l][sl] = key_empty();
                    f.lc[l][sl] = 0;
                    dL -= lco;
                    Lls[pos] = 0;
                }
                bool queued = false;
                if (eval && !is_dense(r.ky, r.kn)) {
                    const int qp = atomicAdd(&qn, 1);
                    if (qp < qcap) {
                        copy_rec(&qrec[qp], &r);
                        queue_tasks(qp, r, l);
                        qslot[qp] = sl;
                        qlco[qp] = lco;
                        qidx[qp] = (short)(ft.lbase[warp][l] + pos);
                        qwarp[qp] = (signed char)warp;
                        queued = true;
                    }
                }
                const bool here = eval && !queued;
                if (__ballot_sync(kFull, here)) {
                    leaf_parents_eval(c, s, b, here, l, lane);
                    if (here) {
                        const Key kb = b.rb[lane];
                        f.lb[l][sl] = kb;
                        f.lc[l][sl] = b.rc[lane];
                        Lls[pos] = kb.s;
                        dL += b.rc[lane] - lco;
                        if (kb.s != 0 && key_better(kb, best)) best = kb;
                    }
                    __syncwarp();
                }
            }
            if (hitj >= 0 && key_better(kc, best)) best = kc;
        }
        for (u64 k = 0; !use_list && rk + B * ((u64)warp + W * 32ull * kScanIlp * k) < n; ++k) {
            u32 slot[kScanIlp];
            u64 sg[kScanIlp], ls[kScanIlp];
#pragma unroll
            for (int u = 0; u < kScanIlp; ++u) {
                const u64 i = rk + B * ((u64)warp + W * ((u64)lane + 32ull * (kScanIlp * k + u)));
                slot[u] = 0;
                sg[u] = ls[u] = 0;
                if (i < n) {
                    slot[u] = front_slot(f.cap[l], soff, (u32)i);
                    sg[u] = force ? ~0ull : __ldcg(f.sig[l] + slot[u]);
                    if (leafp && !force) ls[u] = __ldcg(&f.lb[l][slot[u]].s);
                }
            }
#pragma unroll
            for (int u = 0; u < kScanIlp; ++u) {
                const bool dirty = sg[u] != 0 && (force || (sg[u] & csig) != 0);
                bool cached = leafp && sg[u] != 0 && !dirty;
                if (__ballot_sync(kFull, dirty) || build_list) {
                    Rec &r = b.r[lane];
                    bool changed = false;
                    int kyn = 0;
                    u64 lco = 0;
                    u64 nsg = sg[u];  // the record's signature after this round
                    if (dirty) {
                        load_rec(&r, f.F[l] + slot[u]);
                        if (leafp && !force) lco = __ldcg(f.lc[l] + slot[u]);
                        const int kyo = force ? 0 : (int)r.ky;  // nothing counted before round 0
                        changed = refresh_record(c, Ush, Csh, l, r, force);
                        kyn = r.ky;
                        if (force && leafp && l <= kPadGenes) {  // the key genes, once
                            u16 *po = pad_po(r);
                            for (int q = 0; q < l; ++q) {
                                const u16 v = c.orig[prefix_gene(r.p, q)];
                                int k = q - 1;
                                while (k >= 0 && po[k] > v) {
                                    po[k + 1] = po[k];
                                    --k;
                                }
                                po[k + 1] = v;
                            }
                        }
                        if (changed) {
                            nsg = kyn >= 2 ? sample_sig(r) : 0ull;
                            f.sig[l][slot[u]] = nsg;
                            copy_rec(f.F[l] + slot[u], &r);
                            if (l >= 2) {
                                const u64 fo = kyo >= 2 ? (u64)(kyo - 1) : 0ull, fn = kyn >= 2 ? (u64)(kyn - 1) : 0ull;
                                dA += fn - fo;
                                dV += (fn - fo) * (u64)(hiN - prefix_gene(r.p, l - 1));
                            }
                        } else {
                            cached = leafp;  // nothing covered in it after all
                        }
                    }
                    const bool eval = leafp && changed && kyn >= 2;
                    if (leafp && changed && kyn < 2) {  // no longer shared: no leaf with TP >= 2
                        f.lb[l][slot[u]] = key_empty();
                        f.lc[l][slot[u]] = 0;
                        dL -= lco;
                    }
                    // the warp's list: the records still live after this round, with their
                    // cached best scores (a changed leaf parent's is set when it is evaluated)
                    int lpos = -1;
                    if (build_list) {
                        const bool keep = nsg != 0;
                        const unsigned km = __ballot_sync(kFull, keep);
                        if (lfill + __popc(km) > kList) {
                            lfit = false;
                        } else if (lfit) {
                            if (keep) {
                                lpos = lfill + __popc(km & ((1u << lane) - 1u));
                                lv.slot[warp][lpos] = slot[u];
                                lv.sig[warp][lpos] = nsg;
                                lv.ls[warp][lpos] = leafp && !changed ? ls[u] : 0ull;
                            }
                            lfill += __popc(km);
                        }
                    }
                    // changed leaf parents go to the block's queue (spread over its warps
                    // below); what does not fit is evaluated by this warp
                    bool queued = false;
                    if (eval && !force && !is_dense(r.ky, r.kn)) {
                        const int pos = atomicAdd(&qn, 1);
                        if (pos < qcap) {
                            copy_rec(&qrec[pos], &r);
                            queue_tasks(pos, r, l);
                            qslot[pos] = slot[u];
                            qlco[pos] = lco;
                            qidx[pos] = (short)lpos;
                            qwarp[pos] = (signed char)warp;
                            queued = true;
                        }
                    }
                    const bool here = eval && !queued;
                    if (__ballot_sync(kFull, here)) {
                        leaf_parents_eval(c, s, b, here, l, lane);
                        if (here) {
                            const Key kb = b.rb[lane];
                            f.lb[l][slot[u]] = kb;
                            f.lc[l][slot[u]] = b.rc[lane];
                            if (lpos >= 0) lv.ls[warp][lpos] = kb.s;
                            dL += b.rc[lane] - lco;
                            if (kb.s != 0 && key_better(kb, best)) best = kb;
                        }
                        __syncwarp();
                    }
                }
                if (cached && ls[u] != 0 && ls[u] >= best.s) {  // unchanged: its cached best
                    Key kc;
                    kc.s = ls[u];
                    kc.t0 = __ldcg(&f.lb[l][slot[u]].t0);
                    kc.t1 = __ldcg(&f.lb[l][slot[u]].t1);
                    kc.t2 = __ldcg(&f.lb[l][slot[u]].t2);
                    if (key_better(kc, best)) best = kc;
                }
            }
        }
        if (leafp) {
            // the queued leaf parents: their (record, column word) items spread over all
            // warps of the block, in tasks of up to 32 items of one record; a record's
            // best leaf (packed) and its sum of TP - 1 meet in shared memory
            __syncthreads();
            const int nq = qn < qcap ? qn : qcap;
            if (nq > 0) {
                // every warp forms the records' task prefix itself (nq <= 64: two chunks)
                const int i0 = lane < nq ? qtasks[lane] : 0, i1 = lane + 32 < nq ? qtasks[lane + 32] : 0;
                const int inc0 = warp_incl_scan(i0, lane);
                const int inc1 = __shfl_sync(kFull, inc0, 31) + warp_incl_scan(i1, lane);
                const int T = __shfl_sync(kFull, inc1, 31), nwg = ((c.G - 1) >> 6) + 1;
                for (int tau = warp; tau < T; tau += nwarps) {
                    // its record: the number of records whose tasks end at or before tau
                    const int j = __popc(__ballot_sync(kFull, lane < nq && inc0 <= tau)) +
                                  __popc(__ballot_sync(kFull, lane + 32 < nq && inc1 <= tau));
                    const int e0 = __shfl_sync(kFull, inc0, (j - 1) & 31), e1 = __shfl_sync(kFull, inc1, (j - 33) & 31);
                    const int first = j == 0 ? 0 : (j <= 32 ? e0 : e1);
                    const int lo = qlo[j];
                    const int it = (tau - first) * 32 + lane, wi = (lo >> 6) + it;
                    u64 pk = 0, corr = 0;
                    if (wi < nwg) leaf_item_eval(c, s, qrec[j], wi, range_word(wi, lo, c.G - 1), corr, pk);
                    pk = warp_max_u64(pk);
                    const u32 cs = __reduce_add_sync(kFull, (u32)corr);
                    if (lane == 0) {
                        if (pk) atomicMax(&qbest[j], pk);
                        if (cs) atomicAdd(&qcorr[j], cs);
                    }
                }
                __syncthreads();
                const int j = (int)threadIdx.x;
                if (j < nq) {
                    Key kb = key_empty();
                    if (qbest[j]) {
                        int po[kMaxH - 1];
                        record_po(c, qrec[j], l, po);
                        kb = unpack_leaf(qbest[j], po, l);
                    }
                    f.lb[l][qslot[j]] = kb;
                    f.lc[l][qslot[j]] = qcorr[j];
                    if (kLWarps > 0 && qidx[j] >= 0) lv.ls[qwarp[j]][qidx[j]] = kb.s;
                    dL += qcorr[j] - qlco[j];
                    if (kb.s != 0 && key_better(kb, best)) best = kb;
                }
            }
        }
        if (build_list && lane == 0) ft.lcnt[warp][l] = (short)(lfill - ft.lbase[warp][l]);
        dA = warp_sum_u64(dA);
        dV = warp_sum_u64(dV);
        dL = warp_sum_u64(dL);
        if (lane == 0) {
            deep_add(2 * l + 1, dA);
            deep_add(2 * (l + 1), dV);
            deep_add(2 * h + 1, dL);
        }
    }
    if (build_list && lane == 0) ft.lok[warp] = lfit ? 1 : 0;
    // one block barrier, then three jobs on three warps: the block's best to its slot
    // (first, the round's grid barrier waits for it), the depths' correction changes
    // to the round's counters, the phase's warp cycles to the diagnostics
    Key *wkey = warp_keys();
    warp_cycles(acc, t0, lane);
    {
        const Key wb = warp_max_key(best);
        if (lane == 0) wkey[warp] = wb;
    }
    __syncthreads();
    if (warp == 0) {
        const Key k = warp_max_key(lane < nwarps ? wkey[lane] : key_empty());
        if (lane == 0 && io.overwrite) {
            io.slots[t.rank] = k;
        } else if (lane == 0 && k.s != 0) {
            const Key old = io.slots[t.rank];
            if (key_better(k, old)) io.slots[t.rank] = k;
        }
    }
    if (warp == (nwarps > 1 ? 1 : 0)) {  // deep[i], i = 2e and 2e + 1 for depths e = 1 .. h
        const int i = lane + 2;
        if (i <= 2 * h + 1) {
            u64 d = deep[i];
            if (kLWarps > 0) {
#pragma unroll 4
                for (int w = 0; w < nwarps; ++w) d += wdeep[w][i];
            }
            if (d) atomicAdd(s.cnt + ((size_t)round * h + (i / 2 - 1)) * 2 + (i & 1), d);
        }
    }
    if (warp == (nwarps > 2 ? 2 : nwarps - 1)) {
        const u64 v = lane < nwarps ? warp_cycle_slots()[lane] : 0ull;
        const u64 sum = warp_sum_u64(v), mx = warp_max_u64(v);
        if (lane == 0) {
            atomicAdd(s.work + kWorkWarpSum + 1, sum);
            atomicMax(s.work + (io.par ? kWorkWarpMaxOdd : kWorkWarpMax) + 1, mx);
            atomicAdd(s.work + kWorkWarpN + 1, (u64)nwarps);
        }
    }
    return true;
}

// End of round r of the persistent solve, run by EVERY block of the team on the
// same inputs, so that all of them reach the same decisions without another
// barrier: the winner (largest key of the round's slots), its TP / FP, the next U
// (DelCols on the block's copy Ush, then written to s.U: every block writes the
// same words).  Rank 0 also picks the next round's candidates (cand_sh, and s.cand
// for a later launch), rescores them into the next threshold (next_hint), and
// records the selection and the round state.  Returns true when the solve is done.
__device__ bool end_of_round(const Cohort &c, const Solve &s, int round, const Key *slots, int nslots, const Team &t,
                             u64 *Ush, Key *cand_sh, u64 *next_hint)
{
    __shared__ Key wbest[kMaxWarpsPerBlock];
    __shared__ int gs[kMaxH], os[kMaxH];
    __shared__ int done_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int h = s.h;
    const bool lead = t.rank == 0;
    Key best = key_empty();
    for (int i = threadIdx.x; i < nslots; i += blockDim.x) {
        Key k;
        k.s = __ldcg(&slots[i].s);
        k.t0 = __ldcg(&slots[i].t0);
        k.t1 = __ldcg(&slots[i].t1);
        k.t2 = __ldcg(&slots[i].t2);
        if (key_better(k, best)) best = k;
    }
    // the best kCandidates of the warps' lane bests become next round's candidates
    // (rank 0 keeps them and rescores them into the next threshold; the other blocks
    // need only each warp's best)
    Key mine = best;
    const int per_warp = (kCandidates + nwarps - 1) / nwarps;
    for (int r = 0; r < (lead ? per_warp : 1); ++r) {
        const Key m = warp_max_key(mine);
        const int idx = warp * per_warp + r;
        if (lane == 0 && idx < kCandidates) {
            cand_sh[idx] = m;
            if (lead) s.cand[idx] = m;
        }
        if (m.s != 0 && mine.s == m.s && mine.t0 == m.t0 && mine.t1 == m.t1 && mine.t2 == m.t2) mine = key_empty();
        if (r == 0 && lane == 0) wbest[warp] = m;
    }
    __syncthreads();
    if (warp == 0) {
        best = lane < nwarps ? wbest[lane] : key_empty();
        best = warp_max_key(best);
        const bool last_round = round + 1 >= *(volatile int *)&s.state[kStMaxRounds];
        if (lead && lane < 2) {  // diagnostics: the round's longest warps
            const int mx = ((round & 1) ? kWorkWarpMaxOdd : kWorkWarpMax) + lane;
            s.work[kWorkWarpMaxSum + lane] += __ldcg(&s.work[mx]);
            s.work[mx] = 0;
        }
        bool done = true;
        if (best.s != 0) {
            if (lane < h) {
                const int o = key_get(best, lane);
                os[lane] = o;
                if (!c.TO) gs[lane] = (int)c.inv[o];
            }
            __syncwarp();
            u64 y = 0, n = 0, u = 0;
            // the winner's rows: by original index, or by search position
            const u64 *TR = c.TO ? c.TO : c.T;
            const u64 *NR = c.TO ? c.NO : c.N;
            const int *ri = c.TO ? os : gs;
            if (lane < c.Wt) {
                u = Ush[lane];
                y = u;
#pragma unroll
                for (int i = 0; i < kMaxH; ++i)
                    if (i < h) y &= __ldg(TR + (size_t)ri[i] * c.WTp + lane);
            }
            if (lane < c.Wn) {
                n = ~0ull;
#pragma unroll
                for (int i = 0; i < kMaxH; ++i)
                    if (i < h) n &= __ldg(NR + (size_t)ri[i] * c.WNp + lane);
            }
            int tp = __popcll(y), fp = __popcll(n);
            for (int off = 16; off; off >>= 1) {
                tp += __shfl_xor_sync(kFull, tp, off);
                fp += __shfl_xor_sync(kFull, fp, off);
            }
            __syncwarp();
            if (lane < c.Wt) {
                u &= ~y;
                Ush[lane] = u;
                s.U[lane] = u;
            }
            const unsigned left = __ballot_sync(kFull, u != 0);
            done = !left || last_round;
            if (lead && lane == 0) {
                const int k = *(volatile int *)&s.state[kStK];
                int *r = s.res + (size_t)k * (h + 2);
                for (int i = 0; i < h; ++i) r[i] = os[i];
                r[h] = tp;
                r[h + 1] = fp;
                s.state[kStK] = k + 1;
            }
        }
        if (lane == 0) {
            done_sh = done;
            if (lead) {
                s.state[kStRound] = round + 1;
                if (done) s.state[kStDone] = 1;
            }
        }
    }
    __syncthreads();
    const bool done = done_sh != 0;
    // one block suffices: the threshold is a lower bound whichever blocks have merged
    // into it, and it is first read after the next round's first barrier (h >= 3)
    if (!done && h > 1 && lead) block_rescore(c, s, cand_sh, Ush, next_hint);
    return done;
}

// End of an incremental round, by every block on the same inputs: warp 0 alone
// reduces the blocks' slots to the winner, computes its TP / FP and the tumors it
// covers, applies DelCols to the block's copy of U and keeps the covered tumors
// (Csh) for the next round's update.  The lead block (rank 0) also records the
// selection and finishes the round's counters: depth 1 from its surviving count,
// depths 2..h as the per-sample sums over all tumors (tot) minus the running
// totals (run, to which it adds the round's changes, read together with the
// slots): the corrections, and the per-sample sums of the tumors covered so far,
// which each round's update adds for the tumors the last winner covered.  kk: the lead's
// count of selections; maxr: the round limit.  Returns true when the solve is done.
__device__ bool end_of_round_inc(const Cohort &c, const Solve &s, int round, const Key *slots, int nslots,
                                 const Team &t, u64 *Ush, const u64 *tot, u64 *Csh, u64 *run, int *kk, int maxr)
{
    __shared__ int os[kMaxH];
    __shared__ int done_sh;
    Key *wbest = warp_keys();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int h = s.h;
    const bool lead = t.rank == 0;
    {  // the slots, one per thread (all loads of a thread in flight together)
        Key best = key_empty();
        for (int i = (int)threadIdx.x; i < nslots; i += (int)blockDim.x) {
            Key k;
            k.s = __ldcg(&slots[i].s);
            k.t0 = __ldcg(&slots[i].t0);
            k.t1 = __ldcg(&slots[i].t1);
            k.t2 = __ldcg(&slots[i].t2);
            if (key_better(k, best)) best = k;
        }
        best = warp_max_key(best);
        if (lane == 0) wbest[warp] = best;
    }
    __syncthreads();
    if (warp == 0) {
        u64 dv = 0, da = 0;
        u64 *cv = s.cnt + ((size_t)round * h + lane) * 2;
        if (lead && lane < h) {
            dv = __ldcg(cv);
            da = __ldcg(cv + 1);
        }
        const Key best = warp_max_key(lane < nwarps ? wbest[lane] : key_empty());
        bool done = true;
        u64 ycov = 0;
        if (best.s != 0) {
            if (lane < h) os[lane] = key_get(best, lane);
            __syncwarp();
            const u64 *TR = c.TO ? c.TO : c.T;
            const u64 *NR = c.TO ? c.NO : c.N;
            int ri[kMaxH];
#pragma unroll
            for (int i = 0; i < kMaxH; ++i) ri[i] = i < h ? (c.TO ? os[i] : (int)c.inv[os[i]]) : 0;
            u64 y = 0, n = 0, u = 0;
            if (lane < c.Wt) {
                u = Ush[lane];
                y = u;
#pragma unroll
                for (int i = 0; i < kMaxH; ++i)
                    if (i < h) y &= __ldg(TR + (size_t)ri[i] * c.WTp + lane);
            }
            if (lane < c.Wn) {
                n = ~0ull;
#pragma unroll
                for (int i = 0; i < kMaxH; ++i)
                    if (i < h) n &= __ldg(NR + (size_t)ri[i] * c.WNp + lane);
            }
            const int tp = (int)__reduce_add_sync(kFull, (unsigned)__popcll(y));
            const int fp = (int)__reduce_add_sync(kFull, (unsigned)__popcll(n));
            if (lane < c.Wt) {
                ycov = y;
                u &= ~y;
                Ush[lane] = u;
                s.U[lane] = u;
            }
            const unsigned left = __ballot_sync(kFull, u != 0);
            done = !left || round + 1 >= maxr;
            if (lead && lane == 0) {
                const int k = *kk;
                int *r = s.res + (size_t)k * (h + 2);
                for (int i = 0; i < h; ++i) r[i] = os[i];
                r[h] = tp;
                r[h + 1] = fp;
                s.state[kStK] = k + 1;
                *kk = k + 1;
            }
        }
        if (lead && lane < h) {
            const int l = lane + 1;
            run[2 * l] += dv;
            run[2 * l + 1] += da;
            u64 vis, alive;
            if (l == 1) {
                vis = c.G >= h ? (u64)(c.G - h + 1) : 0ull;
                alive = run[3];
            } else {
                vis = tot[h + lane] - run[2 * l];
                alive = tot[lane] - run[2 * l + 1];
            }
            cv[0] = vis;
            cv[1] = vis - alive;
            s.run[2 * l] = run[2 * l];
            s.run[2 * l + 1] = run[2 * l + 1];
        }
        Csh[lane] = ycov;  // kMaxWords == 32 words, one per lane
        if (lead && lane < c.WTp) s.cov[lane] = ycov;
        if (lane == 0) {
            done_sh = done;
            if (lead) {
                s.state[kStRound] = round + 1;
                if (done) s.state[kStDone] = 1;
            }
        }
    }
    __syncthreads();
    return done_sh != 0;
}

// The greedy loop of one cohort run by a team of co-resident blocks.  A round is
// the depth-2 .. h-1 expansions (depth 1 built on the fly from the gene rows), the
// leaves, a barrier, and the end of round computed redundantly by every block, so
// rounds are separated by h - 1 barriers.  Data indexed by round parity: the slots
// the blocks' bests go to, the frontier counters and the threshold word; rank 0
// clears the next round's set at the start of a round (all reads of it ended
// before the previous round's last barrier).  Returns when the solve is done, a
// frontier overflowed, a barrier timed out (recorded in the cohort's state) or,
// in a batch, the barrier that ended a round carried a yield request.
template <int kQueue, int kLWarps>
__device__ void solve_team(const Cohort &c, const Solve &s, const Frontiers &f, GridSync *gsync, u32 *counts_base,
                           const Team &t, Batch &b, int *yield = nullptr)
{
    __shared__ u64 Ush[kMaxWords];
    __shared__ Key cand_sh[kCandidates];
    __shared__ u64 tot[2 * kMaxH];
    __shared__ u64 Csh[kMaxWords];
    __shared__ u64 run[2 * (kMaxH + 1)];  // incremental rounds, rank 0: the corrections' running totals
    __shared__ FrontTab ftab;
    __shared__ int fm_sh, kk_sh;
    const int h = s.h;
    const bool timer = t.rank == 0 && threadIdx.x == 0;
    u64 tm = timer ? global_ns() : 0;
    auto lap = [&](int phase) {
        if (timer) {
            const u64 now = global_ns();
            atomicAdd(s.work + kWorkPhaseNs + phase, now - tm);
            tm = now;
        }
    };
    if (*(volatile int *)&s.state[kStDone] | *(volatile int *)&s.state[kStError]) return;
    int round = *(volatile int *)&s.state[kStRound];
    const int maxr = *(volatile int *)&s.state[kStMaxRounds];
    for (int w = (int)threadIdx.x; w < kMaxWarpsPerBlock; w += (int)blockDim.x) ftab.lok[w] = 0;
    if (threadIdx.x == 0) {
        ftab.ok = 0;
        kk_sh = *(volatile int *)&s.state[kStK];
    }
    // start of a launch: U and the candidates left by the previous round
    for (int i = threadIdx.x; i < kMaxWords; i += blockDim.x) Ush[i] = i < c.WTp ? __ldcg(&s.U[i]) : 0ull;
    for (int i = threadIdx.x; i < kCandidates; i += blockDim.x) {
        cand_sh[i].s = __ldcg(&s.cand[i].s);
        cand_sh[i].t0 = __ldcg(&s.cand[i].t0);
        cand_sh[i].t1 = __ldcg(&s.cand[i].t1);
        cand_sh[i].t2 = __ldcg(&s.cand[i].t2);
    }
    __syncthreads();
    if (h > 1 && t.rank == 0) block_rescore(c, s, cand_sh, Ush, s.best_hint + (round & 1));
    if (h > 1 && round == 0 && s.prune != MH_PRUNE_OFF && c.CC) {
        // the champions and the first round's threshold, complete before any block
        // starts searching
        if (s.champ && s.prune == MH_PRUNE_PAPER) phase_champions(c, s, t, b);
        if (s.ssum && s.prune == MH_PRUNE_PAPER) phase_sample_sums(c, s, t);
        block_seed(c, s, t, Ush, s.best_hint);
        if (!grid_sync(gsync, s.state, t.size)) return;
    }
    // counting by per-sample sums when every tumor's champion is known (the
    // champions stand for the TP = 1 leaves that this mode never visits)
    bool fm = false;
    if (h > 1 && s.prune == MH_PRUNE_PAPER && c.CC && s.champ && s.ssum) {
        if (threadIdx.x == 0) fm_sh = 1;
        __syncthreads();
        for (int i = threadIdx.x; i < c.Nt; i += blockDim.x)
            if (!__ldcg(s.champ_ok + i)) fm_sh = 0;
        __syncthreads();
        fm = fm_sh != 0;
        if (fm && t.rank == 0) block_sample_totals(c, s, tot);
        // incremental rounds: the tumors covered by the last round's winner
        for (int i = threadIdx.x; i < kMaxWords; i += blockDim.x)
            Csh[i] = (fm && round > 0 && i < c.WTp) ? __ldcg(&s.cov[i]) : 0ull;
        for (int i = threadIdx.x; i < 2 * (kMaxH + 1); i += blockDim.x)
            run[i] = (fm && round > 0) ? __ldcg(s.run + i) : 0ull;
        __syncthreads();
    }
    for (;;) {
        const int par = round & 1;
        // incremental rounds keep round 0's frontiers and their counts (set 0)
        u32 *counts = counts_base + (size_t)(fm ? 0 : par) * kCountWords;
        const RoundIO io{Ush, s.slots + (size_t)par * s.nslots, true, s.best_hint + par, par, fm, fm};
        if (t.rank == 0 && !fm) {  // the next round's counters and threshold start from zero
            u32 *cn = counts_base + (size_t)(par ^ 1) * kCountWords;
            for (int i = threadIdx.x; i < kMaxH * kShards; i += blockDim.x) cn[i * kShardStride] = 0;
            if (threadIdx.x == 0) *(volatile u64 *)(s.best_hint + (par ^ 1)) = 0;
        }
        // on an overflow the team stops; in a batch it also asks the other teams to
        // stop at their next round boundary, so that the host can grow the frontier
        // and relaunch without leaving the team's blocks idle
        auto overflow = [&]() {
            if (t.rank == 0 && threadIdx.x == 0) {
                s.state[kStOverflow] = 1;
                if (yield) {
                    *(volatile int *)yield = 1;
                    __threadfence_system();
                }
            }
        };
        if (h == 1) {
            phase_level1(c, s, round, f, counts, t, io);
            lap(0);
        } else if (fm) {
            // round 0 builds the kept frontiers; every round then updates them
            if (round == 0) {
                if (h == 2) {
                    phase_build1(c, s, f, counts, b, t, Ush);
                    if (!grid_sync(gsync, s.state, t.size)) return;
                }
                for (int l = 2; l <= h - 1; ++l) {
                    if (!phase_expand(c, s, round, l, f, counts, b, t, io)) {
                        overflow();
                        return;
                    }
                    if (!grid_sync(gsync, s.state, t.size)) return;
                }
            }
            lap(1);
            if (!phase_update<kQueue, kLWarps>(c, s, round, f, counts, b, t, io, Csh, round == 0, ftab)) {
                overflow();
                return;
            }
        } else {
            // every block reads the same shard counts after the same barrier, so an
            // overflow is seen by all of them and they leave together
            for (int l = 2; l <= h - 1; ++l) {
                if (!phase_expand(c, s, round, l, f, counts, b, t, io)) {
                    overflow();
                    return;
                }
                if (!grid_sync(gsync, s.state, t.size)) return;
            }
            lap(1);
            if (!phase_leaf(c, s, round, f, counts, b, t, io)) {
                overflow();
                return;
            }
        }
        // the round's last barrier; in a batch its releasing block samples the yield
        // request, so that every block of the team takes the same decision
        if (!grid_sync(gsync, s.state, t.size, yield)) return;
        const bool stop = yield && *(volatile int *)&gsync->flag;
        lap(2);
        const bool done = fm ? end_of_round_inc(c, s, round, io.slots, t.size, t, Ush, tot, Csh, run, &kk_sh, maxr)
                             : end_of_round(c, s, round, io.slots, t.size, t, Ush, cand_sh, s.best_hint + (par ^ 1));
        lap(3);
        if (done) {
            // batch: a team that finished asks the others to stop after their current
            // round, so that the host can hand its blocks to the unfinished cohorts
            if (yield && t.rank == 0 && threadIdx.x == 0) {
                *(volatile int *)yield = 1;  // may be host memory: a plain store, made visible
                __threadfence_system();
            }
            return;
        }
        ++round;
        if (stop) {
            if (t.rank == 0 && threadIdx.x == 0) s.state[kStYield] = 1;
            return;
        }
    }
}

// Diagnostic: one block enters a team barrier sized for two blocks, so the wait
// can only end by its bound; the timeout is recorded in state[kStError].
__global__ void k_barrier_probe(GridSync *g, int *state) { grid_sync(g, state, 2); }

// Two builds of the persistent solve: one block per SM (a cheap grid barrier: the
// small, latency-bound cohorts) and four blocks per SM (more warps to hide memory
// latency: the large ones).
template <int kMinBlocks, int kWarps>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks)
    k_solve(const __grid_constant__ Cohort c, const __grid_constant__ Solve s, const __grid_constant__ Frontiers f,
            GridSync *gsync, u32 *counts, int *yield)
{
    __shared__ Batch scratch[kWarps];
    solve_team<kMinBlocks == 1 ? kEvalQueue : 0, kMinBlocks == 1 ? kWarps : 0>(c, s, f, gsync, counts, grid_team(),
                                                                                scratch[threadIdx.x >> 5], yield);
}

// SM-major number of the calling block (thread 0): SMs are ranked in the order
// their first block arrives, blocks within an SM in arrival order.  Returns -1 if
// the numbering cannot be formed (an SM id out of range, more blocks on an SM than
// expected, or a wait for the SM's rank that did not end).
__device__ int sm_major_block(const BatchMap &m)
{
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    if (smid >= (unsigned)kMaxSmid) return -1;
    const int slot = atomicAdd(&m.tab[smid], 1);
    int r;
    if (slot == 0) {
        r = atomicAdd(&m.tab[2 * kMaxSmid], 1);
        atomicExch(&m.tab[kMaxSmid + smid], r);
    } else {
        unsigned spins = 0;
        while ((r = *(volatile int *)&m.tab[kMaxSmid + smid]) < 0) {
            __nanosleep(32);
            if (++spins > (1u << 22)) return -1;
        }
    }
    if (slot >= m.per_sm || r >= m.num_sms) return -1;
    return r * m.per_sm + slot;
}

// Batched solve: block b (SM-major number, or blockIdx.x if that numbering failed
// anywhere in the grid) works on the cohort whose block range holds b, with the
// blocks of that range as its team; cohorts progress independently.
template <int kMinBlocks, int kWarps>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks)
    k_solve_batch(const BatchItem *items, int n, int *yield, BatchMap map)
{
    __shared__ Batch scratch[kWarps];
    __shared__ int vb_s;
    if (threadIdx.x == 0) {
        vb_s = sm_major_block(map);
        if (vb_s < 0) atomicExch(&map.tab[2 * kMaxSmid + 1], 1);
    }
    if (!grid_sync(map.sync, items[0].s.state, (int)gridDim.x)) return;
    const bool sm_major = *(volatile int *)&map.tab[2 * kMaxSmid + 1] == 0;
    const int vb = sm_major ? vb_s : (int)blockIdx.x;
    int lo = 0, hi = n - 1;  // last item with first_block <= vb
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first_block <= vb) lo = mid; else hi = mid - 1;
    }
    // the block's item in shared memory: the phases read its fields in their inner
    // loops, and shared memory cannot alias the global stores in between (a global
    // copy would be re-read after every store)
    __shared__ BatchItem it;
    static_assert(sizeof(BatchItem) % 4 == 0, "BatchItem is copied as 32-bit words");
    for (int i = threadIdx.x; i < (int)(sizeof(BatchItem) / 4); i += blockDim.x)
        ((int *)&it)[i] = ((const int *)&items[lo])[i];
    __syncthreads();
    Team t{vb - it.first_block, it.nblocks};
    if (t.rank < 0 || t.rank >= t.size) return;
    // a team of whole SMs ranks its blocks SM-minor (rank r on SM r mod #SMs), so
    // that neighbouring work items, handed to neighbouring ranks, go to different SMs
    if (sm_major && it.first_block % map.per_sm == 0 && it.nblocks % map.per_sm == 0) {
        const int nsm = it.nblocks / map.per_sm;
        t.rank = (t.rank % map.per_sm) * nsm + t.rank / map.per_sm;
    }
    solve_team<kMinBlocks == 1 ? kEvalQueue : 0, kMinBlocks == 1 ? kWarps : 0>(it.c, it.s, it.f, it.gsync, it.counts, t,
                                                                                scratch[threadIdx.x >> 5], yield);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers

void launch_transpose(const Cohort &c, const u64 *rows, int row_stride, int samples, u64 *cols, cudaStream_t st)
{
    const long long total = (long long)samples * c.GW;
    if (total == 0) return;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    k_transpose<<<(unsigned)blocks, threads, 0, st>>>(c.G, rows, row_stride, samples, c.GW, cols);
}

void launch_solve_init(const Cohort &c, const Solve &s, int counter_rounds, int max_rounds, u32 *counts, int sets,
                       cudaStream_t st)
{
    cudaMemsetAsync(s.cnt, 0, sizeof(u64) * 2 * (size_t)s.h * (size_t)counter_rounds, st);
    if (s.cut) cudaMemsetAsync(s.cut, 0, sizeof(u64) * (size_t)s.h * (size_t)counter_rounds, st);
    cudaMemsetAsync(s.slots, 0, sizeof(Key) * (size_t)s.nslots * sets, st);
    cudaMemsetAsync(s.cand, 0, sizeof(Key) * (size_t)kCandidates, st);
    cudaMemsetAsync(s.work, 0, sizeof(u64) * kWorkCount, st);
    cudaMemsetAsync(s.best_hint, 0, sizeof(u64) * sets, st);
    cudaMemsetAsync(counts, 0, sizeof(u32) * kCountWords * sets, st);
    k_solve_init<<<1, 64, 0, st>>>(c, s, max_rounds);
}

int level1_grid(const Cohort &c) { return (c.G + kThreads - 1) / kThreads; }

void launch_level1(const Cohort &c, const Solve &s, const Frontiers &f, u32 *counts, cudaStream_t st)
{
    k_level1<<<level1_grid(c), kThreads, 0, st>>>(c, s, f, counts);
}

void launch_expand(const Cohort &c, const Solve &s, int level, const Frontiers &f, u32 *counts, int grid,
                   cudaStream_t st)
{
    k_expand<<<grid, kThreads, 0, st>>>(c, s, level, f, counts);
}

void launch_leaf(const Cohort &c, const Solve &s, const Frontiers &f, u32 *counts, int grid, cudaStream_t st)
{
    k_leaf<<<grid, kThreads, 0, st>>>(c, s, f, counts);
}

void launch_finalize(const Cohort &c, const Solve &s, u32 *counts, cudaStream_t st)
{
    k_finalize<<<1, kThreads, 0, st>>>(c, s, counts);
}

// Coverage of a set of combinations (§IV-D): bit s of tcov (ncov) is set when tumor
// (normal) sample s carries every gene of at least one of the k combinations
// (original indices, k x h).  One thread per (combination, word); the words are
// OR-ed into the masks.
__global__ void k_coverage(const __grid_constant__ Cohort c, const int *genes, int k, int h, u64 *tcov, u64 *ncov)
{
    const int W = c.Wt + c.Wn;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)k * W) return;
    const int j = (int)(t / W), w = (int)(t % W);
    const bool tumor = w < c.Wt;
    const int ww = tumor ? w : w - c.Wt;
    u64 y = ~0ull;
    for (int i = 0; i < h; ++i) {
        const int g = genes[(size_t)j * h + i];
        const u64 *row = tumor ? (c.TO ? c.TO + (size_t)g * c.WTp : c.T + (size_t)c.inv[g] * c.WTp)
                               : (c.NO ? c.NO + (size_t)g * c.WNp : c.N + (size_t)c.inv[g] * c.WNp);
        y &= __ldg(row + ww);
    }
    if (y) atomicOr(tumor ? tcov + ww : ncov + ww, y);
}

void launch_coverage(const Cohort &c, const int *genes, int k, int h, u64 *tcov, u64 *ncov, cudaStream_t st)
{
    const long long total = (long long)k * (c.Wt + c.Wn);
    if (total == 0) return;
    k_coverage<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(c, genes, k, h, tcov, ncov);
}

void launch_finalize_split(const Cohort &c, const Solve &s, u32 *counts, int step, cudaStream_t st)
{
    k_finalize_split<<<1, kThreads, 0, st>>>(c, s, counts, step);
}

int persistent_grid(int num_sms, bool large)
{
    int per_sm = 0;
    const cudaError_t e = large
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<4, kWarpsPerBlock>, kThreads, 0)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve<1, kSmallWarps>, kSmallWarps * 32, 0);
    if (e != cudaSuccess || per_sm < 1) return 0;
    return (large ? per_sm : 1) * num_sms;
}

cudaError_t launch_barrier_probe(GridSync *g, int *state, cudaStream_t st)
{
    k_barrier_probe<<<1, 32, 0, st>>>(g, state);
    return cudaGetLastError();
}

int batch_blocks_per_sm(int build)
{
    int per_sm = 0;
    const cudaError_t e =
        build == 1 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_batch<1, kSmallWarps>,
                                                                   kSmallWarps * 32, 0)
        : build == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_batch<3, kWarpsPerBlock>,
                                                                     kThreads, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_batch<4, kWarpsPerBlock>,
                                                                     kThreads, 0);
    if (e != cudaSuccess) return 0;
    return build == 1 ? (per_sm >= 1 ? 1 : 0) : per_sm;
}

int batch_grid(int num_sms, int build) { return batch_blocks_per_sm(build) * num_sms; }

cudaError_t launch_solve_batch(const BatchItem *d_items, int n, int *d_yield, const BatchMap &m, cudaStream_t st)
{
    const BatchItem *items = d_items;
    int nn = n;
    int *yield = d_yield;
    BatchMap map = m;
    cudaError_t e = cudaMemsetAsync(map.tab, 0, sizeof(int) * kMaxSmid, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(map.tab + kMaxSmid, 0xff, sizeof(int) * kMaxSmid, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(map.tab + 2 * kMaxSmid, 0, sizeof(int) * 2, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(map.sync, 0, sizeof(GridSync), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&items, &nn, &yield, &map};
    const int grid = map.per_sm * map.num_sms;
    const void *fn = map.build == 1   ? (const void *)k_solve_batch<1, kSmallWarps>
                     : map.build == 3 ? (const void *)k_solve_batch<3, kWarpsPerBlock>
                                      : (const void *)k_solve_batch<4, kWarpsPerBlock>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(map.build == 1 ? kSmallWarps * 32 : kThreads), args, 0,
                                       st);
}

cudaError_t launch_solve_persistent(const Cohort &c, const Solve &s, const Frontiers &f, GridSync *gsync,
                                    u32 *counts, int grid, bool large, cudaStream_t st, int *yield)
{
    Cohort cc = c;
    Solve ss = s;
    Frontiers ff = f;
    void *args[] = {&cc, &ss, &ff, &gsync, &counts, &yield};
    const void *fn = large ? (const void *)k_solve<4, kWarpsPerBlock> : (const void *)k_solve<1, kSmallWarps>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(large ? kThreads : kSmallWarps * 32), args, 0, st);
}

}  // namespace mh
