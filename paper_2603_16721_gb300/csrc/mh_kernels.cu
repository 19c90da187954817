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
// Surviving leaves are scored from row popcounts over the non-zero words of the
// prefix only (the other words of the AND are zero).
#include "mh_internal.h"

namespace mh {

namespace {

constexpr unsigned kFull = 0xffffffffu;

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

__device__ __forceinline__ Key warp_max_key(Key k)
{
    for (int off = 16; off; off >>= 1) {
        Key o;
        o.s = __shfl_xor_sync(kFull, k.s, off);
        o.t0 = __shfl_xor_sync(kFull, k.t0, off);
        o.t1 = __shfl_xor_sync(kFull, k.t1, off);
        o.t2 = __shfl_xor_sync(kFull, k.t2, off);
        if (key_better(o, k)) k = o;
    }
    return k;
}

__device__ __forceinline__ u64 warp_sum_u64(u64 v)
{
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
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

// Block-wide best key -> slots[blockIdx.x] (merged with what an earlier launch
// of the same round left there).  All threads of the block must call it.
__device__ void block_commit_best(Key best, Key *slots)
{
    __shared__ Key wbest[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    best = warp_max_key(best);
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (warp == 0) {
        Key k = lane < kWarpsPerBlock ? wbest[lane] : key_empty();
        k = warp_max_key(k);
        if (lane == 0 && k.s != 0) {
            const Key old = slots[blockIdx.x];
            if (key_better(k, old)) slots[blockIdx.x] = k;
        }
    }
}

__device__ __forceinline__ void count_level(const Solve &s, int round, int level, u64 visited, u64 pruned)
{
    u64 *c = s.cnt + ((size_t)round * s.h + (level - 1)) * 2;
    if (visited) atomicAdd(c, visited);
    if (pruned) atomicAdd(c + 1, pruned);
}

// Per-warp scratch of the prefix being expanded.
struct WarpScratch {
    u64 ys[kMaxWords];      // y_{l-1} words
    u64 ns[kMaxWords];      // n_{l-1} words
    u16 samp[kMaxSamples];  // samples set in y_{l-1}
    int po[kMaxH];          // original indices of the prefix genes, ascending
};

// Loads the prefix, forms y_{l-1} / n_{l-1} (lane w holds word w), lists the
// samples of y_{l-1} in ws.samp and returns their number.
__device__ __forceinline__ int warp_prefix_setup(const Cohort &c, const Solve &s, const Prefix &p, int L,
                                                 WarpScratch &ws, unsigned &by, unsigned &bn, int lane,
                                                 bool want_orig)
{
    u64 y = 0, n = 0;
    if (lane < c.Wt) {
        y = s.U[lane];
        for (int i = 0; i < L; ++i) y &= c.T[(size_t)prefix_gene(p, i) * c.WTp + lane];
    }
    if (lane < c.Wn) {
        n = ~0ull;
        for (int i = 0; i < L; ++i) n &= c.N[(size_t)prefix_gene(p, i) * c.WNp + lane];
    }
    ws.ys[lane] = y;
    ws.ns[lane] = n;
    by = __ballot_sync(kFull, y != 0);
    bn = __ballot_sync(kFull, n != 0);
    const int cnt = __popcll(y);
    const int incl = warp_incl_scan(cnt, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    int off = incl - cnt;
    u64 yy = y;
    while (yy) {
        const int b = __ffsll((long long)yy) - 1;
        yy &= yy - 1;
        ws.samp[off++] = (u16)(lane * 64 + b);
    }
    if (want_orig && lane == 0) {
        // insertion sort of the prefix's original indices (L <= 8)
        for (int i = 0; i < L; ++i) {
            const int v = c.orig[prefix_gene(p, i)];
            int j = i - 1;
            while (j >= 0 && ws.po[j] > v) {
                ws.po[j + 1] = ws.po[j];
                --j;
            }
            ws.po[j + 1] = v;
        }
    }
    __syncwarp();
    return total;
}

// OR over the prefix's samples of the 64-gene column word wi, restricted to [lo, hi].
__device__ __forceinline__ u64 sibling_word(const Cohort &c, const WarpScratch &ws, int ky, int wi, int lo,
                                            int hi)
{
    const u64 *col = c.CT + wi;
    u64 m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int j = 0;
    for (; j + 4 <= ky; j += 4) {
        m0 |= col[(size_t)ws.samp[j] * c.GW];
        m1 |= col[(size_t)ws.samp[j + 1] * c.GW];
        m2 |= col[(size_t)ws.samp[j + 2] * c.GW];
        m3 |= col[(size_t)ws.samp[j + 3] * c.GW];
    }
    for (; j < ky; ++j) m0 |= col[(size_t)ws.samp[j] * c.GW];
    u64 m = (m0 | m1) | (m2 | m3);
    if (wi == (lo >> 6)) m &= ~0ull << (lo & 63);
    if (wi == (hi >> 6)) m &= ~0ull >> (63 - (hi & 63));
    return m;
}

__device__ __forceinline__ u64 range_word(int wi, int lo, int hi)
{
    u64 m = ~0ull;
    if (wi == (lo >> 6)) m &= ~0ull << (lo & 63);
    if (wi == (hi >> 6)) m &= ~0ull >> (63 - (hi & 63));
    return m;
}

// Appends the set bits of `a` (children of prefix p at position L) to Fout with
// one atomic per warp.  Entries beyond cap are dropped; the count still grows so
// the host can see the size it needs.
__device__ __forceinline__ void warp_append(u64 a, int wi, const Prefix &p, int L, Prefix *Fout, u32 *nout,
                                            u32 cap, int lane)
{
    const int cnt = __popcll(a);
    const int incl = warp_incl_scan(cnt, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    u32 base = 0;
    if (lane == 0) base = atomicAdd(nout, (u32)total);
    base = __shfl_sync(kFull, base, 0);
    u32 pos = base + (u32)(incl - cnt);
    while (a) {
        const int b = __ffsll((long long)a) - 1;
        a &= a - 1;
        if (pos < cap) Fout[pos] = prefix_with(p, L, wi * 64 + b);
        ++pos;
    }
}

// ---------------------------------------------------------------------------

__global__ void k_transpose(Cohort c, u64 *CT)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)c.Nt * c.GW;
    if (t >= total) return;
    const int s = (int)(t / c.GW), wi = (int)(t % c.GW);
    const int sw = s >> 6, sb = s & 63;
    u64 word = 0;
    for (int b = 0; b < 64; ++b) {
        const int g = wi * 64 + b;
        if (g < c.G) word |= ((c.T[(size_t)g * c.WTp + sw] >> sb) & 1ull) << b;
    }
    CT[t] = word;
}

__global__ void k_solve_init(Cohort c, Solve s)
{
    const int w = threadIdx.x;
    if (w < c.WTp) {
        const int rem = c.Nt - 64 * w;
        s.U[w] = rem >= 64 ? ~0ull : (rem <= 0 ? 0ull : ((1ull << rem) - 1ull));
    }
    if (w < 4) s.state[w] = 0;
}

// Depth 1: y_1(g) = U & x_g for g in [0, G-h] (0-based).  For h = 1 these are
// the leaves and are scored here; otherwise the non-empty ones (all of them with
// pruning off) become the depth-1 frontier.
__global__ void __launch_bounds__(kThreads) k_level1(Cohort c, Solve s, int round, Prefix *F1, u32 *n1, u32 cap1)
{
    if (s.state[1]) return;
    const int lane = threadIdx.x & 31;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int last = c.G - s.h;  // 0-based inclusive bound of depth 1
    const bool in = g <= last;
    bool nonempty = false;
    int tp = 0;
    if (in) {
        const u64 *row = c.T + (size_t)g * c.WTp;
        for (int w = 0; w < c.Wt; ++w) tp += __popcll(row[w] & s.U[w]);
        nonempty = tp > 0;
    }
    const unsigned bin = __ballot_sync(kFull, in), bne = __ballot_sync(kFull, nonempty);
    if (lane == 0) count_level(s, round, 1, (u64)__popc(bin), (u64)__popc(bin & ~bne));
    if (s.h == 1) {
        Key best = key_empty();
        if (nonempty) {
            int fp = 0;
            const u64 *nrow = c.N + (size_t)g * c.WNp;
            for (int w = 0; w < c.Wn; ++w) fp += __popcll(nrow[w]);
            best.s = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
            key_put(best, 0, c.orig[g]);
        }
        block_commit_best(best, s.slots);
        return;
    }
    const bool keep = s.prune ? in : nonempty;
    const unsigned bk = __ballot_sync(kFull, keep);
    if (!bk) return;
    u32 base = 0;
    if (lane == 0) base = atomicAdd(n1, (u32)__popc(bk));
    base = __shfl_sync(kFull, base, 0);
    if (keep) {
        const u32 pos = base + __popc(bk & ((1u << lane) - 1u));
        if (pos < cap1) {
            Prefix p;
            p.w0 = (u64)g;
            p.w1 = 0;
            F1[pos] = p;
        }
    }
}

// Depths 2 .. h-1: one warp per prefix of the depth-(level-1) frontier; the
// non-empty children (all children with pruning off) go to the depth-level frontier.
__global__ void __launch_bounds__(kThreads) k_expand(Cohort c, Solve s, int round, int level, const Prefix *Fin,
                                                     const u32 *nin, Prefix *Fout, u32 *nout, u32 cap)
{
    __shared__ WarpScratch scratch[kWarpsPerBlock];
    if (s.state[1]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpScratch &ws = scratch[warp];
    const u32 count = *nin;
    const int L = level - 1;
    const int hi = c.G - s.h + level - 1;  // 0-based inclusive bound of this depth
    u64 visited = 0, pruned = 0;
    const u32 gw = blockIdx.x * kWarpsPerBlock + warp, nw = gridDim.x * kWarpsPerBlock;
    for (u32 i = gw; i < count; i += nw) {
        const Prefix p = Fin[i];
        unsigned by, bn;
        const int ky = warp_prefix_setup(c, s, p, L, ws, by, bn, lane, false);
        const int lo = prefix_gene(p, L - 1) + 1;
        if (hi >= lo) {
            visited += (u64)(hi - lo + 1);
            u64 alive = 0;
            for (int wb = lo >> 6; wb <= (hi >> 6); wb += 32) {
                const int wi = wb + lane;
                u64 m = 0, a = 0;
                if (wi <= (hi >> 6)) {
                    m = ky ? sibling_word(c, ws, ky, wi, lo, hi) : 0;
                    a = s.prune ? range_word(wi, lo, hi) : m;
                }
                alive += (u64)__popcll(m);
                warp_append(a, wi, p, L, Fout, nout, cap, lane);
            }
            alive = warp_sum_u64(alive);
            pruned += (u64)(hi - lo + 1) - alive;
        }
        __syncwarp();
    }
    if (lane == 0) count_level(s, round, level, visited, pruned);
}

// Depth h (leaves): one warp per prefix of the depth-(h-1) frontier; every
// non-empty leaf is scored S = a_num * TP + a_den * (Nn - FP) and the best
// (score desc, original tuple asc) is kept.
__global__ void __launch_bounds__(kThreads) k_leaf(Cohort c, Solve s, int round, const Prefix *Fin, const u32 *nin)
{
    __shared__ WarpScratch scratch[kWarpsPerBlock];
    Key best = key_empty();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpScratch &ws = scratch[warp];
    const bool done = s.state[1] != 0;
    u64 visited = 0, pruned = 0, words = 0, prefixes = 0;
    if (!done) {
        const u32 count = *nin;
        const int h = s.h, L = h - 1;
        const int hi = c.G - 1;
        const u32 gw = blockIdx.x * kWarpsPerBlock + warp, nw = gridDim.x * kWarpsPerBlock;
        for (u32 i = gw; i < count; i += nw) {
            const Prefix p = Fin[i];
            unsigned by, bn;
            const int ky = warp_prefix_setup(c, s, p, L, ws, by, bn, lane, true);
            const int lo = prefix_gene(p, L - 1) + 1;
            ++prefixes;
            if (hi < lo) continue;
            visited += (u64)(hi - lo + 1);
            u64 alive = 0;
            if (ky) {
                for (int wb = lo >> 6; wb <= (hi >> 6); wb += 32) {
                    const int wi = wb + lane;
                    if (wi > (hi >> 6)) break;
                    words += (u64)ky;
                    u64 m = sibling_word(c, ws, ky, wi, lo, hi);
                    alive += (u64)__popcll(m);
                    while (m) {
                        const int b = __ffsll((long long)m) - 1;
                        m &= m - 1;
                        const int g = wi * 64 + b;
                        const u64 *trow = c.T + (size_t)g * c.WTp;
                        const u64 *nrow = c.N + (size_t)g * c.WNp;
                        int tp = 0, fp = 0;
                        for (unsigned bits = by; bits; bits &= bits - 1) {
                            const int w = __ffs(bits) - 1;
                            tp += __popcll(ws.ys[w] & trow[w]);
                        }
                        for (unsigned bits = bn; bits; bits &= bits - 1) {
                            const int w = __ffs(bits) - 1;
                            fp += __popcll(ws.ns[w] & nrow[w]);
                        }
                        const u64 s1 = s.a_num * (u64)tp + s.a_den * (u64)(c.Nn - fp) + 1;
                        if (s1 < best.s) continue;
                        Key k;
                        k.s = s1;
                        k.t0 = k.t1 = k.t2 = 0;
                        const int o = c.orig[g];
                        int pos = 0;
                        bool placed = false;
                        for (int q = 0; q < L; ++q) {
                            const int v = ws.po[q];
                            if (!placed && o < v) {
                                key_put(k, pos++, o);
                                placed = true;
                            }
                            key_put(k, pos++, v);
                        }
                        if (!placed) key_put(k, pos, o);
                        if (key_better(k, best)) best = k;
                    }
                }
            }
            alive = warp_sum_u64(alive);
            pruned += (u64)(hi - lo + 1) - alive;
            __syncwarp();
        }
        if (lane == 0) {
            count_level(s, round, h, visited, pruned);
            atomicAdd(s.work, words);
            atomicAdd(s.work + 1, prefixes);
        }
    }
    block_commit_best(best, s.slots);
}

// End of a round: reduce the per-block bests, record the winner with its TP / FP,
// clear the tumors it covers (DelCols) and raise the done flag when nothing was
// found or every tumor is covered.  One block.
__global__ void __launch_bounds__(kThreads) k_finalize(Cohort c, Solve s, int round)
{
    __shared__ Key wbest[kWarpsPerBlock];
    __shared__ int gs[kMaxH], os[kMaxH];
    if (s.state[1]) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Key best = key_empty();
    for (int i = threadIdx.x; i < s.nslots; i += blockDim.x) {
        const Key k = s.slots[i];
        if (key_better(k, best)) best = k;
        s.slots[i] = key_empty();
    }
    best = warp_max_key(best);
    if (lane == 0) wbest[warp] = best;
    __syncthreads();
    if (warp != 0) return;
    best = lane < kWarpsPerBlock ? wbest[lane] : key_empty();
    best = warp_max_key(best);
    if (best.s == 0) {
        if (lane == 0) s.state[1] = 1;
        return;
    }
    const int h = s.h;
    if (lane < h) {
        const int o = key_get(best, lane);
        os[lane] = o;
        gs[lane] = (int)c.inv[o];
    }
    __syncwarp();
    u64 y = 0, n = 0;
    if (lane < c.Wt) {
        y = s.U[lane];
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
    u64 u = 0;
    if (lane < c.Wt) {
        u = s.U[lane] & ~y;
        s.U[lane] = u;
    }
    const unsigned left = __ballot_sync(kFull, u != 0);
    if (lane == 0) {
        const int k = s.state[0];
        int *r = s.res + (size_t)k * (h + 2);
        for (int i = 0; i < h; ++i) r[i] = os[i];
        r[h] = tp;
        r[h + 1] = fp;
        s.state[0] = k + 1;
        if (!left) s.state[1] = 1;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers

void launch_transpose(const Cohort &c, u64 *CT, cudaStream_t st)
{
    const long long total = (long long)c.Nt * c.GW;
    if (total == 0) return;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    k_transpose<<<(unsigned)blocks, threads, 0, st>>>(c, CT);
}

void launch_solve_init(const Cohort &c, const Solve &s, int max_rounds, cudaStream_t st)
{
    cudaMemsetAsync(s.cnt, 0, sizeof(u64) * 2 * (size_t)s.h * (size_t)max_rounds, st);
    cudaMemsetAsync(s.slots, 0, sizeof(Key) * (size_t)s.nslots, st);
    cudaMemsetAsync(s.work, 0, sizeof(u64) * 2, st);
    k_solve_init<<<1, 64, 0, st>>>(c, s);
}

int level1_grid(const Cohort &c) { return (c.G + kThreads - 1) / kThreads; }

void launch_level1(const Cohort &c, const Solve &s, int round, Prefix *F1, u32 *n1, u32 cap1, cudaStream_t st)
{
    k_level1<<<level1_grid(c), kThreads, 0, st>>>(c, s, round, F1, n1, cap1);
}

void launch_expand(const Cohort &c, const Solve &s, int round, int level, const Prefix *Fin, const u32 *nin,
                   Prefix *Fout, u32 *nout, u32 cap, int grid, cudaStream_t st)
{
    k_expand<<<grid, kThreads, 0, st>>>(c, s, round, level, Fin, nin, Fout, nout, cap);
}

void launch_leaf(const Cohort &c, const Solve &s, int round, const Prefix *Fin, const u32 *nin, int grid,
                 cudaStream_t st)
{
    k_leaf<<<grid, kThreads, 0, st>>>(c, s, round, Fin, nin);
}

void launch_finalize(const Cohort &c, const Solve &s, int round, cudaStream_t st)
{
    k_finalize<<<1, kThreads, 0, st>>>(c, s, round);
}

}  // namespace mh
