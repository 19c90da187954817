// mh_solve_noalloc: the greedy solve of mh_solve for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while another component
// owns every byte of device memory through its own pool, plug-ins that are handed
// fixed buffers by a host framework, or callers that must not add allocator
// traffic (and its implicit synchronisation) to a latency-critical stream.  For
// them this entry point keeps every piece of scratch -- the sorted cohort store,
// its sample-major copy, the uncovered-tumor mask, the search frontiers, the
// per-block best candidates, the counters and the round state -- in one
// file-scope __device__ array of fixed size.  The caller passes the packed rows
// and the output buffers, both in device memory.  Nothing here calls cudaMalloc,
// cudaFree or any allocating library routine, and the success path touches no
// host heap either.
//
// Every GPU that loads this library keeps the array (kScratchBytes) until the
// process exits.  Every call shares it: calls whose work overlaps on the GPU
// (different streams, different host threads) race on it and must be
// serialised by the caller.  What must start at zero is cleared by each call.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "mh.h"
#include "mh_internal.h"

namespace mh {

namespace {

// Limits of the no-allocation solve.
constexpr int kNaMaxG = 8192;
constexpr int kNaMaxNt = 1024;
constexpr int kNaMaxNn = 1024;
constexpr int kNaMaxH = 4;
constexpr u32 kNaFrontierCap = 1u << 17;  // entries per intermediate depth
constexpr int kNaMaxSlots = 4096;

constexpr int kNaWTp = kNaMaxNt / 64;  // 16 words
constexpr int kNaWNp = kNaMaxNn / 64;
constexpr int kNaGW = kNaMaxG / 64;    // 128 words
constexpr int kNaRounds = kNaMaxNt + 2;

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the pieces inside the scratch array.
constexpr size_t kOffT = 0;
constexpr size_t kOffN = kOffT + align256(sizeof(u64) * kNaMaxG * kNaWTp);
constexpr size_t kOffCT = kOffN + align256(sizeof(u64) * kNaMaxG * kNaWNp);
constexpr size_t kOffCN = kOffCT + align256(sizeof(u64) * kNaMaxNt * kNaGW);
constexpr size_t kOffOrig = kOffCN + align256(sizeof(u64) * kNaMaxNn * kNaGW);
constexpr size_t kOffInv = kOffOrig + align256(sizeof(u16) * kNaMaxG);
constexpr size_t kOffU = kOffInv + align256(sizeof(u32) * kNaMaxG);
constexpr size_t kOffState = kOffU + align256(sizeof(u64) * kNaWTp);
constexpr size_t kOffWork = kOffState + align256(sizeof(int) * kStateWords);
constexpr size_t kOffCounts = kOffWork + align256(sizeof(u64) * (kWorkCount + 1));
constexpr size_t kOffRes = kOffCounts + align256(sizeof(u32) * kCountWords);
constexpr size_t kOffCnt = kOffRes + align256(sizeof(int) * kNaRounds * (kNaMaxH + 2));
constexpr size_t kOffSlots = kOffCnt + align256(sizeof(u64) * 2 * kNaRounds * kNaMaxH);
constexpr size_t kOffCand = kOffSlots + align256(sizeof(Key) * kNaMaxSlots);
constexpr size_t kOffF1 = kOffCand + align256(sizeof(Key) * kCandidates);
constexpr size_t kOffF2 = kOffF1 + align256(sizeof(Rec) * kNaMaxG);
constexpr size_t kOffF3 = kOffF2 + align256(sizeof(Rec) * kNaFrontierCap);
constexpr size_t kScratchBytes = kOffF3 + align256(sizeof(Rec) * kNaFrontierCap);  // about 30 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// 16-bit gene index + 12-bit tumor count: keys are unique, so any sort of them
// is the stable "most sparse first, ties by index" order.
__global__ void k_na_sort_keys(const u64 *bm, int G, int Wt, int Wn, u32 *keys_out)
{
    __shared__ u32 keys[kNaMaxG];
    const int W = Wt + Wn;
    for (int g = threadIdx.x; g < kNaMaxG; g += blockDim.x) {
        u32 key = 0xffffffffu;
        if (g < G) {
            int pc = 0;
            for (int w = 0; w < Wt; ++w) pc += __popcll(bm[(size_t)g * W + w]);
            key = ((u32)pc << 16) | (u32)g;
        }
        keys[g] = key;
    }
    __syncthreads();
    for (int k = 2; k <= kNaMaxG; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < kNaMaxG; i += blockDim.x) {
                const int p = i ^ j;
                if (p > i) {
                    const bool up = (i & k) == 0;
                    const u32 a = keys[i], b = keys[p];
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x) keys_out[g] = keys[g];
}

// Sorted rows into the padded store; flags padding bits that are set.
__global__ void k_na_pack(const u64 *bm, Cohort c, const u32 *keys, u64 *T, u64 *N, u16 *orig, u32 *inv,
                          int *state)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.G) return;
    const int g = (int)(keys[i] & 0xffffu);
    const int W = c.Wt + c.Wn;
    const u64 *row = bm + (size_t)g * W;
    bool bad = false;
    for (int w = 0; w < c.WTp; ++w) {
        const u64 v = w < c.Wt ? row[w] : 0ull;
        if (w == c.Wt - 1 && (c.Nt & 63) && (v >> (c.Nt & 63))) bad = true;
        T[(size_t)i * c.WTp + w] = v;
    }
    for (int w = 0; w < c.WNp; ++w) {
        const u64 v = w < c.Wn ? row[c.Wt + w] : 0ull;
        if (w == c.Wn - 1 && (c.Nn & 63) && (v >> (c.Nn & 63))) bad = true;
        N[(size_t)i * c.WNp + w] = v;
    }
    orig[i] = (u16)g;
    inv[g] = (u32)i;
    if (bad) atomicOr(state + 2, 1);
}

__global__ void k_na_unpack(const int *res, const int *state, int h, int capacity, int32_t *genes, int32_t *tp,
                            int32_t *fp)
{
    const int k = state[0] < capacity ? state[0] : capacity;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
        const int *r = res + (size_t)i * (h + 2);
        for (int j = 0; j < h; ++j) genes[(size_t)i * h + j] = r[j];
        tp[i] = r[h];
        fp[i] = r[h + 1];
    }
}

int na_fail(int code, const char *fmt, ...)
{
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_error_text(buf);
    return code;
}

#define NA_CUDA(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return na_fail(MH_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

// Device address of the scratch array on the current device, looked up on every
// call: an address kept from an earlier call would be stale after a device reset
// or with a new primary context, and the lookup costs little next to a solve.
int scratch_for_current_device(unsigned char **ptr, int *num_sms)
{
    int dev = 0;
    NA_CUDA(cudaGetDevice(&dev));
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return na_fail(MH_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return na_fail(MH_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    *ptr = (unsigned char *)p;
    *num_sms = sms;
    return MH_OK;
}

}  // namespace

}  // namespace mh

using namespace mh;

extern "C" MH_API int mh_solve_noalloc(const uint64_t *d_bitmaps, int32_t G, int32_t Nt, int32_t Nn, int32_t h,
                                       mh_rational alpha, void *stream, int32_t *d_genes, int32_t *d_tp,
                                       int32_t *d_fp, int32_t capacity, int32_t *k_out, int32_t *rounds_out)
{
    if (!d_bitmaps || !d_genes || !d_tp || !d_fp || !k_out)
        return na_fail(MH_EINVAL, "mh_solve_noalloc: NULL input or output pointer");
    if (G < 1 || G > kNaMaxG || Nt < 0 || Nt > kNaMaxNt || Nn < 0 || Nn > kNaMaxNn)
        return na_fail(MH_EINVAL,
                       "mh_solve_noalloc: G=%d Nt=%d Nn=%d exceed the fixed scratch (G <= %d, Nt <= %d, Nn <= %d)",
                       G, Nt, Nn, kNaMaxG, kNaMaxNt, kNaMaxNn);
    if (h < 1 || h > kNaMaxH) return na_fail(MH_EINVAL, "mh_solve_noalloc: h=%d outside [1, %d]", h, kNaMaxH);
    if (alpha.num < 0 || alpha.den <= 0)
        return na_fail(MH_EINVAL, "mh_solve_noalloc: alpha=%d/%d needs num >= 0, den > 0", alpha.num, alpha.den);
    if (capacity < Nt) return na_fail(MH_EINVAL, "mh_solve_noalloc: capacity %d < Nt=%d", capacity, Nt);
    unsigned char *base = nullptr;
    int num_sms = 0;
    int rc = scratch_for_current_device(&base, &num_sms);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;

    Cohort c;
    c.G = G; c.Nt = Nt; c.Nn = Nn;
    c.Wt = (Nt + 63) / 64; c.Wn = (Nn + 63) / 64;
    c.WTp = (c.Wt + 1) & ~1;
    if (c.WTp < 2) c.WTp = 2;
    c.WNp = (c.Wn + 1) & ~1;
    if (c.WNp < 2) c.WNp = 2;
    c.GW = (((G + 63) / 64) + 1) & ~1;
    if (c.GW < 2) c.GW = 2;
    u64 *T = (u64 *)(base + kOffT);
    u64 *N = (u64 *)(base + kOffN);
    u64 *CT = (u64 *)(base + kOffCT);
    u64 *CN = (u64 *)(base + kOffCN);
    u16 *orig = (u16 *)(base + kOffOrig);
    u32 *inv = (u32 *)(base + kOffInv);
    c.T = T; c.N = N; c.CT = CT; c.CN = CN; c.orig = orig; c.inv = inv;
    c.CC = nullptr;  // no running-count table here: every subtree is searched
    c.SL = nullptr;
    c.SO = nullptr;
    c.SLo = nullptr;
    c.GR = nullptr;
    c.GS = nullptr;
    c.TO = nullptr;
    c.NO = nullptr;

    Solve s;
    s.h = h;
    s.prune = MH_PRUNE_PAPER;
    s.a_num = (u64)alpha.num;
    s.a_den = (u64)alpha.den;
    s.U = (u64 *)(base + kOffU);
    s.state = (int *)(base + kOffState);
    s.res = (int *)(base + kOffRes);
    s.cnt = (u64 *)(base + kOffCnt);
    s.slots = (Key *)(base + kOffSlots);
    s.work = (u64 *)(base + kOffWork);
    s.best_hint = s.work + kWorkCount;
    s.cand = (Key *)(base + kOffCand);
    s.champ = nullptr;  // one kernel per phase: no per-sample champions
    s.champ_ok = nullptr;
    s.ssum = nullptr;
    s.gk = nullptr;
    s.cov = nullptr;
    s.run = nullptr;
    s.cut = nullptr;
    s.shard = 0;
    s.nshards = 1;
    s.xbest = nullptr;
    const int leaf_blocks = num_sms * 4;
    s.nslots = level1_grid(c) > leaf_blocks ? level1_grid(c) : leaf_blocks;
    if (s.nslots > kNaMaxSlots) return na_fail(MH_EINVAL, "mh_solve_noalloc: %d SMs exceed the slot array", num_sms);
    u32 *counts = (u32 *)(base + kOffCounts);
    // each frontier is split into kShards equal regions (the region is the cap)
    Frontiers fr;
    for (int l = 0; l < kMaxH; ++l) {
        fr.F[l] = nullptr;
        fr.cap[l] = 0;
        fr.sig[l] = nullptr;
        fr.lb[l] = nullptr;
        fr.lc[l] = nullptr;
    }
    fr.F[1] = (Rec *)(base + kOffF1);
    fr.cap[1] = kNaMaxG / kShards;
    fr.F[2] = (Rec *)(base + kOffF2);
    fr.cap[2] = kNaFrontierCap / kShards;
    fr.F[3] = (Rec *)(base + kOffF3);
    fr.cap[3] = kNaFrontierCap / kShards;
    Rec *F[kMaxH] = {fr.F[0], fr.F[1], fr.F[2], fr.F[3]};
    (void)F;

    // store: sort keys (into the depth-2 frontier area, free at this point), pack, transpose
    u32 *keys = (u32 *)F[2];
    NA_CUDA(cudaMemsetAsync(s.state, 0, sizeof(int) * kStateWords, st));
    k_na_sort_keys<<<1, 1024, 0, st>>>((const u64 *)d_bitmaps, G, c.Wt, c.Wn, keys);
    k_na_pack<<<(G + 255) / 256, 256, 0, st>>>((const u64 *)d_bitmaps, c, keys, T, N, orig, inv, s.state);
    launch_transpose(c, T, c.WTp, Nt, CT, st);
    launch_transpose(c, N, c.WNp, Nn, CN, st);
    NA_CUDA(cudaGetLastError());
    int hs[kStateWords] = {};
    NA_CUDA(cudaMemcpyAsync(hs, s.state, sizeof hs, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if (hs[2]) return na_fail(MH_EINVAL, "mh_solve_noalloc: padding bits past Nt or Nn are set");

    launch_solve_init(c, s, kNaRounds, Nt + 1, counts, 1, st);
    const int grid = leaf_blocks;
    // rounds run on the device; the host enqueues them in growing batches
    int batch = 4, rounds = 0;
    bool done = Nt == 0;
    int st8[kStateWords];
    while (!done) {
        const int n = batch < Nt + 1 - rounds ? batch : Nt + 1 - rounds;
        for (int b = 0; b < n; ++b) {
            launch_level1(c, s, fr, counts, st);
            for (int l = 2; l <= h - 1; ++l) launch_expand(c, s, l, fr, counts, grid, st);
            if (h >= 2) launch_leaf(c, s, fr, counts, grid, st);
            launch_finalize(c, s, counts, st);
        }
        NA_CUDA(cudaGetLastError());
        NA_CUDA(cudaMemcpyAsync(st8, s.state, sizeof st8, cudaMemcpyDeviceToHost, st));
        NA_CUDA(cudaStreamSynchronize(st));
        rounds = st8[4];
        if (st8[3])
            return na_fail(MH_ENOMEM,
                           "mh_solve_noalloc: a search frontier exceeds the fixed scratch (%u prefixes per depth)",
                           kNaFrontierCap);
        done = st8[1] != 0 || rounds >= Nt + 1;
        batch = batch * 2 < 64 ? batch * 2 : 64;
    }
    k_na_unpack<<<4, 256, 0, st>>>(s.res, s.state, h, capacity, d_genes, d_tp, d_fp);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemcpyAsync(st8, s.state, sizeof st8, cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    *k_out = st8[0];
    if (rounds_out) *rounds_out = rounds;
    return MH_OK;
}
