// Host runtime and C ABI of libmh (declared in include/mh.h).
//
// mh_create packs one cohort for the device (sparsity sort of §III-C, padded
// gene-major rows, sample-major tumor copy).  mh_solve runs the greedy loop of
// Algorithm 1; each round is a fixed sequence of kernel launches on the
// handle's stream (depth 1, depths 2..h-1, leaves, finalize) and one 16-byte
// read-back of the round state.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <cmath>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <sys/stat.h>
#include <string>
#include <vector>

#include "mh.h"
#include "mh_internal.h"

using namespace mh;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define MH_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? MH_ENOMEM : MH_ECUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                    \
    } while (0)

// Device memory of handles comes from one stream-ordered pool per device that keeps
// what is freed (release threshold: unlimited), so creating and destroying handles
// (a served request each) neither maps memory again nor synchronises the device.
constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pools[kMaxDevices] = {};

int device_pool(int dev, cudaMemPool_t *out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(MH_ECUDA, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        MH_CUDA(cudaMemPoolCreate(&g_pools[dev], &props));
        unsigned long long keep = ~0ull;
        MH_CUDA(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    *out = g_pools[dev];
    return MH_OK;
}

// Frontier memory of one handle: MH_FRONTIER_BUDGET_MB if set, else 80% of the
// device memory that is free (including what the pool holds unused) when a
// frontier grows.
size_t frontier_budget(int dev = -1)
{
    const char *v = getenv("MH_FRONTIER_BUDGET_MB");
    if (v && *v) {
        const long long mb = atoll(v);
        if (mb > 0) return size_t(mb) << 20;
    }
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return size_t(16) << 30;
    if (dev >= 0 && dev < kMaxDevices && g_pools[dev]) {
        unsigned long long reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(g_pools[dev], cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(g_pools[dev], cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess &&
            reserved > used)
            free_b += (size_t)(reserved - used);
    }
    return (size_t)(free_b * 0.8);
}

// n elements from the device's pool, ordered on stream st.
// Host-side fault injection (mh_set_fault, or MH_FAULT in the environment at the
// first call): the n-th next device allocation fails, or the n-th next solve
// reports that a bounded device wait expired.  Nothing is injected on the device.
std::atomic<int> g_fault_alloc{0}, g_fault_timeout{0};
std::atomic<int> g_fault_env_read{0};

int parse_fault(const char *spec)
{
    if (!spec || !*spec || !strcmp(spec, "none")) {
        g_fault_alloc = 0;
        g_fault_timeout = 0;
        return MH_OK;
    }
    int n = 0;
    if (sscanf(spec, "alloc_fail=%d", &n) == 1 && n > 0) {
        g_fault_alloc = n;
        return MH_OK;
    }
    if (sscanf(spec, "timeout_after=%d", &n) == 1 && n > 0) {
        g_fault_timeout = n;
        return MH_OK;
    }
    return fail(MH_EINVAL, "fault spec '%s': expected none, alloc_fail=N or timeout_after=N (N >= 1)", spec);
}

// Counts an armed fault down; true when it fires.
bool fault_fires(std::atomic<int> &f)
{
    if (!g_fault_env_read.exchange(1)) {
        const char *env = getenv("MH_FAULT");
        if (env && *env) parse_fault(env);
    }
    int v = f.load();
    while (v > 0 && !f.compare_exchange_weak(v, v - 1)) {
    }
    return v == 1;
}

template <typename T>
int dalloc(T **p, size_t n, int64_t *acct, int dev, cudaStream_t st)
{
    *p = nullptr;
    if (n == 0) n = 1;
    if (fault_fires(g_fault_alloc)) return fail(MH_ENOMEM, "injected device allocation failure (mh_set_fault)");
    cudaMemPool_t pool;
    const int rc = device_pool(dev, &pool);
    if (rc) return rc;
    MH_CUDA(cudaMallocFromPoolAsync((void **)p, n * sizeof(T), pool, st));
    if (acct) *acct += (int64_t)(n * sizeof(T));
    return MH_OK;
}

void dfree(void *p, cudaStream_t st)
{
    if (p) cudaFreeAsync(p, st);
}

// Pinned host buffers for the round state read-back (state + frontier counts),
// recycled instead of freed: freeing pinned memory synchronises the device.
constexpr size_t kStateBytes = sizeof(int) * (kStateWords + kCountWords);
std::mutex g_pinned_mutex;
std::vector<int *> g_pinned_free;

int *pinned_state_get()
{
    {
        std::lock_guard<std::mutex> lock(g_pinned_mutex);
        if (!g_pinned_free.empty()) {
            int *p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    int *p = nullptr;
    if (cudaMallocHost((void **)&p, kStateBytes) != cudaSuccess) return nullptr;
    return p;
}

void pinned_state_put(int *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mutex);
    g_pinned_free.push_back(p);
}

// Pinned host buffers for reading a solve's results back (selections, counters,
// cuts, diagnostics in one asynchronous batch of copies), recycled the same way:
// the smallest free one that is large enough, else a new one.
std::vector<std::pair<void *, size_t>> g_pinned_res_free;

void *pinned_res_get(size_t bytes, size_t *got)
{
    {
        std::lock_guard<std::mutex> lock(g_pinned_mutex);
        int best = -1;
        for (int i = 0; i < (int)g_pinned_res_free.size(); ++i)
            if (g_pinned_res_free[i].second >= bytes &&
                (best < 0 || g_pinned_res_free[i].second < g_pinned_res_free[best].second))
                best = i;
        if (best >= 0) {
            auto e = g_pinned_res_free[best];
            g_pinned_res_free.erase(g_pinned_res_free.begin() + best);
            *got = e.second;
            return e.first;
        }
    }
    const size_t want = std::max<size_t>(bytes, 64 << 10);
    void *p = nullptr;
    if (cudaMallocHost(&p, want) != cudaSuccess) return nullptr;
    *got = want;
    return p;
}

void pinned_res_put(void *p, size_t bytes)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mutex);
    g_pinned_res_free.emplace_back(p, bytes);
}

}  // namespace

namespace mh {
void set_error_text(const char *text) { g_last_error = text; }
}  // namespace mh

struct mh_handle {
    int G = 0, Nt = 0, Nn = 0;
    Cohort c{};
    cudaStream_t stream = nullptr;
    int num_sms = 0, dev = 0;
    int64_t device_bytes = 0;
    // cohort store
    unsigned char *dStore = nullptr;      // one block holding every piece below
    u64 *dT = nullptr, *dN = nullptr, *dCT = nullptr, *dCN = nullptr;
    u16 *dOrig = nullptr, *dCC = nullptr, *dSL = nullptr, *dSLo = nullptr;
    u32 *dSO = nullptr;
    u32 *dInv = nullptr;
    // solve workspace (grown on demand)
    int ws_h = 0, ws_rounds = 0, ws_slots = 0;
    u64 *dU = nullptr, *dCnt = nullptr, *dWork = nullptr, *dCut = nullptr;
    int *dState = nullptr, *dRes = nullptr;
    Key *dSlots = nullptr, *dCand = nullptr, *dChamp = nullptr;
    int *dChampOk = nullptr;
    u64 *dSsum = nullptr;                 // per-sample sums of the counters (Nt x 2h)
    u32 *dCounts = nullptr;               // frontier sizes, one per depth, then work-distribution counters
    Rec *dF[kMaxH] = {};               // frontier of depth l at index l
    u32 cap[kMaxH] = {};
    unsigned char *dSide[kMaxH] = {};     // per record slot of depth l: sig, lb, lc (incremental rounds)
    u32 *dGK = nullptr;                   // per gene: uncovered tumors carrying it (incremental rounds)
    u64 *dCov = nullptr;                  // tumors covered by the last round's winner
    int *hState = nullptr;                // pinned: state + frontier counts
    void *hRes = nullptr;                 // pinned: a solve's results on their way back
    size_t hRes_bytes = 0;
    GridSync *dSync = nullptr;            // barrier of the persistent solve
    int coop = 0, pgrid = 0;              // cooperative launch supported; persistent grid size
    std::vector<int> m_s;                 // mutated genes per tumor sample (work estimate of a batch)
    int64_t frontier_bytes = 0;
    cudaEvent_t evk[2] = {};              // around each cooperative launch of a persistent solve
    bool presized[kMaxH] = {};            // frontier of depth l sized from its bound

    // device memory goes back to the pool in the order of the handle's stream
    ~mh_handle()
    {
        for (int i = 0; i < 2; ++i)
            if (evk[i]) cudaEventDestroy(evk[i]);
        for (void *p : {(void *)dStore, (void *)dU,
                        (void *)dCnt, (void *)dCut, (void *)dWork, (void *)dState, (void *)dRes, (void *)dSlots, (void *)dCand, (void *)dChamp, (void *)dChampOk, (void *)dSsum,
                        (void *)dCounts, (void *)dSync})
            dfree(p, stream);
        for (int l = 0; l < kMaxH; ++l) {
            dfree(dF[l], stream);
            dfree(dSide[l], stream);
        }
        dfree(dGK, stream);
        dfree(dCov, stream);
        pinned_state_put(hState);
        pinned_res_put(hRes, hRes_bytes);
    }
};

namespace {

int validate_dims(int32_t G, int32_t Nt, int32_t Nn)
{
    if (G < 1 || G > kMaxGenes) return fail(MH_EINVAL, "G=%d outside [1, %d]", G, kMaxGenes);
    if (Nt < 0 || Nt > kMaxSamples) return fail(MH_EINVAL, "Nt=%d outside [0, %d]", Nt, kMaxSamples);
    if (Nn < 0 || Nn > kMaxWords * 64) return fail(MH_EINVAL, "Nn=%d outside [0, %d]", Nn, kMaxWords * 64);
    return MH_OK;
}

// Builds the device store from host rows (validated here) on the handle's stream;
// with sync, waits for the build to finish.
int build_store(mh_handle *H, const uint64_t *bm, bool sync = true)
{
    const int G = H->G, Nt = H->Nt, Nn = H->Nn;
    const int Wt = (Nt + 63) / 64, Wn = (Nn + 63) / 64, W = Wt + Wn;
    // one pass over the rows: padding bits, each gene's tumor mutations, each
    // tumor's mutated genes
    std::vector<int> pc(G);
    H->m_s.assign(Nt, 0);
    for (int g = 0; g < G; ++g) {
        const uint64_t *row = bm + (size_t)g * W;
        if (Nt % 64 && Wt && (row[Wt - 1] >> (Nt % 64)))
            return fail(MH_EINVAL, "gene %d: tumor padding bits past Nt=%d are set", g, Nt);
        if (Nn % 64 && Wn && (row[Wt + Wn - 1] >> (Nn % 64)))
            return fail(MH_EINVAL, "gene %d: normal padding bits past Nn=%d are set", g, Nn);
        int k = 0;
        for (int w = 0; w < Wt; ++w) {
            k += __builtin_popcountll(row[w]);
            for (uint64_t x = row[w]; x; x &= x - 1) ++H->m_s[w * 64 + __builtin_ctzll(x)];
        }
        pc[g] = k;
    }
    // search order: ascending tumor mutation count, ties by original index (§III-C),
    // by a counting sort (stable)
    std::vector<u32> order(G);
    {
        std::vector<int> start((size_t)Nt + 2, 0);
        for (int g = 0; g < G; ++g) ++start[pc[g] + 1];
        for (int k = 0; k <= Nt; ++k) start[k + 1] += start[k];
        for (int g = 0; g < G; ++g) order[start[pc[g]]++] = (u32)g;
    }
    Cohort &c = H->c;
    c.G = G; c.Nt = Nt; c.Nn = Nn; c.Wt = Wt; c.Wn = Wn;
    c.WTp = std::max(2, (Wt + 1) & ~1);
    c.WNp = std::max(2, (Wn + 1) & ~1);
    c.GW = std::max(2, (((G + 63) / 64) + 1) & ~1);
    // each tumor's genes start at SO[s] in the per-sample lists (its column's popcount
    // is its number of mutated genes)
    std::vector<u32> SO((size_t)Nt + 1, 0);
    for (int s = 0; s < Nt; ++s) SO[s + 1] = SO[s] + (u32)H->m_s[s];
    const size_t nSL = std::max<size_t>(SO[Nt], 1);

    int rc;
    cudaStream_t st = H->stream;
    // the whole store in one device block (256-byte aligned pieces), written by the
    // store kernels from the uploaded rows and permutation
    size_t off = 0;
    auto piece = [&](size_t bytes) {
        const size_t o = off;
        off += (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
        return o;
    };
    const size_t rowsT = (size_t)G * c.WTp, rowsN = (size_t)G * c.WNp;
    const size_t oT = piece(rowsT * sizeof(u64)), oN = piece(rowsN * sizeof(u64));
    const size_t oCT = piece((size_t)Nt * c.GW * sizeof(u64)), oCN = piece((size_t)Nn * c.GW * sizeof(u64));
    const size_t oCC = piece((size_t)Nt * (c.GW + 1) * sizeof(u16)), oSL = piece(nSL * sizeof(u16));
    const size_t oSLo = piece(nSL * sizeof(u16)), oSO = piece(SO.size() * sizeof(u32));
    const size_t oOrig = piece((size_t)G * sizeof(u16)), oInv = piece((size_t)G * sizeof(u32));
    const size_t oGR = piece((size_t)G * sizeof(Rec)), oGS = piece((size_t)G * sizeof(u64));
    const size_t oTO = piece(rowsT * sizeof(u64)), oNO = piece(rowsN * sizeof(u64));
    // scratch for the build: the rows as given, the permutation, the original-order
    // sample-major copy (freed in stream order after the build)
    size_t toff = 0;
    auto tpiece = [&](size_t bytes) {
        const size_t o = toff;
        toff += (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
        return o;
    };
    const size_t tBm = tpiece((size_t)G * W * sizeof(u64)), tOrder = tpiece((size_t)G * sizeof(u32));
    const size_t tCTo = tpiece((size_t)Nt * c.GW * sizeof(u64));
    if ((rc = dalloc(&H->dStore, off, &H->device_bytes, H->dev, st))) return rc;
    unsigned char *scratch = nullptr;
    if ((rc = dalloc(&scratch, toff, nullptr, H->dev, st))) {
        dfree(H->dStore, st);
        H->dStore = nullptr;
        return rc;
    }
    if ((size_t)G * W) MH_CUDA(cudaMemcpyAsync(scratch + tBm, bm, (size_t)G * W * sizeof(u64), cudaMemcpyHostToDevice, st));
    if (G) MH_CUDA(cudaMemcpyAsync(scratch + tOrder, order.data(), (size_t)G * sizeof(u32), cudaMemcpyHostToDevice, st));
    MH_CUDA(cudaMemcpyAsync(H->dStore + oSO, SO.data(), SO.size() * sizeof(u32), cudaMemcpyHostToDevice, st));
    H->dT = (u64 *)(H->dStore + oT);
    H->dN = (u64 *)(H->dStore + oN);
    H->dCT = (u64 *)(H->dStore + oCT);
    H->dCN = (u64 *)(H->dStore + oCN);
    H->dCC = (u16 *)(H->dStore + oCC);
    H->dSL = (u16 *)(H->dStore + oSL);
    H->dSLo = (u16 *)(H->dStore + oSLo);
    H->dSO = (u32 *)(H->dStore + oSO);
    H->dOrig = (u16 *)(H->dStore + oOrig);
    H->dInv = (u32 *)(H->dStore + oInv);
    c.T = H->dT; c.N = H->dN; c.CT = H->dCT; c.CN = H->dCN; c.orig = H->dOrig; c.inv = H->dInv;
    c.CC = Nt ? H->dCC : nullptr;
    c.SL = H->dSL;
    c.SO = H->dSO;
    c.SLo = H->dSLo;
    c.GR = (const Rec *)(H->dStore + oGR);
    c.GS = (const u64 *)(H->dStore + oGS);
    c.TO = (const u64 *)(H->dStore + oTO);
    c.NO = (const u64 *)(H->dStore + oNO);
    StoreBuild b;
    b.c = c;
    b.bm = (const u64 *)(scratch + tBm);
    b.order = (const u32 *)(scratch + tOrder);
    b.SO = H->dSO;
    b.T = H->dT; b.N = H->dN;
    b.TO = (u64 *)(H->dStore + oTO);
    b.NO = (u64 *)(H->dStore + oNO);
    b.CT = H->dCT; b.CN = H->dCN;
    b.CTo = (u64 *)(scratch + tCTo);
    b.CC = H->dCC; b.SL = H->dSL; b.SLo = H->dSLo; b.orig = H->dOrig; b.inv = H->dInv;
    b.GR = (Rec *)(H->dStore + oGR);
    b.GS = (u64 *)(H->dStore + oGS);
    MH_CUDA(launch_store_build(b, st));
    dfree(scratch, st);
    if (sync) MH_CUDA(cudaStreamSynchronize(st));  // build errors surface here
    return MH_OK;
}

int create_common(const uint64_t *bm, int32_t G, int32_t Nt, int32_t Nn, cudaStream_t stream, mh_handle **out,
                  bool sync = true)
{
    mh_handle *H = new (std::nothrow) mh_handle();
    if (!H) return fail(MH_ENOMEM, "host allocation of the handle failed");
    H->G = G; H->Nt = Nt; H->Nn = Nn;
    H->stream = stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    H->dev = dev;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&H->coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) {
        delete H;
        return fail(MH_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    int rc = build_store(H, bm, sync);
    if (rc) {
        delete H;
        return rc;
    }
    *out = H;
    return MH_OK;
}

// Grows the frontier of depth l to at least n records per shard (within the budget),
// with a quarter more room unless `exact`.
int ensure_frontier(mh_handle *H, int l, u64 n, bool exact = false)
{
    if (n <= H->cap[l]) return MH_OK;
    // smallest region: 2048 records per shard, or MH_FRONTIER_MIN_RECORDS
    u64 least = 1u << 11;
    const char *mn = getenv("MH_FRONTIER_MIN_RECORDS");
    if (mn && *mn && atoll(mn) > 0) least = (u64)atoll(mn);
    u64 want = std::max<u64>(exact ? n : n + n / 4, least);
    if (want > 0xffffffffull / kShards) want = 0xffffffffull / kShards;
    const int64_t old_bytes = (int64_t)H->cap[l] * kShards * (int64_t)kSlotBytes;
    const int64_t new_bytes = (int64_t)want * kShards * (int64_t)kSlotBytes;
    const char *fixed = getenv("MH_FRONTIER_BUDGET_MB");
    const bool over = (fixed && *fixed) ? (size_t)(H->frontier_bytes - old_bytes + new_bytes) > frontier_budget()
                                        : (size_t)(new_bytes - old_bytes) > frontier_budget(H->dev);
    if (over || n > want)
        return fail(MH_ENOMEM, "depth-%d frontier needs %llu records per shard (%.1f GB), above the frontier budget",
                    l, (unsigned long long)n, (double)n * kShards * kSlotBytes / 1e9);
    dfree(H->dF[l], H->stream);  // stream-ordered: after the kernels that used it
    dfree(H->dSide[l], H->stream);
    H->dF[l] = nullptr;
    H->dSide[l] = nullptr;
    H->frontier_bytes -= old_bytes;
    H->device_bytes -= old_bytes;
    H->cap[l] = 0;
    int rc = dalloc(&H->dF[l], (size_t)want * kShards, &H->device_bytes, H->dev, H->stream);
    if (rc) return rc;
    rc = dalloc(&H->dSide[l], (size_t)want * kShards * (kSlotBytes - sizeof(Rec)), &H->device_bytes, H->dev,
                H->stream);
    if (rc) return rc;
    H->cap[l] = (u32)want;
    H->frontier_bytes += new_bytes;
    return MH_OK;
}

// After an overflow: grows every depth whose busiest shard outgrew its region.
int grow_overflowed(mh_handle *H, int h, const u32 *hc)
{
    for (int l = 1; l < h; ++l) {
        u32 mx = 0;
        for (int i = 0; i < kShards; ++i) mx = std::max(mx, hc[shard_slot(l, i)]);
        if (mx > H->cap[l]) {
            const int rc = ensure_frontier(H, l, mx);
            if (rc) return rc;
        }
    }
    return MH_OK;
}

int leaf_grid(const mh_handle *H) { return std::max(1, H->num_sms * 4); }

int ensure_workspace(mh_handle *H, int h)
{
    const int rounds = H->Nt + 2;
    const int slots = std::max(std::max(level1_grid(H->c), leaf_grid(H)),
                               std::max(persistent_grid(H->num_sms, true),
                                        std::max(batch_grid(H->num_sms, 3), batch_grid(H->num_sms, 4))));
    int rc;
    const int dev = H->dev;
    cudaStream_t st = H->stream;
    // each piece on its own, so that a call after a failed allocation completes the set
    auto need = [&](auto **p, size_t n) { return *p ? MH_OK : dalloc(p, n, &H->device_bytes, dev, st); };
    const size_t nt1 = (size_t)std::max(H->Nt, 1);
    if ((rc = need(&H->dU, (size_t)H->c.WTp)) || (rc = need(&H->dState, (size_t)kStateWords)) ||
        (rc = need(&H->dWork, (size_t)kWorkCount + 2)) || (rc = need(&H->dCounts, (size_t)kCountSets * kCountWords)) ||
        (rc = need(&H->dCand, (size_t)kCandidates)) || (rc = need(&H->dChamp, nt1)) ||
        (rc = need(&H->dChampOk, nt1)) || (rc = need(&H->dSsum, nt1 * 2 * kMaxH)) ||
        (rc = need(&H->dGK, (size_t)H->G)) || (rc = need(&H->dCov, (size_t)H->c.WTp + 2 * (kMaxH + 1))) ||
        (rc = need(&H->dSync, (size_t)1)))
        return rc;
    if (!H->hState) {
        H->pgrid = H->coop ? persistent_grid(H->num_sms, true) : 0;
        if (!(H->hState = pinned_state_get())) return fail(MH_ENOMEM, "pinned host allocation failed");
    }
    if (h > H->ws_h || rounds > H->ws_rounds) {
        dfree(H->dCnt, st);
        dfree(H->dRes, st);
        dfree(H->dCut, st);
        H->dCnt = nullptr;
        H->dRes = nullptr;
        H->dCut = nullptr;
        const int hh = std::max(h, H->ws_h);
        if ((rc = dalloc(&H->dCnt, (size_t)rounds * hh * 2, &H->device_bytes, dev, st))) return rc;
        if ((rc = dalloc(&H->dCut, (size_t)rounds * hh, &H->device_bytes, dev, st))) return rc;
        if ((rc = dalloc(&H->dRes, (size_t)rounds * (hh + 2), &H->device_bytes, dev, st))) return rc;
        H->ws_h = hh;
        H->ws_rounds = rounds;
    }
    if (slots > H->ws_slots) {
        dfree(H->dSlots, st);
        H->dSlots = nullptr;
        if ((rc = dalloc(&H->dSlots, (size_t)2 * slots, &H->device_bytes, dev, st))) return rc;
        H->ws_slots = slots;
    }
    // depth 1: a warp appends its 32 genes to one of kShards regions
    if ((rc = ensure_frontier(H, 1, (u64)(H->G + kShards - 1) / kShards + 64))) return rc;
    for (int l = 2; l < h; ++l)
        if ((rc = ensure_frontier(H, l, 1))) return rc;
    return MH_OK;
}

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

}  // namespace

namespace {

double work_estimate(const mh_handle *H, int d);

// Expected search work (work_estimate with d = h - 1) above which the served
// runtime treats a request as "large" (it pauses for small ones and at most
// large_slots of them share the GPU).
constexpr double kLargeWork = 4.0e6;

// Build of the single-cohort persistent kernel for a solve: one block of 16 warps
// per SM (the cheaper grid barrier; with single-sample subtrees counted in closed
// form it is the faster build for every cohort measured, c1-c3 and the served
// cohorts), or four blocks of 8 warps per SM with MH_PERSISTENT_BUILD=large.
bool use_large_build(const mh_handle *, int)
{
    const char *v = getenv("MH_PERSISTENT_BUILD");
    return v && !strcmp(v, "large");
}

// Expected depth-l frontier records from sets = sum_s C(m_s, l), the l-gene sets
// that share a tumor (m_s: genes mutated in tumor s).  Nodes with one uncovered
// tumor are counted in closed form and never stored, so a frontier holds the
// l-sets that two or more tumors share: in the first round of the synthetic
// cohorts (c2, c3) 7-9% of `sets` at l = 2 and under 1% at l = 3.  The estimate
// takes 1/8 and 1/64; a frontier that outgrows it grows and its round reruns.
double frontier_records_estimate(double sets, int l) { return sets / (l == 2 ? 8.0 : 64.0); }

// Sizes the frontiers of depths 2..h-1 once per handle from the first-round
// estimate above.  The shards fill unevenly, hence 15% more per shard.  An
// estimate above half the frontier budget is skipped (the frontier then grows when
// it overflows), and so is everything with MH_FRONTIER_PRESIZE=0 (frontiers grown
// on overflow only).
int presize_frontiers(mh_handle *H, int h)
{
    const char *v = getenv("MH_FRONTIER_PRESIZE");
    if (v && v[0] == '0') return MH_OK;
    for (int l = 2; l < h; ++l) {
        if (H->presized[l]) continue;
        H->presized[l] = true;
        double e = 0.0;
        for (int m : H->m_s) {
            double comb = 1.0;
            for (int i = 0; i < l; ++i) comb = comb * (double)(m - i) / (double)(i + 1);
            if (m >= l) e += comb;
        }
        const double per_shard = frontier_records_estimate(e, l) * 1.15 / kShards + 64.0;
        if (per_shard * kShards * sizeof(Rec) > 0.5 * (double)frontier_budget(H->dev)) continue;
        const int rc = ensure_frontier(H, l, (u64)per_shard, true);
        if (rc) return rc;
    }
    return MH_OK;
}

// Validates the options, sizes the workspace and fills the device view of a solve.
int prepare_solve(mh_handle *H, const mh_solve_opts *opts, Solve *s, int *max_rounds)
{
    if (!H || !opts) return fail(MH_EINVAL, "handle or opts is NULL");
    const int h = opts->h;
    if (h < 1 || h > kMaxH) return fail(MH_EINVAL, "h=%d outside [1, %d]", h, kMaxH);
    if (opts->alpha.num < 0 || opts->alpha.den <= 0)
        return fail(MH_EINVAL, "alpha=%d/%d: need num >= 0 and den > 0", opts->alpha.num, opts->alpha.den);
    if (opts->prune != MH_PRUNE_PAPER && opts->prune != MH_PRUNE_OFF && opts->prune != MH_PRUNE_BOUND)
        return fail(MH_EINVAL, "prune=%d is not a pruning mode", opts->prune);
    if (opts->mode != MH_MODE_PERSISTENT && opts->mode != MH_MODE_LAUNCHES)
        return fail(MH_EINVAL, "mode=%d is not an execution mode", opts->mode);
    int rc = ensure_workspace(H, h);
    if (rc) return rc;
    if (opts->prune != MH_PRUNE_OFF && (rc = presize_frontiers(H, h))) return rc;
    s->h = h;
    s->prune = opts->prune;
    s->a_num = (u64)opts->alpha.num;
    s->a_den = (u64)opts->alpha.den;
    s->U = H->dU;
    s->state = H->dState;
    s->res = H->dRes;
    s->cnt = H->dCnt;
    s->slots = H->dSlots;
    s->nslots = H->ws_slots;
    s->cand = H->dCand;
    // per-sample champions and sums serve paper pruning only
    const bool paper = opts->prune == MH_PRUNE_PAPER;
    s->champ = paper ? H->dChamp : nullptr;
    s->champ_ok = paper ? H->dChampOk : nullptr;
    s->ssum = paper ? H->dSsum : nullptr;
    s->gk = H->dGK;
    s->cov = H->dCov;
    s->run = H->dCov + H->c.WTp;
    s->cut = H->dCut;
    s->shard = 0;
    s->nshards = 1;
    s->xbest = nullptr;
    s->work = H->dWork;
    s->best_hint = H->dWork + kWorkCount;
    *max_rounds = H->Nt + 1;
    if (opts->max_rounds > 0) *max_rounds = std::min(*max_rounds, (int)opts->max_rounds);
    return MH_OK;
}

Frontiers frontiers_of(const mh_handle *H)
{
    Frontiers f;
    memset(&f, 0, sizeof f);  // padding included: batch items are compared byte by byte
    for (int l = 0; l < kMaxH; ++l) {
        f.F[l] = H->dF[l];
        f.cap[l] = H->cap[l];
        // side arrays of the slots: lb (Key), then sig and lc (u64)
        const size_t n = (size_t)H->cap[l] * kShards;
        unsigned char *side = H->dSide[l];
        f.lb[l] = side ? (Key *)side : nullptr;
        f.sig[l] = side ? (u64 *)(side + n * sizeof(Key)) : nullptr;
        f.lc[l] = side ? (u64 *)(side + n * (sizeof(Key) + sizeof(u64))) : nullptr;
    }
    return f;
}

// Reads a finished solve back into a new mh_result.  kms: the four phase times
// measured by the caller (used unless the persistent kernel measured them).
int collect_result(mh_handle *H, int h, bool persistent, double solve_ms, const double *kms_in,
                   int64_t launches, int64_t leaf_launches, mh_result **out, double kernel_ms = 0.0)
{
    cudaStream_t st = H->stream;
    // the state, selections, counters, cuts and diagnostics (the arrays at their
    // capacity: Nt + 2 rounds) into one pinned buffer, one wait
    const int cap = std::max(1, H->ws_rounds);
    const size_t bState = sizeof(int) * kStateWords;
    const size_t oRes = (bState + 15) & ~(size_t)15;
    const size_t bRes = sizeof(int) * (size_t)cap * (h + 2);
    const size_t bCnt = sizeof(u64) * (size_t)cap * h * 2;
    const size_t bCut = sizeof(u64) * (size_t)cap * h;
    const size_t oCnt = (oRes + bRes + 15) & ~(size_t)15, oCut = oCnt + bCnt, oWork = oCut + bCut;
    const size_t need = oWork + sizeof(u64) * kWorkCount;
    if (H->hRes_bytes < need) {
        pinned_res_put(H->hRes, H->hRes_bytes);
        H->hRes_bytes = 0;
        H->hRes = pinned_res_get(need, &H->hRes_bytes);
        if (!H->hRes) {
            H->hRes_bytes = 0;
            return fail(MH_ENOMEM, "pinned host allocation of the result failed");
        }
    }
    unsigned char *hb = (unsigned char *)H->hRes;
    cudaError_t e = cudaMemcpyAsync(hb, H->dState, bState, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && H->dRes) e = cudaMemcpyAsync(hb + oRes, H->dRes, bRes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && H->dCnt) e = cudaMemcpyAsync(hb + oCnt, H->dCnt, bCnt, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && H->dCut) e = cudaMemcpyAsync(hb + oCut, H->dCut, bCut, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hb + oWork, H->dWork, sizeof(u64) * kWorkCount, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(MH_ECUDA, "reading the result back failed: %s", cudaGetErrorString(e));
    const int *hs = (const int *)hb;
    const int *res = (const int *)(hb + oRes);
    const u64 *cnt = (const u64 *)(hb + oCnt), *cut = (const u64 *)(hb + oCut), *work = (const u64 *)(hb + oWork);
    const int k = hs[0];
    const int rounds = hs[4];
    if (k < 0 || rounds < 0 || rounds > cap || k > cap) return fail(MH_ECUDA, "inconsistent solve state (k=%d, rounds=%d)", k, rounds);
    mh_result *R = (mh_result *)calloc(1, sizeof(mh_result));
    if (!R) return fail(MH_ENOMEM, "host allocation of the result failed");
    R->h = h;
    R->k = k;
    R->rounds = rounds;
    R->genes = (int32_t *)malloc(sizeof(int32_t) * (size_t)std::max(1, k * h));
    R->tp = (int32_t *)malloc(sizeof(int32_t) * (size_t)std::max(1, k));
    R->fp = (int32_t *)malloc(sizeof(int32_t) * (size_t)std::max(1, k));
    R->visited = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)std::max(1, rounds * h));
    R->pruned = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)std::max(1, rounds * h));
    R->cut = (uint64_t *)calloc((size_t)std::max(1, rounds * h), sizeof(uint64_t));
    if (!R->genes || !R->tp || !R->fp || !R->visited || !R->pruned || !R->cut) {
        mh_result_free(R);
        return fail(MH_ENOMEM, "host allocation of the result failed");
    }
    if (rounds) memcpy(R->cut, cut, sizeof(u64) * (size_t)rounds * h);
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j < h; ++j) R->genes[i * h + j] = res[(size_t)i * (h + 2) + j];
        R->tp[i] = res[(size_t)i * (h + 2) + h];
        R->fp[i] = res[(size_t)i * (h + 2) + h + 1];
    }
    for (int i = 0; i < rounds * h; ++i) {
        R->visited[i] = cnt[(size_t)i * 2];
        R->pruned[i] = cnt[(size_t)i * 2 + 1];
    }
    double kms[4];
    for (int i = 0; i < 4; ++i) kms[i] = kms_in ? kms_in[i] : 0.0;
    if (persistent) {  // phase times measured inside the persistent kernel
        for (int i = 0; i < 4; ++i) kms[i] = (double)work[kWorkPhaseNs + i] * 1e-6;
        leaf_launches = h >= 2 ? rounds : 0;
    }
    R->solve_ms = solve_ms;
    R->kernel_ms = persistent ? kernel_ms : (kms_in ? kms[0] + kms[1] + kms[2] + kms[3] : 0.0);
    R->leaf_ms = kms[2];
    R->level1_ms = kms[0];
    R->expand_ms = kms[1];
    R->finalize_ms = kms[3];
    R->leaf_launches = leaf_launches;
    R->mode = persistent ? MH_MODE_PERSISTENT : MH_MODE_LAUNCHES;
    for (int i = 0; i < 2; ++i) {
        R->diag[i] = work[kWorkWarpSum + i];
        R->diag[2 + i] = work[kWorkWarpMaxSum + i];
        R->diag[4 + i] = work[kWorkWarpN + i];
    }
    R->kernel_launches = launches;
    R->leaf_words = work[kWorkColWords];
    R->leaf_prefixes = work[kWorkPrefixes];
    R->leaf_scored = work[kWorkScored];
    R->leaf_alu_ops = work[kWorkAluOps];
    R->leaf_dense = work[kWorkDense];
    *out = R;
    return MH_OK;
}

}  // namespace

extern "C" {

MH_API const char *mh_last_error(void) { return g_last_error.c_str(); }

MH_API int mh_check_bounded_wait(int32_t *status)
{
    if (!status) return fail(MH_EINVAL, "status is NULL");
    *status = MH_OK;
    GridSync *g = nullptr;
    int *state = nullptr;
    MH_CUDA(cudaMalloc((void **)&g, sizeof(GridSync)));
    cudaError_t e = cudaMalloc((void **)&state, sizeof(int) * kStateWords);
    if (e == cudaSuccess) e = cudaMemset(g, 0, sizeof(GridSync));
    if (e == cudaSuccess) e = cudaMemset(state, 0, sizeof(int) * kStateWords);
    if (e == cudaSuccess) e = launch_barrier_probe(g, state, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int hs[kStateWords] = {};
    if (e == cudaSuccess) e = cudaMemcpy(hs, state, sizeof hs, cudaMemcpyDeviceToHost);
    cudaFree(g);
    cudaFree(state);
    if (e != cudaSuccess) return fail(MH_ECUDA, "mh_check_bounded_wait: %s", cudaGetErrorString(e));
    *status = hs[2] == kErrTimeout ? MH_ETIMEOUT : MH_OK;  // state word 2: error
    return MH_OK;
}

MH_API int mh_create(const uint64_t *bitmaps, int32_t G, int32_t Nt, int32_t Nn, mh_handle **out)
{
    if (!out) return fail(MH_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_dims(G, Nt, Nn);
    if (rc) return rc;
    if (!bitmaps) return fail(MH_EINVAL, "bitmaps is NULL");
    return create_common(bitmaps, G, Nt, Nn, nullptr, out);
}

MH_API int mh_create_device(const uint64_t *d_bitmaps, int32_t G, int32_t Nt, int32_t Nn, void *stream,
                            mh_handle **out)
{
    if (!out) return fail(MH_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate_dims(G, Nt, Nn);
    if (rc) return rc;
    if (!d_bitmaps) return fail(MH_EINVAL, "d_bitmaps is NULL");
    const size_t words = (size_t)G * (size_t)((Nt + 63) / 64 + (Nn + 63) / 64);
    std::vector<uint64_t> host(words);
    cudaStream_t st = (cudaStream_t)stream;
    MH_CUDA(cudaMemcpyAsync(host.data(), d_bitmaps, words * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    MH_CUDA(cudaStreamSynchronize(st));
    return create_common(host.data(), G, Nt, Nn, st, out);
}

MH_API int mh_set_stream(mh_handle *H, void *stream)
{
    if (!H) return fail(MH_EINVAL, "handle is NULL");
    H->stream = (cudaStream_t)stream;
    return MH_OK;
}

MH_API int mh_handle_info(const mh_handle *H, int32_t *G, int32_t *Nt, int32_t *Nn, int64_t *device_bytes)
{
    if (!H) return fail(MH_EINVAL, "handle is NULL");
    if (G) *G = H->G;
    if (Nt) *Nt = H->Nt;
    if (Nn) *Nn = H->Nn;
    if (device_bytes) *device_bytes = H->device_bytes;
    return MH_OK;
}

MH_API void mh_destroy(mh_handle *H)
{
    if (!H) return;
    delete H;  // device memory returns to the pool in stream order: no device-wide wait
}

MH_API void mh_result_free(mh_result *r)
{
    if (!r) return;
    free(r->genes);
    free(r->tp);
    free(r->fp);
    free(r->visited);
    free(r->pruned);
    free(r->cut);
    free(r);
}

MH_API int mh_solve(mh_handle *H, int32_t h, mh_rational alpha, mh_result **out)
{
    mh_solve_opts o;
    memset(&o, 0, sizeof o);
    o.h = h;
    o.alpha = alpha;
    return mh_solve_ex(H, &o, out);
}

MH_API int mh_solve_ex(mh_handle *H, const mh_solve_opts *opts, mh_result **out)
{
    if (!out) return fail(MH_EINVAL, "out is NULL");
    *out = nullptr;
    Solve s;
    int max_rounds = 0;
    int rc = prepare_solve(H, opts, &s, &max_rounds);
    if (rc) return rc;
    const int h = opts->h;
    cudaStream_t st = H->stream;
    const Cohort &c = H->c;

    EventPair total;
    MH_CUDA(cudaEventCreate(&total.a));
    MH_CUDA(cudaEventCreate(&total.b));
    // with time_kernels, events around each kernel of a round: level1 | expand | leaf | finalize
    struct RoundEvents {
        cudaEvent_t ev[5];
        bool valid;
    };
    std::vector<RoundEvents> round_ev;
    auto destroy_events = [&]() {
        cudaEventDestroy(total.a);
        cudaEventDestroy(total.b);
        for (auto &e : round_ev)
            for (int i = 0; i < 5; ++i) cudaEventDestroy(e.ev[i]);
    };
    int64_t launches = 0, leaf_launches = 0;
    const int grid = leaf_grid(H);
    u32 *counts = H->dCounts;

    MH_CUDA(cudaEventRecord(total.a, st));
    launch_solve_init(c, s, H->ws_rounds, max_rounds, counts, kCountSets, st);
    ++launches;
    const bool persistent = opts->mode == MH_MODE_PERSISTENT && H->pgrid > 0 && H->pgrid <= H->ws_slots;
    // one block of 16 warps per SM unless MH_PERSISTENT_BUILD=large
    const bool large = use_large_build(H, h);
    const int pgrid = persistent_grid(H->num_sms, large);
    int rounds_done = 0;
    bool done = H->Nt == 0;  // every tumor covered from the start
    double kernel_ms = 0.0;  // the cooperative launches alone
    if (persistent) {
        for (int i = 0; i < 2; ++i)
            if (!H->evk[i]) MH_CUDA(cudaEventCreate(&H->evk[i]));
        // One cooperative launch runs every round; it returns early only when a
        // frontier overflowed (grown here, then the round is run again).
        while (!done) {
            const Frontiers f = frontiers_of(H);
            MH_CUDA(cudaMemsetAsync(H->dSync, 0, sizeof(GridSync), st));
            MH_CUDA(cudaEventRecord(H->evk[0], st));
            MH_CUDA(launch_solve_persistent(c, s, f, H->dSync, counts, pgrid, large, st));
            MH_CUDA(cudaEventRecord(H->evk[1], st));
            ++launches;
            MH_CUDA(cudaMemcpyAsync(H->hState, H->dState, sizeof(int) * kStateWords, cudaMemcpyDeviceToHost, st));
            MH_CUDA(cudaStreamSynchronize(st));
            const int *hs = H->hState;
            const u32 *hc = (const u32 *)(H->hState + kStateWords);
            rounds_done = hs[4];
            float kx = 0.f;
            cudaEventElapsedTime(&kx, H->evk[0], H->evk[1]);
            kernel_ms += kx;
            if (fault_fires(g_fault_timeout)) {
                destroy_events();
                return fail(MH_ETIMEOUT, "injected timeout (mh_set_fault) after round %d", rounds_done);
            }
            if (hs[2]) {
                destroy_events();
                return fail(MH_ETIMEOUT, "a grid barrier of the persistent solve timed out in round %d", rounds_done);
            }
            if (hs[3]) {  // the frontier counters of the overflowed round (its parity's set)
                MH_CUDA(cudaMemcpy(H->hState + kStateWords, counts + (size_t)(rounds_done & 1) * kCountWords,
                                   sizeof(u32) * kCountWords, cudaMemcpyDeviceToHost));
                if ((rc = grow_overflowed(H, h, hc))) {
                    destroy_events();
                    return rc;
                }
                MH_CUDA(cudaMemsetAsync(H->dCnt + (size_t)rounds_done * h * 2, 0, sizeof(u64) * 2 * h, st));
                MH_CUDA(cudaMemsetAsync(H->dCut + (size_t)rounds_done * h, 0, sizeof(u64) * h, st));
                MH_CUDA(cudaMemsetAsync(counts, 0, sizeof(u32) * kCountSets * kCountWords, st));
                MH_CUDA(cudaMemsetAsync(H->dState + 3, 0, sizeof(int), st));
                continue;
            }
            done = true;
        }
    }
    // Rounds are enqueued in growing batches without waiting: every kernel reads
    // the round index and the done / overflow flags on the device.  After a batch
    // the host reads the state; an overflowed frontier is grown and its round rerun.
    int batch = 4;
    Frontiers fl;
    s.champ = nullptr;  // the per-sample champions are computed by the persistent kernels only
    s.champ_ok = nullptr;
    while (!done) {
        fl = frontiers_of(H);
        const size_t first_ev = round_ev.size();
        const int n = std::min(batch, max_rounds - rounds_done);
        for (int b = 0; b < n; ++b) {
            RoundEvents e{};
            if (opts->time_kernels) {
                for (int i = 0; i < 5; ++i) MH_CUDA(cudaEventCreate(&e.ev[i]));
                e.valid = true;
                MH_CUDA(cudaEventRecord(e.ev[0], st));
            }
            launch_level1(c, s, fl, counts, st);
            ++launches;
            if (opts->time_kernels) MH_CUDA(cudaEventRecord(e.ev[1], st));
            for (int l = 2; l <= h - 1; ++l) {
                launch_expand(c, s, l, fl, counts, grid, st);
                ++launches;
            }
            if (opts->time_kernels) MH_CUDA(cudaEventRecord(e.ev[2], st));
            if (h >= 2) {
                launch_leaf(c, s, fl, counts, grid, st);
                ++launches;
                ++leaf_launches;
            }
            if (opts->time_kernels) MH_CUDA(cudaEventRecord(e.ev[3], st));
            launch_finalize(c, s, counts, st);
            ++launches;
            if (opts->time_kernels) {
                MH_CUDA(cudaEventRecord(e.ev[4], st));
                round_ev.push_back(e);
            }
        }
        MH_CUDA(cudaGetLastError());
        MH_CUDA(cudaMemcpyAsync(H->hState, H->dState, sizeof(int) * kStateWords, cudaMemcpyDeviceToHost, st));
        MH_CUDA(cudaMemcpyAsync(H->hState + kStateWords, counts, sizeof(u32) * kCountWords, cudaMemcpyDeviceToHost,
                                st));
        MH_CUDA(cudaStreamSynchronize(st));
        const int *hs = H->hState;
        const u32 *hc = (const u32 *)(H->hState + kStateWords);
        rounds_done = hs[4];
        if (hs[3]) {
            // a frontier of round rounds_done did not fit: grow it, forget the round's
            // partial counters and frontier sizes, and run the round again
            for (size_t e = first_ev; e < round_ev.size(); ++e) round_ev[e].valid = false;
            if ((rc = grow_overflowed(H, h, hc))) {
                destroy_events();
                return rc;
            }
            MH_CUDA(cudaMemsetAsync(H->dCnt + (size_t)rounds_done * h * 2, 0, sizeof(u64) * 2 * h, st));
                MH_CUDA(cudaMemsetAsync(H->dCut + (size_t)rounds_done * h, 0, sizeof(u64) * h, st));
            MH_CUDA(cudaMemsetAsync(counts, 0, sizeof(u32) * kCountSets * kCountWords, st));
            MH_CUDA(cudaMemsetAsync(H->dState + 3, 0, sizeof(int), st));
            continue;
        }
        done = hs[1] != 0 || rounds_done >= max_rounds;
        batch = std::min(batch * 2, 64);
    }
    MH_CUDA(cudaEventRecord(total.b, st));
    MH_CUDA(cudaStreamSynchronize(st));
    int rounds = 0;
    MH_CUDA(cudaMemcpy(&rounds, H->dState + 4, sizeof(int), cudaMemcpyDeviceToHost));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, total.a, total.b);
    // kernel times of the rounds that ran (launches after the last round return at once)
    double kms[4] = {0, 0, 0, 0};
    int64_t timed = 0;
    for (auto &ev : round_ev) {
        if (!ev.valid || timed >= rounds) continue;
        for (int i = 0; i < 4; ++i) {
            float x = 0.f;
            cudaEventElapsedTime(&x, ev.ev[i], ev.ev[i + 1]);
            kms[i] += x;
        }
        ++timed;
    }
    destroy_events();
    const int64_t ll = opts->time_kernels && !persistent ? (h >= 2 ? timed : 0) : leaf_launches;
    return collect_result(H, h, persistent, ms, kms, launches, ll, out, kernel_ms);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched solve and its autotuner.

namespace {

// Expected search work of a cohort: the gene sets of size d that share a tumor,
// summed over tumors (d = h - 1: the prefixes the leaves hang from; d = h: the
// non-empty leaves), plus the depth-1 scan.
double work_estimate(const mh_handle *H, int d)
{
    double w = (double)H->G;
    for (int m : H->m_s) {
        double comb = 1.0;
        for (int i = 0; i < d; ++i) comb = comb * (double)(m - i) / (double)(i + 1);
        if (m >= d) w += comb;
    }
    return w;
}

// Blocks per cohort: proportional to work^gamma, at least one each, summing to grid.
std::vector<int> split_blocks(const std::vector<double> &work, double gamma, int grid)
{
    const int n = (int)work.size();
    std::vector<double> wt(n);
    double tot = 0;
    for (int i = 0; i < n; ++i) tot += wt[i] = std::pow(std::max(work[i], 1.0), gamma);
    std::vector<int> b(n, 1);
    int left = grid - n;
    std::vector<std::pair<double, int>> frac;
    for (int i = 0; i < n; ++i) {
        const double want = wt[i] / tot * (double)(grid - n);
        const int whole = (int)want;
        b[i] += whole;
        left -= whole;
        frac.push_back({want - whole, i});
    }
    std::sort(frac.begin(), frac.end(), [](auto &a, auto &c) { return a.first > c.first; });
    for (int i = 0; i < n && left > 0; ++i, --left) ++b[frac[i].second];
    return b;
}

std::mutex g_tune_mutex;
std::map<std::string, double> g_tune;  // batch signature -> chosen model (10 * d_extra + gamma)
bool g_tune_loaded = false;

std::string tune_path()
{
    const char *p = getenv("MH_AUTOTUNE_CACHE");
    if (p && *p) return p;
    const char *home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/mh_autotune.txt";
}

// Bucketed shape of a batch: the sorted (h, log2 G, log2 Nt) of its cohorts.
std::string batch_signature(mh_handle *const *hs, const mh_solve_opts *opts, int n, int grid)
{
    std::vector<std::string> parts;
    for (int i = 0; i < n; ++i) {
        std::ostringstream o;
        o << opts[i].h << ":" << (int)std::lround(std::log2((double)hs[i]->G)) << ":"
          << (int)std::lround(std::log2((double)std::max(1, hs[i]->Nt)));
        parts.push_back(o.str());
    }
    std::sort(parts.begin(), parts.end());
    std::ostringstream o;
    o << "grid" << grid;
    for (auto &p : parts) o << "," << p;
    return o.str();
}

bool tune_lookup(const std::string &sig, double *gamma)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (!g_tune_loaded) {
        g_tune_loaded = true;
        std::ifstream in(tune_path());
        std::string key;
        double g;
        while (in >> key >> g) g_tune[key] = g;
    }
    auto it = g_tune.find(sig);
    if (it == g_tune.end()) return false;
    *gamma = it->second;
    return true;
}

void tune_store(const std::string &sig, double gamma)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[sig] = gamma;
    const std::string path = tune_path();
    const size_t slash = path.find_last_of('/');
    if (slash != std::string::npos) {
        const std::string dir = path.substr(0, slash);
        std::string cmd;  // best effort: the cache is an optimisation only
        (void)cmd;
        mkdir(dir.c_str(), 0755);
    }
    std::ofstream out(path, std::ios::trunc);
    for (auto &kv : g_tune) out << kv.first << " " << kv.second << "\n";
}

// Device copy of the batch descriptors (grown on demand, shared by all calls),
// followed by the yield flag, the block-numbering table and the start barrier.
std::mutex g_items_mutex;
BatchItem *g_items = nullptr;
int g_items_cap = 0;

size_t batch_ws_bytes(int n)
{
    return sizeof(BatchItem) * (size_t)n + 256 + sizeof(int) * kBatchTabInts + sizeof(GridSync);
}

BatchMap batch_map_at(BatchItem *items, int cap, int num_sms, int build)
{
    char *base = (char *)items + sizeof(BatchItem) * (size_t)cap + 256;
    return BatchMap{(int *)base, (GridSync *)(base + sizeof(int) * kBatchTabInts), batch_blocks_per_sm(build), num_sms,
                    build};
}

// Blocks per cohort of a batched launch: whole SMs (blocks ~ work^gamma rounded to
// the blocks one SM holds) when there are no more cohorts than SMs.
std::vector<int> split_grid(const std::vector<double> &work, double gamma, int num_sms, int build)
{
    const int per_sm = batch_blocks_per_sm(build);
    if ((int)work.size() > num_sms) return split_blocks(work, gamma, per_sm * num_sms);
    std::vector<int> b = split_blocks(work, gamma, num_sms);
    for (int &x : b) x *= per_sm;
    return b;
}

// One batched run: all cohorts start from "nothing covered"; the grid is split
// between the unfinished cohorts (blocks ~ work^gamma, or the fixed split) and,
// each time a cohort finishes, the launch ends and the remaining cohorts share
// the whole grid again.  *ms receives the run's time (CUDA events).
// The start of a batched solve -- every cohort's round-state initialisation and the
// first cooperative launch over all of them -- is captured into a CUDA graph once
// per launch signature (the items' bytes, which hold every device pointer and size,
// the round limits, the stream and the launch buffers) and replayed when the same
// cohorts are solved again, so a repeated batch costs one graph launch instead of
// some 10 API calls per cohort.  Streams that cannot be captured (the legacy
// default stream, or one already capturing) take the direct launches.
struct StartGraph {
    std::vector<char> key;
    cudaGraphExec_t exec = nullptr;
    BatchItem *h_items = nullptr;  // pinned copy of the items the graph uploads
    int h_cap = 0;
};
StartGraph g_start;  // guarded by g_items_mutex

bool capturable(cudaStream_t st)
{
    if (st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

int run_batch(mh_handle *const *hs, const mh_solve_opts *opts, int n, const std::vector<double> &work, double gamma,
              int build, const std::vector<int> *fixed, double *ms, int *sm_major = nullptr, int *graphed = nullptr,
              bool graph_ok = true)
{
    if (sm_major) *sm_major = 1;
    if (graphed) *graphed = 0;
    cudaStream_t st = hs[0]->stream;
    std::vector<Solve> ss(n);
    std::vector<int> maxr(n);
    for (int i = 0; i < n; ++i) {
        int rc = prepare_solve(hs[i], &opts[i], &ss[i], &maxr[i]);
        if (rc) return rc;
    }
    cudaEvent_t a, b;
    MH_CUDA(cudaEventCreate(&a));
    MH_CUDA(cudaEventCreate(&b));
    MH_CUDA(cudaEventRecord(a, st));
    // every cohort's round state starts from scratch: issued with the first launch
    bool init_pending = true;
    auto issue_init = [&]() {
        for (int i = 0; i < n; ++i)
            launch_solve_init(hs[i]->c, ss[i], hs[i]->ws_rounds, maxr[i], hs[i]->dCounts, kCountSets, st);
    };
    std::lock_guard<std::mutex> lock(g_items_mutex);
    if (g_items_cap < n) {
        cudaFree(g_items);
        g_items = nullptr;
        g_items_cap = 0;
        MH_CUDA(cudaMalloc((void **)&g_items, batch_ws_bytes(n)));
        g_items_cap = n;
    }
    int *d_yield = (int *)((char *)g_items + sizeof(BatchItem) * (size_t)g_items_cap);
    const BatchMap map = batch_map_at(g_items, g_items_cap, hs[0]->num_sms, build);
    std::vector<char> finished(n, 0);
    for (int i = 0; i < n; ++i) finished[i] = hs[i]->Nt == 0;
    for (;;) {
        std::vector<int> act;
        for (int i = 0; i < n; ++i)
            if (!finished[i]) act.push_back(i);
        if (act.empty()) break;
        std::vector<int> blocks;
        if (fixed) {
            for (int i : act) blocks.push_back((*fixed)[i]);
        } else {
            std::vector<double> w;
            for (int i : act) w.push_back(work[i]);
            blocks = split_grid(w, gamma, hs[0]->num_sms, build);
        }
        std::vector<BatchItem> items(act.size());
        memset(items.data(), 0, sizeof(BatchItem) * items.size());  // padding too: the bytes are a graph key
        int first = 0;
        for (size_t k = 0; k < act.size(); ++k) {
            const int i = act[k];
            items[k].c = hs[i]->c;
            items[k].s = ss[i];
            items[k].f = frontiers_of(hs[i]);
            items[k].gsync = hs[i]->dSync;
            items[k].counts = hs[i]->dCounts;
            items[k].first_block = first;
            items[k].nblocks = blocks[k];
            first += blocks[k];
        }
        auto issue_prep = [&]() {
            for (int i : act) {
                cudaMemsetAsync(hs[i]->dSync, 0, sizeof(GridSync), st);
                cudaMemsetAsync(hs[i]->dState + 6, 0, sizeof(int), st);  // yield request
            }
            return cudaMemsetAsync(d_yield, 0, sizeof(int), st);
        };
        // the start of the solve from a captured graph (see StartGraph)
        bool started = false;
        if (graph_ok && init_pending && act.size() > 1 && capturable(st)) {
            std::vector<char> key(sizeof(BatchItem) * items.size());
            memcpy(key.data(), items.data(), key.size());
            auto put = [&](const void *p, size_t bytes) {
                key.insert(key.end(), (const char *)p, (const char *)p + bytes);
            };
            for (int i = 0; i < n; ++i) {
                put(&hs[i]->ws_rounds, sizeof(int));
                put(&maxr[i], sizeof(int));
            }
            put(&st, sizeof st);
            put(&g_items, sizeof g_items);
            put(&map, sizeof map);
            if (g_start.exec && g_start.key == key) {
                started = cudaGraphLaunch(g_start.exec, st) == cudaSuccess;
            } else {
                if (g_start.h_cap < (int)items.size()) {
                    if (g_start.h_items) cudaFreeHost(g_start.h_items);
                    g_start.h_items = nullptr;
                    g_start.h_cap = 0;
                    if (cudaMallocHost((void **)&g_start.h_items, sizeof(BatchItem) * items.size()) == cudaSuccess)
                        g_start.h_cap = (int)items.size();
                }
                cudaGraph_t g = nullptr;
                if (g_start.h_cap >= (int)items.size() &&
                    cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                    memcpy(g_start.h_items, items.data(), sizeof(BatchItem) * items.size());
                    issue_init();
                    issue_prep();
                    cudaMemcpyAsync(g_items, g_start.h_items, sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                                    st);
                    launch_solve_batch(g_items, (int)items.size(), d_yield, map, st);
                    cudaGraphExec_t ex = nullptr;
                    if (cudaStreamEndCapture(st, &g) == cudaSuccess && g &&
                        cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                        if (g_start.exec) cudaGraphExecDestroy(g_start.exec);
                        g_start.exec = ex;
                        g_start.key.swap(key);
                        started = cudaGraphLaunch(ex, st) == cudaSuccess;
                    }
                    if (g) cudaGraphDestroy(g);
                }
                cudaGetLastError();  // a stream that could not be captured: launch directly
            }
            if (started && graphed) *graphed = 1;
        }
        if (init_pending && !started) issue_init();
        init_pending = false;
        if (!started) MH_CUDA(issue_prep());
        if (started) {
            MH_CUDA(cudaStreamSynchronize(st));
            int fell_back = 0;
            MH_CUDA(cudaMemcpy(&fell_back, map.tab + 2 * kMaxSmid + 1, sizeof(int), cudaMemcpyDeviceToHost));
            if (fell_back && sm_major) *sm_major = 0;
        } else if (act.size() == 1 && !fixed) {
            // one cohort left: the single-cohort persistent kernel (its fields are kernel
            // parameters, which the compiler keeps out of registers)
            mh_handle *H = hs[act[0]];
            const bool large = use_large_build(H, opts[act[0]].h);
            MH_CUDA(launch_solve_persistent(H->c, ss[act[0]], frontiers_of(H), H->dSync, H->dCounts,
                                            persistent_grid(H->num_sms, large), large, st));
            MH_CUDA(cudaStreamSynchronize(st));
        } else {
            MH_CUDA(cudaMemcpyAsync(g_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice,
                                    st));
            MH_CUDA(launch_solve_batch(g_items, (int)items.size(), act.size() > 1 ? d_yield : nullptr, map, st));
            MH_CUDA(cudaStreamSynchronize(st));
            int fell_back = 0;  // the launch numbered its blocks by blockIdx.x
            MH_CUDA(cudaMemcpy(&fell_back, map.tab + 2 * kMaxSmid + 1, sizeof(int), cudaMemcpyDeviceToHost));
            if (fell_back && sm_major) *sm_major = 0;
        }
        for (int i : act) {
            mh_handle *H = hs[i];
            MH_CUDA(cudaMemcpy(H->hState, H->dState, sizeof(int) * kStateWords, cudaMemcpyDeviceToHost));
            if (H->hState[2]) return fail(MH_ETIMEOUT, "a team barrier of the batched solve timed out");
            if (H->hState[3]) {
                const int r = H->hState[4];
                MH_CUDA(cudaMemcpy(H->hState + kStateWords, H->dCounts + (size_t)(r & 1) * kCountWords,
                                   sizeof(u32) * kCountWords, cudaMemcpyDeviceToHost));
                int rc = grow_overflowed(H, opts[i].h, (const u32 *)(H->hState + kStateWords));
                if (rc) return rc;
                MH_CUDA(cudaMemsetAsync(H->dCnt + (size_t)r * opts[i].h * 2, 0, sizeof(u64) * 2 * opts[i].h, st));
                MH_CUDA(cudaMemsetAsync(H->dCut + (size_t)r * opts[i].h, 0, sizeof(u64) * opts[i].h, st));
                MH_CUDA(cudaMemsetAsync(H->dCounts, 0, sizeof(u32) * kCountSets * kCountWords, st));
                MH_CUDA(cudaMemsetAsync(H->dState + 3, 0, sizeof(int), st));
            }
            finished[i] = H->hState[1] != 0;
        }
    }
    MH_CUDA(cudaEventRecord(b, st));
    MH_CUDA(cudaEventSynchronize(b));
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = t;
    return MH_OK;
}

// The cohorts one after another, each solved by the single-cohort persistent kernel
// over the whole grid: every cohort's round-state initialisation and launch are
// queued back to back on the stream and the host synchronises once for the batch.
// A cohort whose frontier overflowed is grown and solved again on its own.
// *ms receives the batch's time (CUDA events).
constexpr double kInTurn = 1000.0;  // the autotuner's code for this schedule
int run_in_turn(mh_handle *const *hs, const mh_solve_opts *opts, int n, double *ms)
{
    cudaStream_t st = hs[0]->stream;
    std::vector<Solve> ss(n);
    std::vector<int> maxr(n);
    for (int i = 0; i < n; ++i) {
        int rc = prepare_solve(hs[i], &opts[i], &ss[i], &maxr[i]);
        if (rc) return rc;
    }
    cudaEvent_t a, b;
    MH_CUDA(cudaEventCreate(&a));
    MH_CUDA(cudaEventCreate(&b));
    MH_CUDA(cudaEventRecord(a, st));
    for (int i = 0; i < n; ++i) {
        mh_handle *H = hs[i];
        launch_solve_init(H->c, ss[i], H->ws_rounds, maxr[i], H->dCounts, kCountSets, st);
        if (H->Nt == 0) continue;
        MH_CUDA(cudaMemsetAsync(H->dSync, 0, sizeof(GridSync), st));
        const bool large = use_large_build(H, opts[i].h);
        MH_CUDA(launch_solve_persistent(H->c, ss[i], frontiers_of(H), H->dSync, H->dCounts,
                                        persistent_grid(H->num_sms, large), large, st));
    }
    MH_CUDA(cudaEventRecord(b, st));
    MH_CUDA(cudaEventSynchronize(b));
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    double total = t;
    for (int i = 0; i < n; ++i) {
        mh_handle *H = hs[i];
        MH_CUDA(cudaMemcpy(H->hState, H->dState, sizeof(int) * kStateWords, cudaMemcpyDeviceToHost));
        if (H->hState[2]) return fail(MH_ETIMEOUT, "a grid barrier of the batched solve timed out");
        if (H->hState[3]) {  // overflowed: grown and solved again from the start
            const int r = H->hState[4];
            MH_CUDA(cudaMemcpy(H->hState + kStateWords, H->dCounts + (size_t)(r & 1) * kCountWords,
                               sizeof(u32) * kCountWords, cudaMemcpyDeviceToHost));
            int rc = grow_overflowed(H, opts[i].h, (const u32 *)(H->hState + kStateWords));
            if (rc) return rc;
            MH_CUDA(cudaMemsetAsync(H->dCounts, 0, sizeof(u32) * kCountSets * kCountWords, st));
            std::vector<double> w(1, 1.0);
            double t1 = 0.0;
            rc = run_batch(&hs[i], &opts[i], 1, w, 1.0, kBatchBuilds[0], nullptr, &t1);
            if (rc) return rc;
            total += t1;
        }
    }
    *ms = total;
    return MH_OK;
}

// Groups of k cohorts of similar work (largest first), one group after another; the
// cohorts of a group run concurrently on a split of the grid (blocks ~ work, whole
// SMs, the one-block-per-SM build).  Between the in-turn schedule (k = 1) and the
// whole batch at once.  *ms receives the sum of the groups' times.
constexpr double kGroups = 2000.0;  // the autotuner's code for this schedule is kGroups + k
int run_groups(mh_handle *const *hs, const mh_solve_opts *opts, int n, const std::vector<double> &work, int k,
               double *ms)
{
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return work[a] > work[b]; });
    double total = 0.0;
    for (int g0 = 0; g0 < n; g0 += k) {
        const int m = std::min(k, n - g0);
        std::vector<mh_handle *> gh(m);
        std::vector<mh_solve_opts> go(m);
        std::vector<double> gw(m);
        for (int i = 0; i < m; ++i) {
            gh[i] = hs[idx[g0 + i]];
            go[i] = opts[idx[g0 + i]];
            gw[i] = work[idx[g0 + i]];
        }
        double t = 0.0;
        const int rc = m == 1 ? run_in_turn(gh.data(), go.data(), 1, &t)
                              : run_batch(gh.data(), go.data(), m, gw, 1.0, kBatchBuilds[0], nullptr, &t, nullptr,
                                          nullptr, false);
        if (rc) return rc;
        total += t;
    }
    *ms = total;
    return MH_OK;
}

}  // namespace

extern "C" MH_API int mh_solve_batch(mh_handle *const *handles, const mh_solve_opts *opts, int32_t n,
                                     const int32_t *blocks, mh_result **out)
{
    if (!handles || !opts || !out || n < 1) return fail(MH_EINVAL, "mh_solve_batch: NULL argument or n < 1");
    for (int i = 0; i < n; ++i) {
        out[i] = nullptr;
        if (!handles[i]) return fail(MH_EINVAL, "mh_solve_batch: handle %d is NULL", i);
        for (int j = 0; j < i; ++j)
            if (handles[j] == handles[i]) return fail(MH_EINVAL, "mh_solve_batch: handle %d appears twice", i);
    }
    mh_handle *H0 = handles[0];
    if (!H0->coop) return fail(MH_ECUDA, "mh_solve_batch: the device has no cooperative launch");
    for (int i = 0; i < n; ++i) {  // every handle sizes its workspace (and slot array) now
        Solve tmp;
        int mr;
        int rc = prepare_solve(handles[i], &opts[i], &tmp, &mr);
        if (rc) return rc;
    }
    const int grid = batch_grid(H0->num_sms, 3);  // the smaller of the two builds' grids
    if (grid < n) return fail(MH_EINVAL, "mh_solve_batch: %d cohorts but only %d co-resident blocks", n, grid);
    std::vector<int> b(n);
    if (blocks) {
        long long tot = 0;
        for (int i = 0; i < n; ++i) {
            if (blocks[i] < 1) return fail(MH_EINVAL, "mh_solve_batch: blocks[%d] = %d < 1", i, blocks[i]);
            b[i] = blocks[i];
            tot += blocks[i];
        }
        if (tot > grid) return fail(MH_EINVAL, "mh_solve_batch: %lld blocks requested, %d co-resident", tot, grid);
    }
    // two work models: prefixes (d = h - 1) or leaves (d = h) sharing a tumor
    std::vector<double> work_p(n), work_l(n);
    for (int i = 0; i < n; ++i) {
        work_p[i] = work_estimate(handles[i], opts[i].h - 1);
        work_l[i] = work_estimate(handles[i], opts[i].h);
    }
    double ms = 0.0;
    int rc = MH_OK, smm = 0, graphed = 0;
    // a choice of the autotuner, encoded as 100 * (build == 4) + 10 * model + gamma
    auto run_choice = [&](double choice, double *t, int *smm_out) {
        if (choice >= kGroups) {  // groups of k cohorts, one group after another
            if (smm_out) *smm_out = 1;
            return run_groups(handles, opts, n, work_p, (int)(choice - kGroups), t);
        }
        if (choice >= kInTurn) {  // one cohort after another over the whole grid
            if (smm_out) *smm_out = 1;
            return run_in_turn(handles, opts, n, t);
        }
        // choice = 100 * (index of the build in kBatchBuilds) + 10 * model + gamma
        const int bi = std::min(2, std::max(0, (int)(choice / 100.0)));
        const int build = kBatchBuilds[bi];
        choice -= 100.0 * bi;
        const bool leaves = choice >= 10.0;
        return run_batch(handles, opts, n, leaves ? work_l : work_p, choice - (leaves ? 10.0 : 0.0), build, nullptr,
                         t, smm_out, smm_out ? &graphed : nullptr);
    };
    if (blocks) {
        rc = run_batch(handles, opts, n, work_p, 1.0, 3, &b, &ms, &smm, &graphed);
    } else {
        // autotuner: the cohorts in turn over the whole grid, or concurrently on a split
        // of it -- the kernel build (1, 3 or 4 blocks per SM), the work model and the
        // split exponent gamma (blocks ~ work^gamma) -- chosen by timing each candidate
        // once per batch shape; the choice is cached on disk
        const std::string sig = batch_signature(handles, opts, n, grid);
        double choice = 1.0;
        const char *off = getenv("MH_AUTOTUNE");
        const char *forced = getenv("MH_BATCH_CHOICE");  // a schedule code, bypassing the tuner
        if (forced && *forced) {
            choice = atof(forced);
            rc = run_choice(choice, &ms, &smm);
        } else if ((off && off[0] == '0') || tune_lookup(sig, &choice)) {
            rc = run_choice(choice, &ms, &smm);
        } else {
            const double gammas[] = {0.5, 0.75, 1.0, 1.5, 2.0};
            double best_ms = 1e300, best = 1.0;
            {  // the cohorts in turn, each over the whole grid
                double t = 0.0;
                rc = run_choice(kInTurn, &t, nullptr);
                if (rc) return rc;
                best_ms = t;
                best = kInTurn;
            }
            for (int k : {2, 4}) {  // groups of k cohorts, one group after another
                if (k >= n) break;
                double t = 0.0;
                rc = run_choice(kGroups + k, &t, nullptr);
                if (rc) return rc;
                if (t < best_ms) {
                    best_ms = t;
                    best = kGroups + k;
                }
            }
            for (int bi = 0; bi < 3; ++bi) {
                if (batch_grid(H0->num_sms, kBatchBuilds[bi]) < n) continue;  // a block per cohort at least
                for (int model = 0; model < 2; ++model) {
                    for (double g : gammas) {
                        double t = 0.0;
                        const double cand = 100.0 * bi + 10.0 * model + g;
                        rc = run_choice(cand, &t, nullptr);
                        if (rc) return rc;
                        if (t < best_ms) {
                            best_ms = t;
                            best = cand;
                        }
                    }
                }
            }
            tune_store(sig, best);
            rc = run_choice(best, &ms, &smm);
        }
    }
    if (rc) return rc;
    for (int i = 0; i < n; ++i) {
        rc = collect_result(handles[i], opts[i].h, true, ms, nullptr, 1, 0, &out[i], ms);
        if (rc == MH_OK) {
            out[i]->diag[6] = (uint64_t)smm;
            out[i]->diag[7] = (uint64_t)graphed;
        }
        if (rc) {
            for (int j = 0; j < i; ++j) {
                mh_result_free(out[j]);
                out[j] = nullptr;
            }
            return rc;
        }
    }
    return MH_OK;
}

// ---------------------------------------------------------------------------
// Served runtime: continuous batching of greedy solves.
//
// A scheduler thread keeps a set of active requests, each solved by a team of
// blocks of one cooperative launch of the batched kernel.  The launch ends at the
// next round boundary whenever an active request finishes, or when the scheduler
// raises the yield flag (host memory mapped into the device) because a new request
// is waiting for a free slot; between launches the scheduler retires finished
// requests, admits queued ones within the memory budget (uploading their cohorts),
// and relaunches with the grid split between the active requests again.

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerReq {
    uint64_t ticket = 0;
    std::vector<uint64_t> bm;
    int G = 0, Nt = 0, Nn = 0;
    mh_solve_opts opts{};
    double t_submit = 0, t_done = 0;
    int64_t footprint = 0;
    mh_handle *H = nullptr;
    int status = -1;  // -1 pending, MH_OK done, else the error
    std::string msg;
    mh_result *res = nullptr;
    Solve s{};
    int maxr = 0;
    double work = 0.0;   // expected search work (work_estimate with d = h - 1)
    bool large = false;  // work above kLargeWork
    bool cancel = false; // mh_cancel on an admitted request: retired at the next round boundary
    double t_ran = 0.0;  // last launch that included it (its admission before the first)
    cudaEvent_t built = nullptr;  // end of its store build on the upload stream
};

// Device memory a request needs: its store, workspace and (for h >= 3) the
// frontiers, estimated from the l-gene sets that share a tumor
// (frontier_records_estimate).
int64_t estimate_footprint(const uint64_t *bm, int G, int Nt, int Nn, int h, double *work)
{
    const int Wt = (Nt + 63) / 64, Wn = (Nn + 63) / 64;
    std::vector<int> m(Nt, 0);
    for (int g = 0; g < G; ++g)
        for (int w = 0; w < Wt; ++w)
            for (uint64_t x = bm[(size_t)g * (Wt + Wn) + w]; x; x &= x - 1) ++m[w * 64 + __builtin_ctzll(x)];
    const int64_t gw = ((G + 63) / 64 + 2);
    int64_t bytes = (int64_t)G * (Wt + Wn + 4) * 8 + (int64_t)(Nt + Nn) * gw * 8 + (int64_t)G * (sizeof(Rec) + 12);
    bytes += (int64_t)((G + kShards - 1) / kShards + 64) * kShards * (int64_t)kSlotBytes;
    // sets[d]: the d-gene sets sharing a tumor, summed over tumors
    std::vector<double> sets(std::max(h, 1), 0.0);
    for (int x : m) {
        double comb = 1.0;
        for (int d = 0; d < h; ++d) {
            if (x >= d) sets[d] += comb;
            comb = comb * (double)(x - d) / (double)(d + 1);
        }
    }
    for (int l = 2; l < h; ++l)
        bytes += (int64_t)(frontier_records_estimate(sets[l], l) * 1.25 * (double)kSlotBytes) +
                 (int64_t)(2048 * kShards) * (int64_t)kSlotBytes;
    *work = (double)G + sets[h - 1];  // as work_estimate(H, h - 1)
    return bytes + (64 << 20);
}

}  // namespace

// The batched kernel's build used by the server (four blocks per SM: the faster one
// on a stream of large requests with small ones backfilling).
constexpr int kServerBuild = 1;  // one block of 16 warps per SM: teams of whole SMs

struct mh_server {
    mh_server_opts o{};
    cudaStream_t st = nullptr, st_up = nullptr;  // launches; uploads
    int grid = 0, num_sms = 0;
    int64_t budget = 0, in_use = 0;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<ServerReq *> queue;
    std::vector<ServerReq *> active;
    std::vector<ServerReq *> ready;  // uploaded, joining at the next launch (scheduler thread only)
    std::map<uint64_t, ServerReq *> all;
    bool stop = false;
    uint64_t next_ticket = 1;
    int *h_yield = nullptr, *d_yield = nullptr;
    BatchItem *d_items = nullptr;
    int items_cap = 0;
    int64_t launches = 0;

    void finish(ServerReq *r, int status, const char *msg)
    {
        r->status = status;
        if (msg) r->msg = msg;
        r->t_done = now_s();
        if (r->res) r->res->solve_ms = (r->t_done - r->t_submit) * 1e3;
    }

    // Admission of the queue head when a slot and memory are free: the cohort's
    // rows are uploaded and its store is built on the upload stream without the
    // host waiting (the build's kernels find SMs when the running launch ends at its
    // next round boundary, which the admission asks for); the next launch waits for
    // the build on the device.  The admitted request waits in `ready` for that
    // launch.  Returns true if the head was taken (admitted, or finished with an error).
    bool admit_one()
    {
        ServerReq *r = nullptr;
        {
            std::lock_guard<std::mutex> lock(mu);
            if (queue.empty() || (int)(active.size() + ready.size()) >= o.slots) return false;
            int large = 0;
            for (ServerReq *a : active) large += a->large;
            for (ServerReq *a : ready) large += a->large;
            // the first request in arrival order that may start: a large one waits
            // while large_slots are taken and the smaller ones behind it go first
            auto it = queue.begin();
            while (it != queue.end() && (*it)->large && large >= o.large_slots && (*it)->footprint <= budget) ++it;
            if (it == queue.end()) return false;
            r = *it;
            if (r->footprint > budget) {
                queue.erase(it);
                finish(r, MH_EREJECT, "request needs more device memory than the server budget");
                cv.notify_all();
                return true;
            }
            if (in_use + r->footprint > budget && !(active.empty() && ready.empty())) return false;
            queue.erase(it);
            in_use += r->footprint;
        }
        int rc = create_common(r->bm.data(), r->G, r->Nt, r->Nn, st_up, &r->H, false);
        int maxr = 0;
        if (rc == MH_OK) rc = prepare_solve(r->H, &r->opts, &r->s, &maxr);
        if (rc == MH_OK && (cudaEventCreateWithFlags(&r->built, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventRecord(r->built, st_up) != cudaSuccess))
            rc = fail(MH_ECUDA, "upload failed");
        std::lock_guard<std::mutex> lock(mu);
        if (rc != MH_OK) {
            if (r->built) cudaStreamSynchronize(st_up);  // nothing of it left in flight
            if (r->built) cudaEventDestroy(r->built);
            r->built = nullptr;
            if (r->H) mh_destroy(r->H);
            r->H = nullptr;
            in_use -= r->footprint;
            finish(r, rc, mh_last_error());
            cv.notify_all();
            return true;
        }
        r->H->stream = st;  // from now on ordered with the launches
        r->maxr = maxr;
        r->bm.clear();
        r->bm.shrink_to_fit();
        ready.push_back(r);
        return true;
    }

    // Ready requests join the active set: their round state is initialised on the
    // launch stream, ahead of the next launch.
    void start_ready()
    {
        {
            std::lock_guard<std::mutex> lock(mu);
            std::vector<ServerReq *> keep;
            for (ServerReq *r : ready) {
                if (!r->cancel) {
                    keep.push_back(r);
                    continue;
                }
                if (r->built) {
                    cudaEventSynchronize(r->built);
                    cudaEventDestroy(r->built);
                    r->built = nullptr;
                }
                mh_destroy(r->H);
                r->H = nullptr;
                in_use -= r->footprint;
                finish(r, MH_ECANCELED, "cancelled before it started");
            }
            ready.swap(keep);
            cv.notify_all();
        }
        const double t0 = now_s();
        for (ServerReq *r : ready) {
            r->t_ran = t0;
            if (r->built) {  // its store, built on the upload stream
                cudaStreamWaitEvent(st, r->built, 0);
                cudaEventDestroy(r->built);
                r->built = nullptr;
            }
            launch_solve_init(r->H->c, r->s, r->H->ws_rounds, r->maxr, r->H->dCounts, kCountSets, st);
            if (r->Nt == 0) {
                const int one = 1;
                cudaMemcpyAsync(r->H->dState + 1, &one, sizeof(int), cudaMemcpyHostToDevice, st);
            }
        }
        std::lock_guard<std::mutex> lock(mu);
        active.insert(active.end(), ready.begin(), ready.end());
        ready.clear();
    }

    // Retires finished requests; grows overflowed frontiers.  Returns false on a
    // device error (every active request then fails).
    bool retire()
    {
        std::vector<ServerReq *> keep;
        for (ServerReq *r : active) {
            mh_handle *H = r->H;
            int st8[kStateWords];
            cudaMemcpy(st8, H->dState, sizeof st8, cudaMemcpyDeviceToHost);
            int rc = MH_OK;
            if (r->cancel && !st8[1]) {  // cancelled while running: its state stays behind
                mh_destroy(H);
                r->H = nullptr;
                std::lock_guard<std::mutex> lock(mu);
                in_use -= r->footprint;
                finish(r, MH_ECANCELED, "cancelled while running");
                cv.notify_all();
                continue;
            }
            if (st8[2]) rc = fail(MH_ETIMEOUT, "a team barrier of the served solve timed out");
            if (rc == MH_OK && st8[3]) {
                std::vector<u32> hc(kCountWords);
                cudaMemcpy(hc.data(), H->dCounts + (size_t)(st8[4] & 1) * kCountWords, sizeof(u32) * kCountWords,
                           cudaMemcpyDeviceToHost);
                rc = grow_overflowed(H, r->opts.h, hc.data());
                if (rc == MH_OK) {
                    cudaMemsetAsync(H->dCnt + (size_t)st8[4] * r->opts.h * 2, 0, sizeof(u64) * 2 * r->opts.h, st);
                    cudaMemsetAsync(H->dCut + (size_t)st8[4] * r->opts.h, 0, sizeof(u64) * r->opts.h, st);
                    cudaMemsetAsync(H->dCounts, 0, sizeof(u32) * kCountSets * kCountWords, st);
                    cudaMemsetAsync(H->dState + 3, 0, sizeof(int), st);
                    cudaStreamSynchronize(st);
                    keep.push_back(r);
                    continue;
                }
            }
            if (rc == MH_OK && !st8[1]) {
                keep.push_back(r);
                continue;
            }
            if (rc == MH_OK) rc = collect_result(H, r->opts.h, true, 0.0, nullptr, 1, 0, &r->res);
            mh_destroy(H);
            r->H = nullptr;
            std::lock_guard<std::mutex> lock(mu);
            in_use -= r->footprint;
            finish(r, rc, rc == MH_OK ? nullptr : mh_last_error());
            cv.notify_all();
        }
        std::lock_guard<std::mutex> lock(mu);
        active.swap(keep);
        return true;
    }

    // One launch over the active requests.  Small requests go first: while any is
    // active, the large ones pause at their round boundary (their state stays on the
    // device) and the small ones run batched; the large requests run when no small
    // one is active, a lone one on the single-cohort kernel, several (large_slots >
    // 1) batched together.  Rounds are latency-bound, so solves that share the GPU
    // lose little speed each and gain throughput together.
    void run_active()
    {
        std::vector<ServerReq *> sel;
        // a large request paused longer than large_wait_ms runs in this launch with
        // the small ones (no request waits without bound under a stream of small ones)
        const double t_now = now_s();
        bool starving = false;
        for (ServerReq *r : active)
            if (r->large && (t_now - r->t_ran) * 1e3 > (double)o.large_wait_ms) starving = true;
        for (ServerReq *r : active)
            if (!r->large || starving) sel.push_back(r);
        if (sel.empty()) sel = active;
        for (ServerReq *r : sel) r->t_ran = t_now;
        const int n = (int)sel.size();
        std::vector<double> work(n);
        for (int i = 0; i < n; ++i) work[i] = sel[i]->work;
        const std::vector<int> blocks = split_grid(work, 0.75, num_sms, kServerBuild);
        if (items_cap < n) {
            cudaFree(d_items);
            d_items = nullptr;
            items_cap = 0;
            if (cudaMalloc((void **)&d_items, batch_ws_bytes(n)) != cudaSuccess) return;
            items_cap = n;
        }
        std::vector<BatchItem> items(n);
        int first = 0;
        for (int i = 0; i < n; ++i) {
            mh_handle *H = sel[i]->H;
            items[i].c = H->c;
            items[i].s = sel[i]->s;
            items[i].f = frontiers_of(H);
            items[i].gsync = H->dSync;
            items[i].counts = H->dCounts;
            items[i].first_block = first;
            items[i].nblocks = blocks[i];
            first += blocks[i];
            cudaMemsetAsync(H->dSync, 0, sizeof(GridSync), st);
            cudaMemsetAsync(H->dState + 6, 0, sizeof(int), st);
        }
        *(volatile int *)h_yield = 0;
        cudaEvent_t ev;
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        cudaError_t e;
        if (n == 1) {  // a lone request: the single-cohort persistent kernel, which yields the same way
            ServerReq *r = sel[0];
            mh_handle *H = r->H;
            e = launch_solve_persistent(H->c, r->s, frontiers_of(H), H->dSync, H->dCounts,
                                        persistent_grid(num_sms, use_large_build(H, r->opts.h)),
                                        use_large_build(H, r->opts.h), st, d_yield);
        } else {
            cudaMemcpyAsync(d_items, items.data(), sizeof(BatchItem) * (size_t)n, cudaMemcpyHostToDevice, st);
            e = launch_solve_batch(d_items, n, d_yield, batch_map_at(d_items, items_cap, num_sms, kServerBuild), st);
        }
        if (e != cudaSuccess) {
            cudaEventDestroy(ev);
            return;
        }
        ++launches;
        cudaEventRecord(ev, st);
        // while the launch runs, upload queued requests that fit and ask the launch
        // to end at the next round boundary once one is ready to join
        while (cudaEventQuery(ev) == cudaErrorNotReady) {
            admit_one();
            if (!ready.empty()) *(volatile int *)h_yield = 1;
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        cudaEventDestroy(ev);
    }

    int dev = 0;

    void loop()
    {
        cudaSetDevice(dev);  // the current device is per host thread
        for (;;) {
            {
                std::unique_lock<std::mutex> lock(mu);
                cv.wait(lock, [&] { return stop || !queue.empty() || !active.empty() || !ready.empty(); });
                if (stop && queue.empty() && active.empty() && ready.empty()) return;
            }
            while (admit_one()) {
            }
            start_ready();
            if (active.empty()) continue;
            run_active();
            retire();
        }
    }
};

extern "C" {

MH_API int mh_server_create(const mh_server_opts *opts, mh_server **out)
{
    if (!out) return fail(MH_EINVAL, "out is NULL");
    *out = nullptr;
    mh_server *S = new (std::nothrow) mh_server();
    if (!S) return fail(MH_ENOMEM, "host allocation of the server failed");
    if (opts) S->o = *opts;
    if (S->o.slots <= 0) S->o.slots = 8;
    if (S->o.large_slots <= 0) S->o.large_slots = 2;
    if (S->o.large_wait_ms <= 0) S->o.large_wait_ms = 250;
    int dev = 0, coop = 0;
    cudaError_t e = cudaGetDevice(&dev);
    S->dev = dev;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e == cudaSuccess && !coop) e = cudaErrorNotSupported;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->st_up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&S->h_yield, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&S->d_yield, S->h_yield, 0);
    if (e != cudaSuccess) {
        delete S;
        return fail(MH_ECUDA, "mh_server_create: %s", cudaGetErrorString(e));
    }
    S->grid = batch_grid(S->num_sms, kServerBuild);
    if (S->o.slots > S->grid) S->o.slots = S->grid;
    if (S->o.hbm_budget_bytes > 0) {
        S->budget = S->o.hbm_budget_bytes;
    } else {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        S->budget = (int64_t)(free_b * 0.8);
    }
    S->th = std::thread([S] { S->loop(); });
    *out = S;
    return MH_OK;
}

MH_API int mh_submit(mh_server *S, const uint64_t *bitmaps, int32_t G, int32_t Nt, int32_t Nn, int32_t h,
                     mh_rational alpha, uint64_t *ticket)
{
    if (!S || !ticket) return fail(MH_EINVAL, "server or ticket is NULL");
    int rc = validate_dims(G, Nt, Nn);
    if (rc) return rc;
    if (!bitmaps) return fail(MH_EINVAL, "bitmaps is NULL");
    if (h < 1 || h > kMaxH) return fail(MH_EINVAL, "h=%d outside [1, %d]", h, kMaxH);
    if (alpha.num < 0 || alpha.den <= 0) return fail(MH_EINVAL, "alpha=%d/%d", alpha.num, alpha.den);
    ServerReq *r = new (std::nothrow) ServerReq();
    if (!r) return fail(MH_ENOMEM, "host allocation of the request failed");
    const size_t words = (size_t)G * (size_t)((Nt + 63) / 64 + (Nn + 63) / 64);
    r->bm.assign(bitmaps, bitmaps + words);
    r->G = G;
    r->Nt = Nt;
    r->Nn = Nn;
    r->opts.h = h;
    r->opts.alpha = alpha;
    r->opts.mode = MH_MODE_PERSISTENT;
    r->footprint = estimate_footprint(bitmaps, G, Nt, Nn, h, &r->work);
    r->large = r->work > kLargeWork;
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) {
        delete r;
        return fail(MH_EINVAL, "the server is shutting down");
    }
    r->ticket = S->next_ticket++;
    S->all[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
    S->cv.notify_all();
    return MH_OK;
}

static int take_result(mh_server *S, std::map<uint64_t, ServerReq *>::iterator it, mh_result **out)
{
    ServerReq *r = it->second;
    const int st = r->status;
    if (st == MH_OK) {
        *out = r->res;
        r->res = nullptr;
    } else {
        fail(st, "%s", r->msg.c_str());
    }
    S->all.erase(it);
    delete r;
    return st;
}

MH_API int mh_poll(mh_server *S, uint64_t ticket, mh_result **out)
{
    if (!S || !out) return fail(MH_EINVAL, "server or out is NULL");
    *out = nullptr;
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(MH_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second->status < 0) return MH_EAGAIN;
    return take_result(S, it, out);
}

MH_API int mh_wait(mh_server *S, uint64_t ticket, int32_t timeout_ms, mh_result **out)
{
    if (!S || !out) return fail(MH_EINVAL, "server or out is NULL");
    *out = nullptr;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(MH_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    ServerReq *r = it->second;
    auto ready = [&] { return r->status >= 0; };
    if (timeout_ms < 0) S->cv.wait(lock, ready);
    else if (!S->cv.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) return MH_EAGAIN;
    return take_result(S, S->all.find(ticket), out);
}

MH_API int mh_cancel(mh_server *S, uint64_t ticket)
{
    if (!S) return fail(MH_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(MH_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    ServerReq *r = it->second;
    if (r->status >= 0) return MH_OK;  // finished already: its result stands
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q) {
        if (*q != r) continue;
        S->queue.erase(q);
        S->finish(r, MH_ECANCELED, "cancelled while queued");
        S->cv.notify_all();
        return MH_OK;
    }
    r->cancel = true;                      // admitted: retired at the next round boundary,
    if (S->h_yield) *(volatile int *)S->h_yield = 1;  // which a running launch reaches soon
    return MH_OK;
}

MH_API int mh_set_fault(const char *spec)
{
    g_fault_env_read = 1;  // an explicit setting replaces MH_FAULT
    return parse_fault(spec);
}

MH_API int mh_server_stats(mh_server *S, int64_t *launches, int32_t *queued, int32_t *active, int64_t *bytes_in_use)
{
    if (!S) return fail(MH_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(S->mu);
    if (launches) *launches = S->launches;
    if (queued) *queued = (int32_t)S->queue.size();
    if (active) *active = (int32_t)S->active.size();
    if (bytes_in_use) *bytes_in_use = S->in_use;
    return MH_OK;
}

MH_API void mh_server_destroy(mh_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto &kv : S->all) {
        if (kv.second->res) mh_result_free(kv.second->res);
        delete kv.second;
    }
    cudaFree(S->d_items);
    if (S->h_yield) cudaFreeHost(S->h_yield);
    if (S->st) cudaStreamSynchronize(S->st);
    if (S->st) cudaStreamDestroy(S->st);
    if (S->st_up) cudaStreamDestroy(S->st_up);
    delete S;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Split search: one greedy solve divided over processes by depth-1 genes (the
// lambda units of §III-E), each process searching its share of every round and
// applying the winner merged over all of them.  Runs the one-kernel-per-phase
// path; the merge (largest key, summed counters) is the caller's.

struct mh_shard {
    mh_handle *H = nullptr;
    mh_solve_opts opts{};
    Solve s{};
    int max_rounds = 0;
    int64_t launches = 0, leaf_launches = 0;
    Key *dX = nullptr;  // xbest[0] (the shard's best), xbest[1] (the merged winner)
    bool done = false;
};

namespace {

Key pack_round_key(const mh_round_best *rb, int h)
{
    Key k;
    memset(&k, 0, sizeof k);
    if (!rb->have) return k;
    k.s = (u64)rb->score + 1;
    for (int i = 0; i < h; ++i) {
        const u64 x = (u64)(u16)rb->genes[i] << (16 * (3 - (i & 3)));
        if (i < 4) k.t0 |= x;
        else if (i < 8) k.t1 |= x;
        else k.t2 |= x;
    }
    return k;
}

int shard_state(mh_shard *X, int *hs)
{
    mh_handle *H = X->H;
    MH_CUDA(cudaMemcpyAsync(H->hState, H->dState, sizeof(int) * kStateWords, cudaMemcpyDeviceToHost, H->stream));
    MH_CUDA(cudaMemcpyAsync(H->hState + kStateWords, H->dCounts, sizeof(u32) * kCountWords, cudaMemcpyDeviceToHost,
                            H->stream));
    MH_CUDA(cudaStreamSynchronize(H->stream));
    memcpy(hs, H->hState, sizeof(int) * kStateWords);
    return MH_OK;
}

}  // namespace

extern "C" {

MH_API int mh_shard_begin(mh_handle *H, const mh_solve_opts *opts, int32_t shard, int32_t nshards, mh_shard **out)
{
    if (!out) return fail(MH_EINVAL, "out is NULL");
    *out = nullptr;
    if (nshards < 1 || shard < 0 || shard >= nshards)
        return fail(MH_EINVAL, "shard %d of %d: need 0 <= shard < nshards", shard, nshards);
    if (opts && opts->prune != MH_PRUNE_PAPER && opts->prune != MH_PRUNE_OFF)
        return fail(MH_EINVAL, "split search: prune must be MH_PRUNE_PAPER or MH_PRUNE_OFF");
    mh_shard *X = new (std::nothrow) mh_shard();
    if (!X) return fail(MH_ENOMEM, "host allocation of the split search failed");
    X->H = H;
    if (opts) X->opts = *opts;
    X->opts.mode = MH_MODE_LAUNCHES;
    int rc = prepare_solve(H, &X->opts, &X->s, &X->max_rounds);
    if (!rc) rc = dalloc(&X->dX, 2, &H->device_bytes, H->dev, H->stream);
    if (rc) {
        delete X;
        return rc;
    }
    X->s.champ = nullptr;  // one kernel per phase: no per-sample champions, no sums
    X->s.champ_ok = nullptr;
    X->s.ssum = nullptr;
    X->s.shard = shard;
    X->s.nshards = nshards;
    X->s.xbest = X->dX;
    launch_solve_init(H->c, X->s, H->ws_rounds, X->max_rounds, H->dCounts, kCountSets, H->stream);
    ++X->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dfree(X->dX, H->stream);
        delete X;
        return fail(MH_ECUDA, "starting the split search: %s", cudaGetErrorString(e));
    }
    X->done = H->Nt == 0;
    *out = X;
    return MH_OK;
}

MH_API int mh_shard_search(mh_shard *X, mh_round_best *out)
{
    if (!X || !out) return fail(MH_EINVAL, "shard or out is NULL");
    memset(out, 0, sizeof *out);
    if (X->done) {
        out->done = 1;
        return MH_OK;
    }
    mh_handle *H = X->H;
    const int h = X->opts.h;
    cudaStream_t st = H->stream;
    int hs[kStateWords];
    for (;;) {  // one round of this shard; rerun after growing an overflowed frontier
        const Frontiers fl = frontiers_of(H);
        launch_level1(H->c, X->s, fl, H->dCounts, st);
        for (int l = 2; l <= h - 1; ++l) launch_expand(H->c, X->s, l, fl, H->dCounts, leaf_grid(H), st);
        if (h >= 2) {
            launch_leaf(H->c, X->s, fl, H->dCounts, leaf_grid(H), st);
            ++X->leaf_launches;
        }
        launch_finalize_split(H->c, X->s, H->dCounts, 1, st);
        X->launches += 2 + (h >= 2 ? 1 : 0) + std::max(0, h - 2);
        MH_CUDA(cudaGetLastError());
        int rc = shard_state(X, hs);
        if (rc) return rc;
        if (hs[2]) return fail(MH_ETIMEOUT, "a bounded wait of the split search timed out");
        if (!hs[3]) break;
        const int r = hs[4];
        if ((rc = grow_overflowed(H, h, (const u32 *)(H->hState + kStateWords)))) return rc;
        MH_CUDA(cudaMemsetAsync(H->dCnt + (size_t)r * h * 2, 0, sizeof(u64) * 2 * h, st));
        MH_CUDA(cudaMemsetAsync(H->dCut + (size_t)r * h, 0, sizeof(u64) * h, st));
        MH_CUDA(cudaMemsetAsync(H->dCounts, 0, sizeof(u32) * kCountSets * kCountWords, st));
        MH_CUDA(cudaMemsetAsync(H->dState + 3, 0, sizeof(int), st));
    }
    const int r = hs[4];
    Key k;
    std::vector<u64> cnt((size_t)2 * h);
    MH_CUDA(cudaMemcpyAsync(&k, X->dX, sizeof(Key), cudaMemcpyDeviceToHost, st));
    MH_CUDA(cudaMemcpyAsync(cnt.data(), H->dCnt + (size_t)r * h * 2, sizeof(u64) * 2 * h, cudaMemcpyDeviceToHost,
                            st));
    MH_CUDA(cudaStreamSynchronize(st));
    out->have = k.s != 0;
    if (k.s) {
        out->score = (int64_t)(k.s - 1);
        for (int i = 0; i < h; ++i) {
            const u64 w = i < 4 ? k.t0 : (i < 8 ? k.t1 : k.t2);
            out->genes[i] = (int32_t)((w >> (16 * (3 - (i & 3)))) & 0xffffull);
        }
    }
    for (int l = 0; l < h; ++l) {
        out->visited[l] = cnt[(size_t)l * 2];
        out->pruned[l] = cnt[(size_t)l * 2 + 1];
    }
    return MH_OK;
}

MH_API int mh_shard_commit(mh_shard *X, const mh_round_best *merged, int32_t *done)
{
    if (!X || !merged) return fail(MH_EINVAL, "shard or merged is NULL");
    if (X->done) {
        if (done) *done = 1;
        return MH_OK;
    }
    mh_handle *H = X->H;
    const int h = X->opts.h;
    cudaStream_t st = H->stream;
    int hs[kStateWords];
    int rc = shard_state(X, hs);
    if (rc) return rc;
    const int r = hs[4];
    const Key k = pack_round_key(merged, h);
    std::vector<u64> cnt((size_t)2 * h);
    for (int l = 0; l < h; ++l) {
        cnt[(size_t)l * 2] = merged->visited[l];
        cnt[(size_t)l * 2 + 1] = merged->pruned[l];
    }
    MH_CUDA(cudaMemcpyAsync(X->dX + 1, &k, sizeof(Key), cudaMemcpyHostToDevice, st));
    MH_CUDA(cudaMemcpyAsync(H->dCnt + (size_t)r * h * 2, cnt.data(), sizeof(u64) * 2 * h, cudaMemcpyHostToDevice,
                            st));
    launch_finalize_split(H->c, X->s, H->dCounts, 2, st);
    ++X->launches;
    MH_CUDA(cudaGetLastError());
    if ((rc = shard_state(X, hs))) return rc;
    X->done = hs[1] != 0 || hs[4] >= X->max_rounds;
    if (done) *done = X->done ? 1 : 0;
    return MH_OK;
}

MH_API int mh_shard_result(mh_shard *X, mh_result **out)
{
    if (!X || !out) return fail(MH_EINVAL, "shard or out is NULL");
    *out = nullptr;
    return collect_result(X->H, X->opts.h, false, 0.0, nullptr, X->launches, X->leaf_launches, out);
}

MH_API void mh_shard_free(mh_shard *X)
{
    if (!X) return;
    dfree(X->dX, X->H->stream);
    delete X;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Coverage evaluation (§IV-D)

extern "C" MH_API int mh_evaluate(mh_handle *H, const int32_t *genes, int32_t k, int32_t h, mh_coverage *out,
                                  uint64_t *tumor_covered, uint64_t *normal_covered)
{
    if (!H || !out || (k > 0 && !genes)) return fail(MH_EINVAL, "handle, out or genes is NULL");
    if (k < 0 || h < 1 || h > kMaxH) return fail(MH_EINVAL, "k=%d, h=%d: need k >= 0 and 1 <= h <= %d", k, h, kMaxH);
    for (int64_t i = 0; i < (int64_t)k * h; ++i)
        if (genes[i] < 0 || genes[i] >= H->G) return fail(MH_EINVAL, "gene index %d outside [0, %d)", genes[i], H->G);
    cudaStream_t st = H->stream;
    const Cohort &c = H->c;
    const size_t words = (size_t)c.WTp + c.WNp;
    unsigned char *buf = nullptr;
    const size_t gbytes = ((size_t)std::max(1, k) * h * sizeof(int32_t) + 255) & ~(size_t)255;
    int rc = dalloc(&buf, gbytes + words * sizeof(u64), &H->device_bytes, H->dev, st);
    if (rc) return rc;
    int *dg = (int *)buf;
    u64 *dcov = (u64 *)(buf + gbytes);
    std::vector<u64> cov(words, 0);
    cudaError_t e = cudaMemsetAsync(dcov, 0, words * sizeof(u64), st);
    if (e == cudaSuccess && k)
        e = cudaMemcpyAsync(dg, genes, sizeof(int32_t) * (size_t)k * h, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        launch_coverage(c, dg, k, h, dcov, dcov + c.WTp, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(cov.data(), dcov, words * sizeof(u64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(buf, st);
    if (e != cudaSuccess) return fail(MH_ECUDA, "coverage evaluation failed: %s", cudaGetErrorString(e));
    int tc = 0, nc = 0;
    for (int w = 0; w < c.Wt; ++w) tc += __builtin_popcountll(cov[w]);
    for (int w = 0; w < c.Wn; ++w) nc += __builtin_popcountll(cov[(size_t)c.WTp + w]);
    out->tc = tc;
    out->tt = H->Nt;
    out->nc = nc;
    out->nt = H->Nn;
    out->sensitivity = H->Nt ? (double)tc / H->Nt : 0.0;
    out->specificity = H->Nn ? 1.0 - (double)nc / H->Nn : 0.0;
    if (tumor_covered) memcpy(tumor_covered, cov.data(), sizeof(u64) * (size_t)c.Wt);
    if (normal_covered) memcpy(normal_covered, cov.data() + c.WTp, sizeof(u64) * (size_t)c.Wn);
    return MH_OK;
}
