// Cohort store built on the device (the preprocessing of §III-C and §IV-A: the
// sparsity sort applied to the rows, and the derived layouts the kernels read).
//
// The host validates the rows, counts each gene's and each tumor's mutations,
// sorts the genes (counting sort by tumor mutation count, ties by original index)
// and uploads the packed rows with the permutation; these kernels then write every
// piece of the store in place: rows in search order and in original order, the
// sample-major copies, each tumor's running column counts and gene lists (search
// positions, and original indices ascending), and each gene's static depth-1
// record.  Every piece is a pure function of the rows and the permutation.
#include "mh_internal.h"

namespace mh {

namespace {

// Rows in search order (T, N) and in original order (TO, NO), zero-padded to the
// even strides; orig / inv.  One thread per (gene, word of the wider stride).
__global__ void k_store_rows(const u64 *bm, int W, int Wt, int Wn, int WTp, int WNp, int G, const u32 *order,
                             u64 *T, u64 *N, u64 *TO, u64 *NO, u16 *orig, u32 *inv)
{
    const int Wp = WTp > WNp ? WTp : WNp;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)G * Wp) return;
    const int i = (int)(t / Wp), w = (int)(t % Wp);
    const int g = (int)order[i];
    const u64 *src = bm + (size_t)g * W, *own = bm + (size_t)i * W;
    if (w < WTp) {
        T[(size_t)i * WTp + w] = w < Wt ? src[w] : 0ull;
        TO[(size_t)i * WTp + w] = w < Wt ? own[w] : 0ull;
    }
    if (w < WNp) {
        N[(size_t)i * WNp + w] = w < Wn ? src[Wt + w] : 0ull;
        NO[(size_t)i * WNp + w] = w < Wn ? own[Wt + w] : 0ull;
    }
    if (w == 0) {
        orig[i] = (u16)g;
        inv[g] = (u32)i;
    }
}

// Per tumor s: running popcounts of its sample-major column (CC, GW + 1 entries),
// its genes in search order (SL, from CT) and in original order (SLo, from the
// column over the original-order rows).  One warp per tumor: a lane per column
// word, a warp prefix sum of the words' popcounts placing each word's genes.
__device__ __forceinline__ int warp_incl_sum(int v, int lane)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    return v;
}
__global__ void k_store_lists(const u64 *CT, const u64 *CTo, int Nt, int GW, const u32 *SO, u16 *CC, u16 *SL,
                              u16 *SLo)
{
    const int lane = threadIdx.x & 31;
    const int s = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (s >= Nt) return;  // whole warps leave together
    const u64 *col = CT + (size_t)s * GW, *colo = CTo + (size_t)s * GW;
    u16 *cc = CC + (size_t)s * (GW + 1);
    u32 base = SO[s], baseo = SO[s];
    int run = 0;
    for (int w0 = 0; w0 < GW; w0 += 32) {
        const int w = w0 + lane;
        const u64 x = w < GW ? col[w] : 0ull, xo = w < GW ? colo[w] : 0ull;
        const int n = __popcll(x), no = __popcll(xo);
        const int inc = warp_incl_sum(n, lane), inco = warp_incl_sum(no, lane);
        if (w < GW) cc[w] = (u16)(run + inc - n);
        u32 k = base + (u32)(inc - n), ko = baseo + (u32)(inco - no);
        for (u64 y = x; y; y &= y - 1) SL[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
        for (u64 y = xo; y; y &= y - 1) SLo[ko++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
        const int tot = __shfl_sync(0xffffffffu, inc, 31), toto = __shfl_sync(0xffffffffu, inco, 31);
        run += tot;
        base += (u32)tot;
        baseo += (u32)toto;
    }
    if (lane == 0) cc[GW] = (u16)run;
}

// Static depth-1 record of every gene (search order): all its tumors and normals,
// listed when few, and its tumor signature.  One thread per gene.
__global__ void k_store_records(const u64 *T, const u64 *N, int G, int Wt, int Wn, int WTp, int WNp, Rec *GR, u64 *GS)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= G) return;
    Rec r;
    r.p.w0 = (u64)i;
    r.p.w1 = 0;
    for (int q = 0; q < kListT + kListN; ++q) r.ids[q] = 0;
    r.pad[0] = r.pad[1] = r.pad[2] = 0;
    const u64 *trow = T + (size_t)i * WTp, *nrow = N + (size_t)i * WNp;
    int ky = 0, kn = 0;
    u64 sig = 0;
    for (int w = 0; w < Wt; ++w) {
        ky += __popcll(trow[w]);
        sig |= trow[w];
    }
    for (int w = 0; w < Wn; ++w) kn += __popcll(nrow[w]);
    r.ky = (u16)(ky < 0xffff ? ky : 0xffff);
    r.kn = (u16)(kn < 0xffff ? kn : 0xffff);
    if (ky <= kListT) {
        int k = 0;
        for (int w = 0; w < Wt; ++w)
            for (u64 y = trow[w]; y; y &= y - 1) r.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
    }
    if (kn <= kListN) {
        int k = kListT;
        for (int w = 0; w < Wn; ++w)
            for (u64 y = nrow[w]; y; y &= y - 1) r.ids[k++] = (u16)(w * 64 + __ffsll((long long)y) - 1);
    }
    GR[i] = r;
    GS[i] = sig;
}

}  // namespace

cudaError_t launch_store_build(const StoreBuild &b, cudaStream_t st)
{
    const Cohort &c = b.c;
    const int Wp = c.WTp > c.WNp ? c.WTp : c.WNp;
    const long long nrow = (long long)c.G * Wp;
    if (nrow > 0)
        k_store_rows<<<(unsigned)((nrow + 255) / 256), 256, 0, st>>>(b.bm, c.Wt + c.Wn, c.Wt, c.Wn, c.WTp, c.WNp, c.G,
                                                                      b.order, b.T, b.N, b.TO, b.NO, b.orig, b.inv);
    if (c.Nt > 0) {
        launch_transpose(c, b.T, c.WTp, c.Nt, b.CT, st);
        launch_transpose(c, b.TO, c.WTp, c.Nt, b.CTo, st);
    }
    if (c.Nn > 0) launch_transpose(c, b.N, c.WNp, c.Nn, b.CN, st);
    if (c.Nt > 0)
        k_store_lists<<<(c.Nt + 3) / 4, 128, 0, st>>>(b.CT, b.CTo, c.Nt, c.GW, b.SO, b.CC, b.SL, b.SLo);
    if (c.G > 0) k_store_records<<<(c.G + 127) / 128, 128, 0, st>>>(b.T, b.N, c.G, c.Wt, c.Wn, c.WTp, c.WNp, b.GR, b.GS);
    return cudaGetLastError();
}

}  // namespace mh
