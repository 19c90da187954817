// Diagnostics of libmh with no counterpart in the paper: the measured integer
// throughput of the GPU, the denominator of the search kernels' roofline.
//
// mh_int_peak runs one kernel that keeps every SM's integer pipes busy with one
// kind of 32-bit operation -- LOP3 (three-input logic, the AND / OR of the
// sibling tests), POPC (population count) or IADD -- in eight independent
// dependency chains per thread, with as many resident threads as the SMs hold,
// and returns the operations retired per second (CUDA events around the launch,
// the best of several launches).  The search kernels' executed integer work is
// compared with the LOP3 rate.
#include <cstdint>

#include "mh.h"
#include "mh_internal.h"

namespace mh {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;

template <int OP>
__global__ void __launch_bounds__(kPeakThreads) k_int_peak(unsigned seed, int iters, unsigned *out)
{
    unsigned a[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) a[i] = (seed + 0x9e3779b9u * (threadIdx.x + i)) ^ blockIdx.x;
    const unsigned b = seed ^ 0x85ebca6bu, c = seed + threadIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i) {
                if (OP == 0) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[i]) : "r"(b), "r"(c));
                if (OP == 1) asm volatile("popc.b32 %0, %0;" : "+r"(a[i]));
                if (OP == 2) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[i]) : "r"(b));
            }
        }
    }
    unsigned x = 0;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x ^= a[i];
    if (x == seed) out[blockIdx.x * blockDim.x + threadIdx.x] = x;  // keeps the chains live
}

// One thread follows a chain of dependent loads through a buffer resident in L2
// (ld.global.cg: L1 bypassed), each load on its own 128-byte line; the device
// clock (globaltimer) around the second pass gives the round-trip time of one
// dependent L2 load, the unit of the persistent solve's per-round latency chain.
__global__ void k_l2_fill(u32 *next, u32 n, u32 stride)
{
    const u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) next[i] = (u32)(((unsigned long long)i + stride) % n);
}
__global__ void k_l2_chase(const u32 *next, int steps, unsigned long long *out)
{
    u32 idx = 0;
    unsigned long long t[2] = {0, 0};
    for (int pass = 0; pass < 2; ++pass) {
        unsigned long long t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (int k = 0; k < steps; ++k) idx = __ldcg(next + idx);
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1) : "r"(idx));
        t[pass] = t1 - t0;
    }
    out[0] = t[1];
    out[1] = idx;  // keeps the chain live
}

}  // namespace

}  // namespace mh

using namespace mh;

extern "C" MH_API int mh_l2_latency(double *ns_per_load)
{
    if (!ns_per_load) {
        set_error_text("mh_l2_latency: ns_per_load is NULL");
        return MH_EINVAL;
    }
    constexpr u32 kN = 1u << 20;             // 4 MB of u32: in L2, far beyond L1
    constexpr u32 kStride = 32u * 4099u;      // 128-byte lines apart, visiting many lines
    constexpr int kSteps = 4096;
    u32 *next = nullptr;
    unsigned long long *out = nullptr, h[2] = {0, 0};
    cudaError_t e = cudaMalloc((void **)&next, sizeof(u32) * kN);
    if (e == cudaSuccess) e = cudaMalloc((void **)&out, sizeof(h));
    if (e == cudaSuccess) {
        k_l2_fill<<<(kN + 255) / 256, 256>>>(next, kN, kStride);
        k_l2_chase<<<1, 1>>>(next, kSteps, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, out, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(next);
    cudaFree(out);
    if (e != cudaSuccess) {
        set_error_text(cudaGetErrorString(e));
        return MH_ECUDA;
    }
    *ns_per_load = (double)h[0] / kSteps;
    return MH_OK;
}

extern "C" MH_API int mh_int_peak(int32_t op, double *ops_per_s, double *kernel_ms)
{
    if (!ops_per_s || op < 0 || op > 2) {
        set_error_text("mh_int_peak: op must be 0 (LOP3), 1 (POPC) or 2 (IADD) and ops_per_s non-NULL");
        return MH_EINVAL;
    }
    int dev = 0, sms = 0, per_sm = 0;
    const void *fn = op == 0 ? (const void *)k_int_peak<0> : op == 1 ? (const void *)k_int_peak<1>
                                                                     : (const void *)k_int_peak<2>;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPeakThreads, 0);
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    unsigned *out = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&out, sizeof(unsigned) * (size_t)grid * kPeakThreads);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    const int iters = op == 1 ? 512 : 2048;
    float best = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(ev[0], nullptr);
        if (e != cudaSuccess) break;
        if (op == 0) k_int_peak<0><<<grid, kPeakThreads>>>(12345u + rep, iters, out);
        if (op == 1) k_int_peak<1><<<grid, kPeakThreads>>>(12345u + rep, iters, out);
        if (op == 2) k_int_peak<2><<<grid, kPeakThreads>>>(12345u + rep, iters, out);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(ev[1], nullptr);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;  // launch 0 warms up
    }
    for (int i = 0; i < 2; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (out) cudaFree(out);
    if (e != cudaSuccess || best <= 0.f) {
        set_error_text(e != cudaSuccess ? cudaGetErrorString(e) : "mh_int_peak: no timing");
        return MH_ECUDA;
    }
    const double ops = (double)grid * kPeakThreads * iters * kPeakUnroll * kPeakChains;
    *ops_per_s = ops / (best * 1e-3);
    if (kernel_ms) *kernel_ms = best;
    return MH_OK;
}
