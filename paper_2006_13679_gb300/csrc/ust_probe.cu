// Random-access bandwidth probe: the ceiling of the sampler's memory traffic.
//
// The sampler's work is random 4-byte gathers and atomics into per-tree
// arrays and the CSR. A streaming copy (the HBM figure the roofline is
// usually quoted against) says little about that traffic: every random
// 4-byte access moves a whole 32-byte sector. This probe measures the rate of
// independent random 4-byte loads (L1 bypassed) or atomic adds over a device
// array of a chosen size, so the same kernel gives the L2 rate (arrays well
// inside the 126 MB L2) and the HBM rate (arrays many times larger).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ust_probe.h"

namespace {

// MurmurHash3's 32-bit finaliser (Appleby): a bijection on 32-bit words with
// full avalanche, so consecutive counters give scattered indices.
__device__ __forceinline__ uint32_t fmix32(uint32_t h)
{
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

constexpr int kInFlight = 8;  // independent accesses per thread per iteration

// mode 0: loads through L2 (ld.global.cg); mode 1: atomicAdd. Every thread
// issues iters * kInFlight accesses at hashed indices of a[0 .. mask].
__global__ void __launch_bounds__(256) probe_kernel(int32_t *a, uint32_t mask, int iters, int mode, uint32_t salt,
                                                    int32_t *sink)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t ctr = tid * (uint32_t)(iters * kInFlight) ^ salt;
    int32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        uint32_t idx[kInFlight];
#pragma unroll
        for (int k = 0; k < kInFlight; ++k) idx[k] = fmix32(ctr++) & mask;
        if (mode == 0) {
            int32_t v[kInFlight];
#pragma unroll
            for (int k = 0; k < kInFlight; ++k) v[k] = __ldcg(a + idx[k]);
#pragma unroll
            for (int k = 0; k < kInFlight; ++k) acc += v[k];
        } else if (mode == 1) {
#pragma unroll
            for (int k = 0; k < kInFlight; ++k) atomicAdd(a + idx[k], 1);
        } else {
            // blocks of 16 << (mode - 2) bytes at aligned random positions,
            // read as 16-byte vectors
            const int vecs = 1 << (mode - 2);
            const uint32_t block_mask = ~(uint32_t)(4 * vecs - 1);
#pragma unroll
            for (int k = 0; k < kInFlight; ++k) {
                const int4 *q = reinterpret_cast<const int4 *>(a + (idx[k] & block_mask));
                for (int j = 0; j < vecs; ++j) {
                    const int4 v = __ldcg(q + j);
                    acc += v.x ^ v.w;
                }
            }
        }
    }
    if (acc == 0x7FFFFFFF) sink[tid & 1023] = acc;  // keeps the loads alive
}

}  // namespace

extern "C" int ust_probe_random_access(int64_t bytes, int32_t mode, int32_t reps, void *stream,
                                       double *accesses_per_s)
{
    if (!accesses_per_s || mode < 0 || mode > 4 || reps < 1 || bytes < (1 << 20) || bytes > (1ll << 36))
        return -1;
    // the largest power-of-two word count that fits `bytes`
    uint64_t words = 1;
    while (words * 2 * sizeof(int32_t) <= (uint64_t)bytes && words * 2 <= (1ull << 32)) words *= 2;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -4;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -4;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int32_t *a = nullptr, *sink = nullptr;
    if (cudaMalloc(&a, words * sizeof(int32_t)) != cudaSuccess) return -3;
    if (cudaMalloc(&sink, 1024 * sizeof(int32_t)) != cudaSuccess) {
        cudaFree(a);
        return -3;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    double best = 0.0;
    const int threads = 256, blocks = sms * 8;  // 2048 threads per SM
    const int iters = 128;
    const double per_launch = (double)blocks * threads * iters * kInFlight;
    if (cudaMemsetAsync(a, 0, words * sizeof(int32_t), st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = -4;
    } else {
        for (int r = 0; r <= reps && rc == 0; ++r) {  // launch 0 warms the array into L2 (when it fits)
            cudaEventRecord(e0, st);
            probe_kernel<<<blocks, threads, 0, st>>>(a, (uint32_t)(words - 1), iters, mode, 0x9E3779B9u * (r + 1),
                                                     sink);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = -4;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms > 0.f) best = std::max(best, per_launch / (ms * 1e-3));
        }
        if (cudaGetLastError() != cudaSuccess) rc = -4;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(sink);
    if (rc == 0) *accesses_per_s = best;
    return rc;
}
