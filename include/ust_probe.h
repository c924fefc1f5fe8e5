/*
 * ust_probe.h - measurement helper of libust.so (no counterpart in the
 * paper): the rate of random 4-byte device-memory accesses, the ceiling of
 * the sampler's gather-bound traffic.
 *
 * The sampler of include/ust.h spends its time on random gathers and atomics
 * into per-tree arrays and the CSR (Wilson draws, in-degree peeling, subtree
 * sizes, the interval tests of Algorithm 2). A random 4-byte access moves a
 * whole 32-byte sector, so a streaming copy's bandwidth is not the ceiling
 * of that work. This probe times independent random accesses at hashed
 * indices over one device array, so the same kernel gives the L2 rate
 * (arrays well inside L2) and the HBM rate (arrays far larger than L2).
 */
#ifndef UST_PROBE_H
#define UST_PROBE_H

#include <stdint.h>

#include "ust.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Times `reps` launches (after one warm-up launch that also pulls an
 * L2-sized array into L2) of random accesses over a device array of
 * the largest power-of-two size that fits `bytes` (1 MiB to 64 GiB):
 *   mode 0: 4-byte loads that bypass L1 (ld.global.cg), served by L2 or DRAM;
 *   mode 1: 4-byte atomicAdd of 1 (performed in L2);
 *   modes 2, 3, 4: aligned blocks of 16, 32 or 64 bytes, read as 16-byte
 *   vector loads that bypass L1 (the cost of a random access by its width).
 * 2048 threads per SM each keep 8 independent accesses in flight.
 * *accesses_per_s receives the best launch's accesses (4-byte words or
 * blocks) per second. The array
 * is allocated and freed by the call (cudaMalloc / cudaFree); work runs on
 * `stream` (a cudaStream_t, NULL = legacy default stream), which the call
 * synchronises. Returns 0, -1 (bad argument), -3 (allocation failed) or
 * -4 (CUDA error). */
UST_API int ust_probe_random_access(int64_t bytes, int32_t mode, int32_t reps, void *stream,
                                    double *accesses_per_s);

#ifdef __cplusplus
}
#endif

#endif /* UST_PROBE_H */
