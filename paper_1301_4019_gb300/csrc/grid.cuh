// grid.cuh -- grid-wide synchronisation of cooperative (co-resident) launches: a bounded
// grid barrier on the handle's arrival counter, and the host helpers that size and launch
// such grids.
#pragma once

#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace rsk {
namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier over all CTAs of the (cooperative, hence co-resident) launch, on one
// arrival counter in the handle's ScanGlob that counts up through the launch: barrier k is
// passed when the counter reaches k * gridDim.x. Thread 0 of each CTA arrives with a release
// reduction and polls with acquire loads (the CTA's writes are ordered before the arrival by
// the preceding __syncthreads, and every later read after the poll by the following one).
// The wait is bounded: after the handle's timeout (bar->timeout_ns, 10 s unless set by
// rs_set_barrier_timeout) it records RS_ERR_TIMEOUT and goes on; rs_last_error, which reports
// the status, then resets the counter.
__device__ __forceinline__ void grid_barrier(GridBar* bar, unsigned int& target, int* err) {
  unsigned int* count = &bar->count;
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    unsigned int cur;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(count) : "memory");
    if (static_cast<int>(cur - target) < 0) {
      const unsigned long long t0 = global_ns();
      const unsigned long long limit = __ldcg(&bar->timeout_ns);
      for (;;) {
        __nanosleep(20);
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(count) : "memory");
        if (static_cast<int>(cur - target) >= 0) break;
        if (global_ns() - t0 > limit) {
          flag_error(err, RS_ERR_TIMEOUT);
          break;
        }
      }
    }
  }
  __syncthreads();
}

// Last act of every CTA: one more arrival; the CTA that completes it returns the counter to
// 0 for the next launch (stream order makes the reset visible to it).
__device__ __forceinline__ void grid_exit(GridBar* bar, unsigned int target) {
  if (threadIdx.x == 0 && atomicAdd(&bar->count, 1u) == target + gridDim.x - 1)
    atomicExch(&bar->count, 0u);
}

// Largest co-resident grid of a kernel with kBlock threads (cached per kernel; identical
// devices assumed), 0 when it cannot be determined.
inline int coop_capacity(const void* kernel) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess)
    return 0;
  cache[kernel] = per_sm * sms;
  return per_sm * sms;
}

// Cooperative launch of `grid` CTAs of kBlock threads (grid <= coop_capacity).
template <typename... KArgs, typename... Args>
inline cudaError_t coop_launch(void (*kernel)(KArgs...), int grid, cudaStream_t st,
                               Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

}  // namespace
}  // namespace rsk
