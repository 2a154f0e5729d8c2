// grid_sync.cuh -- bounded software grid barrier for cooperative launches.
#pragma once
#include <cuda_runtime.h>

#include "tab_internal.h"

namespace tab {

constexpr unsigned long long kGridWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ unsigned long long gs_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int gs_ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// All CTAs of the grid are co-resident (cooperative launch).  The last CTA to
// arrive resets the count and bumps the generation; the others spin on the
// generation.  Bounded: after kGridWaitLimitNs, or once another CTA has
// latched an error, DERR_TIMEOUT is latched and false is returned so that
// every CTA leaves.
static __device__ __noinline__ bool grid_sync(GridBar* bar, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int gen = gs_ld_acquire(&bar->gen);
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = gs_gtimer();
      while (gs_ld_acquire(&bar->gen) == gen) {
        if (*(volatile int*)err != 0 || gs_gtimer() - t0 > kGridWaitLimitNs) {
          atomicCAS(err, 0, DERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok && (*(volatile int*)err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace tab
