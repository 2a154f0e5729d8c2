// grid_sync.cuh -- bounded software grid barrier for cooperative launches.
#pragma once
#include <cuda_runtime.h>

#include "tab_internal.h"

namespace tab {


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

__device__ __forceinline__ void gs_red_release(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All CTAs of the grid are co-resident (cooperative launch) and call
// grid_sync the same number of times; `epoch` is a per-thread count of the
// calls so far in this launch (0 at kernel start), and bar->count is 0 at
// launch.  Thread 0 of each CTA adds 1 to the counter with release semantics
// (after the CTA barrier, so every write of the CTA is ordered before it),
// then polls with acquire loads until the counter reaches epoch x gridDim:
// every CTA has arrived, and every CTA's writes before its arrival are
// visible.  The counter only grows, so no CTA has to reset it.  Bounded:
// after limit_ns, or once another CTA has latched an error, DERR_TIMEOUT is
// latched and false is returned so that every CTA leaves.
static __device__ __noinline__ bool grid_sync(GridBar* bar, int* err, unsigned int& epoch,
                                              unsigned long long limit_ns = kDefaultWaitLimitNs) {
  __shared__ int s_ok;
  __syncthreads();
  ++epoch;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = epoch * gridDim.x;
    gs_red_release(&bar->count, 1u);
    const unsigned long long t0 = gs_gtimer();
    while ((int)(gs_ld_acquire(&bar->count) - target) < 0) {
      if (*(volatile int*)err != 0 || gs_gtimer() - t0 > limit_ns) {
        atomicCAS(err, 0, DERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok = ok && (*(volatile int*)err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace tab
