// peaks.cu -- microbenchmarks of the ceilings the tableau kernels are held to
// (tab_measure_peaks in include/tab.h).
//
// Every hot kernel of this library is GF(2) logic on words that sit in shared
// memory, in L2 or in HBM, so its roofline is one of: the integer logic pipe
// (one LOP3 per logic op), the shared-memory port, the L2, or (for the
// streaming measurement engine at large n) HBM.  The per-launch latency of a
// dependent chain of grid barriers bounds the measurement engines as well.
// Each figure below is measured on the current device with CUDA events around
// one launch, after an untimed warm-up launch; nothing changes a GPU setting.
//
//  * logic: every thread runs 8 independent chains of lop3.b32 (inline PTX,
//    so each counted op is exactly one instruction), 2 CTAs of 1,024 threads
//    per SM.  The SM clock over the run is read from clock64 against the
//    global timer on CTA 0, so ops per SM per clock follow as well.
//  * shared memory: 128-bit ld.volatile.shared.v4 of consecutive 16-byte
//    chunks per warp (no bank conflicts), a new address every load,
//    XOR-accumulated so the loads stay live.
//  * L2: 128-bit ld.global.cg (cached in L2 only) over a 64 MiB buffer, which
//    fits GB300's L2, read-only and read-modify-write, many passes in one
//    launch after a warm-up pass.
//  * grid barrier: the library's bounded grid_sync, one CTA per SM in a
//    cooperative launch, 20,000 barriers back to back.
#include <cuda_runtime.h>
#include <stdint.h>

#include "grid_sync.cuh"
#include "tab_internal.h"

namespace tab {

constexpr int kPeakThreads = 1024;
constexpr int kLogicChains = 8;
constexpr int kLogicUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads, 2)
    k_peak_logic(int iters, uint32_t* sink, unsigned long long* clk) {
  uint32_t a[kLogicChains];
#pragma unroll
  for (int j = 0; j < kLogicChains; ++j) a[j] = threadIdx.x * 0x9E3779B9u + j;
  const uint32_t b = blockIdx.x * 0x85EBCA6Bu, c = ~threadIdx.x;
  unsigned long long c0 = 0, t0 = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c0 = clock64();
    t0 = gs_gtimer();
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kLogicUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kLogicChains; ++j)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[j]) : "r"(b), "r"(c));
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < kLogicChains; ++j) x ^= a[j];
  if (x == 0x2545F491u) sink[0] = x;  // keeps the chains live; practically never true
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64() - c0;
    clk[1] = gs_gtimer() - t0;
  }
}

constexpr int kSmemWords = 8192;  // 32 KB per CTA

__global__ void __launch_bounds__(kPeakThreads, 2) k_peak_smem(int iters, uint32_t* sink) {
  __shared__ __align__(16) uint32_t buf[kSmemWords];
  for (int i = threadIdx.x; i < kSmemWords; i += blockDim.x) buf[i] = i * 0x27D4EB2Fu;
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
  constexpr uint32_t kMask = kSmemWords * 4u - 1u;  // 32 KB, a power of two
  uint32_t x0 = 0, x1 = 0, x2 = 0, x3 = 0;
  // each warp reads 512 consecutive bytes per load (4 conflict-free
  // wavefronts); the address moves every load, and the loads are volatile
  // so none is merged with another
  uint32_t off = threadIdx.x * 16u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      uint32_t v0, v1, v2, v3;
      const uint32_t addr = base + ((off + u * 4112u) & kMask);
      asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(v0), "=r"(v1), "=r"(v2), "=r"(v3)
                   : "r"(addr));
      x0 ^= v0;
      x1 ^= v1;
      x2 ^= v2;
      x3 ^= v3;
    }
    off += 528u;
  }
  if ((x0 ^ x1 ^ x2 ^ x3) == 0x2545F491u) sink[0] = x0;
}

__global__ void k_peak_l2(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16,
                          int passes, uint32_t* sink) {
  uint32_t x = 0;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) {
      uint4 v = __ldcg(src + i);
      if (dst) {
        v.x ^= 1u;
        __stcg(dst + i, v);
      } else {
        x ^= v.x ^ v.y ^ v.z ^ v.w;
      }
    }
  }
  if (x == 0x2545F491u) sink[0] = x;
}

__global__ void k_peak_barrier(GridBar* bar, int* err, int rounds) {
  unsigned int epoch = 0;
  for (int i = 0; i < rounds; ++i)
    if (!grid_sync(bar, err, epoch)) return;
}

}  // namespace tab

using namespace tab;

namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" int tab_measure_peaks(tab_peaks* out) {
  if (!out) {
    set_error("null output");
    return TAB_EINVAL;
  }
  int dev = 0, sms = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
    set_error("no CUDA device");
    return TAB_ECUDA;
  }
  *out = tab_peaks{};
  out->sms = sms;
  cudaStream_t s = nullptr;
  uint32_t* sink = nullptr;
  unsigned long long* clk = nullptr;
  uint4* l2buf = nullptr;
  GridBar* bar = nullptr;
  int* err = nullptr;
  const size_t l2_bytes = 64ull << 20;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&sink, 64);
  if (e == cudaSuccess) e = cudaMalloc(&clk, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&l2buf, 2 * l2_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&bar, sizeof(GridBar) + 64);
  if (e == cudaSuccess) err = reinterpret_cast<int*>(bar + 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBar) + 64, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(l2buf, 0x5A, 2 * l2_bytes, s);
  int rc = TAB_OK;
  if (e == cudaSuccess) {
    Timer t;
    float ms = 0.f;
    // logic ops: 2 CTAs of 1,024 threads per SM
    const int lblocks = 2 * sms, liters = 12000;
    k_peak_logic<<<lblocks, kPeakThreads, 0, s>>>(64, sink, clk);
    cudaEventRecord(t.a, s);
    k_peak_logic<<<lblocks, kPeakThreads, 0, s>>>(liters, sink, clk);
    cudaEventRecord(t.b, s);
    e = cudaEventSynchronize(t.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
    unsigned long long hc[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(hc, clk, sizeof hc, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      const double ops = (double)lblocks * kPeakThreads * liters * kLogicUnroll * kLogicChains;
      out->logic_tops = ops / (ms * 1e-3) / 1e12;
      out->sm_clock_mhz = hc[1] ? (double)hc[0] / (double)hc[1] * 1e3 : 0.0;
      if (out->sm_clock_mhz > 0)
        out->logic_ops_per_clk_sm = ops / ((double)hc[0] * sms);
      out->logic_ms = ms;
    }
    // shared memory loads
    const int siters = 6000;
    if (e == cudaSuccess) {
      k_peak_smem<<<lblocks, kPeakThreads, 0, s>>>(16, sink);
      cudaEventRecord(t.a, s);
      k_peak_smem<<<lblocks, kPeakThreads, 0, s>>>(siters, sink);
      cudaEventRecord(t.b, s);
      e = cudaEventSynchronize(t.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
      if (e == cudaSuccess) {
        const double bytes = (double)lblocks * kPeakThreads * siters * 8 * 16;
        out->smem_gbs = bytes / (ms * 1e-3) / 1e9;
        if (out->sm_clock_mhz > 0)
          out->smem_bytes_per_clk_sm = bytes / (ms * 1e-3) / (out->sm_clock_mhz * 1e6) / sms;
      }
    }
    // L2: 64 MiB read-only, then read + write into a second 64 MiB
    const size_t n16 = l2_bytes / 16;
    const int passes = 20;
    const int l2blocks = 4 * sms;
    if (e == cudaSuccess) {
      k_peak_l2<<<l2blocks, 512, 0, s>>>(l2buf, nullptr, n16, 1, sink);
      cudaEventRecord(t.a, s);
      k_peak_l2<<<l2blocks, 512, 0, s>>>(l2buf, nullptr, n16, passes, sink);
      cudaEventRecord(t.b, s);
      e = cudaEventSynchronize(t.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
      if (e == cudaSuccess) out->l2_read_gbs = (double)l2_bytes * passes / (ms * 1e-3) / 1e9;
    }
    if (e == cudaSuccess) {
      uint4* dst = l2buf + n16;
      // 32 MiB source + 32 MiB destination: the whole working set is 64 MiB
      k_peak_l2<<<l2blocks, 512, 0, s>>>(l2buf, dst, n16 / 2, 1, sink);
      cudaEventRecord(t.a, s);
      k_peak_l2<<<l2blocks, 512, 0, s>>>(l2buf, dst, n16 / 2, passes, sink);
      cudaEventRecord(t.b, s);
      e = cudaEventSynchronize(t.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
      if (e == cudaSuccess) out->l2_rw_gbs = (double)l2_bytes * passes / (ms * 1e-3) / 1e9;
    }
    // grid barrier: one CTA of 256 threads per SM, cooperative
    const int rounds = 20000;
    if (e == cudaSuccess && coop) {
      int r = rounds;
      void* args1[] = {&bar, &err, &r};
      int warm = 100;
      void* args0[] = {&bar, &err, &warm};
      e = cudaLaunchCooperativeKernel((const void*)k_peak_barrier, dim3(sms), dim3(256), args0, 0,
                                      s);
      if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);  // counter restarts
      if (e == cudaSuccess) cudaEventRecord(t.a, s);
      if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void*)k_peak_barrier, dim3(sms), dim3(256), args1,
                                        0, s);
      if (e == cudaSuccess) cudaEventRecord(t.b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(t.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
      int herr = 0;
      if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof herr, cudaMemcpyDeviceToHost);
      if (e == cudaSuccess) {
        if (herr != 0) {
          set_error("grid barrier benchmark latched device error %d", herr);
          rc = TAB_ETIMEOUT;
        } else {
          out->grid_barrier_us = ms * 1e3 / rounds;
        }
      }
    }
  }
  if (e != cudaSuccess) {
    set_error("peak benchmark failed: %s", cudaGetErrorString(e));
    rc = TAB_ECUDA;
  }
  if (s) cudaStreamSynchronize(s);
  cudaFree(sink);
  cudaFree(clk);
  cudaFree(l2buf);
  cudaFree(bar);
  if (s) cudaStreamDestroy(s);
  return rc;
}
