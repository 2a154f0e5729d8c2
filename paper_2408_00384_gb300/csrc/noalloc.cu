// noalloc.cu -- Z measurement on a handle without allocating device memory
// (tab_measure_noalloc in include/tab.h).  This entry point has no
// counterpart in the paper; it exists for deployments that cannot allocate.
//
// The other measurement entry points allocate (stream-ordered) device memory
// for the staged qubit list and the outcome log, and the handle's own
// workspace holds the measurement kernel's per-CTA scratch.  Here the staged
// qubit list and every byte of kernel scratch (per-CTA sign partials, base
// signs, deterministic partials, grid-barrier word, error word) live in one
// file-scope __device__ array of fixed size, so the call allocates nothing;
// the caller brings the tableau (e.g. from tab_create_on) and the device
// buffer for the outcomes.  The qubit codes reach the array as kernel
// parameters of small staging launches (copied when each launch is issued),
// so the call keeps no host buffer and issues no host-to-device copy.
//
// The array is one per device per process and keeps what the last call left
// in it: the barrier and error words are cleared at every call, the rest is
// overwritten before it is read.  Calls whose work overlaps on the GPU (e.g.
// on two streams) share the array and race; serialise them on one stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "tab_internal.h"

namespace tab {

constexpr size_t kNoAllocWords = TAB_NOALLOC_SCRATCH_BYTES / sizeof(uint32_t);

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// Host-side device addresses of g_noalloc_scratch, one per device.  In host
// code the symbol itself is only a host stand-in, never a device address.
constexpr int kNoAllocMaxDevices = 128;
static std::mutex g_addr_mu;
static uint32_t* g_addr[kNoAllocMaxDevices];

static int scratch_address(int dev, uint32_t** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("device %d is beyond the %d devices the measurement scratch table holds", dev,
              kNoAllocMaxDevices);
    return TAB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error("cudaGetSymbolAddress of the measurement scratch failed: %s",
                cudaGetErrorString(e));
      return TAB_ECUDA;
    }
    g_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_addr[dev];
  return TAB_OK;
}

// Qubit codes per staging launch: 3,840 bytes of parameters, inside the
// 4 KB kernel-parameter limit.
constexpr int kNoAllocStage = 960;
struct StageCodes {
  uint32_t code[kNoAllocStage];
};

__global__ void k_noalloc_stage(const StageCodes c, int count, uint32_t* __restrict__ dst) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = c.code[i];
}

// Copy a latched device error into the handle's error word (keeps the first).
__global__ void k_noalloc_latch(const int* __restrict__ src, int* __restrict__ dst) {
  const int v = *src;
  if (v != 0) atomicCAS(dst, 0, v);
}

}  // namespace tab

using namespace tab;

extern "C" int tab_measure_noalloc(tab_t h, const int32_t* qubits, int32_t k, int32_t reset,
                                   uint8_t* dev_out_bits) {
  HandleView v;
  int rc = handle_view(h, &v);
  if (rc != TAB_OK) return rc;
  if (k < 0 || (k > 0 && (!qubits || !dev_out_bits))) {
    set_error("bad arguments (k=%d)", k);
    return TAB_EINVAL;
  }
  if (k == 0) return TAB_OK;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != v.dev) {
    set_error("the handle's device must be current");
    return TAB_EINVAL;
  }
  const uint32_t op = reset ? OP_MZR : OP_MZ;
  for (int32_t i = 0; i < k; ++i) {
    if (qubits[i] < 0 || qubits[i] >= v.n) {
      set_error("qubit %d outside [0, %d)", qubits[i], v.n);
      return TAB_ERANGE;
    }
  }
  // layout in the array: [codes | ph | r4 | dp | barrier | error]
  const size_t code_words = ((size_t)k + 63) & ~(size_t)63;
  const int W = 2 * v.Wh;
  int G = std::max(1, v.meas_ctas);
  while (G > 1 && code_words + measure_work_words(v.n, G) > kNoAllocWords) --G;
  if (code_words + measure_work_words(v.n, G) > kNoAllocWords) {
    set_error("k=%d measurements on n=%d qubits need more than the %zu-byte scratch", k, v.n,
              (size_t)TAB_NOALLOC_SCRATCH_BYTES);
    return TAB_ERANGE;
  }
  uint32_t* base = nullptr;
  rc = scratch_address(dev, &base);
  if (rc != TAB_OK) return rc;
  uint32_t* w = base + code_words;
  MeasWork mw;
  mw.ph = w;
  w += (size_t)G * 2 * W;
  mw.r4 = w;
  w += 2 * (size_t)W;
  mw.dp = w;
  w += 2 * (size_t)G;
  mw.bar = reinterpret_cast<GridBar*>(w);
  w += 16;
  mw.err = reinterpret_cast<int*>(w);
  mw.max_ctas = G;
  cudaError_t e = cudaSuccess;
  for (int32_t i0 = 0; i0 < k && e == cudaSuccess; i0 += kNoAllocStage) {
    const int cnt = std::min(kNoAllocStage, k - i0);
    StageCodes sc;
    for (int i = 0; i < cnt; ++i) sc.code[i] = dcode(op, (uint32_t)qubits[i0 + i], 0);
    k_noalloc_stage<<<1, 256, 0, v.stream>>>(sc, cnt, base + i0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, sizeof(int), v.stream);  // error word
  if (e == cudaSuccess)
    e = launch_measure(v.X, v.Z, v.R, v.n, v.Wh, base, k, v.k, v.seed, v.cid, v.shot, dev_out_bits,
                       mw, G, v.stream);
  if (e == cudaSuccess) {
    k_noalloc_latch<<<1, 1, 0, v.stream>>>(mw.err, v.err);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_error("launch failed: %s", cudaGetErrorString(e));
    return TAB_ECUDA;
  }
  handle_advance_k(h, (uint64_t)k);
  return TAB_OK;
}
