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
// buffer for the outcomes.
//
// The array is one per device per process and keeps what the last call left
// in it: the barrier and error words are cleared at every call, the rest is
// overwritten before it is read.  Calls whose work overlaps on the GPU (e.g.
// on two streams) share the array and race; serialise them on one stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "tab_internal.h"

namespace tab {

constexpr size_t kNoAllocWords = TAB_NOALLOC_SCRATCH_BYTES / sizeof(uint32_t);

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// Host-side device addresses of g_noalloc_scratch, one per device.  In host
// code the symbol itself is only a host stand-in, never a device address.
static std::mutex g_addr_mu;
static std::vector<uint32_t*> g_addr;

static int scratch_address(int dev, uint32_t** out) {
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if ((int)g_addr.size() <= dev) g_addr.resize((size_t)dev + 1, nullptr);
  if (!g_addr[(size_t)dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_error("cudaGetSymbolAddress of the measurement scratch failed: %s",
                cudaGetErrorString(e));
      return TAB_ECUDA;
    }
    g_addr[(size_t)dev] = static_cast<uint32_t*>(p);
  }
  *out = g_addr[(size_t)dev];
  return TAB_OK;
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
  std::vector<uint32_t> codes((size_t)k);
  for (int32_t i = 0; i < k; ++i) {
    if (qubits[i] < 0 || qubits[i] >= v.n) {
      set_error("qubit %d outside [0, %d)", qubits[i], v.n);
      return TAB_ERANGE;
    }
    codes[(size_t)i] = dcode(op, (uint32_t)qubits[i], 0);
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
  cudaError_t e = cudaMemcpyAsync(base, codes.data(), (size_t)k * sizeof(uint32_t),
                                  cudaMemcpyHostToDevice, v.stream);
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
