// debug.cu -- the debug build's device index check, run on its own
// (tab_debug_build / tab_debug_check in include/tab.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "tab_internal.h"

namespace tab {

__global__ void k_debug_check(uint32_t index, uint32_t limit, uint32_t* out, int* err) {
  *out = dbg_index(index, limit, err);
}

}  // namespace tab

using namespace tab;

extern "C" int tab_debug_build(void) { return kDebugBuild ? 1 : 0; }

extern "C" int tab_debug_check(uint32_t index, uint32_t limit, uint32_t* checked) {
  if (!checked) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  uint32_t* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed");
    return TAB_ECUDA;
  }
  int rc = TAB_OK;
  uint32_t h[2] = {0u, 0u};
  if (cudaMemset(d, 0, 2 * sizeof(uint32_t)) != cudaSuccess) rc = TAB_ECUDA;
  if (rc == TAB_OK) {
    k_debug_check<<<1, 1>>>(index, limit, d, reinterpret_cast<int*>(d + 1));
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = TAB_ECUDA;
  }
  cudaFree(d);
  if (rc != TAB_OK) {
    set_error("debug check launch failed");
    return rc;
  }
  *checked = h[0];
  if ((int)h[1] == DERR_BOUNDS) {
    set_error("index out of range: %u >= %u", index, limit);
    return TAB_EDEVICE;
  }
  return TAB_OK;
}
