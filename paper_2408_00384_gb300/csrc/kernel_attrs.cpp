// kernel_attrs.cpp -- one-time kernel attributes, per device.
//
// cudaFuncSetAttribute acts on the current device, so a limit raised for a
// handle on device 0 does not hold for a handle on device 1, and launchers
// may run on several host threads at once (shard ranks, server workers).
// The table below records which (kernel, device, limit) has been set; it is
// fixed-size, so checking it never allocates.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "tab_internal.h"

namespace tab {

namespace {
struct AttrEntry {
  const void* fn;
  int bytes;
  uint64_t devices;  // bit d: set on device d
};
constexpr int kAttrEntries = 64;
std::mutex g_attr_mu;
AttrEntry g_attr[kAttrEntries];
int g_attr_used = 0;
}  // namespace

cudaError_t ensure_smem_limit(const void* fn, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_attr_mu);
  AttrEntry* ent = nullptr;
  for (int i = 0; i < g_attr_used; ++i)
    if (g_attr[i].fn == fn && g_attr[i].bytes == bytes) ent = &g_attr[i];
  if (ent && dev < 64 && (ent->devices >> dev & 1u)) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  if (!ent && g_attr_used < kAttrEntries) {
    ent = &g_attr[g_attr_used++];
    ent->fn = fn;
    ent->bytes = bytes;
    ent->devices = 0;
  }
  if (ent && dev < 64) ent->devices |= uint64_t(1) << dev;
  return cudaSuccess;
}

}  // namespace tab
