// philox.cuh -- Philox4x32-10 counter-based generator, written from its
// published definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
// as easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit multiplies
// (multipliers 0xD2511F53, 0xCD9E8D57) with the key bumped by the Weyl
// constants (0x9E3779B9, 0xBB67AE85) between rounds.
#pragma once
#include <stdint.h>

namespace tab {

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint32_t lo0 = 0xD2511F53u * ctr.x, hi0 = mulhi32(0xD2511F53u, ctr.x);
    const uint32_t lo1 = 0xCD9E8D57u * ctr.z, hi1 = mulhi32(0xCD9E8D57u, ctr.z);
    ctr = make_uint4(hi1 ^ ctr.y ^ key.x, lo1, hi0 ^ ctr.w ^ key.y, lo0);
    key.x += 0x9E3779B9u;
    key.y += 0xBB67AE85u;
  }
  return ctr;
}

// Outcome bit of measurement k of (circuit_id, shot) under seed: bit 0 of
// output word 0 for counter (k, shot, cid lo, cid hi), key (seed lo, seed hi).
__host__ __device__ __forceinline__ uint32_t outcome_bit(uint64_t seed, uint64_t cid,
                                                         uint32_t shot, uint64_t k) {
  const uint4 r = philox4x32_10(
      make_uint4((uint32_t)k, shot, (uint32_t)cid, (uint32_t)(cid >> 32)),
      make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  return r.x & 1u;
}

}  // namespace tab
