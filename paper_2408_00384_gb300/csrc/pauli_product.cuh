// pauli_product.cuh -- one warp forms the ordered product of selected rows of
// one tableau column (device helper shared by the expectation and the
// sharded-measurement kernels).
//
// Pauli strings multiply column by column: the product of rows t1 < t2 < ...
// (later rows multiplied on the left) is i^(sum_j e_j) (x) Q_j with Q_j the
// XOR of the rows' (x, z) bits in column j and e_j the exponent of i picked
// up there, sum over the rows of AG's g(row bits, running product bits)
// (Aaronson & Gottesman, PRA 70, 052328, Sec. III): +1 on YZ, XY, ZX and -1
// on YX, XZ, ZY.  Lane l of the warp reads word w0 + l of the column
// (coalesced); the running product before a row is an exclusive prefix XOR
// inside the word plus a warp scan of the word parities.
#pragma once
#include <stdint.h>

namespace tab {

__device__ __forceinline__ uint32_t pp_prefix_xor_inclusive(uint32_t v) {
  v ^= v << 1;
  v ^= v << 2;
  v ^= v << 4;
  v ^= v << 8;
  v ^= v << 16;
  return v;
}

// Column words xc[0 .. nw), zc[0 .. nw) (one bit per row), rows selected by
// sel(w).  Whole warp, convergent.  Returns (in every lane) the exponent sum
// mod 4 and the product's bits (qx, qz).
template <typename Sel>
__device__ __forceinline__ uint32_t pp_column_product(const uint32_t* __restrict__ xc,
                                                      const uint32_t* __restrict__ zc, int nw,
                                                      Sel sel, uint32_t& qx, uint32_t& qz) {
  const int lane = threadIdx.x & 31;
  uint32_t cx = 0u, cz = 0u, e = 0u;
  for (int w0 = 0; w0 < nw; w0 += 32) {
    const int w = w0 + lane;
    const uint32_t m = w < nw ? sel(w) : 0u;
    const uint32_t x1 = m ? __ldg(xc + w) & m : 0u;
    const uint32_t z1 = m ? __ldg(zc + w) & m : 0u;
    const uint32_t ix = pp_prefix_xor_inclusive(x1), iz = pp_prefix_xor_inclusive(z1);
    const uint32_t bx = ix >> 31, bz = iz >> 31;
    uint32_t sx = bx, sz = bz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t tx = __shfl_up_sync(0xffffffffu, sx, o);
      const uint32_t tz = __shfl_up_sync(0xffffffffu, sz, o);
      if (lane >= o) {
        sx ^= tx;
        sz ^= tz;
      }
    }
    const uint32_t inx = (sx ^ bx) ^ cx, inz = (sz ^ bz) ^ cz;  // rows before this word
    const uint32_t x2 = (ix << 1) ^ (0u - inx), z2 = (iz << 1) ^ (0u - inz);
    const uint32_t plus = (x1 & z1 & ~x2 & z2) | (x1 & ~z1 & x2 & z2) | (~x1 & z1 & x2 & ~z2);
    const uint32_t minus = (x1 & z1 & x2 & ~z2) | (x1 & ~z1 & ~x2 & z2) | (~x1 & z1 & x2 & z2);
    e += (uint32_t)__popc(plus) + 3u * (uint32_t)__popc(minus);
    cx ^= __shfl_sync(0xffffffffu, sx, 31);
    cz ^= __shfl_sync(0xffffffffu, sz, 31);
  }
  qx = cx;
  qz = cz;
  return __reduce_add_sync(0xffffffffu, e) & 3u;
}

}  // namespace tab
