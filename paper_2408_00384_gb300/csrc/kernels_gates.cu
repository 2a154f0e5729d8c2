// kernels_gates.cu -- tableau initialisation, fused gate application and
// packing kernels (sm_103a).
//
// Gate rules (Aaronson & Gottesman, PRA 70, 052328, Sec. III, and the products
// of those rules for the other gates), applied to 32 rows at a time, one bit
// per row in a 32-bit word (x = X-plane word, z = Z-plane word, r = sign word):
//   H      r ^= x&z;               swap(x, z)
//   S      r ^= x&z;               z ^= x
//   S^dag  r ^= x&~z;              z ^= x
//   X/Y/Z  r ^= z / x^z / x
//   CNOT   r ^= xc & zt & ~(xt^zc); xt ^= xc; zc ^= zt
//   CZ     r ^= xa & xb & (za^zb); za ^= xb; zb ^= xa
//   SWAP   swap columns
// Rows are independent under gates, so a CTA that owns a 32-row slab of the
// tableau can apply an entire gate segment to it with no communication with
// other CTAs.  Gates within one layer act on disjoint qubits and commute, so
// the CTA's threads take different gates of a layer in parallel; sign
// contributions XOR into a per-thread register and are reduced once at the end.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gate_rules.cuh"
#include "tab_internal.h"

namespace tab {

// ---------------------------------------------------------------- init -----
__global__ void k_init(uint32_t* __restrict__ X, uint32_t* __restrict__ Z,
                       uint32_t* __restrict__ R, int n, int Wh) {
  const int W = 2 * Wh;
  const size_t total = (size_t)n * W;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(i / W), w = (int)(i % W);
    const uint32_t bit = 1u << (a & 31);
    X[i] = (w == (a >> 5)) ? bit : 0u;        // destabilizer a = +X_a
    Z[i] = (w == Wh + (a >> 5)) ? bit : 0u;   // stabilizer a = +Z_a
  }
  if (blockIdx.x == 0)
    for (int w = threadIdx.x; w < W; w += blockDim.x) R[w] = 0u;
}

void launch_init(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh, cudaStream_t s) {
  const size_t total = (size_t)n * 2 * Wh;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_init<<<blocks, 256, 0, s>>>(X, Z, R, n, Wh);
}

// ------------------------------------------------- fused row-slab gates ----
// Grid: one CTA per 32-row slab (row word w = blockIdx.x), W CTAs.  The slab
// of every column (x and z words, 8 bytes per qubit) is staged in shared
// memory, the segment's layers are applied in order with a CTA barrier
// between layers, and the slab is written back.
template <int T>
__global__ void __launch_bounds__(T) k_gates_slab(uint32_t* __restrict__ X, uint32_t* __restrict__ Z,
                                                  uint32_t* __restrict__ R, int n, int W,
                                                  const uint32_t* __restrict__ ops,
                                                  const uint32_t* __restrict__ layer_off,
                                                  int nlayers) {
  extern __shared__ uint32_t sm[];
  uint32_t* sx = sm;      // X-plane word of every column (this slab's 32 rows)
  uint32_t* sz = sm + n;  // Z-plane word of every column
  __shared__ uint32_t s_r;
  const int w = blockIdx.x;
  for (int a = threadIdx.x; a < n; a += T) {
    sx[a] = X[(size_t)a * W + w];
    sz[a] = Z[(size_t)a * W + w];
  }
  if (threadIdx.x == 0) s_r = 0u;
  __syncthreads();

  uint32_t racc = 0u;
  uint32_t lb = __ldg(layer_off);
  for (int L = 0; L < nlayers; ++L) {
    const uint32_t le = __ldg(layer_off + L + 1);
    for (uint32_t g = lb + threadIdx.x; g < le; g += T)
      apply_gate(__ldg(ops + g), sx, sz, 1, 0, racc);
    lb = le;
    __syncthreads();
  }

  for (int a = threadIdx.x; a < n; a += T) {
    X[(size_t)a * W + w] = sx[a];
    Z[(size_t)a * W + w] = sz[a];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) racc ^= __shfl_xor_sync(0xffffffffu, racc, o);
  if ((threadIdx.x & 31) == 0 && racc) atomicXor(&s_r, racc);
  __syncthreads();
  if (threadIdx.x == 0) R[w] ^= s_r;
}

constexpr int kGateThreads = 256;
constexpr int kMaxSmemBytes = 227 * 1024;

int gates_max_n() { return (kMaxSmemBytes - 1024) / 8; }

cudaError_t launch_gates_slab(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int W,
                              const uint32_t* ops, const uint32_t* layer_off, int nlayers,
                              cudaStream_t s) {
  if (nlayers <= 0) return cudaSuccess;
  const size_t smem = (size_t)n * 2 * sizeof(uint32_t);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gates_slab<kGateThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMaxSmemBytes - 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_gates_slab<kGateThreads><<<W, kGateThreads, smem, s>>>(X, Z, R, n, W, ops, layer_off, nlayers);
  return cudaGetLastError();
}

// --------------------------------------------------------- pack / unpack ---
// Unpacked layout: row-major bytes x[i*n + j], z[i*n + j], r[i] for rows
// i in [0, 2n).  Packed row of logical row i: i (destabilizer) or
// 32*Wh + (i - n) (stabilizer).
__global__ void k_pack(uint32_t* __restrict__ X, uint32_t* __restrict__ Z, uint32_t* __restrict__ R,
                       const uint8_t* __restrict__ xs, const uint8_t* __restrict__ zs,
                       const uint8_t* __restrict__ rs, int n, int Wh) {
  const int W = 2 * Wh;
  const size_t total = (size_t)n * W;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total + W;
       i += (size_t)gridDim.x * blockDim.x) {
    const bool sign = i >= total;
    const int a = sign ? 0 : (int)(i / W);
    const int w = sign ? (int)(i - total) : (int)(i % W);
    const int half = w >= Wh;
    uint32_t xw = 0u, zw = 0u;
    for (int b = 0; b < 32; ++b) {
      const int k = (w - (half ? Wh : 0)) * 32 + b;  // row index within the half
      if (k >= n) break;
      const size_t row = (size_t)(half ? n + k : k);
      if (sign) {
        xw |= (uint32_t)(rs[row] & 1u) << b;
      } else {
        xw |= (uint32_t)(xs[row * n + a] & 1u) << b;
        zw |= (uint32_t)(zs[row * n + a] & 1u) << b;
      }
    }
    if (sign) {
      R[w] = xw;
    } else {
      X[(size_t)a * W + w] = xw;
      Z[(size_t)a * W + w] = zw;
    }
  }
}

__global__ void k_unpack(const uint32_t* __restrict__ X, const uint32_t* __restrict__ Z,
                         const uint32_t* __restrict__ R, uint8_t* __restrict__ xs,
                         uint8_t* __restrict__ zs, uint8_t* __restrict__ rs, int n, int Wh) {
  const int W = 2 * Wh;
  const size_t rows = 2 * (size_t)n;
  const size_t total = rows * n;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total + rows;
       e += (size_t)gridDim.x * blockDim.x) {
    if (e >= total) {
      const size_t i = e - total;
      const size_t P = i < (size_t)n ? i : (size_t)32 * Wh + (i - n);
      rs[i] = (uint8_t)((R[P >> 5] >> (P & 31)) & 1u);
      continue;
    }
    const size_t i = e / n, j = e % n;
    const size_t P = i < (size_t)n ? i : (size_t)32 * Wh + (i - n);
    xs[e] = (uint8_t)((X[j * W + (P >> 5)] >> (P & 31)) & 1u);
    zs[e] = (uint8_t)((Z[j * W + (P >> 5)] >> (P & 31)) & 1u);
  }
}

static int grid_for(size_t total) {
  size_t b = (total + 255) / 256;
  if (b > 8192) b = 8192;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_pack(uint32_t* X, uint32_t* Z, uint32_t* R, const uint8_t* xs,
                        const uint8_t* zs, const uint8_t* rs, int n, int Wh, cudaStream_t s) {
  const size_t total = (size_t)n * 2 * Wh + 2 * Wh;
  k_pack<<<grid_for(total), 256, 0, s>>>(X, Z, R, xs, zs, rs, n, Wh);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const uint32_t* X, const uint32_t* Z, const uint32_t* R, uint8_t* xs,
                          uint8_t* zs, uint8_t* rs, int n, int Wh, cudaStream_t s) {
  const size_t total = 2 * (size_t)n * n + 2 * (size_t)n;
  k_unpack<<<grid_for(total), 256, 0, s>>>(X, Z, R, xs, zs, rs, n, Wh);
  return cudaGetLastError();
}

}  // namespace tab
