// kernels_expect.cu -- expectation values <psi|P|psi> of Pauli strings on a
// device-resident stabilizer tableau (sm_103a).
//
// Operation (Aaronson & Gottesman, PRA 70, 052328, Sec. III, applied to a
// general Pauli P instead of Z_a): the state is the +1 eigenstate of the n
// stabilizer rows, so
//  * if P anticommutes with some stabilizer row, <P> = 0;
//  * otherwise +-P is in the stabilizer group: it is the product of the
//    stabilizer rows n+i over the destabilizers i that anticommute with P,
//    and <P> is the sign that product carries.
//
// Design: one CTA per Pauli string.
//  1. Commutation bits c[w] of every row with P: the symplectic product
//     x_row . z_P + z_row . x_P, XOR-accumulated over the columns of P's
//     support (threads split the words and the columns).
//  2. Any stabilizer bit set: <P> = 0 (a barrier with an OR).
//  3. Otherwise the product phase, column by column.  Pauli strings multiply
//     column-wise, so the product of the selected rows (ascending order) is
//     i^(sum_j e_j) (-1)^(sum r) (x) Q_j, with e_j the exponent picked up
//     while multiplying column j's single-qubit Paulis in order.  A warp
//     takes a column: lane l reads stabilizer word Wh + w (w = w0 + l,
//     coalesced), forms each selected row's running product before it (an
//     exclusive prefix XOR inside the word, then a warp scan of the word
//     parities for the carry), and counts AG's g(x1, z1, x2, z2) for
//     "row times running product" bit-sliced: +1 on
//     YZ, XY, ZX and -1 on YX, XZ, ZY.  Q_j must come out equal to P_j.
//  4. E = sum_j e_j + 2 sum r (mod 4) is 0 or 2; <P> = +1 or -1.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pauli_product.cuh"
#include "tab_internal.h"

namespace tab {

constexpr int kExpectThreads = 256;

template <int T>
__global__ void __launch_bounds__(T) k_expect(const uint32_t* __restrict__ X,
                                              const uint32_t* __restrict__ Z,
                                              const uint32_t* __restrict__ R, int n, int Wh,
                                              const uint8_t* __restrict__ codes,
                                              int8_t* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int W = 2 * Wh;
  uint32_t* c = sm;                                       // W commutation words
  uint8_t* p = reinterpret_cast<uint8_t*>(sm + W);        // n codes of this string
  __shared__ uint32_t s_e, s_r, s_bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint8_t* P = codes + (size_t)blockIdx.x * n;
  for (int j = tid; j < n; j += T) p[j] = P[j] & 3u;
  for (int w = tid; w < W; w += T) c[w] = 0u;
  if (tid == 0) s_e = s_r = s_bad = 0u;
  __syncthreads();

  // 1. commutation bits: thread (word w, slice s) XORs columns j = s, s+S, ...
  const int S = W >= T ? 1 : T / W;
  if (tid < (W >= T ? T : W * S)) {
    const int s = W >= T ? 0 : tid / W;
    for (int w = W >= T ? tid : tid % W; w < W; w += W >= T ? T : W) {
      uint32_t acc = 0u;
      for (int j = s; j < n; j += S) {
        const uint32_t pj = p[j];
        if (pj & 1u) acc ^= __ldg(Z + (size_t)j * W + w);
        if (pj & 2u) acc ^= __ldg(X + (size_t)j * W + w);
      }
      if (acc) atomicXor(&c[w], acc);
    }
  }
  __syncthreads();

  // 2. P anticommutes with a stabilizer row: <P> = 0
  int anti = 0;
  for (int w = Wh + tid; w < W; w += T) anti |= c[w] != 0u;
  if (__syncthreads_or(anti)) {
    if (tid == 0) out[blockIdx.x] = 0;
    return;
  }

  // 3. signs of the selected stabilizers, and the column phases
  uint32_t rs = 0u;
  for (int w = tid; w < Wh; w += T) rs ^= __popc(__ldg(R + Wh + w) & c[w]) & 1u;
  if (rs) atomicXor(&s_r, 1u);
  for (int j = warp; j < n; j += T / 32) {
    uint32_t qx, qz;
    const uint32_t e = pp_column_product(X + (size_t)j * W + Wh, Z + (size_t)j * W + Wh, Wh,
                                         [&](int w) { return c[w]; }, qx, qz);
    if (lane == 0) {
      atomicAdd(&s_e, e);
      if (qx != (p[j] & 1u) || qz != (p[j] >> 1)) atomicOr(&s_bad, 1u);
    }
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t E = (s_e + 2u * s_r) & 3u;
    if (s_bad || (E & 1u)) {
      atomicCAS(err, 0, DERR_PHASE);
      out[blockIdx.x] = 0;
    } else {
      out[blockIdx.x] = E == 0u ? 1 : -1;
    }
  }
}

size_t expect_smem_bytes(int n) {
  return (size_t)2 * half_words(n) * sizeof(uint32_t) + (size_t)((n + 15) & ~15);
}

cudaError_t launch_expect(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int Wh,
                          const uint8_t* codes, int k, int8_t* out, int* err, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  const size_t smem = expect_smem_bytes(n);
  cudaError_t e = ensure_smem_limit((const void*)k_expect<kExpectThreads>,
                                    (int)expect_smem_bytes(TAB_MAX_QUBITS));
  if (e != cudaSuccess) return e;
  k_expect<kExpectThreads><<<k, kExpectThreads, smem, s>>>(X, Z, R, n, Wh, codes, out, err);
  return cudaGetLastError();
}

}  // namespace tab
