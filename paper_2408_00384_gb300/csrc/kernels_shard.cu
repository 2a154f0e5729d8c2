// kernels_shard.cu -- per-shard kernels of a row-sharded tableau (sm_103a).
//
// A shard owns the qubit-row indices i in [i0, i1): destabilizer i and its
// partner stabilizer n+i, for all n columns.  Its storage is a tableau of the
// usual layout over those rows: X[j * Ws + w] with Ws = 2 Whs words per
// column, words [0, Whs) holding the destabilizers (row i0 + 32 w + b at bit
// b) and words [Whs, Ws) the stabilizers.  Gates need no exchange (AG Sec.
// III: every row is updated from its own bits), so the gate kernels run on a
// shard unchanged.  A Z measurement (AG Sec. III) runs as these steps, with
// the exchanges between them done by the host:
//  * k_sh_pivot: the smallest local stabilizer row with x_pa = 1 (then an
//    all-reduce of the minimum over the shards);
//  * random case: k_sh_getrow on the owner of p packs row p (then it is
//    broadcast); k_sh_rowsum multiplies every local row h with x_ha = 1 (but
//    p and p-n) by it; k_sh_setrows on the owner copies row p into row p-n
//    and sets row p to Z_a with the Philox outcome as its sign;
//  * deterministic case: k_sh_partial forms the product of the local
//    stabilizer rows selected by their destabilizers' x_ia bits (then the
//    partial products are gathered); k_sh_combine multiplies them in shard
//    order, checks that the result is +-Z_a and writes the outcome.
// Row words are packed one bit per column: x bits in words [0, nw), z bits
// in [nw, 2 nw), the sign (or the exponent of i) in word 2 nw.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pauli_product.cuh"
#include "philox.cuh"
#include "tab_internal.h"

namespace tab {

constexpr int kShThreads = 256;

__global__ void k_sh_init(uint32_t* __restrict__ X, uint32_t* __restrict__ Z,
                          uint32_t* __restrict__ R, int n, int i0, int i1, int Whs) {
  const int Ws = 2 * Whs;
  const size_t plane = (size_t)n * Ws;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < plane;
       k += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(k / Ws), w = (int)(k % Ws);
    const int t = (w < Whs ? w : w - Whs) * 32;  // local row of bit 0
    const int li = j - i0;                        // column j's own row, if local
    const uint32_t bit = (j >= i0 && j < i1 && li >= t && li < t + 32) ? 1u << (li - t) : 0u;
    X[k] = w < Whs ? bit : 0u;
    Z[k] = w < Whs ? 0u : bit;
  }
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < Ws; w += gridDim.x * blockDim.x)
    R[w] = 0u;
}

// smallest local i with x = 1 in column a of stabilizer n+i, or INT32_MAX
__global__ void k_sh_pivot(const uint32_t* __restrict__ X, int Whs, int a, int* piv) {
  __shared__ int best;
  if (threadIdx.x == 0) best = 0x7fffffff;
  __syncthreads();
  const uint32_t* col = X + (size_t)a * 2 * Whs + Whs;
  for (int w = threadIdx.x; w < Whs; w += blockDim.x) {
    const uint32_t v = col[w];
    if (v) atomicMin(&best, w * 32 + __ffs(v) - 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *piv = best;
}

// row = stabilizer at local index li (x bits, z bits, sign)
__global__ void k_sh_getrow(const uint32_t* __restrict__ X, const uint32_t* __restrict__ Z,
                            const uint32_t* __restrict__ R, int n, int Whs, int li,
                            uint32_t* __restrict__ row) {
  const int Ws = 2 * Whs, nw = (n + 31) / 32, w = Whs + li / 32, b = li % 32;
  const int lane = threadIdx.x & 31;
  for (int j0 = (threadIdx.x & ~31); j0 < nw * 32; j0 += blockDim.x) {
    const int j = j0 + lane;
    const bool in = j < n;
    const uint32_t xb = __ballot_sync(0xffffffffu, in && ((X[(size_t)(in ? j : 0) * Ws + w] >> b) & 1u));
    const uint32_t zb = __ballot_sync(0xffffffffu, in && ((Z[(size_t)(in ? j : 0) * Ws + w] >> b) & 1u));
    if (lane == 0) {
      row[j0 / 32] = xb;
      row[nw + j0 / 32] = zb;
    }
  }
  if (threadIdx.x == 0) row[2 * nw] = (R[w] >> b) & 1u;
}

// Every local row h with x_ha = 1, h != p and h != p-n (li >= 0 on the owner
// of p), becomes row_p * row_h with the sign AG's rowsum gives.  One CTA per
// local word; its threads split the columns, each keeping bit-sliced mod-4
// exponent counters (lo, hi) of the 32 rows for its columns, and the
// counters are summed over the threads (mod-4 addition, bit-sliced) before
// the sign update.
__global__ void k_sh_rowsum(uint32_t* __restrict__ X, uint32_t* __restrict__ Z,
                            uint32_t* __restrict__ R, int n, int Whs, int a, int li,
                            const uint32_t* __restrict__ row_g, int* __restrict__ err) {
  extern __shared__ uint32_t row[];  // 2 nw + 1 words, then 2 * blockDim.x counters
  const int Ws = 2 * Whs, nw = (n + 31) / 32, w = blockIdx.x, T = blockDim.x;
  uint32_t* clo = row + 2 * nw + 1;
  uint32_t* chi = clo + T;
  for (int k = threadIdx.x; k < 2 * nw + 1; k += T) row[k] = row_g[k];
  __syncthreads();
  uint32_t m = X[(size_t)a * Ws + w];  // rows with x_ha = 1, read before any update
  if (li >= 0 && (w == li / 32 || w == Whs + li / 32)) m &= ~(1u << (li % 32));
  uint32_t lo = 0u, hi = 0u;
  __syncthreads();  // every thread has read column a before it changes
  if (m) {
    for (int j = threadIdx.x; j < n; j += T) {
      const uint32_t xp = 0u - ((row[j >> 5] >> (j & 31)) & 1u);
      const uint32_t zp = 0u - ((row[nw + (j >> 5)] >> (j & 31)) & 1u);
      if (!(xp | zp)) continue;
      const size_t k = (size_t)j * Ws + w;
      const uint32_t x2 = X[k], z2 = Z[k];
      const uint32_t plus = (xp & zp & ~x2 & z2) | (xp & ~zp & x2 & z2) | (~xp & zp & x2 & ~z2);
      const uint32_t minus = (xp & zp & x2 & ~z2) | (xp & ~zp & ~x2 & z2) | (~xp & zp & x2 & z2);
      hi ^= (lo & plus) | (~lo & minus);
      lo ^= plus | minus;
      X[k] = x2 ^ (m & xp);
      Z[k] = z2 ^ (m & zp);
    }
  }
  clo[threadIdx.x] = lo;
  chi[threadIdx.x] = hi;
  __syncthreads();
  for (int o = T / 2; o > 0; o >>= 1) {  // (lo, hi) + (lo', hi') mod 4, bit-sliced
    if (threadIdx.x < o) {
      const uint32_t l2 = clo[threadIdx.x + o], h2 = chi[threadIdx.x + o];
      const uint32_t l1 = clo[threadIdx.x];
      chi[threadIdx.x] ^= h2 ^ (l1 & l2);
      clo[threadIdx.x] = l1 ^ l2;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && m) {
    if (clo[0] & m) atomicCAS(err, 0, DERR_PHASE);
    R[w] ^= m & ((0u - row[2 * nw]) ^ chi[0]);
  }
}

// Owner of p (local index li): row p-n := row p (the broadcast copy), row
// p := Z_a with sign = the Philox outcome of measurement k, written to *bout.
__global__ void k_sh_setrows(uint32_t* __restrict__ X, uint32_t* __restrict__ Z,
                             uint32_t* __restrict__ R, int n, int Whs, int a, int li,
                             const uint32_t* __restrict__ row, uint64_t seed, uint64_t cid,
                             uint32_t shot, uint64_t k, uint8_t* __restrict__ bout) {
  const int Ws = 2 * Whs, nw = (n + 31) / 32, wd = li / 32, ws = Whs + li / 32;
  const uint32_t bit = 1u << (li % 32);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const size_t c = (size_t)j * Ws;
    const bool xb = (row[j >> 5] >> (j & 31)) & 1u, zb = (row[nw + (j >> 5)] >> (j & 31)) & 1u;
    X[c + wd] = (X[c + wd] & ~bit) | (xb ? bit : 0u);
    Z[c + wd] = (Z[c + wd] & ~bit) | (zb ? bit : 0u);
    X[c + ws] &= ~bit;
    Z[c + ws] = (Z[c + ws] & ~bit) | (j == a ? bit : 0u);
  }
  if (threadIdx.x == 0) {
    const uint32_t b = outcome_bit(seed, cid, shot, k);
    R[wd] = (R[wd] & ~bit) | (row[2 * nw] ? bit : 0u);
    R[ws] = (R[ws] & ~bit) | (b ? bit : 0u);
    *bout = (uint8_t)b;
  }
}

// Product of the local stabilizer rows n+i whose destabilizer has x_ia = 1,
// ascending i: out = x bits, z bits, exponent E (product = i^E (x) P(x, z)).
__global__ void k_sh_partial(const uint32_t* __restrict__ X, const uint32_t* __restrict__ Z,
                             const uint32_t* __restrict__ R, int n, int Whs, int a,
                             uint32_t* __restrict__ out) {
  extern __shared__ uint32_t acc[];  // 2 nw words
  __shared__ uint32_t s_e;
  const int Ws = 2 * Whs, nw = (n + 31) / 32, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < 2 * nw; k += blockDim.x) acc[k] = 0u;
  if (threadIdx.x == 0) s_e = 0u;
  __syncthreads();
  const uint32_t* sel = X + (size_t)a * Ws;  // destabilizer words of column a
  uint32_t rs = 0u;
  for (int w = threadIdx.x; w < Whs; w += blockDim.x) rs += __popc(R[Whs + w] & sel[w]);
  if (rs) atomicAdd(&s_e, 2u * rs);
  for (int j = warp; j < n; j += blockDim.x / 32) {
    uint32_t qx, qz;
    const uint32_t e = pp_column_product(X + (size_t)j * Ws + Whs, Z + (size_t)j * Ws + Whs, Whs,
                                         [&](int w) { return __ldg(sel + w); }, qx, qz);
    if (lane == 0) {
      atomicAdd(&s_e, e);
      if (qx) atomicOr(&acc[j >> 5], 1u << (j & 31));
      if (qz) atomicOr(&acc[nw + (j >> 5)], 1u << (j & 31));
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * nw; k += blockDim.x) out[k] = acc[k];
  if (threadIdx.x == 0) out[2 * nw] = s_e & 3u;
}

// The shards' partial products multiplied in shard order (later ones on the
// left); the result must be +-Z_a, and its sign is the outcome.
__global__ void k_sh_combine(const uint32_t* __restrict__ parts, int shards, int n, int a,
                             uint8_t* __restrict__ bout, int* __restrict__ err) {
  extern __shared__ uint32_t q[];  // running product: 2 nw words
  __shared__ uint32_t s_e, s_bad;
  const int nw = (n + 31) / 32, stride = 2 * nw + 1;
  for (int k = threadIdx.x; k < 2 * nw; k += blockDim.x) q[k] = parts[k];
  if (threadIdx.x == 0) {
    s_e = parts[2 * nw] & 3u;
    s_bad = 0u;
  }
  __syncthreads();
  for (int s = 1; s < shards; ++s) {
    const uint32_t* p = parts + (size_t)s * stride;
    uint32_t e = 0u;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
      const uint32_t x1 = p[w], z1 = p[nw + w], x2 = q[w], z2 = q[nw + w];
      const uint32_t plus = (x1 & z1 & ~x2 & z2) | (x1 & ~z1 & x2 & z2) | (~x1 & z1 & x2 & ~z2);
      const uint32_t minus = (x1 & z1 & x2 & ~z2) | (x1 & ~z1 & ~x2 & z2) | (~x1 & z1 & x2 & z2);
      e += (uint32_t)__popc(plus) + 3u * (uint32_t)__popc(minus);
    }
    if (e) atomicAdd(&s_e, e & 3u);
    __syncthreads();
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
      q[w] ^= p[w];
      q[nw + w] ^= p[nw + w];
    }
    if (threadIdx.x == 0) s_e += p[2 * nw];
    __syncthreads();
  }
  for (int w = threadIdx.x; w < nw; w += blockDim.x) {
    const uint32_t wantz = (a >> 5) == w ? 1u << (a & 31) : 0u;
    if (q[w] != 0u || q[nw + w] != wantz) atomicOr(&s_bad, 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t E = s_e & 3u;
    if (s_bad || (E & 1u)) atomicCAS(err, 0, DERR_PHASE);
    *bout = (uint8_t)(E >> 1);
  }
}

// X on qubit a: the sign of every local row with z_ha = 1 flips
__global__ void k_sh_xgate(const uint32_t* __restrict__ Z, uint32_t* __restrict__ R, int Whs,
                           int a) {
  const int Ws = 2 * Whs;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < Ws; w += gridDim.x * blockDim.x)
    R[w] ^= Z[(size_t)a * Ws + w];
}

// Unpacked rows of the shard into the caller's (2n) x n arrays.
__global__ void k_sh_unpack(const uint32_t* __restrict__ X, const uint32_t* __restrict__ Z,
                            const uint32_t* __restrict__ R, int n, int i0, int i1, int Whs,
                            uint8_t* __restrict__ xs, uint8_t* __restrict__ zs,
                            uint8_t* __restrict__ rs) {
  const int Ws = 2 * Whs, cnt = i1 - i0;
  const size_t total = (size_t)2 * cnt * n;
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (size_t)gridDim.x * blockDim.x) {
    const int t = (int)(k / n), j = (int)(k % n);  // t < cnt: destabilizer, else stabilizer
    const int li = t < cnt ? t : t - cnt;
    const int w = (t < cnt ? 0 : Whs) + li / 32, b = li % 32;
    const size_t row = t < cnt ? (size_t)(i0 + li) : (size_t)(n + i0 + li);
    xs[row * n + j] = (X[(size_t)j * Ws + w] >> b) & 1u;
    zs[row * n + j] = (Z[(size_t)j * Ws + w] >> b) & 1u;
    if (j == 0) rs[row] = (R[w] >> b) & 1u;
  }
}

// ---- launches --------------------------------------------------------------

static unsigned sh_blocks(size_t work) {
  const size_t b = (work + kShThreads - 1) / kShThreads;
  return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t sh_init(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int i0, int i1, int Whs,
                    cudaStream_t s) {
  k_sh_init<<<sh_blocks((size_t)n * 2 * Whs), kShThreads, 0, s>>>(X, Z, R, n, i0, i1, Whs);
  return cudaGetLastError();
}
cudaError_t sh_pivot(const uint32_t* X, int Whs, int a, int* piv, cudaStream_t s) {
  k_sh_pivot<<<1, kShThreads, 0, s>>>(X, Whs, a, piv);
  return cudaGetLastError();
}
cudaError_t sh_getrow(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int Whs,
                      int li, uint32_t* row, cudaStream_t s) {
  k_sh_getrow<<<1, kShThreads, 0, s>>>(X, Z, R, n, Whs, li, row);
  return cudaGetLastError();
}
cudaError_t sh_rowsum(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Whs, int a, int li,
                      const uint32_t* row, int* err, cudaStream_t s) {
  const size_t smem = (size_t)(2 * ((n + 31) / 32) + 1 + 2 * kShThreads) * 4;
  k_sh_rowsum<<<2 * Whs, kShThreads, smem, s>>>(X, Z, R, n, Whs, a, li, row, err);
  return cudaGetLastError();
}
cudaError_t sh_setrows(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Whs, int a, int li,
                       const uint32_t* row, uint64_t seed, uint64_t cid, uint32_t shot,
                       uint64_t k, uint8_t* bout, cudaStream_t s) {
  k_sh_setrows<<<1, kShThreads, 0, s>>>(X, Z, R, n, Whs, a, li, row, seed, cid, shot, k, bout);
  return cudaGetLastError();
}
cudaError_t sh_partial(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int Whs,
                       int a, uint32_t* out, cudaStream_t s) {
  const size_t smem = (size_t)2 * ((n + 31) / 32) * 4;
  k_sh_partial<<<1, kShThreads, smem, s>>>(X, Z, R, n, Whs, a, out);
  return cudaGetLastError();
}
cudaError_t sh_combine(const uint32_t* parts, int shards, int n, int a, uint8_t* bout, int* err,
                       cudaStream_t s) {
  const size_t smem = (size_t)2 * ((n + 31) / 32) * 4;
  k_sh_combine<<<1, kShThreads, smem, s>>>(parts, shards, n, a, bout, err);
  return cudaGetLastError();
}
cudaError_t sh_xgate(const uint32_t* Z, uint32_t* R, int Whs, int a, cudaStream_t s) {
  k_sh_xgate<<<sh_blocks((size_t)2 * Whs), kShThreads, 0, s>>>(Z, R, Whs, a);
  return cudaGetLastError();
}
cudaError_t sh_unpack(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int i0,
                      int i1, int Whs, uint8_t* xs, uint8_t* zs, uint8_t* rs, cudaStream_t s) {
  k_sh_unpack<<<sh_blocks((size_t)2 * (i1 - i0) * n), kShThreads, 0, s>>>(X, Z, R, n, i0, i1,
                                                                           Whs, xs, zs, rs);
  return cudaGetLastError();
}

}  // namespace tab
