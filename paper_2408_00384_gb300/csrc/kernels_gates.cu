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
#include <stdlib.h>

#include <atomic>

#include "clifford1.h"
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

// ------------------------------------------------- TMA ring helpers ------
// The gate kernel streams its block records (the same for every CTA, read
// from L2) into a shared-memory ring with TMA bulk copies (cp.async.bulk,
// completion on one mbarrier per ring slot), several chunks ahead, so no
// thread waits on an L2 round trip per block.  Every wait is bounded.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gate_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity; false after ~1 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gate_gtimer();
  while (!mbar_try_wait(bar, parity))
    if (gate_gtimer() - t0 > 1000000000ull) return false;
  return true;
}
// One TMA bulk copy of `bytes` (multiple of 16, both addresses 16-B aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------ block row-slab gates ----
// Grid: one CTA per 32-row slab (row word w = blockIdx.x), W CTAs.  The slab
// of every column is staged in shared memory with each qubit's x and z words
// side by side (one 8-byte access per qubit; the compiler orders a
// super-layer's records so a half-warp's qubits fall on distinct bank
// pairs), and the slab is written back at the end.  The gate run is compiled
// into two-qubit blocks (blocks.cpp) grouped in super-layers of pairwise-
// disjoint blocks, with one CTA barrier per super-layer.  A thread applies a
// whole block to the slab's 32 rows in registers -- U_0 (x) U_1, the
// entangler, V_0 (x) V_1 -- without branching on the gates, and stores the
// two columns back (exchanged if the block swaps them).  The records (8
// bytes) stream through the TMA ring.
constexpr int kBlkChunk = 512;                  // records per TMA copy (4 KB)
constexpr int kBlkSlots = 16;                   // 64 KB ring (10 slots, 40 KB, for large n)
constexpr int kBlkRing = kBlkChunk * kBlkSlots;

// Single-qubit codes as masks: for code m, {alpha, beta, gamma, delta} and
// {eps, zeta, eta, 0} of clifford1.h as all-ones / all-zero words, two uint4
// per code in shared memory, so applying a code is two vector loads (mostly
// broadcasts: a layer uses few distinct codes) and branch-free LOP3 work.
__device__ __forceinline__ void c1_masks_init(uint4* tab, int tid, int T) {
  for (int m = tid; m < 128; m += T) {
    const uint32_t u = (uint32_t)m;
    tab[2 * m] = make_uint4(0u - (u & 1u), 0u - ((u >> 1) & 1u), 0u - ((u >> 2) & 1u),
                            0u - ((u >> 3) & 1u));
    tab[2 * m + 1] = make_uint4(0u - ((u >> 4) & 1u), 0u - ((u >> 5) & 1u), 0u - ((u >> 6) & 1u), 0u);
  }
}
__device__ __forceinline__ void c1_apply_masks(const uint4* tab, uint32_t m, uint32_t& x,
                                               uint32_t& z, uint32_t& r) {
  const uint4 a = tab[2 * m], e = tab[2 * m + 1];
  r ^= (x & e.x) ^ (z & e.y) ^ (x & z & e.z);
  const uint32_t xn = (x & a.x) ^ (z & a.y);
  z = (x & a.z) ^ (z & a.w);
  x = xn;
}

// NB blocks of one super-layer (pairwise-disjoint qubits) on the slab's 32
// rows, blocks with on[j] false skipped: every load first, then the NB
// independent computations, then every store, so the blocks' dependent
// chains interleave.  Branch-free except where a whole warp usually agrees:
// U_0 (x) U_1 is skipped when both are the identity (every block past a
// qubit's first, as the compiler folds later single-qubit gates into V), and
// a single-qubit block skips its second column's load and store.  The
// entangler is computed as CNOT-or-CZ masks.
template <int NB>
__device__ __forceinline__ void apply_blocks(const uint2 (&rec)[NB], const bool (&on)[NB],
                                             const uint4* c1m, uint2* sxz,
                                             uint32_t& r, int n, int* err) {
  uint32_t qa[NB], qb[NB], m[NB], x0[NB], z0[NB], x1[NB], z1[NB];
  bool two[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    qa[j] = dbg_index(rec[j].x & 0x3FFFu, (uint32_t)n, err);
    qb[j] = dbg_index((rec[j].x >> 14) & 0x3FFFu, (uint32_t)n, err);
    two[j] = on[j] && ((rec[j].x >> 28) & 1u);
    m[j] = rec[j].y;
    const uint2 va = on[j] ? sxz[qa[j]] : make_uint2(0u, 0u);
    const uint2 vb = two[j] ? sxz[qb[j]] : make_uint2(0u, 0u);
    x0[j] = va.x;
    z0[j] = va.y;
    x1[j] = vb.x;
    z1[j] = vb.y;
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if ((m[j] & 0x3FFFu) != (kC1Ident | (kC1Ident << 7))) {
      c1_apply_masks(c1m, m[j] & 0x7Fu, x0[j], z0[j], r);
      c1_apply_masks(c1m, (m[j] >> 7) & 0x7Fu, x1[j], z1[j], r);
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    // CNOT with control in register 0 (the compiler's convention), or CZ
    const uint32_t ent = (rec[j].x >> 29) & 3u;
    const uint32_t cn = ent == 1u ? 0xffffffffu : 0u, cz = ent == 2u ? 0xffffffffu : 0u;
    r ^= (cn & x0[j] & z1[j] & ~(x1[j] ^ z0[j])) ^ (cz & x0[j] & x1[j] & (z0[j] ^ z1[j]));
    const uint32_t x1n = x1[j] ^ (cn & x0[j]);
    const uint32_t z0n = z0[j] ^ (cn & z1[j]) ^ (cz & x1[j]);
    z1[j] ^= cz & x0[j];
    x1[j] = x1n;
    z0[j] = z0n;
    c1_apply_masks(c1m, (m[j] >> 14) & 0x7Fu, x0[j], z0[j], r);
    c1_apply_masks(c1m, (m[j] >> 21) & 0x7Fu, x1[j], z1[j], r);
  }
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const bool sw = (m[j] >> 28) & 1u;
    const uint32_t da = sw ? qb[j] : qa[j], db = sw ? qa[j] : qb[j];
    if (on[j]) sxz[da] = make_uint2(x0[j], z0[j]);
    if (two[j]) sxz[db] = make_uint2(x1[j], z1[j]);
  }
}

template <int T, int SLOTS>
__global__ void __launch_bounds__(T) k_gates_block(uint32_t* __restrict__ X, uint32_t* __restrict__ Z,
                                                   uint32_t* __restrict__ R, int n, int W,
                                                   const uint2* __restrict__ blk,
                                                   const uint32_t* __restrict__ blk_off,
                                                   int nlayers, int* __restrict__ err) {
  extern __shared__ __align__(128) uint32_t sm[];
  uint2* ring = reinterpret_cast<uint2*>(sm);  // block-record ring (SLOTS * kBlkChunk records)
  uint2* sxz = reinterpret_cast<uint2*>(sm + 2 * SLOTS * kBlkChunk);  // (X, Z) words of every column (this slab)
  __shared__ __align__(8) uint64_t bars[SLOTS];
  __shared__ uint4 c1m[256];  // masks of the 128 single-qubit codes
  __shared__ uint32_t s_r;
  __shared__ int s_abort;
  const int w = blockIdx.x, tid = threadIdx.x;
  const uint32_t ob = __ldg(blk_off), oe = __ldg(blk_off + nlayers);
  const uint32_t base = ob & ~1u;  // 16-byte aligned start of the stream
  const int nchunks = (int)((oe - base + kBlkChunk - 1) / kBlkChunk);
  int issued = 0, waited = 0;      // thread 0's pipeline state
  if (tid == 0) {
    for (int i = 0; i < SLOTS; ++i) mbar_init(&bars[i], 1);
    mbar_fence_init();
    s_r = 0u;
    s_abort = 0;
    for (; issued < nchunks && issued < SLOTS; ++issued)
      tma_bulk_g2s(ring + (size_t)issued * kBlkChunk, blk + base + (size_t)issued * kBlkChunk,
                   kBlkChunk * 8, &bars[issued]);
  }
  for (int a = tid; a < n; a += T) sxz[a] = make_uint2(X[(size_t)a * W + w], Z[(size_t)a * W + w]);
  c1_masks_init(c1m, tid, T);
  __syncthreads();

  uint32_t racc = 0u;
  uint32_t prev_lb = ob, lb = ob;
  for (int L = 0; L < nlayers; ++L) {
    const uint32_t le = __ldg(blk_off + L + 1);
    if (tid == 0) {
      // refill slots whose chunk ended before the previous super-layer began
      while (issued < nchunks &&
             (int64_t)base + (int64_t)(issued - SLOTS + 1) * kBlkChunk <= (int64_t)prev_lb) {
        const int slot = issued % SLOTS;
        fence_proxy_async_smem();
        tma_bulk_g2s(ring + (size_t)slot * kBlkChunk, blk + base + (size_t)issued * kBlkChunk,
                     kBlkChunk * 8, &bars[slot]);
        ++issued;
      }
      if (le > lb) {
        const int c_last = (int)((le - 1 - base) / kBlkChunk);
        if (c_last >= issued) {
          atomicCAS(err, 0, DERR_BOUNDS);
          s_abort = 1;
        } else {
          for (; waited <= c_last; ++waited)
            if (!mbar_wait_bounded(&bars[waited % SLOTS], (uint32_t)(waited / SLOTS) & 1u)) {
              atomicCAS(err, 0, DERR_TIMEOUT);
              s_abort = 1;
              break;
            }
        }
      }
    }
    __syncthreads();
    if (s_abort) break;
    // thread tid takes blocks lb + tid, lb + tid + T, ... two at a time
    for (uint32_t g = lb + tid; g < le; g += 2 * T) {
      const uint32_t g2 = g + T;
      const uint2 recs[2] = {ring[(g - base) % (SLOTS * kBlkChunk)],
                             ring[(g2 < le ? g2 - base : g - base) % (SLOTS * kBlkChunk)]};
      const bool on[2] = {true, g2 < le};
      apply_blocks<2>(recs, on, c1m, sxz, racc, n, err);
    }
    prev_lb = lb;
    lb = le;
  }
  // every copy issued must land before the CTA exits
  if (tid == 0)
    for (; waited < issued; ++waited)
      mbar_wait_bounded(&bars[waited % SLOTS], (uint32_t)(waited / SLOTS) & 1u);
  __syncthreads();
  if (s_abort) return;

  for (int a = tid; a < n; a += T) {
    const uint2 v = sxz[a];
    X[(size_t)a * W + w] = v.x;
    Z[(size_t)a * W + w] = v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) racc ^= __shfl_xor_sync(0xffffffffu, racc, o);
  if ((tid & 31) == 0 && racc) atomicXor(&s_r, racc);
  __syncthreads();
  if (tid == 0) R[w] ^= s_r;
}

constexpr int kMaxSmemBytes = 227 * 1024;

// dynamic shared memory of the block kernel: what is left next to its static
// share (mbarriers, code masks: under 5 KB)
constexpr int kBlkDynMax = kMaxSmemBytes - 8192;

int gates_block_max_n() { return (kBlkDynMax - kBlkRing * 8) / 8; }

// Threads per CTA of the block kernel: the kernel is latency-bound per
// super-layer, so a CTA just large enough for two blocks per thread (n/2
// blocks in a full layer, interleaved in pairs) keeps its barrier cheap:
// 128, 256 or 512 threads.  TAB_BLOCK_THREADS overrides (tuning sweeps).
static int block_threads(int n) {
  const int forced = run_config().block_threads;
  if (forced == 128 || forced == 256 || forced == 512) return forced;
  return n <= 512 ? 128 : n <= 1024 ? 256 : 512;
}

template <int T, int SLOTS>
static cudaError_t launch_gates_block_t(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int W,
                                        const uint2* blk, const uint32_t* blk_off, int nlayers,
                                        int* err, cudaStream_t s) {
  const size_t smem = (size_t)SLOTS * kBlkChunk * 8 + (size_t)n * 2 * sizeof(uint32_t);
  // once per device; shard threads may launch concurrently
  const cudaError_t attr =
      ensure_smem_limit((const void*)k_gates_block<T, SLOTS>, kBlkDynMax);
  if (attr != cudaSuccess) return attr;
  k_gates_block<T, SLOTS><<<W, T, smem, s>>>(X, Z, R, n, W, blk, blk_off, nlayers, err);
  return cudaGetLastError();
}

// Ring slots: 16, or 10 where the smaller ring (still two super-layers of at
// most kMaxLayerOps records plus a chunk on each side: 5,120 records) is what
// lets two CTAs share an SM.  The budget is the device's shared memory per SM
// split in two, less the per-CTA reservation and the kernel's static share
// (mbarriers, the code-mask table), queried once per device.
static int block_slots(int n) {
  constexpr int kMaxDev = 64;
  static std::atomic<long long> budget[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 16;
  }
  long long two = budget[dev].load();
  if (two == 0) {
    int per_sm = 0, reserved = 0;
    cudaFuncAttributes fa{};
    if (cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, (const void*)k_gates_block<512, 10>) != cudaSuccess) {
      cudaGetLastError();
      return 16;
    }
    two = (long long)per_sm / 2 - reserved - (long long)fa.sharedSizeBytes;
    budget[dev].store(two > 0 ? two : -1);
  }
  const long long c16 = 16LL * kBlkChunk * 8 + 8LL * n;
  const long long c10 = 10LL * kBlkChunk * 8 + 8LL * n;
  return (c16 > two && c10 <= two) ? 10 : 16;
}

cudaError_t launch_gates_block(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int W,
                               const uint2* blk, const uint32_t* blk_off, int nlayers, int* err,
                               cudaStream_t s, int threads) {
  if (nlayers <= 0) return cudaSuccess;
  if (block_slots(n) == 10)
    return launch_gates_block_t<512, 10>(X, Z, R, n, W, blk, blk_off, nlayers, err, s);
  switch (threads == 128 || threads == 256 || threads == 512 ? threads : block_threads(n)) {
    case 128: return launch_gates_block_t<128, 16>(X, Z, R, n, W, blk, blk_off, nlayers, err, s);
    case 256: return launch_gates_block_t<256, 16>(X, Z, R, n, W, blk, blk_off, nlayers, err, s);
    default: return launch_gates_block_t<512, 16>(X, Z, R, n, W, blk, blk_off, nlayers, err, s);
  }
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
