// measure_resident.cuh -- Z measurement runs on a tableau whose columns stay
// in the shared memory of the CTAs that own them for the whole run.
//
// Operation: Aaronson & Gottesman, PRA 70, 052328, Sec. III, measurement step
// (the formalism of the Clifford backend in arXiv:2408.00384, "Simulation of
// Clifford circuits"):
//   random case: rows h with x_ha = 1 (h != p, p-n) become row_p * row_h with
//     2 r_h' = 2 r_h + 2 r_p + sum_j [x_pj z_pj + x_hj z_hj - x'_hj z'_hj
//                                     + 2 z_pj x_hj]   (mod 4),
//     (x' = x_h ^ x_p, z' = z_h ^ z_p), then row p-n := row p and
//     row p := (-1)^b Z_a;
//   deterministic case: e = sum_{m in T} (2 r_m + |x_m & z_m|)
//                           + 2 sum_{m<l in T} z_m . x_l  (mod 4), outcome e/2.
//
// Ownership.  CTA r of C owns the columns j = r, r+C, r+2C, ... in shared
// memory; within the CTA, warp v owns the local columns v, v+16, v+32, ...
// The sign exponent 2 r_h (mod 4) of every row is kept as a sum of shares:
// one base (CTA 0, warp 0) plus one share per warp, held in that warp's
// registers (bit-sliced, lane l holds words l, l+32, ...).  Every term of the
// rowsum exponent is a sum over columns, and "2 r_p" is the sum of the
// shares of row p, so a warp adds only its own columns' terms and its own
// share of row p: applying a measurement needs no communication inside the
// CTA or between CTAs.  The shares are folded once, at the end.
//
// Blocked measurements.  The X|Z bits a measurement leaves behind depend only
// on X|Z bits (never on signs or outcomes), and the pivot and the mask of rows
// with x_ha = 1 of measurement m depend only on the measured columns.  So a
// batch of K consecutive measurements runs in two phases:
//   phase 1: the measured columns of the batch (pushed by their owners at the
//            end of the previous batch) are replayed through the K
//            measurements, one warp per column, one named barrier per
//            measurement; this gives every measurement's pivot p_m and mask
//            S_m (the measured column at that time);
//   phase 2: every warp applies the K rowsums, in order, to its own columns
//            and its own share -- no barrier at all.
// One CTA barrier between the phases and one cluster/grid barrier per batch.
// A deterministic measurement with reset ends its batch (its outcome, needed
// for the reset, is only known once every share is summed).
//
// The communication policy decides how batches meet:
//   CommCluster -- one thread-block cluster: owners push the next batch's
//                  columns into every CTA's shared memory over DSMEM, and the
//                  hardware cluster barrier publishes them;
//   CommGrid    -- a cooperative grid: owners stage the next batch's columns
//                  in global memory (L2), bounded software grid barrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "grid_sync.cuh"
#include "philox.cuh"
#include "tab_internal.h"

namespace tab {

constexpr int kResThreads = 512;
constexpr int kResWarps = kResThreads / 32;
constexpr int kBatchMax = 32;
constexpr int kResMaxLocalCols = 32 * kResWarps;  // a warp's columns fit one ballot

struct ResArgs {
  uint32_t *X, *Z, *R;  // handle layout: W = 2*Wh words per column
  int n, Wh;
  const uint32_t* mops;
  int nm;
  uint64_t k0, seed, cid;
  uint32_t shot;
  uint8_t* out;
  int* err;
  int kb;  // measurements per batch (1..kBatchMax)
  // CommGrid workspace (global memory)
  uint32_t* stage;  // [2][kb][2][W] measured columns of the next batch
  uint32_t* dp;     // [2][kb][C] deterministic partials
  uint32_t* ph;     // [C][2][W] sign partials for the fold
  uint32_t* r4;     // [2][W] base signs for the fold
  GridBar* bar;
};

struct ResLayout {
  int ncl, Wp;
  size_t words;
};

__host__ __device__ inline ResLayout res_layout(int n, int Wh, int C, int kb) {
  ResLayout L;
  const int W = 2 * Wh;
  L.ncl = (n + C - 1) / C;
  L.Wp = W + 1;
  L.words = 2 * (size_t)L.ncl * L.Wp   // own X, Z columns
            + 4 * (size_t)W             // CTA sign partial (lo, hi), base signs (lo, hi)
            + (size_t)kb * W            // mask of each measurement of the batch
            + 4 * (size_t)kb * W        // measured columns X, Z, double-buffered
            + 2 * (size_t)kb * C;       // deterministic partials, double-buffered
  return L;
}

// Largest batch size (power of two <= cap <= kBatchMax) that fits `limit`
// bytes; 0 if even single measurements do not fit.
__host__ __device__ inline int res_batch_for(int n, int Wh, int C, size_t limit,
                                             int cap = kBatchMax) {
  if ((n + C - 1) / C > kResMaxLocalCols) return 0;
  for (int kb = cap; kb >= 1; kb >>= 1)
    if (res_layout(n, Wh, C, kb).words * 4 <= limit) return kb;
  return 0;
}

// Words per lane of a warp's register share: the smallest of 2, 4, 8, 16
// covering W = 2*Wh words (0 if W > 512).
__host__ __device__ inline int res_words_per_lane(int Wh) {
  const int W = 2 * Wh;
  for (int wl = 2; wl <= 16; wl *= 2)
    if (32 * wl >= W) return wl;
  return 0;
}

__device__ __forceinline__ void res_add4(uint32_t& l, uint32_t& h, uint32_t bl, uint32_t bh) {
  h ^= bh ^ (l & bl);
  l ^= bl;
}
__device__ __forceinline__ uint32_t res_prefix_xor_excl(uint32_t v) {
  uint32_t y = v << 1;
  y ^= y << 1;
  y ^= y << 2;
  y ^= y << 4;
  y ^= y << 8;
  y ^= y << 16;
  return y;
}
__device__ __forceinline__ void res_named_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Shared-memory pointers of the per-CTA state.
struct ResSmem {
  uint32_t *Xs, *Zs, *PHlo, *PHhi, *R4lo, *R4hi, *SM, *TX, *TZ, *dpv;
};

__device__ __forceinline__ ResSmem res_smem(uint32_t* sm, const ResLayout& Ly, int W, int kb) {
  ResSmem s;
  s.Xs = sm;
  s.Zs = s.Xs + (size_t)Ly.ncl * Ly.Wp;
  s.PHlo = s.Zs + (size_t)Ly.ncl * Ly.Wp;
  s.PHhi = s.PHlo + W;
  s.R4lo = s.PHhi + W;
  s.R4hi = s.R4lo + W;
  s.SM = s.R4hi + W;                  // [kb][W] mask of each measurement of the batch
  s.TX = s.SM + (size_t)kb * W;       // [2][kb][W] measured columns, X plane
  s.TZ = s.TX + 2 * (size_t)kb * W;   // [2][kb][W] Z plane
  s.dpv = s.TZ + 2 * (size_t)kb * W;  // [2][kb][C]
  return s;
}

// Per-batch bookkeeping in static shared memory.
struct ResBatch {
  uint32_t code[kBatchMax];  // measurement codes of the batch
  int slot[kBatchMax];       // measured-column slot of each measurement
  int q[kBatchMax];          // qubit of each slot
  int own[kBatchMax];        // slots whose column this CTA owns
  int P[kBatchMax];          // pivot row of each measurement (-1: deterministic)
  uint32_t rbit[kBatchMax];  // Philox outcome bit of each measurement
  uint32_t dacc[kBatchMax];  // this CTA's deterministic partial
  int ptype[kBatchMax];      // previous batch: 1 = deterministic
  int det[kBatchMax];        // previous batch: resolved deterministic outcome
  int D, nown, keff;
  uint32_t plast;            // code of the previous batch's last measurement
};

// Distinct measured qubits of the batch starting at m (first occurrence
// order) and the slots this CTA owns.  Thread 0 only.
__device__ __forceinline__ void res_batch_slots(const uint32_t* mops, int m, int K, int C, int r,
                                                ResBatch& b) {
  int D = 0;
  for (int i = 0; i < K; ++i) {
    b.code[i] = __ldg(mops + m + i);
    const int a = (int)dq1(b.code[i]);
    int d = 0;
    while (d < D && b.q[d] != a) ++d;
    if (d == D) b.q[D++] = a;
    b.slot[i] = d;
  }
  int no = 0;
  for (int d = 0; d < D; ++d)
    if (b.q[d] % C == r) b.own[no++] = d;
  b.D = D;
  b.nown = no;
}

template <int WL, class Comm>
__device__ void measure_resident(const ResArgs& A, Comm& cm, uint32_t* sm) {
  constexpr int NW = kResWarps;
  const int C = cm.size(), r = cm.rank(), tid = threadIdx.x, T = blockDim.x;
  const int n = A.n, Wh = A.Wh, W = 2 * Wh, KB = A.kb;
  const ResLayout Ly = res_layout(n, Wh, C, KB);
  const int Wp = Ly.Wp;
  const int nown = (n - r + C - 1) / C;  // columns owned: r, r+C, ...
  const ResSmem s = res_smem(sm, Ly, W, KB);
  const int lane = tid & 31, warp = tid >> 5;
  const int ncw = warp < nown ? (nown - warp + NW - 1) / NW : 0;  // this warp's columns
  const bool base_warp = (r == 0 && warp == 0);
  __shared__ ResBatch b;

  // this warp's share of every row's sign exponent (lo, hi bit planes)
  uint32_t plo[WL], phi[WL];
#pragma unroll
  for (int k = 0; k < WL; ++k) plo[k] = phi[k] = 0u;

  // ---- load own columns, base signs
  for (int i = tid; i < nown * W; i += T) {
    const int lj = i / W, w = i - lj * W;
    const size_t g = (size_t)(r + lj * C) * W + w;
    s.Xs[(size_t)lj * Wp + w] = A.X[g];
    s.Zs[(size_t)lj * Wp + w] = A.Z[g];
  }
  for (int w = tid; w < W; w += T) {
    s.R4lo[w] = 0u;
    s.R4hi[w] = (r == 0) ? A.R[w] : 0u;
  }
  if (tid == 0) {  // slots of the first batch
    const int K0 = A.nm < KB ? A.nm : KB;
    res_batch_slots(A.mops, 0, K0, C, r, b);
  }
  if (!cm.start()) return;
  cm.stage_columns(s, 0, b, W, Wp, KB);  // first batch's measured columns

  int m = 0, batch = 0, prev_base = 0, prev_count = 0;
  while (m < A.nm) {
    const int par = batch & 1;
    const int K = (A.nm - m < KB) ? A.nm - m : KB;
    // ---- barrier: the previous batch's column updates, staged columns and
    // deterministic partials are visible everywhere
    if (!cm.sync()) return;
    // ---- resolve the previous batch's deterministic outcomes
    if (tid < prev_count && b.ptype[tid]) {
      const uint32_t e = cm.sum_dp(s.dpv, par ^ 1, tid, KB) & 3u;
      if (e & 1u) atomicCAS(A.err, 0, DERR_PHASE);
      b.det[tid] = (int)(e >> 1);
      if (r == 0) A.out[prev_base + tid] = (uint8_t)(e >> 1);
    }
    cm.gather_columns(s, par, b, W, KB);
    if (tid < K) b.rbit[tid] = outcome_bit(A.seed, A.cid, A.shot, A.k0 + (uint64_t)(m + tid));
    if (tid < KB) b.dacc[tid] = 0u;
    if (tid == 0) b.keff = K;
    __syncthreads();
    // a deterministic measure-and-reset ends its batch, so only the last
    // measurement of the previous batch can need its X_a: every sign ^= z_a,
    // added to the share of the warp that owns column a
    if (prev_count > 0 && b.ptype[prev_count - 1] && b.det[prev_count - 1] &&
        dop(b.plast) == OP_MZR) {
      const int pa = (int)dq1(b.plast);
      if (pa % C == r && (pa / C) % NW == warp) {
        const uint32_t* zc = s.Zs + (size_t)(pa / C) * Wp;
#pragma unroll
        for (int k = 0; k < WL; ++k) {
          const int w = lane + 32 * k;
          if (w < W) phi[k] ^= zc[w];
        }
      }
    }

    // ---- phase 1: replay the K measurements on the measured columns only
    const int D = b.D;
    const int np1 = D < NW ? D : NW;
    uint32_t* TXp = s.TX + (size_t)par * KB * W;
    uint32_t* TZp = s.TZ + (size_t)par * KB * W;
    if (warp < np1) {
      for (int i = 0; i < K; ++i) {
        const uint32_t code = b.code[i];
        const int a = (int)dq1(code);
        const int d0 = b.slot[i];
        uint32_t* Si = s.SM + (size_t)i * W;
        if (d0 % NW == warp)
          for (int w = lane; w < W; w += 32) Si[w] = TXp[(size_t)d0 * W + w];
        res_named_sync(1, 32 * np1);
        int pw = -1;
        for (int base = 0; base < Wh && pw < 0; base += 32) {
          const int hw = base + lane;
          const uint32_t bal = __ballot_sync(0xffffffffu, hw < Wh && Si[Wh + hw] != 0u);
          if (bal) pw = Wh + base + __ffs(bal) - 1;
        }
        const int P = pw < 0 ? -1 : pw * 32 + __ffs(Si[pw]) - 1;
        if (warp == 0 && lane == 0) b.P[i] = P;
        if (P < 0) {  // deterministic: X|Z unchanged; with reset the batch ends
          if (dop(code) == OP_MZR) {
            if (warp == 0 && lane == 0) b.keff = i + 1;
            break;
          }
          continue;
        }
        const int wp = P >> 5, wd = (P - 32 * Wh) >> 5;
        const uint32_t bpm = 1u << (P & 31);
        for (int d = warp; d < D; d += NW) {
          uint32_t* tx = TXp + (size_t)d * W;
          uint32_t* tz = TZp + (size_t)d * W;
          const uint32_t XP = (tx[wp] & bpm) ? 0xffffffffu : 0u;
          const uint32_t ZP = (tz[wp] & bpm) ? 0xffffffffu : 0u;
          const bool is_a = b.q[d] == a;
          __syncwarp();
          for (int w = lane; w < W; w += 32) {
            uint32_t Sw = Si[w];
            if (w == wp || w == wd) Sw &= ~bpm;
            uint32_t x = tx[w] ^ (Sw & XP), z = tz[w] ^ (Sw & ZP);
            if (w == wd) {  // row p-n := row p
              x = (x & ~bpm) | (XP & bpm);
              z = (z & ~bpm) | (ZP & bpm);
            }
            if (w == wp) {  // row p := Z_a
              x &= ~bpm;
              z = (z & ~bpm) | (is_a ? bpm : 0u);
            }
            tx[w] = x;
            tz[w] = z;
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    const int keff = b.keff;
    if (r == 0 && tid < keff && b.P[tid] >= 0) A.out[m + tid] = (uint8_t)b.rbit[tid];

    // ---- phase 2: every warp applies the batch to its columns and its share
    for (int i = 0; i < keff; ++i) {
      const uint32_t code = b.code[i];
      const int a = (int)dq1(code);
      const int P = b.P[i];
      const uint32_t* S = s.SM + (size_t)i * W;
      __syncwarp();  // the previous measurement's column writes, across lanes
      if (P >= 0) {
        // ============ random outcome ============
        const uint32_t rbit = b.rbit[i];
        const int wp = P >> 5, wd = (P - 32 * Wh) >> 5;
        const uint32_t bpm = 1u << (P & 31);
        // this warp's share of 2 r_p (and the base, for the base warp)
        uint32_t pl = 0u, ph = 0u;
#pragma unroll
        for (int k = 0; k < WL; ++k) {  // mask select: keeps the shares in registers
          const uint32_t sel = 0u - (uint32_t)(k == (wp >> 5));
          pl |= plo[k] & sel;
          ph |= phi[k] & sel;
        }
        pl = __shfl_sync(0xffffffffu, pl, wp & 31);
        ph = __shfl_sync(0xffffffffu, ph, wp & 31);
        const uint32_t php = ((pl & bpm) ? 1u : 0u) | ((ph & bpm) ? 2u : 0u);
        uint32_t r4p = 0u;
        if (base_warp) r4p = ((s.R4lo[wp] & bpm) ? 1u : 0u) | ((s.R4hi[wp] & bpm) ? 2u : 0u);
        // pivot row over this warp's columns (lane c: column warp + 16 c)
        bool xb = false, zb = false;
        if (lane < ncw) {
          const size_t ii = (size_t)(warp + lane * NW) * Wp + wp;
          xb = (s.Xs[ii] & bpm) != 0u;
          zb = (s.Zs[ii] & bpm) != 0u;
        }
        const uint32_t supx = __ballot_sync(0xffffffffu, xb);
        const uint32_t supz = __ballot_sync(0xffffffffu, zb);
        if (lane < ncw && !xb && !zb) {  // row p is I here: row p-n := row p clears it
          const size_t ii = (size_t)(warp + lane * NW) * Wp + wd;
          s.Xs[ii] &= ~bpm;
          s.Zs[ii] &= ~bpm;
        }
        __syncwarp();
        const int la = (a % C == r) ? a / C : -1;  // local column of qubit a
        const uint32_t scal = ((uint32_t)__popc(supx & supz) + php + r4p) & 3u;
        const uint32_t sup = supx | supz;
#pragma unroll
        for (int k = 0; k < WL; ++k) {
          const int w = lane + 32 * k;
          if (w < W) {
            uint32_t Sw = S[w];
            if (w == wp || w == wd) Sw &= ~bpm;  // S' excludes rows p and p-n
            uint32_t lo = plo[k], hi = phi[k];
            for (uint32_t left = sup; left; left &= left - 1u) {
              const int c = __ffs(left) - 1;
              const uint32_t XP = 0u - ((supx >> c) & 1u), ZP = 0u - ((supz >> c) & 1u);
              const int lj = warp + c * NW;
              const size_t ii = (size_t)lj * Wp + w;
              const uint32_t x = s.Xs[ii], z = s.Zs[ii];
              const uint32_t A0 = x & z, B0 = (x ^ XP) & (z ^ ZP);
              const uint32_t inc = A0 & ~B0 & Sw, dec = B0 & ~A0 & Sw;
              hi ^= ((lo & inc) | (~lo & dec)) ^ (ZP & x & Sw);
              lo ^= inc | dec;
              uint32_t xn = x ^ (XP & Sw), zn = z ^ (ZP & Sw);
              if (w == wd) {  // row p-n := row p
                xn = (xn & ~bpm) | (XP & bpm);
                zn = (zn & ~bpm) | (ZP & bpm);
              }
              if (w == wp) {  // row p := Z_a
                xn &= ~bpm;
                zn = (zn & ~bpm) | ((lj == la) ? bpm : 0u);
              }
              s.Xs[ii] = xn;
              s.Zs[ii] = zn;
            }
            // this warp's share of 2 r_p and of sum_j x_pj z_pj, on every row in S'
            res_add4(lo, hi, (scal & 1u) ? Sw : 0u, (scal & 2u) ? Sw : 0u);
            if (w == wd) {  // share of row p-n := share of row p
              lo = (lo & ~bpm) | ((php & 1u) ? bpm : 0u);
              hi = (hi & ~bpm) | ((php & 2u) ? bpm : 0u);
            }
            if (w == wp) {  // row p := (-1)^b Z_a: shares 0, base 2b
              lo &= ~bpm;
              hi &= ~bpm;
            }
            plo[k] = lo;
            phi[k] = hi;
          }
        }
        if (dop(code) == OP_MZR && rbit && la >= 0 && la % NW == warp) {
          __syncwarp();  // reset: X_a on every row, sign ^= z_a
          const uint32_t* zc = s.Zs + (size_t)la * Wp;
#pragma unroll
          for (int k = 0; k < WL; ++k) {
            const int w = lane + 32 * k;
            if (w < W) phi[k] ^= zc[w];
          }
        }
        if (base_warp) {
          __syncwarp();
          if (lane == 0) {
            s.R4lo[wd] = (s.R4lo[wd] & ~bpm) | ((r4p & 1u) ? bpm : 0u);
            s.R4hi[wd] = (s.R4hi[wd] & ~bpm) | ((r4p & 2u) ? bpm : 0u);
            s.R4lo[wp] &= ~bpm;
            s.R4hi[wp] = (s.R4hi[wp] & ~bpm) | (rbit ? bpm : 0u);
          }
          __syncwarp();
        }
      } else {
        // ============ deterministic outcome: this warp's partial ============
        uint32_t acc = 0u;
#pragma unroll
        for (int k = 0; k < WL; ++k) {
          const int w = lane + 32 * k;
          if (w >= Wh && w < W) {
            const uint32_t t = S[w - Wh];
            acc += __popc(plo[k] & t) + 2u * __popc(phi[k] & t);
            if (base_warp) acc += __popc(s.R4lo[w] & t) + 2u * __popc(s.R4hi[w] & t);
          }
        }
        const uint32_t lt = (1u << lane) - 1u;
        for (int c = 0; c < ncw; ++c) {
          const size_t col = (size_t)(warp + c * NW) * Wp + Wh;
          uint32_t carry = 0u;
          for (int base = 0; base < Wh; base += 32) {
            const int hw = base + lane;
            uint32_t xT = 0u, zT = 0u;
            if (hw < Wh) {
              const uint32_t t = S[hw];
              xT = s.Xs[col + hw] & t;
              zT = s.Zs[col + hw] & t;
            }
            acc += __popc(xT & zT);
            const uint32_t bal = __ballot_sync(0xffffffffu, __popc(zT) & 1);
            const uint32_t cin = (__popc(bal & lt) & 1u) ^ carry;
            const uint32_t zpre = res_prefix_xor_excl(zT) ^ (cin ? 0xffffffffu : 0u);
            acc += 2u * (__popc(xT & zpre) & 1u);
            carry ^= __popc(bal) & 1u;
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && (acc & 3u)) atomicAdd(&b.dacc[i], acc & 3u);
      }
    }
    __syncthreads();

    // ---- publish the deterministic partials; bookkeeping for the next batch
    for (int i = 0; i < keff; ++i)
      if (b.P[i] < 0) cm.publish_dp(s.dpv, par, i, KB, b.dacc[i] & 3u);
    __syncthreads();
    if (tid < keff) b.ptype[tid] = b.P[tid] < 0;
    __syncthreads();
    if (tid == 0) {
      b.plast = b.code[keff - 1];
      const int mn = m + keff;
      const int Kn = (A.nm - mn < KB) ? A.nm - mn : KB;
      if (Kn > 0) res_batch_slots(A.mops, mn, Kn, C, r, b);
      else b.D = b.nown = 0;
    }
    __syncthreads();
    cm.stage_columns(s, par ^ 1, b, W, Wp, KB);  // next batch's measured columns
    prev_base = m;
    prev_count = keff;
    m += keff;
    ++batch;
  }

  // ---- epilogue: last batch's deterministic outcomes, fold, write back
  if (!cm.sync()) return;
  {
    const int par = batch & 1;
    if (tid < prev_count && b.ptype[tid]) {
      const uint32_t e = cm.sum_dp(s.dpv, par ^ 1, tid, KB) & 3u;
      if (e & 1u) atomicCAS(A.err, 0, DERR_PHASE);
      b.det[tid] = (int)(e >> 1);
      if (r == 0) A.out[prev_base + tid] = (uint8_t)(e >> 1);
    }
  }
  for (int w = tid; w < W; w += T) {
    s.PHlo[w] = 0u;
    s.PHhi[w] = 0u;
  }
  __syncthreads();
  if (prev_count > 0 && b.ptype[prev_count - 1] && b.det[prev_count - 1] &&
      dop(b.plast) == OP_MZR) {
    const int pa = (int)dq1(b.plast);
    if (pa % C == r && (pa / C) % NW == warp) {
      const uint32_t* zc = s.Zs + (size_t)(pa / C) * Wp;
#pragma unroll
      for (int k = 0; k < WL; ++k) {
        const int w = lane + 32 * k;
        if (w < W) phi[k] ^= zc[w];
      }
    }
  }
  // the CTA's share: sum of its warps' shares (mod 4).  A bit-sliced add
  // through two atomic XORs is exact under any interleaving: the carry uses
  // the low plane as the atomic returned it, so the adds serialise in the
  // order of the low-plane atomics, and the high plane only takes XORs.
#pragma unroll
  for (int k = 0; k < WL; ++k) {
    const int w = lane + 32 * k;
    if (w < W && (plo[k] | phi[k])) {
      const uint32_t old = atomicXor(&s.PHlo[w], plo[k]);
      atomicXor(&s.PHhi[w], phi[k] ^ (old & plo[k]));
    }
  }
  __syncthreads();
  if (!cm.fold(s, W, A)) return;
  for (int i = tid; i < nown * W; i += T) {
    const int lj = i / W, w = i - lj * W;
    const size_t g = (size_t)(r + lj * C) * W + w;
    A.X[g] = s.Xs[(size_t)lj * Wp + w];
    A.Z[g] = s.Zs[(size_t)lj * Wp + w];
  }
  cm.finish();
}

}  // namespace tab
