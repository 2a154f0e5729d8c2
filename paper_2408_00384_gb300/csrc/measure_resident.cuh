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
// CTA r of C owns the columns j = r, r+C, r+2C, ... in shared memory (column
// stride W+1, odd, so lanes over words and lanes over columns are both bank
// conflict free), together with its own mod-4 sign partials; CTA 0 also keeps
// the base signs.  The true sign of row h is (base + sum_r partial_r) / 2,
// linear in each CTA's share, so a CTA only ever adds its own columns' share
// of a rowsum exponent and nothing is exchanged until the final fold.
//
// Blocked measurements.  The X|Z bits a measurement leaves behind depend only
// on X|Z bits (never on signs or outcomes), and the pivot and the mask of rows
// with x_ha = 1 of measurement m depend only on the measured columns.  So a
// batch of K consecutive measurements runs in two phases:
//   phase 1: every CTA copies the batch's measured columns and replays the K
//            measurements on those columns alone, which gives every
//            measurement's pivot p_m and mask S_m (the column at that time);
//   phase 2: each CTA applies the K rowsums, in order, to its own columns and
//            its own sign partials -- with no communication at all.
// One barrier per batch replaces one per measurement.  A deterministic
// measurement with reset ends its batch (its outcome, needed for the reset,
// is only known once every CTA's partial is in).
//
// The communication policy decides how batches meet:
//   CommCluster -- one thread-block cluster: measured columns are read from
//                  their owners' shared memory over DSMEM, hardware barrier;
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
constexpr int kBatchMax = 32;

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
  int ncl, Wp, GG;
  size_t words;
};

__host__ __device__ inline ResLayout res_layout(int n, int Wh, int C, int kb) {
  ResLayout L;
  const int W = 2 * Wh;
  L.ncl = (n + C - 1) / C;
  L.Wp = W + 1;
  L.GG = kResThreads / W;
  if (L.GG < 1) L.GG = 1;
  L.words = (size_t)2 * L.ncl * L.Wp   // own X, Z columns
            + 4 * (size_t)W             // own sign partials (lo, hi), base signs (lo, hi)
            + 3 * (size_t)kb * W        // batch masks, tracked X and Z columns
            + 2 * (size_t)kb * C        // deterministic partials, double-buffered
            + (size_t)L.ncl             // support list
            + 2 * (size_t)L.GG * W      // group counters
            + (size_t)W;                // new Z column of the measured qubit
  return L;
}

// Largest batch size (power of two <= cap <= kBatchMax) that fits `limit`
// bytes; 0 if even single measurements do not fit.
__host__ __device__ inline int res_batch_for(int n, int Wh, int C, size_t limit,
                                             int cap = kBatchMax) {
  for (int kb = cap; kb >= 1; kb >>= 1)
    if (res_layout(n, Wh, C, kb).words * 4 <= limit) return kb;
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

// Shared-memory pointers of the per-CTA state.
struct ResSmem {
  uint32_t *Xs, *Zs, *PHlo, *PHhi, *R4lo, *R4hi, *SM, *TX, *TZ, *dpv, *supp, *redlo, *redhi, *zA;
};

__device__ __forceinline__ ResSmem res_smem(uint32_t* sm, const ResLayout& Ly, int W, int C, int kb) {
  ResSmem s;
  s.Xs = sm;
  s.Zs = s.Xs + (size_t)Ly.ncl * Ly.Wp;
  s.PHlo = s.Zs + (size_t)Ly.ncl * Ly.Wp;
  s.PHhi = s.PHlo + W;
  s.R4lo = s.PHhi + W;
  s.R4hi = s.R4lo + W;
  s.SM = s.R4hi + W;            // [kb][W] mask of each measurement of the batch
  s.TX = s.SM + (size_t)kb * W; // [kb][W] tracked measured columns, X plane
  s.TZ = s.TX + (size_t)kb * W; // [kb][W] Z plane
  s.dpv = s.TZ + (size_t)kb * W;  // [2][kb][C]
  s.supp = s.dpv + 2 * (size_t)kb * C;
  s.redlo = s.supp + Ly.ncl;
  s.redhi = s.redlo + (size_t)Ly.GG * W;
  s.zA = s.redhi + (size_t)Ly.GG * W;
  return s;
}

// Distinct measured qubits of the batch starting at m (first occurrence
// order): code[i] and slot[i] for each measurement, q[d] for each slot.
// Thread 0 only.
__device__ __forceinline__ int res_batch_slots(const uint32_t* mops, int m, int K, uint32_t* code,
                                               int* slot, int* q) {
  int D = 0;
  for (int i = 0; i < K; ++i) {
    code[i] = __ldg(mops + m + i);
    const int a = (int)dq1(code[i]);
    int d = 0;
    while (d < D && q[d] != a) ++d;
    if (d == D) q[D++] = a;
    slot[i] = d;
  }
  return D;
}

template <class Comm>
__device__ void measure_resident(const ResArgs& A, Comm& cm, uint32_t* sm) {
  const int C = cm.size(), r = cm.rank(), tid = threadIdx.x, T = blockDim.x;
  const int n = A.n, Wh = A.Wh, W = 2 * Wh, KB = A.kb;
  const ResLayout Ly = res_layout(n, Wh, C, KB);
  const int Wp = Ly.Wp, GG = Ly.GG;
  const int nown = (n - r + C - 1) / C;  // columns owned: r, r+C, ...
  const ResSmem s = res_smem(sm, Ly, W, C, KB);
  const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  __shared__ int s_nsupp, s_kc, s_keff, s_D, s_det;
  __shared__ uint32_t s_php, s_r4p, s_acc;
  __shared__ int s_slot[kBatchMax], s_q[kBatchMax], s_P[kBatchMax];
  __shared__ uint32_t s_xp[kBatchMax], s_zp[kBatchMax], s_code[kBatchMax];
  __shared__ int s_ptype[kBatchMax];  // previous batch: 1 = deterministic

  // ---- load own columns, zero partials
  for (int i = tid; i < nown * W; i += T) {
    const int lj = i / W, w = i - lj * W;
    const size_t g = (size_t)(r + lj * C) * W + w;
    s.Xs[(size_t)lj * Wp + w] = A.X[g];
    s.Zs[(size_t)lj * Wp + w] = A.Z[g];
  }
  for (int w = tid; w < W; w += T) {
    s.PHlo[w] = 0u;
    s.PHhi[w] = 0u;
    s.R4lo[w] = 0u;
    s.R4hi[w] = (r == 0) ? A.R[w] : 0u;
  }
  if (tid == 0) {  // slots of the first batch
    const int K0 = A.nm < KB ? A.nm : KB;
    s_D = A.nm > 0 ? res_batch_slots(A.mops, 0, K0, s_code, s_slot, s_q) : 0;
  }
  __syncthreads();
  cm.stage_columns(s, 0, 0, s_D, s_q, W, Wp, A);  // (grid) first batch's columns

  int m = 0, batch = 0, prev_base = 0, prev_count = 0;
  while (m < A.nm) {
    const int par = batch & 1;
    const int K = (A.nm - m < KB) ? A.nm - m : KB;
    // ---- barrier: the previous batch's column updates, staged columns and
    // deterministic partials are visible everywhere
    if (!cm.sync()) return;
    // ---- resolve the previous batch's deterministic outcomes
    for (int i = 0; i < prev_count; ++i) {
      if (!s_ptype[i]) continue;
      if (tid == 0) {
        const uint32_t e = cm.sum_dp(s.dpv, par ^ 1, i, KB) & 3u;
        if (e & 1u) atomicCAS(A.err, 0, DERR_PHASE);
        s_det = (int)(e >> 1);
        if (r == 0) A.out[prev_base + i] = (uint8_t)s_det;
      }
      __syncthreads();
      const uint32_t pc = __ldg(A.mops + prev_base + i);
      const int pa = (int)dq1(pc);
      if (dop(pc) == OP_MZR && s_det && pa % C == r) {  // X on pa: every sign ^= z
        const uint32_t* zc = s.Zs + (size_t)(pa / C) * Wp;
        for (int w = tid; w < W; w += T) s.PHhi[w] ^= zc[w];
      }
      __syncthreads();
    }
    // ---- gather the batch's measured columns (state after the last batch)
    const int D = s_D;
    cm.gather_columns(s, par, D, s_q, W, Wp, A);
    if (!cm.after_gather()) return;

    // ---- phase 1: replay the K measurements on the measured columns only
    if (tid == 0) s_keff = K;
    __syncthreads();
    for (int i = 0; i < K; ++i) {
      const uint32_t code = s_code[i];
      const int a = (int)dq1(code);
      const int d0 = s_slot[i];
      uint32_t* Si = s.SM + (size_t)i * W;
      for (int w = tid; w < W; w += T) Si[w] = s.TX[(size_t)d0 * W + w];
      __syncthreads();
      if (warp == 0) {
        int pw = -1;
        for (int base = 0; base < Wh && pw < 0; base += 32) {
          const int hw = base + lane;
          const uint32_t bal = __ballot_sync(0xffffffffu, hw < Wh && Si[Wh + hw] != 0u);
          if (bal) pw = Wh + base + __ffs(bal) - 1;
        }
        if (lane == 0) s_P[i] = pw < 0 ? -1 : pw * 32 + __ffs(Si[pw]) - 1;
      }
      __syncthreads();
      const int P = s_P[i];
      if (P < 0) {  // deterministic: X|Z unchanged; with reset the batch ends
        if (dop(code) == OP_MZR) {
          if (tid == 0) s_keff = i + 1;
          break;
        }
        continue;
      }
      const int wp = P >> 5, wd = (P - 32 * Wh) >> 5;
      const uint32_t bpm = 1u << (P & 31);
      if (tid < D) {
        s_xp[tid] = (s.TX[(size_t)tid * W + wp] & bpm) ? 0xffffffffu : 0u;
        s_zp[tid] = (s.TZ[(size_t)tid * W + wp] & bpm) ? 0xffffffffu : 0u;
      }
      __syncthreads();
      for (int e = tid; e < D * W; e += T) {
        const int d = e / W, w = e - d * W;
        const uint32_t XP = s_xp[d], ZP = s_zp[d];
        uint32_t Sw = Si[w];
        if (w == wp || w == wd) Sw &= ~bpm;
        uint32_t tx = s.TX[e] ^ (Sw & XP), tz = s.TZ[e] ^ (Sw & ZP);
        if (w == wd) {
          tx = (tx & ~bpm) | (XP & bpm);
          tz = (tz & ~bpm) | (ZP & bpm);
        }
        if (w == wp) {
          tx &= ~bpm;
          tz = (tz & ~bpm) | ((s_q[d] == a) ? bpm : 0u);
        }
        s.TX[e] = tx;
        s.TZ[e] = tz;
      }
      __syncthreads();
    }
    __syncthreads();
    const int keff = s_keff;

    // ---- phase 2: apply the batch's measurements to own columns, in order
    for (int i = 0; i < keff; ++i) {
      const uint32_t code = s_code[i];
      const int a = (int)dq1(code);
      const bool reset = dop(code) == OP_MZR;
      const uint32_t rbit = outcome_bit(A.seed, A.cid, A.shot, A.k0 + (uint64_t)(m + i));
      const uint32_t* S = s.SM + (size_t)i * W;
      const int P = s_P[i];
      if (tid == 0) {
        s_nsupp = 0;
        s_kc = 0;
        s_acc = 0u;
      }
      __syncthreads();
      if (P >= 0) {
        // ============ random outcome ============
        const int Pd = P - 32 * Wh;
        const int wp = P >> 5, wd = Pd >> 5;
        const uint32_t bpm = 1u << (P & 31);
        if (tid == 0) {
          s_php = ((s.PHlo[wp] & bpm) ? 1u : 0u) | ((s.PHhi[wp] & bpm) ? 2u : 0u);
          s_r4p = ((s.R4lo[wp] & bpm) ? 1u : 0u) | ((s.R4hi[wp] & bpm) ? 2u : 0u);
        }
        // support list of the pivot row over own columns (warp-aggregated)
        for (int l0 = tid - lane; l0 < nown; l0 += T) {
          const int lj = l0 + lane;
          uint32_t xp = 0u, zp = 0u;
          if (lj < nown) {
            xp = (s.Xs[(size_t)lj * Wp + wp] & bpm) ? 1u : 0u;
            zp = (s.Zs[(size_t)lj * Wp + wp] & bpm) ? 1u : 0u;
          }
          const uint32_t in = __ballot_sync(0xffffffffu, (xp | zp) != 0u);
          const uint32_t yy = __ballot_sync(0xffffffffu, (xp & zp) != 0u);
          int pos = 0;
          if (lane == 0 && in) {
            pos = atomicAdd(&s_nsupp, __popc(in));
            if (yy) atomicAdd(&s_kc, __popc(yy));
          }
          pos = __shfl_sync(0xffffffffu, pos, 0);
          if (xp | zp) {
            s.supp[pos + __popc(in & ((1u << lane) - 1u))] = (uint32_t)lj | (xp << 30) | (zp << 31);
          } else if (lj < nown) {  // row p is I here: row p-n := row p clears this bit
            s.Xs[(size_t)lj * Wp + wd] &= ~bpm;
            s.Zs[(size_t)lj * Wp + wd] &= ~bpm;
          }
        }
        __syncthreads();
        const int nsupp = s_nsupp;
        const int g = tid / W, w = tid - g * W;
        const int la = (a % C == r) ? a / C : -1;
        if (g < GG) {
          uint32_t lo = 0u, hi = 0u;
          uint32_t Sw = S[w];
          if (w == wp || w == wd) Sw &= ~bpm;  // S' excludes rows p and p-n
          for (int idx = g; idx < nsupp; idx += GG) {
            const uint32_t e = s.supp[idx];
            const int lj = (int)(e & 0x3FFFu);
            const uint32_t XP = (e & (1u << 30)) ? 0xffffffffu : 0u;
            const uint32_t ZP = (e & (1u << 31)) ? 0xffffffffu : 0u;
            const size_t ii = (size_t)lj * Wp + w;
            const uint32_t x = s.Xs[ii], z = s.Zs[ii];
            const uint32_t A0 = x & z, B0 = (x ^ XP) & (z ^ ZP);
            const uint32_t inc = A0 & ~B0, dec = B0 & ~A0;
            hi ^= ((lo & inc) | (~lo & dec)) ^ (ZP & x);
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
            if (lj == la) s.zA[w] = zn;
          }
          s.redlo[g * W + w] = lo;
          s.redhi[g * W + w] = hi;
        }
        __syncthreads();
        if (tid < W) {
          const int ww = tid;
          uint32_t L = 0u, H = 0u;
          for (int gg = 0; gg < GG; ++gg) res_add4(L, H, s.redlo[gg * W + ww], s.redhi[gg * W + ww]);
          // this CTA's share of 2 r_p (its partial of row p, plus the base for
          // CTA 0) and of sum_j x_pj z_pj, added to every row in S'
          uint32_t scal = (uint32_t)s_kc + (s_php & 1u) + 2u * (s_php >> 1);
          if (r == 0) scal += (s_r4p & 1u) + 2u * (s_r4p >> 1);
          scal &= 3u;
          res_add4(L, H, (scal & 1u) ? 0xffffffffu : 0u, (scal & 2u) ? 0xffffffffu : 0u);
          uint32_t Sw = S[ww];
          if (ww == wp || ww == wd) Sw &= ~bpm;
          L &= Sw;
          H &= Sw;
          uint32_t pl = s.PHlo[ww], ph = s.PHhi[ww];
          res_add4(pl, ph, L, H);
          if (ww == wd) {  // sign share of row p-n := that of row p
            pl = (pl & ~bpm) | ((s_php & 1u) ? bpm : 0u);
            ph = (ph & ~bpm) | ((s_php & 2u) ? bpm : 0u);
          }
          if (ww == wp) {
            pl &= ~bpm;
            ph &= ~bpm;
          }
          if (la >= 0 && reset && rbit) ph ^= s.zA[ww];  // reset: X_a on every row
          s.PHlo[ww] = pl;
          s.PHhi[ww] = ph;
          if (r == 0 && (ww == wp || ww == wd)) {
            uint32_t bl = s.R4lo[ww], bh = s.R4hi[ww];
            if (ww == wd) {
              bl = (bl & ~bpm) | ((s_r4p & 1u) ? bpm : 0u);
              bh = (bh & ~bpm) | ((s_r4p & 2u) ? bpm : 0u);
            } else {
              bl &= ~bpm;
              bh = (bh & ~bpm) | (rbit ? bpm : 0u);
            }
            s.R4lo[ww] = bl;
            s.R4hi[ww] = bh;
          }
        }
        if (r == 0 && tid == 0) A.out[m + i] = (uint8_t)rbit;
      } else {
        // ============ deterministic outcome: this CTA's partial ============
        uint32_t acc = 0u;
        for (int hw = tid; hw < Wh; hw += T) {
          const uint32_t t = S[hw];
          acc += __popc(s.PHlo[Wh + hw] & t) + 2u * __popc(s.PHhi[Wh + hw] & t);
          if (r == 0) acc += __popc(s.R4lo[Wh + hw] & t) + 2u * __popc(s.R4hi[Wh + hw] & t);
        }
        const uint32_t lt = (1u << lane) - 1u;
        for (int lj = warp; lj < nown; lj += nw) {
          uint32_t carry = 0u;
          for (int base = 0; base < Wh; base += 32) {
            const int hw = base + lane;
            uint32_t xT = 0u, zT = 0u;
            if (hw < Wh) {
              const uint32_t t = S[hw];
              xT = s.Xs[(size_t)lj * Wp + Wh + hw] & t;
              zT = s.Zs[(size_t)lj * Wp + Wh + hw] & t;
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
        if (lane == 0) atomicAdd(&s_acc, acc & 3u);
        __syncthreads();
        cm.publish_dp(s.dpv, par, i, KB, s_acc & 3u);
      }
      __syncthreads();
    }

    // ---- bookkeeping for the next batch
    if (tid == 0) {
      for (int i = 0; i < keff; ++i) s_ptype[i] = s_P[i] < 0;
      const int mn = m + keff;
      const int Kn = (A.nm - mn < KB) ? A.nm - mn : KB;
      s_D = Kn > 0 ? res_batch_slots(A.mops, mn, Kn, s_code, s_slot, s_q) : 0;
    }
    __syncthreads();
    cm.stage_columns(s, par ^ 1, 1, s_D, s_q, W, Wp, A);  // (grid) next batch's columns
    prev_base = m;
    prev_count = keff;
    m += keff;
    ++batch;
  }

  // ---- epilogue: last batch's deterministic outcomes, fold, write back
  if (!cm.sync()) return;
  const int par = batch & 1;
  for (int i = 0; i < prev_count; ++i) {
    if (!s_ptype[i]) continue;
    if (tid == 0) {
      const uint32_t e = cm.sum_dp(s.dpv, par ^ 1, i, KB) & 3u;
      if (e & 1u) atomicCAS(A.err, 0, DERR_PHASE);
      s_det = (int)(e >> 1);
      if (r == 0) A.out[prev_base + i] = (uint8_t)s_det;
    }
    __syncthreads();
    const uint32_t pc = __ldg(A.mops + prev_base + i);
    const int pa = (int)dq1(pc);
    if (dop(pc) == OP_MZR && s_det && pa % C == r) {
      const uint32_t* zc = s.Zs + (size_t)(pa / C) * Wp;
      for (int w = tid; w < W; w += T) s.PHhi[w] ^= zc[w];
    }
    __syncthreads();
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
