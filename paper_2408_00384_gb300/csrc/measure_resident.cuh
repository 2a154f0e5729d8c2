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
// memory; within the CTA, warp v owns a contiguous block of them.  The sign
// exponent 2 r_h (mod 4) of every row is kept as a sum of shares: one base
// (CTA 0, warp 0) plus one share per warp, held in that warp's registers
// (bit-sliced, lane l holds words l, l+32, ...).  Every term of the rowsum
// exponent is a sum over columns, and "2 r_p" is the sum of the shares of
// row p, so a warp adds only its own columns' terms and its own share of
// row p: applying a measurement needs no communication inside the CTA or
// between CTAs.  The shares are folded once, at the end.
//
// Per column j of the pivot row, (x_pj, z_pj) is X, Z or Y (or I: nothing to
// do), and the exponent terms of a row h in S' reduce to (with a mod-4
// counter lo + 2 hi per row):
//   X: +1 if x_hj z_hj, -1 if !x_hj z_hj              ; x_hj ^= 1
//   Z: +1 if x_hj z_hj, -1 if x_hj !z_hj, +2 if x_hj  ; z_hj ^= 1
//   Y: +1 if x_hj z_hj, -1 if !x_hj !z_hj, +2 if x_hj ; x_hj ^= 1, z_hj ^= 1
// which is what the three column kernels below add, 32 rows per word.
//
// Blocked measurements.  The X|Z bits a measurement leaves behind depend only
// on X|Z bits (never on signs or outcomes), and the pivot and the mask of rows
// with x_ha = 1 of measurement m depend only on the X bits of the measured
// columns: a column's X bits change only through the X bits of the mask and
// of row p (x_hc ^= x_pc for h in S', row p-n := row p, x_pc := 0).  So a
// batch of K consecutive measurements runs in two overlapping phases:
//   phase 1: the X bits of the batch's measured columns (staged by their
//            owners at the end of the previous batch) are copied into shared
//            memory and replayed through the K measurements: a chain warp
//            finds each pivot p_m on the measured column, publishes p_m and
//            the mask S_m (the measured column at that time) with a release
//            store of a counter and applies measurement m to the next two
//            measured columns in registers; helper warps apply it to the
//            other columns still measured later in the batch;
//   phase 2: the CTA's A apply warps, each owning a contiguous block of the
//            CTA's columns, apply the K rowsums, in order, to their columns
//            and their shares, each as soon as the counter shows it published
//            (an acquire load, a bounded wait); the replay and apply warps
//            run concurrently.
// One CTA barrier and one grid barrier per batch.  A deterministic
// measurement with reset ends its batch (its outcome, needed for the reset,
// is only known once every share is summed).  The communication policy
// (CommGrid, kernels_resident.cu) stages the next batch's columns in global
// memory (L2) and meets at a bounded software grid barrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "grid_sync.cuh"
#include "philox.cuh"
#include "tab_internal.h"

namespace tab {

// Warp roles.  Warp 0 and kResHelpers helper warps replay the batch (phase
// 1); the next A warps are apply warps (phase 2), each owning at most 32 of
// the CTA's columns (one ballot); 1 + kResHelpers + A <= kResMaxWarps.  The host picks A from the CTA's columns, one column
// per apply warp where that fits (kernels_resident.cu): the work of one
// measurement is a short dependent chain per warp, so several warps per SM
// hide each other's latency.
constexpr int kResMaxWarps = 16;
constexpr int kBatchMax = 32;                       // largest batch of any instance
constexpr int kResHelpers = 4;                      // helper warps of the replay
constexpr int kResMaxLocalCols = 32 * (kResMaxWarps - 1);  // columns of one CTA
constexpr int kPubSpinMax = 1 << 22;              // polls (64 ns apart) before a wait gives up

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
  int nreplay, napply;  // replay warps R = 1 + kResHelpers, apply warps A (blockDim = 32 (R + A))
  unsigned long long wait_ns;  // limit of each grid-barrier wait
  int skip_arrival;            // test-only fault injection (TAB_DEBUG_SKIP_BARRIER_ARRIVAL)
  // CommGrid workspace (global memory)
  uint32_t* stage;  // [2][kb][W] X bits of the measured columns of the next batch
  uint32_t* dp;     // [2][kb][C] deterministic partials
  uint32_t* ph;     // [C][2][W] sign partials for the fold
  uint32_t* r4;     // [2][W] base signs for the fold
  GridBar* bar;
};

struct ResLayout {
  int ncl, Wp;
  size_t words;
};

// Shared-memory words per CTA.  `push`: the measured columns of the next
// batch land in shared memory (cluster, double-buffered), not in global
// memory (grid).
__host__ __device__ inline ResLayout res_layout(int n, int Wh, int C, int kb, bool push) {
  ResLayout L;
  const int W = 2 * Wh;
  L.ncl = (n + C - 1) / C;
  L.Wp = W + 1;
  L.words = 2 * (size_t)L.ncl * L.Wp            // own X, Z columns
            + 4 * (size_t)W                      // CTA sign partial (lo, hi), base signs (lo, hi)
            + (size_t)kb * W                     // mask of each measurement of the batch
            + (size_t)kb * L.Wp                  // X bits of the batch's measured columns
            + (push ? 4 * (size_t)kb * W : 0)    // measured columns X, Z, double-buffered
            + 2 * (size_t)kb * C;                // deterministic partials, double-buffered
  return L;
}

// Largest batch size (power of two <= cap <= kBatchMax) that fits `limit`
// bytes; 0 if even single measurements do not fit.
__host__ __device__ inline int res_batch_for(int n, int Wh, int C, size_t limit, int cap,
                                             bool push) {
  if ((n + C - 1) / C > kResMaxLocalCols) return 0;
  if (cap > kBatchMax) cap = kBatchMax;
  for (int kb = cap; kb >= 1; kb >>= 1)
    if (res_layout(n, Wh, C, kb, push).words * 4 <= limit) return kb;
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
// publish / observe a counter in shared memory (release / acquire, CTA scope)
__device__ __forceinline__ void res_st_release(int* p, int v) {
  asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"((uint32_t)__cvta_generic_to_shared(p)),
               "r"(v)
               : "memory");
}
__device__ __forceinline__ int res_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.b32 %0, [%1];"
               : "=r"(v)
               : "r"((uint32_t)__cvta_generic_to_shared(p))
               : "memory");
  return v;
}
// Wait until *p >= v (lane 0 polls with acquire loads; warp-wide); false
// when the wait gives up after kPubSpinMax polls.  With `nap`, polls after
// the first 256 are 64 ns apart.
__device__ __forceinline__ bool res_wait_geq(const int* p, int v, bool nap) {
  for (int it = 0; it <= kPubSpinMax; ++it) {
    const int seen = __shfl_sync(0xffffffffu, (threadIdx.x & 31) == 0 ? res_ld_acquire(p) : 0, 0);
    if (seen >= v) return true;
    if (nap && it >= 256) __nanosleep(64);
  }
  return false;
}
// v[k] for a warp-uniform k, without dynamic register indexing
template <int WL>
__device__ __forceinline__ uint32_t res_pick(const uint32_t (&v)[WL], int k) {
  uint32_t o = 0u;
#pragma unroll
  for (int j = 0; j < WL; ++j) o |= v[j] & (0u - (uint32_t)(j == k));
  return o;
}

// Shared-memory pointers of the per-CTA state.
struct ResSmem {
  uint32_t *Xs, *Zs, *PHlo, *PHhi, *R4lo, *R4hi, *SM, *CX, *TX, *TZ, *dpv;
};

__device__ __forceinline__ ResSmem res_smem(uint32_t* sm, const ResLayout& Ly, int W, int kb,
                                            bool push) {
  ResSmem s;
  s.Xs = sm;
  s.Zs = s.Xs + (size_t)Ly.ncl * Ly.Wp;
  s.PHlo = s.Zs + (size_t)Ly.ncl * Ly.Wp;
  s.PHhi = s.PHlo + W;
  s.R4lo = s.PHhi + W;
  s.R4hi = s.R4lo + W;
  s.SM = s.R4hi + W;             // [kb][W] mask of each measurement of the batch
  s.CX = s.SM + (size_t)kb * W;  // [kb][Wp] replayed X bits of the measured columns
  s.TX = s.CX + (size_t)kb * Ly.Wp;  // [2][kb][W] measured columns, X plane (push only)
  s.TZ = s.TX + (push ? 2 * (size_t)kb * W : 0);
  s.dpv = s.TZ + (push ? 2 * (size_t)kb * W : 0);  // [2][kb][C]
  return s;
}

// Per-batch bookkeeping in static shared memory.
struct ResBatch {
  uint32_t code[kBatchMax];  // measurement codes of the batch
  int slot[kBatchMax];       // measured-column slot of each measurement
  int la[kBatchMax];         // local column of the measured qubit in this CTA, or -1
  int lw[kBatchMax];         // warp of this CTA owning that column, or -1
  int q[kBatchMax];          // qubit of each slot
  int last[kBatchMax];       // last measurement of each slot
  uint32_t live[kBatchMax];  // slots measured again after measurement i (bit d: slot d)
  uint32_t hm[kBatchMax];    // live[i] less slot[i+1] and slot[i+2]: the helpers' slots at i
  int s3[kBatchMax];         // slot[i+3], or -1
  int own[kBatchMax];        // slots whose column this CTA owns
  int P[kBatchMax];          // pivot row of each measurement (-1: deterministic)
  uint32_t dacc[kBatchMax];  // this CTA's deterministic partial
  int ptype[kBatchMax];      // previous batch: 1 = deterministic
  int det[kBatchMax];        // previous batch: resolved deterministic outcome
  int D, nown, anydet;
  volatile int keff;         // measurements of the batch (a deterministic reset ends it)
  int npub;                  // measurements whose pivot and mask are published
  int hpri[kResHelpers];     // helper h: updates whose look-ahead column it has applied
  uint32_t plast;            // code of the previous batch's last measurement
};

// Slots of a batch of K <= 32 measurements, lane i holding code i: distinct
// measured qubits in first-occurrence order, each slot's last measurement,
// the slots still needed after each measurement, and the slots, columns and
// apply warps (warp R + local column / cpw) this CTA owns.  Warp-wide (one
// warp).
__device__ __forceinline__ void res_batch_slots(uint32_t code, int K, int C, int r, int cpw,
                                                int R, ResBatch& b, int n, int* err) {
  const int lane = threadIdx.x & 31;
  if (lane < K) code = dbg_code(code, (uint32_t)n, err);
  const bool v = lane < K;
  const int a = v ? (int)dq1(code) : -1 - lane;
  const uint32_t grp = __match_any_sync(0xffffffffu, a);
  const int first = __ffs(grp) - 1;
  const bool lead = v && first == lane;
  const uint32_t firsts = __ballot_sync(0xffffffffu, lead);
  const int slot = __popc(firsts & ((1u << first) - 1u));
  const bool mine = lead && (a % C == r);
  const uint32_t owned = __ballot_sync(0xffffffffu, mine);
  const int lastv = lead ? 31 - __clz(grp) : -1;
  if (v) {
    const int la = (a % C == r) ? a / C : -1;
    b.code[lane] = code;
    b.slot[lane] = slot;
    b.la[lane] = la;
    b.lw[lane] = (la >= 0 && cpw > 0) ? R + la / cpw : -1;
  }
  if (lead) {
    b.q[slot] = a;
    b.last[slot] = lastv;
  }
  __syncwarp();
  const int D = __popc(firsts);
  const int s1 = __shfl_down_sync(0xffffffffu, slot, 1), s2 = __shfl_down_sync(0xffffffffu, slot, 2);
  const int s3 = __shfl_down_sync(0xffffffffu, slot, 3);
  if (v) {  // slots still needed after measurement `lane`
    uint32_t live = 0u;
    for (int d = 0; d < D; ++d)
      if (b.last[d] > lane) live |= 1u << d;
    b.live[lane] = live;
    if (lane + 1 < K) live &= ~(1u << s1);
    if (lane + 2 < K) live &= ~(1u << s2);
    b.hm[lane] = live;
    b.s3[lane] = lane + 3 < K ? s3 : -1;
  }
  if (mine) b.own[__popc(owned & ((1u << lane) - 1u))] = slot;
  if (lane == 0) {
    b.D = D;
    b.nown = __popc(owned);
  }
}

template <int WL, class Comm>
__device__ void measure_resident(const ResArgs& A, Comm& cm, uint32_t* sm) {
  constexpr bool kPush = Comm::kPush;
  const int R = A.nreplay, NA = A.napply;
  const int C = cm.size(), r = cm.rank(), tid = threadIdx.x, T = blockDim.x;
  const int n = A.n, Wh = A.Wh, W = 2 * Wh, KB = A.kb;
  const ResLayout Ly = res_layout(n, Wh, C, KB, kPush);
  const int Wp = Ly.Wp;
  const int nown = (n - r + C - 1) / C;  // columns owned: r, r+C, ...
  const ResSmem s = res_smem(sm, Ly, W, KB, kPush);
  const int lane = tid & 31, warp = tid >> 5;
  const int cpw = (nown + NA - 1) / NA;  // an apply warp's local columns: c0 .. c0+ncw-1
  const int av = warp - R;                 // apply-warp index (negative: a replay warp)
  const int c0 = av * cpw;
  const int ncw = (av < 0 || nown - c0 < 0) ? 0 : (nown - c0 < cpw ? nown - c0 : cpw);
  const bool base_warp = (r == 0 && warp == R);
  const uint32_t lt = (1u << lane) - 1u;
  __shared__ ResBatch b;

  // this warp's share of every row's sign exponent (lo, hi bit planes)
  uint32_t plo[WL], phi[WL];
#pragma unroll
  for (int k = 0; k < WL; ++k) plo[k] = phi[k] = 0u;

  // ---- load own columns, base signs, first batch
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
  if (warp == 0) {
    const int K0 = A.nm < KB ? A.nm : KB;
    const uint32_t c = lane < K0 ? __ldg(A.mops + lane) : 0u;
    res_batch_slots(c, K0, C, r, cpw, R, b, n, A.err);
    if (lane == 0) b.anydet = 0;
  }
  if (!cm.start()) return;
  cm.stage_columns(s, 0, b, W, Wp, KB);  // first batch's measured columns

  int m = 0, batch = 0, prev_base = 0, prev_count = 0;
  while (m < A.nm) {
    const int par = batch & 1;
    const int K = (A.nm - m < KB) ? A.nm - m : KB;
    // outcome bits of the batch (lane i: measurement m+i) and the codes of
    // the batch after it: both known now, their latency hides in the barrier
    const uint32_t my_rbit =
        lane < K ? outcome_bit(A.seed, A.cid, A.shot, A.k0 + (uint64_t)(m + lane)) : 0u;
    uint32_t next_code = 0u;
    if (warp == 0 && lane < KB && m + K + lane < A.nm) next_code = __ldg(A.mops + m + K + lane);
    // ---- barrier: the previous batch's column updates, staged columns and
    // deterministic partials are visible everywhere
    if (!cm.sync()) return;
    // ---- resolve the previous batch's deterministic outcomes
    if (b.anydet) {
      if (tid < prev_count && b.ptype[tid]) {
        const uint32_t e = cm.sum_dp(s.dpv, par ^ 1, tid, KB) & 3u;
        if (e & 1u) atomicCAS(A.err, 0, DERR_PHASE);
        b.det[tid] = (int)(e >> 1);
        if (r == 0) A.out[prev_base + tid] = (uint8_t)(e >> 1);
      }
      __syncthreads();
      // a deterministic measure-and-reset ends its batch, so only the last
      // measurement of the previous batch can need its X_a: every sign ^= z_a,
      // added to the share of the warp that owns column a
      if (b.ptype[prev_count - 1] && b.det[prev_count - 1] && dop(b.plast) == OP_MZR) {
        const int pa = (int)dq1(b.plast);
        if (pa % C == r && R + (pa / C) / cpw == warp) {
          const uint32_t* zc = s.Zs + (size_t)(pa / C) * Wp;
#pragma unroll
          for (int k = 0; k < WL; ++k) {
            const int w = lane + 32 * k;
            if (w < W) phi[k] ^= zc[w];
          }
        }
      }
    }
    if (tid < KB) b.dacc[tid] = 0u;
    if (tid == 0) {
      b.keff = K;
      b.npub = 0;
      for (int h = 0; h < kResHelpers; ++h) b.hpri[h] = 0;
    }
    // the X bits of the batch's measured columns into shared memory for the
    // replay warp, by every thread (independent L2 loads, four in flight)
    {
      const int DW = b.D * W;
      for (int e0 = tid; e0 < DW; e0 += 4 * T) {
        uint32_t v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * T;
          v[u] = e < DW ? cm.slot_word(s, par, e / W, e % W, W, KB) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * T;
          if (e < DW) s.CX[(size_t)(e / W) * Wp + e % W] = v[u];
        }
      }
    }
    __syncthreads();

    // ---- phase 1: replay the batch on the X bits of its measured columns
    // (shared memory, slot d at CX + d*Wp, lane l taking words l, l+32, ...).
    // Warp 0 runs the chain: for measurement i it holds slot[i] and
    // slot[i+1] in registers, current through measurement i-1; it finds the
    // pivot P_i on slot[i], publishes P_i and the mask S_i (release store of
    // npub), then applies measurement i to slot[i+1] and slot[i+2] (stored
    // back) and moves on.  The helper warps apply measurement j to every
    // other slot still measured later in the batch (helper h: slots
    // d = h mod kResHelpers), in order, the slot warp 0 takes next
    // (slot[j+3]) first, after which they bump hpri[h]; warp 0 waits for that
    // before it loads slot[i+2].  So each slot sees the measurements in
    // order, and the chain from one publication to the next is one pivot
    // search and two column updates in registers.
    uint32_t* CX = s.CX;
    // measurement i (pivot P, mask v = S_i less rows p and p-n) on one
    // column's words held by this lane, with xp row p's bit on that column:
    // x ^= v where xp, then row p-n := row p (keep/setd: the bit of row p-n
    // or p in this lane's words) and row p := Z_a (no X)
    struct Upd {
      uint32_t v[WL], keep[WL], setd[WL];
    };
    auto make_upd = [&](const uint32_t (&S)[WL], int P, Upd& u) {
      const int wp = P >> 5, wd = (P - 32 * Wh) >> 5;
      const uint32_t bpm = 1u << (P & 31);
#pragma unroll
      for (int k = 0; k < WL; ++k) {
        const int w = lane + 32 * k;
        const bool pk = w == wp || w == wd;
        u.keep[k] = pk ? ~bpm : 0xffffffffu;
        u.setd[k] = w == wd ? bpm : 0u;
        u.v[k] = S[k] & u.keep[k];
      }
    };
    auto upd_words = [&](uint32_t (&c)[WL], const Upd& u, bool xp) {
      const uint32_t XP = xp ? 0xffffffffu : 0u;
#pragma unroll
      for (int k = 0; k < WL; ++k) c[k] = ((c[k] ^ (u.v[k] & XP)) & u.keep[k]) | (u.setd[k] & XP);
    };
    auto load_col = [&](uint32_t (&c)[WL], int d) {
#pragma unroll
      for (int k = 0; k < WL; ++k) {
        const int w = lane + 32 * k;
        c[k] = (d >= 0 && w < W) ? CX[(size_t)d * Wp + w] : 0u;
      }
    };
    auto store_col = [&](const uint32_t (&c)[WL], int d) {
#pragma unroll
      for (int k = 0; k < WL; ++k) {
        const int w = lane + 32 * k;
        if (w < W) CX[(size_t)d * Wp + w] = c[k];
      }
    };
    constexpr int NQ = kBatchMax / kResHelpers;  // slots per helper: d = kResHelpers q + h
    if (warp == 0) {
      uint32_t ca[WL], cb[WL];
      load_col(ca, b.slot[0]);
      load_col(cb, K > 1 ? b.slot[1] : -1);
      const int k_stab = Wh >> 5;  // first k whose words reach the stabilizer half
      uint32_t code = b.code[0];
      for (int i = 0; i < K; ++i) {
        const int d2 = i + 2 < K ? b.slot[i + 2] : -1;
        const uint32_t code_next = i + 1 < K ? b.code[i + 1] : 0u;
        // has slot[i+2]'s helper applied measurement i-1 to it?  (looked at
        // early; waited for below)
        bool ready = d2 < 0 || res_ld_acquire(&b.hpri[d2 % kResHelpers]) >= i;
        uint32_t* Si = s.SM + (size_t)i * W;
        int P = -1;
#pragma unroll
        for (int k = 0; k < WL; ++k) {
          const int w = lane + 32 * k;
          if (w < W) Si[w] = ca[k];
          if (k < k_stab || P >= 0) continue;  // warp-uniform
          const uint32_t bal = __ballot_sync(0xffffffffu, w >= Wh && ca[k] != 0u);
          if (bal) {
            const int l = __ffs(bal) - 1;
            const uint32_t word = __shfl_sync(0xffffffffu, ca[k], l);
            P = (32 * k + l) * 32 + __ffs(word) - 1;
          }
        }
        if (lane == 0) {
          b.P[i] = P;
          if (P < 0 && dop(code) == OP_MZR) b.keff = i + 1;  // ends the batch
        }
        __syncwarp();
        if (lane == 0) res_st_release(&b.npub, i + 1);
        if (P < 0 && dop(code) == OP_MZR) break;
        if (i + 1 >= K) break;
        if (!__all_sync(0xffffffffu, ready)) {  // wait (every lane polls; bounded)
          for (int it = 0; it <= kPubSpinMax && !ready; ++it)
            ready = res_ld_acquire(&b.hpri[d2 % kResHelpers]) >= i;
          if (!__all_sync(0xffffffffu, ready)) {
            if (lane == 0) atomicCAS(A.err, 0, DERR_TIMEOUT);
            break;
          }
        }
        uint32_t cc[WL];
        load_col(cc, d2);
        if (P >= 0) {  // random outcome: measurement i on slot[i+1] and slot[i+2]
          Upd u;
          make_upd(ca, P, u);
          // row p's bits on slot[i+1] (bit 0) and slot[i+2] (bit 1), from the
          // lane holding word P>>5
          const int wp = P >> 5;
          const uint32_t bb = (res_pick(cb, wp >> 5) >> (P & 31)) & 1u;
          const uint32_t bc = (res_pick(cc, wp >> 5) >> (P & 31)) & 1u;
          const uint32_t bits = __shfl_sync(0xffffffffu, bb | (bc << 1), wp & 31);
          upd_words(cb, u, bits & 1u);
          store_col(cb, b.slot[i + 1]);
          if (d2 >= 0) {
            upd_words(cc, u, (bits >> 1) & 1u);
            store_col(cc, d2);
          }
        }
#pragma unroll
        for (int k = 0; k < WL; ++k) {
          ca[k] = cb[k];
          cb[k] = cc[k];
        }
        code = code_next;
      }
    } else if (warp <= kResHelpers && warp < R) {
      const int h = warp - 1;
      const uint32_t own = 0x11111111u << h;  // slots d = h mod kResHelpers
      static_assert(kResHelpers == 4, "slot ownership mask");
      if constexpr (WL <= 4) {
        // this helper's slots in registers; `held`: slots whose register
        // copy is current through the previous measurement
        uint32_t xr[NQ][WL];
        uint32_t held = 0u;
        for (int j = 0; j < K; ++j) {
          if (!res_wait_geq(&b.npub, j + 1, false)) {
            if (lane == 0) atomicCAS(A.err, 0, DERR_TIMEOUT);
            break;
          }
          __syncwarp();
          const int P = b.P[j];
          const int d3 = b.s3[j];
          const uint32_t mine = P >= 0 ? b.hm[j] & own : 0u;
          if (mine != 0u) {
            // slots last written by warp 0 or by the staging: reload
            const uint32_t rl = mine & ~held;
            if (rl != 0u) {
#pragma unroll
              for (int q = 0; q < NQ; ++q)
                if ((rl >> (kResHelpers * q + h)) & 1u) load_col(xr[q], kResHelpers * q + h);
            }
            uint32_t Sr[WL];
            load_col(Sr, -1);
#pragma unroll
            for (int k = 0; k < WL; ++k) {
              const int w = lane + 32 * k;
              if (w < W) Sr[k] = s.SM[(size_t)j * W + w];
            }
            Upd u;
            make_upd(Sr, P, u);
            // row p's bit on each slot, from the lane holding word P>>5
            const int wp = P >> 5;
            uint32_t gl = 0u;
#pragma unroll
            for (int q = 0; q < NQ; ++q) gl |= ((res_pick(xr[q], wp >> 5) >> (P & 31)) & 1u) << q;
            const uint32_t g = __shfl_sync(0xffffffffu, gl, wp & 31);
            if (d3 >= 0 && ((mine >> d3) & 1u)) {  // warp 0's next slot first
              const int qp = d3 / kResHelpers;
              uint32_t c[WL];
#pragma unroll
              for (int k = 0; k < WL; ++k) {
                c[k] = 0u;
#pragma unroll
                for (int q = 0; q < NQ; ++q) c[k] |= xr[q][k] & (0u - (uint32_t)(q == qp));
              }
              upd_words(c, u, (g >> qp) & 1u);
              store_col(c, d3);
              __syncwarp();
            }
            if (lane == 0) res_st_release(&b.hpri[h], j + 1);
            // every slot of `mine` (the one above again, identically)
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
              const uint32_t act = 0u - ((mine >> (kResHelpers * q + h)) & 1u);
              uint32_t c[WL];
#pragma unroll
              for (int k = 0; k < WL; ++k) c[k] = xr[q][k];
              upd_words(c, u, (g >> q) & 1u);
#pragma unroll
              for (int k = 0; k < WL; ++k) xr[q][k] = (c[k] & act) | (xr[q][k] & ~act);
            }
            held = mine;
          } else if (P >= 0) {
            held = 0u;
            if (lane == 0) res_st_release(&b.hpri[h], j + 1);
          } else {
            // a deterministic measurement changes no X bit: the register
            // copies stay current; warp 0 loads slot[j+3] next, so store it
            // if this helper holds it
            if (d3 >= 0 && ((held >> d3) & 1u)) {
              const int qp = d3 / kResHelpers;
#pragma unroll
              for (int q = 0; q < NQ; ++q)
                if (q == qp) store_col(xr[q], d3);
              __syncwarp();
            }
            if (lane == 0) res_st_release(&b.hpri[h], j + 1);
          }
          if (__shfl_sync(0xffffffffu, lane == 0 ? b.keff : 0, 0) == j + 1) break;  // batch ends here
        }
      } else {
        // this helper's slots in shared memory (CX), updated in place
        for (int j = 0; j < K; ++j) {
          if (!res_wait_geq(&b.npub, j + 1, false)) {
            if (lane == 0) atomicCAS(A.err, 0, DERR_TIMEOUT);
            break;
          }
          __syncwarp();
          const int P = b.P[j];
          const int d3 = b.s3[j];
          uint32_t mine = P >= 0 ? b.hm[j] & own : 0u;
          if (mine != 0u) {
            const uint32_t bpm = 1u << (P & 31);
            uint32_t Sr[WL];
#pragma unroll
            for (int k = 0; k < WL; ++k) {
              const int w = lane + 32 * k;
              Sr[k] = w < W ? s.SM[(size_t)j * W + w] : 0u;
            }
            Upd u;
            make_upd(Sr, P, u);
            // row p's bit on each of this helper's slots (lane d: slot d)
            const uint32_t g = __ballot_sync(
                0xffffffffu, ((mine >> lane) & 1u) && ((CX[(size_t)lane * Wp + (P >> 5)] & bpm) != 0u));
            __syncwarp();
            if (d3 >= 0 && ((mine >> d3) & 1u)) {  // warp 0's next slot first
              uint32_t c[WL];
              load_col(c, d3);
              upd_words(c, u, (g >> d3) & 1u);
              store_col(c, d3);
              mine &= ~(1u << d3);
              __syncwarp();
            }
            if (lane == 0) res_st_release(&b.hpri[h], j + 1);
            for (uint32_t l = mine; l != 0u; l &= l - 1u) {
              const int d = __ffs(l) - 1;
              uint32_t c[WL];
              load_col(c, d);
              upd_words(c, u, (g >> d) & 1u);
              store_col(c, d);
            }
            __syncwarp();
          } else if (lane == 0) {
            res_st_release(&b.hpri[h], j + 1);
          }
          if (__shfl_sync(0xffffffffu, lane == 0 ? b.keff : 0, 0) == j + 1) break;  // batch ends here
        }
      }
    }

    // ---- phase 2: every apply warp with columns (and the base warp) applies
    // the batch to its columns and its share, each measurement as soon as it
    // is published; a warp without columns keeps a zero share and has no work
    if (ncw > 0 || base_warp) {
      int seen = 0;
      for (int i = 0; i < K; ++i) {
        if (i >= seen) {  // wait for measurement i (bounded)
          for (int it = 0;; ++it) {
            seen = __shfl_sync(0xffffffffu, lane == 0 ? res_ld_acquire(&b.npub) : 0, 0);
            if (seen > i || it > kPubSpinMax) break;
            if (it >= 256) __nanosleep(64);
          }
          if (seen <= i) {
            if (lane == 0) atomicCAS(A.err, 0, DERR_TIMEOUT);
            break;
          }
        }
        const uint32_t code = b.code[i];
        const int P = b.P[i];
        const uint32_t* S = s.SM + (size_t)i * W;
        const uint32_t rbit = __shfl_sync(0xffffffffu, my_rbit, i);
        __syncwarp();  // the previous measurement's column writes, across lanes
        if (P >= 0) {
          // ============ random outcome ============
          const int wp = P >> 5, wd = (P - 32 * Wh) >> 5;
          const uint32_t bpm = 1u << (P & 31);
          const int la = b.la[i];  // local column of qubit a (or -1)
          // this warp's share of 2 r_p (and the base, for the base warp)
          const uint32_t pl = __shfl_sync(0xffffffffu, res_pick(plo, wp >> 5), wp & 31);
          const uint32_t ph = __shfl_sync(0xffffffffu, res_pick(phi, wp >> 5), wp & 31);
          const uint32_t php = ((pl & bpm) ? 1u : 0u) | ((ph & bpm) ? 2u : 0u);
          uint32_t r4p = 0u;
          if (base_warp) r4p = ((s.R4lo[wp] & bpm) ? 1u : 0u) | ((s.R4hi[wp] & bpm) ? 2u : 0u);
          // pivot row over this warp's columns (lane c: local column c0 + c)
          bool xb = false, zb = false;
          if (lane < ncw) {
            const size_t ii = (size_t)(c0 + lane) * Wp + wp;
            xb = (s.Xs[ii] & bpm) != 0u;
            zb = (s.Zs[ii] & bpm) != 0u;
          }
          const uint32_t supx = __ballot_sync(0xffffffffu, xb);
          const uint32_t supz = __ballot_sync(0xffffffffu, zb);
          const uint32_t scal = ((uint32_t)__popc(supx & supz) + php + r4p) & 3u;
          // S': rows with x_ha = 1 other than p and p-n
          uint32_t Sw[WL];
#pragma unroll
          for (int k = 0; k < WL; ++k) {
            const int w = lane + 32 * k;
            Sw[k] = w < W ? S[w] : 0u;
            if (w == wp || w == wd) Sw[k] &= ~bpm;
          }
          // the rowsum on every column where row p is X, Z or Y
          for (uint32_t left = supx | supz; left; left &= left - 1u) {
            const int c = __ffs(left) - 1;
            const bool cx = (supx >> c) & 1u, cz = (supz >> c) & 1u;
            uint32_t* xc = s.Xs + (size_t)(c0 + c) * Wp;
            uint32_t* zc = s.Zs + (size_t)(c0 + c) * Wp;
            if (cx && !cz) {  // X
#pragma unroll
              for (int k = 0; k < WL; ++k) {
                const int w = lane + 32 * k;
                if (w < W) {
                  const uint32_t x = xc[w], t = zc[w] & Sw[k];
                  phi[k] ^= t & ~(x ^ plo[k]);
                  plo[k] ^= t;
                  xc[w] = x ^ Sw[k];
                }
              }
            } else if (!cx) {  // Z
#pragma unroll
              for (int k = 0; k < WL; ++k) {
                const int w = lane + 32 * k;
                if (w < W) {
                  const uint32_t z = zc[w], t = xc[w] & Sw[k];
                  phi[k] ^= t & (z ^ plo[k]);
                  plo[k] ^= t;
                  zc[w] = z ^ Sw[k];
                }
              }
            } else {  // Y
#pragma unroll
              for (int k = 0; k < WL; ++k) {
                const int w = lane + 32 * k;
                if (w < W) {
                  const uint32_t x = xc[w], z = zc[w];
                  const uint32_t e = ~(x ^ z) & Sw[k];
                  phi[k] ^= (e & ~(x ^ plo[k])) ^ (x & Sw[k]);
                  plo[k] ^= e;
                  xc[w] = x ^ Sw[k];
                  zc[w] = z ^ Sw[k];
                }
              }
            }
          }
          __syncwarp();
          // rows p-n and p of every column of this warp: row p-n := row p,
          // row p := Z_a (lane c: local column c0 + c)
          if (lane < ncw) {
            const int lj = c0 + lane;
            uint32_t* xc = s.Xs + (size_t)lj * Wp;
            uint32_t* zc = s.Zs + (size_t)lj * Wp;
            xc[wd] = (xc[wd] & ~bpm) | (xb ? bpm : 0u);
            zc[wd] = (zc[wd] & ~bpm) | (zb ? bpm : 0u);
            xc[wp] &= ~bpm;
            zc[wp] = (zc[wp] & ~bpm) | ((lj == la) ? bpm : 0u);
          }
          // this warp's share of 2 r_p and of sum_j x_pj z_pj, on every row in S'
#pragma unroll
          for (int k = 0; k < WL; ++k) {
            const int w = lane + 32 * k;
            uint32_t lo = plo[k], hi = phi[k];
            res_add4(lo, hi, (scal & 1u) ? Sw[k] : 0u, (scal & 2u) ? Sw[k] : 0u);
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
          if (dop(code) == OP_MZR && rbit && b.lw[i] == warp) {
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
          for (int c = 0; c < ncw; ++c) {
            const size_t col = (size_t)(c0 + c) * Wp + Wh;
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
        if (__shfl_sync(0xffffffffu, lane == 0 ? b.keff : 0, 0) == i + 1) break;  // batch ends here
      }
    }
    __syncthreads();
    const int keff = b.keff;
    if (r == 0 && warp == 0 && lane < keff && b.P[lane] >= 0)
      A.out[m + lane] = (uint8_t)my_rbit;

    // ---- publish the deterministic partials; bookkeeping for the next batch
    int anydet = 0;
    for (int i = 0; i < keff; ++i)
      if (b.P[i] < 0) {
        cm.publish_dp(s.dpv, par, i, KB, b.dacc[i] & 3u);
        anydet = 1;
      }
    __syncthreads();
    if (tid < keff) b.ptype[tid] = b.P[tid] < 0;
    if (tid == 0) {
      b.plast = b.code[keff - 1];
      b.anydet = anydet;
    }
    __syncthreads();
    if (warp == 0) {
      const int mn = m + keff;
      const int Kn = (A.nm - mn < KB) ? A.nm - mn : KB;
      if (keff != K && lane < Kn) next_code = __ldg(A.mops + mn + lane);  // batch ended early
      res_batch_slots(next_code, Kn > 0 ? Kn : 0, C, r, cpw, R, b, n, A.err);
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
  if (b.anydet) {
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
  if (b.anydet && b.ptype[prev_count - 1] && b.det[prev_count - 1] && dop(b.plast) == OP_MZR) {
    const int pa = (int)dq1(b.plast);
    if (pa % C == r && R + (pa / C) / cpw == warp) {
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
