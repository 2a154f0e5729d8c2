// kernels_sct.cu -- single-CTA tableau engine (whole tableau resident in
// shared memory) and the persistent batched launch built on it (sm_103a).
//
// For n <= 640 a complete tableau (2 planes x n columns x 2n rows, plus signs)
// fits in one CTA's shared memory, so gates and measurements need only CTA
// barriers.  Operations are those of Aaronson & Gottesman, PRA 70, 052328,
// Sec. III (the formalism of the Clifford backend in arXiv:2408.00384,
// "Simulation of Clifford circuits"):
//  * gates: column updates (gate_rules.cuh); the lanes of a warp take the
//    words of one column, so one gate is one conflict-free shared-memory sweep;
//  * measurement of Z_a: pivot by warp ballot over the stabilizer half of
//    column a; random case -- rowsum of the pivot row into every row with
//    x_ha = 1 with the exponent
//      2 r_h' = 2 r_h + 2 r_p + sum_j [x_pj z_pj + x_hj z_hj - x'_hj z'_hj
//                                      + 2 z_pj x_hj]   (mod 4)
//    kept as bit-sliced mod-4 counters (x' = x_h ^ x_p, z' = z_h ^ z_p), then
//    row p-n := row p and row p := (-1)^b Z_a; deterministic case -- the sign
//    of the product of the selected stabilizer rows,
//      e = sum_m (2 r_m + |x_m & z_m|) + 2 sum_{m<l} z_m . x_l   (mod 4),
//    whose pairwise term is a prefix-parity scan down each column.
//
// Shared-memory layout: Whc = ceil(n/32) words per half, Wc = 2*Whc per
// column, column stride Wp = Wc | 1 (odd, so both "lanes over words of one
// column" and "lanes over columns at one word" are bank-conflict free).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gate_rules.cuh"
#include "philox.cuh"
#include "sct.h"
#include "tab_internal.h"

namespace tab {

constexpr int kSctThreads = 512;
constexpr uint32_t kNoiseKeyTag = 0x4E4F4953u;  // noise draws use a key of their own
constexpr unsigned long long kReadyWaitNs = 2000000000ull;

__host__ __device__ inline int sct_whc(int n) { return (n + 31) / 32; }
__host__ __device__ inline int sct_wc(int n) { return 2 * sct_whc(n); }
__host__ __device__ inline int sct_wp(int n) { return sct_wc(n) | 1; }

size_t sct_image_words(int n) {
  return ((size_t)2 * n * sct_wp(n) + sct_wc(n) + 3) & ~(size_t)3;
}

__host__ __device__ inline size_t sct_smem_words(int n, int threads) {
  const int Wc = sct_wc(n);
  int GG = threads / Wc;
  if (GG < 1) GG = 1;
  if (GG > n) GG = n;
  (void)GG;
  return (size_t)2 * n * sct_wp(n) + 2 * (size_t)Wc + 3 * (size_t)n + 2 * (size_t)sct_wp(n);
}

size_t sct_smem_bytes(int n, int threads) { return sizeof(uint32_t) * sct_smem_words(n, threads); }

// Extra shared memory of the terminal-measurement sampler for a circuit of n
// qubits, K terminal measurements and `shots` shots (sct_form_pass and
// sct_sample): K coefficient columns, a list of K columns, and one K-bit
// random vector per shot.
size_t sct_sampler_bytes(int n, int K, int shots) {
  const size_t FW = ((size_t)K + 31) / 32;
  return sizeof(uint32_t) * ((size_t)K * sct_wp(n) + (size_t)K + (size_t)shots * FW);
}

struct Sct {
  int n, Whc, Wc, Wp, GG;
  uint32_t *X, *Z, *R, *sS, *supp, *redlo, *redhi;  // supp: [3][n] (X, Z, Y columns)
  int* err;  // the launch's error word (debug-build index checks)
  unsigned long long* work;  // BatchArgs::work (null: not counting)
};

__device__ __forceinline__ void sct_setup(Sct& s, uint32_t* base, int n, int* err) {
  s.n = n;
  s.err = err;
  s.work = nullptr;
  s.Whc = sct_whc(n);
  s.Wc = 2 * s.Whc;
  s.Wp = s.Wc | 1;
  s.GG = (int)blockDim.x / s.Wc;
  if (s.GG < 1) s.GG = 1;
  if (s.GG > n) s.GG = n;  // a group per column at most
  s.X = base;
  s.Z = s.X + (size_t)n * s.Wp;
  s.R = s.Z + (size_t)n * s.Wp;
  s.sS = s.R + s.Wc;
  s.supp = s.sS + s.Wc;
  s.redlo = s.supp + 3 * n;  // per-word sign counters of a rowsum (low, high plane)
  s.redhi = s.redlo + s.Wp;
}

__device__ __forceinline__ unsigned long long sct_gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t prefix_xor_exclusive(uint32_t v) {
  uint32_t y = v << 1;
  y ^= y << 1;
  y ^= y << 2;
  y ^= y << 4;
  y ^= y << 8;
  y ^= y << 16;
  return y;
}

__device__ __forceinline__ void add4s(uint32_t& l, uint32_t& h, uint32_t bl, uint32_t bh) {
  h ^= bh ^ (l & bl);
  l ^= bl;
}

// |0^n>: destabilizer i = +X_i, stabilizer i = +Z_i.
__device__ void sct_identity(const Sct& s) {
  const int tot = s.n * s.Wp;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int a = i / s.Wp, w = i - a * s.Wp;
    const uint32_t bit = 1u << (a & 31);
    s.X[i] = (w == (a >> 5)) ? bit : 0u;
    s.Z[i] = (w == s.Whc + (a >> 5)) ? bit : 0u;
  }
  for (int w = threadIdx.x; w < s.Wc; w += blockDim.x) s.R[w] = 0u;
}

// Apply layers [0, nl) of a gate segment; layer_off[L]..layer_off[L+1].
__device__ void sct_gates(const Sct& s, const uint32_t* __restrict__ ops,
                          const uint32_t* __restrict__ layer_off, int nl,
                          const uint8_t* npauli = nullptr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t r0 = 0u, r1 = 0u;
  uint32_t lb = __ldg(layer_off);
  if (s.Wc >= 32) {  // one gate per warp, lanes over words
    const bool two = lane + 32 < s.Wc;
    for (int L = 0; L < nl; ++L) {
      const uint32_t le = __ldg(layer_off + L + 1);
      for (uint32_t g = lb + warp; g < le; g += nw) {
        const uint32_t code = dbg_code(__ldg(ops + g), (uint32_t)s.n, s.err);
        apply_gate(code, s.X, s.Z, s.Wp, lane, r0, npauli);
        if (two) apply_gate(code, s.X, s.Z, s.Wp, lane + 32, r1, npauli);
      }
      lb = le;
      __syncthreads();
    }
    if (r0) atomicXor(&s.R[lane], r0);
    if (two && r1) atomicXor(&s.R[lane + 32], r1);
  } else {  // several gates per warp, Wc lanes each
    const int sub = 32 / s.Wc, gsub = lane / s.Wc, w = lane - gsub * s.Wc;
    const bool active = gsub < sub;
    for (int L = 0; L < nl; ++L) {
      const uint32_t le = __ldg(layer_off + L + 1);
      if (active)
        for (uint32_t g = lb + warp * sub + gsub; g < le; g += nw * sub)
          apply_gate(dbg_code(__ldg(ops + g), (uint32_t)s.n, s.err), s.X, s.Z, s.Wp, w, r0, npauli);
      lb = le;
      __syncthreads();
    }
    if (active && r0) atomicXor(&s.R[w], r0);
  }
  __syncthreads();
}

// Measure Z_a (code = MZ / MZR on qubit a) with pre-drawn bit rbit.  Returns
// the outcome (same value in every thread).  `next_code` (kNoNext: none) is
// the measurement that follows with no gate in between: a random-outcome
// measurement then also does the next one's pivot phase (its column's X bits
// are final once the rowsum is done) inside its last phase, and sets *pre;
// the next call, given *pre, skips that phase and its barrier.
constexpr uint32_t kNoNext = 0xFFFFFFFFu;
// kCount: instances that update the work counters (s.work) are separate
// from the ones timed, which carry no counting code.
template <bool kCount = false>
__device__ int sct_measure(const Sct& s, uint32_t code, uint32_t rbit, int* err,
                           uint32_t next_code = kNoNext, bool* pre = nullptr) {
  __shared__ int s_pw;
  __shared__ uint32_t s_cnt;  // list lengths: X in bits 0-9, Z 10-19, Y 20-29
  static_assert(TAB_BATCH_MAX_QUBITS < 1024, "list lengths are packed in 10-bit fields");
  __shared__ uint32_t s_acc;
  const int tid = threadIdx.x, T = blockDim.x;
  const int a = (int)dbg_index(dq1(code), (uint32_t)s.n, err);
  const bool reset = dop(code) == OP_MZR;
  const int n = s.n, Whc = s.Whc, Wc = s.Wc, Wp = s.Wp;
  const uint32_t* xa = s.X + (size_t)a * Wp;
  if (!(pre && *pre)) {  // pivot phase: the mask S, zeroed counters, the pivot word
    for (int w = tid; w < Wc; w += T) {
      s.sS[w] = xa[w];
      s.redlo[w] = 0u;
      s.redhi[w] = 0u;
    }
    if (tid < 32) {
      const uint32_t v = (tid < Whc) ? xa[Whc + tid] : 0u;
      const uint32_t bal = __ballot_sync(0xffffffffu, v != 0u);
      if (tid == 0) {
        s_pw = bal ? Whc + __ffs(bal) - 1 : -1;
        s_cnt = 0u;
        s_acc = 0u;
      }
    }
    __syncthreads();
  }
  const int pw = s_pw;
  if (pw >= 0) {
    // ---------------- random outcome ----------------
    const int P = pw * 32 + __ffs(s.sS[pw]) - 1;
    const int Pd = P - 32 * Whc;
    const int wp = pw, wd = Pd >> 5;
    const uint32_t bpm = 1u << (P & 31);
    const uint32_t rp = (s.R[wp] & bpm) ? 1u : 0u;
    const int lane = tid & 31;
    // row p on every column: the columns where it is X, Z or Y go to three
    // lists (warp-aggregated appends).  Rows p-n and p are rewritten here, on
    // every column (row p-n := row p, row p := Z_a): the rowsum below leaves
    // both rows alone (S' excludes them), and their exponent counters are
    // never read.
    uint32_t* lX = s.supp;
    uint32_t* lZ = s.supp + n;
    uint32_t* lY = s.supp + 2 * n;
    for (int j0 = tid - lane; j0 < n; j0 += T) {  // warp-uniform trip count
      const int j = j0 + lane;
      uint32_t xp = 0u, zp = 0u;
      if (j < n) {
        uint32_t* xc = s.X + (size_t)j * Wp;
        uint32_t* zc = s.Z + (size_t)j * Wp;
        xp = (xc[wp] & bpm) ? 1u : 0u;
        zp = (zc[wp] & bpm) ? 1u : 0u;
        xc[wd] = (xc[wd] & ~bpm) | (xp ? bpm : 0u);
        zc[wd] = (zc[wd] & ~bpm) | (zp ? bpm : 0u);
        xc[wp] &= ~bpm;
        zc[wp] = (zc[wp] & ~bpm) | ((j == a) ? bpm : 0u);
      }
      const uint32_t bx = __ballot_sync(0xffffffffu, xp & ~zp);
      const uint32_t bz = __ballot_sync(0xffffffffu, ~xp & zp);
      const uint32_t by = __ballot_sync(0xffffffffu, xp & zp);
      // one atomic for the three list lengths (packed 10-bit fields)
      uint32_t old = 0u;
      if (lane == 0 && (bx | bz | by))
        old = atomicAdd(&s_cnt, (uint32_t)__popc(bx) | ((uint32_t)__popc(bz) << 10) |
                                    ((uint32_t)__popc(by) << 20));
      old = __shfl_sync(0xffffffffu, old, 0);
      const int ox = (int)(old & 1023u), oz = (int)((old >> 10) & 1023u),
                oy = (int)((old >> 20) & 1023u);
      const uint32_t lt = (1u << lane) - 1u;
      if (xp & ~zp) lX[ox + __popc(bx & lt)] = (uint32_t)j;
      if (~xp & zp) lZ[oz + __popc(bz & lt)] = (uint32_t)j;
      if (xp & zp) lY[oy + __popc(by & lt)] = (uint32_t)j;
    }
    __syncthreads();
    const uint32_t cnt = s_cnt;
    const int nx = (int)(cnt & 1023u), nz = (int)((cnt >> 10) & 1023u), ny = (int)((cnt >> 20) & 1023u);
    if (kCount && s.work && tid == 0) {  // work counters: the pivot row's support
      atomicAdd(s.work, (unsigned long long)(nx + nz + ny) * (unsigned long long)Wc);
      atomicAdd(s.work + 2, 1ull);
    }
    const int g = tid / Wc, w = tid - g * Wc;
    if (g < s.GG) {
      // per row h of this word: rows in S' (x_ha = 1, h != p, p-n) take
      // row p into them; the exponent counter (lo, hi) adds, per column,
      //   X: +1 if x z, -1 if !x z         Z: +1 if x z, -1 if x !z, +2 if x
      //   Y: +1 if x z, -1 if !x !z, +2 if x
      // (the terms of 2 r_h' above with row p's bits fixed); rows outside S'
      // get counts too, but only S' rows are read
      uint32_t lo = 0u, hi = 0u, lo2 = 0u, hi2 = 0u;
      uint32_t Sw = s.sS[w];
      if (w == wp || w == wd) Sw &= ~bpm;  // S' excludes rows p and p-n
      // two columns per iteration, each into a counter of its own (summed
      // at the end: addition mod 4 is associative), so the two columns'
      // loads and updates are independent chains
      const int GG = s.GG;
      int idx = g;
      for (; idx + GG < nx; idx += 2 * GG) {
        const size_t i0 = (size_t)lX[idx] * Wp + w, i1 = (size_t)lX[idx + GG] * Wp + w;
        const uint32_t x0 = s.X[i0], z0 = s.Z[i0], x1 = s.X[i1], z1 = s.Z[i1];
        hi ^= z0 & ~(x0 ^ lo);
        lo ^= z0;
        hi2 ^= z1 & ~(x1 ^ lo2);
        lo2 ^= z1;
        s.X[i0] = x0 ^ Sw;
        s.X[i1] = x1 ^ Sw;
      }
      if (idx < nx) {
        const size_t i = (size_t)lX[idx] * Wp + w;
        const uint32_t x = s.X[i], z = s.Z[i];
        hi ^= z & ~(x ^ lo);
        lo ^= z;
        s.X[i] = x ^ Sw;
      }
      for (idx = g; idx + GG < nz; idx += 2 * GG) {
        const size_t i0 = (size_t)lZ[idx] * Wp + w, i1 = (size_t)lZ[idx + GG] * Wp + w;
        const uint32_t x0 = s.X[i0], z0 = s.Z[i0], x1 = s.X[i1], z1 = s.Z[i1];
        hi ^= x0 & (z0 ^ lo);
        lo ^= x0;
        hi2 ^= x1 & (z1 ^ lo2);
        lo2 ^= x1;
        s.Z[i0] = z0 ^ Sw;
        s.Z[i1] = z1 ^ Sw;
      }
      if (idx < nz) {
        const size_t i = (size_t)lZ[idx] * Wp + w;
        const uint32_t x = s.X[i], z = s.Z[i];
        hi2 ^= x & (z ^ lo2);
        lo2 ^= x;
        s.Z[i] = z ^ Sw;
      }
      for (idx = g; idx + GG < ny; idx += 2 * GG) {
        const size_t i0 = (size_t)lY[idx] * Wp + w, i1 = (size_t)lY[idx + GG] * Wp + w;
        const uint32_t x0 = s.X[i0], z0 = s.Z[i0], x1 = s.X[i1], z1 = s.Z[i1];
        const uint32_t e0 = ~(x0 ^ z0), e1 = ~(x1 ^ z1);
        hi ^= (e0 & ~(x0 ^ lo)) ^ x0;
        lo ^= e0;
        hi2 ^= (e1 & ~(x1 ^ lo2)) ^ x1;
        lo2 ^= e1;
        s.X[i0] = x0 ^ Sw;
        s.Z[i0] = z0 ^ Sw;
        s.X[i1] = x1 ^ Sw;
        s.Z[i1] = z1 ^ Sw;
      }
      if (idx < ny) {
        const size_t i = (size_t)lY[idx] * Wp + w;
        const uint32_t x = s.X[i], z = s.Z[i];
        const uint32_t e = ~(x ^ z);
        hi ^= (e & ~(x ^ lo)) ^ x;
        lo ^= e;
        s.X[i] = x ^ Sw;
        s.Z[i] = z ^ Sw;
      }
      add4s(lo, hi, lo2, hi2);
      // this group's counters into the word's accumulator: a bit-sliced add
      // through two atomic XORs, exact under any interleaving (the carry
      // uses the low plane as the atomic returned it, so the adds serialise
      // in the order of the low-plane atomics; the high plane only takes
      // XORs)
      if (lo | hi) {
        const uint32_t old = atomicXor(&s.redlo[w], lo);
        atomicXor(&s.redhi[w], hi ^ (old & lo));
      }
    }
    __syncthreads();
    // every word: the summed counters, row p's share and the sign update;
    // then (with a next measurement) that measurement's pivot phase, each
    // thread on the words it has just read
    const bool nxt = next_code != kNoNext;
    const uint32_t* xn = s.X + (size_t)(nxt ? dbg_index(dq1(next_code), (uint32_t)n, err) : 0u) * Wp;
    for (int ww = tid; ww < Wc; ww += T) {
      uint32_t L = s.redlo[ww], H = s.redhi[ww];
      const uint32_t scal = ((uint32_t)ny + 2u * rp) & 3u;
      add4s(L, H, (scal & 1u) ? 0xffffffffu : 0u, (scal & 2u) ? 0xffffffffu : 0u);
      uint32_t Sw = s.sS[ww];
      if (ww == wp || ww == wd) Sw &= ~bpm;
      if (L & Sw) atomicCAS(err, 0, DERR_PHASE);
      uint32_t r = s.R[ww] ^ (H & Sw);
      if (ww == wd) r = (r & ~bpm) | (rp ? bpm : 0u);
      if (ww == wp) r = (r & ~bpm) | (rbit ? bpm : 0u);
      if (reset && rbit) r ^= s.Z[(size_t)a * Wp + ww];  // X_a on every row
      s.R[ww] = r;
      if (nxt) {
        s.sS[ww] = xn[ww];
        s.redlo[ww] = 0u;
        s.redhi[ww] = 0u;
      }
    }
    // the next pivot word on the last warp, beside the per-word updates of
    // the first (T >= 64; Whc <= 20 words fit one warp)
    const int pt = tid - (T - 32);
    if (nxt && pt >= 0) {
      const uint32_t v = (pt < Whc) ? xn[Whc + pt] : 0u;
      const uint32_t bal = __ballot_sync(0xffffffffu, v != 0u);
      if (pt == 0) {
        s_pw = bal ? Whc + __ffs(bal) - 1 : -1;
        s_cnt = 0u;
        s_acc = 0u;
      }
    }
    __syncthreads();
    if (pre) *pre = nxt;
    return (int)rbit;
  }
  // ---------------- deterministic outcome ----------------
  if (kCount && s.work && tid == 0) {  // work counters: the rows multiplied
    uint32_t k = 0u;
    for (int hw = 0; hw < Whc; ++hw) k += __popc(s.sS[hw]);
    atomicAdd(s.work + 1, (unsigned long long)k * (unsigned long long)Wc);
    atomicAdd(s.work + 3, 1ull);
  }
  const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;  // (random case returned above)
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t acc = 0u;
  for (int j = warp; j < n; j += nw) {
    uint32_t carry = 0u;
    for (int base = 0; base < Whc; base += 32) {
      const int hw = base + lane;
      uint32_t xT = 0u, zT = 0u;
      if (hw < Whc) {
        const uint32_t t = s.sS[hw];
        xT = s.X[(size_t)j * Wp + Whc + hw] & t;
        zT = s.Z[(size_t)j * Wp + Whc + hw] & t;
      }
      acc += __popc(xT & zT);
      const uint32_t bal = __ballot_sync(0xffffffffu, __popc(zT) & 1);
      const uint32_t cin = (__popc(bal & lt) & 1u) ^ carry;
      const uint32_t zpre = prefix_xor_exclusive(zT) ^ (cin ? 0xffffffffu : 0u);
      acc += 2u * (__popc(xT & zpre) & 1u);
      carry ^= __popc(bal) & 1u;
    }
  }
  for (int hw = tid; hw < Whc; hw += T) acc += 2u * __popc(s.R[Whc + hw] & s.sS[hw]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) atomicAdd(&s_acc, acc & 3u);
  __syncthreads();
  const uint32_t e = s_acc & 3u;
  if ((e & 1u) && tid == 0) atomicCAS(err, 0, DERR_PHASE);
  const int out = (int)(e >> 1);
  if (reset && out)
    for (int w = tid; w < Wc; w += T) s.R[w] ^= s.Z[(size_t)a * Wp + w];
  __syncthreads();
  if (pre) *pre = false;
  return out;
}

// ------------------------------------------ terminal-measurement sampler ---
// When a circuit's measurements are all at its end (Z only, no reset), which
// measurements are random, their pivots and masks, and every X|Z update are
// the same in every shot: none of them reads a sign or an outcome.  Every
// sign, and so every deterministic outcome, is then an affine function over
// GF(2) of the random bits b_0, b_1, ... of the earlier random measurements
// (a rowsum adds row p's sign plus an X|Z-only term; row p of measurement i
// becomes b_i).  So the terminal run is done once per circuit with each sign
// kept as such a form -- R holds the constant part, and column j of F (the
// tableau's column layout) holds the coefficient of b_j -- and every shot is
// evaluated from its own Philox bits.  The outcomes are those of running the
// shot itself, bit for bit.
//
// forms[i*(1+FW)]: bit 0 = measurement i is random (outcome b_i), bit 1 =
// constant of a deterministic outcome; words 1..FW: its coefficients.
template <bool kCount = false>
__device__ void sct_form_pass(const Sct& s, const uint32_t* __restrict__ ops, uint32_t op_begin,
                              int K, uint32_t* F, int* fpl, uint32_t* forms, int FW, int* err) {
  __shared__ int s_fpw, s_nf;
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
  const int Wc = s.Wc, Wp = s.Wp, Whc = s.Whc;
  const uint32_t lt = (1u << lane) - 1u;
  for (size_t e = tid; e < (size_t)K * Wp; e += T) F[e] = 0u;
  __syncthreads();
  for (int i = 0; i < K; ++i) {
    const uint32_t code = __ldg(ops + op_begin + i);
    // X|Z bits, pivot, mask and the constant parts of the signs, with b_i = 0
    const int c = sct_measure<kCount>(s, code, 0u, err);
    // s.sS still holds the measured column's X plane before the measurement
    if (tid < 32) {
      const uint32_t v = (tid < Whc) ? s.sS[Whc + tid] : 0u;
      const uint32_t bal = __ballot_sync(0xffffffffu, v != 0u);
      if (tid == 0) {
        s_fpw = bal ? Whc + __ffs(bal) - 1 : -1;
        s_nf = 0;
      }
    }
    __syncthreads();
    uint32_t* hdr = forms + (size_t)i * (1 + FW);
    const int pw = s_fpw;
    if (pw >= 0) {
      const int P = pw * 32 + __ffs(s.sS[pw]) - 1;
      const int wp = pw, wd = (P - 32 * Whc) >> 5;
      const uint32_t bpm = 1u << (P & 31);
      // columns whose bit p is set: row p's form has b_j; the others only
      // lose row p-n's bit (row p-n := row p)
      for (int j0 = tid - lane; j0 < i; j0 += T) {  // warp-uniform trip count
        const int j = j0 + lane;
        const bool f = j < i && (F[(size_t)j * Wp + wp] & bpm);
        const uint32_t bal = __ballot_sync(0xffffffffu, f);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(&s_nf, __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (f) fpl[base + __popc(bal & lt)] = j;
        else if (j < i) F[(size_t)j * Wp + wd] &= ~bpm;
      }
      __syncthreads();
      const int nf = s_nf;
      for (int e = tid; e < nf * Wc; e += T) {
        const int idx = e / Wc, w = e - idx * Wc;
        uint32_t* col = F + (size_t)fpl[idx] * Wp;
        uint32_t Sw = s.sS[w];
        if (w == wp || w == wd) Sw &= ~bpm;  // S' excludes rows p and p-n
        uint32_t v = col[w] ^ Sw;
        if (w == wd) v |= bpm;   // row p-n := row p
        if (w == wp) v &= ~bpm;  // row p := b_i
        col[w] = v;
      }
      if (tid == 0) {
        F[(size_t)i * Wp + wp] |= bpm;
        hdr[0] = 1u;
      }
    } else {
      // deterministic: coefficient of b_j = parity of column j over the
      // stabilizer rows the destabilizer column selects
      for (int f = warp; f < FW; f += nw) {
        const int j = f * 32 + lane;
        uint32_t acc = 0u;
        if (j < i)
          for (int hw = 0; hw < Whc; ++hw) acc += __popc(F[(size_t)j * Wp + Whc + hw] & s.sS[hw]);
        const uint32_t word = __ballot_sync(0xffffffffu, acc & 1u);
        if (lane == 0) hdr[1 + f] = word;
      }
      if (tid == 0) hdr[0] = (uint32_t)c << 1;
    }
    __syncthreads();
  }
}

// Outcomes of every shot from the forms: random ones are the shot's Philox
// bits, deterministic ones constant ^ parity(coefficients & bits).
__device__ void sct_sample(const uint32_t* forms, int K, int FW, int shots, uint64_t seed,
                           uint64_t cid, uint8_t* out, uint32_t* Bs) {
  const int tid = threadIdx.x, T = blockDim.x;
  for (int e = tid; e < shots * FW; e += T) Bs[e] = 0u;
  __syncthreads();
  for (int e = tid; e < shots * K; e += T) {
    const int sh = e / K, i = e - sh * K;
    if (__ldcg(forms + (size_t)i * (1 + FW)) & 1u) {
      const uint32_t b = outcome_bit(seed, cid, (uint32_t)sh, (uint64_t)i);
      out[(size_t)sh * K + i] = (uint8_t)b;
      if (b) atomicOr(Bs + (size_t)sh * FW + (i >> 5), 1u << (i & 31));
    }
  }
  __syncthreads();
  for (int e = tid; e < shots * K; e += T) {
    const int sh = e / K, i = e - sh * K;
    const uint32_t* h = forms + (size_t)i * (1 + FW);
    const uint32_t hd = __ldcg(h);
    if (hd & 1u) continue;
    uint32_t o = (hd >> 1) & 1u;
    for (int f = 0; f < FW; ++f) o ^= __popc(__ldcg(h + 1 + f) & Bs[(size_t)sh * FW + f]) & 1u;
    out[(size_t)sh * K + i] = (uint8_t)o;
  }
}

// -------------------------------------------- global <-> shared transfers ---
// Image layout (batched scratch): the shared-memory X, Z planes then R.
__device__ void sct_store_image(const Sct& s, uint32_t* __restrict__ img) {
  const size_t tot = (size_t)2 * s.n * s.Wp + s.Wc;
  for (size_t i = threadIdx.x; i < tot; i += blockDim.x) img[i] = s.X[i];
}
__device__ void sct_load_image(const Sct& s, const uint32_t* __restrict__ img) {
  const size_t tot = (size_t)2 * s.n * s.Wp + s.Wc;
  for (size_t i = threadIdx.x; i < tot; i += blockDim.x) s.X[i] = __ldcg(img + i);
}
// Handle layout: Wh words per half (multiple of 4), W = 2*Wh per column.
__device__ void sct_load_global(const Sct& s, const uint32_t* X, const uint32_t* Z,
                                const uint32_t* R, int Wh) {
  const int W = 2 * Wh;
  const int tot = s.n * s.Wc;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int a = i / s.Wc, w = i - a * s.Wc;
    const int gw = w < s.Whc ? w : Wh + (w - s.Whc);
    s.X[(size_t)a * s.Wp + w] = X[(size_t)a * W + gw];
    s.Z[(size_t)a * s.Wp + w] = Z[(size_t)a * W + gw];
  }
  for (int w = threadIdx.x; w < s.Wc; w += blockDim.x)
    s.R[w] = R[w < s.Whc ? w : Wh + (w - s.Whc)];
}
__device__ void sct_store_global(const Sct& s, uint32_t* X, uint32_t* Z, uint32_t* R, int Wh) {
  const int W = 2 * Wh;
  const int tot = s.n * s.Wc;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int a = i / s.Wc, w = i - a * s.Wc;
    const int gw = w < s.Whc ? w : Wh + (w - s.Whc);
    X[(size_t)a * W + gw] = s.X[(size_t)a * s.Wp + w];
    Z[(size_t)a * W + gw] = s.Z[(size_t)a * s.Wp + w];
  }
  for (int w = threadIdx.x; w < s.Wc; w += blockDim.x) R[w < s.Whc ? w : Wh + (w - s.Whc)] = s.R[w];
}

// Run segments [seg_begin, seg_end) of a program on the resident tableau.
// Outcome k of this run goes to out[k]; k0 is the first measurement index.
template <bool kCount = false>
__device__ void sct_run_segments(const Sct& s, const Seg* __restrict__ segs, int seg_begin,
                                 int seg_end, const uint32_t* __restrict__ ops,
                                 const uint32_t* __restrict__ layer_off, uint64_t seed,
                                 uint64_t cid, uint32_t shot, uint64_t k0, uint8_t* out,
                                 int* err, const uint8_t* npauli = nullptr) {
  uint64_t k = k0;
  int o = 0;
  for (int si = seg_begin; si < seg_end; ++si) {
    const Seg g = segs[si];
    if (g.kind == 0) {
      sct_gates(s, ops, layer_off + g.layer_begin, (int)(g.layer_end - g.layer_begin), npauli);
    } else {
      __shared__ uint32_t s_rbits;  // outcome bits of the current 32 measurements
      uint32_t next_code = __ldg(ops + g.op_begin);  // fetched one step ahead
      bool pre = false;  // the next measurement's pivot phase is done
      for (uint32_t op = g.op_begin; op < g.op_end; ++op) {
        const uint32_t code = next_code;
        next_code = op + 1 < g.op_end ? __ldg(ops + op + 1) : kNoNext;
        const uint32_t t = (op - g.op_begin) & 31u;
        if (t == 0u) {  // warp 0 draws the next 32 outcome bits (lane i: k + i)
          if (threadIdx.x < 32) {
            const uint32_t b = outcome_bit(seed, cid, shot, k + threadIdx.x);
            const uint32_t bits = __ballot_sync(0xffffffffu, b != 0u);
            if (threadIdx.x == 0) s_rbits = bits;
          }
          __syncthreads();
        }
        const uint32_t rbit = (s_rbits >> t) & 1u;
        const int m = sct_measure<kCount>(s, code, rbit, err, next_code, &pre);
        if (threadIdx.x == 0) out[o] = (uint8_t)m;
        ++k;
        ++o;
      }
    }
  }
}

// ---------------------------------------------- plain path, one tableau ---
__global__ void __launch_bounds__(kSctThreads) k_sct_program(SctProgArgs A) {
  extern __shared__ uint32_t smem[];
  Sct s;
  sct_setup(s, smem, A.n, A.err);
  sct_load_global(s, A.X, A.Z, A.R, A.Wh);
  __syncthreads();
  sct_run_segments(s, A.segs, 0, A.nsegs, A.ops, A.layer_off, A.seed, A.cid, A.shot, A.k0,
                   A.out, A.err);
  __syncthreads();
  sct_store_global(s, A.X, A.Z, A.R, A.Wh);
}

cudaError_t launch_sct_program(const SctProgArgs& A, cudaStream_t st) {
  cudaError_t e = ensure_smem_limit((const void*)k_sct_program,
                                    (int)sct_smem_bytes(TAB_BATCH_MAX_QUBITS, kSctThreads));
  if (e != cudaSuccess) return e;
  k_sct_program<<<1, kSctThreads, sct_smem_bytes(A.n, kSctThreads), st>>>(A);
  return cudaGetLastError();
}

// ------------------------------------------------------- batched launch ---
// Work items: one "prefix" item per circuit (identity, then the gates before
// the first measurement; the resulting image is stored and its ready flag
// released) followed by one item per (circuit, shot) (wait for the flag, load
// the image, run the rest of the circuit with that shot's outcome stream).
// Items are dequeued in order from one atomic counter; every prefix item is
// dequeued before any shot item, and prefix items never wait, so every wait
// ends.  Waits are bounded anyway and latch DERR_TIMEOUT.
template <int T, bool kCount>
__global__ void __launch_bounds__(T) k_batch(BatchArgs A) {
  extern __shared__ uint32_t smem[];
  __shared__ unsigned int s_item;
  __shared__ int s_stop;
  const uint64_t seed = A.seed;
  uint8_t* out = A.out;
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(A.queue, 1u);
      s_stop = *(volatile int*)A.err != 0;
    }
    __syncthreads();
    const unsigned int it = s_item;
    const int stop = s_stop;
    __syncthreads();
    if (stop || it >= (unsigned int)A.nitems) break;
    const uint64_t item = A.items[it];
    const uint32_t ci = dbg_index((uint32_t)item, (uint32_t)A.ncirc, A.err),
                   shot = (uint32_t)(item >> 32);
    const BatchCirc C = A.circs[ci];
    Sct s;
    sct_setup(s, smem, C.n, A.err);
    s.work = kCount ? A.work : nullptr;
    uint32_t* img = A.img + C.img_off;
    if (shot == 0xFFFFFFFFu) {
      sct_identity(s);
      __syncthreads();
      if (C.n_prefix) {
        const Seg g = A.segs[C.seg_begin];
        sct_gates(s, A.ops, A.layer_off + g.layer_begin, (int)(g.layer_end - g.layer_begin));
      }
      if (C.sampled) {  // terminal measurements: one pass for every shot
        const int K = (int)C.n_meas, FW = (K + 31) / 32;
        uint32_t* F = smem + sct_smem_words(C.n, (int)blockDim.x);
        int* fpl = reinterpret_cast<int*>(F + (size_t)K * s.Wp);
        uint32_t* Bs = reinterpret_cast<uint32_t*>(fpl + K);
        const Seg g = A.segs[C.seg_begin + C.n_prefix];
        sct_form_pass<kCount>(s, A.ops, g.op_begin, K, F, fpl, img, FW, A.err);
        __syncthreads();
        sct_sample(img, K, FW, C.shots, seed, C.cid, out + C.out_off, Bs);
        __syncthreads();
        continue;
      }
      sct_store_image(s, img);
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(A.ready + ci, 1);
      }
    } else {
      if (threadIdx.x == 0) {
        const unsigned long long t0 = sct_gtimer();
        int ok = 1;
        while (atomicAdd(A.ready + ci, 0) == 0) {
          if (*(volatile int*)A.err != 0 || sct_gtimer() - t0 > kReadyWaitNs) {
            atomicCAS(A.err, 0, DERR_TIMEOUT);
            ok = 0;
            break;
          }
        }
        __threadfence();
        s_stop = !ok;
      }
      __syncthreads();
      if (s_stop) break;
      sct_load_image(s, img);
      // this shot's noise draws: op j fires when word 0 >> 4 of its Philox
      // block (counter (j, shot, cid lo, cid hi), key (seed lo, seed hi ^
      // tag)) is below its 28-bit probability; DEPOL1 then takes X, Y or Z by
      // floor(word 1 * 3 / 2^32)
      uint8_t* npauli = reinterpret_cast<uint8_t*>(smem + sct_smem_words(C.n, (int)blockDim.x));
      for (uint32_t j = threadIdx.x; j < C.n_noise; j += blockDim.x) {
        const uint32_t e = __ldg(A.noise + C.noise_off + j), kind = e >> 28;
        const uint4 rr = philox4x32_10(
            make_uint4(j, shot, (uint32_t)C.cid, (uint32_t)(C.cid >> 32)),
            make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ kNoiseKeyTag));
        uint8_t p = 0;
        if ((rr.x >> 4) < (e & 0xFFFFFFFu))
          p = kind == 1u ? (uint8_t)OP_X
                         : kind == 2u ? (uint8_t)OP_Z
                                      : (uint8_t)(OP_X + (uint32_t)(((uint64_t)rr.y * 3u) >> 32));
        npauli[j] = p;
      }
      __syncthreads();
      sct_run_segments<kCount>(s, A.segs, (int)(C.seg_begin + C.n_prefix), (int)C.seg_end, A.ops,
                       A.layer_off, seed, C.cid, shot, 0,
                       out + C.out_off + (uint64_t)shot * C.n_meas, A.err, npauli);
    }
    __syncthreads();
  }
}

// Thread counts the batched kernel is built for; the autotuner
// (tab_batch_tune) times each on the batch itself.
static const void* batch_kernel_for(int threads, bool count = false) {
  switch (threads) {
    case 128: return count ? (const void*)k_batch<128, true> : (const void*)k_batch<128, false>;
    case 256: return count ? (const void*)k_batch<256, true> : (const void*)k_batch<256, false>;
    case 512: return count ? (const void*)k_batch<512, true> : (const void*)k_batch<512, false>;
    case 1024: return count ? (const void*)k_batch<1024, true> : (const void*)k_batch<1024, false>;
    default: return nullptr;
  }
}

const void* batch_kernel_ptr(int threads, bool count) { return batch_kernel_for(threads, count); }

cudaError_t prepare_batch_kernel(int threads) {
  // the largest tableau, or a sampled circuit's tableau plus its forms; both
  // instances (timed and counting)
  for (const bool count : {false, true}) {
    const void* fn = batch_kernel_for(threads, count);
    if (!fn) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               227 * 1024 - 2048);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Resident CTAs per SM for `threads` and `smem` bytes (0: does not launch).
int batch_ctas_per_sm(int threads, size_t smem) {
  const void* fn = batch_kernel_for(threads);
  if (!fn || prepare_batch_kernel(threads) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    v = 0;
  }
  return v < 0 ? 0 : v;
}

}  // namespace tab
