// kernels_measure.cu -- Z measurement of a device-resident tableau (sm_103a).
//
// Operation (Aaronson & Gottesman, PRA 70, 052328, Sec. III; the measurement
// step of the Clifford backend in arXiv:2408.00384, "Simulation of Clifford
// circuits"): to measure Z_a,
//  * random case -- some stabilizer row p has x_pa = 1 (p = the smallest):
//    every other row h with x_ha = 1 becomes row_p * row_h, row p-n becomes
//    row p, row p becomes +-Z_a with the sign = the outcome bit;
//  * deterministic case -- the outcome is the sign of the product of the
//    stabilizer rows n+i over the destabilizers i with x_ia = 1.
//
// Design: one cooperative persistent launch runs a whole run of measurements.
// CTA c owns the qubit columns j = c, c+G, c+2G, ...; threads own 4-word
// quads of rows.  Per measurement there is exactly one grid barrier:
//  - every CTA reads column a (the mask of rows with x_ha = 1) and finds the
//    same pivot p;
//  - every CTA updates only its own columns, reading the pivot row's bits
//    from those columns.
// Sign bookkeeping is lazy and linear: the true sign of row h is
// (R4[h] + sum_c PH[c][h]) / 2 with mod-4 partials PH[c] owned by CTA c, so a
// CTA adds its columns' share of every rowsum exponent to its own partial and
// no CTA ever reads another's partial until the final fold.  Writing the
// rowsum exponent of row_p * row_h in the form (i^e X^x Z^z with
// e = 2r + |x&z|, products adding e_p + e_h + 2 z_p.x_h):
//   2 r_h' = 2 r_h + 2 r_p + sum_j [x_pj z_pj + x_hj z_hj - x'_hj z'_hj
//                                   + 2 z_pj x_hj]        (mod 4),
// with x' = x_h ^ x_p, z' = z_h ^ z_p.  The column-a X plane after a random
// measurement is known in closed form (only row p-n is set); its write is
// deferred by one measurement so no CTA overwrites it while others read it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "grid_sync.cuh"
#include "philox.cuh"
#include "tab_internal.h"

namespace tab {

constexpr int kMeasThreads = 512;

struct MArgs {
  uint32_t* X;
  uint32_t* Z;
  uint32_t* R;
  int n, Wh, W;
  const uint32_t* mops;
  int nm;
  uint64_t k0, seed, cid;
  uint32_t shot;
  uint8_t* out;
  uint32_t* ph;  // [G][2][W]
  uint32_t* r4;  // [2][W]
  uint32_t* dp;  // [2][G]
  unsigned long long wait_ns;  // limit of each grid-barrier wait
  GridBar* bar;
  int* err;
  unsigned long long* work;  // MeasWork::work (null: not counting)
};

// mod-4 bit-sliced add: (h, l) += (bh, bl)
__device__ __forceinline__ void add4(uint32_t& l, uint32_t& h, uint32_t bl, uint32_t bh) {
  h ^= bh ^ (l & bl);
  l ^= bl;
}

__device__ __forceinline__ uint32_t prefix_xor_excl(uint32_t v) {
  uint32_t y = v << 1;
  y ^= y << 1;
  y ^= y << 2;
  y ^= y << 4;
  y ^= y << 8;
  y ^= y << 16;
  return y;
}

// Deterministic outcome: sum of the G partials (mod 4) of buffer `buf`.
// Returns the outcome (0/1) or -1 on an odd total; called by one warp.
__device__ int det_outcome_warp(const uint32_t* dp, int G) {
  uint32_t s = 0;
  for (int i = threadIdx.x & 31; i < G; i += 32) s += __ldcg(dp + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  s &= 3u;
  return (s & 1u) ? -1 : (int)(s >> 1);
}

__global__ void __launch_bounds__(kMeasThreads) k_measure(MArgs A) {
  unsigned int epoch = 0;  // grid barriers passed (grid_sync)
  extern __shared__ uint32_t smem[];
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
  const int n = A.n, Wh = A.Wh, W = A.W, Q = W / 4;
  const int ncols = (n - c + G - 1) / G;  // columns owned by this CTA
  uint32_t* sS = smem;                    // [W] mask (column a, X plane)
  uint32_t* sZA = sS + W;                 // [W] new Z column a (reset term)
  uint32_t* sSupp = sZA + W;              // [ncols] support list of the pivot row
  uint32_t* sRed = sSupp + ((ncols + 3) & ~3);  // [GG][Q][8] partial counters
  __shared__ int s_pw, s_nsupp, s_kc, s_det_out;
  __shared__ uint32_t s_rbits;  // outcome bits of the current 32 measurements
  __shared__ uint32_t s_php, s_r4p;  // row p's own partial / base sign: bit0 lo, bit1 hi

  uint32_t* PHlo = A.ph + (size_t)c * 2 * W;
  uint32_t* PHhi = PHlo + W;
  uint32_t* R4lo = A.r4;
  uint32_t* R4hi = A.r4 + W;

  // initial partials: zero; base = current signs (as 2*r)
  for (int w = tid; w < W; w += blockDim.x) {
    PHlo[w] = 0u;
    PHhi[w] = 0u;
    if (c == 0) {
      R4lo[w] = 0u;
      R4hi[w] = A.R[w];
    }
  }
  __syncthreads();

  const int GG = (Q <= (int)blockDim.x) ? (int)blockDim.x / Q : 1;
  int pend_a = -1, pend_pd = -1;              // column whose X write is deferred
  int prev_det = 0, prev_a = 0, prev_reset = 0;  // unresolved deterministic outcome

  uint32_t next_code = A.nm > 0 ? __ldg(A.mops) : 0u;  // fetched one step ahead
  for (int m = 0; m < A.nm; ++m) {
    const uint32_t code = next_code;
    if (m + 1 < A.nm) next_code = __ldg(A.mops + m + 1);
    if (m > 0 && !grid_sync(A.bar, A.err, epoch, A.wait_ns)) return;
    // ---- resolve the previous deterministic outcome (needs every CTA's partial)
    if (prev_det) {
      const uint32_t* dbuf = A.dp + (size_t)((m - 1) & 1) * G;
      const bool owner = (prev_a % G) == c;
      if (tid < 32 && (c == 0 || (owner && prev_reset))) {
        const int o = det_outcome_warp(dbuf, G);
        if (tid == 0) {
          if (o < 0) atomicCAS(A.err, 0, DERR_PHASE);
          s_det_out = o < 0 ? 0 : o;
          if (c == 0) A.out[m - 1] = (uint8_t)s_det_out;
        }
      }
      __syncthreads();
      if (owner && prev_reset && s_det_out) {  // X on qubit prev_a: r_i ^= z_i,prev_a
        const uint32_t* zc = A.Z + (size_t)prev_a * W;
        for (int w = tid; w < W; w += blockDim.x) PHhi[w] ^= zc[w];
      }
      prev_det = 0;
    }

    const int a = (int)dbg_index(dq1(code), (uint32_t)A.n, A.err);
    const int reset = dop(code) == OP_MZR;
    // outcome bits of measurements m .. m+31, drawn by warp 0 once every 32
    // measurements (lane i: measurement m+i); read after the barrier below
    if ((m & 31) == 0 && tid < 32) {
      const uint32_t b = outcome_bit(A.seed, A.cid, A.shot, A.k0 + (uint64_t)(m + tid));
      const uint32_t bits = __ballot_sync(0xffffffffu, b != 0u);
      if (tid == 0) s_rbits = bits;
    }

    // ---- phase A: mask S = X column a, pivot p = first stabilizer row in S
    if (tid == 0) s_pw = 0x7fffffff;
    for (int w = tid; w < W; w += blockDim.x) {
      uint32_t v;
      if (a == pend_a) v = (w == (pend_pd >> 5)) ? (1u << (pend_pd & 31)) : 0u;
      else v = __ldcg(A.X + (size_t)a * W + w);
      sS[w] = v;
    }
    __syncthreads();
    for (int w = Wh + tid; w < W; w += blockDim.x)
      if (sS[w]) atomicMin(&s_pw, w);
    __syncthreads();
    const int pw = s_pw;

    // ---- phase B: materialize the deferred column (its owner only).  No CTA
    // reads that column from memory in phase A (a == pend_a uses the closed
    // form), so the write cannot race with a reader.
    if (pend_a >= 0 && (pend_a % G) == c) {
      uint32_t* xc = A.X + (size_t)pend_a * W;
      for (int w = tid; w < W; w += blockDim.x)
        xc[w] = (w == (pend_pd >> 5)) ? (1u << (pend_pd & 31)) : 0u;
    }
    pend_a = -1;
    __syncthreads();
    const uint32_t rbit = (s_rbits >> (m & 31)) & 1u;

    if (pw != 0x7fffffff) {
      // ================= random outcome =================
      const int P = pw * 32 + (__ffs(sS[pw]) - 1);
      const int Pd = P - 32 * Wh;
      const int wp = P >> 5, wd = Pd >> 5;
      const uint32_t bpm = 1u << (P & 31);
      if (tid == 0) {
        s_nsupp = 0;
        s_kc = 0;
        const uint32_t plo = (PHlo[wp] & bpm) ? 1u : 0u, phi = (PHhi[wp] & bpm) ? 1u : 0u;
        s_php = plo | (phi << 1);
        if (c == 0) {
          const uint32_t blo = (R4lo[wp] & bpm) ? 1u : 0u, bhi = (R4hi[wp] & bpm) ? 1u : 0u;
          s_r4p = blo | (bhi << 1);
        }
      }
      __syncthreads();
      // pre-pass: pivot-row bits of own columns; clear row p-n where row p is I
      for (int idx = tid; idx < ncols; idx += blockDim.x) {
        const int j = c + idx * G;
        const uint32_t xw = __ldcg(A.X + (size_t)j * W + wp);
        const uint32_t zw = __ldcg(A.Z + (size_t)j * W + wp);
        const uint32_t xp = (xw & bpm) ? 1u : 0u, zp = (zw & bpm) ? 1u : 0u;
        if (xp | zp) {
          const int pos = atomicAdd(&s_nsupp, 1);
          sSupp[pos] = (uint32_t)j | (xp << 30) | (zp << 31);
          if (xp & zp) atomicAdd(&s_kc, 1);
        } else {
          uint32_t* xd = A.X + (size_t)j * W + wd;
          uint32_t* zd = A.Z + (size_t)j * W + wd;
          const uint32_t xv = __ldcg(xd), zv = __ldcg(zd);
          if (xv & bpm) *xd = xv & ~bpm;
          if (zv & bpm) *zd = zv & ~bpm;
        }
      }
      __syncthreads();
      const int nsupp = s_nsupp;
      if (A.work && tid == 0) {  // work counters: this CTA's support columns
        atomicAdd(A.work, (unsigned long long)nsupp);
        if (c == 0) atomicAdd(A.work + 2, 1ull);
      }
      // scalar added to every row in S': this CTA's share of
      // 2 r_p (= its partial of row p, plus the base for CTA 0) + sum x_pj z_pj
      uint32_t scal = (uint32_t)s_kc + (s_php & 1u) + 2u * (s_php >> 1);
      if (c == 0) scal += (s_r4p & 1u) + 2u * (s_r4p >> 1);
      scal &= 3u;
      const bool own_a = (a % G) == c;
      // main pass: threads own quads q of rows, groups g split the support list
      const int q = tid % Q, g = tid / Q;
      if (g < GG) {
        uint32_t lo[4] = {0u, 0u, 0u, 0u}, hi[4] = {0u, 0u, 0u, 0u};
        uint32_t sm4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int w = 4 * q + k;
          uint32_t s = sS[w];
          if (w == wp || w == wd) s &= ~bpm;  // S' excludes rows p and p-n
          sm4[k] = s;
        }
        for (int idx = g; idx < nsupp; idx += GG) {
          const uint32_t e = sSupp[idx];
          const int j = (int)(e & 0x3FFFu);
          const uint32_t XP = (e & (1u << 30)) ? 0xffffffffu : 0u;
          const uint32_t ZP = (e & (1u << 31)) ? 0xffffffffu : 0u;
          uint4* xq = reinterpret_cast<uint4*>(A.X + (size_t)j * W) + q;
          uint4* zq = reinterpret_cast<uint4*>(A.Z + (size_t)j * W) + q;
          const uint4 xv = __ldcg(xq), zv = __ldcg(zq);
          uint32_t xs[4] = {xv.x, xv.y, xv.z, xv.w}, zs[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t x = xs[k], z = zs[k];
            const uint32_t A0 = x & z;
            const uint32_t B0 = (x ^ XP) & (z ^ ZP);
            const uint32_t inc = A0 & ~B0, dec = B0 & ~A0;
            hi[k] ^= ((lo[k] & inc) | (~lo[k] & dec)) ^ (ZP & x);
            lo[k] ^= inc | dec;
            uint32_t xn = x ^ (XP & sm4[k]);
            uint32_t zn = z ^ (ZP & sm4[k]);
            const int w = 4 * q + k;
            if (w == wd) {  // row p-n := row p
              xn = (xn & ~bpm) | (XP & bpm);
              zn = (zn & ~bpm) | (ZP & bpm);
            }
            if (w == wp) {  // row p := Z_a
              xn &= ~bpm;
              zn = (zn & ~bpm) | ((j == a) ? bpm : 0u);
            }
            xs[k] = xn;
            zs[k] = zn;
          }
          if (j != a) *xq = make_uint4(xs[0], xs[1], xs[2], xs[3]);
          *zq = make_uint4(zs[0], zs[1], zs[2], zs[3]);
          if (j == a) {
#pragma unroll
            for (int k = 0; k < 4; ++k) sZA[4 * q + k] = zs[k];
          }
        }
        uint32_t* red = sRed + ((size_t)g * Q + q) * 8;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          red[k] = lo[k];
          red[4 + k] = hi[k];
        }
      }
      __syncthreads();
      // combine groups, add the scalar, mask by S', fold into own partial
      if (tid < Q) {
        const uint32_t s0 = (scal & 1u) ? 0xffffffffu : 0u, s1 = (scal & 2u) ? 0xffffffffu : 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int w = 4 * tid + k;
          uint32_t L = 0u, H = 0u;
          for (int gg = 0; gg < GG; ++gg) {
            const uint32_t* red = sRed + ((size_t)gg * Q + tid) * 8;
            add4(L, H, red[k], red[4 + k]);
          }
          add4(L, H, s0, s1);
          uint32_t s = sS[w];
          if (w == wp || w == wd) s &= ~bpm;
          L &= s;
          H &= s;
          uint32_t pl = PHlo[w], phh = PHhi[w];
          add4(pl, phh, L, H);
          if (w == wd) {  // sign partial of row p-n := that of row p
            pl = (pl & ~bpm) | ((s_php & 1u) ? bpm : 0u);
            phh = (phh & ~bpm) | ((s_php & 2u) ? bpm : 0u);
          }
          if (w == wp) {
            pl &= ~bpm;
            phh &= ~bpm;
          }
          if (own_a && reset && rbit) phh ^= sZA[w];  // reset: X_a on every row
          PHlo[w] = pl;
          PHhi[w] = phh;
          if (c == 0 && (w == wp || w == wd)) {
            uint32_t bl = R4lo[w], bh = R4hi[w];
            if (w == wd) {  // base sign of row p-n := that of row p
              bl = (bl & ~bpm) | ((s_r4p & 1u) ? bpm : 0u);
              bh = (bh & ~bpm) | ((s_r4p & 2u) ? bpm : 0u);
            } else {
              bl &= ~bpm;
              bh = (bh & ~bpm) | (rbit ? bpm : 0u);
            }
            R4lo[w] = bl;
            R4hi[w] = bh;
          }
        }
      }
      if (c == 0 && tid == 0) A.out[m] = (uint8_t)rbit;
      pend_a = a;
      pend_pd = Pd;
      __syncthreads();
    } else {
      // ================= deterministic outcome =================
      // T = stabilizer rows n+i for destabilizers i in S; e = sum_{m in T}
      // (2 r_m + |x_m & z_m|) + 2 sum_{m<l in T} z_m . x_l  (mod 4)
      uint32_t acc = 0u;
      if (A.work && c == 0) {  // work counters: the rows multiplied
        uint32_t k = 0u;
        for (int w = tid; w < Wh; w += blockDim.x) k += __popc(sS[w]);
        if (k) atomicAdd(A.work + 1, (unsigned long long)k);
        if (tid == 0) atomicAdd(A.work + 3, 1ull);
      }
      for (int w = Wh + tid; w < W; w += blockDim.x) {
        const uint32_t t = sS[w - Wh];
        acc += __popc(PHlo[w] & t) + 2u * __popc(PHhi[w] & t);
        if (c == 0) acc += __popc(R4lo[w] & t) + 2u * __popc(R4hi[w] & t);
      }
      const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
      const uint32_t lt = (1u << lane) - 1u;
      for (int idx = warp; idx < ncols; idx += nwarps) {
        const int j = c + idx * G;
        uint32_t carry = 0u;
        for (int base = 0; base < Wh; base += 32) {
          const int hw = base + lane;
          uint32_t xT = 0u, zT = 0u;
          if (hw < Wh) {
            const uint32_t t = sS[hw];
            xT = __ldcg(A.X + (size_t)j * W + Wh + hw) & t;
            zT = __ldcg(A.Z + (size_t)j * W + Wh + hw) & t;
          }
          acc += __popc(xT & zT);
          const uint32_t bal = __ballot_sync(0xffffffffu, __popc(zT) & 1);
          const uint32_t cin = (__popc(bal & lt) & 1u) ^ carry;
          const uint32_t zpre = prefix_xor_excl(zT) ^ (cin ? 0xffffffffu : 0u);
          acc += 2u * (__popc(xT & zpre) & 1u);
          carry ^= __popc(bal) & 1u;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      __shared__ uint32_t s_acc;
      if (tid == 0) s_acc = 0u;
      __syncthreads();
      if (lane == 0) atomicAdd(&s_acc, acc & 3u);
      __syncthreads();
      if (tid == 0) A.dp[(size_t)(m & 1) * G + c] = s_acc & 3u;
      prev_det = 1;
      prev_a = a;
      prev_reset = reset;
      __syncthreads();
    }
  }

  // ---- epilogue: resolve the last deterministic outcome, materialize the
  // deferred column, fold the partial signs into R
  if (!grid_sync(A.bar, A.err, epoch, A.wait_ns)) return;
  if (prev_det) {
    const uint32_t* dbuf = A.dp + (size_t)((A.nm - 1) & 1) * G;
    const bool owner = (prev_a % G) == c;
    if (tid < 32 && (c == 0 || (owner && prev_reset))) {
      const int o = det_outcome_warp(dbuf, G);
      if (tid == 0) {
        if (o < 0) atomicCAS(A.err, 0, DERR_PHASE);
        s_det_out = o < 0 ? 0 : o;
        if (c == 0) A.out[A.nm - 1] = (uint8_t)s_det_out;
      }
    }
    __syncthreads();
    if (owner && prev_reset && s_det_out) {
      const uint32_t* zc = A.Z + (size_t)prev_a * W;
      for (int w = tid; w < W; w += blockDim.x) PHhi[w] ^= zc[w];
    }
  }
  if (pend_a >= 0 && (pend_a % G) == c) {
    uint32_t* xc = A.X + (size_t)pend_a * W;
    for (int w = tid; w < W; w += blockDim.x)
      xc[w] = (w == (pend_pd >> 5)) ? (1u << (pend_pd & 31)) : 0u;
  }
  if (!grid_sync(A.bar, A.err, epoch, A.wait_ns)) return;
  for (int w = c * blockDim.x + tid; w < W; w += G * blockDim.x) {
    uint32_t L = __ldcg(R4lo + w), H = __ldcg(R4hi + w);
    for (int cc = 0; cc < G; ++cc) {
      const uint32_t* p = A.ph + (size_t)cc * 2 * W;
      add4(L, H, __ldcg(p + w), __ldcg(p + W + w));
    }
    if (L != 0u) atomicCAS(A.err, 0, DERR_PHASE);
    A.R[w] = H;
  }
}

size_t measure_work_words(int n, int max_ctas) {
  const int W = 2 * half_words(n);
  // ph + r4 + dp + barrier(2) + err(1), rounded
  return (size_t)max_ctas * 2 * W + 2 * (size_t)W + 2 * (size_t)max_ctas + 64;
}

static size_t meas_smem_bytes(int n, int W, int G) {
  const int ncols = (n + G - 1) / G;
  const int Q = W / 4;
  const int GG = (Q <= kMeasThreads) ? kMeasThreads / Q : 1;
  return sizeof(uint32_t) * (2 * (size_t)W + ((ncols + 3) & ~3) + (size_t)GG * Q * 8);
}

int measure_ctas_for(int n, int sm_count, int max_ctas) {
  int g = n / 6;  // about six columns per CTA at least
  if (g > sm_count) g = sm_count;
  if (g > max_ctas) g = max_ctas;
  if (g < 1) g = 1;
  return g;
}

cudaError_t launch_measure(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh,
                           const uint32_t* mops, int nm, uint64_t k0, uint64_t seed,
                           uint64_t cid, uint32_t shot, uint8_t* out, const MeasWork& mw,
                           int ctas, cudaStream_t s) {
  if (nm <= 0) return cudaSuccess;
  MArgs A;
  A.X = X; A.Z = Z; A.R = R;
  A.n = n; A.Wh = Wh; A.W = 2 * Wh;
  A.mops = mops; A.nm = nm;
  A.k0 = k0; A.seed = seed; A.cid = cid; A.shot = shot;
  A.out = out;
  A.ph = mw.ph; A.r4 = mw.r4; A.dp = mw.dp; A.bar = mw.bar; A.err = mw.err;
  A.work = mw.work;
  A.wait_ns = run_wait_limit_ns();
  const size_t smem = meas_smem_bytes(n, A.W, ctas);
  cudaError_t e = ensure_smem_limit((const void*)k_measure, 200 * 1024);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(mw.bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)k_measure, dim3(ctas), dim3(kMeasThreads), args,
                                     smem, s);
}

}  // namespace tab
