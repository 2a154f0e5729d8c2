// kernels_cluster.cu -- Z measurement runs on a tableau held entirely in the
// shared memory of one thread-block cluster (sm_103a, DSMEM).
//
// Operation: Aaronson & Gottesman, PRA 70, 052328, Sec. III, measurement
// step (the formalism of the Clifford backend in arXiv:2408.00384,
// "Simulation of Clifford circuits"); same arithmetic as k_measure:
//   random case: rows h with x_ha = 1 (h != p, p-n) become row_p * row_h with
//     2 r_h' = 2 r_h + 2 r_p + sum_j [x_pj z_pj + x_hj z_hj - x'_hj z'_hj
//                                     + 2 z_pj x_hj]   (mod 4),
//     then row p-n := row p, row p := (-1)^b Z_a;
//   deterministic case: e = sum_{m in T} (2 r_m + |x_m & z_m|)
//                           + 2 sum_{m<l in T} z_m . x_l  (mod 4), outcome e/2.
//
// For n up to about 2,500 the whole tableau (n columns x W words x 2 planes)
// fits in the shared memory of a 16-CTA cluster.  CTA r owns the columns
// j = r, r+C, r+2C, ...; every per-CTA quantity (its columns, its mod-4 sign
// partials) stays in its own shared memory for the whole run.  Per
// measurement the owner of the measured column writes that column (the mask of
// rows with x_ha = 1) straight into every CTA's shared memory over DSMEM, and
// one hardware cluster barrier separates measurements -- no global-memory
// round trip and no software grid barrier on the critical path.
#include <cuda_runtime.h>
#include <stdint.h>

#include "philox.cuh"
#include "tab_internal.h"

namespace tab {

constexpr int kClThreads = 512;
constexpr int kClMaxSmem = 226 * 1024;  // dynamic; static shared memory comes on top

struct ClArgs {
  uint32_t *X, *Z, *R;  // handle layout: W = 2*Wh words per column
  int n, Wh;
  const uint32_t* mops;
  int nm;
  uint64_t k0, seed, cid;
  uint32_t shot;
  uint8_t* out;
  int* err;
};

__device__ __forceinline__ uint32_t cl_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(cl_smem(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_st(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t cl_ld(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_nrank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_add4(uint32_t& l, uint32_t& h, uint32_t bl, uint32_t bh) {
  h ^= bh ^ (l & bl);
  l ^= bl;
}
__device__ __forceinline__ uint32_t cl_prefix_xor_excl(uint32_t v) {
  uint32_t y = v << 1;
  y ^= y << 1;
  y ^= y << 2;
  y ^= y << 4;
  y ^= y << 8;
  y ^= y << 16;
  return y;
}

struct ClLayout {
  int ncl, Wp, GG;
  size_t words;
};

__host__ __device__ inline ClLayout cl_layout(int n, int Wh, int C) {
  ClLayout L;
  const int W = 2 * Wh;
  L.ncl = (n + C - 1) / C;
  L.Wp = W + 1;
  L.GG = kClThreads / W;
  if (L.GG < 1) L.GG = 1;
  L.words = (size_t)2 * L.ncl * L.Wp       // own X, Z columns
            + 4 * (size_t)W                 // own sign partials (lo, hi), base signs (lo, hi)
            + 2 * (size_t)W                 // mask, double-buffered
            + 2 * (size_t)C                 // deterministic partials, double-buffered
            + (size_t)L.ncl                 // support list
            + 2 * (size_t)L.GG * W          // group counters
            + (size_t)W;                    // new Z column of the measured qubit
  return L;
}

__global__ void __launch_bounds__(kClThreads) k_measure_cluster(ClArgs A) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int C = (int)cl_nrank(), r = (int)cl_rank(), tid = threadIdx.x, T = blockDim.x;
  const int n = A.n, Wh = A.Wh, W = 2 * Wh;
  const ClLayout Ly = cl_layout(n, Wh, C);
  const int Wp = Ly.Wp, GG = Ly.GG;
  const int nown = (n - r + C - 1) / C;  // columns owned: r, r+C, ...
  uint32_t* Xs = sm;
  uint32_t* Zs = Xs + (size_t)Ly.ncl * Wp;
  uint32_t* PHlo = Zs + (size_t)Ly.ncl * Wp;
  uint32_t* PHhi = PHlo + W;
  uint32_t* R4lo = PHhi + W;
  uint32_t* R4hi = R4lo + W;
  uint32_t* mask = R4hi + W;     // [2][W]
  uint32_t* dpv = mask + 2 * W;  // [2][C]
  uint32_t* supp = dpv + 2 * C;  // [ncl]
  uint32_t* redlo = supp + Ly.ncl;
  uint32_t* redhi = redlo + (size_t)GG * W;
  uint32_t* zA = redhi + (size_t)GG * W;
  __shared__ int s_pw, s_nsupp, s_kc, s_det;
  __shared__ uint32_t s_php, s_r4p, s_acc;

  // ---- load own columns, zero partials
  for (int i = tid; i < nown * W; i += T) {
    const int lj = i / W, w = i - lj * W;
    const size_t g = (size_t)(r + lj * C) * W + w;
    Xs[(size_t)lj * Wp + w] = A.X[g];
    Zs[(size_t)lj * Wp + w] = A.Z[g];
  }
  for (int w = tid; w < W; w += T) {
    PHlo[w] = 0u;
    PHhi[w] = 0u;
    R4lo[w] = 0u;
    R4hi[w] = (r == 0) ? A.R[w] : 0u;
  }
  __syncthreads();

  int prev_det = 0, prev_a = 0, prev_reset = 0;
  for (int m = 0; m < A.nm; ++m) {
    const int buf = m & 1;
    const uint32_t code = __ldg(A.mops + m);
    const int a = (int)dq1(code);
    const bool reset = dop(code) == OP_MZR;
    const uint32_t rbit = outcome_bit(A.seed, A.cid, A.shot, A.k0 + (uint64_t)m);
    // 1. the owner of column a writes it into every CTA's mask buffer
    if (a % C == r) {
      const uint32_t* xa = Xs + (size_t)(a / C) * Wp;
      for (int i = tid; i < C * W; i += T) {
        const int t = i / W, w = i - t * W;
        cl_st(cl_map(mask + buf * W + w, (uint32_t)t), xa[w]);
      }
    }
    // 2. every write of the previous measurement and this mask are visible
    cl_sync();
    // 3. resolve the previous deterministic outcome
    if (prev_det) {
      if (tid == 0) {
        uint32_t e = 0;
        for (int t = 0; t < C; ++t) e += dpv[(buf ^ 1) * C + t];
        e &= 3u;
        if (e & 1u) atomicCAS(A.err, 0, DERR_PHASE);
        s_det = (int)(e >> 1);
        if (r == 0) A.out[m - 1] = (uint8_t)s_det;
      }
      __syncthreads();
      if (prev_reset && s_det && prev_a % C == r) {  // X on prev_a: every sign ^= z
        const uint32_t* zc = Zs + (size_t)(prev_a / C) * Wp;
        for (int w = tid; w < W; w += T) PHhi[w] ^= zc[w];
      }
      prev_det = 0;
    }
    // 4. pivot: first stabilizer row in the mask
    const uint32_t* S = mask + buf * W;
    if (tid < 32) {
      int pw = -1;
      for (int base = 0; base < Wh && pw < 0; base += 32) {
        const int hw = base + tid;
        const uint32_t bal = __ballot_sync(0xffffffffu, hw < Wh && S[Wh + hw] != 0u);
        if (bal) pw = Wh + base + __ffs(bal) - 1;
      }
      if (tid == 0) {
        s_pw = pw;
        s_nsupp = 0;
        s_kc = 0;
        s_acc = 0u;
      }
    }
    __syncthreads();
    const int pw = s_pw;
    if (pw >= 0) {
      // ============ random outcome ============
      const int P = pw * 32 + __ffs(S[pw]) - 1;
      const int Pd = P - 32 * Wh;
      const int wp = pw, wd = Pd >> 5;
      const uint32_t bpm = 1u << (P & 31);
      if (tid == 0) {
        s_php = ((PHlo[wp] & bpm) ? 1u : 0u) | ((PHhi[wp] & bpm) ? 2u : 0u);
        s_r4p = ((R4lo[wp] & bpm) ? 1u : 0u) | ((R4hi[wp] & bpm) ? 2u : 0u);
      }
      for (int lj = tid; lj < nown; lj += T) {
        uint32_t* xc = Xs + (size_t)lj * Wp;
        uint32_t* zc = Zs + (size_t)lj * Wp;
        const uint32_t xp = (xc[wp] & bpm) ? 1u : 0u, zp = (zc[wp] & bpm) ? 1u : 0u;
        if (xp | zp) {
          const int pos = atomicAdd(&s_nsupp, 1);
          supp[pos] = (uint32_t)lj | (xp << 30) | (zp << 31);
          if (xp & zp) atomicAdd(&s_kc, 1);
        } else {  // row p is I here: row p-n := row p clears this bit
          xc[wd] &= ~bpm;
          zc[wd] &= ~bpm;
        }
      }
      __syncthreads();
      const int nsupp = s_nsupp;
      const int g = tid / W, w = tid - g * W;
      const int la = (a % C == r) ? a / C : -1;
      if (g < GG) {
        uint32_t lo = 0u, hi = 0u;
        uint32_t Sw = S[w];
        if (w == wp || w == wd) Sw &= ~bpm;
        for (int idx = g; idx < nsupp; idx += GG) {
          const uint32_t e = supp[idx];
          const int lj = (int)(e & 0x3FFFu);
          const uint32_t XP = (e & (1u << 30)) ? 0xffffffffu : 0u;
          const uint32_t ZP = (e & (1u << 31)) ? 0xffffffffu : 0u;
          const size_t i = (size_t)lj * Wp + w;
          const uint32_t x = Xs[i], z = Zs[i];
          const uint32_t A0 = x & z, B0 = (x ^ XP) & (z ^ ZP);
          const uint32_t inc = A0 & ~B0, dec = B0 & ~A0;
          hi ^= ((lo & inc) | (~lo & dec)) ^ (ZP & x);
          lo ^= inc | dec;
          uint32_t xn = x ^ (XP & Sw), zn = z ^ (ZP & Sw);
          if (w == wd) {
            xn = (xn & ~bpm) | (XP & bpm);
            zn = (zn & ~bpm) | (ZP & bpm);
          }
          if (w == wp) {
            xn &= ~bpm;
            zn = (zn & ~bpm) | ((lj == la) ? bpm : 0u);
          }
          Xs[i] = xn;
          Zs[i] = zn;
          if (lj == la) zA[w] = zn;
        }
        redlo[g * W + w] = lo;
        redhi[g * W + w] = hi;
      }
      __syncthreads();
      if (tid < W) {
        const int ww = tid;
        uint32_t L = 0u, H = 0u;
        for (int gg = 0; gg < GG; ++gg) cl_add4(L, H, redlo[gg * W + ww], redhi[gg * W + ww]);
        uint32_t scal = (uint32_t)s_kc + (s_php & 1u) + 2u * (s_php >> 1);
        if (r == 0) scal += (s_r4p & 1u) + 2u * (s_r4p >> 1);
        scal &= 3u;
        cl_add4(L, H, (scal & 1u) ? 0xffffffffu : 0u, (scal & 2u) ? 0xffffffffu : 0u);
        uint32_t Sw = S[ww];
        if (ww == wp || ww == wd) Sw &= ~bpm;
        L &= Sw;
        H &= Sw;
        uint32_t pl = PHlo[ww], ph = PHhi[ww];
        cl_add4(pl, ph, L, H);
        if (ww == wd) {
          pl = (pl & ~bpm) | ((s_php & 1u) ? bpm : 0u);
          ph = (ph & ~bpm) | ((s_php & 2u) ? bpm : 0u);
        }
        if (ww == wp) {
          pl &= ~bpm;
          ph &= ~bpm;
        }
        if (la >= 0 && reset && rbit) ph ^= zA[ww];
        PHlo[ww] = pl;
        PHhi[ww] = ph;
        if (r == 0 && (ww == wp || ww == wd)) {
          uint32_t bl = R4lo[ww], bh = R4hi[ww];
          if (ww == wd) {
            bl = (bl & ~bpm) | ((s_r4p & 1u) ? bpm : 0u);
            bh = (bh & ~bpm) | ((s_r4p & 2u) ? bpm : 0u);
          } else {
            bl &= ~bpm;
            bh = (bh & ~bpm) | (rbit ? bpm : 0u);
          }
          R4lo[ww] = bl;
          R4hi[ww] = bh;
        }
      }
      if (r == 0 && tid == 0) A.out[m] = (uint8_t)rbit;
    } else {
      // ============ deterministic outcome ============
      uint32_t acc = 0u;
      for (int hw = tid; hw < Wh; hw += T) {
        const uint32_t t = S[hw];
        acc += __popc(PHlo[Wh + hw] & t) + 2u * __popc(PHhi[Wh + hw] & t);
        if (r == 0) acc += __popc(R4lo[Wh + hw] & t) + 2u * __popc(R4hi[Wh + hw] & t);
      }
      const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
      const uint32_t lt = (1u << lane) - 1u;
      for (int lj = warp; lj < nown; lj += nw) {
        uint32_t carry = 0u;
        for (int base = 0; base < Wh; base += 32) {
          const int hw = base + lane;
          uint32_t xT = 0u, zT = 0u;
          if (hw < Wh) {
            const uint32_t t = S[hw];
            xT = Xs[(size_t)lj * Wp + Wh + hw] & t;
            zT = Zs[(size_t)lj * Wp + Wh + hw] & t;
          }
          acc += __popc(xT & zT);
          const uint32_t bal = __ballot_sync(0xffffffffu, __popc(zT) & 1);
          const uint32_t cin = (__popc(bal & lt) & 1u) ^ carry;
          const uint32_t zpre = cl_prefix_xor_excl(zT) ^ (cin ? 0xffffffffu : 0u);
          acc += 2u * (__popc(xT & zpre) & 1u);
          carry ^= __popc(bal) & 1u;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) atomicAdd(&s_acc, acc & 3u);
      __syncthreads();
      if (tid < C) cl_st(cl_map(dpv + buf * C + r, (uint32_t)tid), s_acc & 3u);
      prev_det = 1;
      prev_a = a;
      prev_reset = reset;
    }
    __syncthreads();
  }

  // ---- epilogue: last deterministic outcome, fold the signs, write back
  cl_sync();
  if (prev_det) {
    if (tid == 0) {
      uint32_t e = 0;
      for (int t = 0; t < C; ++t) e += dpv[((A.nm - 1) & 1) * C + t];
      e &= 3u;
      if (e & 1u) atomicCAS(A.err, 0, DERR_PHASE);
      s_det = (int)(e >> 1);
      if (r == 0) A.out[A.nm - 1] = (uint8_t)s_det;
    }
    __syncthreads();
    if (prev_reset && s_det && prev_a % C == r) {
      const uint32_t* zc = Zs + (size_t)(prev_a / C) * Wp;
      for (int w = tid; w < W; w += T) PHhi[w] ^= zc[w];
    }
  }
  cl_sync();
  for (int w = r + C * tid; w < W; w += C * T) {
    uint32_t L = cl_ld(cl_map(R4lo + w, 0)), H = cl_ld(cl_map(R4hi + w, 0));
    for (int t = 0; t < C; ++t) cl_add4(L, H, cl_ld(cl_map(PHlo + w, (uint32_t)t)),
                                        cl_ld(cl_map(PHhi + w, (uint32_t)t)));
    if (L != 0u) atomicCAS(A.err, 0, DERR_PHASE);
    A.R[w] = H;
  }
  for (int i = tid; i < nown * W; i += T) {
    const int lj = i / W, w = i - lj * W;
    const size_t g = (size_t)(r + lj * C) * W + w;
    A.X[g] = Xs[(size_t)lj * Wp + w];
    A.Z[g] = Zs[(size_t)lj * Wp + w];
  }
  cl_sync();  // no CTA leaves while another may still read its shared memory
}

// Cluster size for n qubits (0 if the tableau does not fit one cluster).
int cluster_size_for(int n, int Wh) {
  static int max_c = -1;
  if (max_c < 0) {
    max_c = 0;
    if (cudaFuncSetAttribute(k_measure_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_measure_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kClMaxSmem) == cudaSuccess) {
      for (int c = 16; c >= 2 && max_c == 0; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(kClThreads);
        cfg.dynamicSmemBytes = kClMaxSmem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_measure_cluster, &cfg) == cudaSuccess &&
            nclusters > 0)
          max_c = c;
      }
    }
    cudaGetLastError();  // a failed probe must not leave an error behind
  }
  if (max_c == 0 || 2 * Wh > kClThreads) return 0;
  // the largest cluster spreads the tableau thinnest; if it does not fit, no
  // smaller one does
  return cl_layout(n, Wh, max_c).words * 4 <= (size_t)kClMaxSmem ? max_c : 0;
}

cudaError_t launch_measure_cluster(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh,
                                   const uint32_t* mops, int nm, uint64_t k0, uint64_t seed,
                                   uint64_t cid, uint32_t shot, uint8_t* out, int* err, int C,
                                   cudaStream_t s) {
  if (nm <= 0) return cudaSuccess;
  ClArgs A;
  A.X = X;
  A.Z = Z;
  A.R = R;
  A.n = n;
  A.Wh = Wh;
  A.mops = mops;
  A.nm = nm;
  A.k0 = k0;
  A.seed = seed;
  A.cid = cid;
  A.shot = shot;
  A.out = out;
  A.err = err;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kClThreads);
  cfg.dynamicSmemBytes = cl_layout(n, Wh, C).words * 4;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_measure_cluster, A);
}

}  // namespace tab
