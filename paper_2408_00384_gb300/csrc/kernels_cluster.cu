// kernels_cluster.cu -- measurement runs on a tableau resident in shared
// memory across CTAs (measure_resident.cuh), with two communication policies:
//
//  * k_measure_cluster: one thread-block cluster of up to 16 CTAs holds the
//    whole tableau (n up to about 2,500).  The measured column is written
//    straight into every CTA's shared memory with DSMEM stores, and one
//    hardware cluster barrier separates measurements -- no global-memory round
//    trip and no software grid barrier on the critical path.
//  * k_measure_resident: a cooperative grid of up to one CTA per SM holds the
//    tableau (n up to about 8,000).  The measured column goes through a
//    double-buffered global buffer (L2) and a bounded software grid barrier;
//    the column updates themselves never leave shared memory.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include <algorithm>

#include "measure_resident.cuh"
#include "tab_internal.h"

namespace tab {

// Measurements per batch: TAB_MEAS_BATCH (1, 2, 4, ..., 32) caps it for
// tuning sweeps; the default is the largest that fits.
static int batch_cap() {
  static int cap = 0;
  if (cap == 0) {
    cap = kBatchMax;
    if (const char* e = getenv("TAB_MEAS_BATCH")) {
      const int v = atoi(e);
      if (v >= 1 && v <= kBatchMax && (v & (v - 1)) == 0) cap = v;
    }
  }
  return cap;
}


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

// One thread-block cluster: DSMEM and the hardware cluster barrier.
struct CommCluster {
  static constexpr bool kPush = true;
  int C, r;
  __device__ CommCluster() : C((int)cl_nrank()), r((int)cl_rank()) {}
  __device__ int size() const { return C; }
  __device__ int rank() const { return r; }
  // every CTA of the cluster runs before anyone touches its shared memory
  __device__ bool start() {
    cl_sync();
    return true;
  }
  __device__ bool sync() {
    cl_sync();
    return true;
  }
  // owners push the measured columns (their current state) into buffer
  // `buf` of every CTA; the next cluster barrier publishes them
  __device__ void stage_columns(const ResSmem& s, int buf, const ResBatch& b, int W, int Wp,
                                int KB) {
    const int per = b.nown * W;
    for (int e = threadIdx.x; e < per * C; e += blockDim.x) {
      const int dst = e / per, rem = e - dst * per;
      const int j = rem / W, w = rem - j * W;
      const int d = b.own[j];
      const size_t off = (size_t)(b.q[d] / C) * Wp + w;
      const size_t to = ((size_t)buf * KB + d) * W + w;
      cl_st(cl_map(s.TX + to, (uint32_t)dst), s.Xs[off]);
      cl_st(cl_map(s.TZ + to, (uint32_t)dst), s.Zs[off]);
    }
  }
  // word w of slot d's measured column (plane 0: X, 1: Z), pushed by its owner
  __device__ uint32_t slot_word(const ResSmem& s, int buf, int d, int w, int plane, int W,
                                int KB) const {
    return (plane ? s.TZ : s.TX)[((size_t)buf * KB + d) * W + w];
  }
  __device__ void publish_dp(uint32_t* dpv, int buf, int i, int kb, uint32_t v) {
    if ((int)threadIdx.x < C)
      cl_st(cl_map(dpv + ((size_t)buf * kb + i) * C + r, threadIdx.x), v);
  }
  __device__ uint32_t sum_dp(const uint32_t* dpv, int buf, int i, int kb) {
    uint32_t e = 0;
    for (int t = 0; t < C; ++t) e += dpv[((size_t)buf * kb + i) * C + t];
    return e;
  }
  // fold every CTA's sign partials (and CTA 0's base) into R
  __device__ bool fold(const ResSmem& s, int W, const ResArgs& A) {
    cl_sync();
    for (int w = r + C * (int)threadIdx.x; w < W; w += C * (int)blockDim.x) {
      uint32_t L = cl_ld(cl_map(s.R4lo + w, 0)), H = cl_ld(cl_map(s.R4hi + w, 0));
      for (int t = 0; t < C; ++t)
        res_add4(L, H, cl_ld(cl_map(s.PHlo + w, (uint32_t)t)), cl_ld(cl_map(s.PHhi + w, (uint32_t)t)));
      if (L != 0u) atomicCAS(A.err, 0, DERR_PHASE);
      A.R[w] = H;
    }
    return true;
  }
  // no CTA leaves while another may still read its shared memory
  __device__ void finish() { cl_sync(); }
};

// A cooperative grid: owners stage measured columns in global memory (L2),
// global deterministic partials, bounded grid barrier.
struct CommGrid {
  static constexpr bool kPush = false;
  const ResArgs& A;
  int C, r;
  __device__ explicit CommGrid(const ResArgs& a) : A(a), C((int)gridDim.x), r((int)blockIdx.x) {}
  __device__ int size() const { return C; }
  __device__ int rank() const { return r; }
  __device__ bool start() {
    __syncthreads();
    return true;
  }
  __device__ bool sync() { return grid_sync(A.bar, A.err); }
  // owners write the measured columns (their current state) to stage[buf]
  __device__ void stage_columns(const ResSmem& s, int buf, const ResBatch& b, int W, int Wp,
                                int KB) {
    for (int e = threadIdx.x; e < b.nown * W; e += blockDim.x) {
      const int j = e / W, w = e - j * W;
      const int d = b.own[j];
      const size_t off = (size_t)(b.q[d] / C) * Wp + w;
      uint32_t* dst = A.stage + (((size_t)buf * KB + d) * 2) * W;
      dst[w] = s.Xs[off];
      dst[W + w] = s.Zs[off];
    }
  }
  // word w of slot d's measured column (plane 0: X, 1: Z), staged in L2
  __device__ uint32_t slot_word(const ResSmem&, int buf, int d, int w, int plane, int W,
                                int KB) const {
    return __ldcg(A.stage + (((size_t)buf * KB + d) * 2 + plane) * W + w);
  }
  __device__ void publish_dp(uint32_t*, int buf, int i, int kb, uint32_t v) {
    if (threadIdx.x == 0) A.dp[((size_t)buf * kb + i) * C + r] = v;
  }
  __device__ uint32_t sum_dp(const uint32_t*, int buf, int i, int kb) {
    uint32_t e = 0;
    for (int t = 0; t < C; ++t) e += __ldcg(A.dp + ((size_t)buf * kb + i) * C + t);
    return e;
  }
  __device__ bool fold(const ResSmem& s, int W, const ResArgs&) {
    uint32_t* mine = A.ph + (size_t)r * 2 * W;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
      mine[w] = s.PHlo[w];
      mine[W + w] = s.PHhi[w];
      if (r == 0) {
        A.r4[w] = s.R4lo[w];
        A.r4[W + w] = s.R4hi[w];
      }
    }
    if (!grid_sync(A.bar, A.err)) return false;
    for (int w = r * (int)blockDim.x + threadIdx.x; w < W; w += C * (int)blockDim.x) {
      uint32_t L = __ldcg(A.r4 + w), H = __ldcg(A.r4 + W + w);
      for (int t = 0; t < C; ++t)
        res_add4(L, H, __ldcg(A.ph + (size_t)t * 2 * W + w), __ldcg(A.ph + (size_t)t * 2 * W + W + w));
      if (L != 0u) atomicCAS(A.err, 0, DERR_PHASE);
      A.R[w] = H;
    }
    return true;
  }
  __device__ void finish() {}
};

template <int WL>
__global__ void __launch_bounds__(32 * res_warps(WL)) k_measure_cluster(ResArgs A) {
  extern __shared__ __align__(16) uint32_t sm[];
  CommCluster cm;
  measure_resident<WL>(A, cm, sm);
}

template <int WL>
__global__ void __launch_bounds__(32 * res_warps(WL)) k_measure_resident(ResArgs A) {
  extern __shared__ __align__(16) uint32_t sm[];
  CommGrid cm(A);
  measure_resident<WL>(A, cm, sm);
}

// Kernel instance for the register share of W = 2*Wh words.
static const void* cluster_kernel(int wl) {
  switch (wl) {
    case 2: return (const void*)k_measure_cluster<2>;
    case 4: return (const void*)k_measure_cluster<4>;
    case 8: return (const void*)k_measure_cluster<8>;
    default: return nullptr;
  }
}
static const void* resident_kernel(int wl) {
  switch (wl) {
    case 2: return (const void*)k_measure_resident<2>;
    case 4: return (const void*)k_measure_resident<4>;
    case 8: return (const void*)k_measure_resident<8>;
    case 16: return (const void*)k_measure_resident<16>;
    default: return nullptr;
  }
}

// Dynamic shared memory every measurement kernel instance can take: the
// device's opt-in maximum per block less the largest static share.
static int res_dyn_limit() {
  static int lim = -1;
  if (lim < 0) {
    int dev = 0, optin = 0;
    size_t stat = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      optin = 0;
    for (int wl = 2; wl <= 16; wl *= 2) {
      const void* fns[2] = {cluster_kernel(wl), resident_kernel(wl)};
      for (const void* fn : fns) {
        cudaFuncAttributes fa;
        if (fn != nullptr && cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.sharedSizeBytes > stat)
          stat = fa.sharedSizeBytes;
      }
    }
    cudaGetLastError();
    lim = optin > (int)stat + 1024 ? (optin - (int)stat) & ~255 : 0;
  }
  return lim;
}

// Cluster size for n qubits (0 if the tableau does not fit one cluster).
int cluster_size_for(int n, int Wh) {
  static int max_c = -1;
  if (max_c < 0) {
    max_c = 0;
    bool ok = true;
    for (int wl = 2; wl <= 8; wl *= 2)
      ok = ok &&
           cudaFuncSetAttribute(cluster_kernel(wl), cudaFuncAttributeNonPortableClusterSizeAllowed,
                                1) == cudaSuccess &&
           cudaFuncSetAttribute(cluster_kernel(wl), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                res_dyn_limit()) == cudaSuccess;
    if (ok) {
      for (int c = 16; c >= 2 && max_c == 0; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(32 * res_warps(8));
        cfg.dynamicSmemBytes = res_dyn_limit();
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, cluster_kernel(8), &cfg) == cudaSuccess &&
            nclusters > 0)
          max_c = c;
      }
    }
    cudaGetLastError();  // a failed probe must not leave an error behind
  }
  const int wl = res_words_per_lane(Wh);
  if (max_c == 0 || wl == 0 || cluster_kernel(wl) == nullptr) return 0;
  // Preferred size: TAB_CLUSTER_SIZE (2..16, a power of two) if set, else the
  // largest supported.  A smaller cluster has a cheaper barrier and more work
  // per CTA; the smallest size at least the preferred one that fits is used.
  static int pref = -1;
  if (pref < 0) {
    pref = max_c;
    if (const char* e = getenv("TAB_CLUSTER_SIZE")) {
      const int v = atoi(e);
      if (v >= 2 && v <= max_c && (v & (v - 1)) == 0) pref = v;
    }
  }
  for (int c = pref; c <= max_c; c *= 2)
    if (res_batch_for(n, Wh, c, res_dyn_limit(), kBatchMax, true) >= 4) return c;
  return 0;
}

static ResArgs res_args(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh, const uint32_t* mops,
                        int nm, uint64_t k0, uint64_t seed, uint64_t cid, uint32_t shot,
                        uint8_t* out, int* err) {
  ResArgs A = {};
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
  return A;
}

cudaError_t launch_measure_cluster(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh,
                                   const uint32_t* mops, int nm, uint64_t k0, uint64_t seed,
                                   uint64_t cid, uint32_t shot, uint8_t* out, int* err, int C,
                                   cudaStream_t s) {
  if (nm <= 0) return cudaSuccess;
  const int wl = res_words_per_lane(Wh);
  const void* fn = cluster_kernel(wl);
  if (fn == nullptr) return cudaErrorInvalidValue;
  ResArgs A = res_args(X, Z, R, n, Wh, mops, nm, k0, seed, cid, shot, out, err);
  A.kb = res_batch_for(n, Wh, C, res_dyn_limit(), std::min(batch_cap(), res_warps(wl)), true);
  if (A.kb == 0) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(32 * res_warps(wl));
  cfg.dynamicSmemBytes = res_layout(n, Wh, C, A.kb, true).words * 4;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  void* args[] = {&A};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// CTAs for the grid-resident engine (0 if the tableau does not fit): one
// per SM -- phase 2 of a batch is spread over more columns-owning warps the
// more CTAs there are, and the per-batch barrier costs about the same -- or
// TAB_GRID_CTAS if set and the share fits (tuning sweeps).
int resident_ctas_for(int n, int Wh, int sm_count) {
  static int pref = -1;
  if (pref < 0) {
    pref = 0;
    if (const char* e = getenv("TAB_GRID_CTAS")) pref = atoi(e);
  }
  const int wl = res_words_per_lane(Wh);
  if (wl == 0) return 0;
  if (ensure_smem_limit(resident_kernel(wl), res_dyn_limit()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (pref >= 2 && pref <= sm_count &&
      res_batch_for(n, Wh, pref, res_dyn_limit(), kBatchMax, false) >= 4)
    return pref;
  return res_batch_for(n, Wh, sm_count, res_dyn_limit(), kBatchMax, false) >= 4 ? sm_count : 0;
}

size_t resident_work_words(int n, int max_ctas) {
  const int W = 2 * half_words(n);
  return 4 * (size_t)kBatchMax * W          // staged columns [2][kb][2][W]
         + 2 * (size_t)kBatchMax * max_ctas // deterministic partials [2][kb][G]
         + (size_t)max_ctas * 2 * W         // sign partials for the fold
         + 2 * (size_t)W + 16;              // base signs
}

cudaError_t launch_measure_resident(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh,
                                    const uint32_t* mops, int nm, uint64_t k0, uint64_t seed,
                                    uint64_t cid, uint32_t shot, uint8_t* out, int* err,
                                    uint32_t* work, GridBar* bar, int G, cudaStream_t s) {
  if (nm <= 0) return cudaSuccess;
  const int wl = res_words_per_lane(Wh);
  const void* fn = resident_kernel(wl);
  if (fn == nullptr) return cudaErrorInvalidValue;
  ResArgs A = res_args(X, Z, R, n, Wh, mops, nm, k0, seed, cid, shot, out, err);
  const int W = 2 * Wh;
  A.kb = res_batch_for(n, Wh, G, res_dyn_limit(), std::min(batch_cap(), res_warps(wl)), false);
  if (A.kb == 0) return cudaErrorInvalidValue;
  A.stage = work;
  A.dp = A.stage + 4 * (size_t)A.kb * W;
  A.ph = A.dp + 2 * (size_t)A.kb * G;
  A.r4 = A.ph + (size_t)G * 2 * W;
  A.bar = bar;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(32 * res_warps(wl)), args,
                                     res_layout(n, Wh, G, A.kb, false).words * 4, s);
}

}  // namespace tab
