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

constexpr int kClMaxSmem = 226 * 1024;  // dynamic; static shared memory comes on top

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
  int C, r;
  __device__ CommCluster() : C((int)cl_nrank()), r((int)cl_rank()) {}
  __device__ int size() const { return C; }
  __device__ int rank() const { return r; }
  __device__ bool sync() {
    cl_sync();
    return true;
  }
  __device__ void stage_columns(const ResSmem&, int, int, int, const int*, int, int,
                                const ResArgs&) {}
  // read the measured columns from their owners' shared memory
  __device__ void gather_columns(const ResSmem& s, int, int D, const int* q, int W, int Wp,
                                 const ResArgs&) {
    for (int e = threadIdx.x; e < D * W; e += blockDim.x) {
      const int d = e / W, w = e - d * W;
      const int a = q[d];
      const size_t off = (size_t)(a / C) * Wp + w;
      s.TX[e] = cl_ld(cl_map(s.Xs + off, (uint32_t)(a % C)));
      s.TZ[e] = cl_ld(cl_map(s.Zs + off, (uint32_t)(a % C)));
    }
  }
  // nobody may change a column before every CTA has read it
  __device__ bool after_gather() {
    cl_sync();
    return true;
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
  const ResArgs& A;
  int C, r;
  __device__ explicit CommGrid(const ResArgs& a) : A(a), C((int)gridDim.x), r((int)blockIdx.x) {}
  __device__ int size() const { return C; }
  __device__ int rank() const { return r; }
  __device__ bool sync() { return grid_sync(A.bar, A.err); }
  // owners write the next batch's measured columns (their current state)
  __device__ void stage_columns(const ResSmem& s, int buf, int, int D, const int* q, int W, int Wp,
                                const ResArgs&) {
    const int KB = A.kb;
    for (int e = threadIdx.x; e < D * W; e += blockDim.x) {
      const int d = e / W, w = e - d * W;
      const int a = q[d];
      if (a % C != r) continue;
      const size_t off = (size_t)(a / C) * Wp + w;
      uint32_t* dst = A.stage + (((size_t)buf * KB + d) * 2) * W;
      dst[w] = s.Xs[off];
      dst[W + w] = s.Zs[off];
    }
  }
  __device__ void gather_columns(const ResSmem& s, int buf, int D, const int*, int W, int,
                                 const ResArgs&) {
    const int KB = A.kb;
    for (int e = threadIdx.x; e < D * W; e += blockDim.x) {
      const int d = e / W, w = e - d * W;
      const uint32_t* src = A.stage + (((size_t)buf * KB + d) * 2) * W;
      s.TX[e] = __ldcg(src + w);
      s.TZ[e] = __ldcg(src + W + w);
    }
    __syncthreads();
  }
  __device__ bool after_gather() { return true; }
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

__global__ void __launch_bounds__(kResThreads) k_measure_cluster(ResArgs A) {
  extern __shared__ __align__(16) uint32_t sm[];
  CommCluster cm;
  measure_resident(A, cm, sm);
}

__global__ void __launch_bounds__(kResThreads) k_measure_resident(ResArgs A) {
  extern __shared__ __align__(16) uint32_t sm[];
  CommGrid cm(A);
  measure_resident(A, cm, sm);
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
        cfg.blockDim = dim3(kResThreads);
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
  if (max_c == 0 || 2 * Wh > kResThreads) return 0;
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
    if (res_batch_for(n, Wh, c, kClMaxSmem) >= 4) return c;
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
  ResArgs A = res_args(X, Z, R, n, Wh, mops, nm, k0, seed, cid, shot, out, err);
  A.kb = res_batch_for(n, Wh, C, kClMaxSmem, batch_cap());
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)C);
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = res_layout(n, Wh, C, A.kb).words * 4;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_measure_cluster, A);
}

// CTAs for the grid-resident engine (0 if the tableau does not fit): the
// smallest count whose share fits, so that the barrier stays cheap, but at
// least enough CTAs to keep per-CTA work short.
int resident_ctas_for(int n, int Wh, int sm_count) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_measure_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kClMaxSmem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    attr = true;
  }
  if (2 * Wh > kResThreads) return 0;
  for (int g = 16; g <= sm_count; g += 8)
    if (res_batch_for(n, Wh, g, kClMaxSmem) >= 4 && (n + g - 1) / g < (1 << 14)) return g;
  return 0;
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
  ResArgs A = res_args(X, Z, R, n, Wh, mops, nm, k0, seed, cid, shot, out, err);
  const int W = 2 * Wh;
  A.kb = res_batch_for(n, Wh, G, kClMaxSmem, batch_cap());
  A.stage = work;
  A.dp = A.stage + 4 * (size_t)A.kb * W;
  A.ph = A.dp + 2 * (size_t)A.kb * G;
  A.r4 = A.ph + (size_t)G * 2 * W;
  A.bar = bar;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel((const void*)k_measure_resident, dim3((unsigned)G),
                                     dim3(kResThreads), args, res_layout(n, Wh, G, A.kb).words * 4, s);
}

}  // namespace tab
