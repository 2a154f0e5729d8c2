// kernels_resident.cu -- measurement runs on a tableau resident in shared
// memory across the CTAs of a cooperative grid (measure_resident.cuh): up to
// one CTA per SM holds the tableau (n up to about 8,000).  The measured
// columns of each batch go through a double-buffered global buffer (L2) and a
// bounded software grid barrier; the column updates themselves never leave
// shared memory.
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
  const int v = run_config().meas_batch;
  return v >= 1 && v <= kBatchMax ? v : kBatchMax;
}


// A cooperative grid: owners stage measured columns in global memory (L2),
// global deterministic partials, bounded grid barrier.
struct CommGrid {
  static constexpr bool kPush = false;
  const ResArgs& A;
  int C, r;
  unsigned int epoch = 0;  // grid barriers passed (grid_sync)
  __device__ explicit CommGrid(const ResArgs& a) : A(a), C((int)gridDim.x), r((int)blockIdx.x) {}
  __device__ int size() const { return C; }
  __device__ int rank() const { return r; }
  __device__ bool start() {
    __syncthreads();
    return true;
  }
  // test-only fault injection: the last CTA leaves without arriving, so the
  // others' bounded wait runs out
  __device__ bool sync() {
    if (A.skip_arrival && r == C - 1) return false;
    return grid_sync(A.bar, A.err, epoch, A.wait_ns);
  }
  // owners write the X bits of the measured columns (their current state)
  // to stage[buf]
  __device__ void stage_columns(const ResSmem& s, int buf, const ResBatch& b, int W, int Wp,
                                int KB) {
    for (int e = threadIdx.x; e < b.nown * W; e += blockDim.x) {
      const int j = e / W, w = e - j * W;
      const int d = b.own[j];
      A.stage[((size_t)buf * KB + d) * W + w] = s.Xs[(size_t)(b.q[d] / C) * Wp + w];
    }
  }
  // word w of the X bits of slot d's measured column, staged in L2
  __device__ uint32_t slot_word(const ResSmem&, int buf, int d, int w, int W, int KB) const {
    return __ldcg(A.stage + ((size_t)buf * KB + d) * W + w);
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
    if (!grid_sync(A.bar, A.err, epoch, A.wait_ns)) return false;
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
__global__ void __launch_bounds__(32 * kResMaxWarps, 1) k_measure_resident(const __grid_constant__ ResArgs A) {
  extern __shared__ __align__(16) uint32_t sm[];
  CommGrid cm(A);
  measure_resident<WL>(A, cm, sm);
}

// Kernel instance for the register share of W = 2*Wh words.
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
      const void* fn = resident_kernel(wl);
      cudaFuncAttributes fa;
      if (fn != nullptr && cudaFuncGetAttributes(&fa, fn) == cudaSuccess && fa.sharedSizeBytes > stat)
        stat = fa.sharedSizeBytes;
    }
    cudaGetLastError();
    lim = optin > (int)stat + 1024 ? (optin - (int)stat) & ~255 : 0;
  }
  return lim;
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

// CTAs for the grid-resident engine (0 if the tableau does not fit): one
// per SM -- phase 2 of a batch is spread over more columns-owning warps the
// more CTAs there are, and the per-batch barrier costs about the same -- or
// TAB_GRID_CTAS if set and the share fits (tuning sweeps).
int resident_ctas_for(int n, int Wh, int sm_count) {
  const int pref = run_config().grid_ctas;
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
  return 2 * (size_t)kBatchMax * W          // staged X bits of measured columns [2][kb][W]
         + 2 * (size_t)kBatchMax * max_ctas // deterministic partials [2][kb][G]
         + (size_t)max_ctas * 2 * W         // sign partials for the fold
         + 2 * (size_t)W + 16;              // base signs
}

cudaError_t launch_measure_resident(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Wh,
                                    const uint32_t* mops, int nm, uint64_t k0, uint64_t seed,
                                    uint64_t cid, uint32_t shot, uint8_t* out, int* err,
                                    uint32_t* work, GridBar* bar, int G, cudaStream_t s,
                                    int batch) {
  if (nm <= 0) return cudaSuccess;
  const int wl = res_words_per_lane(Wh);
  const void* fn = resident_kernel(wl);
  if (fn == nullptr) return cudaErrorInvalidValue;
  ResArgs A = res_args(X, Z, R, n, Wh, mops, nm, k0, seed, cid, shot, out, err);
  const int W = 2 * Wh;
  const int cap = batch >= 1 && batch <= kBatchMax ? batch : batch_cap();
  A.kb = res_batch_for(n, Wh, G, res_dyn_limit(), cap, false);
  if (A.kb == 0) return cudaErrorInvalidValue;
  // the replay chain warp and its helpers; apply warps: one column each
  // where the CTA's warp budget allows, at most 32 columns each
  A.nreplay = 1 + kResHelpers;
  const int nown = (n + G - 1) / G;
  int napply = std::min(nown, kResMaxWarps - A.nreplay);
  napply = std::max(napply, (nown + 31) / 32);
  napply = std::max(1, std::min(napply, kResMaxWarps - A.nreplay));
  if ((nown + napply - 1) / napply > 32) return cudaErrorInvalidValue;
  A.napply = napply;
  A.wait_ns = run_wait_limit_ns();
  A.skip_arrival = (run_config().debug & TAB_DEBUG_SKIP_BARRIER_ARRIVAL) ? 1 : 0;
  A.stage = work;
  A.dp = A.stage + 2 * (size_t)A.kb * W;
  A.ph = A.dp + 2 * (size_t)A.kb * G;
  A.r4 = A.ph + (size_t)G * 2 * W;
  A.bar = bar;
  cudaError_t e = cudaMemsetAsync(bar, 0, sizeof(GridBar), s);
  if (e != cudaSuccess) return e;
  void* args[] = {&A};
  return cudaLaunchCooperativeKernel(fn, dim3((unsigned)G), dim3(32 * (A.nreplay + A.napply)),
                                     args, res_layout(n, Wh, G, A.kb, false).words * 4, s);
}

}  // namespace tab
