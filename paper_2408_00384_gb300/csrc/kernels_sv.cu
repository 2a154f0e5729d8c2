// kernels_sv.cu -- state vector of a small device-resident stabilizer
// tableau (sm_103a).
//
// The state is the common +1 eigenvector of the n stabilizer rows S_i
// (Aaronson & Gottesman, PRA 70, 052328, Sec. III), so for any basis state
// |b> with <psi|b> != 0,
//     prod_i (I + S_i) / 2 |b>  =  <psi|b> |psi>.
// The host takes b from Z measurements of a copy of the tableau (their
// outcomes always lie in the support).  Here: one launch unpacks the n
// stabilizer rows into (x mask, z mask, sign); then one launch per row
// applies (I + S_i) / 2 in place -- S = (-1)^r i^|x&z| X^x Z^z sends |y> to
// (-1)^r i^|x&z| (-1)^(z.y) |y ^ x>, so each thread updates the pair
// (y, y ^ x) (or scales y alone when x = 0); then the norm and the first
// nonzero amplitude are reduced and one launch rescales, making that
// amplitude real and positive.  Basis index bit q is qubit q.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "tab_internal.h"

namespace tab {

struct SvRow {
  uint32_t x, z, r;
};

__global__ void k_sv_rows(const uint32_t* __restrict__ X, const uint32_t* __restrict__ Z,
                          const uint32_t* __restrict__ R, int n, int Wh, SvRow* rows) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int W = 2 * Wh, w = Wh + i / 32, b = i % 32;  // stabilizer n+i: packed row 32 Wh + i
  uint32_t xm = 0u, zm = 0u;
  for (int j = 0; j < n; ++j) {
    xm |= ((X[(size_t)j * W + w] >> b) & 1u) << j;
    zm |= ((Z[(size_t)j * W + w] >> b) & 1u) << j;
  }
  rows[i] = SvRow{xm, zm, (R[w] >> b) & 1u};
}

__device__ __forceinline__ float2 cmul_phase(float2 v, int q) {  // v * i^q
  switch (q & 3) {
    case 0: return v;
    case 1: return make_float2(-v.y, v.x);
    case 2: return make_float2(-v.x, -v.y);
    default: return make_float2(v.y, -v.x);
  }
}

// v <- (I + S) v / 2 for S = rows[i]; `pairs` threads (2^(n-1) when x != 0,
// else 2^n single amplitudes)
__global__ void k_sv_project(float2* __restrict__ v, const SvRow* __restrict__ rows, int i,
                             int n) {
  const SvRow s = rows[i];
  const int q0 = 2 * (int)s.r + __popc(s.x & s.z);  // S = i^q0 X^x Z^z
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s.x == 0u) {
    if (tid >= (1ull << n)) return;
    const uint32_t y = (uint32_t)tid;
    const int q = q0 + 2 * (__popc(s.z & y) & 1);  // eigenvalue i^q, q even
    v[y] = (q & 2) ? make_float2(0.f, 0.f) : v[y];
    return;
  }
  if (tid >= (1ull << (n - 1))) return;
  // y runs over the indices with bit hb clear; its partner is y ^ x
  const int hb = 31 - __clz(s.x);
  const uint32_t lo = (uint32_t)tid & ((1u << hb) - 1u);
  const uint32_t y = (((uint32_t)tid >> hb) << (hb + 1)) | lo;
  const uint32_t yp = y ^ s.x;
  const float2 a = v[y], b = v[yp];
  // (S v)[y] = i^q0 (-1)^(z.yp) v[yp], (S v)[yp] = i^q0 (-1)^(z.y) v[y]
  const float2 sa = cmul_phase(b, q0 + 2 * (__popc(s.z & yp) & 1));
  const float2 sb = cmul_phase(a, q0 + 2 * (__popc(s.z & y) & 1));
  v[y] = make_float2(0.5f * (a.x + sa.x), 0.5f * (a.y + sa.y));
  v[yp] = make_float2(0.5f * (b.x + sb.x), 0.5f * (b.y + sb.y));
}

// sum |v|^2 (double) and the smallest index with |v|^2 above `thresh`
__global__ void k_sv_reduce(const float2* __restrict__ v, uint64_t len, double* norm2,
                            unsigned long long* first, float thresh) {
  __shared__ double part[32];
  double acc = 0.0;
  unsigned long long mine = ~0ull;
  for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < len;
       y += (uint64_t)gridDim.x * blockDim.x) {
    const float2 a = v[y];
    const float m = a.x * a.x + a.y * a.y;
    acc += (double)m;
    if (m > thresh && y < mine) mine = y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mine, o);
    mine = t < mine ? t : mine;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    part[wid] = acc;
    if (mine != ~0ull) atomicMin(first, mine);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
    atomicAdd(norm2, s);
  }
}

// the factor conj(a0) / (|a0| |v|), a0 the first nonzero amplitude (1 when
// there is none, which a valid tableau never gives)
__global__ void k_sv_factor(const float2* __restrict__ v, uint64_t len, const double* norm2,
                            const unsigned long long* first, float2* factor) {
  float2 f = make_float2(1.f, 0.f);
  if (*first < len && *norm2 > 0.0) {
    const float2 a0 = v[*first];
    const double m = sqrt((double)a0.x * a0.x + (double)a0.y * a0.y);
    const double sc = 1.0 / (sqrt(*norm2) * m);
    f = make_float2((float)(a0.x * sc), (float)(-a0.y * sc));
  }
  *factor = f;
}

__global__ void k_sv_scale(float2* __restrict__ v, uint64_t len, const float2* factor) {
  const float cr = factor->x, ci = factor->y;
  for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < len;
       y += (uint64_t)gridDim.x * blockDim.x) {
    const float2 a = v[y];
    v[y] = make_float2(a.x * cr - a.y * ci, a.x * ci + a.y * cr);
  }
}

// Fill v (2^n complex, device) with the state of the tableau, given a basis
// state b in its support.  `work`: device scratch of sv_work_bytes(n).
size_t sv_work_bytes(int n) { return 64 + (size_t)n * sizeof(SvRow); }

cudaError_t launch_statevector(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n,
                               int Wh, uint32_t b, float2* v, void* work, cudaStream_t s) {
  const uint64_t len = 1ull << n;
  double* norm2 = reinterpret_cast<double*>(work);
  unsigned long long* first = reinterpret_cast<unsigned long long*>(norm2 + 1);
  float2* factor = reinterpret_cast<float2*>(first + 1);
  SvRow* rows = reinterpret_cast<SvRow*>(static_cast<char*>(work) + 64);
  cudaError_t e = cudaMemsetAsync(v, 0, len * sizeof(float2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(norm2, 0, sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(first, 0xFF, sizeof(unsigned long long), s);
  const float one[2] = {1.f, 0.f};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(v + b, one, sizeof(float2), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_sv_rows<<<(n + 63) / 64, 64, 0, s>>>(X, Z, R, n, Wh, rows);
  for (int i = 0; i < n; ++i) {
    const uint64_t threads = len;  // enough for either form
    k_sv_project<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(v, rows, i, n);
  }
  const unsigned blocks = (unsigned)std::min<uint64_t>((len + 255) / 256, 152 * 8);
  // every step halves a sum of two amplitudes whose components are short
  // dyadic rationals, exact in float: zero amplitudes are exactly zero and
  // "nonzero" needs no tolerance
  k_sv_reduce<<<blocks, 256, 0, s>>>(v, len, norm2, first, 0.f);
  k_sv_factor<<<1, 1, 0, s>>>(v, len, norm2, first, factor);
  k_sv_scale<<<blocks, 256, 0, s>>>(v, len, factor);
  return cudaGetLastError();
}

}  // namespace tab
