// sct.h -- argument blocks of the single-CTA engine (kernels_sct.cu): the
// plain-path program kernel for one small tableau and the batched launch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tab_internal.h"

namespace tab {

struct SctProgArgs {
  uint32_t *X, *Z, *R;  // handle layout (Wh words per half)
  int n, Wh;
  const Seg* segs;
  int nsegs;
  const uint32_t* ops;
  const uint32_t* layer_off;
  uint64_t seed, cid;
  uint32_t shot;
  uint64_t k0;   // first measurement index
  uint8_t* out;  // outcome k0 + i goes to out[i]
  int* err;
};

struct BatchCirc {
  int32_t n;
  int32_t shots;
  uint32_t seg_begin, seg_end;  // into the batch's segment table
  uint32_t n_prefix;            // 1 if the first segment is shared gates
  uint32_t n_meas;              // measurement ops per shot
  uint64_t cid;
  uint64_t out_off;             // byte offset of shot 0's outcomes
  uint64_t img_off;             // word offset of the shared-prefix image (or the
                                // outcome forms of a sampled circuit)
  uint32_t sampled;             // 1: terminal measurements by the sampler
  uint32_t n_noise;             // noise ops (drawn per shot), entries noise_off ..
  uint64_t noise_off;           //   of the batch's noise table
};

struct BatchArgs {
  const BatchCirc* circs;
  const Seg* segs;
  const uint32_t* ops;
  const uint32_t* layer_off;
  const uint64_t* items;  // circuit | shot << 32 (shot = ~0: prefix item)
  const uint32_t* noise;  // noise table: kind << 28 | probability (kProgNoise)
  int nitems;
  int ncirc;              // circuits (entries of circs)
  uint32_t* img;
  int* ready;
  unsigned int* queue;
  int* err;
  uint64_t seed;  // Philox key of this run
  uint8_t* out;   // outcome buffer of this run
  // work counters (tab_batch_count_work; null: off): [0] the pivot rows'
  // support columns times the tableau's words per column, over random
  // outcomes, [1] the rows multiplied times the words per column, over
  // deterministic ones, [2] / [3] random / deterministic measurements
  unsigned long long* work = nullptr;
};

size_t sct_image_words(int n);
// Shared memory of one tableau of n qubits run by a CTA of `threads`.
size_t sct_smem_bytes(int n, int threads);
// Extra shared memory of the terminal-measurement sampler (K measurements).
size_t sct_sampler_bytes(int n, int K, int shots);
cudaError_t launch_sct_program(const SctProgArgs& A, cudaStream_t st);
// Batched kernel instances: threads per CTA in {128, 256, 512, 1024}.
constexpr int kBatchThreadChoices[4] = {128, 256, 512, 1024};
constexpr int kBatchDefaultThreads = 512;
int batch_ctas_per_sm(int threads, size_t smem);
cudaError_t prepare_batch_kernel(int threads);
// The batched kernel for `threads`; `count`: the instance that updates the
// work counters (BatchArgs::work).
const void* batch_kernel_ptr(int threads, bool count = false);

}  // namespace tab
