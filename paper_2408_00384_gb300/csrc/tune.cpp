// tune.cpp -- autotuner of the plain path's launch shape (tab_tune in
// include/tab.h) and its persisted cache.
//
// The shapes tried are the ones the kernels are built for: the measurement
// engine (single-CTA where the tableau fits one CTA, grid-resident where it
// fits the grid's shared memory, streaming), the grid-resident engine's
// measurements per batch (8, 16, 32), and the block gate kernel's threads
// per CTA (128, 256, 512).  The engine and batch are chosen first (the
// measurement runs dominate the time where they differ), then the gate
// kernel's CTA size with that engine.  Every shape computes the same
// tableau and outcomes; the tuner checks that each run's outcome log equals
// the first run's, and refuses (TAB_EDEVICE) if one does not.
//
// Cache: TAB_AUTOTUNE_CACHE names a text file with one entry per line,
//   {"key": "<gpu>|n<bucket>|g<bucket>|m<bucket>", "engine": E,
//    "block_threads": T, "meas_batch": B, "best_ms": M}
// keyed by the GPU name, the qubit count rounded up to a power of two, and
// log2 buckets of the program's gates per qubit and measurement count.  A
// hit applies the stored shape without timing; a tuning run rewrites the
// file (all entries, through a temporary file and a rename).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tab_internal.h"

namespace tab {

namespace {

struct Shape {
  int engine = TAB_ENGINE_AUTO, threads = 0, batch = 0;
  float ms = 0.f;
};

std::mutex g_cache_mu;

int log2_bucket(double v) {
  int b = 0;
  while (v >= 2.0) {
    v /= 2.0;
    ++b;
  }
  return b;
}

std::string cache_key(int n, int64_t n_gates, int64_t n_meas) {
  int dev = 0;
  cudaDeviceProp prop{};
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    snprintf(prop.name, sizeof prop.name, "unknown");
  }
  int nb = 1;
  while (nb < n) nb *= 2;
  char buf[400];
  snprintf(buf, sizeof buf, "%s|n%d|g%d|m%d", prop.name, nb,
           log2_bucket((double)n_gates / (double)(n > 0 ? n : 1)), log2_bucket((double)n_meas + 1));
  for (char* c = buf; *c; ++c)
    if (*c == '"' || *c == '\n') *c = '_';
  return buf;
}

// Entries of the cache file (missing file: none).  Lines it cannot read are
// skipped.
std::map<std::string, Shape> read_cache(const char* path) {
  std::map<std::string, Shape> m;
  FILE* f = fopen(path, "r");
  if (!f) return m;
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    const char* k = strstr(line, "\"key\": \"");
    if (!k) continue;
    k += 8;
    const char* e = strchr(k, '"');
    if (!e) continue;
    Shape s;
    const char* p = strstr(e, "\"engine\":");
    const char* q = strstr(e, "\"block_threads\":");
    const char* r = strstr(e, "\"meas_batch\":");
    const char* t = strstr(e, "\"best_ms\":");
    if (!p || !q || !r) continue;
    s.engine = atoi(p + 9);
    s.threads = atoi(q + 16);
    s.batch = atoi(r + 13);
    s.ms = t ? (float)atof(t + 10) : 0.f;
    m[std::string(k, (size_t)(e - k))] = s;
  }
  fclose(f);
  return m;
}

bool write_cache(const char* path, const std::map<std::string, Shape>& m) {
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) return false;
  for (const auto& kv : m)
    fprintf(f,
            "{\"key\": \"%s\", \"engine\": %d, \"block_threads\": %d, \"meas_batch\": %d, "
            "\"best_ms\": %.4f}\n",
            kv.first.c_str(), kv.second.engine, kv.second.threads, kv.second.batch,
            (double)kv.second.ms);
  const bool ok = fclose(f) == 0;
  return ok && rename(tmp.c_str(), path) == 0;
}

}  // namespace

}  // namespace tab

using namespace tab;

extern "C" int tab_tune(tab_t h, tab_prog_t p, int32_t reps, tab_tuned* out) {
  HandleView v;
  int rc = handle_view(h, &v);
  if (rc != TAB_OK) return rc;
  if (!p || !out) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  int64_t n_gates = 0, n_meas = 0, n_layers = 0;
  rc = tab_prog_info(p, &n_gates, &n_meas, &n_layers);
  if (rc != TAB_OK) return rc;
  *out = tab_tuned{};
  const char* path = getenv("TAB_AUTOTUNE_CACHE");
  const std::string key = cache_key(v.n, n_gates, n_meas);
  if (path && reps >= 0) {
    std::map<std::string, Shape> m;
    {
      std::lock_guard<std::mutex> lk(g_cache_mu);
      m = read_cache(path);
    }
    auto it = m.find(key);
    if (it != m.end() && tab_set_engine(h, it->second.engine) == TAB_OK) {
      handle_set_shape(h, it->second.threads, it->second.batch);
      out->engine = it->second.engine;
      out->block_threads = it->second.threads;
      out->meas_batch = it->second.batch;
      out->best_ms = it->second.ms;
      out->from_cache = 1;
      return tab_reset(h);
    }
  }
  const int runs = reps > 0 ? reps : 3;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("cudaEventCreate failed");
    return TAB_ECUDA;
  }
  std::vector<uint8_t> want((size_t)n_meas + 1), got((size_t)n_meas + 1);
  bool have_want = false;
  int tried = 0;
  // time `runs` runs of the program from |0^n> with the current shape (the
  // handle's RNG settings each time); check the first run's outcomes
  auto time_shape = [&](float* ms) -> int {
    float total = 0.f;
    for (int i = 0; i < runs; ++i) {
      int r = tab_reset(h);
      if (r == TAB_OK && cudaEventRecord(e0, v.stream) != cudaSuccess) r = TAB_ECUDA;
      if (r == TAB_OK) r = tab_run(h, p);
      if (r == TAB_OK && cudaEventRecord(e1, v.stream) != cudaSuccess) r = TAB_ECUDA;
      if (r == TAB_OK) r = tab_sync(h);
      if (r != TAB_OK) return r;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      total += t;
      if (i == 0) {
        int64_t cnt = 0;
        r = tab_read_outcomes(h, got.data(), (int64_t)got.size(), &cnt);
        if (r != TAB_OK) return r;
        if (!have_want) {
          want = got;
          have_want = true;
        } else if (memcmp(want.data(), got.data(), (size_t)cnt) != 0) {
          set_error("launch shapes disagree on the outcomes");
          return TAB_EDEVICE;
        }
      }
    }
    *ms = total / (float)runs;
    ++tried;
    return TAB_OK;
  };
  int saved_threads = 0, saved_batch = 0;
  handle_get_shape(h, &saved_threads, &saved_batch);
  Shape best;
  best.ms = -1.f;
  // engines (and batches) first, with the default gate kernel shape
  const int engines[3] = {TAB_ENGINE_SINGLE_CTA, TAB_ENGINE_GRID, TAB_ENGINE_STREAM};
  const int batches[3] = {8, 16, 32};
  for (int e : engines) {
    if (tab_set_engine(h, e) != TAB_OK) continue;
    int resolved = 0, ctas = 0;
    tab_engine_resolved(h, &resolved, &ctas);
    if (resolved != e) continue;  // the engine does not hold this tableau
    const int nb = e == TAB_ENGINE_GRID ? 3 : 1;
    for (int bi = 0; bi < nb; ++bi) {
      const int batch = e == TAB_ENGINE_GRID ? batches[bi] : 0;
      handle_set_shape(h, 0, batch);
      float ms = 0.f;
      rc = time_shape(&ms);
      if (rc != TAB_OK) break;
      if (best.ms < 0.f || ms < best.ms) {
        best.engine = e;
        best.batch = batch;
        best.ms = ms;
      }
    }
    if (rc != TAB_OK) break;
  }
  // then the gate kernel's threads per CTA with that engine
  if (rc == TAB_OK && best.ms >= 0.f && best.engine != TAB_ENGINE_SINGLE_CTA) {
    tab_set_engine(h, best.engine);
    for (int t : {128, 256, 512}) {
      handle_set_shape(h, t, best.batch);
      float ms = 0.f;
      rc = time_shape(&ms);
      if (rc != TAB_OK) break;
      if (ms < best.ms) {
        best.threads = t;
        best.ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TAB_OK || best.ms < 0.f) {
    handle_set_shape(h, saved_threads, saved_batch);
    if (rc == TAB_OK) {
      set_error("no launch shape ran");
      rc = TAB_ECUDA;
    }
    return rc;
  }
  tab_set_engine(h, best.engine);
  handle_set_shape(h, best.threads, best.batch);
  out->engine = best.engine;
  out->block_threads = best.threads;
  out->meas_batch = best.batch;
  out->best_ms = best.ms;
  out->tried = tried;
  if (path) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    std::map<std::string, Shape> m = read_cache(path);
    m[key] = best;
    if (!write_cache(path, m)) {
      set_error("cannot write the autotune cache %s", path);
      return TAB_EINVAL;
    }
  }
  return tab_reset(h);
}
