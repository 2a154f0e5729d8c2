// config.cpp -- the process-wide run-time configuration (tab_get_config /
// tab_set_config in include/tab.h).
//
// The launch-shape knobs start from the environment (TAB_BLOCK_THREADS,
// TAB_MEAS_BATCH, TAB_GRID_CTAS, TAB_BATCH_CHUNKS; read once, on first use) and can then be
// changed through the C ABI.  Launchers read a copy of the whole struct per
// launch, under a mutex, so a change takes effect for launches issued after
// tab_set_config returns.
#include <stdlib.h>

#include <mutex>

#include "tab_internal.h"

namespace tab {

namespace {

std::mutex g_cfg_mu;
bool g_cfg_init = false;
tab_config g_cfg;

int env_int(const char* name) {
  const char* e = getenv(name);
  return e ? atoi(e) : 0;
}

bool valid_batch(int v) { return v == 0 || (v >= 1 && v <= 32 && (v & (v - 1)) == 0); }
bool valid_threads(int v) { return v == 0 || v == 128 || v == 256 || v == 512; }

void init_locked() {
  if (g_cfg_init) return;
  g_cfg = tab_config{};
  const int bt = env_int("TAB_BLOCK_THREADS");
  if (valid_threads(bt)) g_cfg.block_threads = bt;
  const int mb = env_int("TAB_MEAS_BATCH");
  if (valid_batch(mb)) g_cfg.meas_batch = mb;
  const int gc = env_int("TAB_GRID_CTAS");
  if (gc >= 0) g_cfg.grid_ctas = gc;
  const int bc = env_int("TAB_BATCH_CHUNKS");
  if (bc >= 0 && bc <= kMaxBatchChunks) g_cfg.batch_chunks = bc;
  g_cfg_init = true;
}

}  // namespace

tab_config run_config() {
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  init_locked();
  return g_cfg;
}

unsigned long long run_wait_limit_ns() {
  const tab_config c = run_config();
  return c.wait_limit_ns ? (unsigned long long)c.wait_limit_ns : kDefaultWaitLimitNs;
}

}  // namespace tab

using namespace tab;

extern "C" int tab_get_config(tab_config* out) {
  if (!out) {
    set_error("null output");
    return TAB_EINVAL;
  }
  *out = run_config();
  return TAB_OK;
}

extern "C" int tab_set_config(const tab_config* cfg) {
  if (!cfg) {
    set_error("null configuration");
    return TAB_EINVAL;
  }
  if (!valid_threads(cfg->block_threads)) {
    set_error("block_threads %d is not 0, 128, 256 or 512", cfg->block_threads);
    return TAB_EINVAL;
  }
  if (!valid_batch(cfg->meas_batch)) {
    set_error("meas_batch %d is not 0 or a power of two in [1, 32]", cfg->meas_batch);
    return TAB_EINVAL;
  }
  if (cfg->grid_ctas < 0) {
    set_error("grid_ctas %d < 0", cfg->grid_ctas);
    return TAB_EINVAL;
  }
  if (cfg->batch_chunks < 0 || cfg->batch_chunks > kMaxBatchChunks) {
    set_error("batch_chunks %d outside [0, %d]", cfg->batch_chunks, kMaxBatchChunks);
    return TAB_EINVAL;
  }
  if (cfg->reserved != 0) {
    set_error("reserved field is %d, not 0", cfg->reserved);
    return TAB_EINVAL;
  }
  if (cfg->debug & ~(uint32_t)TAB_DEBUG_SKIP_BARRIER_ARRIVAL) {
    set_error("unknown debug flags 0x%x", cfg->debug);
    return TAB_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_cfg_mu);
  init_locked();
  g_cfg = *cfg;
  return TAB_OK;
}
