// serve.cpp -- continuous-batching request server over device-resident
// tableaus (tab_server_* in include/tab.h).
//
// A worker thread owns the device side.  Requests wait in a FIFO; one is
// admitted when a slot is free and its tableau fits the device-memory budget.
// Admission compiles the circuit, allocates its tableau, and enqueues the
// whole program (gate runs and mid-circuit measurement runs) plus the
// device-to-host copy of its outcomes on one of the server's streams; the
// tableau stays on the device from the first gate to the last measurement.
// Requests on different streams overlap on the GPU; a finished request
// (completion event reached) returns its slot and memory, and the next
// waiting request is admitted at once.  Every request draws its outcomes from
// its own Philox stream (circuit_id, shot), so its result does not depend on
// what else is in flight.
//
// Failures are detected on the host: a request larger than the whole budget
// or with an invalid gate is rejected before anything is launched; a request
// whose completion is not seen within its deadline (fault injection drops a
// completion on purpose) fails with TAB_ETIMEOUT, and its slot is reclaimed
// after its stream has drained.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tab_internal.h"
#include "trace.h"

using namespace tab;

namespace tab {
int handle_outcomes_async(tab_t h, uint8_t* host, cudaStream_t* used_stream);
int handle_apply_program(tab_t h, const HostProgram& hp);
int grid_compile_mode(int n);
int handle_set_meas_ctas(tab_t h, int ctas);
size_t handle_device_bytes(int32_t n);
}

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Req {
  int64_t ticket = 0;
  int32_t n = 0, shots = 1;
  uint64_t cid = 0;
  HostProgram prog;           // compiled at submit, in the caller's thread
  std::vector<HostProgram> shot_progs;  // with noise ops: one program per shot
  int64_t n_meas = 0;
  size_t bytes = 0;
  tab_t h = nullptr;
  void* dmem = nullptr;       // stream-ordered allocation holding the tableau
  int stream_idx = -1;
  cudaEvent_t done = nullptr;
  uint8_t* pinned = nullptr;  // outcomes, all shots
  std::vector<uint8_t> out;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = TAB_REQ_PENDING;
  int status = TAB_OK;
  char msg[256] = {0};
  bool drop_completion = false;
};

}  // namespace

struct tab_server_s {
  tab_server_config cfg{};
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::vector<Req*> running;
  std::unordered_map<int64_t, Req*> reqs;
  std::vector<cudaStream_t> streams;       // single-SM requests
  std::vector<int> stream_load;
  std::vector<cudaStream_t> grid_streams;  // grid-wide requests, highest priority
  std::vector<int> grid_busy;              // 1 while a request owns that stream
  int grid_running = 0;  // running requests on grid-wide engines
  size_t mem_used = 0;
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  tab_server_stats st{};
};

namespace {

void finish(tab_server_s* S, Req* r, int status, const char* msg) {
  r->status = status;
  if (msg) snprintf(r->msg, sizeof r->msg, "%s", msg);
  r->t_done = now_s();
  r->state = status == TAB_OK ? TAB_REQ_DONE : TAB_REQ_FAILED;
  if (status == TAB_OK) {
    S->st.completed++;
  } else {
    S->st.failed++;
  }
}

cudaStream_t request_stream(tab_server_s* S, const Req* r) {
  return r->n > TAB_BATCH_MAX_QUBITS ? S->grid_streams[(size_t)r->stream_idx]
                                     : S->streams[(size_t)r->stream_idx];
}

void release(tab_server_s* S, Req* r) {
  if (r->h) {
    tab_destroy(r->h);  // waits for the request's stream work first
    r->h = nullptr;
  }
  if (r->dmem) {  // stream-ordered free: no device-wide synchronization
    cudaFreeAsync(r->dmem, request_stream(S, r));
    r->dmem = nullptr;
  }
  if (r->done) {
    cudaEventDestroy(r->done);
    r->done = nullptr;
  }
  if (r->n > TAB_BATCH_MAX_QUBITS) {
    S->grid_running--;
    if (r->stream_idx >= 0) S->grid_busy[(size_t)r->stream_idx] = 0;
  } else if (r->stream_idx >= 0) {
    S->stream_load[(size_t)r->stream_idx]--;
  }
  S->mem_used -= r->bytes;
  r->bytes = 0;
}

// Admit one request: allocate, upload and enqueue its compiled program.
// Called by the worker thread without the lock.
int admit(tab_server_s* S, Req* r) {
  int si = 0;
  if (r->n > TAB_BATCH_MAX_QUBITS) {
    // at most grid_streams.size() grid-wide requests run at once: take a free one
    while (si + 1 < (int)S->grid_busy.size() && S->grid_busy[(size_t)si]) ++si;
    S->grid_busy[(size_t)si] = 1;
    r->stream_idx = si;
  } else {
    for (size_t i = 1; i < S->streams.size(); ++i)
      if (S->stream_load[i] < S->stream_load[(size_t)si]) si = (int)i;
    r->stream_idx = si;
    S->stream_load[(size_t)si]++;
  }
  cudaStream_t st = request_stream(S, r);
  const size_t hb = handle_device_bytes(r->n);
  int rc = TAB_OK;
  if (cudaMallocAsync(&r->dmem, hb, st) != cudaSuccess) {
    cudaGetLastError();
    r->dmem = nullptr;
    set_error("device allocation of %zu bytes failed", hb);
    rc = TAB_ENOMEM;
  }
  if (rc == TAB_OK) rc = tab_create_on(r->n, r->dmem, hb, st, &r->h);
  // small tableaus run whole on one SM; larger ones on the grid-wide engines
  if (rc == TAB_OK && r->n <= TAB_BATCH_MAX_QUBITS) rc = tab_set_engine(r->h, TAB_ENGINE_SINGLE_CTA);
  if (rc == TAB_OK && S->cfg.meas_ctas > 0) rc = handle_set_meas_ctas(r->h, S->cfg.meas_ctas);
  for (int32_t s = 0; rc == TAB_OK && s < r->shots; ++s) {
    if (s > 0) rc = tab_reset(r->h);
    if (rc == TAB_OK) rc = tab_set_rng(r->h, S->cfg.seed, r->cid, (uint32_t)s);
    if (rc == TAB_OK)
      rc = handle_apply_program(r->h, r->shot_progs.empty() ? r->prog : r->shot_progs[(size_t)s]);
    if (rc == TAB_OK && r->n_meas > 0) {
      cudaStream_t used = nullptr;
      rc = handle_outcomes_async(r->h, r->pinned + (size_t)s * r->n_meas, &used);
    }
  }
  if (rc == TAB_OK) {
    if (cudaEventCreateWithFlags(&r->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(r->done, st) != cudaSuccess) {
      set_error("event record failed");
      rc = TAB_ECUDA;
    }
  }
  r->t_admit = now_s();
  return rc;
}

void worker_main(tab_server_s* S) {
  // stream_load and the running set are only touched by this thread
  cudaSetDevice(S->dev);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    if (S->stop && S->pending.empty() && S->running.empty()) break;
    bool progressed = false;
    // ---- completions
    for (size_t i = 0; i < S->running.size();) {
      Req* r = S->running[i];
      bool fin = false;
      if (!r->drop_completion) {
        const cudaError_t q = cudaEventQuery(r->done);
        if (q == cudaSuccess) {
          const int rc = tab_sync(r->h);  // latched device errors of this request
          r->out.assign(r->pinned, r->pinned + (size_t)r->n_meas * r->shots);
          finish(S, r, rc, rc == TAB_OK ? nullptr : tab_last_error());
          fin = true;
        } else if (q != cudaErrorNotReady) {
          finish(S, r, TAB_ECUDA, cudaGetErrorString(q));
          fin = true;
        }
      }
      if (!fin && S->cfg.request_timeout_s > 0 &&
          now_s() - r->t_admit > S->cfg.request_timeout_s) {
        finish(S, r, TAB_ETIMEOUT, "request completion not observed before its deadline");
        fin = true;
      }
      if (fin) {
        release(S, r);
        S->running[i] = S->running.back();
        S->running.pop_back();
        progressed = true;
        S->cv_done.notify_all();
      } else {
        ++i;
      }
    }
    // ---- admissions (FIFO, memory- and slot-limited)
    while (!S->pending.empty() && (int)S->running.size() < S->cfg.max_inflight) {
      Req* r = S->pending.front();
      if (r->bytes > S->cfg.mem_budget_bytes) {  // can never fit: reject
        S->pending.pop_front();
        S->st.rejected++;
        finish(S, r, TAB_ENOMEM, "request needs more device memory than the server budget");
        S->cv_done.notify_all();
        continue;
      }
      if (S->mem_used + r->bytes > S->cfg.mem_budget_bytes) break;
      const bool grid = r->n > TAB_BATCH_MAX_QUBITS;
      if (grid && S->grid_running >= std::max(1, S->cfg.max_grid_inflight)) {
        // FIFO among grid-wide requests; small ones behind it may still go
        bool admitted_small = false;
        for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
          Req* q = *it;
          if (q->n > TAB_BATCH_MAX_QUBITS || q->bytes > S->cfg.mem_budget_bytes ||
              S->mem_used + q->bytes > S->cfg.mem_budget_bytes)
            continue;
          S->pending.erase(it);
          S->pending.push_front(q);
          admitted_small = true;
          break;
        }
        if (!admitted_small) break;
        continue;
      }
      if (grid) S->grid_running++;
      S->pending.pop_front();
      S->mem_used += r->bytes;
      S->st.peak_mem = std::max<uint64_t>(S->st.peak_mem, S->mem_used);
      // upload and enqueue without the lock: only this thread touches the
      // running set, memory accounting and streams
      lk.unlock();
      const int rc = admit(S, r);
      lk.lock();
      if (rc != TAB_OK) {
        finish(S, r, rc, tab_last_error());
        release(S, r);
        S->cv_done.notify_all();
      } else {
        r->state = TAB_REQ_RUNNING;
        S->running.push_back(r);
        S->st.peak_inflight = std::max<int64_t>(S->st.peak_inflight, (int64_t)S->running.size());
      }
      progressed = true;
    }
    if (!progressed) {
      if (S->running.empty() && S->pending.empty() && !S->stop) {
        S->cv_work.wait(lk);
      } else {
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
}

}  // namespace

extern "C" {

int tab_server_create(const tab_server_config* cfg, tab_server_t* out) {
  if (!cfg || !out) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  *out = nullptr;
  if (cfg->max_inflight < 1 || cfg->n_streams < 1 || cfg->mem_budget_bytes == 0) {
    set_error("bad server configuration");
    return TAB_EINVAL;
  }
  tab_server_s* S = new (std::nothrow) tab_server_s();
  if (!S) {
    set_error("host allocation failed");
    return TAB_ENOMEM;
  }
  S->cfg = *cfg;
  if (cudaGetDevice(&S->dev) != cudaSuccess) {
    delete S;
    set_error("no CUDA device");
    return TAB_ECUDA;
  }
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);  // hi is numerically lowest
  const int ngrid = std::max(1, cfg->max_grid_inflight);
  for (int i = 0; i < cfg->n_streams + ngrid; ++i) {
    cudaStream_t st;
    const bool grid = i >= cfg->n_streams;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, grid ? prio_hi : prio_lo) !=
        cudaSuccess) {
      for (cudaStream_t x : S->streams) cudaStreamDestroy(x);
      for (cudaStream_t x : S->grid_streams) cudaStreamDestroy(x);
      delete S;
      set_error("stream creation failed");
      return TAB_ECUDA;
    }
    if (grid) {
      S->grid_streams.push_back(st);
      S->grid_busy.push_back(0);
    } else {
      S->streams.push_back(st);
      S->stream_load.push_back(0);
    }
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return TAB_OK;
}

int tab_server_submit(tab_server_t S, const tab_circuit* c, int64_t* ticket) {
  tab::TraceRange trace_("tab_server_submit");
  if (!S || !c || !ticket) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  if (c->n < 1 || c->n > TAB_MAX_QUBITS || c->shots < 1 || c->n_gates < 0 ||
      (c->n_gates > 0 && !c->gates)) {
    set_error("bad request");
    return TAB_EINVAL;
  }
  // validate now: a corrupted request is refused before it reaches the device
  int64_t ext = 0;
  int vrc = validate_program(c->n, c->gates, c->n_gates, &ext);
  if (vrc != TAB_OK) return vrc;
  int64_t nm = 0;
  bool noise = false;
  for (int64_t i = 0; i < c->n_gates; ++i) {
    const uint32_t op = (uint32_t)(c->gates[i] >> 56);
    nm += (op == TAB_MZ || op == TAB_MZR || op == TAB_MX || op == TAB_MY);
    noise = noise || op == TAB_DEPOL1 || op == TAB_XERR || op == TAB_ZERR;
  }
  Req* r = new (std::nothrow) Req();
  if (!r) {
    set_error("host allocation failed");
    return TAB_ENOMEM;
  }
  // single-SM requests need layers; grid-wide ones the form their gate kernel
  // reads.  Extended ops are lowered as tab_apply lowers them: X / Y
  // measurements once, noise ops drawn for each shot (its own program).
  const int mode = c->n <= TAB_BATCH_MAX_QUBITS ? kProgLayers : grid_compile_mode(c->n);
  int crc = TAB_OK;
  std::vector<tab_gate> low;
  if (!ext) {
    crc = build_program(c->n, c->gates, c->n_gates, &r->prog, mode);
  } else if (!noise) {
    crc = lower_for_runs(c->n, c->gates, c->n_gates, false, 0, 0, 0, low);
    if (crc == TAB_OK) crc = build_program(c->n, low.data(), (int64_t)low.size(), &r->prog, mode);
  } else {
    r->shot_progs.resize((size_t)c->shots);
    for (int32_t sh = 0; crc == TAB_OK && sh < c->shots; ++sh) {
      crc = lower_for_runs(c->n, c->gates, c->n_gates, false, S->cfg.seed, c->circuit_id,
                           (uint32_t)sh, low);
      if (crc == TAB_OK)
        crc = build_program(c->n, low.data(), (int64_t)low.size(), &r->shot_progs[(size_t)sh],
                            mode);
    }
  }
  if (crc != TAB_OK) {
    delete r;
    return crc;
  }
  r->n = c->n;
  r->shots = c->shots;
  r->cid = c->circuit_id;
  r->n_meas = nm;
  r->bytes = handle_device_bytes(c->n) + (size_t)c->n_gates * 4 + 8192 +
             (size_t)nm * c->shots;
  const size_t ob = std::max<size_t>((size_t)nm * c->shots, 1);
  if (cudaMallocHost((void**)&r->pinned, ob) != cudaSuccess) {
    delete r;
    set_error("pinned allocation failed");
    return TAB_ENOMEM;
  }
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> g(S->mu);
    r->ticket = S->next_ticket++;
    S->reqs[r->ticket] = r;
    S->pending.push_back(r);
    S->st.submitted++;
  }
  S->cv_work.notify_one();
  *ticket = r->ticket;
  return TAB_OK;
}

int tab_server_query(tab_server_t S, int64_t ticket, int* state) {
  if (!S || !state) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("unknown ticket %lld", (long long)ticket);
    return TAB_EINVAL;
  }
  *state = it->second->state;
  return TAB_OK;
}

int tab_server_wait(tab_server_t S, int64_t ticket, double timeout_s, uint8_t* out, int64_t cap,
                    int64_t* count, double* latency_s) {
  if (!S) {
    set_error("null server");
    return TAB_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("unknown ticket %lld", (long long)ticket);
    return TAB_EINVAL;
  }
  Req* r = it->second;
  const auto pred = [&] { return r->state == TAB_REQ_DONE || r->state == TAB_REQ_FAILED; };
  if (timeout_s < 0) {
    S->cv_done.wait(lk, pred);
  } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
    set_error("request %lld not finished within %.3f s", (long long)ticket, timeout_s);
    return TAB_ESTATE;
  }
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  if (count) *count = (int64_t)r->out.size();
  const int status = r->status;
  if (status == TAB_OK && out) memcpy(out, r->out.data(), (size_t)std::min<int64_t>(cap, (int64_t)r->out.size()));
  if (status != TAB_OK) set_error("%s", r->msg);
  S->reqs.erase(it);
  cudaFreeHost(r->pinned);
  delete r;
  return status;
}

int tab_server_inject(tab_server_t S, int64_t ticket, int kind) {
  if (!S) {
    set_error("null server");
    return TAB_EINVAL;
  }
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("unknown ticket %lld", (long long)ticket);
    return TAB_EINVAL;
  }
  if (kind != TAB_FAULT_DROP_COMPLETION) {
    set_error("unknown fault kind %d", kind);
    return TAB_EINVAL;
  }
  it->second->drop_completion = true;
  return TAB_OK;
}

int tab_server_stats_get(tab_server_t S, tab_server_stats* out) {
  if (!S || !out) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->st;
  out->inflight = (int64_t)S->running.size();
  out->queued = (int64_t)S->pending.size();
  out->mem_used = S->mem_used;
  return TAB_OK;
}

int tab_server_destroy(tab_server_t S) {
  if (!S) return TAB_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& kv : S->reqs) {
    if (kv.second->pinned) cudaFreeHost(kv.second->pinned);
    delete kv.second;
  }
  for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
  for (cudaStream_t st : S->grid_streams) cudaStreamDestroy(st);
  delete S;
  return TAB_OK;
}

}  // extern "C"
