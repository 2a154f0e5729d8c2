// tab_api.cpp -- C-ABI entry points of libtab (declared in include/tab.h):
// handle lifetime, stream binding, gate application, measurement, outcome
// log, import/export and error reporting.  All tableau arithmetic happens in
// the CUDA kernels; this file validates, marshals and launches.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <thread>
#include <memory>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "philox.cuh"
#include "pool.h"
#include "sct.h"
#include "tab_internal.h"
#include "trace.h"

namespace tab {
const char* last_error();
}

using namespace tab;

#define CU(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                  \
      return TAB_ECUDA;                                                           \
    }                                                                             \
  } while (0)

struct tab_s {
  int32_t n = 0, Wh = 0, W = 0;
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_mem = true;
  void* base = nullptr;
  uint32_t *X = nullptr, *Z = nullptr, *R = nullptr;
  MeasWork mw{};
  int meas_ctas = 1;
  uint32_t* rw = nullptr;     // grid-resident measurement workspace
  GridBar* rbar = nullptr;
  int res_ctas = 0;           // CTAs of the grid-resident engine (0: does not fit)
  uint64_t seed = 1, cid = 0;
  uint32_t shot = 0;
  uint64_t k = 0;             // next measurement index
  uint64_t noise_k = 0;       // next noise-op index (TAB_DEPOL1 / TAB_XERR / TAB_ZERR)
  uint8_t* log = nullptr;     // device outcome log
  int64_t log_cap = 0, log_len = 0;
  int64_t launches = 0;
  int64_t h2d_bytes = 0, d2h_bytes = 0;  // host <-> device copies made for callers
  int sticky = TAB_OK;        // latched device error
  int engine = TAB_ENGINE_AUTO;
  int shape_threads = 0, shape_batch = 0;  // tuned launch shape (0: default)
  // pinned staging areas for program uploads (one H2D copy per upload), used
  // in turn: an upload waits only for the copy out of the area it reuses
  struct Stage {
    uint8_t* p = nullptr;  // pinned host buffer
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool pending = false;
    uint8_t* dev = nullptr;  // device buffer the copy goes to (stream-ordered reuse)
    size_t dcap = 0;
    cudaEvent_t done = nullptr;  // after the kernels that read `dev` (side-stream uploads)
    bool done_pending = false;
  };
  cudaStream_t cstream = nullptr;  // copy stream of the pipelined apply's uploads
  static constexpr int kStages = 4;
  Stage stg[kStages];
  int stg_next = 0;
  std::vector<HostProgram> pipe;  // chunk programs of the pipelined apply (reused)
  HostProgram pipe_merged;        // consecutive chunks taken as one program (no records)
  std::vector<uint2*> pipe_pin;   // per chunk: its block records in pinned memory
  std::vector<size_t> pipe_cap;   //   and that buffer's capacity (records)
  cudaEvent_t pipe_end = nullptr; // after the last copy out of the pinned buffers
  static constexpr int kPipeEv = 4;
  cudaEvent_t pipe_ev[kPipeEv] = {};  // ends of the pipelined apply's launches
  unsigned long long* workc = nullptr;  // work counters (tab_count_work), 4 words
};

struct tab_prog_s {
  HostProgram hp;
  uint32_t* d_ops = nullptr;
  uint32_t* d_layer = nullptr;
  Seg* d_segs = nullptr;
  uint2* d_blk = nullptr;
  uint32_t* d_blk_off = nullptr;
};

// Device copy of a compiled program.
struct DevProg {
  uint32_t* ops = nullptr;
  uint32_t* layer = nullptr;
  Seg* segs = nullptr;
  uint2* blk = nullptr;       // block records, for the block gate kernel
  uint32_t* blk_off = nullptr;
  void* base = nullptr;       // single allocation holding all of the above (staged uploads)
  bool kept = false;          // base is a staging area's device buffer: not freed after use
  int stage = -1;             // that staging area
};

namespace {


int sm_count_of(int dev) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) v = 1;
  return v < 1 ? 1 : v;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct Sizes {
  size_t planes, sign, work, rwork, total;
};

Sizes sizes_for(int n, int max_ctas) {
  const int Wh = half_words(n), W = 2 * Wh;
  Sizes s;
  s.planes = align256((size_t)n * W * 4);
  s.sign = align256((size_t)W * 4);
  s.work = align256(measure_work_words(n, max_ctas) * 4);
  s.rwork = align256(resident_work_words(n, max_ctas) * 4 + sizeof(GridBar) + 64);
  s.total = 2 * s.planes + s.sign + s.work + s.rwork;
  return s;
}

int check_handle(tab_t h) {
  if (!h) {
    set_error("null handle");
    return TAB_EINVAL;
  }
  if (h->sticky != TAB_OK) {
    set_error("handle unusable after an earlier device error");
    return h->sticky;
  }
  return TAB_OK;
}

// Read back the device error word (synchronous) and latch it.
int poll_device_error(tab_t h) {
  int err = 0;
  cudaError_t e = cudaMemcpyAsync(&err, h->mw.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    set_error("device error: %s", cudaGetErrorString(e));
    h->sticky = TAB_ECUDA;
    return TAB_ECUDA;
  }
  if (err == DERR_TIMEOUT) {
    set_error("a device-side wait timed out");
    h->sticky = TAB_ETIMEOUT;
    return TAB_ETIMEOUT;
  }
  if (err == DERR_BOUNDS) {
    set_error("device reported an index out of range (debug build check)");
    h->sticky = TAB_EDEVICE;
    return TAB_EDEVICE;
  }
  if (err != 0) {
    set_error("device reported inconsistency code %d", err);
    h->sticky = TAB_EDEVICE;
    return TAB_EDEVICE;
  }
  return TAB_OK;
}

int setup(tab_t h, int32_t n, void* mem, bool own) {
  h->n = n;
  h->Wh = half_words(n);
  h->W = 2 * h->Wh;
  CU(cudaGetDevice(&h->dev));
  const int sms = sm_count_of(h->dev);
  h->mw.max_ctas = sms;
  const Sizes s = sizes_for(n, sms);
  char* b = static_cast<char*>(mem);
  h->base = mem;
  h->own_mem = own;
  h->X = reinterpret_cast<uint32_t*>(b);
  h->Z = reinterpret_cast<uint32_t*>(b + s.planes);
  h->R = reinterpret_cast<uint32_t*>(b + 2 * s.planes);
  uint32_t* w = reinterpret_cast<uint32_t*>(b + 2 * s.planes + s.sign);
  h->mw.ph = w;
  w += (size_t)sms * 2 * h->W;
  h->mw.r4 = w;
  w += 2 * (size_t)h->W;
  h->mw.dp = w;
  w += 2 * (size_t)sms;
  h->mw.bar = reinterpret_cast<GridBar*>(w);
  w += 16;
  h->mw.err = reinterpret_cast<int*>(w);
  h->meas_ctas = measure_ctas_for(n, sms, sms);
  char* rb = b + 2 * s.planes + s.sign + s.work;
  h->rbar = reinterpret_cast<GridBar*>(rb);
  h->rw = reinterpret_cast<uint32_t*>(rb + 64);
  h->res_ctas = resident_ctas_for(n, h->Wh, sms);
  CU(cudaMemsetAsync(h->mw.err, 0, sizeof(int), h->stream));
  launch_init(h->X, h->Z, h->R, n, h->Wh, h->stream);
  h->launches++;
  CU(cudaGetLastError());
  return TAB_OK;
}

int ensure_log(tab_t h, int64_t extra) {
  const int64_t need = h->log_len + extra;
  if (need <= h->log_cap) return TAB_OK;
  int64_t cap = h->log_cap ? h->log_cap : 4096;
  while (cap < need) cap *= 2;
  uint8_t* nl = nullptr;
  CU(cudaMallocAsync((void**)&nl, (size_t)cap, h->stream));
  if (h->log_len) CU(cudaMemcpyAsync(nl, h->log, (size_t)h->log_len, cudaMemcpyDeviceToDevice, h->stream));
  if (h->log) CU(cudaFreeAsync(h->log, h->stream));
  h->log = nl;
  h->log_cap = cap;
  return TAB_OK;
}

bool use_single_cta(tab_t h) {
  if (h->engine == TAB_ENGINE_SINGLE_CTA) return true;
  if (h->engine != TAB_ENGINE_AUTO) return false;
  return h->n <= 256;
}

// Engine that runs a run of measurements on this handle (single-CTA runs the
// whole program), and its CTA count: grid-resident where the tableau fits the
// grid's shared memory and the selected engine allows, else streaming.
int measure_engine(tab_t h, int* ctas) {
  if (use_single_cta(h)) {
    *ctas = 1;
    return TAB_ENGINE_SINGLE_CTA;
  }
  const bool any = h->engine == TAB_ENGINE_AUTO;
  const int G = (any || h->engine == TAB_ENGINE_GRID) ? h->res_ctas : 0;
  if (G > 0) {
    *ctas = G;
    return TAB_ENGINE_GRID;
  }
  *ctas = h->meas_ctas;
  return TAB_ENGINE_STREAM;
}

// Enqueue the program.  Measurement segments use `seed`.
int run_program(tab_t h, const HostProgram& hp, const DevProg& dp, uint64_t seed) {
  if (hp.n_meas) {
    int rc = ensure_log(h, hp.n_meas);
    if (rc != TAB_OK) return rc;
  }
  if (hp.segs.empty()) return TAB_OK;
  if (use_single_cta(h)) {
    SctProgArgs A;
    A.X = h->X;
    A.Z = h->Z;
    A.R = h->R;
    A.n = h->n;
    A.Wh = h->Wh;
    A.segs = dp.segs;
    A.nsegs = (int)hp.segs.size();
    A.ops = dp.ops;
    A.layer_off = dp.layer;
    A.seed = seed;
    A.cid = h->cid;
    A.shot = h->shot;
    A.k0 = h->k;
    A.out = h->log + h->log_len;
    A.err = h->mw.err;
    CU(launch_sct_program(A, h->stream));
    h->launches++;
    h->k += (uint64_t)hp.n_meas;
    h->log_len += hp.n_meas;
    return TAB_OK;
  }
  if (hp.n_gates > 0 && !(hp.mode & kProgBlocks)) {
    set_error("the program has no block records for the multi-CTA gate kernel");
    return TAB_EINVAL;
  }
  for (size_t si = 0; si < hp.segs.size(); ++si) {
    const Seg& s = hp.segs[si];
    if (s.kind == 0) {
      {
        // gate runs that follow one another with adjacent super-layer offsets
        // (pieces of one list compiled apart) run as one launch: the shared
        // bound between two runs is an empty super-layer
        size_t sj = si;
        while (sj + 1 < hp.segs.size() && hp.segs[sj + 1].kind == 0 &&
               hp.segs[sj + 1].blk_begin == hp.segs[sj].blk_end + 1)
          ++sj;
        CU(launch_gates_block(h->X, h->Z, h->R, h->n, h->W, dp.blk, dp.blk_off + s.blk_begin,
                              (int)(hp.segs[sj].blk_end - s.blk_begin), h->mw.err, h->stream,
                              h->shape_threads));
        si = sj;
      }
      h->launches++;
    } else {
      const int nm = (int)(s.op_end - s.op_begin);
      int ctas = 0;
      const int me = measure_engine(h, &ctas);
      if (me == TAB_ENGINE_GRID)
        CU(launch_measure_resident(h->X, h->Z, h->R, h->n, h->Wh, dp.ops + s.op_begin, nm, h->k,
                                   seed, h->cid, h->shot, h->log + h->log_len, h->mw.err, h->rw,
                                   h->rbar, ctas, h->stream, h->shape_batch));
      else
        CU(launch_measure(h->X, h->Z, h->R, h->n, h->Wh, dp.ops + s.op_begin, nm, h->k, seed,
                          h->cid, h->shot, h->log + h->log_len, h->mw, h->meas_ctas, h->stream));
      h->launches++;
      h->k += (uint64_t)nm;
      h->log_len += nm;
    }
  }
  return TAB_OK;
}

int upload(const HostProgram& hp, DevProg* d, cudaStream_t s, bool async_alloc) {
  const size_t ob = (hp.ops.size() + kOpsPad) * 4;  // TMA chunks may read past the end
  const size_t lb = std::max<size_t>(hp.layer_off.size(), 1) * 4;
  const size_t sb = std::max<size_t>(hp.segs.size(), 1) * sizeof(Seg);
  if (async_alloc) {
    CU(cudaMallocAsync((void**)&d->ops, ob, s));
    CU(cudaMallocAsync((void**)&d->layer, lb, s));
    CU(cudaMallocAsync((void**)&d->segs, sb, s));
  } else {
    CU(cudaMalloc((void**)&d->ops, ob));
    CU(cudaMalloc((void**)&d->layer, lb));
    CU(cudaMalloc((void**)&d->segs, sb));
  }
  if (!hp.ops.empty())
    CU(cudaMemcpyAsync(d->ops, hp.ops.data(), hp.ops.size() * 4, cudaMemcpyHostToDevice, s));
  CU(cudaMemsetAsync(d->ops + hp.ops.size(), 0, (size_t)kOpsPad * 4, s));
  if (!hp.layer_off.empty())
    CU(cudaMemcpyAsync(d->layer, hp.layer_off.data(), hp.layer_off.size() * 4,
                       cudaMemcpyHostToDevice, s));
  if (!hp.segs.empty())
    CU(cudaMemcpyAsync(d->segs, hp.segs.data(), hp.segs.size() * sizeof(Seg),
                       cudaMemcpyHostToDevice, s));
  // block records (padded like ops: TMA chunks may read past the end)
  if (hp.mode & kProgBlocks) {
    const size_t bb = (hp.blk.size() + kOpsPad) * sizeof(uint2);
    const size_t bo = std::max<size_t>(hp.blk_off.size(), 1) * 4;
    if (async_alloc) {
      CU(cudaMallocAsync((void**)&d->blk, bb, s));
      CU(cudaMallocAsync((void**)&d->blk_off, bo, s));
    } else {
      CU(cudaMalloc((void**)&d->blk, bb));
      CU(cudaMalloc((void**)&d->blk_off, bo));
    }
    if (!hp.blk.empty())
      CU(cudaMemcpyAsync(d->blk, hp.blk.data(), hp.blk.size() * sizeof(uint2),
                         cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(d->blk + hp.blk.size(), 0, (size_t)kOpsPad * sizeof(uint2), s));
    if (!hp.blk_off.empty())
      CU(cudaMemcpyAsync(d->blk_off, hp.blk_off.data(), hp.blk_off.size() * 4,
                         cudaMemcpyHostToDevice, s));
  }
  return TAB_OK;
}

void free_async(DevProg& d, cudaStream_t s) {
  if (d.kept) return;
  if (d.base) {
    cudaFreeAsync(d.base, s);
    return;
  }
  if (d.ops) cudaFreeAsync(d.ops, s);
  if (d.layer) cudaFreeAsync(d.layer, s);
  if (d.segs) cudaFreeAsync(d.segs, s);
  if (d.blk) cudaFreeAsync(d.blk, s);
  if (d.blk_off) cudaFreeAsync(d.blk_off, s);
}

// Upload a compiled program through the handle's next staging area: one
// asynchronous copy from its pinned host buffer into its device buffer.  The
// host buffer is reused once the copy out of it has completed, so up to
// kStages uploads can be in flight behind the kernels of earlier ones; the
// device buffer is rewritten only by later work on the handle's stream, after
// the kernels that read it.  Programs above kKeptMax bytes get a device
// allocation of their own, freed after use.
// With `ext` the block records are not in hp.blk but in ext->n pinned host
// buffers, copied in order straight into the device buffer.
struct ExtBlocks {
  const uint2* const* ptr;
  const size_t* cnt;
  int n;
  size_t total;
};

// With `side` the copies run on the handle's copy stream, after the kernels
// that last read this staging area's device buffer (its `done` event, which
// the caller records once the program has run), and the handle's stream
// waits for them: a program's upload overlaps the previous program's kernels.
int upload_staged(tab_t h, const HostProgram& hp, DevProg* d, const ExtBlocks* ext = nullptr,
                  bool side = false) {
  const bool want_blk = (hp.mode & kProgBlocks) != 0;
  const size_t nblk = ext ? ext->total : hp.blk.size();
  const size_t ob = align256((hp.ops.size() + kOpsPad) * 4);
  const size_t lb = align256(std::max<size_t>(hp.layer_off.size(), 1) * 4);
  const size_t sb = align256(std::max<size_t>(hp.segs.size(), 1) * sizeof(Seg));
  const size_t bb = want_blk ? align256((nblk + kOpsPad) * sizeof(uint2)) : 0;
  const size_t bo = want_blk ? align256(std::max<size_t>(hp.blk_off.size(), 1) * 4) : 0;
  const size_t total = ob + lb + sb + bb + bo;
  const int stage = h->stg_next;
  tab_s::Stage& sg = h->stg[stage];
  h->stg_next = (h->stg_next + 1) % tab_s::kStages;
  if (sg.pending) {
    CU(cudaEventSynchronize(sg.ev));
    sg.pending = false;
  }
  if (sg.cap < total) {
    if (sg.p) cudaFreeHost(sg.p);
    sg.p = nullptr;
    sg.cap = 0;
    const size_t cap = total + total / 4;
    CU(cudaMallocHost((void**)&sg.p, cap));
    sg.cap = cap;
  }
  if (!sg.ev) CU(cudaEventCreateWithFlags(&sg.ev, cudaEventDisableTiming));
  uint8_t* st = sg.p;
  uint32_t* ops = reinterpret_cast<uint32_t*>(st);
  if (!hp.ops.empty()) memcpy(ops, hp.ops.data(), hp.ops.size() * 4);
  memset(ops + hp.ops.size(), 0, (size_t)kOpsPad * 4);
  if (!hp.layer_off.empty()) memcpy(st + ob, hp.layer_off.data(), hp.layer_off.size() * 4);
  if (!hp.segs.empty()) memcpy(st + ob + lb, hp.segs.data(), hp.segs.size() * sizeof(Seg));
  if (want_blk) {
    uint8_t* b0 = st + ob + lb + sb;
    if (!hp.blk.empty()) {  // large programs: the copy into pinned memory in pieces
      const size_t bytes = hp.blk.size() * sizeof(uint2);
      const int pieces = bytes >= ((size_t)1 << 20) ? pool_threads() : 1;
      const uint8_t* src = reinterpret_cast<const uint8_t*>(hp.blk.data());
      pool_run(pieces, [&](int i) {
        const size_t a = bytes * (size_t)i / (size_t)pieces;
        const size_t e = bytes * (size_t)(i + 1) / (size_t)pieces;
        memcpy(b0 + a, src + a, e - a);
      });
    }
    memset(b0 + nblk * sizeof(uint2), 0, (size_t)kOpsPad * sizeof(uint2));
    if (!hp.blk_off.empty()) memcpy(b0 + bb, hp.blk_off.data(), hp.blk_off.size() * 4);
  }
  constexpr size_t kKeptMax = (size_t)64 << 20;
  uint8_t* dev = nullptr;
  d->kept = total <= kKeptMax;
  d->stage = stage;
  side = side && d->kept;  // a buffer of its own is allocated in the handle's stream order
  bool grown = false;
  if (side && !h->cstream) CU(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
  if (side && !sg.done) CU(cudaEventCreateWithFlags(&sg.done, cudaEventDisableTiming));
  cudaStream_t cs = side ? h->cstream : h->stream;
  if (d->kept) {
    if (sg.dcap < total) {
      if (sg.dev) CU(cudaFreeAsync(sg.dev, h->stream));
      sg.dev = nullptr;
      sg.dcap = 0;
      const size_t cap = std::min(kKeptMax, total + total / 4);
      CU(cudaMallocAsync((void**)&sg.dev, cap, h->stream));
      sg.dcap = cap;
      grown = true;
    }
    dev = sg.dev;
  } else {
    CU(cudaMallocAsync((void**)&dev, total, h->stream));
  }
  if (side) {  // after the last kernels that read this buffer (and a new allocation)
    if (grown) {
      CU(cudaEventRecord(sg.done, h->stream));
      sg.done_pending = true;
    }
    if (sg.done_pending) CU(cudaStreamWaitEvent(cs, sg.done, 0));
    sg.done_pending = false;
  }
  if (ext && want_blk) {
    // everything but the records through the staging area, the records from
    // the parts' own pinned buffers
    const size_t rec0 = ob + lb + sb, recb = nblk * sizeof(uint2);
    CU(cudaMemcpyAsync(dev, st, rec0, cudaMemcpyHostToDevice, cs));
    size_t at = rec0;
    for (int i = 0; i < ext->n; ++i) {
      const size_t b = ext->cnt[i] * sizeof(uint2);
      if (b) CU(cudaMemcpyAsync(dev + at, ext->ptr[i], b, cudaMemcpyHostToDevice, cs));
      at += b;
    }
    CU(cudaMemcpyAsync(dev + rec0 + recb, st + rec0 + recb, total - rec0 - recb,
                       cudaMemcpyHostToDevice, cs));
  } else {
    CU(cudaMemcpyAsync(dev, st, total, cudaMemcpyHostToDevice, cs));
  }
  h->h2d_bytes += (int64_t)total;
  CU(cudaEventRecord(sg.ev, cs));
  sg.pending = true;
  if (side) CU(cudaStreamWaitEvent(h->stream, sg.ev, 0));
  d->base = dev;
  d->ops = reinterpret_cast<uint32_t*>(dev);
  d->layer = reinterpret_cast<uint32_t*>(dev + ob);
  d->segs = reinterpret_cast<Seg*>(dev + ob + lb);
  d->blk = want_blk ? reinterpret_cast<uint2*>(dev + ob + lb + sb) : nullptr;
  d->blk_off = want_blk ? reinterpret_cast<uint32_t*>(dev + ob + lb + sb + bb) : nullptr;
  return TAB_OK;
}

// Compile forms for a call on this handle: ASAP layers for the single-CTA
// engine, else the block records the multi-CTA gate kernel reads.
int compile_mode_for(tab_t h) { return use_single_cta(h) ? kProgLayers : kProgBlocks; }

}  // namespace

extern "C" {

const char* tab_last_error(void) { return tab::last_error(); }

size_t tab_bytes_required(int32_t n) {
  if (n < 1 || n > TAB_MAX_QUBITS) return 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  return sizes_for(n, sm_count_of(dev)).total;
}

int tab_create(int32_t n, tab_t* out) {
  if (!out) {
    set_error("null output pointer");
    return TAB_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || n > TAB_MAX_QUBITS) {
    set_error("n=%d outside [1, %d]", n, TAB_MAX_QUBITS);
    return TAB_ERANGE;
  }
  int dev = 0;
  CU(cudaGetDevice(&dev));
  const size_t bytes = sizes_for(n, sm_count_of(dev)).total;
  void* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes failed", bytes);
    return TAB_ENOMEM;
  }
  tab_t h = new (std::nothrow) tab_s();
  if (!h) {
    cudaFree(mem);
    set_error("host allocation failed");
    return TAB_ENOMEM;
  }
  int rc = setup(h, n, mem, true);
  if (rc != TAB_OK) {
    cudaFree(mem);
    delete h;
    return rc;
  }
  *out = h;
  return TAB_OK;
}

int tab_create_on(int32_t n, void* dev_ptr, size_t bytes, void* cuda_stream, tab_t* out) {
  if (!out || !dev_ptr) {
    set_error("null pointer argument");
    return TAB_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || n > TAB_MAX_QUBITS) {
    set_error("n=%d outside [1, %d]", n, TAB_MAX_QUBITS);
    return TAB_ERANGE;
  }
  if (((uintptr_t)dev_ptr & 255) != 0) {
    set_error("caller memory must be 256-byte aligned");
    return TAB_EINVAL;
  }
  const size_t need = tab_bytes_required(n);
  if (bytes < need) {
    set_error("caller memory too small: %zu < %zu bytes", bytes, need);
    return TAB_ENOMEM;
  }
  tab_t h = new (std::nothrow) tab_s();
  if (!h) {
    set_error("host allocation failed");
    return TAB_ENOMEM;
  }
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  int rc = setup(h, n, dev_ptr, false);
  if (rc != TAB_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return TAB_OK;
}

int tab_destroy(tab_t h) {
  if (!h) return TAB_OK;
  cudaStreamSynchronize(h->stream);
  if (h->log) cudaFreeAsync(h->log, h->stream);
  for (tab_s::Stage& sg : h->stg)
    if (sg.dev) cudaFreeAsync(sg.dev, h->stream);
  cudaStreamSynchronize(h->stream);
  if (h->own_mem && h->base) cudaFree(h->base);
  for (tab_s::Stage& sg : h->stg) {
    if (sg.p) cudaFreeHost(sg.p);
    if (sg.ev) cudaEventDestroy(sg.ev);
  }
  for (cudaEvent_t ev : h->pipe_ev)
    if (ev) cudaEventDestroy(ev);
  for (tab_s::Stage& sg : h->stg)
    if (sg.done) cudaEventDestroy(sg.done);
  if (h->cstream) {
    cudaStreamSynchronize(h->cstream);
    cudaStreamDestroy(h->cstream);
  }
  for (uint2* p : h->pipe_pin)
    if (p) cudaFreeHost(p);
  if (h->pipe_end) cudaEventDestroy(h->pipe_end);
  if (h->workc) cudaFree(h->workc);
  delete h;
  return TAB_OK;
}

int tab_num_qubits(tab_t h, int32_t* n) {
  if (!h || !n) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  *n = h->n;
  return TAB_OK;
}

int tab_set_stream(tab_t h, void* cuda_stream) {
  if (!h) {
    set_error("null handle");
    return TAB_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (s != h->stream) {
    // the staging buffers are reused in the order of the handle's stream
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
      set_error("cuda: %s", cudaGetErrorString(e));
      return TAB_ECUDA;
    }
  }
  h->stream = s;
  return TAB_OK;
}

int tab_set_rng(tab_t h, uint64_t seed, uint64_t circuit_id, uint32_t shot) {
  int rc = check_handle(h);
  if (rc) return rc;
  h->seed = seed;
  h->cid = circuit_id;
  h->shot = shot;
  h->k = 0;
  h->noise_k = 0;
  return TAB_OK;
}

int tab_reset(tab_t h) {
  // an error latched on the device by a bounded wait or a consistency check
  // leaves the CUDA context usable: reset clears it (after the failed work
  // has drained) and re-initialises the tableau
  if (h && (h->sticky == TAB_ETIMEOUT || h->sticky == TAB_EDEVICE)) {
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaMemsetAsync(h->mw.err, 0, sizeof(int), h->stream));
    h->sticky = TAB_OK;
  }
  int rc = check_handle(h);
  if (rc) return rc;
  launch_init(h->X, h->Z, h->R, h->n, h->Wh, h->stream);
  h->launches++;
  CU(cudaGetLastError());
  h->k = 0;
  h->noise_k = 0;
  h->log_len = 0;
  return TAB_OK;
}

// Largest chunk (words) of the pipelined tab_apply: TAB_APPLY_CHUNK when set
// (0 turns the pipeline off), else about a quarter of the list per compile
// thread, within [2^13, 2^16] -- several rounds of chunks, so that the GPU
// work of the last round, which no compile hides, stays short.
static int64_t apply_chunk(int64_t count) {
  static int64_t env = -2;
  if (env == -2) {
    const char* e = getenv("TAB_APPLY_CHUNK");
    env = e ? std::max<int64_t>(0, atoll(e)) : -1;
  }
  if (env >= 0) return env;
  const int64_t per = count / (4 * (int64_t)std::max(1, pool_threads() - 1));
  return std::min<int64_t>((int64_t)1 << 16, std::max<int64_t>((int64_t)1 << 13, per));
}

// tab_apply for a long list on the block-kernel engines, once the whole list
// has been validated (nothing runs if any word is bad): its chunks are
// compiled by the host pool in list order while one pool thread uploads and
// launches them, so the GPU starts on the first chunk while later ones are
// still being compiled.  The chunks grow from 2^13 words (the GPU starts
// early) to `chunk` and shrink again over the tail; the launcher takes every
// chunk compiled by the time it is free as one program (one upload, one gate
// launch per gate run).
static int apply_pipelined(tab_t h, const tab_gate* gates, int64_t count, int64_t chunk) {
  // chunk bounds: doubling from 2^13 words up to `chunk`, then `chunk`, and
  // over the tail guided sizes (a share of what is left per compile thread,
  // at least 2^12), so the last chunks finish close together and little GPU
  // work is still queued when the host is done
  const int64_t T = std::max(1, pool_threads() - 1), lo = (int64_t)1 << 12;
  std::vector<int64_t> bnd(1, 0);
  for (int64_t s = std::min<int64_t>(chunk, (int64_t)1 << 13); bnd.back() < count;
       s = std::min<int64_t>(chunk, 2 * s)) {
    const int64_t left = count - bnd.back();
    const int64_t step = 2 * left > T * chunk ? s : std::max(lo, std::min(s, left / T));
    bnd.push_back(std::min<int64_t>(count, bnd.back() + step));
  }
  const int nc = (int)bnd.size() - 1;
  if (h->pipe.size() < (size_t)nc) h->pipe.resize((size_t)nc);
  if (h->pipe_pin.size() < (size_t)nc) {
    h->pipe_pin.resize((size_t)nc, nullptr);
    h->pipe_cap.resize((size_t)nc, 0);
  }
  // the previous call's copies out of the pinned record buffers are done
  // before the compile threads write them again
  if (h->pipe_end) CU(cudaEventSynchronize(h->pipe_end));
  // the uploads run on the copy stream: it first waits for everything already
  // queued on the handle's stream (earlier programs may still read the
  // staging areas' device buffers)
  if (!h->cstream) CU(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
  if (!h->pipe_end) CU(cudaEventCreateWithFlags(&h->pipe_end, cudaEventDisableTiming));
  CU(cudaEventRecord(h->pipe_end, h->stream));
  CU(cudaStreamWaitEvent(h->cstream, h->pipe_end, 0));
  std::vector<HostProgram>& parts = h->pipe;
  std::unique_ptr<std::atomic<int>[]> state(new std::atomic<int>[(size_t)nc]);
  for (int i = 0; i < nc; ++i) state[i].store(0);
  int crc = TAB_OK;
  std::string cmsg;
  pool_run(nc + 1, [&](int idx) {
    if (idx == 0) {  // the launcher (indices are taken in order: it starts first)
      cudaSetDevice(h->dev);
      for (cudaEvent_t& ev : h->pipe_ev)
        if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) ev = nullptr;
      // launches recorded, and known finished: with two still queued on the
      // GPU, the launcher keeps merging chunks instead of adding a third
      // (fewer, larger launches while the GPU is behind)
      int issued = 0, finished = 0;
      auto in_flight = [&]() {
        while (finished < issued) {
          cudaEvent_t ev = h->pipe_ev[finished % tab_s::kPipeEv];
          if (ev && cudaEventQuery(ev) != cudaSuccess) break;
          ++finished;
        }
        return issued - finished;
      };
      for (int i = 0; i < nc;) {
        while (state[i].load(std::memory_order_acquire) == 0) std::this_thread::yield();
        int j = i + 1;
        for (;;) {
          while (j < nc && state[j].load(std::memory_order_acquire) != 0) ++j;
          if (j == nc || in_flight() < 2) break;
          std::this_thread::yield();
        }
        int r = TAB_OK;
        for (int c = i; c < j; ++c)
          if (state[c].load(std::memory_order_relaxed) < 0) r = TAB_EINVAL;
        if (r != TAB_OK && crc == TAB_OK) cmsg = "chunk compile failed";
        // chunks i .. j-1 as one program: the small arrays merged here, the
        // block records copied from each chunk's pinned buffer
        const HostProgram* hp = &h->pipe_merged;
        std::vector<size_t> cnt((size_t)(j - i));
        ExtBlocks ext{&h->pipe_pin[(size_t)i], cnt.data(), j - i, 0};
        if (r == TAB_OK && crc == TAB_OK) {
          concat_programs(h->pipe_merged, &parts[(size_t)i], (size_t)(j - i), false);
          for (int c = i; c < j; ++c) {
            cnt[(size_t)(c - i)] = parts[(size_t)c].blk.size();
            ext.total += parts[(size_t)c].blk.size();
          }
        }
        if (r == TAB_OK && crc == TAB_OK && hp->n_gates + hp->n_meas > 0) {
          DevProg d;
          r = upload_staged(h, *hp, &d, &ext, true);
          if (r == TAB_OK) r = run_program(h, *hp, d, h->seed);
          if (r == TAB_OK && d.kept) {  // the staging area's buffer is free after these kernels
            tab_s::Stage& sg = h->stg[d.stage];
            if (sg.done && cudaEventRecord(sg.done, h->stream) == cudaSuccess) sg.done_pending = true;
          }
          free_async(d, h->stream);
          if (r != TAB_OK) cmsg = last_error();
          cudaEvent_t ev = h->pipe_ev[issued % tab_s::kPipeEv];
          if (r == TAB_OK && ev && cudaEventRecord(ev, h->stream) == cudaSuccess) ++issued;
        }
        if (r != TAB_OK && crc == TAB_OK) crc = r;
        i = j;
      }
      return;
    }
    const int i = idx - 1;
    const int64_t b = bnd[(size_t)i], e = bnd[(size_t)i + 1];
    int r = build_validated_blocks(h->n, gates + b, e - b, &parts[(size_t)i]);
    const size_t nb = parts[(size_t)i].blk.size();
    if (r == TAB_OK && nb > h->pipe_cap[(size_t)i]) {  // grow this chunk's pinned buffer
      if (h->pipe_pin[(size_t)i]) cudaFreeHost(h->pipe_pin[(size_t)i]);
      h->pipe_pin[(size_t)i] = nullptr;
      h->pipe_cap[(size_t)i] = 0;
      const size_t cap = nb + nb / 4 + 64;
      if (cudaMallocHost((void**)&h->pipe_pin[(size_t)i], cap * sizeof(uint2)) == cudaSuccess)
        h->pipe_cap[(size_t)i] = cap;
      else
        r = TAB_ENOMEM;
    }
    if (r == TAB_OK && nb)
      memcpy(h->pipe_pin[(size_t)i], parts[(size_t)i].blk.data(), nb * sizeof(uint2));
    state[i].store(r == TAB_OK ? 1 : -1, std::memory_order_release);
  });
  if (!h->pipe_end) CU(cudaEventCreateWithFlags(&h->pipe_end, cudaEventDisableTiming));
  CU(cudaEventRecord(h->pipe_end, h->stream));
  if (crc != TAB_OK) set_error("%s", cmsg.c_str());
  return crc;
}

// Extended ops (tab.h) lowered to base ops.
//  * A noise op becomes the Pauli its Philox draw selects, or nothing.  The
//    draw uses the RNG context (seed, circuit, shot) and the noise counter
//    *noise_k, which this advances; with noise_k == nullptr noise ops are
//    rejected.
//  * MX and MY are Z measurements between basis changes (MX: H, MZ, H; MY:
//    S^dag H, MZ, H S).  A maximal run of consecutive measurement ops (MZ,
//    MZR, MX, MY) on pairwise distinct qubits is lowered as: every
//    pre-rotation, then the Z measurements in their order, then every
//    post-rotation.  A one-qubit gate on qubit b commutes with everything a Z
//    measurement of qubit a != b does to the tableau (it conjugates every row
//    alike, and conjugation respects row products and signs), so the result is
//    the one of the ops taken one by one, and the run stays one measurement
//    segment.
// The list has been validated with extended ops allowed.  Plain words are
// copied in spans.
static int lower_ops(int32_t n, const tab_gate* g, int64_t count, uint64_t seed, uint64_t cid,
                     uint32_t shot, uint64_t* noise_k, std::vector<tab_gate>& out,
                     bool keep_noise = false) {
  constexpr uint32_t kNoiseKeyTag = 0x4E4F4953u;  // noise draws use a key of their own
  out.clear();
  out.reserve((size_t)count + (size_t)count / 4 + 8);
  auto put = [&](uint32_t op, uint64_t q) { out.push_back(tab_make_gate(op, (uint32_t)q, 0)); };
  auto op_of = [&](int64_t i) { return (uint32_t)(g[i] >> 56); };
  auto q1_of = [&](int64_t i) { return (g[i] >> 28) & 0xFFFFFFFull; };
  auto is_meas = [](uint32_t op) {
    return op == TAB_MZ || op == TAB_MZR || op == TAB_MX || op == TAB_MY;
  };
  std::vector<uint32_t> seen((size_t)n, 0u);  // run stamp per qubit
  uint32_t stamp = 0;
  int64_t span = 0;  // first plain word not yet copied
  for (int64_t i = 0; i < count; ++i) {
    const uint32_t op = op_of(i);
    if (op < TAB_MX && !is_meas(op)) continue;  // plain gate word
    out.insert(out.end(), g + span, g + i);
    if (is_meas(op)) {
      // the run: consecutive measurement ops on distinct qubits
      ++stamp;
      int64_t e = i;
      bool ext = false;
      while (e < count && is_meas(op_of(e)) && seen[(size_t)q1_of(e)] != stamp) {
        seen[(size_t)q1_of(e)] = stamp;
        ext = ext || op_of(e) == TAB_MX || op_of(e) == TAB_MY;
        ++e;
      }
      if (!ext) {  // plain measurements only: copy them as they are
        out.insert(out.end(), g + i, g + e);
      } else {
        for (int64_t k = i; k < e; ++k) {
          if (op_of(k) == TAB_MY) put(TAB_SDG, q1_of(k));
          if (op_of(k) == TAB_MX || op_of(k) == TAB_MY) put(TAB_H, q1_of(k));
        }
        for (int64_t k = i; k < e; ++k) put(op_of(k) == TAB_MZR ? TAB_MZR : TAB_MZ, q1_of(k));
        for (int64_t k = i; k < e; ++k) {
          if (op_of(k) == TAB_MX || op_of(k) == TAB_MY) put(TAB_H, q1_of(k));
          if (op_of(k) == TAB_MY) put(TAB_S, q1_of(k));
        }
      }
      span = e;
      i = e - 1;
      continue;
    }
    // a noise op
    if (keep_noise) {  // kept as it is, for a per-shot draw on the device
      out.push_back(g[i]);
      span = i + 1;
      continue;
    }
    if (!noise_k) {
      set_error("gate %lld: noise ops are accepted by tab_apply only", (long long)i);
      return TAB_EINVAL;
    }
    const uint64_t j = (*noise_k)++;
    const uint4 r = philox4x32_10(make_uint4((uint32_t)j, shot, (uint32_t)cid, (uint32_t)(cid >> 32)),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ kNoiseKeyTag));
    if ((r.x >> 4) < (uint32_t)(g[i] & 0xFFFFFFFull)) {
      static const uint32_t kDepol[3] = {TAB_X, TAB_Y, TAB_Z};
      const uint32_t pauli = op == TAB_XERR   ? (uint32_t)TAB_X
                             : op == TAB_ZERR ? (uint32_t)TAB_Z
                                              : kDepol[((uint64_t)r.y * 3u) >> 32];
      put(pauli, q1_of(i));
    }
    span = i + 1;
  }
  out.insert(out.end(), g + span, g + count);
  return TAB_OK;
}

static int lower_extended(tab_t h, int32_t n, const tab_gate* g, int64_t count,
                          std::vector<tab_gate>& out) {
  if (!h) return lower_ops(n, g, count, 0, 0, 0, nullptr, out);
  return lower_ops(n, g, count, h->seed, h->cid, h->shot, &h->noise_k, out);
}

int tab_lower_ops(int32_t n, const tab_gate* gates, int64_t count, uint64_t seed,
                  uint64_t circuit_id, uint32_t shot, uint64_t* noise_counter, tab_gate* out,
                  int64_t out_cap, int64_t* out_count) {
  if (n < 1 || n > TAB_MAX_QUBITS) {
    set_error("n=%d outside [1, %d]", n, TAB_MAX_QUBITS);
    return TAB_ERANGE;
  }
  if (!out_count || (out_cap > 0 && !out)) {
    set_error("null output pointer");
    return TAB_EINVAL;
  }
  int64_t ext = 0;
  int rc = validate_program(n, gates, count, &ext);
  if (rc) return rc;
  std::vector<tab_gate> low;
  uint64_t nk = noise_counter ? *noise_counter : 0;
  rc = lower_ops(n, gates, count, seed, circuit_id, shot, &nk, low);
  if (rc) return rc;
  *out_count = (int64_t)low.size();
  if ((int64_t)low.size() > out_cap) {
    set_error("output needs %lld words", (long long)low.size());
    return TAB_ENOMEM;
  }
  if (!low.empty()) memcpy(out, low.data(), low.size() * sizeof(tab_gate));
  if (noise_counter) *noise_counter = nk;
  return TAB_OK;
}

int tab_apply(tab_t h, const tab_gate* gates, int64_t count) {
  tab::TraceRange trace_("tab_apply");
  int rc = check_handle(h);
  if (rc) return rc;
  int64_t ext = 0;
  rc = validate_program(h->n, gates, count, &ext);
  if (rc) return rc;
  std::vector<tab_gate> lowered;
  if (ext) {
    rc = lower_extended(h, h->n, gates, count, lowered);
    if (rc) return rc;
    gates = lowered.data();
    count = (int64_t)lowered.size();
  }
  if (compile_mode_for(h) == kProgBlocks && count >= ((int64_t)1 << 17) && pool_threads() >= 3) {
    const int64_t chunk = apply_chunk(count);
    if (chunk > 0) return apply_pipelined(h, gates, count, chunk);
  }
  HostProgram hp;
  rc = build_program(h->n, gates, count, &hp, compile_mode_for(h));
  if (rc) return rc;
  if (hp.n_gates + hp.n_meas == 0) return TAB_OK;
  DevProg d;
  rc = upload_staged(h, hp, &d);
  if (rc == TAB_OK) rc = run_program(h, hp, d, h->seed);
  free_async(d, h->stream);
  return rc;
}

int tab_prog_create(int32_t n, const tab_gate* gates, int64_t count, tab_prog_t* out) {
  tab::TraceRange trace_("tab_prog_create");
  if (!out) {
    set_error("null output pointer");
    return TAB_EINVAL;
  }
  *out = nullptr;
  tab_prog_t p = new (std::nothrow) tab_prog_s();
  if (!p) {
    set_error("host allocation failed");
    return TAB_ENOMEM;
  }
  // extended ops other than noise are lowered first
  int64_t ext = 0;
  std::vector<tab_gate> lowered;
  int rc = (n >= 1 && n <= TAB_MAX_QUBITS) ? validate_program(n, gates, count, &ext) : TAB_OK;
  if (rc == TAB_OK && ext) {
    rc = lower_extended(nullptr, n, gates, count, lowered);
    gates = lowered.data();
    count = (int64_t)lowered.size();
  }
  // both forms: the program may run on any engine
  if (rc == TAB_OK)
    rc = build_program(n, gates, count, &p->hp, kProgLayers | kProgBlocks | kProgBankOrder);
  if (rc == TAB_OK) {
    DevProg d;
    rc = upload(p->hp, &d, nullptr, false);
    p->d_ops = d.ops;
    p->d_layer = d.layer;
    p->d_segs = d.segs;
    p->d_blk = d.blk;
    p->d_blk_off = d.blk_off;
  }
  if (rc == TAB_OK) {
    cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
      set_error("upload failed: %s", cudaGetErrorString(e));
      rc = TAB_ECUDA;
    }
  }
  if (rc != TAB_OK) {
    tab_prog_destroy(p);
    return rc;
  }
  *out = p;
  return TAB_OK;
}

int tab_prog_destroy(tab_prog_t p) {
  if (!p) return TAB_OK;
  if (p->d_ops) cudaFree(p->d_ops);
  if (p->d_layer) cudaFree(p->d_layer);
  if (p->d_segs) cudaFree(p->d_segs);
  if (p->d_blk) cudaFree(p->d_blk);
  if (p->d_blk_off) cudaFree(p->d_blk_off);
  delete p;
  return TAB_OK;
}

int tab_prog_info(tab_prog_t p, int64_t* n_gates, int64_t* n_meas, int64_t* n_layers) {
  if (!p) {
    set_error("null program");
    return TAB_EINVAL;
  }
  if (n_gates) *n_gates = p->hp.n_gates;
  if (n_meas) *n_meas = p->hp.n_meas;
  if (n_layers) {
    int64_t L = 0;
    for (const Seg& s : p->hp.segs)
      if (s.kind == 0) L += s.layer_end - s.layer_begin;
    *n_layers = L;
  }
  return TAB_OK;
}

int tab_run(tab_t h, tab_prog_t p) {
  tab::TraceRange trace_("tab_run");
  int rc = check_handle(h);
  if (rc) return rc;
  if (!p) {
    set_error("null program");
    return TAB_EINVAL;
  }
  if (p->hp.n != h->n) {
    set_error("program built for n=%d, handle has n=%d", p->hp.n, h->n);
    return TAB_EINVAL;
  }
  DevProg d;
  d.ops = p->d_ops;
  d.layer = p->d_layer;
  d.segs = p->d_segs;
  d.blk = p->d_blk;
  d.blk_off = p->d_blk_off;
  return run_program(h, p->hp, d, h->seed);
}

static int measure_common(tab_t h, const int32_t* qubits, int32_t k, uint64_t seed,
                          int64_t* first) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (k < 0 || (k > 0 && !qubits)) {
    set_error("bad qubit list");
    return TAB_EINVAL;
  }
  std::vector<tab_gate> g((size_t)k);
  for (int32_t i = 0; i < k; ++i) {
    if (qubits[i] < 0 || qubits[i] >= h->n) {
      set_error("qubit %d outside [0, %d)", qubits[i], h->n);
      return TAB_ERANGE;
    }
    g[(size_t)i] = tab_make_gate(TAB_MZ, (uint32_t)qubits[i], 0);
  }
  HostProgram hp;
  rc = build_program(h->n, g.data(), k, &hp, compile_mode_for(h));  // measurements only
  if (rc) return rc;
  *first = h->log_len;
  if (hp.ops.empty()) return TAB_OK;
  DevProg d;
  rc = upload_staged(h, hp, &d);
  if (rc == TAB_OK) rc = run_program(h, hp, d, seed);
  free_async(d, h->stream);
  return rc;
}

int tab_measure(tab_t h, const int32_t* qubits, int32_t k, uint64_t seed, uint8_t* out_bits) {
  tab::TraceRange trace_("tab_measure");
  if (k > 0 && !out_bits) {
    set_error("null output buffer");
    return TAB_EINVAL;
  }
  int64_t first = 0;
  int rc = measure_common(h, qubits, k, seed, &first);
  if (rc) return rc;
  if (k > 0) CU(cudaMemcpyAsync(out_bits, h->log + first, (size_t)k, cudaMemcpyDeviceToHost, h->stream));
  return poll_device_error(h);
}

int tab_measure_async(tab_t h, const int32_t* qubits, int32_t k, uint8_t* dev_out_bits) {
  tab::TraceRange trace_("tab_measure_async");
  if (k > 0 && !dev_out_bits) {
    set_error("null output buffer");
    return TAB_EINVAL;
  }
  int64_t first = 0;
  int rc = measure_common(h, qubits, k, h ? h->seed : 0, &first);
  if (rc) return rc;
  if (k > 0)
    CU(cudaMemcpyAsync(dev_out_bits, h->log + first, (size_t)k, cudaMemcpyDeviceToDevice, h->stream));
  return TAB_OK;
}

int tab_expect(tab_t h, const uint8_t* paulis, int32_t k, int8_t* out) {
  tab::TraceRange trace_("tab_expect");
  int rc = check_handle(h);
  if (rc) return rc;
  if (k < 0 || (k > 0 && (!paulis || !out))) {
    set_error("bad Pauli list (k=%d)", k);
    return TAB_EINVAL;
  }
  if (k == 0) return TAB_OK;
  const size_t bytes = (size_t)k * (size_t)h->n;
  for (size_t i = 0; i < bytes; ++i)
    if (paulis[i] > 3u) {
      set_error("Pauli %lld, qubit %lld: code %u is not 0..3", (long long)(i / h->n),
                (long long)(i % h->n), (unsigned)paulis[i]);
      return TAB_EINVAL;
    }
  uint8_t* d = nullptr;
  CU(cudaMallocAsync((void**)&d, bytes + (size_t)k, h->stream));
  CU(cudaMemcpyAsync(d, paulis, bytes, cudaMemcpyHostToDevice, h->stream));
  h->h2d_bytes += (int64_t)bytes;
  int8_t* dout = reinterpret_cast<int8_t*>(d + bytes);
  cudaError_t e = launch_expect(h->X, h->Z, h->R, h->n, h->Wh, d, k, dout, h->mw.err, h->stream);
  if (e == cudaSuccess) {
    h->launches++;
    e = cudaMemcpyAsync(out, dout, (size_t)k, cudaMemcpyDeviceToHost, h->stream);
    h->d2h_bytes += k;
  }
  cudaFreeAsync(d, h->stream);
  if (e != cudaSuccess) {
    set_error("cuda: %s", cudaGetErrorString(e));
    return TAB_ECUDA;
  }
  return poll_device_error(h);
}

int tab_statevector(tab_t h, float* amps, int64_t len) {
  tab::TraceRange trace_("tab_statevector");
  int rc = check_handle(h);
  if (rc) return rc;
  const int n = h->n;
  if (n > TAB_SV_MAX_QUBITS) {
    set_error("n=%d above the state-vector limit %d", n, TAB_SV_MAX_QUBITS);
    return TAB_ERANGE;
  }
  if (!amps || len < ((int64_t)2 << n)) {
    set_error("amplitude buffer needs %lld floats", (long long)((int64_t)2 << n));
    return TAB_EINVAL;
  }
  // a basis state in the support: the Z outcomes of every qubit of a copy
  tab_t c = nullptr;
  rc = tab_create(n, &c);
  if (rc) return rc;
  rc = tab_set_stream(c, h->stream);
  uint32_t b = 0u;
  if (rc == TAB_OK) {
    const size_t planes = (size_t)n * h->W * 4;
    cudaError_t e = cudaMemcpyAsync(c->X, h->X, planes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->Z, h->Z, planes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->R, h->R, (size_t)h->W * 4, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) {
      set_error("cuda: %s", cudaGetErrorString(e));
      rc = TAB_ECUDA;
    }
  }
  if (rc == TAB_OK) {
    std::vector<int32_t> q((size_t)n);
    for (int i = 0; i < n; ++i) q[(size_t)i] = i;
    std::vector<uint8_t> bits((size_t)n);
    rc = tab_measure(c, q.data(), n, 1, bits.data());
    for (int i = 0; rc == TAB_OK && i < n; ++i) b |= (uint32_t)(bits[(size_t)i] & 1u) << i;
  }
  tab_destroy(c);
  if (rc) return rc;
  const size_t vb = (size_t)8 << n;
  char* d = nullptr;
  CU(cudaMallocAsync((void**)&d, vb + sv_work_bytes(n), h->stream));
  cudaError_t e = launch_statevector(h->X, h->Z, h->R, n, h->Wh, b, reinterpret_cast<float2*>(d),
                                     d + vb, h->stream);
  if (e == cudaSuccess) {
    h->launches += n + 5;
    e = cudaMemcpyAsync(amps, d, vb, cudaMemcpyDeviceToHost, h->stream);
    h->d2h_bytes += (int64_t)vb;
  }
  cudaFreeAsync(d, h->stream);
  if (e != cudaSuccess) {
    set_error("cuda: %s", cudaGetErrorString(e));
    return TAB_ECUDA;
  }
  return poll_device_error(h);
}

int tab_read_outcomes(tab_t h, uint8_t* out, int64_t max, int64_t* count) {
  tab::TraceRange trace_("tab_read_outcomes");
  int rc = check_handle(h);
  if (rc) return rc;
  if (count) *count = h->log_len;
  const int64_t nb = std::min<int64_t>(max, h->log_len);
  if (nb > 0) {
    if (!out) {
      set_error("null output buffer");
      return TAB_EINVAL;
    }
    CU(cudaMemcpyAsync(out, h->log, (size_t)nb, cudaMemcpyDeviceToHost, h->stream));
    h->d2h_bytes += (int64_t)nb;
  }
  return poll_device_error(h);
}

int tab_clear_outcomes(tab_t h) {
  int rc = check_handle(h);
  if (rc) return rc;
  h->log_len = 0;
  return TAB_OK;
}

int tab_set_engine(tab_t h, int engine) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (engine != TAB_ENGINE_AUTO && engine != TAB_ENGINE_SINGLE_CTA &&
      engine != TAB_ENGINE_GRID && engine != TAB_ENGINE_STREAM) {
    set_error("unknown engine %d", engine);
    return TAB_EINVAL;
  }
  if (engine == TAB_ENGINE_SINGLE_CTA && h->n > TAB_BATCH_MAX_QUBITS) {
    set_error("single-CTA engine needs n <= %d (n=%d)", TAB_BATCH_MAX_QUBITS, h->n);
    return TAB_ERANGE;
  }
  h->engine = engine;
  return TAB_OK;
}

int tab_engine_resolved(tab_t h, int* engine, int* ctas) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!engine || !ctas) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  *engine = measure_engine(h, ctas);
  return TAB_OK;
}

int tab_transfer_bytes(tab_t h, int64_t* h2d, int64_t* d2h) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h2d) *h2d = h->h2d_bytes;
  if (d2h) *d2h = h->d2h_bytes;
  return TAB_OK;
}

int tab_kernel_launches(tab_t h, int64_t* count) {
  if (!h || !count) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  *count = h->launches;
  return TAB_OK;
}

int tab_export(tab_t h, uint8_t* x, uint8_t* z, uint8_t* r) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!x || !z || !r) {
    set_error("null output buffer");
    return TAB_EINVAL;
  }
  const size_t cells = 2 * (size_t)h->n * h->n, rows = 2 * (size_t)h->n;
  uint8_t* d = nullptr;
  CU(cudaMallocAsync((void**)&d, 2 * cells + rows, h->stream));
  CU(launch_unpack(h->X, h->Z, h->R, d, d + cells, d + 2 * cells, h->n, h->Wh, h->stream));
  h->launches++;
  CU(cudaMemcpyAsync(x, d, cells, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaMemcpyAsync(z, d + cells, cells, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaMemcpyAsync(r, d + 2 * cells, rows, cudaMemcpyDeviceToHost, h->stream));
  h->d2h_bytes += (int64_t)(2 * cells + rows);
  CU(cudaFreeAsync(d, h->stream));
  return poll_device_error(h);
}

int tab_import(tab_t h, const uint8_t* x, const uint8_t* z, const uint8_t* r, uint64_t meas_counter) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!x || !z || !r) {
    set_error("null input buffer");
    return TAB_EINVAL;
  }
  const size_t cells = 2 * (size_t)h->n * h->n, rows = 2 * (size_t)h->n;
  uint8_t* d = nullptr;
  CU(cudaMallocAsync((void**)&d, 2 * cells + rows, h->stream));
  CU(cudaMemcpyAsync(d, x, cells, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(d + cells, z, cells, cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(d + 2 * cells, r, rows, cudaMemcpyHostToDevice, h->stream));
  h->h2d_bytes += (int64_t)(2 * cells + rows);
  CU(launch_pack(h->X, h->Z, h->R, d, d + cells, d + 2 * cells, h->n, h->Wh, h->stream));
  h->launches++;
  CU(cudaFreeAsync(d, h->stream));
  h->k = meas_counter;
  return poll_device_error(h);
}

int tab_sync(tab_t h) {
  int rc = check_handle(h);
  if (rc) return rc;
  return poll_device_error(h);
}

int tab_count_work(tab_t h, int32_t on) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (on && !h->workc) {
    void* p = nullptr;
    if (cudaMalloc(&p, 4 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of the work counters failed");
      return TAB_ENOMEM;
    }
    h->workc = static_cast<unsigned long long*>(p);
  }
  if (on) CU(cudaMemsetAsync(h->workc, 0, 4 * sizeof(unsigned long long), h->stream));
  h->mw.work = on ? h->workc : nullptr;
  return TAB_OK;
}

int tab_work_counts(tab_t h, int64_t* counts) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!counts) {
    set_error("null output");
    return TAB_EINVAL;
  }
  unsigned long long v[4] = {0ull, 0ull, 0ull, 0ull};
  if (h->workc) {
    CU(cudaMemcpyAsync(v, h->workc, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  for (int i = 0; i < 4; ++i) counts[i] = (int64_t)v[i];
  return TAB_OK;
}

}  // extern "C"

namespace tab {
int lower_for_runs(int32_t n, const tab_gate* g, int64_t count, bool keep_noise, uint64_t seed,
                   uint64_t cid, uint32_t shot, std::vector<tab_gate>& out) {
  uint64_t nk = 0;
  return lower_ops(n, g, count, seed, cid, shot, &nk, out, keep_noise);
}
}  // namespace tab

namespace tab {

// Internal helpers for the request server (not part of the C ABI).
int handle_outcomes_async(tab_t h, uint8_t* host, cudaStream_t* used_stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (h->log_len > 0)
    CU(cudaMemcpyAsync(host, h->log, (size_t)h->log_len, cudaMemcpyDeviceToHost, h->stream));
  if (used_stream) *used_stream = h->stream;
  return TAB_OK;
}

int handle_set_meas_ctas(tab_t h, int ctas) {
  int rc = check_handle(h);
  if (rc) return rc;
  h->meas_ctas = std::max(1, std::min(ctas, h->mw.max_ctas));
  return TAB_OK;
}

size_t handle_device_bytes(int32_t n) { return tab_bytes_required(n); }

// Compile forms a request of n qubits needs on a multi-CTA engine handle.
int grid_compile_mode(int) { return kProgBlocks; }

// Enqueue an already compiled program (the request server compiles at submit).
int handle_apply_program(tab_t h, const HostProgram& hp) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (hp.n != h->n) {
    set_error("program built for n=%d, handle has n=%d", hp.n, h->n);
    return TAB_EINVAL;
  }
  if (hp.n_gates + hp.n_meas == 0) return TAB_OK;
  if (hp.n_gates > 0 && !(hp.mode & kProgLayers) && use_single_cta(h)) {
    set_error("the single-CTA engine needs a layered program");
    return TAB_EINVAL;
  }
  DevProg d;
  rc = upload_staged(h, hp, &d);
  if (rc == TAB_OK) rc = run_program(h, hp, d, h->seed);
  free_async(d, h->stream);
  return rc;
}

int handle_view(tab_t h, HandleView* v) {
  int rc = check_handle(h);
  if (rc) return rc;
  v->n = h->n;
  v->Wh = h->Wh;
  v->dev = h->dev;
  v->X = h->X;
  v->Z = h->Z;
  v->R = h->R;
  v->stream = h->stream;
  v->seed = h->seed;
  v->cid = h->cid;
  v->k = h->k;
  v->shot = h->shot;
  v->err = h->mw.err;
  v->meas_ctas = h->meas_ctas;
  return TAB_OK;
}

void handle_set_shape(tab_t h, int block_threads, int meas_batch) {
  h->shape_threads = block_threads;
  h->shape_batch = meas_batch;
}

void handle_get_shape(tab_t h, int* block_threads, int* meas_batch) {
  *block_threads = h->shape_threads;
  *meas_batch = h->shape_batch;
}

void handle_advance_k(tab_t h, uint64_t dk) {
  h->k += dk;
  h->launches++;
}

}  // namespace tab
