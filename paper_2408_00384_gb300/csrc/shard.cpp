// shard.cpp -- a tableau whose rows are split over shards driven by host
// threads (the row-slab sharding of one large tableau; the ranks here are
// threads of one process, the exchanges go through HostComm).
//
// Shard s owns the qubit-row indices [i0, i1) -- destabilizer i and
// stabilizer n+i together, so the pivot's partner row p-n and the
// deterministic case's selection stay local -- and holds them for every
// column in the layout of kernels_shard.cu.  tab_sharded_apply compiles the
// gate list once (block program, uploaded once) and then runs it on every
// shard at once, one thread per shard:
//  * a gate run: the block gate kernel on the shard's row words (rows are
//    independent under gates: no exchange);
//  * a measurement of Z_a (AG Sec. III): local pivot candidates, an
//    all-reduce of the minimum; in the random case the owner's row p is
//    broadcast, every shard applies the rowsums to its rows and the owner
//    rewrites rows p-n and p; in the deterministic case the shards' partial
//    products are gathered on shard 0, which multiplies them; the outcome
//    is broadcast (MZR applies X where it is 1).
// Outcomes use the same Philox stream as a single tableau, so the two give
// identical results.
#include <cuda_runtime.h>
#include <stdio.h>

#include <algorithm>
#include <limits>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "shard_comm.h"
#include "tab_internal.h"
#include "trace.h"

namespace tab {

cudaError_t sh_init(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int i0, int i1, int Whs,
                    cudaStream_t s);
cudaError_t sh_pivot(const uint32_t* X, int Whs, int a, int* piv, cudaStream_t s);
cudaError_t sh_getrow(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int Whs,
                      int li, uint32_t* row, cudaStream_t s);
cudaError_t sh_rowsum(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Whs, int a, int li,
                      const uint32_t* row, int* err, cudaStream_t s);
cudaError_t sh_setrows(uint32_t* X, uint32_t* Z, uint32_t* R, int n, int Whs, int a, int li,
                       const uint32_t* row, uint64_t seed, uint64_t cid, uint32_t shot,
                       uint64_t k, uint8_t* bout, cudaStream_t s);
cudaError_t sh_partial(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int Whs,
                       int a, uint32_t* out, cudaStream_t s);
cudaError_t sh_combine(const uint32_t* parts, int shards, int n, int a, uint8_t* bout, int* err,
                       cudaStream_t s);
cudaError_t sh_xgate(const uint32_t* Z, uint32_t* R, int Whs, int a, cudaStream_t s);
cudaError_t sh_unpack(const uint32_t* X, const uint32_t* Z, const uint32_t* R, int n, int i0,
                      int i1, int Whs, uint8_t* xs, uint8_t* zs, uint8_t* rs, cudaStream_t s);

namespace {

struct Shard {
  int i0 = 0, i1 = 0, Whs = 0;
  cudaStream_t st = nullptr;
  char* mem = nullptr;            // X, Z, R, row, part, parts, err, piv, bout
  uint32_t *X = nullptr, *Z = nullptr, *R = nullptr;
  uint32_t *row = nullptr, *part = nullptr, *parts = nullptr;
  int* err = nullptr;
  int* piv = nullptr;
  uint8_t* bout = nullptr;
  uint32_t* host = nullptr;       // pinned: row / partial staging, then scalars
};

}  // namespace

}  // namespace tab

struct tab_shard_s {
  int32_t n = 0, S = 0, Wh = 0, nw = 0;
  int dev = 0;
  uint64_t seed = 1, cid = 0, k = 0;
  uint32_t shot = 0;
  std::vector<tab::Shard> sh;
  std::vector<uint8_t> log;
  int sticky = TAB_OK;
};

namespace tab {
namespace {

#define SH_CU(call)                                                          \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      set_error("cuda: %s (%s)", cudaGetErrorString(e_), #call);             \
      return TAB_ECUDA;                                                      \
    }                                                                        \
  } while (0)

size_t row_words(int n) { return (size_t)2 * ((n + 31) / 32) + 1; }

void free_shard(Shard& s) {
  if (s.st) cudaStreamSynchronize(s.st);
  if (s.mem) cudaFree(s.mem);
  if (s.host) cudaFreeHost(s.host);
  if (s.st) cudaStreamDestroy(s.st);
  s = Shard();
}

int alloc_shard(tab_shard_t h, Shard& s) {
  const size_t plane = (size_t)h->n * 2 * s.Whs * 4, rw = row_words(h->n) * 4;
  const size_t bytes = 2 * plane + (size_t)2 * s.Whs * 4 + 2 * rw + rw * (size_t)h->S + 64;
  SH_CU(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
  SH_CU(cudaMalloc((void**)&s.mem, bytes));
  SH_CU(cudaMallocHost((void**)&s.host, rw * (size_t)h->S + 64));
  char* b = s.mem;
  s.X = reinterpret_cast<uint32_t*>(b);
  s.Z = reinterpret_cast<uint32_t*>(b + plane);
  s.R = reinterpret_cast<uint32_t*>(b + 2 * plane);
  s.row = reinterpret_cast<uint32_t*>(b + 2 * plane + (size_t)2 * s.Whs * 4);
  s.part = s.row + row_words(h->n);
  s.parts = s.part + row_words(h->n);
  char* tail = reinterpret_cast<char*>(s.parts + row_words(h->n) * (size_t)h->S);
  s.err = reinterpret_cast<int*>(tail);
  s.piv = reinterpret_cast<int*>(tail + 16);
  s.bout = reinterpret_cast<uint8_t*>(tail + 32);
  SH_CU(cudaMemsetAsync(s.err, 0, sizeof(int), s.st));
  SH_CU(sh_init(s.X, s.Z, s.R, h->n, s.i0, s.i1, s.Whs, s.st));
  return TAB_OK;
}

// one rank's pass over a compiled program
struct RankCtx {
  tab_shard_t h;
  const HostProgram* hp;
  const uint2* blk;
  const uint32_t* blk_off;
  HostComm* comm;
  std::vector<uint8_t>* outcomes;  // shard 0 appends
  std::string msg;
};

int sync_check(Shard& s) {
  int err = 0;
  SH_CU(cudaMemcpyAsync(&err, s.err, sizeof(int), cudaMemcpyDeviceToHost, s.st));
  SH_CU(cudaStreamSynchronize(s.st));
  if (err == DERR_TIMEOUT) {
    set_error("a device-side wait timed out");
    return TAB_ETIMEOUT;
  }
  if (err) {
    set_error("device reported inconsistency code %d", err);
    return TAB_EDEVICE;
  }
  return TAB_OK;
}

int measure_one(RankCtx& c, int rank, int a, bool reset, uint64_t k) {
  tab_shard_t h = c.h;
  Shard& s = h->sh[(size_t)rank];
  const size_t rw = row_words(h->n);
  // 1. pivot: local candidate, then the minimum over the shards
  SH_CU(sh_pivot(s.X, s.Whs, a, s.piv, s.st));
  int local = 0;
  SH_CU(cudaMemcpyAsync(&local, s.piv, sizeof(int), cudaMemcpyDeviceToHost, s.st));
  SH_CU(cudaStreamSynchronize(s.st));
  const int64_t none = std::numeric_limits<int64_t>::max();
  const int64_t cand = local == 0x7fffffff ? none : (int64_t)s.i0 + local;
  int64_t p = none;
  if (!c.comm->allreduce_min(rank, cand, &p)) return TAB_ESTATE;
  uint8_t b = 0;
  if (p != none) {
    // 2. random case: broadcast row p, rowsums everywhere, owner rewrites p-n, p
    int owner = 0;
    while (!(p >= h->sh[(size_t)owner].i0 && p < h->sh[(size_t)owner].i1)) ++owner;
    const int li = rank == owner ? (int)(p - s.i0) : -1;
    if (rank == owner) {
      SH_CU(sh_getrow(s.X, s.Z, s.R, h->n, s.Whs, li, s.row, s.st));
      SH_CU(cudaMemcpyAsync(s.host, s.row, rw * 4, cudaMemcpyDeviceToHost, s.st));
      SH_CU(cudaStreamSynchronize(s.st));
    }
    if (!c.comm->broadcast(rank, owner, s.host, rw * 4)) return TAB_ESTATE;
    if (rank != owner) SH_CU(cudaMemcpyAsync(s.row, s.host, rw * 4, cudaMemcpyHostToDevice, s.st));
    SH_CU(sh_rowsum(s.X, s.Z, s.R, h->n, s.Whs, a, li, s.row, s.err, s.st));
    if (rank == owner) {
      SH_CU(sh_setrows(s.X, s.Z, s.R, h->n, s.Whs, a, li, s.row, h->seed, h->cid, h->shot, k,
                       s.bout, s.st));
      SH_CU(cudaMemcpyAsync(&b, s.bout, 1, cudaMemcpyDeviceToHost, s.st));
    }
    int rc = sync_check(s);
    if (rc) return rc;
    if (!c.comm->broadcast(rank, owner, &b, 1)) return TAB_ESTATE;
  } else {
    // 3. deterministic case: partial products gathered and combined on shard 0
    SH_CU(sh_partial(s.X, s.Z, s.R, h->n, s.Whs, a, s.part, s.st));
    SH_CU(cudaMemcpyAsync(s.host, s.part, rw * 4, cudaMemcpyDeviceToHost, s.st));
    SH_CU(cudaStreamSynchronize(s.st));
    std::vector<uint32_t> all(rank == 0 ? rw * (size_t)h->S : 0);
    if (!c.comm->gather(rank, 0, s.host, rw * 4, all.data())) return TAB_ESTATE;
    if (rank == 0) {
      SH_CU(cudaMemcpyAsync(s.parts, all.data(), all.size() * 4, cudaMemcpyHostToDevice, s.st));
      SH_CU(sh_combine(s.parts, h->S, h->n, a, s.bout, s.err, s.st));
      SH_CU(cudaMemcpyAsync(&b, s.bout, 1, cudaMemcpyDeviceToHost, s.st));
      int rc = sync_check(s);
      if (rc) return rc;
    }
    if (!c.comm->broadcast(rank, 0, &b, 1)) return TAB_ESTATE;
  }
  if (rank == 0) c.outcomes->push_back(b);
  if (reset && b) SH_CU(sh_xgate(s.Z, s.R, s.Whs, a, s.st));
  return TAB_OK;
}

int rank_main(RankCtx& c, int rank) {
  tab_shard_t h = c.h;
  Shard& s = h->sh[(size_t)rank];
  SH_CU(cudaSetDevice(h->dev));
  uint64_t k = h->k;
  for (const Seg& g : c.hp->segs) {
    if (g.kind == 0) {
      if (g.blk_end > g.blk_begin)
        SH_CU(launch_gates_block(s.X, s.Z, s.R, h->n, 2 * s.Whs, c.blk, c.blk_off + g.blk_begin,
                                 (int)(g.blk_end - g.blk_begin), s.err, s.st));
      continue;
    }
    for (uint32_t o = g.op_begin; o < g.op_end; ++o) {
      const uint32_t code = c.hp->ops[o];
      const int rc = measure_one(c, rank, (int)dq1(code), dop(code) == TAB_MZR, k++);
      if (rc) return rc;
    }
  }
  return sync_check(s);
}

}  // namespace
}  // namespace tab

using namespace tab;

int tab_sharded_create(int32_t n, int32_t shards, tab_shard_t* out) {
  if (!out) {
    set_error("null output pointer");
    return TAB_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || n > TAB_MAX_QUBITS || n > gates_block_max_n()) {
    set_error("n=%d outside [1, %d]", n, std::min(TAB_MAX_QUBITS, gates_block_max_n()));
    return TAB_ERANGE;
  }
  const int Wh = half_words(n), used = (n + 31) / 32;
  if (shards < 1 || shards > used) {
    set_error("shards=%d outside [1, %d] (one 32-row word at least per shard)", shards, used);
    return TAB_ERANGE;
  }
  std::unique_ptr<tab_shard_s> h(new (std::nothrow) tab_shard_s());
  if (!h) {
    set_error("host allocation failed");
    return TAB_ENOMEM;
  }
  h->n = n;
  h->S = shards;
  h->Wh = Wh;
  h->nw = used;
  SH_CU(cudaGetDevice(&h->dev));
  h->sh.resize((size_t)shards);
  for (int s = 0; s < shards; ++s) {  // row words split as evenly as possible
    const int d0 = used * s / shards, d1 = used * (s + 1) / shards;
    Shard& q = h->sh[(size_t)s];
    q.i0 = 32 * d0;
    q.i1 = std::min(n, 32 * d1);
    q.Whs = d1 - d0;
    const int rc = alloc_shard(h.get(), q);
    if (rc) {
      for (Shard& x : h->sh) free_shard(x);
      return rc;
    }
  }
  for (Shard& q : h->sh) SH_CU(cudaStreamSynchronize(q.st));
  *out = h.release();
  return TAB_OK;
}

int tab_sharded_destroy(tab_shard_t h) {
  if (!h) return TAB_OK;
  for (Shard& s : h->sh) free_shard(s);
  delete h;
  return TAB_OK;
}

int tab_sharded_set_rng(tab_shard_t h, uint64_t seed, uint64_t circuit_id, uint32_t shot) {
  if (!h) {
    set_error("null handle");
    return TAB_EINVAL;
  }
  h->seed = seed;
  h->cid = circuit_id;
  h->shot = shot;
  h->k = 0;
  return TAB_OK;
}

int tab_sharded_apply(tab_shard_t h, const tab_gate* gates, int64_t count) {
  tab::TraceRange trace_("tab_sharded_apply");
  if (!h) {
    set_error("null handle");
    return TAB_EINVAL;
  }
  if (h->sticky != TAB_OK) {
    set_error("handle unusable after an earlier error");
    return h->sticky;
  }
  HostProgram hp;
  int rc = build_program(h->n, gates, count, &hp, kProgBlocks);
  if (rc) return rc;
  if (hp.n_gates + hp.n_meas == 0) return TAB_OK;
  // the block program once, read by every shard
  uint2* blk = nullptr;
  uint32_t* off = nullptr;
  const size_t nb = hp.blk.size() + kOpsPad, no = std::max<size_t>(hp.blk_off.size(), 1);
  SH_CU(cudaMalloc((void**)&blk, nb * sizeof(uint2)));
  if (cudaMalloc((void**)&off, no * 4) != cudaSuccess) {
    cudaFree(blk);
    set_error("cudaMalloc failed");
    return TAB_ENOMEM;
  }
  cudaMemset(blk, 0, nb * sizeof(uint2));
  if (!hp.blk.empty()) cudaMemcpy(blk, hp.blk.data(), hp.blk.size() * sizeof(uint2), cudaMemcpyHostToDevice);
  if (!hp.blk_off.empty()) cudaMemcpy(off, hp.blk_off.data(), hp.blk_off.size() * 4, cudaMemcpyHostToDevice);
  HostComm comm(h->S);
  std::vector<uint8_t> outcomes;
  std::vector<RankCtx> ctx((size_t)h->S, RankCtx{h, &hp, blk, off, &comm, &outcomes, {}});
  std::vector<int> rcs((size_t)h->S, TAB_OK);
  std::vector<std::thread> th;
  for (int r = 0; r < h->S; ++r)
    th.emplace_back([&, r] {
      rcs[(size_t)r] = rank_main(ctx[(size_t)r], r);
      if (rcs[(size_t)r] != TAB_OK) {
        ctx[(size_t)r].msg = tab_last_error();
        comm.abort();
      }
    });
  for (auto& t : th) t.join();
  cudaFree(blk);
  cudaFree(off);
  // the first failure that is not another rank's abort
  for (int r = 0; r < h->S; ++r)
    if (rcs[(size_t)r] != TAB_OK && rcs[(size_t)r] != TAB_ESTATE) {
      set_error("shard %d: %s", r, ctx[(size_t)r].msg.c_str());
      h->sticky = rcs[(size_t)r];
      return rcs[(size_t)r];
    }
  for (int r = 0; r < h->S; ++r)
    if (rcs[(size_t)r] != TAB_OK) {
      set_error("shard %d: %s", r, ctx[(size_t)r].msg.c_str());
      h->sticky = rcs[(size_t)r];
      return rcs[(size_t)r];
    }
  h->k += (uint64_t)outcomes.size();
  h->log.insert(h->log.end(), outcomes.begin(), outcomes.end());
  return TAB_OK;
}

int tab_sharded_read_outcomes(tab_shard_t h, uint8_t* out, int64_t max, int64_t* count) {
  if (!h) {
    set_error("null handle");
    return TAB_EINVAL;
  }
  if (count) *count = (int64_t)h->log.size();
  const int64_t nb = std::min<int64_t>(max, (int64_t)h->log.size());
  if (nb > 0) {
    if (!out) {
      set_error("null output buffer");
      return TAB_EINVAL;
    }
    memcpy(out, h->log.data(), (size_t)nb);
  }
  return TAB_OK;
}

int tab_sharded_export(tab_shard_t h, uint8_t* x, uint8_t* z, uint8_t* r) {
  if (!h || !x || !z || !r) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  const int n = h->n;
  const size_t cells = (size_t)2 * n * n;
  uint8_t* d = nullptr;
  SH_CU(cudaMalloc((void**)&d, 2 * cells + 2 * (size_t)n));
  int rc = TAB_OK;
  for (Shard& s : h->sh) {
    cudaError_t e = sh_unpack(s.X, s.Z, s.R, n, s.i0, s.i1, s.Whs, d, d + cells, d + 2 * cells, s.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s.st);
    if (e != cudaSuccess) {
      set_error("cuda: %s", cudaGetErrorString(e));
      rc = TAB_ECUDA;
      break;
    }
  }
  if (rc == TAB_OK) {
    cudaError_t e = cudaMemcpy(x, d, cells, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(z, d + cells, cells, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(r, d + 2 * cells, 2 * (size_t)n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      set_error("cuda: %s", cudaGetErrorString(e));
      rc = TAB_ECUDA;
    }
  }
  cudaFree(d);
  return rc;
}
