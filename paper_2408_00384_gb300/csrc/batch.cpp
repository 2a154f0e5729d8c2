// batch.cpp -- batched runs of many independent circuits and shots in one
// persistent launch (tab_batch_* in include/tab.h).
//
// Packing: every circuit's gate list is compiled (validated, ASAP-layered)
// and the programs are concatenated into one op table, one layer-offset table
// and one segment table.  Work items are one shared-prefix item per circuit
// (the gates before its first measurement, run once) and one item per
// (circuit, shot) (the rest of the circuit with that shot's outcome stream).
// Items are ordered prefix-first, each class by decreasing estimated cost, so
// the persistent CTAs pull the long items first and the tail stays short.
// A replay is a CUDA graph: a memset of the queue / ready flags / error word
// and the kernel, whose (seed, output) arguments are updated in place.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "pool.h"
#include "sct.h"
#include "tab_internal.h"
#include "trace.h"

using namespace tab;

#define CUB(call)                                                             \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));              \
      return TAB_ECUDA;                                                       \
    }                                                                         \
  } while (0)

struct tab_batch_s {
  int m = 0;
  int64_t n_gates = 0, n_meas = 0, out_bytes = 0;
  int64_t h2d_bytes = 0;                    // compiled tables copied to the device
  int max_n = 1;
  bool sample = false;                      // terminal measurements by the sampler
  int nsampled = 0;
  std::vector<int32_t> cn, ck, cshots;      // per circuit: n, terminal K, shots
  std::vector<int32_t> cnoise;              // per circuit: noise ops (drawn per shot)
  std::vector<uint8_t> csampled;
  int sms = 1;
  int nitems = 0;
  // Size classes: circuits whose tableaus take the same number of CTAs per
  // SM run in a persistent launch of their own, shaped for them (threads,
  // shared memory, CTAs).  In the batch's graph each class's launch follows
  // the control memset and starts as soon as every CTA of the class before it
  // is running (largest tableaus first), so its CTAs take the SMs that the
  // earlier classes leave as their queues run dry: no class waits for the
  // tail of the one before.
  struct Class {
    int lo_n = 0, max_n = 0;         // qubit range of the class
    int item_begin = 0, item_end = 0;
    int threads = kBatchDefaultThreads;  // CTA shape (tab_batch_tune sets it per class)
    size_t smem = 0;
    int ctas = 1;
    BatchArgs args{};
    cudaGraphNode_t knode = nullptr;
  };
  std::vector<Class> cls;
  std::vector<int32_t> ccls;  // per circuit: its class
  // device
  void* dmem = nullptr;
  BatchArgs args{};     // fields shared by the classes' launches
  void* ctl = nullptr;  // error word, queue counters, ready flags (zeroed per run)
  size_t ctl_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  unsigned long long* workc = nullptr;  // work counters (tab_batch_count_work), 4 words
};

namespace {

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }
int configure(tab_batch_s* B, int k, int threads);

// CTA size a class starts with (before tab_batch_tune): about one thread per
// two tableau words of a 32-qubit group, 128 .. 512.
int default_threads(int max_n) { return max_n <= 128 ? 128 : max_n <= 256 ? 256 : 512; }

// Shared memory a batch kernel CTA of `threads` may take (the device's opt-in
// maximum less a margin for the kernel's static shared memory).
constexpr size_t kBatchSmemLimit = 227 * 1024 - 2048;

// One circuit of a batch: extended ops lowered (MX / MY as in tab_apply;
// noise ops kept, drawn per shot on the device), then compiled into ASAP
// layers.  The shared prefix -- gates run once per circuit, before any shot
// -- ends at the first measurement or noise op, so a circuit with noise
// compiles its prefix and the rest apart.  *prefix: 1 if the program's first
// segment is that prefix.
// A word array left uninitialized on allocation (std::vector would zero it).
struct RawWords {
  std::unique_ptr<uint32_t[]> p;
  size_t n;
  explicit RawWords(size_t count) : p(new uint32_t[count]), n(count) {}
  uint32_t* data() { return p.get(); }
  uint32_t* begin() { return p.get(); }
  size_t size() const { return n; }
  bool empty() const { return n == 0; }
  uint32_t& operator[](size_t i) { return p[i]; }
};

int compile_circuit(const tab_circuit& tc, std::vector<tab_gate>& low, HostProgram& hp,
                    uint8_t* prefix) {
  int64_t ext = 0;
  int rc = validate_program(tc.n, tc.gates, tc.n_gates, &ext);
  if (rc != TAB_OK) return rc;
  const tab_gate* g = tc.gates;
  int64_t count = tc.n_gates;
  bool noise = false;
  if (ext) {
    rc = lower_for_runs(tc.n, tc.gates, tc.n_gates, true, 0, 0, 0, low);
    if (rc != TAB_OK) return rc;
    g = low.data();
    count = (int64_t)low.size();
    for (int64_t i = 0; i < count && !noise; ++i) {
      const uint32_t op = (uint32_t)(g[i] >> 56);
      noise = op == TAB_DEPOL1 || op == TAB_XERR || op == TAB_ZERR;
    }
  }
  if (!noise) {
    // a list with no extended ops was validated above; a lowered list is
    // checked again on its way in
    rc = ext ? build_program(tc.n, g, count, &hp) : build_validated(tc.n, g, count, &hp, kProgLayers);
    *prefix = (!hp.segs.empty() && hp.segs[0].kind == 0) ? 1 : 0;
    return rc;
  }
  int64_t cut = 0;
  while (cut < count) {
    const uint32_t op = (uint32_t)(g[cut] >> 56);
    if (op == TAB_MZ || op == TAB_MZR || op == TAB_DEPOL1 || op == TAB_XERR || op == TAB_ZERR) break;
    ++cut;
  }
  HostProgram part[2];
  rc = build_program(tc.n, g, cut, &part[0]);
  if (rc == TAB_OK) rc = build_program(tc.n, g + cut, count - cut, &part[1], kProgLayers | kProgNoise);
  if (rc != TAB_OK) return rc;
  if (part[1].noise.size() > 0x3FFFu) {
    set_error("more than %u noise ops in one circuit", 0x3FFFu);
    return TAB_ERANGE;
  }
  concat_programs(hp, part, 2);
  *prefix = part[0].segs.empty() ? 0 : 1;
  return TAB_OK;
}

int build_batch(const tab_circuit* circuits, int32_t m, const int64_t* out_offsets,
                tab_batch_s* B) {
  if (m < 0 || (m > 0 && !circuits)) {
    set_error("bad circuit array");
    return TAB_EINVAL;
  }
  for (int32_t c = 0; c < m; ++c) {
    const tab_circuit& tc = circuits[c];
    if (tc.n < 1 || tc.n > TAB_BATCH_MAX_QUBITS) {
      set_error("circuit %d: n=%d outside [1, %d]", c, tc.n, TAB_BATCH_MAX_QUBITS);
      return TAB_ERANGE;
    }
    if (tc.shots < 1) {
      set_error("circuit %d: shots=%d < 1", c, tc.shots);
      return TAB_EINVAL;
    }
  }
  // ---- compile every circuit on the host pool (circuits claimed one at a
  // time: their sizes differ by orders of magnitude); the error message is
  // per thread, so a failing circuit keeps its own
  std::vector<HostProgram> progs((size_t)m);
  std::vector<int> rcs((size_t)m, TAB_OK);
  std::vector<uint8_t> prefix((size_t)m, 0);
  std::vector<std::string> msgs((size_t)m);
  {
    std::atomic<int> next{0};
    pool_run(pool_threads(), [&](int) {
      std::vector<tab_gate> low;
      for (;;) {
        const int c = next.fetch_add(1);
        if (c >= m) break;
        const tab_circuit& tc = circuits[c];
        HostProgram& hp = progs[(size_t)c];
        int rc = compile_circuit(tc, low, hp, &prefix[(size_t)c]);
        rcs[(size_t)c] = rc;
        if (rc != TAB_OK) msgs[(size_t)c] = tab_last_error();
      }
    });
  }
  for (int32_t c = 0; c < m; ++c)
    if (rcs[(size_t)c] != TAB_OK) {
      set_error("circuit %d: %s", c, msgs[(size_t)c].c_str());
      return rcs[(size_t)c];
    }
  // ---- offsets of each circuit in the concatenated tables (in order)
  std::vector<size_t> o_ops((size_t)m + 1, 0), o_lo((size_t)m + 1, 0), o_seg((size_t)m + 1, 0);
  for (int32_t c = 0; c < m; ++c) {
    const HostProgram& hp = progs[(size_t)c];
    o_ops[(size_t)c + 1] = o_ops[(size_t)c] + hp.ops.size();
    o_lo[(size_t)c + 1] = o_lo[(size_t)c] + hp.layer_off.size();
    o_seg[(size_t)c + 1] = o_seg[(size_t)c] + hp.segs.size();
  }
  // the concatenated tables are written in full by the parallel fill below,
  // so they are allocated without the serial zeroing of a std::vector
  RawWords ops(o_ops[(size_t)m]), layer_off(o_lo[(size_t)m]);
  std::vector<uint32_t> noise;
  std::vector<Seg> segs(o_seg[(size_t)m]);
  std::vector<BatchCirc> circs((size_t)m);
  std::vector<double> pre_cost((size_t)m), shot_cost((size_t)m);
  uint64_t img_words = 0, noise_words = 0;
  int64_t out_packed = 0, out_max = 0;
  for (int32_t c = 0; c < m; ++c) {
    const tab_circuit& tc = circuits[c];
    const HostProgram& hp = progs[(size_t)c];
    BatchCirc& bc = circs[(size_t)c];
    bc.n = tc.n;
    bc.shots = tc.shots;
    bc.seg_begin = (uint32_t)o_seg[(size_t)c];
    bc.seg_end = (uint32_t)o_seg[(size_t)c + 1];
    bc.n_prefix = prefix[(size_t)c];
    bc.n_noise = (uint32_t)hp.noise.size();
    bc.noise_off = noise_words;
    noise_words += hp.noise.size();
    bc.n_meas = (uint32_t)hp.n_meas;
    bc.cid = tc.circuit_id;
    bc.img_off = img_words;
    img_words += sct_image_words(tc.n);
    // terminal measurements only (one MZ run after the gates): the sampler
    // runs them once and evaluates every shot from the outcome forms
    bc.sampled = 0;
    if (B->sample && hp.n_meas > 0 && hp.noise.empty() &&
        hp.segs.size() == (size_t)bc.n_prefix + 1 &&
        hp.segs.back().kind == 1) {
      const Seg& ms = hp.segs.back();
      bool mz = true;
      for (uint32_t i = ms.op_begin; i < ms.op_end && mz; ++i) mz = dop(hp.ops[i]) == OP_MZ;
      const size_t K = (size_t)hp.n_meas, FW = (K + 31) / 32;
      if (mz && K * (1 + FW) <= sct_image_words(tc.n) &&
          sct_smem_bytes(tc.n, 1024) + sct_sampler_bytes(tc.n, (int)K, tc.shots) <= kBatchSmemLimit)
        bc.sampled = 1;
    }
    B->nsampled += (int)bc.sampled;
    B->cn.push_back(tc.n);
    B->ck.push_back((int32_t)hp.n_meas);
    B->cshots.push_back(tc.shots);
    B->cnoise.push_back((int32_t)hp.noise.size());
    B->csampled.push_back((uint8_t)bc.sampled);
    const int64_t span = (int64_t)tc.shots * hp.n_meas;
    bc.out_off = (uint64_t)(out_offsets ? out_offsets[c] : out_packed);
    out_packed += span;
    out_max = std::max<int64_t>(out_max, (int64_t)bc.out_off + span);
    double pre = 0, rest = 0;
    const double wc = 2.0 * ((tc.n + 31) / 32);
    for (size_t i = 0; i < hp.segs.size(); ++i) {
      const Seg& s = hp.segs[i];
      const double len = (double)(s.op_end - s.op_begin);
      if (s.kind == 0) (i == 0 && bc.n_prefix ? pre : rest) += len * wc + (s.layer_end - s.layer_begin) * 8.0;
      else rest += len * (double)tc.n * wc;
    }
    // a sampled circuit is one item: prefix, one terminal pass, every shot
    pre_cost[(size_t)c] = bc.sampled ? pre + rest + (double)tc.shots * hp.n_meas : pre;
    shot_cost[(size_t)c] = rest;
    B->n_gates += hp.n_gates;
    B->n_meas += span;
    B->max_n = std::max(B->max_n, tc.n);
  }
  noise.resize(noise_words);
  // ---- fill the concatenated tables, circuits in parallel
  {
    std::atomic<int> next{0};
    pool_run(pool_threads(), [&](int) {
      for (;;) {
        const int c = next.fetch_add(1);
        if (c >= m) break;
        HostProgram& hp = progs[(size_t)c];
        const uint32_t op_base = (uint32_t)o_ops[(size_t)c], lo_base = (uint32_t)o_lo[(size_t)c];
        std::copy(hp.ops.begin(), hp.ops.end(), ops.begin() + (ptrdiff_t)op_base);
        std::copy(hp.noise.begin(), hp.noise.end(),
                  noise.begin() + (ptrdiff_t)circs[(size_t)c].noise_off);
        for (size_t i = 0; i < hp.layer_off.size(); ++i)
          layer_off[lo_base + i] = hp.layer_off[i] + op_base;
        for (size_t i = 0; i < hp.segs.size(); ++i) {
          Seg sg = hp.segs[i];
          sg.op_begin += op_base;
          sg.op_end += op_base;
          sg.layer_begin += lo_base;
          sg.layer_end += lo_base;
          segs[o_seg[(size_t)c] + i] = sg;
        }
        hp = HostProgram();  // release this circuit's arrays
      }
    });
  }
  B->m = m;
  B->out_bytes = out_max;
  // ---- size classes: 32-qubit groups (one tableau word per 32 qubits, so
  // one shared-memory footprint per group) merged while they take the same
  // CTAs per SM at their default CTA size; the largest first
  {
    std::vector<int> occ_of(TAB_BATCH_MAX_QUBITS / 32 + 2, 0);
    for (int g = 1; g <= TAB_BATCH_MAX_QUBITS / 32; ++g) {
      const int nn = 32 * g, T = default_threads(nn);
      occ_of[(size_t)g] = batch_ctas_per_sm(T, sct_smem_bytes(nn, T));
    }
    int top = 0;
    for (int32_t c = 0; c < m; ++c) top = std::max(top, (circuits[c].n + 31) / 32);
    B->ccls.assign((size_t)m, 0);
    std::vector<int> cls_of_group((size_t)top + 1, -1);
    for (int g = top; g >= 1; --g) {
      if (B->cls.empty() || occ_of[(size_t)g] != occ_of[(size_t)(B->cls.back().lo_n + 31) / 32] ||
          default_threads(32 * g) != default_threads(B->cls.back().max_n)) {
        tab_batch_s::Class k;
        k.max_n = 32 * g;
        B->cls.push_back(k);
      }
      B->cls.back().lo_n = 32 * (g - 1) + 1;
      cls_of_group[(size_t)g] = (int)B->cls.size() - 1;
    }
    for (int32_t c = 0; c < m; ++c) B->ccls[(size_t)c] = cls_of_group[(size_t)((circuits[c].n + 31) / 32)];
    for (auto& k : B->cls) k.threads = default_threads(k.max_n);
  }
  // ---- work items per class, longest first within each: the class's
  // prefix items, then its shot items (grouped per circuit)
  std::vector<uint64_t> items;
  std::vector<int32_t> order((size_t)m);
  std::iota(order.begin(), order.end(), 0);
  std::vector<int32_t> by_pre = order, by_shot = order;
  std::stable_sort(by_pre.begin(), by_pre.end(),
                   [&](int32_t a, int32_t b) { return pre_cost[(size_t)a] > pre_cost[(size_t)b]; });
  std::stable_sort(by_shot.begin(), by_shot.end(),
                   [&](int32_t a, int32_t b) { return shot_cost[(size_t)a] > shot_cost[(size_t)b]; });
  for (size_t k = 0; k < B->cls.size(); ++k) {
    B->cls[k].item_begin = (int)items.size();
    for (int32_t c : by_pre)
      if (B->ccls[(size_t)c] == (int32_t)k) items.push_back((uint64_t)(uint32_t)c | (0xFFFFFFFFull << 32));
    for (int32_t c : by_shot) {
      if (B->ccls[(size_t)c] != (int32_t)k || circs[(size_t)c].n_meas == 0 || circs[(size_t)c].sampled)
        continue;
      for (int32_t s = 0; s < circs[(size_t)c].shots; ++s)
        items.push_back((uint64_t)(uint32_t)c | ((uint64_t)(uint32_t)s << 32));
    }
    B->cls[k].item_end = (int)items.size();
  }
  B->nitems = (int)items.size();
  // ---- device image: one allocation
  const size_t b_circs = a256(circs.size() * sizeof(BatchCirc) + 1);
  const size_t b_segs = a256(segs.size() * sizeof(Seg) + 1);
  const size_t b_ops = a256(ops.size() * 4 + 4);
  const size_t b_lo = a256(layer_off.size() * 4 + 4);
  const size_t b_items = a256(items.size() * 8 + 8);
  const size_t b_img = a256(img_words * 4 + 16);
  const size_t b_noise = a256(noise.size() * 4 + 4);
  const size_t q_bytes = ((B->cls.size() * 4) + 15) & ~(size_t)15;  // queue counters
  B->ctl_bytes = a256(16 + q_bytes + (size_t)m * 4 + 4);
  const size_t total = b_circs + b_segs + b_ops + b_lo + b_items + b_img + b_noise + B->ctl_bytes;
  B->h2d_bytes = (int64_t)(circs.size() * sizeof(BatchCirc) + segs.size() * sizeof(Seg) +
                           ops.size() * 4 + layer_off.size() * 4 + items.size() * 8 +
                           noise.size() * 4);
  if (cudaMalloc(&B->dmem, total) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %zu bytes for the batch failed", total);
    return TAB_ENOMEM;
  }
  char* p = static_cast<char*>(B->dmem);
  BatchArgs& A = B->args;
  A.circs = reinterpret_cast<const BatchCirc*>(p);
  CUB(cudaMemcpy(p, circs.data(), circs.size() * sizeof(BatchCirc), cudaMemcpyHostToDevice));
  p += b_circs;
  A.segs = reinterpret_cast<const Seg*>(p);
  if (!segs.empty()) CUB(cudaMemcpy(p, segs.data(), segs.size() * sizeof(Seg), cudaMemcpyHostToDevice));
  p += b_segs;
  A.ops = reinterpret_cast<const uint32_t*>(p);
  if (!ops.empty()) CUB(cudaMemcpy(p, ops.data(), ops.size() * 4, cudaMemcpyHostToDevice));
  p += b_ops;
  A.layer_off = reinterpret_cast<const uint32_t*>(p);
  if (!layer_off.empty())
    CUB(cudaMemcpy(p, layer_off.data(), layer_off.size() * 4, cudaMemcpyHostToDevice));
  p += b_lo;
  A.items = reinterpret_cast<const uint64_t*>(p);
  if (!items.empty()) CUB(cudaMemcpy(p, items.data(), items.size() * 8, cudaMemcpyHostToDevice));
  p += b_items;
  A.img = reinterpret_cast<uint32_t*>(p);
  p += b_img;
  A.noise = reinterpret_cast<const uint32_t*>(p);
  if (!noise.empty()) CUB(cudaMemcpy(p, noise.data(), noise.size() * 4, cudaMemcpyHostToDevice));
  p += b_noise;
  B->ctl = p;
  A.err = reinterpret_cast<int*>(p);
  A.ready = reinterpret_cast<int*>(p + 16 + q_bytes);
  A.ncirc = (int)circs.size();
  int dev = 0;
  CUB(cudaGetDevice(&dev));
  CUB(cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev));
  for (size_t k = 0; k < B->cls.size(); ++k) {
    tab_batch_s::Class& K = B->cls[k];
    K.args = A;
    K.args.items = A.items + K.item_begin;
    K.args.nitems = K.item_end - K.item_begin;
    K.args.queue = reinterpret_cast<unsigned int*>(p + 16) + k;
    const int rc = configure(B, (int)k, K.threads);
    if (rc != TAB_OK) return rc;
  }
  return TAB_OK;
}

// CTA shape of class k's persistent launch: `threads` per CTA, shared memory
// for the class's largest tableau (with a shot's noise draws or a sampled
// circuit's forms), and as many CTAs as fit on the GPU at once.
int configure(tab_batch_s* B, int k, int threads) {
  tab_batch_s::Class& K = B->cls[(size_t)k];
  size_t smem = sct_smem_bytes(K.max_n, threads);
  for (size_t c = 0; c < B->cn.size(); ++c) {
    if (B->ccls[c] != k) continue;
    if (B->cnoise[c])  // a shot's noise draws follow its tableau
      smem = std::max(smem, sct_smem_bytes(B->cn[c], threads) + (((size_t)B->cnoise[c] + 3) & ~(size_t)3));
    if (B->csampled[c])
      smem = std::max(smem, sct_smem_bytes(B->cn[c], threads) +
                                sct_sampler_bytes(B->cn[c], B->ck[c], B->cshots[c]));
  }
  const int occ = batch_ctas_per_sm(threads, smem);
  if (occ <= 0) {
    set_error("the batched kernel does not launch with %d threads", threads);
    return TAB_ECUDA;
  }
  K.threads = threads;
  K.smem = smem;
  K.ctas = std::max(1, std::min(std::max(K.args.nitems, 1), B->sms * occ));
  return TAB_OK;
}

int make_graph(tab_batch_s* B) {
  CUB(cudaGraphCreate(&B->graph, 0));
  cudaMemsetParams mp{};
  mp.dst = B->ctl;
  mp.value = 0;
  mp.elementSize = 1;
  mp.width = B->ctl_bytes;
  mp.height = 1;
  mp.pitch = 0;
  cudaGraphNode_t mset, prev = nullptr;
  CUB(cudaGraphAddMemsetNode(&mset, B->graph, nullptr, 0, &mp));
  for (auto& K : B->cls) {
    if (K.args.nitems == 0) {
      K.knode = nullptr;
      continue;
    }
    void* kargs[] = {&K.args};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(batch_kernel_ptr(K.threads));
    kp.gridDim = dim3(K.ctas);
    kp.blockDim = dim3(K.threads);
    kp.sharedMemBytes = (unsigned)K.smem;
    kp.kernelParams = kargs;
    CUB(cudaGraphAddKernelNode(&K.knode, B->graph, &mset, 1, &kp));
    if (prev) {  // launches once every CTA of the class before it has begun
      cudaGraphEdgeData ed{};
      ed.from_port = cudaGraphKernelNodePortLaunchCompletion;
      ed.type = cudaGraphDependencyTypeProgrammatic;
      CUB(cudaGraphAddDependencies(B->graph, &prev, &K.knode, &ed, 1));
    }
    prev = K.knode;
  }
  CUB(cudaGraphInstantiate(&B->gexec, B->graph, 0));
  return TAB_OK;
}

// Kernel attributes of every class's CTA shape.
int prepare_classes(tab_batch_s* B) {
  for (const auto& K : B->cls)
    if (prepare_batch_kernel(K.threads) != cudaSuccess) {
      set_error("kernel attribute setup failed");
      return TAB_ECUDA;
    }
  return TAB_OK;
}

}  // namespace

extern "C" {

int tab_batch_create(const tab_circuit* circuits, int32_t m, tab_batch_t* out) {
  return tab_batch_create_ex(circuits, m, 0u, out);
}

int tab_batch_create_ex(const tab_circuit* circuits, int32_t m, uint32_t flags,
                        tab_batch_t* out) {
  if (!out) {
    set_error("null output pointer");
    return TAB_EINVAL;
  }
  if (flags & ~(uint32_t)TAB_BATCH_SAMPLE_TERMINAL) {
    set_error("unknown batch flags 0x%x", flags);
    return TAB_EINVAL;
  }
  *out = nullptr;
  tab_batch_s* B = new (std::nothrow) tab_batch_s();
  if (!B) {
    set_error("host allocation failed");
    return TAB_ENOMEM;
  }
  B->sample = (flags & TAB_BATCH_SAMPLE_TERMINAL) != 0;
  int rc = build_batch(circuits, m, nullptr, B);
  if (rc == TAB_OK) rc = prepare_classes(B);
  if (rc != TAB_OK) {
    tab_batch_destroy(B);
    return rc;
  }
  *out = B;
  return TAB_OK;
}

int tab_batch_destroy(tab_batch_t B) {
  if (!B) return TAB_OK;
  cudaDeviceSynchronize();
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->dmem) cudaFree(B->dmem);
  if (B->workc) cudaFree(B->workc);
  delete B;
  return TAB_OK;
}

int tab_batch_count_work(tab_batch_t B, int32_t on) {
  if (!B) {
    set_error("null batch");
    return TAB_EINVAL;
  }
  if (on && !B->workc) {
    void* p = nullptr;
    if (cudaMalloc(&p, 4 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc of the work counters failed");
      return TAB_ENOMEM;
    }
    B->workc = static_cast<unsigned long long*>(p);
  }
  if (on) CUB(cudaMemset(B->workc, 0, 4 * sizeof(unsigned long long)));
  unsigned long long* w = on ? B->workc : nullptr;
  B->args.work = w;
  for (auto& K : B->cls) K.args.work = w;
  return TAB_OK;
}

int tab_batch_work_counts(tab_batch_t B, int64_t* counts) {
  if (!B || !counts) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  unsigned long long v[4] = {0ull, 0ull, 0ull, 0ull};
  if (B->workc) CUB(cudaMemcpy(v, B->workc, sizeof v, cudaMemcpyDeviceToHost));
  for (int i = 0; i < 4; ++i) counts[i] = (int64_t)v[i];
  return TAB_OK;
}

int tab_batch_info(tab_batch_t B, int64_t* n_gates, int64_t* n_meas, int64_t* out_bytes) {
  if (!B) {
    set_error("null batch");
    return TAB_EINVAL;
  }
  if (n_gates) *n_gates = B->n_gates;
  if (n_meas) *n_meas = B->n_meas;
  if (out_bytes) *out_bytes = B->out_bytes;
  return TAB_OK;
}

int tab_batch_h2d_bytes(tab_batch_t B, int64_t* bytes) {
  if (!B || !bytes) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  *bytes = B->h2d_bytes;
  return TAB_OK;
}

int tab_batch_launches(tab_batch_t B, int64_t* count) {
  if (!B || !count) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  int64_t n = 0;
  for (const auto& K : B->cls) n += K.args.nitems > 0;
  *count = n;
  return TAB_OK;
}

int tab_batch_exec(tab_batch_t B, uint64_t seed, uint8_t* dev_out, void* cuda_stream) {
  tab::TraceRange trace_("tab_batch_exec");
  if (!B) {
    set_error("null batch");
    return TAB_EINVAL;
  }
  if (B->out_bytes > 0 && !dev_out) {
    set_error("null output buffer");
    return TAB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  B->args.seed = seed;
  B->args.out = dev_out;
  for (auto& K : B->cls) {
    K.args.seed = seed;
    K.args.out = dev_out;
  }
  if (B->args.work) {  // counting: the counting instances, one class after another
    CUB(cudaMemsetAsync(B->ctl, 0, B->ctl_bytes, st));
    for (auto& K : B->cls) {
      if (K.args.nitems == 0) continue;
      void* kargs[] = {&K.args};
      CUB(cudaLaunchKernel(batch_kernel_ptr(K.threads, true), dim3(K.ctas), dim3(K.threads), kargs,
                           K.smem, st));
    }
    return TAB_OK;
  }
  if (!B->gexec) {
    int rc = make_graph(B);
    if (rc != TAB_OK) return rc;
  } else {
    for (auto& K : B->cls) {
      if (!K.knode) continue;
      void* kargs[] = {&K.args};
      cudaKernelNodeParams kp{};
      kp.func = const_cast<void*>(batch_kernel_ptr(K.threads));
      kp.gridDim = dim3(K.ctas);
      kp.blockDim = dim3(K.threads);
      kp.sharedMemBytes = (unsigned)K.smem;
      kp.kernelParams = kargs;
      CUB(cudaGraphExecKernelNodeSetParams(B->gexec, K.knode, &kp));
    }
  }
  CUB(cudaGraphLaunch(B->gexec, st));
  return TAB_OK;
}

}  // extern "C"

static int batch_error(tab_batch_t B, void* cuda_stream) {
  int err = 0;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  CUB(cudaMemcpyAsync(&err, B->args.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUB(cudaStreamSynchronize(st));
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

extern "C" {

int tab_meas_counts(const tab_circuit* circuits, int32_t m, int64_t* counts) {
  if (m < 0 || (m > 0 && (!circuits || !counts))) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  std::atomic<int> next{0};
  pool_run(pool_threads(), [&](int) {
    for (;;) {
      const int c = next.fetch_add(1);
      if (c >= m) break;
      const tab_gate* g = circuits[c].gates;
      int64_t nm = 0;
      for (int64_t i = 0; g && i < circuits[c].n_gates; ++i) {
        const uint32_t op = (uint32_t)(g[i] >> 56);
        nm += (op == TAB_MZ) | (op == TAB_MZR) | (op == TAB_MX) | (op == TAB_MY);
      }
      counts[c] = nm;
    }
  });
  return TAB_OK;
}

int tab_batch_meas_counts(tab_batch_t B, int64_t* counts) {
  if (!B || !counts) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  for (size_t c = 0; c < B->ck.size(); ++c) counts[c] = B->ck[c];
  return TAB_OK;
}

}  // extern "C"

// tab_batch_run's default chunking of large lists: chunks, and the share
// of the gates in the first (measured on the 4,096-circuit family with the
// box's 16 host cores: 0.1 of the gates in the first of 5 chunks ran end to
// end in 401 ms, four equal chunks in 443-577 ms, 0.12 / 0.06 of 4 chunks
// in 415 / 422 ms).
constexpr int kAutoChunks = 5;
constexpr double kFirstChunkShare = 0.1;

// tab_batch_run and tab_batch_run_packed: out_offsets (caller's layout) or
// packed output; with packed output, `capacity` (< 0: unchecked) bounds the
// bytes written and counts (optional) receives every circuit's n_meas.
static int batch_run(const tab_circuit* circuits, int32_t m, uint64_t seed, uint8_t* out_bits,
                     const int64_t* out_offsets, int64_t capacity, int64_t* counts_out) {
  if (m < 0 || (m > 0 && !circuits)) {
    set_error("bad circuit array");
    return TAB_EINVAL;
  }
  int64_t gates = 0;
  for (int32_t c = 0; c < m; ++c) gates += std::max<int64_t>(circuits[c].n_gates, 0);
  // Contiguous chunks of about equal gate count, compiled in order on the
  // host pool and launched on two streams in turn: the device runs chunk k
  // (and the tail of chunk k-1) while the host compiles chunk k+1.
  const int cfg_chunks = run_config().batch_chunks;
  // By default large lists take kAutoChunks chunks, the first of them a
  // small one (its compile is the part the device cannot overlap); a
  // configured count cuts equal chunks.
  int K = cfg_chunks > 0 ? cfg_chunks
                         : (m >= 256 && gates >= ((int64_t)1 << 24)) ? kAutoChunks : 1;
  K = std::max(1, std::min(K, m));
  // chunk boundaries by gate count: chunk 0 takes first_share of the gates,
  // the others equal parts of the rest
  const double first_share = K <= 1 ? 1.0 : cfg_chunks > 0 ? 1.0 / K : kFirstChunkShare;
  const std::vector<int32_t> cut = batch_chunk_cuts(circuits, m, K, first_share);
  // Output.  Caller's offsets: one device buffer spanning them all (sized
  // from the measurement counts first), spans copied back at the end.
  // Packed: each chunk's outcomes are packed in a device buffer of its own
  // and copied to the next free bytes of out_bits behind the chunk's launch
  // (pinned out_bits) or after the last launch (pageable).
  int rc = TAB_OK;
  std::vector<int64_t> counts, offs;
  int64_t out_end = 0;
  if (out_offsets) {
    counts.assign((size_t)m + 1, 0);
    offs.assign((size_t)m + 1, 0);
    rc = tab_meas_counts(circuits, m, counts.data());
    if (rc != TAB_OK) return rc;
    for (int32_t c = 0; c < m; ++c) {
      const int64_t span = counts[(size_t)c] * std::max(circuits[c].shots, 0);
      offs[(size_t)c] = out_offsets[c];
      out_end = std::max(out_end, offs[(size_t)c] + span);
    }
    if (out_end > 0 && !out_bits) {
      set_error("null output buffer");
      return TAB_EINVAL;
    }
  }
  bool pinned = false;
  if (out_bits) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, out_bits) == cudaSuccess)
      pinned = pa.type == cudaMemoryTypeHost;
    cudaGetLastError();
  }
  cudaStream_t st[2] = {nullptr, nullptr};
  for (auto& s : st)
    if (rc == TAB_OK && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      set_error("stream creation failed");
      rc = TAB_ECUDA;
    }
  uint8_t* dout = nullptr;
  if (rc == TAB_OK && out_end > 0 && cudaMalloc((void**)&dout, (size_t)out_end) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of %lld output bytes failed", (long long)out_end);
    rc = TAB_ENOMEM;
  }
  std::vector<tab_batch_s*> parts;
  std::vector<uint8_t*> pout;   // packed: per chunk device outcomes
  std::vector<int64_t> pbase;   // packed: where the chunk's outcomes go in out_bits
  int64_t base = 0;
  for (size_t k = 0; rc == TAB_OK && k + 1 < cut.size(); ++k) {
    const int32_t c0 = cut[k], mk = cut[k + 1] - cut[k];
    tab_batch_s* B = new (std::nothrow) tab_batch_s();
    if (!B) {
      set_error("host allocation failed");
      rc = TAB_ENOMEM;
      break;
    }
    parts.push_back(B);
    rc = build_batch(circuits + c0, mk, out_offsets ? offs.data() + c0 : nullptr, B);
    if (rc == TAB_OK) rc = prepare_classes(B);
    if (rc != TAB_OK) break;
    if (counts_out)
      for (int32_t c = 0; c < mk; ++c) counts_out[c0 + c] = B->ck[(size_t)c];
    uint8_t* dk = dout;
    if (!out_offsets) {
      dk = nullptr;
      if (B->out_bytes > 0 && !out_bits) {
        set_error("null output buffer");
        rc = TAB_EINVAL;
        break;
      }
      if (capacity >= 0 && base + B->out_bytes > capacity) {
        set_error("the outcomes of circuits 0..%d take %lld bytes, more than the %lld given",
                  cut[k + 1] - 1, (long long)(base + B->out_bytes), (long long)capacity);
        rc = TAB_ERANGE;
        break;
      }
      if (B->out_bytes > 0 && cudaMalloc((void**)&dk, (size_t)B->out_bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %lld output bytes failed", (long long)B->out_bytes);
        rc = TAB_ENOMEM;
        break;
      }
      pout.push_back(dk);
      pbase.push_back(base);
    }
    cudaStream_t s = st[k & 1];
    rc = tab_batch_exec(B, seed, dk, s);
    if (rc == TAB_OK && !out_offsets && pinned && B->out_bytes > 0 &&
        cudaMemcpyAsync(out_bits + base, dk, (size_t)B->out_bytes, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess) {
      set_error("outcome copy failed");
      rc = TAB_ECUDA;
    }
    base += B->out_bytes;
  }
  for (cudaStream_t s : st)
    if (s && cudaStreamSynchronize(s) != cudaSuccess && rc == TAB_OK) {
      set_error("batch run failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = TAB_ECUDA;
    }
  for (tab_batch_s* B : parts)
    if (rc == TAB_OK) rc = batch_error(B, st[0]);
  if (rc == TAB_OK && out_offsets && out_end > 0) {
    // copy only the spans written, leave the rest untouched
    for (int32_t c = 0; c < m; ++c) {
      const int64_t span = counts[(size_t)c] * circuits[c].shots;
      if (span && cudaMemcpy(out_bits + offs[(size_t)c], dout + offs[(size_t)c], (size_t)span,
                             cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("outcome copy failed");
        rc = TAB_ECUDA;
        break;
      }
    }
  }
  if (rc == TAB_OK && !out_offsets && !pinned)
    for (size_t k = 0; k < pout.size() && rc == TAB_OK; ++k) {
      const int64_t bytes = parts[k]->out_bytes;
      if (bytes > 0 && cudaMemcpy(out_bits + pbase[k], pout[k], (size_t)bytes,
                                  cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("outcome copy failed");
        rc = TAB_ECUDA;
      }
    }
  if (dout) cudaFree(dout);
  for (uint8_t* p : pout)
    if (p) cudaFree(p);
  for (tab_batch_s* B : parts) tab_batch_destroy(B);
  for (cudaStream_t s : st)
    if (s) cudaStreamDestroy(s);
  return rc;
}

extern "C" {

int tab_batch_run(const tab_circuit* circuits, int32_t m, uint64_t seed, uint8_t* out_bits,
                  const int64_t* out_offsets) {
  tab::TraceRange trace_("tab_batch_run");
  return batch_run(circuits, m, seed, out_bits, out_offsets, -1, nullptr);
}

int tab_batch_run_packed(const tab_circuit* circuits, int32_t m, uint64_t seed,
                         uint8_t* out_bits, int64_t out_capacity, int64_t* counts) {
  tab::TraceRange trace_("tab_batch_run_packed");
  if (out_capacity < 0) {
    set_error("out_capacity %lld < 0", (long long)out_capacity);
    return TAB_EINVAL;
  }
  return batch_run(circuits, m, seed, out_bits, nullptr, out_capacity, counts);
}

// Autotuner: run each size class's launch alone with every CTA size the
// kernel is built for (shared memory sized to the class's largest tableau;
// as many CTAs as fit), time each run with events on `cuda_stream`, keep the
// fastest per class for later tab_batch_exec replays.  The runs write the
// same outcomes as an exec with this seed would.  *threads_out: the CTA size
// of the first (largest-qubit) class; *best_ms_out: the sum of the classes'
// best times.
int tab_batch_tune(tab_batch_t B, uint64_t seed, uint8_t* dev_out, void* cuda_stream,
                   int32_t* threads_out, float* best_ms_out) {
  if (!B) {
    set_error("null batch");
    return TAB_EINVAL;
  }
  if (B->out_bytes > 0 && !dev_out) {
    set_error("null output buffer");
    return TAB_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUB(cudaEventCreate(&e0));
  CUB(cudaEventCreate(&e1));
  int rc = TAB_OK;
  float total_ms = 0.f;
  for (size_t k = 0; k < B->cls.size() && rc == TAB_OK; ++k) {
    tab_batch_s::Class& K = B->cls[k];
    if (K.args.nitems == 0) continue;
    K.args.seed = seed;
    K.args.out = dev_out;
    int best = -1;
    float best_ms = 0.f;
    for (int threads : kBatchThreadChoices) {
      if (prepare_batch_kernel(threads) != cudaSuccess || configure(B, (int)k, threads) != TAB_OK) {
        cudaGetLastError();
        continue;
      }
      void* kargs[] = {&K.args};
      cudaError_t e = cudaMemsetAsync(B->ctl, 0, B->ctl_bytes, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess)
        e = cudaLaunchKernel(batch_kernel_ptr(threads), dim3(K.ctas), dim3(threads), kargs, K.smem,
                             st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e != cudaSuccess) {
        set_error("tuning launch failed: %s", cudaGetErrorString(e));
        rc = TAB_ECUDA;
        break;
      }
      rc = batch_error(B, cuda_stream);
      if (rc != TAB_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best < 0 || ms < best_ms) {
        best = threads;
        best_ms = ms;
      }
    }
    if (rc != TAB_OK) break;
    if (best < 0) {
      set_error("no CTA shape of the batched kernel launches for qubits %d..%d", K.lo_n, K.max_n);
      rc = TAB_ECUDA;
      break;
    }
    rc = configure(B, (int)k, best);
    total_ms += best_ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TAB_OK) return rc;
  if (B->gexec) cudaGraphExecDestroy(B->gexec);  // rebuilt with the new shapes
  if (B->graph) cudaGraphDestroy(B->graph);
  B->gexec = nullptr;
  B->graph = nullptr;
  if (threads_out) *threads_out = B->cls.empty() ? 0 : B->cls[0].threads;
  if (best_ms_out) *best_ms_out = total_ms;
  return TAB_OK;
}

int tab_batch_sampled(tab_batch_t B, int32_t* circuits) {
  if (!B || !circuits) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  *circuits = B->nsampled;
  return TAB_OK;
}

int tab_batch_config(tab_batch_t B, int32_t* threads, int32_t* ctas, int64_t* smem_bytes) {
  if (!B) {
    set_error("null batch");
    return TAB_EINVAL;
  }
  const bool any = !B->cls.empty();
  if (threads) *threads = any ? B->cls[0].threads : 0;
  if (ctas) *ctas = any ? B->cls[0].ctas : 0;
  if (smem_bytes) *smem_bytes = any ? (int64_t)B->cls[0].smem : 0;
  return TAB_OK;
}

int tab_batch_classes(tab_batch_t B, int32_t* count) {
  if (!B || !count) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  *count = (int32_t)B->cls.size();
  return TAB_OK;
}

int tab_batch_class(tab_batch_t B, int32_t k, tab_batch_class_info* out) {
  if (!B || !out) {
    set_error("null argument");
    return TAB_EINVAL;
  }
  if (k < 0 || k >= (int32_t)B->cls.size()) {
    set_error("class %d outside [0, %d)", k, (int)B->cls.size());
    return TAB_ERANGE;
  }
  const tab_batch_s::Class& K = B->cls[(size_t)k];
  out->lo_n = K.lo_n;
  out->max_n = K.max_n;
  out->threads = K.threads;
  out->ctas = K.ctas;
  out->smem_bytes = (int64_t)K.smem;
  out->items = K.item_end - K.item_begin;
  return TAB_OK;
}

}  // extern "C"
