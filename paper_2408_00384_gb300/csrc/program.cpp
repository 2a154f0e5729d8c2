// program.cpp -- compile a gate list into the device program format:
// validation, split into gate / measurement segments, and ASAP layering.
//
// Gates acting on disjoint qubits commute exactly, so the conjugation they
// apply to every tableau row (AG Sec. III) is the same in any order.  ASAP
// layering gives each gate the layer 1 + max(layer of the previous gate on
// each of its qubits): per-qubit program order is kept, and the gates of one
// layer act on pairwise-disjoint qubits, so a kernel may apply them in
// parallel.  Within a layer gates are grouped by op code so that neighbouring
// threads take the same branch.  A measurement touches every row, so it ends
// the gate segment before it.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "pool.h"
#include "tab_internal.h"

namespace tab {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char* last_error() { return g_last_error.c_str(); }

// Every word of gates[begin, end) is a valid gate for n qubits (index i in
// messages is the position in the whole list).  Extended ops (TAB_MX ..
// TAB_ZERR, one-qubit) are valid only when `ext` is given; *ext then counts
// them.
static int validate(int32_t n, const tab_gate* gates, int64_t begin, int64_t end,
                    int64_t* ext = nullptr) {
  // fast pass: one flag over the whole range without data-dependent branches
  // (two-qubit ops are CNOT, CZ, SWAP = 7, 8, 9); the exact scan below runs
  // only when some word is bad, to name the first one
  uint64_t bad = 0;
  const uint64_t un = (uint64_t)n;
  for (int64_t i = begin; i < end; ++i) {
    const uint64_t g = gates[i];
    const uint64_t op = g >> 56;
    const uint64_t q1 = (g >> 28) & 0xFFFFFFFull, q2 = g & 0xFFFFFFFull;
    const uint64_t two = (uint64_t)(op - TAB_CNOT) <= (uint64_t)(TAB_SWAP - TAB_CNOT);
    bad |= (uint64_t)(op > TAB_BARRIER) | ((uint64_t)(op != TAB_BARRIER) & (uint64_t)(q1 >= un)) |
           (two & ((uint64_t)(q2 >= un) | (uint64_t)(q1 == q2)));
  }
  if (!bad) return TAB_OK;
  int64_t n_ext = 0;
  for (int64_t i = begin; i < end; ++i) {
    const uint64_t g = gates[i];
    const uint32_t op = (uint32_t)(g >> 56);
    const uint64_t q1 = (g >> 28) & 0xFFFFFFFull, q2 = g & 0xFFFFFFFull;
    if (op > TAB_BARRIER && op <= TAB_ZERR && ext != nullptr) {
      if (q1 >= (uint64_t)n) {
        set_error("gate %lld: qubit %llu >= n=%d", (long long)i, (unsigned long long)q1, n);
        return TAB_ERANGE;
      }
      ++n_ext;
      continue;
    }
    if (op > TAB_BARRIER) {
      set_error(op <= TAB_ZERR ? "gate %lld: op %u is not accepted here"
                               : "gate %lld: unknown op %u",
                (long long)i, op);
      return TAB_EINVAL;
    }
    if (op == TAB_BARRIER) continue;
    if (q1 >= (uint64_t)n) {
      set_error("gate %lld: qubit %llu >= n=%d", (long long)i, (unsigned long long)q1, n);
      return TAB_ERANGE;
    }
    if (op == TAB_CNOT || op == TAB_CZ || op == TAB_SWAP) {
      if (q2 >= (uint64_t)n) {
        set_error("gate %lld: qubit %llu >= n=%d", (long long)i, (unsigned long long)q2, n);
        return TAB_ERANGE;
      }
      if (q1 == q2) {
        set_error("gate %lld: two-qubit op on one qubit %llu", (long long)i,
                  (unsigned long long)q1);
        return TAB_EINVAL;
      }
    }
  }
  if (ext) *ext += n_ext;
  return TAB_OK;
}

// Compile a validated gate list into the forms `mode` names.
static int build_range(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out,
                       int mode);

void concat_programs(HostProgram& P, const HostProgram* part, size_t T, bool with_blk) {
  std::vector<size_t> o_ops(T + 1, 0), o_blk(T + 1, 0), o_loff(T + 1, 0),
      o_boff(T + 1, 0), o_segs(T + 1, 0), o_meas(T + 1, 0), o_noise(T + 1, 0);
  for (size_t t = 0; t < T; ++t) {
    o_ops[t + 1] = o_ops[t] + part[t].ops.size();
    o_blk[t + 1] = o_blk[t] + part[t].blk.size();
    o_loff[t + 1] = o_loff[t] + part[t].layer_off.size();
    o_boff[t + 1] = o_boff[t] + part[t].blk_off.size();
    o_segs[t + 1] = o_segs[t] + part[t].segs.size();
    o_meas[t + 1] = o_meas[t] + (size_t)part[t].n_meas;
    o_noise[t + 1] = o_noise[t] + part[t].noise.size();
  }
  P.clear(part[0].n);
  P.mode = part[0].mode;
  P.ops.resize(o_ops[T]);
  if (with_blk) P.blk.resize(o_blk[T]);
  P.layer_off.resize(o_loff[T]);
  P.blk_off.resize(o_boff[T]);
  P.segs.resize(o_segs[T]);
  P.noise.resize(o_noise[T]);
  for (size_t t = 0; t < T; ++t) {
    P.n_gates += part[t].n_gates;
    P.n_meas += part[t].n_meas;
  }
  pool_run((int)T, [&](int ti) {
    const size_t t = (size_t)ti;
    const HostProgram& Q = part[t];
    std::copy(Q.ops.begin(), Q.ops.end(), P.ops.begin() + (ptrdiff_t)o_ops[t]);
    std::copy(Q.noise.begin(), Q.noise.end(), P.noise.begin() + (ptrdiff_t)o_noise[t]);
    if (o_noise[t])  // noise ordinals count from the first part's first noise op
      for (size_t i = o_ops[t]; i < o_ops[t + 1]; ++i)
        if (dop(P.ops[i]) == OP_NOISE) P.ops[i] += (uint32_t)o_noise[t];
    if (with_blk) std::copy(Q.blk.begin(), Q.blk.end(), P.blk.begin() + (ptrdiff_t)o_blk[t]);
    for (size_t i = 0; i < Q.layer_off.size(); ++i)
      P.layer_off[o_loff[t] + i] = Q.layer_off[i] + (uint32_t)o_ops[t];
    for (size_t i = 0; i < Q.blk_off.size(); ++i)
      P.blk_off[o_boff[t] + i] = Q.blk_off[i] + (uint32_t)o_blk[t];
    for (size_t i = 0; i < Q.segs.size(); ++i) {
      Seg s = Q.segs[i];
      s.op_begin += (uint32_t)o_ops[t];
      s.op_end += (uint32_t)o_ops[t];
      s.layer_begin += (uint32_t)o_loff[t];
      s.layer_end += (uint32_t)o_loff[t];
      s.blk_begin += (uint32_t)o_boff[t];
      s.blk_end += (uint32_t)o_boff[t];
      s.meas_before += (uint32_t)o_meas[t];
      P.segs[o_segs[t] + i] = s;
    }
  });
}

int validate_program(int32_t n, const tab_gate* gates, int64_t count, int64_t* ext) {
  if (n < 1 || n > TAB_MAX_QUBITS) {
    set_error("n=%d outside [1, %d]", n, TAB_MAX_QUBITS);
    return TAB_ERANGE;
  }
  if (count < 0 || (count > 0 && gates == nullptr)) {
    set_error("bad gate list (count=%lld)", (long long)count);
    return TAB_EINVAL;
  }
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(count >> 16, pool_threads()));
  std::vector<int> rcs((size_t)T, TAB_OK);
  std::vector<int64_t> nx((size_t)T, 0);
  std::vector<std::string> msg((size_t)T);
  pool_run(T, [&](int t) {
    rcs[(size_t)t] = validate(n, gates, count * t / T, count * (t + 1) / T,
                              ext ? &nx[(size_t)t] : nullptr);
    if (rcs[(size_t)t] != TAB_OK) msg[(size_t)t] = last_error();
  });
  for (int t = 0; t < T; ++t)  // the first bad word in list order
    if (rcs[(size_t)t] != TAB_OK) {
      set_error("%s", msg[(size_t)t].c_str());
      return rcs[(size_t)t];
    }
  if (ext)
    for (int t = 0; t < T; ++t) *ext += nx[(size_t)t];
  return TAB_OK;
}

int build_validated(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out, int mode) {
  return build_range(n, gates, count, out, mode);
}

int build_validated_blocks(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out) {
  return build_range(n, gates, count, out, kProgBlocks);
}

int build_program(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out,
                  int mode) {
  if (n < 1 || n > TAB_MAX_QUBITS) {
    set_error("n=%d outside [1, %d]", n, TAB_MAX_QUBITS);
    return TAB_ERANGE;
  }
  if (count < 0 || (count > 0 && gates == nullptr)) {
    set_error("bad gate list (count=%lld)", (long long)count);
    return TAB_EINVAL;
  }
  // Long lists compiled to blocks only (the multi-CTA engines' per-call path)
  // are cut into chunks that the pool's threads validate and compile at once;
  // each chunk's gates become gate runs of their own, concatenated in order.
  const int64_t kChunk = 1 << 16;
  if ((mode & ~kProgBankOrder) == kProgBlocks && count >= 2 * kChunk) {
    const int T = (int)std::min<int64_t>(count / kChunk, pool_threads());
    if (T >= 2) {
      std::vector<HostProgram> part((size_t)T);
      std::vector<int> rcs((size_t)T, TAB_OK);
      std::vector<std::string> msg((size_t)T);
      pool_run(T, [&](int t) {
        const int64_t b = count * t / T, e = count * (t + 1) / T;
        int rc = validate(n, gates, b, e);
        if (rc == TAB_OK) rc = build_range(n, gates + b, e - b, &part[(size_t)t], mode);
        rcs[(size_t)t] = rc;
        if (rc != TAB_OK) msg[(size_t)t] = last_error();
      });
      for (int t = 0; t < T; ++t)
        if (rcs[(size_t)t] != TAB_OK) {
          set_error("%s", msg[(size_t)t].c_str());
          return rcs[(size_t)t];
        }
      concat_programs(*out, part.data(), part.size());
      return TAB_OK;
    }
  }
  int64_t n_ext = 0;
  const int vrc = validate(n, gates, 0, count, (mode & kProgNoise) ? &n_ext : nullptr);
  if (vrc != TAB_OK) return vrc;

  return build_range(n, gates, count, out, mode);
}

static int build_range(int32_t n, const tab_gate* gates, int64_t count, HostProgram* out,
                       int mode) {
  const bool layers = (mode & kProgLayers) != 0, blocks = (mode & kProgBlocks) != 0;
  HostProgram& P = *out;
  P.clear(n);
  P.mode = mode & (kProgLayers | kProgBlocks);
  if (layers) P.ops.reserve((size_t)count);
  // one builder per thread, kept between calls with its arrays' capacity
  static thread_local BlockBuilder bb;
  bb.bank_order_on = (mode & kProgBankOrder) != 0;
  if (blocks) {
    bb.reset(n, (size_t)count / 2 + 16);
    P.blk.reserve((size_t)count / 2 + 16);
  }
  int64_t run_gates = 0;  // gates in the open gate run
  std::vector<int64_t> last((size_t)n, -1);  // global layer of the last gate per qubit
  int64_t nlayers = 0;                       // layers emitted so far (global)
  // The open segment's gate codes with their bucket keys (layer - first
  // layer of the segment) * kOps + op, and the count per bucket, kept as the
  // gates arrive: a layer is at most one past the segment's last, so the
  // count table grows a layer at a time.
  constexpr int kOps = 13;  // device op codes 0..12
  // (plain arrays with a fill index: a segment holds at most every gate,
  // and the per-gate appends stay inline in the loop)
  std::unique_ptr<uint32_t[]> seg_buf(layers && count > 0 ? new uint32_t[2 * (size_t)count] : nullptr);
  uint32_t* const seg_codes = seg_buf.get();
  uint32_t* const seg_key = layers && count > 0 ? seg_buf.get() + count : nullptr;
  size_t nseg = 0;
  std::vector<uint32_t> cnt;

  // Each gate segment owns one contiguous run of layer_off entries:
  // layer_off[layer_begin] = op_begin, layer_off[layer_begin + L + 1] = end
  // of layer L, layer_off[layer_end] = op_end.
  auto flush_gates = [&]() {
    if (run_gates == 0) return;
    run_gates = 0;
    if (!layers) {  // blocks only: the run owns no gate codes
      Seg s{};
      s.kind = 0;
      s.op_begin = s.op_end = (uint32_t)P.ops.size();
      s.meas_before = (uint32_t)P.n_meas;
      s.layer_begin = s.layer_end = (uint32_t)P.layer_off.size();
      bb.emit(P, s);
      bb.reset(n, 0);
      P.segs.push_back(s);
      return;
    }
    // counting sort by (layer, op): layer sizes first, then the bucket
    // starts in place of the counts
    const int64_t nl = (int64_t)(cnt.size() / kOps);
    std::vector<uint32_t> lsz((size_t)nl);
    uint32_t acc = 0;
    for (int64_t L = 0; L < nl; ++L) {
      const uint32_t l0 = acc;
      for (int o = 0; o < kOps; ++o) {
        const uint32_t c = cnt[(size_t)L * kOps + o];
        cnt[(size_t)L * kOps + o] = acc;
        acc += c;
      }
      lsz[(size_t)L] = acc - l0;
    }
    const uint32_t op_base = (uint32_t)P.ops.size();
    P.ops.resize(P.ops.size() + nseg);
    uint32_t* dst = P.ops.data() + op_base;
    for (size_t i = 0; i < nseg; ++i) dst[cnt[seg_key[i]]++] = seg_codes[i];
    Seg s{};
    s.kind = 0;
    s.op_begin = op_base;
    s.op_end = op_base + (uint32_t)nseg;
    s.meas_before = (uint32_t)P.n_meas;
    s.layer_begin = (uint32_t)P.layer_off.size();
    P.layer_off.push_back(op_base);
    uint32_t run = op_base;
    for (int64_t L = 0; L < nl; ++L) {
      uint32_t sz = lsz[(size_t)L];
      // a layer larger than kMaxLayerOps becomes consecutive sub-layers (its
      // gates are pairwise disjoint, so any split keeps the result)
      while (sz > (uint32_t)kMaxLayerOps) {
        run += kMaxLayerOps;
        sz -= kMaxLayerOps;
        P.layer_off.push_back(run);
      }
      run += sz;
      P.layer_off.push_back(run);
    }
    s.layer_end = (uint32_t)P.layer_off.size() - 1;
    if (blocks) {
      bb.emit(P, s);
      bb.reset(n, 0);
    } else {
      s.blk_begin = s.blk_end = (uint32_t)P.blk_off.size();
    }
    P.segs.push_back(s);
    nlayers += nl;
    nseg = 0;
    cnt.clear();
  };

  for (int64_t i = 0; i < count; ++i) {
    const uint64_t g = gates[i];
    uint32_t op = (uint32_t)(g >> 56);
    uint32_t q1 = (uint32_t)((g >> 28) & 0xFFFFFFFull), q2 = (uint32_t)(g & 0xFFFFFFFull);
    if (op == TAB_BARRIER || op == TAB_I) continue;
    if (op > TAB_BARRIER) {
      // kProgNoise: a noise op becomes a one-qubit OP_NOISE code whose second
      // field is its ordinal (the device draws it per shot); any other
      // extended op must have been lowered already
      const bool noise = op == TAB_DEPOL1 || op == TAB_XERR || op == TAB_ZERR;
      if (!noise || !(mode & kProgNoise) || !layers || blocks || P.noise.size() > 0x3FFFu) {
        set_error("gate %lld: op %u is not accepted here", (long long)i, op);
        return TAB_EINVAL;
      }
      const uint32_t kind = op == TAB_DEPOL1 ? 0u : op == TAB_XERR ? 1u : 2u;
      P.noise.push_back(kind << 28 | (q2 & 0xFFFFFFFu));
      op = OP_NOISE;
      q2 = (uint32_t)P.noise.size() - 1u;
    }
    if (op == TAB_MZ || op == TAB_MZR) {
      flush_gates();
      if (P.segs.empty() || P.segs.back().kind != 1) {
        Seg s{};
        s.kind = 1;
        s.op_begin = s.op_end = (uint32_t)P.ops.size();
        s.meas_before = (uint32_t)P.n_meas;
        P.segs.push_back(s);
      }
      P.ops.push_back(dcode(op, q1, 0));
      P.segs.back().op_end++;
      P.n_meas++;
      continue;
    }
    const bool two = (op == TAB_CNOT || op == TAB_CZ || op == TAB_SWAP);
    ++run_gates;
    if (op != OP_NOISE) P.n_gates++;
    if (blocks) bb.add(op, q1, two ? q2 : 0);
    if (!layers) continue;
    int64_t L = std::max<int64_t>(last[q1], nlayers - 1);
    if (two) L = std::max<int64_t>(L, last[q2]);
    L += 1;
    last[q1] = L;
    if (two) last[q2] = L;
    const size_t key = (size_t)(L - nlayers) * kOps + op;
    if (key >= cnt.size()) cnt.resize(cnt.size() + kOps, 0);  // a new layer
    cnt[key]++;
    seg_codes[nseg] = dcode(op, q1, (two || op == OP_NOISE) ? q2 : 0);
    seg_key[nseg++] = (uint32_t)key;
  }
  flush_gates();
  return TAB_OK;
}

}  // namespace tab
