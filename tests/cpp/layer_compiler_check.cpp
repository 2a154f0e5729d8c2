// Host check of the layered compile (program.cpp, kProgLayers): random gate
// lists over every gate kind, with measurement runs, barriers, identities and
// (with kProgNoise) Pauli noise ops, are compiled and the result is checked
// against the list itself:
//  * segments: gate runs and measurement runs alternate as in the list, and
//    every measurement run holds the list's MZ / MZR codes in order;
//  * every gate run's codes are the list's gates of that run (BARRIER and I
//    dropped), each exactly once;
//  * the gates of one layer act on pairwise-disjoint qubits and are grouped
//    by op code (layers above kMaxLayerOps are split and keep the order);
//  * each qubit meets its gates in list order, and each gate sits in its
//    ASAP layer (one past the latest earlier gate on any of its qubits),
//    computed here independently;
//  * gate and measurement counts, noise ordinals and the noise table.
// The validated entry (build_validated) must give the same program as
// build_program.  Exit status 0 on success; prints "bad <count>".
#include <algorithm>
#include <cstdio>
#include <random>
#include <vector>
#include "tab_internal.h"
namespace tab {
const char* last_error();
}
using namespace tab;

static int bad = 0;
#define CHECK(c, ...)            \
  do {                           \
    if (!(c)) {                  \
      if (bad < 20) {            \
        printf(__VA_ARGS__);     \
        printf("\n");            \
      }                          \
      ++bad;                     \
    }                            \
  } while (0)

static tab_gate G(uint32_t op, uint32_t a, uint32_t b) {
  return (tab_gate)op << 56 | (tab_gate)a << 28 | b;
}

static bool two_qubit(uint32_t op) { return op == TAB_CNOT || op == TAB_CZ || op == TAB_SWAP; }

// The list's device op for a gate word (noise ops: OP_NOISE), or -1 when it
// is dropped (BARRIER, I) or a measurement.
static int dev_op(uint32_t op) {
  if (op == TAB_BARRIER || op == TAB_I || op == TAB_MZ || op == TAB_MZR) return -1;
  if (op == TAB_DEPOL1 || op == TAB_XERR || op == TAB_ZERR) return OP_NOISE;
  return (int)op;
}

static void check_list(int n, const std::vector<tab_gate>& g, bool noise) {
  const int mode = kProgLayers | (noise ? kProgNoise : 0);
  HostProgram P;
  int rc = build_program(n, g.data(), (int64_t)g.size(), &P, mode);
  CHECK(rc == TAB_OK, "build_program rc %d: %s", rc, last_error());
  if (rc != TAB_OK) return;
  if (!noise) {
    HostProgram Q;
    rc = build_validated(n, g.data(), (int64_t)g.size(), &Q, kProgLayers);
    CHECK(rc == TAB_OK && Q.ops == P.ops && Q.layer_off == P.layer_off && Q.segs.size() == P.segs.size(),
          "build_validated differs");
  }
  // expected runs: maximal runs of gates (dropped words ignored) and of
  // measurements, in list order
  struct Run {
    bool meas;
    std::vector<size_t> idx;  // list positions
  };
  std::vector<Run> runs;
  for (size_t i = 0; i < g.size(); ++i) {
    const uint32_t op = (uint32_t)(g[i] >> 56);
    const bool m = op == TAB_MZ || op == TAB_MZR;
    if (!m && dev_op(op) < 0) continue;
    if (runs.empty() || runs.back().meas != m) runs.push_back({m, {}});
    runs.back().idx.push_back(i);
  }
  CHECK(P.segs.size() == runs.size(), "segments %zu, runs %zu", P.segs.size(), runs.size());
  if (P.segs.size() != runs.size()) return;
  int64_t n_gates = 0, n_meas = 0, noise_seen = 0;
  for (size_t si = 0; si < runs.size(); ++si) {
    const Seg& s = P.segs[si];
    const Run& R = runs[si];
    CHECK((s.kind == 1) == R.meas, "segment %zu kind %u", si, s.kind);
    CHECK(s.meas_before == (uint32_t)n_meas, "segment %zu meas_before %u, want %lld", si,
          s.meas_before, (long long)n_meas);
    if (R.meas) {
      CHECK(s.op_end - s.op_begin == R.idx.size(), "segment %zu: %u codes for %zu measurements", si,
            s.op_end - s.op_begin, R.idx.size());
      for (size_t k = 0; k < R.idx.size() && s.op_begin + k < s.op_end; ++k) {
        const tab_gate w = g[R.idx[k]];
        const uint32_t c = P.ops[s.op_begin + k];
        CHECK(dop(c) == (uint32_t)(w >> 56) && dq1(c) == (uint32_t)((w >> 28) & 0xFFFFFFF),
              "segment %zu measurement %zu code %08x", si, k, c);
      }
      n_meas += (int64_t)R.idx.size();
      continue;
    }
    // the run's gates, their ASAP layers computed here
    std::vector<int> last(n, -1), want_layer;
    std::vector<uint32_t> want_code;
    for (size_t i : R.idx) {
      const uint32_t op = (uint32_t)(g[i] >> 56);
      const uint32_t a = (uint32_t)((g[i] >> 28) & 0xFFFFFFF), b = (uint32_t)(g[i] & 0xFFFFFFF);
      const bool two = two_qubit(op);
      int L = last[a];
      if (two) L = std::max(L, last[b]);
      ++L;
      last[a] = L;
      if (two) last[b] = L;
      want_layer.push_back(L);
      const int d = dev_op(op);
      if (d == OP_NOISE) {
        // the code's second field is the op's ordinal in the noise table
        want_code.push_back(dcode(OP_NOISE, a, (uint32_t)noise_seen));
        const uint32_t kind = op == TAB_DEPOL1 ? 0u : op == TAB_XERR ? 1u : 2u;
        CHECK((size_t)noise_seen < P.noise.size() &&
                  P.noise[(size_t)noise_seen] == (kind << 28 | (b & 0xFFFFFFFu)),
              "noise table entry %lld", (long long)noise_seen);
        ++noise_seen;
      } else {
        want_code.push_back(dcode((uint32_t)d, a, two ? b : 0u));
        ++n_gates;
      }
    }
    int depth = 0;
    for (int L : want_layer) depth = std::max(depth, L + 1);
    const uint32_t lb = s.layer_begin, le = s.layer_end;
    CHECK(P.layer_off[lb] == s.op_begin && P.layer_off[le] == s.op_end, "segment %zu layer bounds",
          si);
    CHECK(s.op_end - s.op_begin == want_code.size(), "segment %zu: %u codes for %zu gates", si,
          s.op_end - s.op_begin, want_code.size());
    // each code -> its compiled layer
    std::vector<int> got_layer(s.op_end - s.op_begin, -1);
    for (uint32_t L = lb; L < le; ++L) {
      std::vector<char> used(n, 0);
      uint32_t prev_op = 0;
      for (uint32_t i = P.layer_off[L]; i < P.layer_off[L + 1]; ++i) {
        const uint32_t c = P.ops[i], op = dop(c);
        const uint32_t a = dq1(c), b = dq2(c);
        CHECK(op >= prev_op, "segment %zu layer %u: ops not grouped", si, L);
        prev_op = op;
        CHECK(a < (uint32_t)n && !used[a], "segment %zu layer %u: qubit %u twice", si, L, a);
        if (a < (uint32_t)n) used[a] = 1;
        if (two_qubit(op)) {
          CHECK(b < (uint32_t)n && !used[b], "segment %zu layer %u: qubit %u twice", si, L, b);
          if (b < (uint32_t)n) used[b] = 1;
        }
        got_layer[i - s.op_begin] = (int)(L - lb);
      }
    }
    // multiset of codes, and per qubit the order of its gates: walk the
    // compiled codes in order and match each against the list's next
    // unmatched gate on its first qubit
    std::vector<std::vector<size_t>> per_q(n);
    for (size_t k = 0; k < want_code.size(); ++k) per_q[dq1(want_code[k])].push_back(k);
    std::vector<size_t> next_q(n, 0);
    std::vector<int> layer_of_gate(want_code.size(), -1);
    for (uint32_t i = s.op_begin; i < s.op_end; ++i) {
      const uint32_t c = P.ops[i], a = dq1(c);
      if (a >= (uint32_t)n || next_q[a] >= per_q[a].size()) {
        CHECK(false, "segment %zu: extra code %08x", si, c);
        continue;
      }
      const size_t k = per_q[a][next_q[a]++];
      CHECK(want_code[k] == c, "segment %zu: code %08x where the list has %08x", si, c,
            want_code[k]);
      layer_of_gate[k] = got_layer[i - s.op_begin];
    }
    // ASAP layers: with no layer above kMaxLayerOps codes every gate sits
    // in exactly its ASAP layer; otherwise a large layer is split into
    // consecutive sub-layers, and the compiled layer grows with the ASAP one
    std::vector<int> asap_size(depth, 0);
    for (int L : want_layer) ++asap_size[L];
    int largest = 0;
    for (int v : asap_size) largest = std::max(largest, v);
    const bool split = largest > kMaxLayerOps;
    if (!split) {
      CHECK((int)(le - lb) == depth, "segment %zu: %u layers for ASAP depth %d", si, le - lb, depth);
      for (size_t k = 0; k < want_code.size(); ++k)
        CHECK(layer_of_gate[k] == want_layer[k], "segment %zu: gate %zu in layer %d, ASAP %d", si, k,
              layer_of_gate[k], want_layer[k]);
    } else {
      for (size_t k = 0; k + 1 < want_code.size(); ++k)
        for (size_t k2 = k + 1; k2 < want_code.size() && k2 < k + 64; ++k2)
          if (want_layer[k] < want_layer[k2])
            CHECK(layer_of_gate[k] < layer_of_gate[k2],
                  "segment %zu: gates %zu, %zu out of layer order", si, k, k2);
    }
    // per qubit, the second qubit's order too
    for (size_t k = 0; k < want_code.size(); ++k) {
      const uint32_t c = want_code[k];
      if (!two_qubit(dop(c))) continue;
      for (size_t k2 = k + 1; k2 < want_code.size(); ++k2) {
        const uint32_t c2 = want_code[k2];
        const bool shares = dq1(c2) == dq2(c) || (two_qubit(dop(c2)) && dq2(c2) == dq2(c));
        if (shares) {
          CHECK(layer_of_gate[k] < layer_of_gate[k2], "segment %zu: qubit %u order", si, dq2(c));
          break;
        }
      }
    }
    CHECK((int)(le - lb) >= depth, "segment %zu: %u layers for ASAP depth %d", si, le - lb, depth);
  }
  CHECK(P.n_gates == n_gates, "n_gates %lld, want %lld", (long long)P.n_gates, (long long)n_gates);
  CHECK(P.n_meas == n_meas, "n_meas %lld, want %lld", (long long)P.n_meas, (long long)n_meas);
  CHECK((int64_t)P.noise.size() == noise_seen, "noise table %zu, want %lld", P.noise.size(),
        (long long)noise_seen);
}

int main() {
  std::mt19937_64 rng(20240801);
  const uint32_t one[] = {TAB_H, TAB_S, TAB_SDG, TAB_X, TAB_Y, TAB_Z, TAB_I, TAB_BARRIER};
  int lists = 0;
  for (int trial = 0; trial < 400; ++trial) {
    const bool noise = trial % 3 == 2;
    const int n = 1 + (int)(rng() % 200);
    const int len = (int)(rng() % 3000);
    std::vector<tab_gate> g;
    for (int i = 0; i < len; ++i) {
      const uint32_t a = (uint32_t)(rng() % n);
      const int r = (int)(rng() % 100);
      if (r < 45) {
        g.push_back(G(one[rng() % 8], a, 0));
      } else if (r < 80 && n > 1) {
        uint32_t b = (uint32_t)(rng() % (n - 1));
        if (b >= a) ++b;
        const uint32_t op = r < 65 ? TAB_CNOT : r < 75 ? TAB_CZ : TAB_SWAP;
        g.push_back(G(op, a, b));
      } else if (r < 90 && noise) {
        const uint32_t op = r < 84 ? TAB_DEPOL1 : r < 87 ? TAB_XERR : TAB_ZERR;
        g.push_back(G(op, a, (uint32_t)(rng() & 0xFFFFFFF)));
      } else {
        // a run of measurements
        const int k = 1 + (int)(rng() % 6);
        for (int j = 0; j < k; ++j)
          g.push_back(G(rng() % 2 ? TAB_MZ : TAB_MZR, (uint32_t)(rng() % n), 0));
      }
    }
    check_list(n, g, noise);
    ++lists;
  }
  // layers above kMaxLayerOps: one layer of 3000 H, then 1500 CNOTs
  {
    const int n = 3000;
    std::vector<tab_gate> g;
    for (int a = 0; a < n; ++a) g.push_back(G(TAB_H, a, 0));
    for (int a = 0; a + 1 < n; a += 2) g.push_back(G(TAB_CNOT, a, a + 1));
    g.push_back(G(TAB_MZ, 7, 0));
    check_list(n, g, false);
    HostProgram P;
    build_program(n, g.data(), (int64_t)g.size(), &P, kProgLayers);
    // 3000 H in two sub-layers (2048 + 952), then one layer of 1500 CNOTs
    const Seg& s = P.segs[0];
    CHECK(s.layer_end - s.layer_begin == 3, "split layers: %u", s.layer_end - s.layer_begin);
    CHECK(P.layer_off[s.layer_begin + 1] - P.layer_off[s.layer_begin] == (uint32_t)kMaxLayerOps,
          "first sub-layer size");
    ++lists;
  }
  printf("lists %d bad %d\n", lists, bad);
  return bad ? 1 : 0;
}
