// blocks.cpp -- compile a gate run into two-qubit blocks for the block gate
// kernel.
//
// Rows of the tableau are independent under gates (Aaronson & Gottesman,
// PRA 70, 052328, Sec. III), so one thread can apply a whole sequence of
// gates on a qubit pair to 32 rows held in registers.  A block is
//   U_0 (x) U_1, then one entangler (none, CNOT either way, or CZ), then
//   V_0 (x) V_1, then an optional swap of the two columns on the way out,
// where U, V are single-qubit Cliffords (clifford1.h: any run of H, S, S^dag,
// X, Y, Z on one qubit is one 7-bit code).  A SWAP never costs a gate: it
// swaps which register holds which qubit for the rest of the block.
//
// Blocks are assigned to super-layers greedily, in program order:
//  * a gate on qubits that all sit in the latest block of those qubits is
//    folded into it (single-qubit gates always; an entangler if the block
//    has none yet);
//  * two single-qubit blocks (or one and an untouched qubit) that are the
//    latest on their qubits merge into one two-qubit block, at the later of
//    their super-layers -- nothing later depends on them yet;
//  * otherwise the gate opens a block one super-layer above the latest
//    blocks of its qubits.
// So per-qubit gate order is kept, and the blocks of one super-layer act on
// pairwise-disjoint qubits: a kernel may apply them in parallel.
#include <algorithm>
#include <vector>

#include "clifford1.h"
#include "tab_internal.h"

namespace tab {

// c1_compose as a table: entry [b][a] is b after a (7-bit codes)
static const uint8_t* c1_table() {
  static const std::vector<uint8_t> t = [] {
    std::vector<uint8_t> v(128 * 128);
    for (uint32_t b = 0; b < 128; ++b)
      for (uint32_t a = 0; a < 128; ++a) v[b * 128 + a] = (uint8_t)c1_compose(b, a);
    return v;
  }();
  return t.data();
}

// row of c1_table for each gate op (tab_op numbering, 4 bits)
static const uint8_t* c1_row_of_op() {
  static const std::vector<uint8_t> t = [] {
    std::vector<uint8_t> v(16);
    for (uint32_t op = 0; op < 16; ++op) v[op] = (uint8_t)c1_of_op(op);
    return v;
  }();
  return t.data();
}

void BlockBuilder::reset(int32_t n, size_t hint) {
  if (!comp_) {
    comp_ = c1_table();
    code_ = c1_row_of_op();
  }
  if ((int32_t)q_.size() < n) q_.assign((size_t)n, QSlot{-1, 0u, 0u});
  ++seg_;
  blk_.clear();
  if (hint > blk_.capacity()) blk_.reserve(hint);
}

// One gate (tab_op numbering) of the current run.
void BlockBuilder::add(uint32_t op, uint32_t a, uint32_t b) {
  auto latest = [&](uint32_t q) -> int32_t { return q_[q].stamp == seg_ ? q_[q].cur : -1; };
  auto bind = [&](uint32_t q, int32_t B, uint8_t role) { q_[q] = QSlot{B, seg_, role}; };
  auto open = [&](uint32_t qa, uint32_t qb, bool two, int32_t layer) -> int32_t {
    BlkRec k{};
    k.qa = (uint16_t)qa;
    k.qb = (uint16_t)(two ? qb : 0u);
    k.layer = layer;
    k.has_b = two;
    k.U[0] = k.U[1] = k.V[0] = k.V[1] = kC1Ident;
    blk_.push_back(k);
    const int32_t B = (int32_t)blk_.size() - 1;
    bind(qa, B, 0);
    if (two) bind(qb, B, 1);
    return B;
  };
  const bool two = op - TAB_CNOT <= (uint32_t)(TAB_SWAP - TAB_CNOT);
  if (!two) {
    const uint8_t* tab = comp_ + 128u * code_[op & 15u];
    int32_t B = latest(a);
    if (B < 0) B = open(a, 0, false, 0);
    BlkRec& k = blk_[(size_t)B];
    uint8_t* c = (k.ent ? k.V : k.U) + q_[a].role;
    *c = tab[*c];
    return;
  }
  int32_t Ba = latest(a), Bb = latest(b);
  int32_t B = -1;
  if (Ba >= 0 && Ba == Bb) {
    B = Ba;  // both qubits in one block
    if (op != TAB_SWAP && blk_[(size_t)B].ent) B = -1;
  } else {
    const bool sa = Ba < 0 || !blk_[(size_t)Ba].has_b;
    const bool sb = Bb < 0 || !blk_[(size_t)Bb].has_b;
    if (sa && sb) {  // single-qubit blocks (or untouched qubits): merge
      if (Ba >= 0 && Bb >= 0) {
        BlkRec& ka = blk_[(size_t)Ba];
        BlkRec& kb = blk_[(size_t)Bb];
        ka.qb = (uint16_t)b;
        ka.has_b = 1;
        ka.U[1] = kb.U[0];
        ka.layer = std::max(ka.layer, kb.layer);
        kb.dead = 1;
        bind(b, Ba, 1);
        B = Ba;
      } else if (Ba >= 0) {
        BlkRec& ka = blk_[(size_t)Ba];
        ka.qb = (uint16_t)b;
        ka.has_b = 1;
        bind(b, Ba, 1);
        B = Ba;
      } else if (Bb >= 0) {
        BlkRec& kb = blk_[(size_t)Bb];
        kb.qb = (uint16_t)a;
        kb.has_b = 1;
        bind(a, Bb, 1);
        B = Bb;
      } else {
        B = open(a, b, true, 0);
      }
    }
  }
  if (B < 0) {
    int32_t L = 0;
    if (Ba >= 0) L = std::max(L, blk_[(size_t)Ba].layer + 1);
    if (Bb >= 0) L = std::max(L, blk_[(size_t)Bb].layer + 1);
    B = open(a, b, true, L);
  }
  BlkRec& k = blk_[(size_t)B];
  const uint32_t ra = q_[a].role, rb = q_[b].role;
  if (op == TAB_SWAP) {  // relabel: the registers stay, the qubits trade places
    k.swp ^= 1;
    q_[a].role = rb;
    q_[b].role = ra;
  } else if (op == TAB_CNOT) {
    k.ent = 1;
    k.dir = (uint8_t)ra;  // 0: control in register 0, target in 1; 1: the reverse
  } else {
    k.ent = 2;  // CZ is symmetric
  }
}

// Within one super-layer, reorder each kind group's records so that every
// aligned window of 32 records (the records one warp takes together) reads
// its first qubits, and its second qubits, from 32 distinct shared-memory
// banks: distinct qa mod 32 and, among two-qubit blocks, distinct qb mod 32.
// The blocks of a super-layer act on disjoint qubits and commute, so any
// order gives the same tableau; groups stay contiguous (warp-uniform paths).
// Greedy: each window slot takes the first record within kScan of the
// group's remaining records that fits the window, else the next one.
static void bank_order(uint2* recs, const uint32_t* group_size, int ngroups) {
  constexpr size_t kScan = 64;
  uint32_t used_a = 0u, used_b = 0u;
  int slot = 0;
  size_t at = 0;
  for (int g = 0; g < ngroups; ++g) {
    uint2* G = recs + at;
    const size_t size = group_size[g];
    for (size_t k = 0; k < size; ++k) {
      size_t pick = k;
      for (size_t j = k; j < size && j < k + kScan; ++j) {
        const uint32_t qa = G[j].x & 31u, qb = (G[j].x >> 14) & 31u, two = (G[j].x >> 28) & 1u;
        if (!((used_a >> qa) & 1u) && !(two && ((used_b >> qb) & 1u))) {
          pick = j;
          break;
        }
      }
      std::swap(G[k], G[pick]);
      used_a |= 1u << (G[k].x & 31u);
      if ((G[k].x >> 28) & 1u) used_b |= 1u << ((G[k].x >> 14) & 31u);
      if (++slot == 32) {
        slot = 0;
        used_a = used_b = 0u;
      }
    }
    at += size;
  }
}

// Emit the run's blocks, grouped by super-layer and, inside one, by kind
// (single- or two-qubit, entangler, whether the U codes are identities, and
// the class -- identity, H, S or other -- of each V code) so that the threads
// of a warp take the same path: identity codes are skipped and H / S take
// their two-operation forms.  A CNOT is stored with its control in register
// 0 (the block's two registers relabelled if needed: the qubits, the U and
// the V codes trade places; the swap flag keeps its meaning).  Super-layers
// above kMaxLayerOps blocks become consecutive sub-layers.  Appends to P.blk
// and P.blk_off and sets s.blk_begin / s.blk_end.
void BlockBuilder::emit(HostProgram& P, Seg& s) {
  // (1q | 2q none / CNOT / CZ) x (U identity) x (V_0 class) x (V_1 class);
  // the sort key of each live block and its record are formed in one pass
  // (table lookups in place of data-dependent branches)
  const int kKinds = 128;
  static const std::vector<uint8_t> cls = [] {
    std::vector<uint8_t> v(128, 3);
    v[kC1Ident] = 0;
    v[kC1H] = 1;
    v[kC1S] = 2;
    return v;
  }();
  const size_t nb = blk_.size();
  key_.resize(nb);
  rec_.resize(nb);
  int32_t top = 0;
  size_t live = 0;
  for (size_t i = 0; i < nb; ++i) {
    BlkRec& k = blk_[i];
    if (k.dead) {
      key_[i] = UINT32_MAX;
      continue;
    }
    if (k.has_b && k.ent == 1 && k.dir == 1) {
      std::swap(k.qa, k.qb);
      std::swap(k.U[0], k.U[1]);
      std::swap(k.V[0], k.V[1]);
      k.dir = 0;
    }
    const uint32_t e = k.has_b ? 1u + k.ent : 0u;
    const uint32_t u = ((k.U[0] ^ kC1Ident) | (k.U[1] ^ kC1Ident)) != 0;
    key_[i] = (uint32_t)k.layer * kKinds + ((e * 2 + u) * 4 + cls[k.V[0]]) * 4 + cls[k.V[1]];
    rec_[i] = make_uint2((uint32_t)k.qa | ((uint32_t)k.qb << 14) | ((uint32_t)k.has_b << 28) |
                             ((uint32_t)k.ent << 29) | ((uint32_t)k.dir << 31),
                         (uint32_t)k.U[0] | ((uint32_t)k.U[1] << 7) | ((uint32_t)k.V[0] << 14) |
                             ((uint32_t)k.V[1] << 21) | ((uint32_t)k.swp << 28));
    top = std::max(top, k.layer + 1);
    ++live;
  }
  std::vector<uint32_t>& cnt = cnt_;
  cnt.assign((size_t)top * kKinds + 1, 0u);
  for (size_t i = 0; i < nb; ++i)
    if (key_[i] != UINT32_MAX) cnt[key_[i]]++;
  std::vector<uint32_t> pos(cnt.size(), 0u);
  uint32_t acc = 0;
  for (size_t i = 0; i < cnt.size(); ++i) {
    pos[i] = acc;
    acc += cnt[i];
  }
  const uint32_t base = (uint32_t)P.blk.size();
  P.blk.resize(P.blk.size() + live);
  uint2* out = P.blk.data() + base;
  for (size_t i = 0; i < nb; ++i)
    if (key_[i] != UINT32_MAX) out[pos[key_[i]]++] = rec_[i];
  s.blk_begin = (uint32_t)P.blk_off.size();
  P.blk_off.push_back(base);
  uint32_t run = base;
  for (int32_t L = 0; L < top; ++L) {
    uint32_t sz = 0;
    for (int t = 0; t < kKinds; ++t) sz += cnt[(size_t)L * kKinds + t];
    bank_order(P.blk.data() + run, cnt.data() + (size_t)L * kKinds, kKinds);
    while (sz > (uint32_t)kMaxLayerOps) {
      run += kMaxLayerOps;
      sz -= kMaxLayerOps;
      P.blk_off.push_back(run);
    }
    run += sz;
    P.blk_off.push_back(run);
  }
  s.blk_end = (uint32_t)P.blk_off.size() - 1;
  blk_.clear();
}

}  // namespace tab
