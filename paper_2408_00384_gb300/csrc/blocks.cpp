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

// Within one super-layer, reorder each group's records so that every aligned
// window of 16 records (the records one half-warp takes together) reads its
// first qubits, and its second qubits, from as many distinct shared-memory
// bank pairs as the group allows.  The gate kernel keeps a qubit's X and Z
// words side by side (one 8-byte load per qubit, 16 bank pairs), so the key
// is qa mod 16, and qb mod 16 for two-qubit blocks.  The blocks of a
// super-layer act on disjoint qubits and commute, so any order gives the
// same tableau; groups stay contiguous.  Greedy over buckets keyed by
// (qa mod 16, qb mod 16): each window slot takes, among the residues the
// window has not used yet, the first residue with the most records left and
// then the second residue with the most records left (so the buckets drain
// evenly and the last windows are not left with one residue), else any
// record.
static void bank_order(uint2* recs, const uint32_t* group_size, int ngroups) {
  constexpr int kR = 16;  // residues (64-bit words: 16 bank pairs), window of kR records
  constexpr int kB = kR * (kR + 1);  // qb residue kR: a single-qubit block
  thread_local std::vector<uint2> tmp;
  thread_local std::vector<int32_t> next;
  int32_t head[kB];
  uint64_t row[kR];  // row[i] bit j: bucket (i, j) is not empty
  int cnt_a[kR], cnt_b[kR + 1];  // records left with each first / second residue
  uint32_t used_a = 0u, used_b = 0u;
  int slot = 0;
  size_t at = 0;
  for (int g = 0; g < ngroups; ++g) {
    const size_t size = group_size[g];
    uint2* G = recs + at;
    at += size;
    if (size == 0) continue;
    tmp.assign(G, G + size);
    next.assign(size, -1);
    for (int b = 0; b < kB; ++b) head[b] = -1;
    for (int i = 0; i < kR; ++i) row[i] = 0u;
    for (int i = 0; i < kR; ++i) cnt_a[i] = 0;
    for (int j = 0; j <= kR; ++j) cnt_b[j] = 0;
    for (size_t k = size; k-- > 0;) {
      const uint32_t qa = tmp[k].x & (kR - 1u);
      const uint32_t qb = ((tmp[k].x >> 28) & 1u) ? (tmp[k].x >> 14) & (kR - 1u) : (uint32_t)kR;
      const int b = (int)(qa * (kR + 1) + qb);
      next[k] = head[b];
      head[b] = (int32_t)k;
      row[qa] |= 1ull << qb;
      ++cnt_a[qa];
      ++cnt_b[qb];
    }
    for (size_t k = 0; k < size; ++k) {
      int pick_b = -1, best_a = -1;
      const uint64_t free_b = ((uint64_t)(~used_b) & ((1ull << kR) - 1u)) | (1ull << kR);
      for (uint32_t rows = ~used_a & ((1u << kR) - 1u); rows; rows &= rows - 1u) {
        const int i = __builtin_ctz(rows);
        if (cnt_a[i] > best_a && (row[i] & free_b)) {
          best_a = cnt_a[i];
          pick_b = i;
        }
      }
      if (pick_b >= 0) {
        const int i = pick_b;
        int best_b = -1;
        for (uint64_t m = row[i] & free_b; m; m &= m - 1u) {
          const int j = __builtin_ctzll(m);
          if (cnt_b[j] > best_b) {
            best_b = cnt_b[j];
            pick_b = i * (kR + 1) + j;
          }
        }
      }
      // no bucket fits the window: a record whose first residue is free, or
      // whose second residue is free, else any record
      for (uint32_t rows = ~used_a & ((1u << kR) - 1u); rows && pick_b < 0; rows &= rows - 1u) {
        const int i = __builtin_ctz(rows);
        if (row[i]) pick_b = i * (kR + 1) + __builtin_ctzll(row[i]);
      }
      for (int i = 0; i < kR && pick_b < 0; ++i)
        if (row[i] & free_b) pick_b = i * (kR + 1) + __builtin_ctzll(row[i] & free_b);
      for (int i = 0; i < kR && pick_b < 0; ++i)
        if (row[i]) pick_b = i * (kR + 1) + __builtin_ctzll(row[i]);
      const int32_t idx = head[pick_b];
      head[pick_b] = next[(size_t)idx];
      --cnt_a[pick_b / (kR + 1)];
      --cnt_b[pick_b % (kR + 1)];
      if (head[pick_b] < 0) row[pick_b / (kR + 1)] &= ~(1ull << (pick_b % (kR + 1)));
      G[k] = tmp[(size_t)idx];
      used_a |= 1u << (pick_b / (kR + 1));
      if (pick_b % (kR + 1) < kR) used_b |= 1u << (pick_b % (kR + 1));
      if (++slot == kR) {
        slot = 0;
        used_a = used_b = 0u;
      }
    }
  }
}

// Emit the run's blocks, grouped by super-layer and, inside one, into
// single- and two-qubit blocks (a warp of one kind takes one path), each
// group in bank order where bank_order_on.  A CNOT is stored with its
// control in register 0 (the block's two registers relabelled if needed: the
// qubits, the U and the V codes trade places; the swap flag keeps its
// meaning).  Super-layers above
// kMaxLayerOps blocks become consecutive sub-layers.  Appends to P.blk and
// P.blk_off and sets s.blk_begin / s.blk_end.
void BlockBuilder::emit(HostProgram& P, Seg& s) {
  const int kKinds = 2;
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
    key_[i] = (uint32_t)k.layer * kKinds + (k.has_b ? 1u : 0u);
    rec_[i] = make_uint2((uint32_t)k.qa | ((uint32_t)k.qb << 14) | ((uint32_t)k.has_b << 28) |
                             ((uint32_t)k.ent << 29),
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
    if (bank_order_on) bank_order(P.blk.data() + run, cnt.data() + (size_t)L * kKinds, kKinds);
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
