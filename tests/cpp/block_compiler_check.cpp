// Host check of the block compiler (blocks.cpp): random gate lists over every
// gate kind are compiled into two-qubit blocks, the blocks are applied to
// random 32-row words with the block formulas of the device kernel, and the
// result must equal the gates applied one at a time with the Aaronson &
// Gottesman rules (PRA 70, 052328, Sec. III).  Each super-layer must act on
// pairwise-disjoint qubits.  The pipelined apply's host side (chunks
// compiled apart, merged without their records, adjacent gate runs taken as
// one) must give the same result.  Exit status 0 on success.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>
#include "tab_internal.h"
#include "clifford1.h"
using namespace tab;
static void c1h(uint32_t m, uint32_t& x, uint32_t& z, uint32_t& r) {
  const uint32_t al = 0u - (m & 1u), be = 0u - ((m >> 1) & 1u), ga = 0u - ((m >> 2) & 1u),
                 de = 0u - ((m >> 3) & 1u), ep = 0u - ((m >> 4) & 1u), ze = 0u - ((m >> 5) & 1u),
                 et = 0u - ((m >> 6) & 1u);
  r ^= (ep & x) ^ (ze & z) ^ (et & x & z);
  const uint32_t xn = (al & x) ^ (be & z);
  z = (ga & x) ^ (de & z);
  x = xn;
}
static void blockh(uint2 rec, std::vector<uint32_t>& sx, std::vector<uint32_t>& sz, uint32_t& r) {
  const uint32_t qa = rec.x & 0x3FFFu, qb = (rec.x >> 14) & 0x3FFFu;
  const bool two = (rec.x >> 28) & 1u;
  // emitted records keep a CNOT's control in register 0 (bit 31 is 0)
  const uint32_t ent = (rec.x >> 29) & 3u, dir = rec.x >> 31, m = rec.y;
  uint32_t x0 = sx[qa], z0 = sz[qa];
  c1h(m & 0x7F, x0, z0, r);
  if (!two) { sx[qa] = x0; sz[qa] = z0; return; }
  uint32_t x1 = sx[qb], z1 = sz[qb];
  c1h((m >> 7) & 0x7F, x1, z1, r);
  if (ent == 1) {
    uint32_t xc = dir ? x1 : x0, zc = dir ? z1 : z0, xt = dir ? x0 : x1, zt = dir ? z0 : z1;
    r ^= xc & zt & ~(xt ^ zc);
    uint32_t xt2 = xt ^ xc, zc2 = zc ^ zt;
    x0 = dir ? xt2 : xc; z0 = dir ? zt : zc2; x1 = dir ? xc : xt2; z1 = dir ? zc2 : zt;
  } else if (ent == 2) {
    r ^= x0 & x1 & (z0 ^ z1);
    uint32_t z0n = z0 ^ x1; z1 ^= x0; z0 = z0n;
  }
  c1h((m >> 14) & 0x7F, x0, z0, r);
  c1h((m >> 21) & 0x7F, x1, z1, r);
  const bool sw = (m >> 28) & 1u;
  uint32_t da = sw ? qb : qa, db = sw ? qa : qb;
  sx[da] = x0; sz[da] = z0; sx[db] = x1; sz[db] = z1;
}
// the gates one at a time: AG rules (and their products for Y, Z, S^dag, CZ)
// on 32 rows
static void gate(uint32_t op, uint32_t a, uint32_t b, std::vector<uint32_t>& X, std::vector<uint32_t>& Z, uint32_t& r) {
  uint32_t &xa = X[a], &za = Z[a];
  switch (op) {
    case TAB_X: r ^= za; break;
    case TAB_Y: r ^= xa ^ za; break;
    case TAB_Z: r ^= xa; break;
    case TAB_H: { r ^= xa & za; uint32_t t = xa; xa = za; za = t; break; }
    case TAB_S: r ^= xa & za; za ^= xa; break;
    case TAB_SDG: r ^= xa & ~za; za ^= xa; break;
    case TAB_CNOT: { uint32_t &xt = X[b], &zt = Z[b]; r ^= xa & zt & ~(xt ^ za); xt ^= xa; za ^= zt; break; }
    case TAB_CZ: { uint32_t &xb = X[b], &zb = Z[b]; r ^= xa & xb & (za ^ zb); uint32_t zan = za ^ xb; zb ^= xa; za = zan; break; }
    case TAB_SWAP: { std::swap(X[a], X[b]); std::swap(Z[a], Z[b]); break; }
  }
}
int main() {
  std::mt19937_64 rng(12345);
  int bad = 0, cases = 0;
  long long blocks = 0, gates_total = 0, layers = 0;
  for (int t = 0; t < 3000; ++t) {
    const int n = 1 + (int)(rng() % 40);
    const int ng = (int)(rng() % 300);
    std::vector<tab_gate> g;
    for (int i = 0; i < ng; ++i) {
      uint32_t op = 1 + (uint32_t)(rng() % 9);  // X..SWAP
      uint32_t a = (uint32_t)(rng() % n), b = (uint32_t)(rng() % n);
      const bool two = op >= TAB_CNOT;
      if (two && n < 2) op = TAB_H;
      if (op >= TAB_CNOT) while (b == a) b = (uint32_t)(rng() % n);
      g.push_back(tab_make_gate(op, a, op >= TAB_CNOT ? b : 0));
    }
    HostProgram hp;  // every other circuit also with the bank order of replayed programs
    const int mode = kProgBlocks | ((rng() & 1) ? kProgBankOrder : 0);
    if (build_program(n, g.data(), (int64_t)g.size(), &hp, mode) != TAB_OK) { printf("build failed\n"); return 1; }
    std::vector<uint32_t> X(n), Z(n), X2, Z2;
    for (int a = 0; a < n; ++a) { X[a] = (uint32_t)rng(); Z[a] = (uint32_t)rng(); }
    uint32_t r = (uint32_t)rng(), r2 = r;
    X2 = X; Z2 = Z;
    for (auto w : g) gate((uint32_t)(w >> 56), (uint32_t)((w >> 28) & 0xFFFFFFF), (uint32_t)(w & 0xFFFFFFF), X, Z, r);
    for (const Seg& s : hp.segs) {
      if (s.kind != 0) continue;
      for (uint32_t L = s.blk_begin; L < s.blk_end; ++L) {
        // disjointness check within a super-layer
        std::vector<int> seen(n, 0);
        for (uint32_t i = hp.blk_off[L]; i < hp.blk_off[L + 1]; ++i) {
          const uint2 rec = hp.blk[i];
          const uint32_t qa = rec.x & 0x3FFF, qb = (rec.x >> 14) & 0x3FFF; const bool two = (rec.x >> 28) & 1;
          if (seen[qa]++ || (two && seen[qb]++)) { printf("overlap in layer\n"); ++bad; }
          blockh(rec, X2, Z2, r2);
          ++blocks;
        }
        ++layers;
      }
    }
    gates_total += ng;
    ++cases;
    if (X != X2 || Z != Z2 || r != r2) { if (bad < 5) printf("mismatch case %d n=%d ng=%d\n", t, n, ng); ++bad; }
  }
  printf("cases %d bad %d gates %lld blocks %lld superlayers %lld\n", cases, bad, gates_total, blocks, layers);
  // a list long enough to be compiled in chunks by worker threads (each chunk
  // its own gate runs, appended in order)
  {
    const int n = 300, ng = 600000;
    std::vector<tab_gate> g;
    for (int i = 0; i < ng; ++i) {
      uint32_t op = 1 + (uint32_t)(rng() % 9);
      uint32_t a = (uint32_t)(rng() % n), b = (uint32_t)(rng() % n);
      if (op >= TAB_CNOT) while (b == a) b = (uint32_t)(rng() % n);
      g.push_back(tab_make_gate(op, a, op >= TAB_CNOT ? b : 0));
    }
    HostProgram hp;
    if (build_program(n, g.data(), (int64_t)g.size(), &hp, kProgBlocks) != TAB_OK) return 1;
    std::vector<uint32_t> X(n), Z(n);
    for (int a = 0; a < n; ++a) { X[a] = (uint32_t)rng(); Z[a] = (uint32_t)rng(); }
    uint32_t r = (uint32_t)rng(), r2 = r;
    std::vector<uint32_t> X2 = X, Z2 = Z;
    for (auto w : g) gate((uint32_t)(w >> 56), (uint32_t)((w >> 28) & 0xFFFFFFF), (uint32_t)(w & 0xFFFFFFF), X, Z, r);
    int runs = 0;
    for (const Seg& s : hp.segs) {
      if (s.kind != 0) continue;
      ++runs;
      for (uint32_t L = s.blk_begin; L < s.blk_end; ++L)
        for (uint32_t i = hp.blk_off[L]; i < hp.blk_off[L + 1]; ++i) blockh(hp.blk[i], X2, Z2, r2);
    }
    const bool ok = X == X2 && Z == Z2 && r == r2 && hp.n_gates == ng;
    printf("long list: %d gates, %d gate runs, %s\n", ng, runs, ok ? "equal" : "MISMATCH");
    if (!ok) ++bad;
  }
  // random-layer circuit shape: n=1000, 50 layers, H/S per qubit, n/2 CNOT:CZ
  // 3:1 -- one super-layer per layer
  {
    const int n = 1000; std::vector<tab_gate> g;
    for (int L = 0; L < 50; ++L) {
      for (int a = 0; a < n; ++a) g.push_back(tab_make_gate(rng() & 1 ? TAB_H : TAB_S, a, 0));
      std::vector<int> p(n); for (int i = 0; i < n; ++i) p[i] = i; std::shuffle(p.begin(), p.end(), rng);
      for (int i = 0; i + 1 < n; i += 2) g.push_back(tab_make_gate(rng() % 4 ? TAB_CNOT : TAB_CZ, p[i], p[i + 1]));
    }
    HostProgram hp; build_program(n, g.data(), (int64_t)g.size(), &hp, kProgBlocks | kProgBankOrder);
    // windows of 16 records (one half-warp's 8-byte loads): how many read
    // 16 distinct bank pairs for both qubits (the bank order's goal), and
    // the worst bank-pair load
    long long win = 0, distinct = 0; int worst = 0;
    for (size_t L = 0; L + 1 < hp.blk_off.size(); ++L) {
      for (uint32_t w0 = hp.blk_off[L]; w0 < hp.blk_off[L + 1]; w0 += 16) {
        uint32_t ma = 0, mb = 0; bool ok = true; int ca[16] = {0}, cb[16] = {0};
        for (uint32_t i = w0; i < std::min(hp.blk_off[L + 1], w0 + 16); ++i) {
          const uint32_t a = hp.blk[i].x & 15u, b = (hp.blk[i].x >> 14) & 15u;
          ok = ok && !((ma >> a) & 1u) && !((mb >> b) & 1u);
          ma |= 1u << a; mb |= 1u << b;
          worst = std::max(worst, std::max(++ca[a], ++cb[b]));
          if (hp.blk[i].x >> 31) { printf("record bit 31 set\n"); ++bad; }
        }
        ++win; distinct += ok;
      }
    }
    printf("layer circuit: %zu gates -> %zu blocks, %zu super-layers; windows %lld, "
           "conflict-free %lld, worst bank load %d\n", g.size(), hp.blk.size(), hp.blk_off.size() - 1,
           win, distinct, worst);
    if (hp.blk_off.size() - 1 != 50 || hp.blk.size() != 25000) ++bad;
  }
  // the pipelined apply's host side: chunks compiled apart (build_validated_
  // blocks), groups of consecutive chunks merged without their records
  // (concat_programs with_blk = false) while the records are concatenated on
  // their own, and adjacent gate runs taken as one run over the shared bound
  // (an empty super-layer) -- the result must equal the gates one at a time
  {
    const int n = 200, ng = 300000;
    std::vector<tab_gate> g;
    for (int i = 0; i < ng; ++i) {
      uint32_t op = 1 + (uint32_t)(rng() % 9);
      uint32_t a = (uint32_t)(rng() % n), b = (uint32_t)(rng() % n);
      if (op >= TAB_CNOT) while (b == a) b = (uint32_t)(rng() % n);
      g.push_back(tab_make_gate(op, a, op >= TAB_CNOT ? b : 0));
    }
    std::vector<int64_t> bnd{0};
    for (int64_t s = 1 << 12; bnd.back() < ng; s = std::min<int64_t>(1 << 15, s * 2))
      bnd.push_back(std::min<int64_t>(ng, bnd.back() + s));
    const int nc = (int)bnd.size() - 1;
    std::vector<HostProgram> parts((size_t)nc);
    for (int c = 0; c < nc; ++c)
      if (build_validated_blocks(n, g.data() + bnd[c], bnd[c + 1] - bnd[c], &parts[(size_t)c]) != TAB_OK)
        return 1;
    std::vector<uint32_t> X(n), Z(n);
    for (int a = 0; a < n; ++a) { X[a] = (uint32_t)rng(); Z[a] = (uint32_t)rng(); }
    uint32_t r = (uint32_t)rng(), r2 = r;
    std::vector<uint32_t> X2 = X, Z2 = Z;
    for (auto w : g) gate((uint32_t)(w >> 56), (uint32_t)((w >> 28) & 0xFFFFFFF), (uint32_t)(w & 0xFFFFFFF), X, Z, r);
    int launches = 0;
    for (int i = 0; i < nc;) {
      const int j = std::min(nc, i + 1 + (int)(rng() % 5));  // merge 1..5 chunks
      HostProgram M;
      concat_programs(M, &parts[(size_t)i], (size_t)(j - i), false);
      std::vector<uint2> rec;
      for (int c = i; c < j; ++c) rec.insert(rec.end(), parts[(size_t)c].blk.begin(), parts[(size_t)c].blk.end());
      if (!M.blk.empty()) ++bad;
      for (size_t si = 0; si < M.segs.size(); ++si) {
        if (M.segs[si].kind != 0) continue;
        size_t sj = si;
        while (sj + 1 < M.segs.size() && M.segs[sj + 1].kind == 0 &&
               M.segs[sj + 1].blk_begin == M.segs[sj].blk_end + 1)
          ++sj;
        ++launches;
        for (uint32_t L = M.segs[si].blk_begin; L < M.segs[sj].blk_end; ++L)
          for (uint32_t k = M.blk_off[L]; k < M.blk_off[L + 1]; ++k) blockh(rec[k], X2, Z2, r2);
        si = sj;
      }
      i = j;
    }
    const bool ok = X == X2 && Z == Z2 && r == r2;
    printf("pipelined merge: %d chunks, %d launches, %s\n", nc, launches, ok ? "equal" : "MISMATCH");
    if (!ok) ++bad;
  }
  return bad != 0;
}
