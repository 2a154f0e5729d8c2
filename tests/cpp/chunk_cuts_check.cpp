// Host check of tab_batch_run's chunking (batch_chunk_cuts): for random
// circuit lists (gate counts spread over orders of magnitude, empty and
// negative counts among them), chunk counts and shares, the bounds start at
// 0, end at m and grow strictly (no empty chunk), there are at most K
// chunks, and each cut is the first circuit at which the running gate count
// reaches its target (first_share of the gates, then equal parts of the
// rest), checked against a direct restatement of that rule.  Exit status 0
// on success; prints "bad <count>".
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>
#include "tab_internal.h"
using namespace tab;

int main() {
  std::mt19937_64 rng(7);
  int bad = 0, cases = 0;
  for (int trial = 0; trial < 3000; ++trial) {
    const int32_t m = (int32_t)(rng() % 300);
    std::vector<tab_circuit> cs((size_t)m);
    int64_t total = 0;
    for (auto& c : cs) {
      const int r = (int)(rng() % 10);
      c.n_gates = r == 0 ? 0 : r == 1 ? -5 : (int64_t)std::exp2((double)(rng() % 20));
      total += c.n_gates > 0 ? c.n_gates : 0;
    }
    const int K = 1 + (int)(rng() % 9);
    const double share = trial % 2 ? 0.1 : 1.0 / K;
    const std::vector<int32_t> cut = batch_chunk_cuts(cs.data(), m, K, share);
    ++cases;
    bool ok = !cut.empty() && cut.front() == 0 && cut.back() == m;
    for (size_t i = 1; ok && i < cut.size(); ++i) ok = cut[i] > cut[i - 1];
    ok = ok && (int)cut.size() - 1 <= (m > 0 ? K : 0) && (m > 0 || cut.size() == 1);
    // the rule, restated: walk the circuits; cut after circuit c when the
    // running count reaches the next target, at most one cut per circuit
    std::vector<int32_t> want(1, 0);
    int64_t run = 0;
    int k = 1;
    for (int32_t c = 0; c < m && k < K; ++c) {
      run += cs[(size_t)c].n_gates > 0 ? cs[(size_t)c].n_gates : 0;
      const double t = (double)total * (share + (1.0 - share) * (k - 1) / (double)(K - 1));
      if ((double)run >= t) {
        want.push_back(c + 1);
        ++k;
      }
    }
    if (want.back() != m) want.push_back(m);
    ok = ok && want == cut;
    if (!ok) {
      if (bad < 10) printf("m=%d K=%d share=%.2f: %zu bounds\n", m, K, share, cut.size());
      ++bad;
    }
  }
  // equal circuits, equal chunks: 100 circuits of 10 gates in 4 chunks
  {
    std::vector<tab_circuit> cs(100);
    for (auto& c : cs) c.n_gates = 10;
    const std::vector<int32_t> cut = batch_chunk_cuts(cs.data(), 100, 4, 0.25);
    if (cut != std::vector<int32_t>({0, 25, 50, 75, 100})) {
      printf("equal chunks wrong\n");
      ++bad;
    }
    const std::vector<int32_t> cut2 = batch_chunk_cuts(cs.data(), 100, 5, 0.1);
    if (cut2 != std::vector<int32_t>({0, 10, 33, 55, 78, 100})) {
      printf("first-share chunks wrong:");
      for (int32_t v : cut2) printf(" %d", v);
      printf("\n");
      ++bad;
    }
  }
  printf("cases %d bad %d\n", cases, bad);
  return bad ? 1 : 0;
}
