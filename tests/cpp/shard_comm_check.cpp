// Host check of the thread-rank collectives (shard_comm.h): ranks as threads
// run many rounds of all-reduce-min, broadcast from a rotating root and
// gather, and every rank checks every result; then one rank aborts in the
// middle and the others must leave their collectives (no rank left waiting);
// then one rank never arrives and the others must give up after the limit.
// Exit status 0 on success.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "shard_comm.h"

using tab::HostComm;

int main() {
  const int R = 4, rounds = 2000;
  std::atomic<int> bad{0};
  {
    HostComm comm(R, 10.0);
    std::vector<std::thread> th;
    for (int r = 0; r < R; ++r)
      th.emplace_back([&, r] {
        for (int it = 0; it < rounds; ++it) {
          int64_t m = -1;
          const int64_t mine = (int64_t)((it * 7 + r * 13) % 29) - 5;
          if (!comm.allreduce_min(r, mine, &m)) { bad++; return; }
          int64_t want = 1 << 30;
          for (int q = 0; q < R; ++q) want = std::min<int64_t>(want, (int64_t)((it * 7 + q * 13) % 29) - 5);
          if (m != want) bad++;
          const int root = it % R;
          uint32_t buf[3] = {0, 0, 0};
          if (r == root) { buf[0] = (uint32_t)it; buf[1] = (uint32_t)root; buf[2] = 0xABCDu; }
          if (!comm.broadcast(r, root, buf, sizeof buf)) { bad++; return; }
          if (buf[0] != (uint32_t)it || buf[1] != (uint32_t)root || buf[2] != 0xABCDu) bad++;
          uint64_t v = (uint64_t)it * 100 + (uint64_t)r;
          std::vector<uint64_t> all(R, 0);
          if (!comm.gather(r, 1, &v, sizeof v, all.data())) { bad++; return; }
          if (r == 1)
            for (int q = 0; q < R; ++q)
              if (all[(size_t)q] != (uint64_t)it * 100 + (uint64_t)q) bad++;
        }
      });
    for (auto& t : th) t.join();
  }
  std::atomic<int> left{0};
  {
    HostComm comm(R, 10.0);
    std::vector<std::thread> th;
    for (int r = 0; r < R; ++r)
      th.emplace_back([&, r] {
        for (int it = 0; it < rounds; ++it) {
          if (r == 2 && it == 500) { comm.abort(); break; }
          int64_t m;
          if (!comm.allreduce_min(r, it, &m)) break;
        }
        left++;
      });
    for (auto& t : th) t.join();
  }
  // a rank that never arrives: the others give up after the limit
  std::atomic<int> timed_out{0};
  {
    HostComm comm(R, 0.2);
    std::vector<std::thread> th;
    for (int r = 0; r < R - 1; ++r)  // rank R-1 never joins
      th.emplace_back([&, r] {
        int64_t m;
        if (!comm.allreduce_min(r, r, &m)) timed_out++;
      });
    for (auto& t : th) t.join();
  }
  printf("bad %d left %d timed_out %d\n", bad.load(), left.load(), timed_out.load());
  return (bad.load() == 0 && left.load() == R && timed_out.load() == R - 1) ? 0 : 1;
}
