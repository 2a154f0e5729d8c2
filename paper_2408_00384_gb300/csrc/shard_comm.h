// shard_comm.h -- collectives for ranks that are host threads of one process:
// the exchange steps of a row-sharded tableau (barrier, all-reduce of a
// minimum, broadcast and gather of byte buffers).
//
// Every collective is entered by all ranks in the same order.  A rank that
// fails calls abort(); from then on every collective returns false at once
// (and a wait that outlasts the limit aborts too), so no rank is left
// waiting on one that has gone.  A barrier spins for a few microseconds
// before it blocks: the exchanges of a measurement are short and frequent.
#pragma once
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <limits>
#include <mutex>
#include <vector>

namespace tab {

class HostComm {
 public:
  explicit HostComm(int ranks, double limit_s = 60.0)
      : ranks_(ranks), limit_(limit_s), vals_((size_t)ranks, 0), srcs_((size_t)ranks, nullptr) {}
  int size() const { return ranks_; }

  void abort() {
    std::lock_guard<std::mutex> lk(m_);
    aborted_.store(true);
    cv_.notify_all();
  }
  bool aborted() { return aborted_.load(); }

  // false when aborted (or when the wait outlasts the limit, which aborts)
  bool barrier() {
    if (aborted_.load()) return false;
    const uint64_t gen = gen_.load(std::memory_order_acquire);
    if (arrived_.fetch_add(1, std::memory_order_acq_rel) + 1 == ranks_) {
      arrived_.store(0, std::memory_order_relaxed);
      {
        std::lock_guard<std::mutex> lk(m_);
        gen_.fetch_add(1, std::memory_order_release);
      }
      cv_.notify_all();
      return !aborted_.load();
    }
    // spin a little (the other ranks are usually microseconds away), then block
    const auto t0 = std::chrono::steady_clock::now();
    while (std::chrono::steady_clock::now() - t0 < std::chrono::microseconds(50)) {
      if (gen_.load(std::memory_order_acquire) != gen) return !aborted_.load();
      if (aborted_.load()) return false;
    }
    std::unique_lock<std::mutex> lk(m_);
    const bool ok = cv_.wait_for(lk, std::chrono::duration<double>(limit_), [&] {
      return gen_.load(std::memory_order_acquire) != gen || aborted_.load();
    });
    if (!ok) {
      aborted_.store(true);
      cv_.notify_all();
    }
    return !aborted_.load();
  }

  // the minimum of every rank's v, returned to every rank
  bool allreduce_min(int rank, int64_t v, int64_t* out) {
    vals_[(size_t)rank] = v;
    if (!barrier()) return false;
    int64_t m = std::numeric_limits<int64_t>::max();
    for (int64_t x : vals_) m = x < m ? x : m;
    *out = m;
    return barrier();
  }

  // root's `bytes` at buf copied into buf on every other rank
  bool broadcast(int rank, int root, void* buf, size_t bytes) {
    if (rank == root) srcs_[(size_t)root] = buf;
    if (!barrier()) return false;
    if (rank != root) memcpy(buf, srcs_[(size_t)root], bytes);
    return barrier();
  }

  // rank r's `bytes` at in -> offset r * bytes of out on root
  bool gather(int rank, int root, const void* in, size_t bytes, void* out) {
    srcs_[(size_t)rank] = in;
    if (!barrier()) return false;
    if (rank == root)
      for (int r = 0; r < ranks_; ++r)
        memcpy(static_cast<char*>(out) + (size_t)r * bytes, srcs_[(size_t)r], bytes);
    return barrier();
  }

 private:
  std::mutex m_;
  std::condition_variable cv_;
  const int ranks_;
  const double limit_;
  std::atomic<int> arrived_{0};
  std::atomic<uint64_t> gen_{0};
  std::atomic<bool> aborted_{false};
  std::vector<int64_t> vals_;
  std::vector<const void*> srcs_;
};

}  // namespace tab
