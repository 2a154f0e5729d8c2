// pool.cpp -- persistent host worker threads for pool_run (pool.h).
//
// The workers start on first use (one fewer than the hardware threads, at
// most 15) and sleep on a condition variable between jobs.  A job hands out
// indices from an atomic counter; the caller takes indices too and then waits
// until every index has finished.  A pool_run called from inside a job runs
// its indices on the calling thread.
#include "pool.h"

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

namespace tab {

namespace {

thread_local bool t_in_job = false;  // this thread is running a job's index

class Pool {
 public:
  Pool() {
    const unsigned hw = std::thread::hardware_concurrency();
    const int nw = (int)std::min<unsigned>(hw > 1 ? hw - 1 : 0, 15u);
    for (int i = 0; i < nw; ++i) workers_.emplace_back([this] { loop(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(m_);
      stop_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (auto& t : workers_) t.join();
  }
  int threads() const { return (int)workers_.size() + 1; }

  void run(int n, const std::function<void(int)>& fn) {
    if (n <= 0) return;
    if (n == 1 || workers_.empty() || t_in_job) {
      for (int i = 0; i < n; ++i) fn(i);
      return;
    }
    std::lock_guard<std::mutex> job_lock(job_m_);  // one job at a time
    {
      std::lock_guard<std::mutex> lk(m_);
      fn_ = &fn;
      n_ = n;
      next_.store(0);
      done_.store(0);
      ++gen_;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(m_);
    done_cv_.wait(lk, [&] { return done_.load() == n_; });
    fn_ = nullptr;
  }

 private:
  void work() {
    for (;;) {
      const int i = next_.fetch_add(1);
      if (i >= n_) return;
      t_in_job = true;
      (*fn_)(i);
      t_in_job = false;
      if (done_.fetch_add(1) + 1 == n_) {
        std::lock_guard<std::mutex> lk(m_);
        done_cv_.notify_all();
      }
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(m_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
        if (stop_) return;
        if (fn_ == nullptr) continue;
      }
      work();
    }
  }

  std::vector<std::thread> workers_;
  std::mutex m_, job_m_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* fn_ = nullptr;
  int n_ = 0;
  std::atomic<int> next_{0}, done_{0};
  uint64_t gen_ = 0;
  bool stop_ = false;
};

Pool& pool() {
  static Pool p;
  return p;
}

}  // namespace

void pool_run(int n, const std::function<void(int)>& fn) { pool().run(n, fn); }
int pool_threads() { return pool().threads(); }

}  // namespace tab
