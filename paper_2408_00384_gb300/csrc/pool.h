// pool.h -- a small persistent host thread pool for the runtime's parallel
// steps (chunked program compilation, the merge of the chunks, and copies of
// large compiled programs into the pinned staging buffer).
#pragma once
#include <functional>

namespace tab {

// Run fn(0) .. fn(n-1) on the pool's workers and the calling thread; returns
// when all have finished.  Calls from several threads at once are
// serialised.  With n <= 1, no workers, or a call made from inside another
// pool_run job, fn runs on the calling thread.
void pool_run(int n, const std::function<void(int)>& fn);

// Threads available to pool_run (workers + the caller).
int pool_threads();

}  // namespace tab
