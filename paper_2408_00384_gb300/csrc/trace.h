// trace.h -- NVTX ranges around the C-ABI calls, so a profiler's timeline
// shows which library call issued which launches.  NVTX 3 is header-only:
// with no tool attached a range costs a check of a null callback.  Without
// the header (another toolkit) the ranges compile to nothing.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define TAB_HAVE_NVTX 1
#endif
#endif

namespace tab {

class TraceRange {
 public:
  explicit TraceRange(const char* name) {
#ifdef TAB_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~TraceRange() {
#ifdef TAB_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace tab
