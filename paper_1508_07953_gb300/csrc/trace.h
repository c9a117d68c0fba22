// trace.h -- NVTX ranges around the library's host entry points (a frame, a
// batched step, a served tick, an anchor-loop frame), so that a timeline
// profiler shows the launches grouped by the call that issued them.  With no
// profiler attached the push/pop calls return at once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace riann {

class NvtxRange {
 public:
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace riann
