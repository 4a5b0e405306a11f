// NVTX ranges around the library's entry points, so that a profiler attached
// to the process (Nsight Systems, or ncu --nvtx) can attribute the host calls
// and the kernels they enqueue to a phase: frame ingest, initialisation, the
// solve, the energy, batches, the network.  NVTX v3 is header-only; without a
// tool attached a range costs a branch.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace gid {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace gid
