// Host-side kernel launch with an optional programmatic dependency on the
// previous kernel of the stream (programmatic dependent launch).
//
// While the calling thread's flag is set (PdlScope), launches made through
// launch_pdl carry cudaLaunchAttributeProgrammaticStreamSerialization: the
// kernel may be scheduled as soon as every CTA of the previous kernel has
// executed griddepcontrol.launch_dependents, runs its prologue, and waits in
// griddepcontrol.wait (ptx::grid_dep_wait) for that kernel to complete before
// it touches shared data.  Only kernels with that wait may be launched this
// way; with the flag clear the launch is an ordinary stream-ordered one.
#pragma once

#include <cuda_runtime.h>

namespace th {

inline bool& pdl_flag() {
  thread_local bool on = false;
  return on;
}

struct PdlScope {
  bool prev;
  explicit PdlScope(bool on) : prev(pdl_flag()) { pdl_flag() = on; }
  ~PdlScope() { pdl_flag() = prev; }
  PdlScope(const PdlScope&) = delete;
  PdlScope& operator=(const PdlScope&) = delete;
};

// cluster > 0 adds a thread-block cluster of that many CTAs along x
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int cluster,
                       const Args&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (cluster > 0) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (pdl_flag()) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  cfg.attrs = na ? attr : nullptr;
  cfg.numAttrs = na;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace th
