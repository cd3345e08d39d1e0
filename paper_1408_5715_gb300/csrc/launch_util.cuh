// launch_util.cuh -- kernel launches with programmatic dependent launch.
//
// A time loop is a chain of kernels, each reading what the previous one
// wrote.  Launched with programmatic stream serialisation, kernel j+1 is set
// up while kernel j runs; its blocks wait in `griddepcontrol.wait` (a
// hardware wait for the previous grid to complete and its memory to be
// visible) before touching any data.  The kernels do not signal an early
// launch (`griddepcontrol.launch_dependents`): measured on GB300, letting the
// next grid's blocks take SM slots during the previous step's last wave
// slowed the persistent shapes by up to 8 %, while the implicit signal at
// grid completion still hides the launch gap (1-6 % per step on meshes of 1M
// and 65k cells).  Without a programmatic predecessor the wait returns at
// once, so the kernels are correct under any launch.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace fv {
namespace {

// First statement of every kernel launched in a programmatic chain.
__device__ __forceinline__ void chain_entry() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_chained(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem,
                           cudaStream_t s, bool programmatic, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  if (programmatic) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace
}  // namespace fv
