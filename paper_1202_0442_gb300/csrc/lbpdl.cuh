// lbpdl.cuh -- programmatic dependent launch of the kernels of an
// iteration.
//
// A kernel launched with launch_pdl may be scheduled while the kernel
// before it in the stream drains: its blocks are placed once every block of
// that kernel has exited, without waiting for the kernel's completion to
// travel back through the front end.  Each such kernel calls dep_wait()
// (griddepcontrol.wait) before its first global-memory access; it returns
// once the previous kernel has completed and its writes are visible.  The
// order of the stream is therefore kept exactly (same results bit for bit);
// only the launch latency between two dependent kernels is hidden.  A
// kernel launched the ordinary way passes dep_wait() at once.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace lbk {

__device__ __forceinline__ void dep_wait() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

template <class... P, class... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace lbk
