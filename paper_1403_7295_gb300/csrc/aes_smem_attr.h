// aes_smem_attr.h — host launch helpers: the one-time opt-in of a kernel to a
// large dynamic shared-memory carve-out, per device (cudaFuncSetAttribute is
// per function and device; repeating it on every launch costs host time on
// small calls), and launches with programmatic stream serialisation.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

namespace aesgpu {

template <class Kernel>
inline cudaError_t ensure_dynamic_smem(Kernel kern, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;  // (kernel, device) already opted in
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const std::pair<const void*, int> key{reinterpret_cast<const void*>(kern), dev};
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(key)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.insert(key);
  return e;
}

// Launch with programmatic stream serialisation: the kernel may start (and
// fill its shared-memory tables) while the previous kernel in the stream
// finishes; the kernel executes griddepcontrol.wait before touching any
// memory another grid may write (the caller's buffers), which returns once
// the previous grid has completed and its writes are visible.  Only kernels
// that do so may be launched this way.
template <typename Kern, typename... Args>
inline cudaError_t launch_pdl(Kern kern, unsigned grid, unsigned block, size_t smem, cudaStream_t stream,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace aesgpu
