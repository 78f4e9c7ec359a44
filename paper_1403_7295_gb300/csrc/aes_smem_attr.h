// aes_smem_attr.h — one-time opt-in of a kernel to a large dynamic
// shared-memory carve-out, per device (cudaFuncSetAttribute is per function
// and device; repeating it on every launch costs host time on small calls).
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

}  // namespace aesgpu
