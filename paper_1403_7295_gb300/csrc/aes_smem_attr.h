// aes_smem_attr.h — host launch helpers: the one-time opt-in of a kernel to a
// large dynamic shared-memory carve-out, per CUDA context (cudaFuncSetAttribute
// applies to the function in the current context; repeating it on every
// launch costs host time on small calls), and launches with programmatic
// stream serialisation.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <set>
#include <utility>

namespace aesgpu {

// ID of the calling thread's current CUDA context (unique for the life of
// the process; a context made after cudaDeviceReset gets a new one), or 0
// when no context is current yet.  The two driver calls are fetched through
// the runtime, so the library needs no link against the driver library.
// Returns false if the driver does not offer them.
inline bool current_context_id(unsigned long long* id) {
  using GetCurrentFn = CUresult (*)(CUcontext*);
  using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
  struct Calls {
    GetCurrentFn get_current = nullptr;
    GetIdFn get_id = nullptr;
  };
  static const Calls calls = [] {
    Calls c;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void* f1 = nullptr;
    void* f2 = nullptr;
    // cuCtxGetId exists from CUDA 12.0 on.
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2) {
      c.get_current = reinterpret_cast<GetCurrentFn>(f1);
      c.get_id = reinterpret_cast<GetIdFn>(f2);
    }
    return c;
  }();
  if (calls.get_current == nullptr) return false;
  CUcontext ctx = nullptr;
  if (calls.get_current(&ctx) != CUDA_SUCCESS) return false;
  *id = 0;
  return ctx == nullptr || calls.get_id(ctx, id) == CUDA_SUCCESS;
}

// The one-time opt-in of a kernel to `bytes` of dynamic shared memory.  The
// attribute belongs to the kernel as loaded in one CUDA context, so the
// opt-in is remembered per (kernel, context ID); a context without an ID
// yet (none current) is opted in every time.
template <class Kernel>
inline cudaError_t ensure_dynamic_smem(Kernel kern, int bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, unsigned long long>> done;  // (kernel, context) already opted in
  unsigned long long ctx = 0;
  if (!current_context_id(&ctx)) ctx = 0;
  const std::pair<const void*, unsigned long long> key{reinterpret_cast<const void*>(kern), ctx};
  std::lock_guard<std::mutex> lock(mu);
  if (ctx != 0 && done.count(key)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && ctx != 0) done.insert(key);
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
