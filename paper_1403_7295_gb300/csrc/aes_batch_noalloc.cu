// aes_batch_noalloc.cu — aes_batch_submit for callers that cannot allocate:
// the batch pipeline's workspace (per-message block offsets, chunk totals,
// work counters, the lane path's bins and order) lives in one file-scope
// device array instead of a caller buffer.  The work itself is the ordinary aes_batch_submit path.
#include <cuda_runtime.h>

#include <mutex>

#include "aes_batch.h"
#include "aes_smem_attr.h"
#include "aesgpu.h"

namespace {

// Layout of the batch workspace for n messages: offsets (n + 1 words),
// chunk totals (one word per 4096 messages), work counters, then the lane
// path's bins (n halfwords), bin counts, cursors and a count (2 x 1536 + 1 words) and
// order (n + 96 words), each rounded up to 256 bytes.
constexpr size_t round256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
constexpr size_t workspace_for(size_t n) {
  return round256(8 * (n + 1)) + round256(8 * ((n + 4095) / 4096)) + 256 + round256(2 * n) +
         round256(8 * 1536 + 4) + round256(4 * (n + 96));
}
constexpr size_t kScratchBytes = workspace_for(AES_BATCH_NOALLOC_MAX_MSGS);  // 931,328 bytes

// Held by every device that loads the library, for the life of the process.
static __device__ __align__(256) unsigned char g_batch_scratch[kScratchBytes];

// Device address of g_batch_scratch per device ordinal, looked up with that
// device current and kept with the ID of the CUDA context it was looked up
// in.  The host-side symbol is only a handle: its own address is not usable
// on the device.  A new context on the device (after cudaDeviceReset, or a
// driver-API context made current) has a new ID and gets a fresh lookup, so
// a stale address from a destroyed context is never handed to a kernel.
constexpr int kMaxDevices = 64;
struct ScratchEntry {
  unsigned long long ctx_id;
  void* ptr;
};
std::mutex g_mu;
ScratchEntry g_scratch[kMaxDevices] = {};

aes_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return aesgpu::record_cuda_failure(e);
  if (dev < 0 || dev >= kMaxDevices) return AES_ERR_ARG;
  unsigned long long id = 0;
  if (!aesgpu::current_context_id(&id)) return aesgpu::record_cuda_failure(cudaErrorNotSupported);
  std::lock_guard<std::mutex> lock(g_mu);
  ScratchEntry& entry = g_scratch[dev];
  if (id == 0 || entry.ptr == nullptr || entry.ctx_id != id) {
    if (aesgpu::batch_workspace_bytes(AES_BATCH_NOALLOC_MAX_MSGS) > kScratchBytes)
      return AES_ERR_NOMEM;  // layout drifted from the sizing above
    void* p = nullptr;
    // Binds (or creates) the device's primary context when none is current.
    e = cudaGetSymbolAddress(&p, g_batch_scratch);
    if (e != cudaSuccess) return aesgpu::record_cuda_failure(e);
    if (!aesgpu::current_context_id(&id) || id == 0) return aesgpu::record_cuda_failure(cudaErrorNotSupported);
    entry = ScratchEntry{id, p};
  }
  *out = entry.ptr;
  return AES_OK;
}

}  // namespace

extern "C" aes_status aes_batch_submit_noalloc(const aes_batch* b, void* stream) {
  if (b == nullptr) return AES_ERR_ARG;
  if (b->n_msgs > AES_BATCH_NOALLOC_MAX_MSGS) return AES_ERR_NOMEM;
  if (b->n_msgs == 0) return AES_OK;
  void* ws = nullptr;
  const aes_status s = scratch_for_current_device(&ws);
  if (s != AES_OK) return s;
  // Nothing needs clearing here: the pipeline itself resets the work
  // counters and bin counts and rewrites every offset the later kernels read.
  return aes_batch_submit_ex(b, ws, kScratchBytes, stream, nullptr);
}
