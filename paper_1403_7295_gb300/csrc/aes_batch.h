// aes_batch.h — internal interface of the batched (many-message) kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "aesgpu.h"

namespace aesgpu {

enum : uint32_t { kBatchCtr = 0, kBatchEcbEnc = 1, kBatchEcbDec = 2 };

// Kernel-side view of one batch (passed by value as a kernel parameter).
struct BatchArgs {
  uint32_t n;   // messages
  uint32_t op;  // kBatch*
  const uint8_t* in;
  uint8_t* out;
  const uint64_t* in_off;
  const uint64_t* in_len;
  const uint64_t* out_off;
  const uint8_t* keys;
  const uint32_t* key_bits;
  const aes_key_schedule* schedules;
  const uint32_t* sched_idx;
  uint32_t n_sched;
  uint32_t tile_blocks;
  uint32_t flags;  // AES_BATCH_IN_PADDED | AES_BATCH_OUT_PADDED
  const uint8_t* iv;
  uint64_t* out_len;
  int32_t* status;
  // workspace
  uint64_t* blk_off;    // [n + 1] first global block of each message; [n] = total
  uint64_t* chunk_sum;  // [nchunks] per-chunk totals, then chunk offsets
  unsigned long long* tile_counter;   // next tile of the long-message block space
  unsigned long long* short_counter;  // next group of messages for the short-message phase
  uint32_t nchunks;
};

size_t batch_workspace_bytes(uint32_t n);
void batch_bind_workspace(BatchArgs* a, void* ws);
cudaError_t launch_batch(const BatchArgs& a, int cta, int grid, cudaStream_t s);

// Sets the calling thread's aes_last_cuda_error() and returns AES_ERR_CUDA.
aes_status record_cuda_failure(cudaError_t e);

}  // namespace aesgpu
