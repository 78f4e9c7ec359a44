// aes_batch.h — internal interface of the batched (many-message) kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "aesgpu.h"

namespace aesgpu {

enum : uint32_t { kBatchCtr = 0, kBatchEcbEnc = 1, kBatchEcbDec = 2 };

// Short CTR messages of fewer than kLaneMax blocks take the lane path
// (aes_batch_lanes.cu), sorted into bins by (key-size class, 511 - blocks):
// class c = (nr - 10) / 2 holds bins [512c, 512c + 512), longest messages
// first.  A lane walks its message's blocks one after another, so longer
// messages (up to the short-phase limit of 512 blocks) stay with the
// persistent kernel's per-warp groups, which spread a message over 32 lanes.
constexpr uint32_t kLaneMax = 128;
constexpr uint32_t kLaneBins = 3 * 512;
constexpr uint16_t kLaneNoBin = 0xFFFF;  // the message is not on the lane path

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
  uint64_t* blk_off;    // [n + 1] first block of each message in the long-message space, counted from
                        // its chunk's first block (blk_start adds the chunk offset); [n] = total
  uint64_t* chunk_sum;  // [nchunks] per-chunk totals, then chunk offsets
  unsigned long long* tile_counter;   // next tile of the long-message block space
  unsigned long long* short_counter;  // next group of messages for the short-message phase
  unsigned int* scan_done;            // count-kernel CTAs finished (the last one scans the chunk totals)
  uint32_t nchunks;
  // The lane path of short CTR messages (one lane per message); all null when
  // the persistent kernel's per-warp groups run them instead.
  uint16_t* lane_bin;     // [n] each message's bin, kLaneNoBin if not on the lane path
  uint32_t* lane_hist;    // [kLaneBins] messages per bin, then each bin's first position in lane_order
  uint32_t* lane_cursor;  // [kLaneBins] positions of each bin handed out so far; then one word:
                          // the short messages left to the per-warp groups (kLaneMax blocks or more)
  uint32_t* lane_order;   // [n + 96] messages in bin order; each class starts at a multiple of 32,
                          // the gaps hold kLaneNoMsg
  uint32_t* lane_info;    // [5] chunks of 32 positions in all, then the first chunk of classes 0, 1, 2
                          // and the end of class 2 (= the total)
  unsigned long long* lane_counter;  // [3] next chunk of each class for the lane kernel
};

constexpr uint32_t kLaneNoMsg = 0xFFFFFFFFu;

size_t batch_workspace_bytes(uint32_t n);
// lanes: bind the lane path's arrays (CTR batches whose short messages take it)
void batch_bind_workspace(BatchArgs* a, void* ws, bool lanes);
cudaError_t launch_batch(const BatchArgs& a, int cta, int grid, cudaStream_t s);

// The lane path's steps (aes_batch_lanes.cu): the scatter into bin order,
// enqueued before the persistent kernel, then the lane kernel, enqueued after it.
// (The bin starts, gaps and chunk ranges are computed by the count kernel's
// last CTA.)
cudaError_t launch_batch_lanes_sort(const BatchArgs& a, cudaStream_t s);
cudaError_t launch_batch_lanes(const BatchArgs& a, int grid, cudaStream_t s);
// Bounded waits of the lane kernel that gave up since the last call; resets the count.
cudaError_t take_lane_timeouts(unsigned int* out);

// Sets the calling thread's aes_last_cuda_error() and returns AES_ERR_CUDA.
aes_status record_cuda_failure(cudaError_t e);

}  // namespace aesgpu
