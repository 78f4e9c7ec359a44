// aes_internal.h — launch interfaces between the C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace aesgpu {

enum class Op : int { kEcbEncrypt = 0, kEcbDecrypt = 1, kCtr = 2 };

// Round keys travel in the kernel's parameter block (constant bank), so every
// AddRoundKey reads a uniform constant operand.
struct RoundKeys {
  uint32_t w[60];
};

// CTR parameters, precomputed on the host per launch.  With the nonce fixed,
// columns 0..2 of the state after the initial AddRoundKey are the same for
// every block, so 12 of the 16 first-round lookups are folded into c1[]:
//   round-1 column j = c1[j] ^ T_{3-j}[byte 3-j of (counter word ^ rk0w3)].
struct CtrParams {
  uint32_t ctr0;    // counter value of block 0 of this launch
  uint32_t rk0w3;   // round-0 key word 3
  uint32_t c1[4];   // folded round-1 columns (round-1 key included)
  uint32_t iv_w[4]; // IV words (little-endian), used by the partial tail block
  // run-cached CTR kernel only, set at launch for its grid: runs done one per
  // warp in whole waves, and log2 of the pieces each later run is split into
  uint64_t whole_runs;
  uint32_t tail_shift;
};

struct LaunchShape {
  int cta_threads;
  int blocks_per_thread;
  int grid_ctas;
};

// T-table launches, one per operation (each returns the launch's CUDA error).
#define AESGPU_DECLARE_LAUNCH(name)                                                          \
  cudaError_t name(int nr, const void* in, void* out, uint64_t nblocks, uint32_t tail_bytes, \
                   const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,        \
                   cudaStream_t stream);
AESGPU_DECLARE_LAUNCH(launch_ttable_enc)
AESGPU_DECLARE_LAUNCH(launch_ttable_dec)
AESGPU_DECLARE_LAUNCH(launch_ttable_ctr)
AESGPU_DECLARE_LAUNCH(launch_ttable_ctr_bulk)  // CTR with TMA-staged input (cta_threads from the shape)
#undef AESGPU_DECLARE_LAUNCH
// Given-up bounded waits of the TMA-staged kernel on the current device since
// the last call (then reset); synchronises with the device.
cudaError_t take_bulk_timeouts(unsigned int* out);

// Bitsliced launches (32 blocks per thread, 128-thread CTAs).  Decryption takes
// the encryption schedule (plain InvCipher order).
cudaError_t launch_bitslice(Op op, int nr, const void* in, void* out, uint64_t nblocks,
                            uint32_t tail_bytes, const RoundKeys& rk, const CtrParams& cp,
                            const LaunchShape& shape, cudaStream_t stream);
constexpr int kBitsliceThreads = 128;
constexpr int kBitsliceBlocksPerCta = 4 * 512;  // 4 warps x 512 blocks per iteration

// CBC decryption (rk: the equivalent inverse schedule; cp.iv_w: the IV) and
// XTS (rk1: data key, encryption or equivalent inverse schedule; rk2: tweak
// key, encryption schedule; nblocks a multiple of 32, sector_blocks too).
cudaError_t launch_cbc_decrypt(int nr, const void* in, void* out, uint64_t nblocks, const RoundKeys& rk,
                               const CtrParams& cp, const LaunchShape& shape, cudaStream_t stream);
cudaError_t launch_xts_mode(bool decrypt, int nr, int nr_tweak, const void* in, void* out,
                            uint64_t nblocks, const RoundKeys& rk1, const RoundKeys& rk2,
                            uint64_t first_sector, uint32_t sector_blocks, const LaunchShape& shape,
                            cudaStream_t stream);

// Dynamic shared memory of the T-table kernels (bytes).
constexpr int kTtableSmemEnc = 128 * 1024;
constexpr int kTtableSmemDec = 192 * 1024;

}  // namespace aesgpu
