// aes_batch.cu — batched varlen AES: many messages, each with its own key
// and IV, in one persistent launch (the paper's chunk-per-thread scheme of
// §IV.B with chunks = messages, mapped onto blocks of a GPU grid).
//
// Pipeline on the caller's stream:
//   0. a memset of the work counters (and, on the lane path of short CTR
//      messages, the bin counts).
//   1. batch_count_scan  per message: validate, count 16-byte blocks
//      (CTR ceil(len/16); ECB+PKCS#7 encrypt floor(len/16)+1; decrypt len/16),
//      write status/out_len, exclusive-scan the counts of long messages
//      (kShortMax blocks or more) inside chunks of 4096 messages.  The last
//      CTA to finish scans the chunk totals into chunk offsets and writes the
//      grand total: blk_start(m) = the chunk offset + m's offset in its chunk.
//   2. (lane path) the scatter of short CTR messages into bin order.
//   3. batch_kernel      persistent CTAs.  Long messages: the CTA claims tiles of
//      `tile_blocks` blocks of the long-message space with an atomic counter,
//      finds the tile's messages by a 32-way warp search over blk_start, expands
//      their keys on the device into shared memory (one thread per message,
//      FIPS-197 §5.2; the equivalent inverse schedule for ECB decryption), and
//      its warps run the T-table rounds of aes_ttable.cuh with round keys read
//      from shared memory (one 128-bit broadcast load per round) or, in the
//      512-thread build, held in registers across a span.  Short messages
//      (1 .. kShortMax-1 blocks), afterwards: every warp on its own claims
//      groups of consecutive messages, expands their keys into its own slots
//      and runs their blocks, with no CTA barrier (so key expansion and claims
//      of one warp overlap the rounds of the others, and the phase fills the
//      tail of the tile phase).
//
// The 1024-thread builds are compiled here; the 512-thread builds in
// aes_batch_regkeys.cu, which includes this file with AES_BATCH_REGKEYS_TU.
#include "aes_batch.h"
#include "aes_smem_attr.h"
#include "aes_ttable.cuh"

namespace aesgpu {
namespace {

constexpr uint32_t kScanThreads = 1024;
constexpr uint32_t kScanItems = 4;
constexpr uint32_t kRkStride = 68;  // words per schedule slot: 16-B aligned, skews banks by 4

template <int OPB>
struct WindowSize;
template <>
struct WindowSize<kBatchCtr> {
  static constexpr int value = 256;
};
template <>
struct WindowSize<kBatchEcbEnc> {
  static constexpr int value = 256;
};
template <>
struct WindowSize<kBatchEcbDec> {
  static constexpr int value = 96;
};

// One message of the current window.  Its round keys live in the schedule
// slot rk[0 .. 4(nr+1)); for CTR, words 60..63 hold the folded round-1
// columns and word 64 the round-0 key word 3.
struct Slot {
  uint64_t blk_start;  // global index of the message's first block
  uint64_t blk_end;
  uint64_t full_end;   // first global block that is not a whole 16-byte input block
  uint64_t src0, dst0; // byte address of (virtual) global block 0 of this message
  uint32_t nr, msg;
  uint32_t rem;        // len mod 16
  uint32_t ctr_base;   // CTR: counter of global block g is ctr_base + (uint32)g
};
constexpr uint32_t kCtrC1 = 60, kCtrRk0w3 = 64;

// Messages of fewer blocks than this go through the per-warp short phase.
constexpr uint64_t kShortMax = 512;

// Messages per warp group in the short phase: a warp's share of the window
// slots of a 1024-thread CTA.
template <int OPB>
constexpr uint32_t kGroup = WindowSize<OPB>::value / 32;

template <int OPB>
constexpr size_t batch_table_bytes() {
  return OPB == kBatchEcbDec ? 192 * 1024 : 128 * 1024;
}

template <int OPB>
constexpr size_t batch_smem_bytes() {
  return batch_table_bytes<OPB>() + WindowSize<OPB>::value * (kRkStride * 4 + sizeof(Slot));
}

// ---------------------------------------------------------------- scan ----

// Validation and block count of message m: its status and (for a valid
// message) its 16-byte blocks and output length (0 for a decryption, whose
// length is known after the padding check).  A rejected message has 0 blocks.
__device__ __forceinline__ uint64_t message_blocks(const BatchArgs& a, uint32_t m, int32_t* status,
                                                   uint64_t* out_len) {
  const uint64_t len = a.in_len[m];
  int32_t st = AES_OK;
  if ((a.in_off[m] | a.out_off[m]) & 15u) st = AES_ERR_ALIGN;
  if (a.keys != nullptr) {
    const uint32_t bits = a.key_bits[m];
    if (bits != 128 && bits != 192 && bits != 256) st = AES_ERR_KEYSIZE;
  } else {
    const uint32_t idx = a.sched_idx[m];
    if (idx >= a.n_sched) {
      st = AES_ERR_ARG;
    } else {
      const uint32_t bits = a.schedules[idx].key_bits, nr = a.schedules[idx].nr;
      if (!((bits == 128 && nr == 10) || (bits == 192 && nr == 12) || (bits == 256 && nr == 14)))
        st = AES_ERR_KEYSIZE;
    }
  }
  uint64_t nb = 0, olen = 0;
  if (a.op == kBatchCtr) {
    nb = (len + 15) / 16;
    olen = len;
  } else if (a.op == kBatchEcbEnc) {
    nb = len / 16 + 1;
    olen = 16 * nb;
  } else {
    if (len == 0 || (len & 15u)) st = AES_ERR_LENGTH;
    nb = len / 16;
    olen = 0;  // set after the padding check
  }
  if (st != AES_OK) nb = olen = 0;
  *status = st;
  *out_len = olen;
  return nb;
}

// Rounds of message m's key (valid once message_blocks accepted it).
__device__ __forceinline__ uint32_t message_rounds(const BatchArgs& a, uint32_t m) {
  return a.keys != nullptr ? a.key_bits[m] / 32 + 6 : a.schedules[a.sched_idx[m]].nr;
}

// Bin of a short CTR message on the lane path: its key-size class, then
// longest first.
__device__ __forceinline__ uint32_t lane_bin_of(uint32_t nr, uint64_t nb) {
  return (nr - 10) / 2 * 512 + (511 - static_cast<uint32_t>(nb));
}

// Count-kernel step for message m: write its status and output length and
// return its size in the long-message block space (0 for short messages).
// On the lane path (lane_hist: the CTA's bin counts in shared memory, then
// its count of short messages left to the per-warp groups) a message of
// fewer than kLaneMax blocks also gets its bin, counted in lane_hist.
__device__ __forceinline__ uint64_t count_blocks(const BatchArgs& a, uint32_t m, uint32_t* lane_hist) {
  int32_t st;
  uint64_t olen;
  const uint64_t nb = message_blocks(a, m, &st, &olen);
  if (a.status) a.status[m] = st;
  if (a.out_len) a.out_len[m] = olen;
  if (lane_hist != nullptr) {
    uint16_t bin = kLaneNoBin;
    if (nb > 0 && nb < kLaneMax) {  // nb > 0: the message was accepted
      const uint32_t b = lane_bin_of(message_rounds(a, m), nb);
      atomicAdd(lane_hist + b, 1u);
      bin = static_cast<uint16_t>(b);
    } else if (nb >= kLaneMax && nb < kShortMax) {
      atomicAdd(lane_hist + kLaneBins, 1u);
    }
    a.lane_bin[m] = bin;
  }
  return nb >= kShortMax ? nb : 0;
}

// On the lane path: whether the persistent kernel's per-warp groups have
// short messages to run (those of kLaneMax blocks or more).
__device__ __forceinline__ bool groups_have_work(const BatchArgs& a) {
  return a.lane_bin == nullptr || a.lane_cursor[kLaneBins] != 0;
}

// Exclusive scan of one value per thread across the CTA; *total = CTA sum.
__device__ __forceinline__ uint64_t cta_exclusive_scan(uint64_t v, uint64_t* sh, uint64_t* total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= static_cast<uint32_t>(o)) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < nwarps ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= static_cast<uint32_t>(o)) w += y;
    }
    sh[32 + lane] = w;  // inclusive warp prefixes
  }
  __syncthreads();
  const uint64_t before = warp ? sh[32 + warp - 1] : 0;
  *total = sh[32 + nwarps - 1];
  __syncthreads();  // sh may be reused by the caller
  return before + x - v;
}

// Messages per chunk of the count kernel (one CTA).
constexpr uint32_t kChunkMsgs = kScanThreads * kScanItems;

// First block of message m in the long-message space (m == n: the total).
__device__ __forceinline__ uint64_t blk_start(const BatchArgs& a, uint64_t m) {
  return m >= a.n ? a.blk_off[a.n] : a.blk_off[m] + a.chunk_sum[m / kChunkMsgs];
}

#if !defined(AES_BATCH_REGKEYS_TU) && !defined(AES_BATCH_LANES_TU)  // run from aes_batch.cu's entry point only
// Lane path, by the count kernel's last CTA: each bin's first position in
// lane_order (each key-size class from a multiple of 32), written over the
// bin counts; the class gaps filled with kLaneNoMsg; the chunk range of each
// class.  Threads 512.. add nothing to the scans.
__device__ void lane_bin_starts(const BatchArgs& a, uint64_t* sh) {
  uint64_t base = 0;  // first position of the class
  for (uint32_t c = 0; c < 3; ++c) {
    const uint32_t b = c * 512 + threadIdx.x;
    uint64_t total;
    const uint64_t ex = cta_exclusive_scan(threadIdx.x < 512 ? __ldcg(a.lane_hist + b) : 0, sh, &total);
    if (threadIdx.x < 512) a.lane_hist[b] = static_cast<uint32_t>(base + ex);
    const uint64_t end = base + total, next = (end + 31) & ~static_cast<uint64_t>(31);
    if (threadIdx.x < next - end) a.lane_order[end + threadIdx.x] = kLaneNoMsg;
    if (threadIdx.x == 0) a.lane_info[1 + c] = static_cast<uint32_t>(base / 32);
    base = next;
  }
  if (threadIdx.x == 0) a.lane_info[0] = a.lane_info[4] = static_cast<uint32_t>(base / 32);
}

__global__ void __launch_bounds__(kScanThreads, 2) batch_count_scan(const BatchArgs a) {
  __shared__ uint64_t sh[64];
  __shared__ uint32_t lane_hist[kLaneBins + 1];  // the lane path's bin counts of this CTA's messages, and
                                                 // its short messages left to the per-warp groups
  __shared__ bool s_last;
  const bool lanes = a.lane_bin != nullptr;
  if (lanes) {
    for (uint32_t i = threadIdx.x; i <= kLaneBins; i += blockDim.x) lane_hist[i] = 0;
    __syncthreads();
  }
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kChunkMsgs + static_cast<uint64_t>(threadIdx.x) * kScanItems;
  uint64_t cnt[kScanItems], sum = 0;
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    const uint64_t m = base + k;
    cnt[k] = m < a.n ? count_blocks(a, static_cast<uint32_t>(m), lanes ? lane_hist : nullptr) : 0;
    sum += cnt[k];
  }
  uint64_t total;
  uint64_t run = cta_exclusive_scan(sum, sh, &total);  // its barriers also order the bin counts
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    const uint64_t m = base + k;
    if (m < a.n) a.blk_off[m] = run;  // from the chunk's first block
    run += cnt[k];
  }
  if (lanes) {
    for (uint32_t i = threadIdx.x; i < kLaneBins; i += blockDim.x)
      if (lane_hist[i] != 0) atomicAdd(a.lane_hist + i, lane_hist[i]);
    if (threadIdx.x == 0 && lane_hist[kLaneBins] != 0) atomicAdd(a.lane_cursor + kLaneBins, lane_hist[kLaneBins]);
  }
  if (threadIdx.x == 0) a.chunk_sum[blockIdx.x] = total;
  // The last CTA to finish turns the chunk totals into chunk offsets and
  // writes the grand total (and, on the lane path, the bin starts).
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(a.scan_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  uint64_t carry = 0;
  for (uint32_t c0 = 0; c0 < a.nchunks; c0 += blockDim.x) {
    const uint32_t c = c0 + threadIdx.x;
    const uint64_t v = c < a.nchunks ? __ldcg(a.chunk_sum + c) : 0;  // other CTAs' totals, from L2
    uint64_t t;
    const uint64_t ex = cta_exclusive_scan(v, sh, &t);
    if (c < a.nchunks) a.chunk_sum[c] = carry + ex;
    carry += t;
  }
  if (threadIdx.x == 0) a.blk_off[a.n] = carry;
  if (lanes) lane_bin_starts(a, sh);
}
#endif  // !AES_BATCH_REGKEYS_TU && !AES_BATCH_LANES_TU

// ------------------------------------------------------------ persistent ----

// Largest m in [0, n) with blk_start(m) <= g (non-decreasing, blk_start(0) = 0),
// by a 32-way search: each step narrows the range 32-fold.  Whole warp calls.
__device__ __forceinline__ uint32_t warp_find(const BatchArgs& a, uint32_t n, uint64_t g) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t step = (hi - lo + 31) / 32;
    const uint64_t idx = static_cast<uint64_t>(lo) + static_cast<uint64_t>(lane) * step;
    const bool ok = lane == 0 || (idx < hi && blk_start(a, idx) <= g);
    const uint32_t mask = __ballot_sync(0xffffffffu, ok);
    const uint32_t last = 31 - __clz(mask);
    lo = lo + last * step;
    hi = min(hi, lo + step);
  }
  return lo;
}

// S(x) for each byte of w.  `sb` points at a replicated table whose byte 0 is S(x).
__device__ __forceinline__ uint32_t sub_word(const Tabs& T, const char* sb, uint32_t off,
                                             uint32_t w) {
  const uint32_t a = T.ld(sb, w, off, 0x5504), b = T.ld(sb, w, off, 0x5514);
  const uint32_t c = T.ld(sb, w, off, 0x5524), d = T.ld(sb, w, off, 0x5534);
  return __byte_perm(__byte_perm(a, b, 0x0040), __byte_perm(c, d, 0x0040), 0x5410);
}

__device__ __forceinline__ uint32_t load_le32(const uint8_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// FIPS-197 §5.2 into rk[0 .. 4(nr+1)).  key: 4-byte aligned, NK words.  The
// last NK words live in registers (w[i mod NK]), so the dependency chain has
// no shared-memory round trips; rk[] is only written.
template <int NK>
__device__ __forceinline__ void expand_key_nk(const Tabs& T, const char* sb, uint32_t sb_off,
                                              const uint8_t* key, uint32_t* rk) {
  constexpr int kWords = 4 * (NK + 7);
  uint32_t w[NK];
  uint32_t q[4];  // the round key being assembled: written as one 128-bit store (rk is 16-byte aligned)
#pragma unroll
  for (int i = 0; i < NK; ++i) {
    w[i] = load_le32(key + 4 * i);
    q[i & 3] = w[i];
    if ((i & 3) == 3) *reinterpret_cast<uint4*>(rk + i - 3) = make_uint4(q[0], q[1], q[2], q[3]);
  }
  uint32_t rcon = 1;
#pragma unroll
  for (int i = NK; i < kWords; ++i) {
    uint32_t t = w[(i - 1) % NK];
    if (i % NK == 0) {
      t = sub_word(T, sb, sb_off, __funnelshift_r(t, t, 8)) ^ rcon;  // RotWord, SubWord, Rcon
      rcon = ((rcon << 1) ^ ((rcon & 0x80u) ? 0x1Bu : 0u)) & 0xFFu;
    } else if (NK == 8 && i % NK == 4) {
      t = sub_word(T, sb, sb_off, t);
    }
    w[i % NK] ^= t;  // w[i] = w[i - NK] ^ t
    q[i & 3] = w[i % NK];
    if ((i & 3) == 3) *reinterpret_cast<uint4*>(rk + i - 3) = make_uint4(q[0], q[1], q[2], q[3]);
  }
}

__device__ void expand_key(const Tabs& T, const char* sb, uint32_t sb_off, const uint8_t* key,
                           uint32_t nk, uint32_t* rk) {
  if (nk == 4) expand_key_nk<4>(T, sb, sb_off, key, rk);
  else if (nk == 6) expand_key_nk<6>(T, sb, sb_off, key, rk);
  else expand_key_nk<8>(T, sb, sb_off, key, rk);
}

// Turn an encryption schedule into the equivalent inverse cipher's (FIPS-197
// §5.3.5), in place.  InvMixColumns(w) = sum_i TDi[S(byte i of w)], since each
// td word applies the inverse S-box first.  One unit (r <= nr / 2, column c)
// swaps word c of rounds r and nr - r, applying InvMixColumns to each unless
// it lands in round 0 or nr; units touch disjoint words, so they may run on
// different threads at once.
__device__ __forceinline__ void decrypt_schedule_unit(const Tabs& T, const char* sb, uint32_t sb_off,
                                                      uint32_t nr, uint32_t* rk, uint32_t r, uint32_t c) {
  auto inv_mix = [&](uint32_t w) {
    const uint32_t s = sub_word(T, sb, sb_off, w);
    return T.t0(s) ^ T.t1(s) ^ T.t2(s) ^ T.t3(s);
  };
  const uint32_t q = nr - r;
  const uint32_t a = rk[4 * r + c], b = rk[4 * q + c];
  const uint32_t na = (q == 0 || q == nr) ? b : inv_mix(b);  // new round r from old round q
  const uint32_t nb = (r == 0 || r == nr) ? a : inv_mix(a);  // new round q from old round r
  rk[4 * r + c] = na;
  if (q != r) rk[4 * q + c] = nb;
}

__device__ void to_decrypt_schedule(const Tabs& T, const char* sb, uint32_t sb_off, uint32_t nr,
                                    uint32_t* rk) {
  for (uint32_t r = 0; r <= nr / 2; ++r)
    for (uint32_t c = 0; c < 4; ++c) decrypt_schedule_unit(T, sb, sb_off, nr, rk, r, c);
}

__device__ __forceinline__ uint4 lds128(const uint32_t* p) {
  return *reinterpret_cast<const uint4*>(p);
}

template <int NR>
__device__ __forceinline__ State enc_rounds_smem(const Tabs& T, State s, const uint32_t* rk,
                                                 int first) {
#pragma unroll
  for (int r = 1; r < NR; ++r) {
    if (r < first) continue;
    const uint4 k = lds128(rk + 4 * r);
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
    enc_round(T, s, kk);
  }
  const uint4 k = lds128(rk + 4 * NR);
  const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
  enc_final(T, s, kk);
  return s;
}

template <int NR>
__device__ __forceinline__ State dec_rounds_smem(const Tabs& T, State s, const uint32_t* rk) {
#pragma unroll
  for (int r = 1; r < NR; ++r) {
    const uint4 k = lds128(rk + 4 * r);
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
    dec_round(T, s, kk);
  }
  const uint4 k = lds128(rk + 4 * NR);
  const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
  dec_final(T, s, kk);
  return s;
}

__device__ __forceinline__ State enc_any(const Tabs& T, State s, const uint32_t* rk, uint32_t nr,
                                         int first) {
  switch (nr) {
    case 10: return enc_rounds_smem<10>(T, s, rk, first);
    case 12: return enc_rounds_smem<12>(T, s, rk, first);
    default: return enc_rounds_smem<14>(T, s, rk, first);
  }
}

__device__ __forceinline__ State dec_any(const Tabs& T, State s, const uint32_t* rk, uint32_t nr) {
  switch (nr) {
    case 10: return dec_rounds_smem<10>(T, s, rk);
    case 12: return dec_rounds_smem<12>(T, s, rk);
    default: return dec_rounds_smem<14>(T, s, rk);
  }
}

// Rounds for a warp whose lanes may hold keys of different sizes.  Rounds
// 1..9 are full rounds for every key size; rounds 10..13 run up to the
// warp's largest round count, each lane masked to its own, then every lane
// takes its final round.  One compact body serves all sizes: per-size
// unrolled copies interleaved in one warp thrash the instruction cache.
__device__ __forceinline__ State enc_lanes(const Tabs& T, State s, const uint32_t* rk, uint32_t nr,
                                           int first) {
  const uint32_t nr_max = __reduce_max_sync(__activemask(), nr);
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    if (r < first) continue;
    const uint4 k = lds128(rk + 4 * r);
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
    enc_round(T, s, kk);
  }
#pragma unroll
  for (int r = 10; r < 14; ++r) {
    if (static_cast<uint32_t>(r) >= nr_max) break;
    if (static_cast<uint32_t>(r) < nr) {
      const uint4 k = lds128(rk + 4 * r);
      const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
      enc_round(T, s, kk);
    }
  }
  const uint4 k = lds128(rk + 4 * nr);
  const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
  enc_final(T, s, kk);
  return s;
}

__device__ __forceinline__ State dec_lanes(const Tabs& T, State s, const uint32_t* rk, uint32_t nr) {
  const uint32_t nr_max = __reduce_max_sync(__activemask(), nr);
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    const uint4 k = lds128(rk + 4 * r);
    const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
    dec_round(T, s, kk);
  }
#pragma unroll
  for (int r = 10; r < 14; ++r) {
    if (static_cast<uint32_t>(r) >= nr_max) break;
    if (static_cast<uint32_t>(r) < nr) {
      const uint4 k = lds128(rk + 4 * r);
      const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
      dec_round(T, s, kk);
    }
  }
  const uint4 k = lds128(rk + 4 * nr);
  const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
  dec_final(T, s, kk);
  return s;
}

__device__ __forceinline__ uint32_t state_byte(const State& s, uint32_t k) {
  const uint32_t w = k < 4 ? s.s0 : k < 8 ? s.s1 : k < 12 ? s.s2 : s.s3;
  return (w >> (8 * (k & 3))) & 0xFFu;
}

// Fill a slot with message m occupying blocks [blk_start, blk_end) of the
// block space being worked on: block range, addresses, key schedule, CTR
// constants.
template <int OPB>
__device__ void fill_slot(const BatchArgs& a, const Tabs& T, const char* sb, uint32_t sb_off,
                          uint32_t m, uint64_t blk_start, uint64_t blk_end, Slot& sl, uint32_t* rk) {
  sl.blk_start = blk_start;
  sl.blk_end = blk_end;
  sl.msg = m;
  sl.nr = 10;
  if (sl.blk_end == sl.blk_start) return;  // empty or rejected: never selected
  const uint64_t len = a.in_len[m];
  sl.rem = static_cast<uint32_t>(len & 15u);
  sl.full_end = sl.blk_start + len / 16;
  sl.src0 = reinterpret_cast<uint64_t>(a.in) + a.in_off[m] - 16 * sl.blk_start;
  sl.dst0 = reinterpret_cast<uint64_t>(a.out) + a.out_off[m] - 16 * sl.blk_start;
  if (a.keys != nullptr) {
    const uint32_t bits = a.key_bits[m];
    const uint32_t nk = bits / 32, nr = nk + 6;
    sl.nr = nr;
    expand_key(T, sb, sb_off, a.keys + 32ull * m, nk, rk);
    if (OPB == kBatchEcbDec) to_decrypt_schedule(T, sb, sb_off, nr, rk);
  } else {
    const aes_key_schedule& ks = a.schedules[a.sched_idx[m]];
    const uint32_t nr = ks.nr;
    sl.nr = nr;
    const uint32_t* src = OPB == kBatchEcbDec ? ks.rk_dec : ks.rk_enc;
    const uint32_t nw = 4 * (nr + 1);
    // read-only loads, independent of the shared-memory stores: all in flight together
#pragma unroll
    for (uint32_t i = 0; i < 60; ++i)
      if (i < nw) rk[i] = __ldg(src + i);
  }
  if (OPB == kBatchCtr) {
    const uint4 ivw = *reinterpret_cast<const uint4*>(a.iv + 16ull * m);
    const uint32_t iv_w[4] = {ivw.x, ivw.y, ivw.z, ivw.w};
    sl.ctr_base = __byte_perm(ivw.w, 0, 0x0123) - static_cast<uint32_t>(sl.blk_start);
    uint32_t s[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] = iv_w[c] ^ rk[c];
    s[3] = 0;  // the counter column: looked up per block
    rk[kCtrRk0w3] = rk[3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t acc = rk[4 + j];
      // row i of round-1 column j comes from column j+i; column 3 (the counter) stays on the device
      if (((j + 0) & 3) != 3) acc ^= T.t0(s[(j + 0) & 3]);
      if (((j + 1) & 3) != 3) acc ^= T.t1(s[(j + 1) & 3]);
      if (((j + 2) & 3) != 3) acc ^= T.t2(s[(j + 2) & 3]);
      if (((j + 3) & 3) != 3) acc ^= T.t3(s[(j + 3) & 3]);
      rk[kCtrC1 + j] = acc;
    }
  }
}

// A window slot of the tile phase: message m at its place in the long-message space.
template <int OPB>
__device__ __forceinline__ void load_slot(const BatchArgs& a, const Tabs& T, const char* sb,
                                          uint32_t sb_off, uint32_t m, Slot& sl, uint32_t* rk) {
  fill_slot<OPB>(a, T, sb, sb_off, m, blk_start(a, m), blk_start(a, m + 1ull), sl, rk);
}

// The message a thread is working in, cached in registers and rebased to the
// tile: blocks t0 + [s, e) of the tile belong to it, blocks below f are whole.
struct Cur {
  uint32_t s, e, f;
  uint32_t nr;     // rounds | rem << 8 | (message ends in this tile) << 16
  uint32_t ctr;    // counter of tile block 0 (CTR)
  uint32_t slot;
  uint64_t src, dst;  // byte address of tile block 0 in this message's input / output
};

// The message of tile block gr.  A thread's blocks only move forward through
// a window, so the search starts at its current slot and steps forward a few
// slots (short messages: usually one step) before falling back to a binary
// search over the rest of the window.
__device__ __forceinline__ void select_message(const Slot* slots, uint32_t wn, uint64_t t0,
                                               uint64_t t1, uint32_t gr, Cur& c) {
  const uint64_t g = t0 + gr;
  uint32_t lo = c.slot, hi = wn;  // last slot whose first block is <= g, in [lo, hi)
#pragma unroll 1
  for (int i = 0; i < 3 && lo + 1 < hi; ++i) {
    if (slots[lo + 1].blk_start > g) hi = lo + 1;
    else ++lo;
  }
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (slots[mid].blk_start <= g) lo = mid;
    else hi = mid;
  }
  const Slot& sl = slots[lo];
  const uint64_t bs = max(sl.blk_start, t0), be = min(sl.blk_end, t1);
  const uint64_t bf = min(max(sl.full_end, t0), t1);
  c.s = static_cast<uint32_t>(bs - t0);
  c.e = static_cast<uint32_t>(be - t0);
  c.f = static_cast<uint32_t>(bf - t0);
  c.nr = sl.nr | (sl.rem << 8) | ((sl.blk_end <= t1 ? 1u : 0u) << 16);
  c.ctr = sl.ctr_base + static_cast<uint32_t>(t0);
  c.slot = lo;
  c.src = sl.src0 + 16 * t0;
  c.dst = sl.dst0 + 16 * t0;
}

// Bytes [0, n) of a 16-byte-aligned block, zero above (n < 16): whole words
// first, then the bytes of the last word.  Every load is independent of the
// others, so they are in flight together.
__device__ __forceinline__ uint4 load_partial(const uint8_t* p, uint32_t n) {
  uint32_t w[4] = {0, 0, 0, 0};
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) {
    if (4 * q + 4 <= n) {
      w[q] = __ldcs(reinterpret_cast<const unsigned int*>(p + 4 * q));
    } else {
#pragma unroll
      for (uint32_t b = 0; b < 3; ++b)
        if (4 * q + b < n) w[q] |= static_cast<uint32_t>(__ldcs(p + 4 * q + b)) << (8 * b);
    }
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Store bytes [0, n) of v at a 16-byte-aligned address (n < 16).
__device__ __forceinline__ void store_partial(uint8_t* p, const uint4& v, uint32_t n) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (uint32_t q = 0; q < 4; ++q) {
    if (4 * q + 4 <= n) {
      __stcs(reinterpret_cast<unsigned int*>(p + 4 * q), w[q]);
    } else {
#pragma unroll
      for (uint32_t b = 0; b < 3; ++b)
        if (4 * q + b < n) p[4 * q + b] = static_cast<uint8_t>(w[q] >> (8 * b));
    }
  }
}

// Input of tile block gr of the current message: a whole block, or the
// leading `rem` bytes of the last one (zero above).
// (With AES_BATCH_IN_PADDED a ragged last block is read whole: the bytes past
// the message up to the 16-byte boundary are the caller's padding.  A last
// block without message bytes, the PKCS#7 block of an aligned length, is
// never read.)
template <int OPB>
__device__ __forceinline__ uint4 load_block(const BatchArgs& a, const Cur& c, uint32_t gr) {
  const uint32_t rem = (c.nr >> 8) & 0xFFu;
  if (OPB == kBatchEcbDec || gr < c.f || (rem != 0 && (a.flags & AES_BATCH_IN_PADDED)))
    return __ldcs(reinterpret_cast<const uint4*>(c.src + 16ull * gr));
  return load_partial(reinterpret_cast<const uint8_t*>(c.src + 16ull * gr), rem);
}

// Per-thread cache of one CTR counter run (256 aligned counters of one
// message): after round 1 only column 0 depends on the counter's low byte,
// so round 2 is d_j ^ (one lookup) for the whole run.
struct RunCache {
  uint32_t run, slot;    // counter >> 8 and window slot + 1 (0: empty)
  uint32_t xr, c10;      // counter word of the run start ^ rk0 word 3; folded round-1 column 0
  uint32_t d0, d1, d2, d3;
};

template <int OPB>
__device__ __forceinline__ void process_block(const BatchArgs& a, const Tabs& T, const Slot* slots,
                                              const uint32_t* rk, const Cur& c, uint32_t gr,
                                              const uint4& v_in, RunCache& rc) {
  const uint32_t nr = c.nr & 0xFFu, rem = (c.nr >> 8) & 0xFFu;
  const bool full = gr < c.f;
  uint8_t* dst = reinterpret_cast<uint8_t*>(c.dst + 16ull * gr);
  if (OPB == kBatchCtr) {
    const uint32_t ctr = c.ctr + gr;
    // tile-phase messages are long (>= kShortMax blocks): counter runs are cached per lane
    if ((ctr >> 8) != rc.run || c.slot + 1 != rc.slot) {  // a new run: its round-1/2 constants
      rc.run = ctr >> 8;
      rc.slot = c.slot + 1;
      rc.xr = __byte_perm(ctr & ~255u, 0, 0x0123) ^ rk[kCtrRk0w3];
      const uint4 c1 = lds128(rk + kCtrC1);
      rc.c10 = c1.x;
      const uint32_t s1 = c1.y ^ T.t2(rc.xr), s2 = c1.z ^ T.t1(rc.xr), s3 = c1.w ^ T.t0(rc.xr);
      const uint4 k2 = lds128(rk + 8);
      rc.d0 = k2.x ^ T.t1(s1) ^ T.t2(s2) ^ T.t3(s3);
      rc.d1 = k2.y ^ T.t0(s1) ^ T.t1(s2) ^ T.t2(s3);
      rc.d2 = k2.z ^ T.t0(s2) ^ T.t1(s3) ^ T.t3(s1);
      rc.d3 = k2.w ^ T.t0(s3) ^ T.t2(s1) ^ T.t3(s2);
    }
    const uint32_t s0 = rc.c10 ^ T.t3(rc.xr ^ ((ctr & 255u) << 24));
    State s{rc.d0 ^ T.t0(s0), rc.d1 ^ T.t3(s0), rc.d2 ^ T.t2(s0), rc.d3 ^ T.t1(s0)};
    s = enc_any(T, s, rk, nr, 3);
    if (full || (a.flags & AES_BATCH_OUT_PADDED)) {
      __stcs(reinterpret_cast<uint4*>(dst),
             make_uint4(v_in.x ^ s.s0, v_in.y ^ s.s1, v_in.z ^ s.s2, v_in.w ^ s.s3));
    } else {  // partial last block (v_in holds its `rem` bytes): the leading `rem` bytes
      store_partial(dst, make_uint4(v_in.x ^ s.s0, v_in.y ^ s.s1, v_in.z ^ s.s2, v_in.w ^ s.s3), rem);
    }
  } else if (OPB == kBatchEcbEnc) {
    uint4 v = v_in;
    if (!full) {  // last block: rem message bytes (in v_in) then PKCS#7 pad bytes of value 16 - rem
      const uint32_t pad = (16 - rem) * 0x01010101u;
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t keep = rem >= 4 * q + 4 ? 4 : rem > 4 * q ? rem - 4 * q : 0;  // message bytes in word q
        const uint32_t mask = keep == 4 ? 0xFFFFFFFFu : (1u << (8 * keep)) - 1;
        w[q] = (w[q] & mask) | (pad & ~mask);
      }
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    const uint4 k0 = lds128(rk);
    State s{v.x ^ k0.x, v.y ^ k0.y, v.z ^ k0.z, v.w ^ k0.w};
    s = enc_any(T, s, rk, nr, 1);
    __stcs(reinterpret_cast<uint4*>(dst), make_uint4(s.s0, s.s1, s.s2, s.s3));
  } else {
    const uint4 k0 = lds128(rk);
    State s{v_in.x ^ k0.x, v_in.y ^ k0.y, v_in.z ^ k0.z, v_in.w ^ k0.w};
    s = dec_any(T, s, rk, nr);
    __stcs(reinterpret_cast<uint4*>(dst), make_uint4(s.s0, s.s1, s.s2, s.s3));
    if (((c.nr >> 16) & 1u) && gr + 1 == c.e) {  // the message's last block: check PKCS#7
      const Slot& sl = slots[c.slot];
      const uint32_t p = state_byte(s, 15);
      bool ok = p >= 1 && p <= 16;
      for (uint32_t k = 16 - (ok ? p : 0); k < 16; ++k) ok = ok && state_byte(s, k) == p;
      if (a.status) a.status[sl.msg] = ok ? AES_OK : AES_ERR_PADDING;
      if (a.out_len) a.out_len[sl.msg] = ok ? 16 * (sl.blk_end - sl.blk_start) - p : 0;
    }
  }
}

// Round-key source of the span loop: shared memory (one 128-bit broadcast
// load per round), or registers loaded once per span (kRegKeys: 512-thread
// CTAs, whose 128 registers per thread hold a whole schedule).
template <int NR, bool kRegKeys, int kFirstWord>
struct SpanKeys {
  uint32_t w[kRegKeys ? 4 * (NR + 1) - kFirstWord : 1];
  const uint32_t* rk;
  __device__ __forceinline__ explicit SpanKeys(const uint32_t* src) : rk(src) {
    if (kRegKeys) {
#pragma unroll
      for (int i = kFirstWord; i < 4 * (NR + 1); i += 4) {
        const uint4 k = lds128(src + i);
        w[i - kFirstWord] = k.x;
        w[i - kFirstWord + 1] = k.y;
        w[i - kFirstWord + 2] = k.z;
        w[i - kFirstWord + 3] = k.w;
      }
    }
  }
  // words 4r .. 4r+3
  __device__ __forceinline__ void round(int r, uint32_t kk[4]) const {
    if (kRegKeys) {
#pragma unroll
      for (int j = 0; j < 4; ++j) kk[j] = w[4 * r - kFirstWord + j];
    } else {
      const uint4 k = lds128(rk + 4 * r);
      kk[0] = k.x;
      kk[1] = k.y;
      kk[2] = k.z;
      kk[3] = k.w;
    }
  }
};

template <int NR, bool kRegKeys, int kFirstWord>
__device__ __forceinline__ State enc_rounds_keys(const Tabs& T, State s, const SpanKeys<NR, kRegKeys, kFirstWord>& K,
                                                 int first) {
#pragma unroll
  for (int r = 1; r < NR; ++r) {
    if (r < first) continue;
    uint32_t kk[4];
    K.round(r, kk);
    enc_round(T, s, kk);
  }
  uint32_t kk[4];
  K.round(NR, kk);
  enc_final(T, s, kk);
  return s;
}

template <int NR, bool kRegKeys>
__device__ __forceinline__ State dec_rounds_keys(const Tabs& T, State s, const SpanKeys<NR, kRegKeys, 0>& K) {
#pragma unroll
  for (int r = 1; r < NR; ++r) {
    uint32_t kk[4];
    K.round(r, kk);
    dec_round(T, s, kk);
  }
  uint32_t kk[4];
  K.round(NR, kk);
  dec_final(T, s, kk);
  return s;
}

// A whole span (256 blocks) inside one message, every block whole: the same
// work as process_block with the round count fixed and no per-block checks.
template <int OPB, int NR, bool kRegKeys>
__device__ __forceinline__ void span_fast(const BatchArgs& a, const Tabs& T, const Slot* slots,
                                          const uint32_t* rk, const Cur& c, uint32_t span,
                                          uint32_t lane, RunCache& rc) {
  // CTR's rounds 1-2 come from the run cache: its loop reads keys from round 3
  constexpr int kFirstWord = OPB == kBatchCtr ? 12 : 0;
  const SpanKeys<NR, kRegKeys, kFirstWord> K(rk);
  const uint4* src = reinterpret_cast<const uint4*>(c.src) + span + lane;
  uint4* dst = reinterpret_cast<uint4*>(c.dst) + span + lane;
  uint4 v = __ldcs(src);
#pragma unroll 1
  for (uint32_t k = 0; k < 8; ++k) {
    uint4 vn = v;
    if (k < 7) vn = __ldcs(src + 32 * (k + 1));
    State s;
    if constexpr (OPB == kBatchCtr) {
      const uint32_t ctr = c.ctr + span + 32 * k + lane;
      if ((ctr >> 8) != rc.run || c.slot + 1 != rc.slot) {
        rc.run = ctr >> 8;
        rc.slot = c.slot + 1;
        rc.xr = __byte_perm(ctr & ~255u, 0, 0x0123) ^ rk[kCtrRk0w3];
        const uint4 c1 = lds128(rk + kCtrC1);
        rc.c10 = c1.x;
        const uint32_t s1 = c1.y ^ T.t2(rc.xr), s2 = c1.z ^ T.t1(rc.xr), s3 = c1.w ^ T.t0(rc.xr);
        const uint4 k2 = lds128(rk + 8);
        rc.d0 = k2.x ^ T.t1(s1) ^ T.t2(s2) ^ T.t3(s3);
        rc.d1 = k2.y ^ T.t0(s1) ^ T.t1(s2) ^ T.t2(s3);
        rc.d2 = k2.z ^ T.t0(s2) ^ T.t1(s3) ^ T.t3(s1);
        rc.d3 = k2.w ^ T.t0(s3) ^ T.t2(s1) ^ T.t3(s2);
      }
      const uint32_t s0 = rc.c10 ^ T.t3(rc.xr ^ ((ctr & 255u) << 24));
      s = State{rc.d0 ^ T.t0(s0), rc.d1 ^ T.t3(s0), rc.d2 ^ T.t2(s0), rc.d3 ^ T.t1(s0)};
      s = enc_rounds_keys<NR>(T, s, K, 3);
      __stcs(dst + 32 * k, make_uint4(v.x ^ s.s0, v.y ^ s.s1, v.z ^ s.s2, v.w ^ s.s3));
    } else if constexpr (OPB == kBatchEcbEnc) {
      uint32_t k0[4];
      K.round(0, k0);
      s = State{v.x ^ k0[0], v.y ^ k0[1], v.z ^ k0[2], v.w ^ k0[3]};
      s = enc_rounds_keys<NR>(T, s, K, 1);
      __stcs(dst + 32 * k, make_uint4(s.s0, s.s1, s.s2, s.s3));
    } else {
      uint32_t k0[4];
      K.round(0, k0);
      s = State{v.x ^ k0[0], v.y ^ k0[1], v.z ^ k0[2], v.w ^ k0[3]};
      s = dec_rounds_keys<NR>(T, s, K);
      __stcs(dst + 32 * k, make_uint4(s.s0, s.s1, s.s2, s.s3));
      const uint32_t gr = span + 32 * k + lane;
      if (((c.nr >> 16) & 1u) && gr + 1 == c.e) {  // the message's last block: check PKCS#7
        const Slot& sl = slots[c.slot];
        const uint32_t p = state_byte(s, 15);
        bool ok = p >= 1 && p <= 16;
        for (uint32_t q = 16 - (ok ? p : 0); q < 16; ++q) ok = ok && state_byte(s, q) == p;
        if (a.status) a.status[sl.msg] = ok ? AES_OK : AES_ERR_PADDING;
        if (a.out_len) a.out_len[sl.msg] = ok ? 16 * (sl.blk_end - sl.blk_start) - p : 0;
      }
    }
    v = vn;
  }
}

// Blocks g_begin + 32k + lane < g_end of the slots' block space (tile blocks
// t0 + gr), each in the message select_message finds for it; the lane's next
// block is loaded before the current one's rounds when it is in the same message.
template <int OPB>
__device__ __forceinline__ void run_blocks(const BatchArgs& a, const Tabs& T, const Slot* slots,
                                           const uint32_t* rk_all, uint32_t wn, uint64_t t0, uint64_t t1,
                                           uint32_t g_begin, uint32_t g_end, uint32_t lane, Cur& c,
                                           RunCache& rc) {
  uint4 next = make_uint4(0, 0, 0, 0);
  bool have_next = false;
#pragma unroll 1
  for (uint32_t gr = g_begin + lane; gr < g_end; gr += 32) {
    if (gr < c.s || gr >= c.e) select_message(slots, wn, t0, t1, gr, c);
    uint4 v = next;
    if (!have_next) v = load_block<OPB>(a, c, gr);
    const uint32_t gn = gr + 32;
    have_next = gn < g_end && gn < c.e;
    if (have_next) next = load_block<OPB>(a, c, gn);
    process_block<OPB>(a, T, slots, rk_all + c.slot * kRkStride, c, gr, v, rc);
  }
}

// Tile size when the caller gives none: about 4 tiles per CTA of the
// long-message blocks (so CTAs finish close together while each tile's
// serial part, the claim, window load and barriers, stays small against
// its blocks), a whole number of CTA widths, at most 65536 blocks (measured
// best for large batches).
__device__ __forceinline__ uint32_t auto_tile(uint64_t total, uint32_t ctas, uint32_t cta_threads) {
  uint64_t t = (total + 4ull * ctas - 1) / (4ull * ctas);
  t = (t + cta_threads - 1) / cta_threads * cta_threads;
  return static_cast<uint32_t>(t < cta_threads ? cta_threads : t > 65536 ? 65536 : t);
}

// Warp 0: claim the next tile and find its first and last message.
__device__ __forceinline__ void claim_tile(const BatchArgs& a, uint64_t total, uint32_t tile,
                                           unsigned long long* s_tile, uint32_t* s_mlo,
                                           uint32_t* s_mhi) {
  const uint32_t lane = threadIdx.x & 31;
  unsigned long long t = 0;
  if (lane == 0) t = atomicAdd(a.tile_counter, 1ull);
  t = __shfl_sync(0xffffffffu, t, 0);
  const uint64_t t0 = t * tile;
  uint32_t mlo = 0, mhi = 0;
  if (t0 < total) {
    mlo = warp_find(a, a.n, t0);
    mhi = warp_find(a, a.n, min(t0 + tile, total) - 1);
  }
  if (lane == 0) {
    *s_tile = t;
    *s_mlo = mlo;
    *s_mhi = mhi;
  }
}

// ------------------------------------------------------ short messages ----
//
// After the tile phase every warp works alone on groups of kGroup consecutive
// messages.  A group's valid short messages are numbered by round count,
// then by position (compact index ci), and laid end to end in that order in
// a group block space; lane l of a warp step
// takes group block base + l.  The message of each lane's block follows from
// one ballot (messages starting at or before `base`) and one OR-reduction (a
// bit for every message starting inside the step), so there is no search.

// One message of a group (block numbers relative to the group).
struct GroupMsg {
  uint64_t src0, dst0;  // byte address of (virtual) group block 0 in the message's input / output
  uint32_t ctr0;        // CTR: counter of group block 0; ECB: the message's first group block
  uint32_t info;        // nr | rem << 8 | lane of the message in the group << 16
  uint32_t full_end;    // first group block that is not a whole 16-byte input block
  uint32_t end;         // first group block after the message
};
static_assert(sizeof(GroupMsg) == 32, "two 128-bit loads per record");

// Words per round-key slot in the short phase.  CTR slots add, after the
// round keys (0..59) and the folded round-1 columns (60..63): word 64 the
// round-0 key word 3, 65 the cached counter run (counter >> 8), 66 that run's
// column-3 input xr, 67 its round-1 column 0 without the counter byte, and
// 68..71 its round-2 columns without the column-0 term.
template <int OPB>
constexpr uint32_t kShortStride = OPB == kBatchCtr ? 72 : kRkStride;
constexpr uint32_t kRunWords = 64, kRunD = 68;

// Per-warp region: kGroup round-key slots, kGroup records, kGroup start blocks.
template <int OPB>
constexpr uint32_t kWarpRegion =
    static_cast<uint32_t>(WindowSize<OPB>::value * (kRkStride * 4 + sizeof(Slot)) / 32) & ~15u;
template <int OPB>
constexpr bool region_fits() {
  return kGroup<OPB> * (kShortStride<OPB> * 4 + sizeof(GroupMsg) + 4) <= kWarpRegion<OPB>;
}
static_assert(region_fits<kBatchCtr>() && region_fits<kBatchEcbEnc>() && region_fits<kBatchEcbDec>(),
              "short-phase groups exceed a warp's share of the window region");

// A lane's current message in the short phase, kept in registers while the
// lane's blocks stay in it: its record and, for CTR, the cached counter run
// (run, xr, c10) and that run's round-2 columns d, so a block in the cached
// run reads no per-message word from shared memory.
struct ShortCur {
  GroupMsg r;
  uint32_t run, xr, c10;
  uint4 d;
};

template <int OPB>
__device__ __forceinline__ void load_short_cur(const uint32_t* wrk, const GroupMsg* rec, uint32_t ci,
                                               ShortCur& c) {
  c.r = rec[ci];
  if (OPB == kBatchCtr) {
    const uint32_t* rk = wrk + (c.r.info >> 16) * kShortStride<OPB>;
    const uint4 q = lds128(rk + kRunWords);  // rk0 word 3, cached run, xr, c10
    c.run = q.y;
    c.xr = q.z;
    c.c10 = q.w;
    c.d = lds128(rk + kRunD);
  }
}

template <int OPB>
__device__ __forceinline__ void short_block(const BatchArgs& a, const Tabs& T, const uint32_t* wrk,
                                            const ShortCur& c, uint32_t gr, unsigned long long m0) {
  const GroupMsg& r = c.r;
  const uint32_t nr = r.info & 0xFFu, rem = (r.info >> 8) & 0xFFu, j = r.info >> 16;
  const uint32_t* rk = wrk + j * kShortStride<OPB>;
  const bool full = gr < r.full_end;
  const uint8_t* src = reinterpret_cast<const uint8_t*>(r.src0 + 16ull * gr);
  uint8_t* dst = reinterpret_cast<uint8_t*>(r.dst0 + 16ull * gr);
  uint4 v;  // a ragged last block whole only under AES_BATCH_IN_PADDED; an empty one never
  if (OPB == kBatchEcbDec || full || (rem != 0 && (a.flags & AES_BATCH_IN_PADDED)))
    v = __ldcs(reinterpret_cast<const uint4*>(src));
  else
    v = load_partial(src, rem);
  if (OPB == kBatchCtr) {
    const uint32_t ctr = r.ctr0 + gr;
    uint32_t xr = c.xr;
    uint4 d = c.d;
    if ((ctr >> 8) != c.run) {  // outside the cached run: that run's constants (15 lookups)
      xr = __byte_perm(ctr & ~255u, 0, 0x0123) ^ rk[kCtrRk0w3];
      const uint4 c1 = lds128(rk + kCtrC1), k2 = lds128(rk + 8);
      const uint32_t s1 = c1.y ^ T.t2(xr), s2 = c1.z ^ T.t1(xr), s3 = c1.w ^ T.t0(xr);
      d = make_uint4(k2.x ^ T.t1(s1) ^ T.t2(s2) ^ T.t3(s3), k2.y ^ T.t0(s1) ^ T.t1(s2) ^ T.t2(s3),
                     k2.z ^ T.t0(s2) ^ T.t1(s3) ^ T.t3(s1), k2.w ^ T.t0(s3) ^ T.t2(s1) ^ T.t3(s2));
    }
    // rounds 1-2: only round-1 column 0 depends on the counter's low byte
    const uint32_t s0 = c.c10 ^ T.t3(xr ^ ((ctr & 255u) << 24));
    State s{d.x ^ T.t0(s0), d.y ^ T.t3(s0), d.z ^ T.t2(s0), d.w ^ T.t1(s0)};
    s = enc_lanes(T, s, rk, nr, 3);
    const uint4 o = make_uint4(v.x ^ s.s0, v.y ^ s.s1, v.z ^ s.s2, v.w ^ s.s3);
    if (full || (a.flags & AES_BATCH_OUT_PADDED)) __stcs(reinterpret_cast<uint4*>(dst), o);
    else store_partial(dst, o, rem);
  } else if (OPB == kBatchEcbEnc) {
    if (!full) {  // last block: rem message bytes then PKCS#7 pad bytes of value 16 - rem
      const uint32_t pad = (16 - rem) * 0x01010101u;
      uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (uint32_t q = 0; q < 4; ++q) {
        const uint32_t keep = rem >= 4 * q + 4 ? 4 : rem > 4 * q ? rem - 4 * q : 0;
        const uint32_t mask = keep == 4 ? 0xFFFFFFFFu : (1u << (8 * keep)) - 1;
        w[q] = (w[q] & mask) | (pad & ~mask);
      }
      v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    const uint4 k0 = lds128(rk);
    State s{v.x ^ k0.x, v.y ^ k0.y, v.z ^ k0.z, v.w ^ k0.w};
    s = enc_lanes(T, s, rk, nr, 1);
    __stcs(reinterpret_cast<uint4*>(dst), make_uint4(s.s0, s.s1, s.s2, s.s3));
  } else {
    const uint4 k0 = lds128(rk);
    State s{v.x ^ k0.x, v.y ^ k0.y, v.z ^ k0.z, v.w ^ k0.w};
    s = dec_lanes(T, s, rk, nr);
    __stcs(reinterpret_cast<uint4*>(dst), make_uint4(s.s0, s.s1, s.s2, s.s3));
    if (gr + 1 == r.end) {  // the message's last block: check PKCS#7
      const uint32_t p = state_byte(s, 15);
      bool ok = p >= 1 && p <= 16;
      for (uint32_t q = 16 - (ok ? p : 0); q < 16; ++q) ok = ok && state_byte(s, q) == p;
      const uint32_t m = static_cast<uint32_t>(m0 + j);
      if (a.status) a.status[m] = ok ? AES_OK : AES_ERR_PADDING;
      if (a.out_len) a.out_len[m] = ok ? 16ull * (r.end - r.ctr0) - p : 0;
    }
  }
}

template <int OPB>
__device__ void short_phase(const BatchArgs& a, const Tabs& T, const char* sb, uint32_t sb_off,
                            char* region, uint32_t warp, uint32_t lane) {
  constexpr uint32_t G = kGroup<OPB>;
  char* wbase = region + warp * kWarpRegion<OPB>;
  uint32_t* wrk = reinterpret_cast<uint32_t*>(wbase);
  GroupMsg* rec = reinterpret_cast<GroupMsg*>(wbase + G * kShortStride<OPB> * 4);
  uint32_t* first = reinterpret_cast<uint32_t*>(wbase + G * (kShortStride<OPB> * 4 + sizeof(GroupMsg)));
  unsigned long long m0 = 0;
  if (lane == 0) m0 = atomicAdd(a.short_counter, static_cast<unsigned long long>(G));
  m0 = __shfl_sync(0xffffffffu, m0, 0);
  while (m0 < a.n) {
    unsigned long long m1 = 0;  // the next group, claimed now so its latency overlaps this one
    if (lane == 0) m1 = atomicAdd(a.short_counter, static_cast<unsigned long long>(G));
    uint32_t nb = 0;
    uint64_t len = 0;
    if (lane < G && m0 + lane < a.n) {
      int32_t st;
      uint64_t olen;
      const uint64_t b = message_blocks(a, static_cast<uint32_t>(m0 + lane), &st, &olen);
      const bool on_lanes = OPB == kBatchCtr && a.lane_bin != nullptr && b < kLaneMax;
      if (st == AES_OK && b > 0 && b < kShortMax && !on_lanes) {
        nb = static_cast<uint32_t>(b);
        len = a.in_len[m0 + lane];
      }
    }
    const uint32_t valid = __ballot_sync(0xffffffffu, nb > 0);
    uint32_t nr = 0;  // the lane's message's rounds (0: no message)
    const uint32_t* sched = nullptr;  // its resident schedule, copied below by the whole warp
    if (nb > 0) {
      const uint32_t m = static_cast<uint32_t>(m0 + lane);
      if (a.keys != nullptr) {
        const uint32_t nk = a.key_bits[m] / 32;
        nr = nk + 6;
        expand_key(T, sb, sb_off, a.keys + 32ull * m, nk, wrk + lane * kShortStride<OPB>);
      } else {
        const aes_key_schedule& ks = a.schedules[a.sched_idx[m]];
        nr = ks.nr;
        sched = OPB == kBatchEcbDec ? ks.rk_dec : ks.rk_enc;
      }
    }
    if (a.keys == nullptr) {
      // Resident schedules: slot j's 4(nr + 1) words as coalesced loads by the
      // warp's lanes (a lane copying its own would issue 60 scattered loads).
#pragma unroll 1
      for (uint32_t j = 0; j < G; ++j) {
        const uint32_t nw = min(4 * (__shfl_sync(0xffffffffu, nr, j) + 1), 60u);  // nr was validated: 10, 12, 14
        const uint64_t p = __shfl_sync(0xffffffffu, reinterpret_cast<uint64_t>(sched), j);
        if (nw > 4) {
          const uint32_t* src = reinterpret_cast<const uint32_t*>(p);
          uint32_t* dst = wrk + j * kShortStride<OPB>;
          for (uint32_t w = lane; w < nw; w += 32) dst[w] = __ldg(src + w);
        }
      }
    }
    // The group's messages are laid end to end ordered by round count, then
    // by lane (ci), so that a warp step mixes key sizes as rarely as the
    // group allows: rounds 10-13 run masked, a step paying for its longest
    // key.  b0 = blocks of the messages before this one in that order.
    const uint32_t r10 = __ballot_sync(0xffffffffu, nr == 10), r12 = __ballot_sync(0xffffffffu, nr == 12);
    const uint32_t r14 = valid & ~(r10 | r12);
    const uint32_t lower = nr == 12 ? r10 : nr == 14 ? (r10 | r12) : 0u;
    const uint32_t peers = nr == 10 ? r10 : nr == 12 ? r12 : r14;
    const uint32_t ci = __popc(lower) + __popc(peers & ((1u << lane) - 1));
    uint32_t b0 = 0;
#pragma unroll
    for (uint32_t j = 0; j < G; ++j) {
      const uint32_t nb_j = __shfl_sync(0xffffffffu, nb, j), ci_j = __shfl_sync(0xffffffffu, ci, j);
      if (nb_j > 0 && ci_j < ci) b0 += nb_j;
    }
    const uint32_t nblk = __reduce_add_sync(0xffffffffu, nb);
    __syncwarp();
    if (nb > 0) {
      const uint32_t m = static_cast<uint32_t>(m0 + lane);
      uint32_t* rk = wrk + lane * kShortStride<OPB>;
      GroupMsg r;
      r.src0 = reinterpret_cast<uint64_t>(a.in) + a.in_off[m] - 16ull * b0;
      r.dst0 = reinterpret_cast<uint64_t>(a.out) + a.out_off[m] - 16ull * b0;
      r.ctr0 = b0;
      if (OPB == kBatchCtr) {
        const uint4 ivw = *reinterpret_cast<const uint4*>(a.iv + 16ull * m);
        r.ctr0 = __byte_perm(ivw.w, 0, 0x0123) - b0;
        const uint4 k0 = lds128(rk), k1 = lds128(rk + 4), k2 = lds128(rk + 8);
        const uint32_t s0 = ivw.x ^ k0.x, s1 = ivw.y ^ k0.y, s2 = ivw.z ^ k0.z;
        // round-1 columns without the counter column's lookups (column 3 of the state)
        const uint32_t c1x = k1.x ^ T.t0(s0) ^ T.t1(s1) ^ T.t2(s2);
        const uint32_t c1y0 = k1.y ^ T.t0(s1) ^ T.t1(s2) ^ T.t3(s0);
        const uint32_t c1z0 = k1.z ^ T.t0(s2) ^ T.t2(s0) ^ T.t3(s1);
        const uint32_t c1w0 = k1.w ^ T.t1(s0) ^ T.t2(s1) ^ T.t3(s2);
        // the counter run holding most of the message's blocks (a message of
        // < 512 blocks spans at most three runs): its round-1/2 constants
        const uint32_t c_first = r.ctr0 + b0;
        const uint32_t in_first = 256 - (c_first & 255u);
        const uint32_t run = (c_first >> 8) + (nb > 2 * in_first ? 1 : 0);
        const uint32_t xr = __byte_perm(run << 8, 0, 0x0123) ^ k0.w;
        const uint32_t c1y = c1y0 ^ T.t2(xr), c1z = c1z0 ^ T.t1(xr), c1w = c1w0 ^ T.t0(xr);
        // words 60..71 of the slot, three 128-bit stores: c1, then (rk0 word 3,
        // run, xr, c1 column 0), then the run's round-2 columns
        *reinterpret_cast<uint4*>(rk + kCtrC1) = make_uint4(c1x, c1y0, c1z0, c1w0);
        *reinterpret_cast<uint4*>(rk + kRunWords) = make_uint4(k0.w, run, xr, c1x);
        *reinterpret_cast<uint4*>(rk + kRunD) =
            make_uint4(k2.x ^ T.t1(c1y) ^ T.t2(c1z) ^ T.t3(c1w), k2.y ^ T.t0(c1y) ^ T.t1(c1z) ^ T.t2(c1w),
                       k2.z ^ T.t0(c1z) ^ T.t1(c1w) ^ T.t3(c1y), k2.w ^ T.t0(c1w) ^ T.t2(c1y) ^ T.t3(c1z));
      }
      r.info = nr | static_cast<uint32_t>(len & 15u) << 8 | lane << 16;
      r.full_end = b0 + static_cast<uint32_t>(len / 16);
      r.end = b0 + nb;
      rec[ci] = r;
      first[ci] = b0;
    }
    __syncwarp();
    if (OPB == kBatchEcbDec && a.keys != nullptr) {
      // Equivalent-inverse-cipher schedules: slot j's units (round r = lane / 4
      // <= nr / 2, column lane % 4) on the warp's lanes, one slot at a time,
      // instead of one lane working through a whole schedule alone.
#pragma unroll 1
      for (uint32_t j = 0; j < G; ++j) {
        const uint32_t nr_j = __shfl_sync(0xffffffffu, nr, j);
        if (nr_j != 0 && lane / 4 <= nr_j / 2)
          decrypt_schedule_unit(T, sb, sb_off, nr_j, wrk + j * kShortStride<OPB>, lane / 4, lane % 4);
      }
      __syncwarp();
    }
    const uint32_t ng = __popc(valid);
    const uint32_t my_first = lane < ng ? first[lane] : 0xFFFFFFFFu;
    uint32_t cur = 0xFFFFFFFFu;
    ShortCur sc{};
#pragma unroll 1
    for (uint32_t base = 0; base < nblk; base += 32) {
      const uint32_t gr = base + lane;
      // messages starting at or before `base`, and a bit for each start inside the step
      const uint32_t c0 = __popc(__ballot_sync(0xffffffffu, my_first <= base)) - 1;
      const uint32_t d = my_first - base;
      const uint32_t starts = __reduce_or_sync(0xffffffffu, (my_first > base && d < 32) ? 1u << d : 0u);
      const uint32_t ci = c0 + __popc(starts & (0xFFFFFFFFu >> (31 - lane)));
      if (gr < nblk) {
        if (ci != cur) {
          cur = ci;
          load_short_cur<OPB>(wrk, rec, ci, sc);
        }
        short_block<OPB>(a, T, wrk, sc, gr, m0);
      }
    }
    __syncwarp();  // the slots are refilled next
    m0 = __shfl_sync(0xffffffffu, m1, 0);
  }
}

// kRegKeys: the 512-thread build (128 registers per thread), whose span loop
// keeps the message's round keys in registers.
template <int OPB, bool kRegKeys>
__global__ void __launch_bounds__(kRegKeys ? 512 : 1024, 1) batch_kernel(const __grid_constant__ BatchArgs a) {
  constexpr int kWin = WindowSize<OPB>::value;
  constexpr bool kDec = OPB == kBatchEcbDec;
  extern __shared__ __align__(16) uint32_t smem[];
  // the claimed tile, double-buffered: tile i reads entry i & 1 while warp 0
  // writes tile i + 1 into the other entry
  __shared__ unsigned long long s_tile[2];
  __shared__ uint32_t s_mlo[2], s_mhi[2];
  __shared__ uint32_t s_span;  // next 256-block span of the current window

  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // The lane kernel, launched next on the lane path, may start on SMs this
  // grid leaves (it shares no data with this kernel and waits for its
  // completion before it ends).
  pdl_launch_dependents();
  const uint64_t total = a.blk_off[a.n];
  if (total == 0 && !groups_have_work(a)) return;  // lane path: no long message, no group work
  const uint32_t tile = a.tile_blocks ? a.tile_blocks : auto_tile(total, gridDim.x, blockDim.x);
  if (warp == 0) claim_tile(a, total, tile, &s_tile[0], &s_mlo[0], &s_mhi[0]);  // overlaps the table fill

  fill_tables<kDec>(smem);
  if (kDec) {  // forward S-box (all four bytes) beside the inverse one, for key expansion
    const int nwarps = blockDim.x >> 5;
    for (int x = warp; x < 256; x += nwarps)
      smem[kRegionC / 4 + x * 64 + 32 + lane] = kDevTables.sbox[x] * 0x01010101u;
  }
  uint32_t* rk_all = smem + batch_table_bytes<OPB>() / 4;
  Slot* slots = reinterpret_cast<Slot*>(rk_all + kWin * kRkStride);

  const char* base = reinterpret_cast<const char*>(smem);
  const Tabs T{base, base + kRegionB, base + kRegionC, lane * 4, lane * 4 + 128};
  // S-box source for key expansion: byte 0 of te2 (encryption tables) or the
  // forward S-box words in the upper half of region C (decryption tables).
  const char* sb = kDec ? T.c : T.b;
  const uint32_t sb_off = kDec ? T.hi : T.lo;
  // Window slots are loaded by warps 1.. first, so warp 0 can look ahead.
  const uint32_t first_slot = tid >= 32 ? tid - 32 : tid + blockDim.x - 32;

  for (uint32_t it = 0;; ++it) {
    __syncthreads();  // tile `it` is visible (and, first time, the tables)
    const uint32_t cur = it & 1;
    const uint64_t t0 = s_tile[cur] * tile;
    const uint32_t m_lo = s_mlo[cur], m_hi = s_mhi[cur];
    if (t0 >= total) break;
    const uint64_t t1 = min(t0 + tile, total);
    for (uint32_t w0 = m_lo; w0 <= m_hi; w0 += kWin) {
      const uint32_t wn = min(static_cast<uint32_t>(kWin), m_hi - w0 + 1);
      for (uint32_t sl = first_slot; sl < wn; sl += blockDim.x)
        load_slot<OPB>(a, T, sb, sb_off, w0 + sl, slots[sl], rk_all + sl * kRkStride);
      if (tid == blockDim.x - 1) s_span = 0;
      __syncthreads();
      // Look ahead while the others start on the window: warp 0 claims tile
      // it + 1 into the other entry (last read before this tile's barrier)
      // and joins the spans afterwards.
      if (w0 == m_lo && warp == 0)
        claim_tile(a, total, tile, &s_tile[cur ^ 1], &s_mlo[cur ^ 1], &s_mhi[cur ^ 1]);
      const uint32_t gr0 = static_cast<uint32_t>(max(t0, slots[0].blk_start) - t0);
      const uint32_t gr1 = static_cast<uint32_t>(min(t1, slots[wn - 1].blk_end) - t0);
      Cur c{1, 0, 0, 0, 0, 0, 0, 0};  // empty: the first block selects its message
      RunCache rc{0, 0, 0, 0, 0, 0, 0, 0};
      // Warps claim spans of 256 consecutive blocks from a shared counter (so
      // they finish the window together); lane l takes blocks 32k + l of the
      // span (coalesced), so a lane's blocks share counter runs.
      for (;;) {
        uint32_t sp = 0;
        if (lane == 0) sp = atomicAdd(&s_span, 1u);
        sp = __shfl_sync(0xffffffffu, sp, 0);
        const uint32_t span = gr0 + sp * 256;
        if (span >= gr1) break;
        if (span + 256 <= gr1) {
          // every lane takes the message of the span's first block; if that
          // message holds the whole span in whole blocks, run the fast loop
          if (span < c.s || span >= c.e) select_message(slots, wn, t0, t1, span, c);
          const bool whole = span >= c.s && span + 256 <= c.f;
          if (whole) {
            const uint32_t* rk = rk_all + c.slot * kRkStride;
            switch (c.nr & 0xFFu) {
              case 10: span_fast<OPB, 10, kRegKeys>(a, T, slots, rk, c, span, lane, rc); break;
              case 12: span_fast<OPB, 12, kRegKeys>(a, T, slots, rk, c, span, lane, rc); break;
              default: span_fast<OPB, 14, kRegKeys>(a, T, slots, rk, c, span, lane, rc); break;
            }
            continue;
          }
        }
        run_blocks<OPB>(a, T, slots, rk_all, wn, t0, t1, span, min(span + 256, gr1), lane, c, rc);
      }
      __syncthreads();
    }
  }

  if (groups_have_work(a))  // on the lane path only the short messages of kLaneMax blocks or more
    short_phase<OPB>(a, T, sb, sb_off, reinterpret_cast<char*>(rk_all), warp, lane);
}

// The persistent kernel of one build (kRegKeys: the 512-thread one).
template <int OPB, bool kRegKeys>
cudaError_t launch_build(const BatchArgs& a, int cta, int grid, cudaStream_t s) {
  constexpr size_t smem = batch_smem_bytes<OPB>();
  static_assert(smem + 64 <= 227 * 1024, "batch kernel shared memory over the 227 KB limit");
  auto kern = batch_kernel<OPB, kRegKeys>;
  cudaError_t e = ensure_dynamic_smem(kern, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<grid, cta, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

#if defined(AES_BATCH_REGKEYS_TU)
// This translation unit (aes_batch_regkeys.cu) holds the 512-thread builds.
cudaError_t launch_batch_regkeys(const BatchArgs& a, int cta, int grid, cudaStream_t s) {
  switch (a.op) {
    case kBatchCtr: return launch_build<kBatchCtr, true>(a, cta, grid, s);
    case kBatchEcbEnc: return launch_build<kBatchEcbEnc, true>(a, cta, grid, s);
    case kBatchEcbDec: return launch_build<kBatchEcbDec, true>(a, cta, grid, s);
  }
  return cudaErrorInvalidValue;
}
#elif !defined(AES_BATCH_LANES_TU)
cudaError_t launch_batch_regkeys(const BatchArgs& a, int cta, int grid, cudaStream_t s);

// Workspace layout, each part rounded up to 256 bytes: block offsets
// (n + 1 words), chunk totals, the work counters and lane_info, the lane
// path's bin counts, cursors and group-message count (cleared together with
// the counters by one memset), then its bins (n halfwords) and order
// (n + 96 words).
constexpr size_t kCounterBytes = 256;
constexpr size_t kLaneCountBytes = (8 * kLaneBins + 4 + 255) & ~static_cast<size_t>(255);

size_t batch_workspace_bytes(uint32_t n) {
  const size_t nchunks = (static_cast<size_t>(n) + kChunkMsgs - 1) / kChunkMsgs;
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  return up(8 * (static_cast<size_t>(n) + 1)) + up(8 * (nchunks > 0 ? nchunks : 1)) + kCounterBytes +
         kLaneCountBytes + up(2 * static_cast<size_t>(n)) + up(4 * (static_cast<size_t>(n) + 96));
}

void batch_bind_workspace(BatchArgs* a, void* ws, bool lanes) {
  auto up = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
  const size_t nchunks = (static_cast<size_t>(a->n) + kChunkMsgs - 1) / kChunkMsgs;
  char* p = static_cast<char*>(ws);
  a->blk_off = reinterpret_cast<uint64_t*>(p);
  p += up(8 * (static_cast<size_t>(a->n) + 1));
  a->chunk_sum = reinterpret_cast<uint64_t*>(p);
  p += up(8 * (nchunks > 0 ? nchunks : 1));
  a->tile_counter = reinterpret_cast<unsigned long long*>(p);  // bytes 0..7 of the counters
  a->short_counter = a->tile_counter + 1;                       // 8..15
  a->scan_done = reinterpret_cast<unsigned int*>(p + 48);       // 48..51
  a->nchunks = static_cast<uint32_t>(nchunks);
  a->lane_bin = nullptr;
  a->lane_hist = a->lane_cursor = a->lane_order = a->lane_info = nullptr;
  a->lane_counter = nullptr;
  if (!lanes) return;
  a->lane_counter = a->tile_counter + 2;  // three counters, 16..39
  a->lane_info = reinterpret_cast<uint32_t*>(p + 64);  // 64..83
  p += kCounterBytes;
  a->lane_hist = reinterpret_cast<uint32_t*>(p);
  a->lane_cursor = a->lane_hist + kLaneBins;
  p += kLaneCountBytes;
  a->lane_bin = reinterpret_cast<uint16_t*>(p);
  p += up(2 * static_cast<size_t>(a->n));
  a->lane_order = reinterpret_cast<uint32_t*>(p);
}

// Enqueue the pipeline: the counters (and on the lane path the bin counts)
// cleared, the count kernel (whose last CTA finishes the scans), on the lane
// path the scatter into bin order, the persistent kernel (which then leaves
// the short messages of fewer than kLaneMax blocks alone), and on the lane
// path the lane kernel, launched with programmatic stream serialisation so
// its CTAs start on the SMs the persistent kernel's CTAs leave.
cudaError_t launch_batch(const BatchArgs& a, int cta, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.tile_counter, 0, kCounterBytes + (a.lane_bin != nullptr ? kLaneCountBytes : 0), s);
  if (e != cudaSuccess) return e;
  batch_count_scan<<<a.nchunks, kScanThreads, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (a.lane_bin != nullptr) {
    e = launch_batch_lanes_sort(a, s);
    if (e != cudaSuccess) return e;
  }
  if (cta <= 512) {
    e = launch_batch_regkeys(a, cta, grid, s);
  } else {
    switch (a.op) {
      case kBatchCtr: e = launch_build<kBatchCtr, false>(a, cta, grid, s); break;
      case kBatchEcbEnc: e = launch_build<kBatchEcbEnc, false>(a, cta, grid, s); break;
      case kBatchEcbDec: e = launch_build<kBatchEcbDec, false>(a, cta, grid, s); break;
      default: return cudaErrorInvalidValue;
    }
  }
  if (e != cudaSuccess || a.lane_bin == nullptr) return e;
  return launch_batch_lanes(a, grid, s);
}
#endif  // AES_BATCH_REGKEYS_TU / !AES_BATCH_LANES_TU

}  // namespace aesgpu
