// aes_batch_lanes.cu — the batch's short CTR messages, one lane per message.
//
// SP 800-38A §6.5 CTR on each message with its own key (FIPS-197 §5.2
// expansion on the device) and IV: the paper's chunk-per-thread split of
// §IV.B with chunk = message, here one message per GPU lane.
//
// Messages of kLaneMax (128) blocks or more stay with the persistent kernel's
// per-warp groups: a lane walks its message one block after another, so a
// chunk of long messages would be a long serial tail.
//
// Why a lane per message.  In the per-warp group phase of aes_batch.cu the
// 32 lanes of a warp step work on blocks of two or three messages at once, so
// every round's key comes from shared memory: a 128-bit load costs four
// shared-memory wavefronts per round, on the pipe the T-table lookups already
// saturate.  Here a lane owns one message from its first block to its last,
// so the message's whole schedule sits in the lane's registers (the round
// count is a template parameter, every index a constant), and round keys
// cost no shared-memory traffic at all.
//
// Steps (after aes_batch.cu's count kernel has binned every accepted short
// message by (key-size class, 511 - blocks)):
//   1. lanes_scatter  per message chunk of the count kernel: places its
//                     messages with a per-CTA rank and one global cursor add
//                     per bin, from the bin starts the count kernel's last
//                     CTA computed (each key-size class from a multiple of
//                     32, bins longest first, the class gaps filled with
//                     kLaneNoMsg).
//   2. batch_lanes_kernel  persistent, 512 threads (128 registers, room for
//                     an AES-256 schedule).  A warp claims 32 consecutive
//                     positions (one key-size class, nearly equal lengths)
//                     and walks the messages in stages of 8 blocks: each lane
//                     copies its message's next 8 whole blocks into its own
//                     shared-memory slot with one TMA bulk copy, computes the
//                     keystream two blocks at a time with the counter-run
//                     caching of the single-buffer kernel (rounds 1-2 mostly
//                     precomputed per run of 256 counters), and stores each
//                     result block with a plain 128-bit streaming store.  A
//                     ragged last block (without the padded flags) is read
//                     and written byte-exactly instead.  While a chunk runs,
//                     the warp claims the next one, looks up its messages and
//                     prefetches their descriptors into L2.
//
// Measured choices (packet-sized batch, 1M messages of 16-1500 bytes):
// results written back through the slot by TMA bulk stores ran at 797 GB/s
// against 828 GB/s for the plain stores (a bulk copy's operands must be
// warp-uniform, so every per-lane copy costs the warp a loop over its
// lanes); plain per-lane loads instead of the bulk copies, 560 GB/s (each
// load touches 32 different lines); one block per iteration 745 GB/s, four
// for AES-128 673 GB/s.
//
// A lane's slot holds its 8 blocks and, at bytes 128..159, the words a new
// counter run needs (round-0 key word 3, the round-1 columns without the
// counter terms, the round-2 key), kept out of registers.  Slots are 176
// bytes apart (11 groups of four banks), so the eight lanes of each
// quarter-warp read their j-th blocks, and their run words, on distinct bank
// groups.  Waits on a warp's mbarrier are bounded (about a second of SM
// clock); a warp that gives up counts it (take_lane_timeouts), lets its
// copy land, and stops.  No cluster, no multicast: every copy moves this
// GPU's memory into the issuing CTA's own shared memory.
#define AES_BATCH_LANES_TU 1
#include "aes_batch.cu"

namespace aesgpu {
namespace {

constexpr uint32_t kLaneThreads = 512;
constexpr uint32_t kLaneWarps = kLaneThreads / 32;
constexpr uint32_t kLaneStage = 8;                       // blocks per lane per stage
constexpr uint32_t kLaneRun = 16 * kLaneStage;           // the run words' offset in a slot
constexpr uint32_t kLaneSlot = 16 * kLaneStage + 48;     // bytes between two lanes' slots
constexpr uint32_t kLaneStageBytes = kLaneWarps * 32 * kLaneSlot;
constexpr int kLaneSmem = 128 * 1024 + kLaneStageBytes + kLaneWarps * 8;  // tables, slots, mbarriers
static_assert(kLaneSmem <= 227 * 1024, "lane kernel shared memory over the 227 KB limit");

// Bounded waits that gave up (read and cleared by take_lane_timeouts).
__device__ unsigned int g_lane_timeouts = 0;

// ------------------------------------------------------------------ sort ----

// The count kernel's partition: kScanItems consecutive messages per thread.
// lane_hist holds each bin's first position (the count kernel's last CTA).
__global__ void __launch_bounds__(kScanThreads) lanes_scatter(const BatchArgs a) {
  __shared__ uint32_t cnt[kLaneBins], first[kLaneBins];
  for (uint32_t i = threadIdx.x; i < kLaneBins; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const uint64_t m0 = static_cast<uint64_t>(blockIdx.x) * kChunkMsgs + static_cast<uint64_t>(threadIdx.x) * kScanItems;
  uint32_t bin[kScanItems], rank[kScanItems];
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k) {
    bin[k] = m0 + k < a.n ? a.lane_bin[m0 + k] : kLaneNoBin;
    rank[k] = bin[k] != kLaneNoBin ? atomicAdd(&cnt[bin[k]], 1u) : 0;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kLaneBins; i += blockDim.x)
    if (cnt[i] != 0) first[i] = a.lane_hist[i] + atomicAdd(a.lane_cursor + i, cnt[i]);
  __syncthreads();
#pragma unroll
  for (uint32_t k = 0; k < kScanItems; ++k)
    if (bin[k] != kLaneNoBin) a.lane_order[first[bin[k]] + rank[k]] = static_cast<uint32_t>(m0 + k);
}

// ----------------------------------------------------------- TMA helpers ----

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
// global -> this CTA's shared memory, completing `bytes` of the mbarrier's transaction count
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// --------------------------------------------------------------- cipher ----

// FIPS-197 §5.2 into registers: w[i] for i < 4(NK + 7), every index a
// compile-time constant once unrolled.  key: 16-byte aligned.
template <int NK>
__device__ __forceinline__ void expand_key_regs(const Tabs& T, const uint8_t* key, uint32_t (&w)[4 * (NK + 7)]) {
  const uint4 k0 = *reinterpret_cast<const uint4*>(key);
  w[0] = k0.x;
  w[1] = k0.y;
  w[2] = k0.z;
  w[3] = k0.w;
  if (NK > 4) {
    const uint4 k1 = *reinterpret_cast<const uint4*>(key + 16);
    const uint32_t hi[4] = {k1.x, k1.y, k1.z, k1.w};
#pragma unroll
    for (int i = 4; i < NK; ++i) w[i] = hi[i - 4];
  }
  uint32_t rcon = 1;
#pragma unroll
  for (int i = NK; i < 4 * (NK + 7); ++i) {
    uint32_t t = w[i - 1];
    if (i % NK == 0) {
      t = sub_word(T, T.b, T.lo, __funnelshift_r(t, t, 8)) ^ rcon;  // RotWord, SubWord, Rcon
      rcon = ((rcon << 1) ^ ((rcon & 0x80u) ? 0x1Bu : 0u)) & 0xFFu;
    } else if (NK == 8 && i % NK == 4) {
      t = sub_word(T, T.b, T.lo, t);
    }
    w[i] = w[i - NK] ^ t;
  }
}

// One chunk (32 positions of lane_order, one key-size class) on one warp.
// m: this lane's message, kLaneNoMsg for a gap; parity: the warp mbarrier's
// next phase parity.  The warp's next chunk is claimed (from `counter`,
// chunks from `first`) after this chunk's first stage, once every warp has
// made its first claim, so no warp takes two chunks while another waits for
// one; its messages are looked up a stage later (next, m_next: kLaneNoMsg at
// or past `end`) and their descriptors prefetched into L2 a stage after
// that, so the next chunk starts without those round trips.  Returns the
// parity after the chunk (bit 0), or kLaneGaveUp if a wait gave up.
constexpr uint32_t kLaneGaveUp = 2;
template <int NR>
__device__ __forceinline__ uint32_t lanes_chunk(const BatchArgs& a, const Tabs& T, uint32_t m, char* slot,
                                                uint32_t slot_s, uint32_t mbar, uint32_t parity, uint32_t first,
                                                unsigned long long* counter, uint32_t end, uint32_t& next,
                                                uint32_t& m_next) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t step = 0;  // next chunk: 0 to claim, 1 to look up, 2 to prefetch, 3 done
  constexpr int NK = NR - 6;
  constexpr long long kWaitLimit = 2000000000ll;  // SM clocks, ~1 s at 2 GHz
  uint32_t w[4 * (NR + 1)];
  uint32_t nb = 0, in_full = 0, out_full = 0, rem = 0, ctr0 = 0, c10 = 0;
  const uint8_t* src = nullptr;
  uint8_t* dst = nullptr;
  if (m != kLaneNoMsg) {
    const uint64_t len = a.in_len[m];
    nb = static_cast<uint32_t>((len + 15) / 16);
    rem = static_cast<uint32_t>(len & 15u);
    in_full = (a.flags & AES_BATCH_IN_PADDED) ? nb : static_cast<uint32_t>(len / 16);
    out_full = (a.flags & AES_BATCH_OUT_PADDED) ? nb : static_cast<uint32_t>(len / 16);
    src = a.in + a.in_off[m];
    dst = a.out + a.out_off[m];
    if (a.keys != nullptr) {
      expand_key_regs<NK>(T, a.keys + 32ull * m, w);
    } else {
      const uint32_t* rk = a.schedules[a.sched_idx[m]].rk_enc;
#pragma unroll
      for (int i = 0; i < 4 * (NR + 1); ++i) w[i] = __ldg(rk + i);
    }
    const uint4 ivw = *reinterpret_cast<const uint4*>(a.iv + 16ull * m);
    ctr0 = __byte_perm(ivw.w, 0, 0x0123);
    const uint32_t s0 = ivw.x ^ w[0], s1 = ivw.y ^ w[1], s2 = ivw.z ^ w[2];
    // round-1 columns without the counter byte's terms: column 0 stays in a
    // register, the other three go to the run words with the round-2 key
    c10 = w[4] ^ T.t0(s0) ^ T.t1(s1) ^ T.t2(s2);
    *reinterpret_cast<uint4*>(slot + kLaneRun) =
        make_uint4(w[3], w[5] ^ T.t0(s1) ^ T.t1(s2) ^ T.t3(s0), w[6] ^ T.t0(s2) ^ T.t2(s0) ^ T.t3(s1),
                   w[7] ^ T.t1(s0) ^ T.t2(s1) ^ T.t3(s2));
    *reinterpret_cast<uint4*>(slot + kLaneRun + 16) = make_uint4(w[8], w[9], w[10], w[11]);
  }
  const uint32_t nbmax = __reduce_max_sync(0xffffffffu, nb);
  uint32_t run = 0xFFFFFFFFu, xr = 0;  // the cached counter run (counter >> 8 never reaches 2^24)
  uint4 d = make_uint4(0, 0, 0, 0);    // its round-2 columns without the column-0 terms
  for (uint32_t s0 = 0; s0 < nbmax; s0 += kLaneStage) {
    const uint32_t e = min(s0 + kLaneStage, nb);  // this stage: blocks [s0, e) (none when e <= s0)
    const uint32_t ein = min(s0 + kLaneStage, in_full);
    const uint32_t nin = ein > s0 ? ein - s0 : 0;
    fence_proxy_async();  // this lane's reads of its slot come before the copy's writes
    if (nin != 0) bulk_load(slot_s, src + 16ull * s0, 16 * nin, mbar);
    else mbar_arrive(mbar);
    const bool ok = mbar_wait_bounded(mbar, parity, kWaitLimit);
    if (!__all_sync(0xffffffffu, ok)) {
      if (!ok) {
        atomicAdd(&g_lane_timeouts, 1u);
        mbar_wait_bounded(mbar, parity, kWaitLimit);  // let the copy land before the warp leaves
      }
      __syncwarp();
      return kLaneGaveUp;
    }
    parity ^= 1u;
    // Two blocks per iteration, their rounds interleaved, so each lane has two
    // independent dependency chains in flight (a stage's odd last block pairs
    // with a dummy whose result is dropped).
#pragma unroll 1
    for (uint32_t s = s0; s < e; s += 2) {
      char* p = slot + 16 * (s - s0);
      const bool two = s + 1 < e;
      // a ragged last input block (without AES_BATCH_IN_PADDED) is read exactly
      const uint4 v0 = s < in_full ? *reinterpret_cast<const uint4*>(p) : load_partial(src + 16ull * s, rem);
      uint4 v1 = make_uint4(0, 0, 0, 0);
      if (two) v1 = s + 1 < in_full ? *reinterpret_cast<const uint4*>(p + 16) : load_partial(src + 16ull * (s + 1), rem);
      State st[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint32_t ctr = ctr0 + s + k;  // modulo 2^32
        if ((ctr >> 8) != run) {  // a new counter run: its constants (15 lookups)
          run = ctr >> 8;
          const uint4 c = *reinterpret_cast<const uint4*>(slot + kLaneRun);  // rk0 word 3, round-1 columns 1-3
          const uint4 k2 = *reinterpret_cast<const uint4*>(slot + kLaneRun + 16);
          xr = __byte_perm(ctr & ~255u, 0, 0x0123) ^ c.x;
          const uint32_t s1 = c.y ^ T.t2(xr), s2 = c.z ^ T.t1(xr), s3 = c.w ^ T.t0(xr);
          d = make_uint4(k2.x ^ T.t1(s1) ^ T.t2(s2) ^ T.t3(s3), k2.y ^ T.t0(s1) ^ T.t1(s2) ^ T.t2(s3),
                         k2.z ^ T.t0(s2) ^ T.t1(s3) ^ T.t3(s1), k2.w ^ T.t0(s3) ^ T.t2(s1) ^ T.t3(s2));
        }
        // rounds 1-2: only round-1 column 0 depends on the counter's low byte
        const uint32_t x0 = c10 ^ T.t3(xr ^ ((ctr & 255u) << 24));
        st[k] = State{d.x ^ T.t0(x0), d.y ^ T.t3(x0), d.z ^ T.t2(x0), d.w ^ T.t1(x0)};
      }
#pragma unroll
      for (int r = 3; r < NR; ++r) {
        enc_round(T, st[0], &w[4 * r]);
        enc_round(T, st[1], &w[4 * r]);
      }
      enc_final(T, st[0], &w[4 * NR]);
      enc_final(T, st[1], &w[4 * NR]);
      const uint4 o0 = xor4(v0, st[0]);
      if (s < out_full) __stcs(reinterpret_cast<uint4*>(dst + 16ull * s), o0);
      else store_partial(dst + 16ull * s, o0, rem);
      if (two) {
        const uint4 o1 = xor4(v1, st[1]);
        if (s + 1 < out_full) __stcs(reinterpret_cast<uint4*>(dst + 16ull * (s + 1)), o1);
        else store_partial(dst + 16ull * (s + 1), o1, rem);
      }
    }
    if (step == 0) {
      if (lane == 0) next = first + static_cast<uint32_t>(atomicAdd(counter, 1ull));
    } else if (step == 1) {
      next = __shfl_sync(0xffffffffu, next, 0);
      m_next = next < end ? a.lane_order[32ull * next + lane] : kLaneNoMsg;
    } else if (step == 2 && m_next != kLaneNoMsg) {
      prefetch_l2(a.in_len + m_next);
      prefetch_l2(a.in_off + m_next);
      prefetch_l2(a.out_off + m_next);
      prefetch_l2(a.iv + 16ull * m_next);
      if (a.keys != nullptr) prefetch_l2(a.keys + 32ull * m_next);
    }
    ++step;
  }
  if (step == 0 && lane == 0) next = first + static_cast<uint32_t>(atomicAdd(counter, 1ull));
  if (step <= 1) {
    next = __shfl_sync(0xffffffffu, next, 0);
    m_next = next < end ? a.lane_order[32ull * next + lane] : kLaneNoMsg;
  }
  return parity;
}

// The chunks of key-size class c, claimed from the class's own counter, each
// one while the chunk before it runs.
template <int NR>
__device__ __forceinline__ uint32_t lanes_class(const BatchArgs& a, const Tabs& T, uint32_t c, char* slot,
                                                uint32_t slot_s, uint32_t mbar, uint32_t parity) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t first = a.lane_info[1 + c], end = a.lane_info[2 + c];
  uint32_t chunk = 0;
  if (lane == 0) chunk = first + static_cast<uint32_t>(atomicAdd(a.lane_counter + c, 1ull));
  chunk = __shfl_sync(0xffffffffu, chunk, 0);
  if (chunk >= end) return parity;
  uint32_t m = a.lane_order[32ull * chunk + lane];
  for (;;) {
    uint32_t next = 0, m_next = kLaneNoMsg;
    parity = lanes_chunk<NR>(a, T, m, slot, slot_s, mbar, parity, first, a.lane_counter + c, end, next, m_next);
    if (parity == kLaneGaveUp || next >= end) return parity;
    m = m_next;
  }
}

__global__ void __launch_bounds__(kLaneThreads, 1) batch_lanes_kernel(const __grid_constant__ BatchArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  fill_tables<false>(smem);
  char* stage = reinterpret_cast<char*>(smem) + 128 * 1024;
  char* slot = stage + (warp * 32 + lane) * kLaneSlot;
  const uint32_t slot_s = smem_addr(slot);
  const uint32_t mbar = smem_addr(stage + kLaneStageBytes) + 8 * warp;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 32;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const char* base = reinterpret_cast<const char*>(smem);
  const Tabs T{base, base + kRegionB, base + kRegionC, lane * 4, lane * 4 + 128};
  // The classes one after another, each from its own chunk counter: the
  // three key sizes' bodies never share live ranges (taken from one loop, or
  // as calls, they spilled).
  uint32_t parity = 0;
  parity = lanes_class<10>(a, T, 0, slot, slot_s, mbar, parity);
  if (parity != kLaneGaveUp) parity = lanes_class<12>(a, T, 1, slot, slot_s, mbar, parity);
  if (parity != kLaneGaveUp) parity = lanes_class<14>(a, T, 2, slot, slot_s, mbar, parity);
  // Launched after the persistent kernel with programmatic serialisation:
  // this grid completes only once that one has, so the batch keeps stream order.
  pdl_wait_previous();
}

}  // namespace

cudaError_t launch_batch_lanes_sort(const BatchArgs& a, cudaStream_t s) {
  lanes_scatter<<<a.nchunks, kScanThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch_lanes(const BatchArgs& a, int grid, cudaStream_t s) {
  cudaError_t e = ensure_dynamic_smem(batch_lanes_kernel, kLaneSmem);
  if (e != cudaSuccess) return e;
  return launch_pdl(batch_lanes_kernel, static_cast<unsigned>(grid), kLaneThreads, kLaneSmem, s, a);
}

cudaError_t take_lane_timeouts(unsigned int* out) {
  unsigned int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_lane_timeouts, sizeof(v));
  if (e != cudaSuccess) return e;
  if (v != 0) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_lane_timeouts, &zero, sizeof(zero));
    if (e != cudaSuccess) return e;
  }
  *out = v;
  return cudaSuccess;
}

}  // namespace aesgpu
