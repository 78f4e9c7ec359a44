// aes_ttable.cuh — single-buffer AES kernels, T-table round variant.
//
// One 16-byte AES block per thread-iteration, held as four 32-bit column words
// (little-endian: byte r of column c is state row r, FIPS-197 §3.4).  A full
// round (paper Fig. 1 step 3: SubBytes, ShiftRows, MixColumns, AddRoundKey)
// is, per output column j,
//   t_j = T0[s_j.b0] ^ T1[s_{j+1}.b1] ^ T2[s_{j+2}.b2] ^ T3[s_{j+3}.b3] ^ rk_j
// where Ti = te0 rotated left by 8i bits; ShiftRows is the choice of source
// column and MixColumns is folded into the table words.  The final round
// (Fig. 1 step 4) picks the plain S-box byte out of the same words.
// Decryption uses the equivalent inverse cipher (FIPS-197 §5.3.5): td0 tables
// with the source columns shifted the other way, and the inverse S-box.
//
// Tables live in shared memory, replicated once per lane: row x of a table is
// 32 copies of the word, so lane l always reads bank l and a warp's 32
// lookups never conflict.  One PRMT builds a lookup address: the state byte
// goes to bits 8..15 (row x at x*256 bytes) and the lane's byte offset to
// bits 0..7.  Two tables share each 256-byte row (lanes at +0 and +128).
//
// Launch: a persistent grid (one CTA per SM by default; the tables take
// 128 KiB, 192 KiB for decryption), grid-stride over blocks, `BPT` blocks per
// thread per iteration for instruction-level parallelism, 128-bit streaming
// loads and stores that coalesce across the warp.
#pragma once
#include "aes_internal.h"
#include "aes_tables.cuh"

namespace aesgpu {
namespace {

__device__ const AesTables kDevTables = make_tables();

constexpr uint32_t kRegionB = 64 * 1024;   // te2|te3 (td2|td3)
constexpr uint32_t kRegionC = 128 * 1024;  // is4 (decryption only)

__device__ __forceinline__ uint32_t rotl(uint32_t v, int k) { return __funnelshift_l(v, v, k); }

// Shared-memory lookups.  a/b/c are the region bases; lo = lane*4 selects the
// first table of a row, hi = lane*4 + 128 the second.
struct Tabs {
  const char* a;
  const char* b;
  const char* c;
  uint32_t lo, hi;
  // word at base + (byte k of x) * 256 + lane offset; sel = 0x55k4
  __device__ __forceinline__ uint32_t ld(const char* base, uint32_t x, uint32_t lane_off,
                                         uint32_t sel) const {
    return *reinterpret_cast<const uint32_t*>(base + __byte_perm(x, lane_off, sel));
  }
  // Ti[byte i of x]
  __device__ __forceinline__ uint32_t t0(uint32_t x) const { return ld(a, x, lo, 0x5504); }
  __device__ __forceinline__ uint32_t t1(uint32_t x) const { return ld(a, x, hi, 0x5514); }
  __device__ __forceinline__ uint32_t t2(uint32_t x) const { return ld(b, x, lo, 0x5524); }
  __device__ __forceinline__ uint32_t t3(uint32_t x) const { return ld(b, x, hi, 0x5534); }
};

// Byte 0 of a, byte 1 of b, byte 2 of c, byte 3 of d.
__device__ __forceinline__ uint32_t merge_bytes(uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  return __byte_perm(__byte_perm(a, b, 0x0050), __byte_perm(c, d, 0x7200), 0x7610);
}

struct State {
  uint32_t s0, s1, s2, s3;
};

__device__ __forceinline__ void enc_round(const Tabs& T, State& s, const uint32_t* k) {
  const uint32_t t0 = T.t0(s.s0) ^ T.t1(s.s1) ^ T.t2(s.s2) ^ T.t3(s.s3) ^ k[0];
  const uint32_t t1 = T.t0(s.s1) ^ T.t1(s.s2) ^ T.t2(s.s3) ^ T.t3(s.s0) ^ k[1];
  const uint32_t t2 = T.t0(s.s2) ^ T.t1(s.s3) ^ T.t2(s.s0) ^ T.t3(s.s1) ^ k[2];
  const uint32_t t3 = T.t0(s.s3) ^ T.t1(s.s0) ^ T.t2(s.s1) ^ T.t3(s.s2) ^ k[3];
  s = State{t0, t1, t2, t3};
}

// Final encryption round: S(x) is byte 0 of te2, byte 1 of te3, byte 2 of
// te0 and byte 3 of te1, so column j is assembled from those four lookups.
__device__ __forceinline__ uint32_t enc_final_col(const Tabs& T, uint32_t a, uint32_t b,
                                                  uint32_t c, uint32_t d, uint32_t k) {
  return merge_bytes(T.ld(T.b, a, T.lo, 0x5504), T.ld(T.b, b, T.hi, 0x5514),
                     T.ld(T.a, c, T.lo, 0x5524), T.ld(T.a, d, T.hi, 0x5534)) ^ k;
}

__device__ __forceinline__ void enc_final(const Tabs& T, State& s, const uint32_t* k) {
  const uint32_t f0 = enc_final_col(T, s.s0, s.s1, s.s2, s.s3, k[0]);
  const uint32_t f1 = enc_final_col(T, s.s1, s.s2, s.s3, s.s0, k[1]);
  const uint32_t f2 = enc_final_col(T, s.s2, s.s3, s.s0, s.s1, k[2]);
  const uint32_t f3 = enc_final_col(T, s.s3, s.s0, s.s1, s.s2, k[3]);
  s = State{f0, f1, f2, f3};
}

// Inverse round: InvShiftRows takes row r of column j from column j - r.
__device__ __forceinline__ void dec_round(const Tabs& T, State& s, const uint32_t* k) {
  const uint32_t t0 = T.t0(s.s0) ^ T.t1(s.s3) ^ T.t2(s.s2) ^ T.t3(s.s1) ^ k[0];
  const uint32_t t1 = T.t0(s.s1) ^ T.t1(s.s0) ^ T.t2(s.s3) ^ T.t3(s.s2) ^ k[1];
  const uint32_t t2 = T.t0(s.s2) ^ T.t1(s.s1) ^ T.t2(s.s0) ^ T.t3(s.s3) ^ k[2];
  const uint32_t t3 = T.t0(s.s3) ^ T.t1(s.s2) ^ T.t2(s.s1) ^ T.t3(s.s0) ^ k[3];
  s = State{t0, t1, t2, t3};
}

__device__ __forceinline__ uint32_t dec_final_col(const Tabs& T, uint32_t a, uint32_t b,
                                                  uint32_t c, uint32_t d, uint32_t k) {
  return merge_bytes(T.ld(T.c, a, T.lo, 0x5504), T.ld(T.c, b, T.lo, 0x5514),
                     T.ld(T.c, c, T.lo, 0x5524), T.ld(T.c, d, T.lo, 0x5534)) ^ k;
}

__device__ __forceinline__ void dec_final(const Tabs& T, State& s, const uint32_t* k) {
  const uint32_t f0 = dec_final_col(T, s.s0, s.s3, s.s2, s.s1, k[0]);
  const uint32_t f1 = dec_final_col(T, s.s1, s.s0, s.s3, s.s2, k[1]);
  const uint32_t f2 = dec_final_col(T, s.s2, s.s1, s.s0, s.s3, k[2]);
  const uint32_t f3 = dec_final_col(T, s.s3, s.s2, s.s1, s.s0, k[3]);
  s = State{f0, f1, f2, f3};
}

// Programmatic dependent launch (the single-buffer launches set it): a grid
// lets the next launch in its stream queue its CTAs at once, and each grid
// fills its tables (from the never-written kDevTables) before waiting for the
// previous grid's completion and memory, so one call's table fill and launch
// latency overlap the previous call's last wave.  Both are no-ops for a
// launch without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait_previous() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Fill the replicated tables; warp w writes rows w, w + nwarps, ...
template <bool kDec>
__device__ __forceinline__ void fill_tables(uint32_t* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int x = warp; x < 256; x += nwarps) {
    const uint32_t v = kDec ? kDevTables.td0[x] : kDevTables.te0[x];
    uint32_t* ra = sm + x * 64;
    uint32_t* rb = sm + kRegionB / 4 + x * 64;
    ra[lane] = v;
    ra[32 + lane] = rotl(v, 8);
    rb[lane] = rotl(v, 16);
    rb[32 + lane] = rotl(v, 24);
    if (kDec) sm[kRegionC / 4 + x * 64 + lane] = kDevTables.is4[x];
  }
}

// Full cipher of one block whose state already had round key 0 added.
template <int NR>
__device__ __forceinline__ void encrypt_rounds(const Tabs& T, State& s, const RoundKeys& rk,
                                               int first_round) {
#pragma unroll
  for (int r = 1; r < NR; ++r)
    if (r >= first_round) enc_round(T, s, &rk.w[4 * r]);
  enc_final(T, s, &rk.w[4 * NR]);
}

// CTR keystream of block `idx` (see CtrParams: round 1 is partly folded).
template <int NR>
__device__ __forceinline__ State ctr_keystream(const Tabs& T, const RoundKeys& rk,
                                               const CtrParams& cp, uint64_t idx) {
  const uint32_t ctr = cp.ctr0 + static_cast<uint32_t>(idx);  // modulo 2^32
  const uint32_t x = __byte_perm(ctr, 0, 0x0123) ^ cp.rk0w3;  // big-endian counter word
  State s{cp.c1[0] ^ T.t3(x), cp.c1[1] ^ T.t2(x), cp.c1[2] ^ T.t1(x), cp.c1[3] ^ T.t0(x)};
  encrypt_rounds<NR>(T, s, rk, 2);
  return s;
}

__device__ __forceinline__ uint4 xor4(uint4 v, const State& s) {
  return make_uint4(v.x ^ s.s0, v.y ^ s.s1, v.z ^ s.s2, v.w ^ s.s3);
}

template <Op OP, int NR, int BPT>
__global__ void __launch_bounds__(1024, 1)
    ttable_kernel(const uint4* in, uint4* out, uint64_t nblocks, uint32_t tail_bytes,
                  const __grid_constant__ RoundKeys rk, const __grid_constant__ CtrParams cp) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr bool kDec = (OP == Op::kEcbDecrypt);
  pdl_launch_dependents();
  fill_tables<kDec>(smem);
  __syncthreads();
  pdl_wait_previous();  // the caller's buffers are touched only after this point

  const uint32_t lane = threadIdx.x & 31;
  const char* base = reinterpret_cast<const char*>(smem);
  const Tabs T{base, base + kRegionB, base + kRegionC, lane * 4, lane * 4 + 128};

  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x * BPT;
  for (uint64_t i0 = static_cast<uint64_t>(blockIdx.x) * blockDim.x * BPT + threadIdx.x;
       i0 < nblocks; i0 += stride) {
    uint4 v[BPT];
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      const uint64_t idx = i0 + static_cast<uint64_t>(k) * blockDim.x;
      v[k] = idx < nblocks ? __ldcs(in + idx) : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
      const uint64_t idx = i0 + static_cast<uint64_t>(k) * blockDim.x;
      uint4 r;
      if constexpr (OP == Op::kCtr) {
        r = xor4(v[k], ctr_keystream<NR>(T, rk, cp, idx));
      } else if constexpr (OP == Op::kEcbEncrypt) {
        State s{v[k].x ^ rk.w[0], v[k].y ^ rk.w[1], v[k].z ^ rk.w[2], v[k].w ^ rk.w[3]};
        encrypt_rounds<NR>(T, s, rk, 1);
        r = make_uint4(s.s0, s.s1, s.s2, s.s3);
      } else {
        State s{v[k].x ^ rk.w[0], v[k].y ^ rk.w[1], v[k].z ^ rk.w[2], v[k].w ^ rk.w[3]};
#pragma unroll
        for (int rr = 1; rr < NR; ++rr) dec_round(T, s, &rk.w[4 * rr]);
        dec_final(T, s, &rk.w[4 * NR]);
        r = make_uint4(s.s0, s.s1, s.s2, s.s3);
      }
      if (idx < nblocks) __stcs(out + idx, r);
    }
  }

  // CTR partial last block: its leading keystream bytes, one thread.
  if constexpr (OP == Op::kCtr) {
    if (tail_bytes != 0 && blockIdx.x == 0 && threadIdx.x == 0) {
      const State s = ctr_keystream<NR>(T, rk, cp, nblocks);
      const uint8_t* src = reinterpret_cast<const uint8_t*>(in + nblocks);
      uint8_t* dst = reinterpret_cast<uint8_t*>(out + nblocks);
      for (uint32_t b = 0; b < tail_bytes; ++b) {
        const uint32_t w = b < 4 ? s.s0 : b < 8 ? s.s1 : b < 12 ? s.s2 : s.s3;
        dst[b] = src[b] ^ static_cast<uint8_t>(w >> (8 * (b & 3)));
      }
    }
  }
}

// CTR with two cached rounds.  Counters that share their upper 24 bits
// (a run of 256 aligned counters) give the same state columns 1..3 after
// round 1 (only the counter's low byte, in column 0 of the round-1 output,
// changes), so 12 of round 2's 16 lookups are the same for the whole run.
// A warp walks one such run at a time, lane l taking counters 32k + l
// (k = 0..7, coalesced 512-byte accesses per k); each lane computes the run's
// constants once (3 + 12 lookups) and then spends 1 + 4 lookups per block on
// rounds 1-2 instead of 4 + 16.
//
// Runs that fill whole waves of the grid's warps go one per warp.  The runs
// of the last, partial wave are split into ctr_tail_pieces() pieces of 8/P
// steps each.  A piece costs its steps plus its own setup: the run's
// constants (15 lookups) and a loop that is not unrolled, about a quarter
// step together.  P is chosen so the busiest warp's share of that wave costs
// least, the fewest pieces on a tie: ceil(runs * P / warps) pieces of
// 4 * 8 / P + 1 quarter steps.  (At 64 MiB, 1,792 tail runs over 4,864
// warps: three one-step pieces, 15 quarter steps, against one four-step
// piece, 17.  At 16 MiB the 4,096 runs stay whole, one per warp of a
// 128-CTA grid: 33 against 35 for seven one-step pieces.)  The launch
// computes the split for its grid (CtrParams::whole_runs, tail_shift); a
// last wave left whole (P = 1) joins the full waves' loop.
__host__ __device__ __forceinline__ uint32_t ctr_tail_pieces(uint64_t tail_runs, uint64_t warps) {
  if (tail_runs == 0 || warps == 0) return 1;
  uint32_t best = 1;
  uint64_t best_cost = ~0ull;
  for (uint32_t p = 1; p <= 8; p *= 2) {
    const uint64_t cost = (tail_runs * p + warps - 1) / warps * (32 / p + 1);
    if (cost < best_cost) {
      best_cost = cost;
      best = p;
    }
  }
  return best;
}

// Steps [k0, k1) of one run.  kWhole: the whole run (k0 = 0, k1 = 8, known
// at compile time, unrolled by two); otherwise a piece, not unrolled.
template <int NR, bool kWhole>
__device__ __forceinline__ void ctr_run_steps(const Tabs& T, const uint4* in, uint4* out,
                                              uint64_t nblocks, uint64_t units, uint32_t tail_bytes,
                                              const RoundKeys& rk, const CtrParams& cp, uint32_t off0,
                                              uint64_t run, uint32_t k0, uint32_t k1, uint32_t lane) {
  if (kWhole) {
    k0 = 0;
    k1 = 8;
  }
  // counter of position 0 of this run (modulo 2^32); its low byte is 0
  const uint32_t ctr_run = (cp.ctr0 & ~255u) + static_cast<uint32_t>(run) * 256u;
  const uint32_t xr = __byte_perm(ctr_run, 0, 0x0123) ^ cp.rk0w3;  // byte 3 still to add
  const uint32_t s1 = cp.c1[1] ^ T.t2(xr), s2 = cp.c1[2] ^ T.t1(xr), s3 = cp.c1[3] ^ T.t0(xr);
  const uint32_t d0 = rk.w[8] ^ T.t1(s1) ^ T.t2(s2) ^ T.t3(s3);
  const uint32_t d1 = rk.w[9] ^ T.t0(s1) ^ T.t1(s2) ^ T.t2(s3);
  const uint32_t d2 = rk.w[10] ^ T.t0(s2) ^ T.t1(s3) ^ T.t3(s1);
  const uint32_t d3 = rk.w[11] ^ T.t0(s3) ^ T.t2(s1) ^ T.t3(s2);
  const int64_t first = static_cast<int64_t>(run) * 256 - off0;  // block index of position 0
#pragma unroll(kWhole ? 2 : 1)
  for (uint32_t k = k0; k < k1; ++k) {
    const uint32_t t = 32 * k + lane;
    const int64_t idx = first + t;
    if (idx < 0 || static_cast<uint64_t>(idx) >= units) continue;
    const bool full = static_cast<uint64_t>(idx) < nblocks;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (full) v = __ldcs(in + idx);
    const uint32_t s0 = cp.c1[0] ^ T.t3(xr ^ (t << 24));
    State s{d0 ^ T.t0(s0), d1 ^ T.t3(s0), d2 ^ T.t2(s0), d3 ^ T.t1(s0)};
    encrypt_rounds<NR>(T, s, rk, 3);
    if (full) {
      __stcs(out + idx, xor4(v, s));
    } else {  // partial last block: its leading keystream bytes
      const uint8_t* src = reinterpret_cast<const uint8_t*>(in + nblocks);
      uint8_t* dst = reinterpret_cast<uint8_t*>(out + nblocks);
      for (uint32_t b = 0; b < tail_bytes; ++b) {
        const uint32_t w = b < 4 ? s.s0 : b < 8 ? s.s1 : b < 12 ? s.s2 : s.s3;
        dst[b] = src[b] ^ static_cast<uint8_t>(w >> (8 * (b & 3)));
      }
    }
  }
}

template <int NR>
__global__ void __launch_bounds__(1024, 1)
    ttable_ctr_cached_kernel(const uint4* in, uint4* out, uint64_t nblocks, uint32_t tail_bytes,
                             const __grid_constant__ RoundKeys rk,
                             const __grid_constant__ CtrParams cp) {
  extern __shared__ __align__(16) uint32_t smem[];
  pdl_launch_dependents();
  fill_tables<false>(smem);
  __syncthreads();
  pdl_wait_previous();  // the caller's buffers are touched only after this point
  const uint32_t lane = threadIdx.x & 31;
  const char* base = reinterpret_cast<const char*>(smem);
  const Tabs T{base, base + kRegionB, base + kRegionC, lane * 4, lane * 4 + 128};

  const uint32_t off0 = cp.ctr0 & 255u;  // position of block 0 inside its run
  const uint64_t units = nblocks + (tail_bytes ? 1 : 0);
  const uint64_t runs = (units + off0 + 255) / 256;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
  const uint64_t wid = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t whole = cp.whole_runs;  // runs one per warp: the full waves, and a last wave left unsplit
  for (uint64_t run = wid; run < whole; run += warps)
    ctr_run_steps<NR, true>(T, in, out, nblocks, units, tail_bytes, rk, cp, off0, run, 0, 8, lane);
  const uint32_t shift = cp.tail_shift, steps = 8u >> shift;
  for (uint64_t piece = wid; piece < ((runs - whole) << shift); piece += warps) {
    const uint32_t k0 = (static_cast<uint32_t>(piece) & ((1u << shift) - 1)) * steps;
    ctr_run_steps<NR, false>(T, in, out, nblocks, units, tail_bytes, rk, cp, off0, whole + (piece >> shift),
                             k0, k0 + steps, lane);
  }
}

// ---------------------------------------------------------------------------
// TMA-staged variant of the run-cached CTR kernel (AES_VARIANT_TTABLE_BULK).
//
// The same rounds and counter-run caching, but each half run of input (128
// blocks, 2 KiB) is brought into a per-warp shared-memory buffer by one
// cp.async.bulk copy (the TMA engine, no LSU instructions) issued before the
// half run's keystream is computed, so the copy overlaps the rounds; the
// lanes then read their blocks from shared memory (LDS.128), XOR and store.
// Runs not wholly inside the buffer, and the split tail pieces, take the
// plain loads of ctr_run_steps.  No cluster, no multicast: every copy reads
// this GPU's own buffer into the issuing CTA's shared memory.
//
// Each wait on the buffer's mbarrier is bounded (about a second of SM
// clock): a warp whose copy has not landed by then counts the timeout in
// *timeouts, waits (again bounded) for its copy to finish, writes nothing
// more and returns.
constexpr uint32_t kBulkHalf = 128;                   // blocks per staged copy
constexpr uint32_t kBulkBytes = kBulkHalf * 16;       // 2 KiB per warp
__host__ __device__ constexpr int bulk_smem_bytes(int warps) {
  return kTtableSmemEnc + warps * static_cast<int>(kBulkBytes) + warps * 8;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// true once the mbarrier's phase with parity `parity` has completed, false
// after `limit` SM clocks
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

template <int NR>
__global__ void __launch_bounds__(1024, 1)
    ttable_ctr_bulk_kernel(const uint4* in, uint4* out, uint64_t nblocks, uint32_t tail_bytes,
                           const __grid_constant__ RoundKeys rk, const __grid_constant__ CtrParams cp,
                           unsigned int* timeouts) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr long long kWaitLimit = 2000000000ll;  // SM clocks, ~1 s at 2 GHz
  pdl_launch_dependents();
  fill_tables<false>(smem);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  char* stage_p = reinterpret_cast<char*>(smem) + kTtableSmemEnc + warp * kBulkBytes;
  const uint32_t stage = smem_addr(stage_p);
  const uint32_t mbar = smem_addr(reinterpret_cast<char*>(smem) + kTtableSmemEnc + nwarps * kBulkBytes) + 8 * warp;
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait_previous();  // the caller's buffers are touched only after this point
  const char* base = reinterpret_cast<const char*>(smem);
  const Tabs T{base, base + kRegionB, base + kRegionC, lane * 4, lane * 4 + 128};

  const uint32_t off0 = cp.ctr0 & 255u;
  const uint64_t units = nblocks + (tail_bytes ? 1 : 0);
  const uint64_t runs = (units + off0 + 255) / 256;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * nwarps;
  const uint64_t wid = static_cast<uint64_t>(blockIdx.x) * nwarps + warp;
  const uint64_t whole = cp.whole_runs;
  uint32_t parity = 0;
  for (uint64_t run = wid; run < whole; run += warps) {
    const int64_t first = static_cast<int64_t>(run) * 256 - off0;
    if (first < 0 || static_cast<uint64_t>(first) + 256 > nblocks) {  // a partial run: plain loads
      ctr_run_steps<NR, true>(T, in, out, nblocks, units, tail_bytes, rk, cp, off0, run, 0, 8, lane);
      continue;
    }
    const uint32_t ctr_run = (cp.ctr0 & ~255u) + static_cast<uint32_t>(run) * 256u;
    const uint32_t xr = __byte_perm(ctr_run, 0, 0x0123) ^ cp.rk0w3;
    const uint32_t s1 = cp.c1[1] ^ T.t2(xr), s2 = cp.c1[2] ^ T.t1(xr), s3 = cp.c1[3] ^ T.t0(xr);
    const uint32_t d0 = rk.w[8] ^ T.t1(s1) ^ T.t2(s2) ^ T.t3(s3);
    const uint32_t d1 = rk.w[9] ^ T.t0(s1) ^ T.t1(s2) ^ T.t2(s3);
    const uint32_t d2 = rk.w[10] ^ T.t0(s2) ^ T.t1(s3) ^ T.t3(s1);
    const uint32_t d3 = rk.w[11] ^ T.t0(s3) ^ T.t2(s1) ^ T.t3(s2);
#pragma unroll 1
    for (uint32_t h = 0; h < 2; ++h) {
      const uint4* src = in + first + kBulkHalf * h;
      __syncwarp();  // every lane's reads of the previous half are done
      if (lane == 0) {
        // order those generic-proxy reads before the copy's async-proxy writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(kBulkBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(stage),
            "l"(src), "r"(kBulkBytes), "r"(mbar)
            : "memory");
      }
      State ks[4];
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) {
        const uint32_t t = 32 * (4 * h + j) + lane;
        const uint32_t x0 = cp.c1[0] ^ T.t3(xr ^ (t << 24));
        State s{d0 ^ T.t0(x0), d1 ^ T.t3(x0), d2 ^ T.t2(x0), d3 ^ T.t1(x0)};
        encrypt_rounds<NR>(T, s, rk, 3);
        ks[j] = s;
      }
      if (!mbar_wait_bounded(mbar, parity, kWaitLimit)) {
        if (lane == 0) atomicAdd(timeouts, 1u);
        mbar_wait_bounded(mbar, parity, kWaitLimit);  // let the copy finish before the warp leaves
        return;
      }
      parity ^= 1u;
#pragma unroll
      for (uint32_t j = 0; j < 4; ++j) {
        const uint4 v = *reinterpret_cast<const uint4*>(stage_p + 16 * (32 * j + lane));
        __stcs(out + first + kBulkHalf * h + 32 * j + lane, xor4(v, ks[j]));
      }
    }
  }
  const uint32_t shift = cp.tail_shift, steps = 8u >> shift;
  for (uint64_t piece = wid; piece < ((runs - whole) << shift); piece += warps) {
    const uint32_t k0 = (static_cast<uint32_t>(piece) & ((1u << shift) - 1)) * steps;
    ctr_run_steps<NR, false>(T, in, out, nblocks, units, tail_bytes, rk, cp, off0, whole + (piece >> shift),
                             k0, k0 + steps, lane);
  }
}

}  // namespace
}  // namespace aesgpu
