// aes_modes.cu — the two other block-parallel modes on the T-table rounds:
//
// CBC decryption (SP 800-38A §6.2):  P_j = InvCipher(C_j) ^ C_{j-1}, C_{-1} = IV.
//   Each thread decrypts one block (equivalent inverse cipher, as ECB) and XORs
//   the preceding ciphertext block, which the neighbouring lane has just
//   loaded (so it comes from L1).  In place is refused by the C ABI: a block's
//   predecessor must still be ciphertext when it is read.
//
// XTS (IEEE 1619 / SP 800-38E, data units a multiple of 512 bytes, no
// ciphertext stealing):  for block j of data unit u,
//   T_u = Cipher_K2(LE128(first_sector + u)),  T_uj = T_u * alpha^j in GF(2^128),
//   C = Cipher_K1(P ^ T_uj) ^ T_uj   (decryption: InvCipher_K1 in the middle).
//   A warp owns 32 chunks of 32 blocks; lane l computes T_u for chunk l's unit
//   (one tweak encryption per lane per 1024 blocks), chunk k's tweak reaches
//   all lanes by shuffle, and block 32q + l of a unit gets
//   T_u * alpha^(32q) (carried from chunk to chunk) * alpha^l, each factor a
//   128-bit shift whose shifted-out bits fold back times {87} (the reduction
//   polynomial x^128 + x^7 + x^2 + x + 1).
//   Decryption tables hold td0..3 and the inverse S-box; the tweak cipher runs
//   there on te0 alone (its rotations give te1..3), kept in the spare half of
//   the inverse S-box rows.
#include "aes_internal.h"
#include "aes_smem_attr.h"
#include "aes_ttable.cuh"

namespace aesgpu {
namespace {

// ---------------------------------------------------------------- CBC ----

template <int NR>
__global__ void __launch_bounds__(1024, 1)
    cbc_decrypt_kernel(const uint4* in, uint4* out, uint64_t nblocks,
                       const __grid_constant__ RoundKeys rk, const __grid_constant__ CtrParams cp) {
  extern __shared__ __align__(16) uint32_t smem[];
  pdl_launch_dependents();
  fill_tables<true>(smem);
  __syncthreads();
  pdl_wait_previous();  // the caller's buffers are touched only after this point
  const uint32_t lane = threadIdx.x & 31;
  const char* base = reinterpret_cast<const char*>(smem);
  const Tabs T{base, base + kRegionB, base + kRegionC, lane * 4, lane * 4 + 128};
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t idx = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nblocks;
       idx += stride) {
    const uint4 c = __ldg(in + idx);
    const uint4 prev = idx ? __ldg(in + idx - 1) : make_uint4(cp.iv_w[0], cp.iv_w[1], cp.iv_w[2], cp.iv_w[3]);
    State s{c.x ^ rk.w[0], c.y ^ rk.w[1], c.z ^ rk.w[2], c.w ^ rk.w[3]};
#pragma unroll
    for (int r = 1; r < NR; ++r) dec_round(T, s, &rk.w[4 * r]);
    dec_final(T, s, &rk.w[4 * NR]);
    __stcs(out + idx, make_uint4(s.s0 ^ prev.x, s.s1 ^ prev.y, s.s2 ^ prev.z, s.s3 ^ prev.w));
  }
}

// ---------------------------------------------------------------- XTS ----

struct Tweak {
  uint32_t w0, w1, w2, w3;  // little-endian 128-bit value, w0 least significant
};

// clmul(h, {87}) for h < 2^32: h ^ h<<1 ^ h<<2 ^ h<<7 as a 64-bit value.
__device__ __forceinline__ uint64_t fold87(uint32_t h) {
  const uint64_t x = h;
  return x ^ (x << 1) ^ (x << 2) ^ (x << 7);
}

// t * alpha^r, 0 <= r < 32: shift the 128-bit value left by r, fold back the
// r bits shifted out (h * alpha^128 = h * (alpha^7 + alpha^2 + alpha + 1)).
__device__ __forceinline__ Tweak mul_alpha_r(const Tweak& t, uint32_t r) {
  const uint32_t h = r ? (t.w3 >> (32 - r)) : 0u;
  Tweak o{t.w0 << r, __funnelshift_l(t.w0, t.w1, r), __funnelshift_l(t.w1, t.w2, r),
          __funnelshift_l(t.w2, t.w3, r)};
  const uint64_t f = fold87(h);
  o.w0 ^= static_cast<uint32_t>(f);
  o.w1 ^= static_cast<uint32_t>(f >> 32);
  return o;
}

// t * alpha^32: move up one word, fold back the top word.
__device__ __forceinline__ Tweak mul_alpha32(const Tweak& t) {
  const uint64_t f = fold87(t.w3);
  return Tweak{static_cast<uint32_t>(f), t.w0 ^ static_cast<uint32_t>(f >> 32), t.w1, t.w2};
}

// Cipher with only te0 (Ti = rotl(te0, 8i)) in the upper half of region C.
struct Te0Only {
  const char* c;
  uint32_t hi;
  __device__ __forceinline__ uint32_t t(uint32_t x, int i) const {
    const uint32_t v = *reinterpret_cast<const uint32_t*>(c + __byte_perm(x, hi, 0x5504 | (i << 4)));
    return i ? __funnelshift_l(v, v, 8 * i) : v;
  }
};

__device__ __forceinline__ State encrypt_te0(const Te0Only& T, State s, const RoundKeys& rk, int nr) {
  s = State{s.s0 ^ rk.w[0], s.s1 ^ rk.w[1], s.s2 ^ rk.w[2], s.s3 ^ rk.w[3]};
  for (int r = 1; r < nr; ++r) {
    const uint32_t* k = &rk.w[4 * r];
    const uint32_t t0 = T.t(s.s0, 0) ^ T.t(s.s1, 1) ^ T.t(s.s2, 2) ^ T.t(s.s3, 3) ^ k[0];
    const uint32_t t1 = T.t(s.s1, 0) ^ T.t(s.s2, 1) ^ T.t(s.s3, 2) ^ T.t(s.s0, 3) ^ k[1];
    const uint32_t t2 = T.t(s.s2, 0) ^ T.t(s.s3, 1) ^ T.t(s.s0, 2) ^ T.t(s.s1, 3) ^ k[2];
    const uint32_t t3 = T.t(s.s3, 0) ^ T.t(s.s0, 1) ^ T.t(s.s1, 2) ^ T.t(s.s2, 3) ^ k[3];
    s = State{t0, t1, t2, t3};
  }
  // final round: S(x) is byte 1 of te0
  auto fin = [&](uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t k) {
    const uint32_t va = *reinterpret_cast<const uint32_t*>(T.c + __byte_perm(a, T.hi, 0x5504));
    const uint32_t vb = *reinterpret_cast<const uint32_t*>(T.c + __byte_perm(b, T.hi, 0x5514));
    const uint32_t vc = *reinterpret_cast<const uint32_t*>(T.c + __byte_perm(c, T.hi, 0x5524));
    const uint32_t vd = *reinterpret_cast<const uint32_t*>(T.c + __byte_perm(d, T.hi, 0x5534));
    return __byte_perm(__byte_perm(va, vb, 0x0051), __byte_perm(vc, vd, 0x5100), 0x7610) ^ k;
  };
  const uint32_t* k = &rk.w[4 * nr];
  return State{fin(s.s0, s.s1, s.s2, s.s3, k[0]), fin(s.s1, s.s2, s.s3, s.s0, k[1]),
               fin(s.s2, s.s3, s.s0, s.s1, k[2]), fin(s.s3, s.s0, s.s1, s.s2, k[3])};
}

struct XtsParams {
  uint64_t first_sector;
  uint32_t sector_blocks;  // a multiple of 32
  uint32_t nr_tweak;
};

template <bool kDec, int NR>
__global__ void __launch_bounds__(1024, 1)
    xts_kernel(const uint4* in, uint4* out, uint64_t nblocks, const __grid_constant__ RoundKeys rk1,
               const __grid_constant__ RoundKeys rk2, const __grid_constant__ XtsParams xp) {
  extern __shared__ __align__(16) uint32_t smem[];
  pdl_launch_dependents();
  fill_tables<kDec>(smem);
  if (kDec) {  // te0 replicas in the upper half of each inverse S-box row, for the tweak cipher
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int x = warp; x < 256; x += nwarps) smem[kRegionC / 4 + x * 64 + 32 + lane] = kDevTables.te0[x];
  }
  __syncthreads();
  pdl_wait_previous();  // the caller's buffers are touched only after this point
  const uint32_t lane = threadIdx.x & 31;
  const char* base = reinterpret_cast<const char*>(smem);
  const Tabs T{base, base + kRegionB, base + kRegionC, lane * 4, lane * 4 + 128};
  const Te0Only T0{base + kRegionC, lane * 4 + 128};

  const uint64_t nchunks = nblocks / 32;  // nblocks is a multiple of 32
  const uint64_t groups = (nchunks + 31) / 32;
  const uint64_t warps = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
  for (uint64_t g = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
       g < groups; g += warps) {
    // lane l: the encrypted tweak of the unit holding chunk 32g + l
    const uint64_t my_chunk = 32 * g + lane;
    const uint64_t unit = (my_chunk * 32) / xp.sector_blocks;
    const uint64_t tv = xp.first_sector + unit;
    State t{static_cast<uint32_t>(tv), static_cast<uint32_t>(tv >> 32), 0u, 0u};
    if (kDec) {
      t = encrypt_te0(T0, t, rk2, static_cast<int>(xp.nr_tweak));
    } else {
      t = State{t.s0 ^ rk2.w[0], t.s1 ^ rk2.w[1], t.s2 ^ rk2.w[2], t.s3 ^ rk2.w[3]};
      for (int r = 1; r < static_cast<int>(xp.nr_tweak); ++r) enc_round(T, t, &rk2.w[4 * r]);
      enc_final(T, t, &rk2.w[4 * xp.nr_tweak]);
    }
    Tweak tq{0, 0, 0, 0};  // tweak of the current chunk's first block (uniform over the warp)
    for (uint32_t k = 0; k < 32; ++k) {
      const uint64_t chunk = 32 * g + k;
      if (chunk >= nchunks) break;
      const uint32_t jb = static_cast<uint32_t>((chunk * 32) % xp.sector_blocks);
      if (k == 0 || jb == 0) {  // a new unit (or the group's first chunk): its tweak from lane k
        tq = Tweak{__shfl_sync(0xffffffffu, t.s0, k), __shfl_sync(0xffffffffu, t.s1, k),
                   __shfl_sync(0xffffffffu, t.s2, k), __shfl_sync(0xffffffffu, t.s3, k)};
        for (uint32_t q = 0; q < jb / 32; ++q) tq = mul_alpha32(tq);
      } else {
        tq = mul_alpha32(tq);  // the next 32 blocks of the same unit
      }
      const Tweak tj = mul_alpha_r(tq, lane);
      const uint64_t idx = chunk * 32 + lane;
      const uint4 v = __ldcs(in + idx);
      State s{v.x ^ tj.w0 ^ rk1.w[0], v.y ^ tj.w1 ^ rk1.w[1], v.z ^ tj.w2 ^ rk1.w[2], v.w ^ tj.w3 ^ rk1.w[3]};
      if (kDec) {
#pragma unroll
        for (int r = 1; r < NR; ++r) dec_round(T, s, &rk1.w[4 * r]);
        dec_final(T, s, &rk1.w[4 * NR]);
      } else {
        encrypt_rounds<NR>(T, s, rk1, 1);
      }
      __stcs(out + idx, make_uint4(s.s0 ^ tj.w0, s.s1 ^ tj.w1, s.s2 ^ tj.w2, s.s3 ^ tj.w3));
    }
  }
}

template <int NR>
cudaError_t launch_cbc(const void* in, void* out, uint64_t nblocks, const RoundKeys& rk,
                       const CtrParams& cp, const LaunchShape& shape, cudaStream_t stream) {
  auto kern = cbc_decrypt_kernel<NR>;
  cudaError_t e = ensure_dynamic_smem(kern, kTtableSmemDec);
  if (e != cudaSuccess) return e;
  const uint64_t needed = (nblocks + shape.cta_threads - 1) / shape.cta_threads;
  const uint64_t ctas = static_cast<uint64_t>(shape.grid_ctas);  // positive: resolved by the caller
  const uint64_t grid = ctas < needed ? ctas : (needed ? needed : 1);
  return launch_pdl(kern, static_cast<unsigned>(grid), shape.cta_threads, kTtableSmemDec, stream,
                    static_cast<const uint4*>(in), static_cast<uint4*>(out), nblocks, rk, cp);
}

template <bool kDec, int NR>
cudaError_t launch_xts(const void* in, void* out, uint64_t nblocks, const RoundKeys& rk1,
                       const RoundKeys& rk2, const XtsParams& xp, const LaunchShape& shape,
                       cudaStream_t stream) {
  auto kern = xts_kernel<kDec, NR>;
  const int smem = kDec ? kTtableSmemDec : kTtableSmemEnc;
  cudaError_t e = ensure_dynamic_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const uint64_t groups = (nblocks / 32 + 31) / 32;
  const uint64_t warps_per_cta = shape.cta_threads / 32;
  const uint64_t needed = (groups + warps_per_cta - 1) / warps_per_cta;
  const uint64_t ctas = static_cast<uint64_t>(shape.grid_ctas);  // positive: resolved by the caller
  const uint64_t grid = ctas < needed ? ctas : (needed ? needed : 1);
  return launch_pdl(kern, static_cast<unsigned>(grid), shape.cta_threads, static_cast<size_t>(smem), stream,
                    static_cast<const uint4*>(in), static_cast<uint4*>(out), nblocks, rk1, rk2, xp);
}

}  // namespace

cudaError_t launch_cbc_decrypt(int nr, const void* in, void* out, uint64_t nblocks, const RoundKeys& rk,
                               const CtrParams& cp, const LaunchShape& shape, cudaStream_t stream) {
  switch (nr) {
    case 10: return launch_cbc<10>(in, out, nblocks, rk, cp, shape, stream);
    case 12: return launch_cbc<12>(in, out, nblocks, rk, cp, shape, stream);
    case 14: return launch_cbc<14>(in, out, nblocks, rk, cp, shape, stream);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_xts_mode(bool decrypt, int nr, int nr_tweak, const void* in, void* out,
                            uint64_t nblocks, const RoundKeys& rk1, const RoundKeys& rk2,
                            uint64_t first_sector, uint32_t sector_blocks, const LaunchShape& shape,
                            cudaStream_t stream) {
  const XtsParams xp{first_sector, sector_blocks, static_cast<uint32_t>(nr_tweak)};
  switch ((decrypt ? 100 : 0) + nr) {
    case 10: return launch_xts<false, 10>(in, out, nblocks, rk1, rk2, xp, shape, stream);
    case 12: return launch_xts<false, 12>(in, out, nblocks, rk1, rk2, xp, shape, stream);
    case 14: return launch_xts<false, 14>(in, out, nblocks, rk1, rk2, xp, shape, stream);
    case 110: return launch_xts<true, 10>(in, out, nblocks, rk1, rk2, xp, shape, stream);
    case 112: return launch_xts<true, 12>(in, out, nblocks, rk1, rk2, xp, shape, stream);
    case 114: return launch_xts<true, 14>(in, out, nblocks, rk1, rk2, xp, shape, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace aesgpu
