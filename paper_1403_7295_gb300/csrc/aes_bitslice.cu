// aes_bitslice.cu — single-buffer AES kernels, bitsliced round variant.
//
// Each thread carries 16 AES blocks as 64 bit-slice words.  Register
// st[32h + 8r + b] (h = 0, 1; r = row; b = bit) holds bit b of state byte
// (row r, column h) of the 16 blocks in its low half and bit b of byte
// (row r, column h + 2) in its high half, block k in bit k (low) / 16 + k
// (high).  Stacking column word h of the 16 blocks over column word h + 2
// gives a 32x32 bit matrix whose transpose is exactly st[32h .. 32h + 31].
//
// A round (paper Fig. 1 step 3) is then:
//   SubBytes     the S-box circuit of aes_bitslice_circuit.cuh on the 8 slices
//                of each (row, column pair): no table, no data-dependent address;
//   ShiftRows    row 2 moves by two columns = swap the halves of its registers;
//                rows 1 and 3 exchange the two registers of a pair, one of them
//                half-swapped;
//   MixColumns   out_r = a_r ^ t ^ xtime(a_r ^ a_{r+1}), t = a_0 ^ a_1 ^ a_2 ^ a_3,
//                on both packed columns at once;
//   AddRoundKey  XOR with masks (all ones per half where the key bit is set).
// Decryption follows FIPS-197 §5.3 in its plain order, with InvMixColumns as
// MixColumns after a'_r = a_r ^ 4(a_r ^ a_{r+2}) (circulant (05 00 04 00)).
//
// Work split: a warp owns 512 consecutive blocks; lane l takes blocks
// base + 32k + l (k = 0..15), so each warp-wide load and store is 512
// contiguous bytes.  The rounds are logic on the ALU pipe; the round-key
// masks are broadcast shared-memory loads.
#include "aes_bitslice_circuit.cuh"
#include "aes_internal.h"

namespace aesgpu {
namespace {

constexpr int kBsThreads = kBitsliceThreads;
constexpr int kBlocksPerThread = 16;

__device__ __forceinline__ uint32_t bswap32(uint32_t v) { return __byte_perm(v, 0, 0x0123); }
__device__ __forceinline__ uint32_t swap_halves(uint32_t v) { return __byte_perm(v, 0, 0x1032); }

// In-place transpose of a 32x32 bit matrix: bit j of a[k] <-> bit k of a[j].
// Quadrant swaps: halves and bytes by PRMT, nibbles / pairs / bits by masks.
__device__ __forceinline__ void transpose32(uint32_t* a) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t x = a[k], y = a[k + 16];
    a[k] = __byte_perm(x, y, 0x5410);
    a[k + 16] = __byte_perm(x, y, 0x7632);
  }
#pragma unroll
  for (int k = 0; k < 32; k = (k + 9) & ~8) {
    const uint32_t x = a[k], y = a[k + 8];
    a[k] = __byte_perm(x, y, 0x6240);
    a[k + 8] = __byte_perm(x, y, 0x7351);
  }
#pragma unroll
  for (int k = 0; k < 32; k = (k + 5) & ~4) {
    const uint32_t t = ((a[k] >> 4) ^ a[k + 4]) & 0x0F0F0F0Fu;
    a[k + 4] ^= t;
    a[k] ^= t << 4;
  }
#pragma unroll
  for (int k = 0; k < 32; k = (k + 3) & ~2) {
    const uint32_t t = ((a[k] >> 2) ^ a[k + 2]) & 0x33333333u;
    a[k + 2] ^= t;
    a[k] ^= t << 2;
  }
#pragma unroll
  for (int k = 0; k < 32; k += 2) {
    const uint32_t t = ((a[k] >> 1) ^ a[k + 1]) & 0x55555555u;
    a[k + 1] ^= t;
    a[k] ^= t << 1;
  }
}

__device__ __forceinline__ void sub_bytes(uint32_t* st) {
#pragma unroll
  for (int g = 0; g < 8; ++g) {  // (column pair, row) groups of 8 slices
    uint32_t* x = st + 8 * g;
    bs_sbox(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
  }
}

__device__ __forceinline__ void inv_sub_bytes(uint32_t* st) {
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    uint32_t* x = st + 8 * g;
    bs_inv_sbox(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
  }
}

// ShiftRows (DIR = +1: new column c = old c + r) or InvShiftRows (DIR = -1).
// Pair registers: P0 = (col 0 | col 2), P1 = (col 1 | col 3).
//   shift by 1: new P0 = (c1 | c3) = P1, new P1 = (c2 | c0) = swap(P0)
//   shift by 2: new P0 = swap(P0), new P1 = swap(P1)
//   shift by 3: new P0 = (c3 | c1) = swap(P1), new P1 = (c0 | c2) = P0
template <int DIR>
__device__ __forceinline__ void shift_rows(uint32_t* st) {
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    {  // row 1
      uint32_t& p0 = st[8 * 1 + b];
      uint32_t& p1 = st[32 + 8 * 1 + b];
      const uint32_t o0 = p0, o1 = p1;
      if (DIR > 0) { p0 = o1; p1 = swap_halves(o0); }
      else { p0 = swap_halves(o1); p1 = o0; }
    }
    {  // row 2
      st[8 * 2 + b] = swap_halves(st[8 * 2 + b]);
      st[32 + 8 * 2 + b] = swap_halves(st[32 + 8 * 2 + b]);
    }
    {  // row 3
      uint32_t& p0 = st[8 * 3 + b];
      uint32_t& p1 = st[32 + 8 * 3 + b];
      const uint32_t o0 = p0, o1 = p1;
      if (DIR > 0) { p0 = swap_halves(o1); p1 = o0; }
      else { p0 = o1; p1 = swap_halves(o0); }
    }
  }
}

// y = x * {02} on 8 slices (bit 0 first): shift up, reduce by x^8 = x^4 + x^3 + x + 1.
__device__ __forceinline__ void xtime8(const uint32_t* x, uint32_t* y) {
  y[0] = x[7];
  y[1] = x[0] ^ x[7];
  y[2] = x[1];
  y[3] = x[2] ^ x[7];
  y[4] = x[3] ^ x[7];
  y[5] = x[4];
  y[6] = x[5];
  y[7] = x[6];
}

// MixColumns on the column pair h, in place:
// out_r = a_r ^ t ^ xtime(a_r ^ a_{r+1}),  t = a_0 ^ a_1 ^ a_2 ^ a_3.
__device__ __forceinline__ void mix_pair(uint32_t* st, int h) {
  uint32_t* a = st + 32 * h;  // row r at a + 8r
  uint32_t t[8], a0[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    a0[b] = a[b];
    t[b] = a[b] ^ a[8 + b] ^ a[16 + b] ^ a[24 + b];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    uint32_t u[8], xt[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) u[b] = a[8 * r + b] ^ (r == 3 ? a0[b] : a[8 * (r + 1) + b]);
    xtime8(u, xt);
#pragma unroll
    for (int b = 0; b < 8; ++b) a[8 * r + b] ^= t[b] ^ xt[b];
  }
}

__device__ __forceinline__ void mix_columns(uint32_t* st) {
  mix_pair(st, 0);
  mix_pair(st, 1);
}

// InvMixColumns = MixColumns after a'_r = a_r ^ 4 (a_r ^ a_{r+2}).
__device__ __forceinline__ void inv_mix_columns(uint32_t* st) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t* a = st + 32 * h;
#pragma unroll
    for (int r = 0; r < 2; ++r) {  // v = a_r ^ a_{r+2} serves rows r and r + 2
      uint32_t v[8], x2[8], x4[8];
#pragma unroll
      for (int b = 0; b < 8; ++b) v[b] = a[8 * r + b] ^ a[8 * (r + 2) + b];
      xtime8(v, x2);
      xtime8(x2, x4);
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        a[8 * r + b] ^= x4[b];
        a[8 * (r + 2) + b] ^= x4[b];
      }
    }
    mix_pair(st, h);
  }
}

__device__ __forceinline__ void add_round_key(uint32_t* st, const uint32_t* mask) {
#pragma unroll
  for (int q = 0; q < 64; q += 4) {
    const uint4 m = *reinterpret_cast<const uint4*>(mask + q);
    st[q] ^= m.x;
    st[q + 1] ^= m.y;
    st[q + 2] ^= m.z;
    st[q + 3] ^= m.w;
  }
}

// Pack the four column words of 16 blocks (w[c][k]) into slices: rows 0..15
// of matrix h are column h, rows 16..31 column h + 2.
__device__ __forceinline__ void to_slices(uint32_t* st) { transpose32(st); transpose32(st + 32); }

template <Op OP, int NR>
__global__ void __launch_bounds__(kBsThreads)
    bitslice_kernel(const uint4* in, uint4* out, uint64_t nblocks, uint32_t tail_bytes,
                    const __grid_constant__ RoundKeys rk, const __grid_constant__ CtrParams cp) {
  // masks[r][32h + j]: low half all ones if bit j of round-key word 4r + h is
  // set, high half likewise for word 4r + h + 2
  __shared__ __align__(16) uint32_t masks[(NR + 1) * 64];
  for (int i = threadIdx.x; i < (NR + 1) * 64; i += blockDim.x) {
    const int r = i / 64, h = (i % 64) / 32, j = i % 32;
    const uint32_t lo = (rk.w[4 * r + h] >> j) & 1u, hi = (rk.w[4 * r + h + 2] >> j) & 1u;
    masks[i] = (lo ? 0x0000FFFFu : 0u) | (hi ? 0xFFFF0000u : 0u);
  }
  __syncthreads();

  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps_total = static_cast<uint64_t>(gridDim.x) * (blockDim.x / 32);
  const uint64_t units = nblocks + (tail_bytes ? 1 : 0);  // the partial CTR block too
  const uint64_t chunks = (units + 511) / 512;
  for (uint64_t chunk = static_cast<uint64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
       chunk < chunks; chunk += warps_total) {
    const uint64_t base = chunk * 512 + lane;
    // st[32h + k] = column h of block k, st[32h + 16 + k] = column h + 2 of block k
    uint32_t st[64];
#pragma unroll
    for (int k = 0; k < kBlocksPerThread; ++k) {
      const uint64_t idx = base + 32ull * k;
      uint4 v;
      if constexpr (OP == Op::kCtr) {
        v = make_uint4(cp.iv_w[0], cp.iv_w[1], cp.iv_w[2],
                       bswap32(cp.ctr0 + static_cast<uint32_t>(idx)));
      } else {
        v = idx < nblocks ? __ldcs(in + idx) : make_uint4(0, 0, 0, 0);
      }
      st[k] = v.x;
      st[16 + k] = v.z;
      st[32 + k] = v.y;
      st[48 + k] = v.w;
    }
    to_slices(st);

    if constexpr (OP == Op::kEcbDecrypt) {
      add_round_key(st, masks + NR * 64);
#pragma unroll 1
      for (int r = NR - 1; r >= 1; --r) {
        shift_rows<-1>(st);
        inv_sub_bytes(st);
        add_round_key(st, masks + r * 64);
        inv_mix_columns(st);
      }
      shift_rows<-1>(st);
      inv_sub_bytes(st);
      add_round_key(st, masks);
    } else {
      add_round_key(st, masks);
#pragma unroll 1
      for (int r = 1; r < NR; ++r) {
        sub_bytes(st);
        shift_rows<1>(st);
        mix_columns(st);
        add_round_key(st, masks + r * 64);
      }
      sub_bytes(st);
      shift_rows<1>(st);
      add_round_key(st, masks + NR * 64);
    }

    to_slices(st);  // the transpose is its own inverse: back to column words
    if constexpr (OP == Op::kCtr) {
      // The data to XOR: eight blocks' loads issued together, then their
      // stores (in and out may be the same buffer, so a load cannot move
      // above an earlier store; one at a time would wait a memory round
      // trip per block).
#pragma unroll
      for (int g = 0; g < kBlocksPerThread; g += 8) {
        uint4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const uint64_t idx = base + 32ull * (g + j);
          v[j] = idx < nblocks ? __ldcs(in + idx) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int k = g + j;
          const uint64_t idx = base + 32ull * k;
          const uint4 r = make_uint4(st[k], st[32 + k], st[16 + k], st[48 + k]);
          if (idx < nblocks) {
            __stcs(out + idx, make_uint4(v[j].x ^ r.x, v[j].y ^ r.y, v[j].z ^ r.z, v[j].w ^ r.w));
          } else if (idx == nblocks && tail_bytes) {  // partial last block
            const uint8_t* src = reinterpret_cast<const uint8_t*>(in + nblocks);
            uint8_t* dst = reinterpret_cast<uint8_t*>(out + nblocks);
            for (uint32_t b = 0; b < tail_bytes; ++b) {
              const uint32_t w = b < 4 ? r.x : b < 8 ? r.y : b < 12 ? r.z : r.w;
              dst[b] = src[b] ^ static_cast<uint8_t>(w >> (8 * (b & 3)));
            }
          }
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < kBlocksPerThread; ++k) {
        const uint64_t idx = base + 32ull * k;
        if (idx < nblocks) __stcs(out + idx, make_uint4(st[k], st[32 + k], st[16 + k], st[48 + k]));
      }
    }
  }
}

template <Op OP, int NR>
cudaError_t launch_bs(const void* in, void* out, uint64_t nblocks, uint32_t tail, const RoundKeys& rk,
                      const CtrParams& cp, const LaunchShape& shape, cudaStream_t stream) {
  auto kern = bitslice_kernel<OP, NR>;
  int grid = shape.grid_ctas;
  if (grid == 0) {  // as many CTAs as fit on every SM at once
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBsThreads, 0);
    if (e != cudaSuccess) return e;
    grid = sms * (per_sm > 0 ? per_sm : 1);
  }
  const uint64_t units = nblocks + (tail ? 1 : 0);
  const uint64_t needed = (units + kBitsliceBlocksPerCta - 1) / kBitsliceBlocksPerCta;
  if (static_cast<uint64_t>(grid) > needed) grid = static_cast<int>(needed > 0 ? needed : 1);
  kern<<<grid, kBsThreads, 0, stream>>>(static_cast<const uint4*>(in), static_cast<uint4*>(out),
                                        nblocks, tail, rk, cp);
  return cudaGetLastError();
}

template <Op OP>
cudaError_t dispatch_bs(int nr, const void* in, void* out, uint64_t nblocks, uint32_t tail,
                        const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                        cudaStream_t stream) {
  switch (nr) {
    case 10: return launch_bs<OP, 10>(in, out, nblocks, tail, rk, cp, shape, stream);
    case 12: return launch_bs<OP, 12>(in, out, nblocks, tail, rk, cp, shape, stream);
    case 14: return launch_bs<OP, 14>(in, out, nblocks, tail, rk, cp, shape, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_bitslice(Op op, int nr, const void* in, void* out, uint64_t nblocks,
                            uint32_t tail_bytes, const RoundKeys& rk, const CtrParams& cp,
                            const LaunchShape& shape, cudaStream_t stream) {
  switch (op) {
    case Op::kEcbEncrypt: return dispatch_bs<Op::kEcbEncrypt>(nr, in, out, nblocks, 0, rk, cp, shape, stream);
    case Op::kEcbDecrypt: return dispatch_bs<Op::kEcbDecrypt>(nr, in, out, nblocks, 0, rk, cp, shape, stream);
    case Op::kCtr: return dispatch_bs<Op::kCtr>(nr, in, out, nblocks, tail_bytes, rk, cp, shape, stream);
  }
  return cudaErrorInvalidValue;
}

}  // namespace aesgpu
