// aes_tables.cuh — AES constant tables of the GPU library, generated at
// compile time from GF(2^8) arithmetic (FIPS-197 §4.2, §5.1.1).
//
// Route: every nonzero field element is a power of the generator {03}; the
// exp/log tables of {03} give the multiplicative inverse as
// exp[255 - log x], and the S-box is that inverse through the affine map of
// FIPS-197 eq. (5.1), written bit by bit.  From the S-box come the lookup
// words the round kernels use (little-endian byte order, byte 0 = row 0):
//   te0[x] = ( 2*S(x),  S(x),   S(x),   3*S(x) )   (SubBytes+MixColumns, row 0)
//   td0[x] = ( e*IS(x), 9*IS(x), d*IS(x), b*IS(x) ) (InvSubBytes+InvMixColumns)
//   is4[x] = IS(x) in all four bytes              (final inverse round)
// Rows 1..3 are byte rotations of row 0 and are built when the kernels fill
// shared memory.
#pragma once
#include <cstdint>

namespace aesgpu {

struct GfTables {
  uint8_t exp[256];
  uint8_t log[256];
};

constexpr uint8_t gf_xtime(uint8_t a) {
  return (uint8_t)((a << 1) ^ ((a & 0x80) ? 0x1B : 0x00));
}

constexpr GfTables make_gf() {
  GfTables g{};
  uint8_t e = 1;
  for (int i = 0; i < 255; ++i) {
    g.exp[i] = e;
    g.log[e] = (uint8_t)i;
    e = (uint8_t)(gf_xtime(e) ^ e);  // e * {03}
  }
  g.exp[255] = g.exp[0];
  return g;
}

constexpr GfTables kGf = make_gf();

constexpr uint8_t gf_mul(uint8_t a, uint8_t b) {
  return (a == 0 || b == 0) ? 0 : kGf.exp[(kGf.log[a] + kGf.log[b]) % 255];
}

constexpr uint8_t gf_inverse(uint8_t a) {
  return a == 0 ? 0 : kGf.exp[(255 - kGf.log[a]) % 255];
}

// FIPS-197 eq. (5.1): b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i, c = {63}.
constexpr uint8_t affine(uint8_t b) {
  uint8_t out = 0;
  for (int i = 0; i < 8; ++i) {
    int bit = ((b >> i) ^ (b >> ((i + 4) & 7)) ^ (b >> ((i + 5) & 7)) ^ (b >> ((i + 6) & 7)) ^
               (b >> ((i + 7) & 7)) ^ (0x63 >> i)) & 1;
    out = (uint8_t)(out | (bit << i));
  }
  return out;
}

struct AesTables {
  uint8_t sbox[256];
  uint8_t inv_sbox[256];
  uint32_t te0[256];
  uint32_t td0[256];
  uint32_t is4[256];
};

constexpr uint32_t pack(uint8_t b0, uint8_t b1, uint8_t b2, uint8_t b3) {
  return (uint32_t)b0 | ((uint32_t)b1 << 8) | ((uint32_t)b2 << 16) | ((uint32_t)b3 << 24);
}

constexpr AesTables make_tables() {
  AesTables t{};
  for (int x = 0; x < 256; ++x) t.sbox[x] = affine(gf_inverse((uint8_t)x));
  for (int x = 0; x < 256; ++x) t.inv_sbox[t.sbox[x]] = (uint8_t)x;
  for (int x = 0; x < 256; ++x) {
    const uint8_t s = t.sbox[x], is = t.inv_sbox[x];
    t.te0[x] = pack(gf_mul(s, 2), s, s, gf_mul(s, 3));
    t.td0[x] = pack(gf_mul(is, 14), gf_mul(is, 9), gf_mul(is, 13), gf_mul(is, 11));
    t.is4[x] = pack(is, is, is, is);
  }
  return t;
}

// One copy for host code (key schedules, CTR precomputation).
constexpr AesTables kHostTables = make_tables();

constexpr uint32_t rotl32(uint32_t v, int k) { return (v << k) | (v >> (32 - k)); }

}  // namespace aesgpu
