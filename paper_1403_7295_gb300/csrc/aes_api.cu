// aes_api.cu — the C ABI of libaesgpu.so: key expansion on the host, argument
// validation, launch-shape choice and dispatch to the round kernels.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "aes_batch.h"
#include "aes_internal.h"
#include "aes_tables.cuh"
#include "aesgpu.h"

namespace aesgpu {
namespace {

thread_local int g_last_cuda_error = 0;

aes_status cuda_failure(cudaError_t e) {
  g_last_cuda_error = static_cast<int>(e);
  return AES_ERR_CUDA;
}

constexpr const AesTables& H = kHostTables;

uint32_t load_le32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

uint32_t sub_word(uint32_t w) {
  return pack(H.sbox[w & 0xFF], H.sbox[(w >> 8) & 0xFF], H.sbox[(w >> 16) & 0xFF],
              H.sbox[w >> 24]);
}

// InvMixColumns of one column word (FIPS-197 §5.3.3), for the equivalent
// inverse cipher's schedule.
uint32_t inv_mix_word(uint32_t w) {
  const uint8_t a0 = w & 0xFF, a1 = (w >> 8) & 0xFF, a2 = (w >> 16) & 0xFF, a3 = w >> 24;
  auto m = [](uint8_t a, uint8_t b) { return gf_mul(a, b); };
  return pack(m(a0, 14) ^ m(a1, 11) ^ m(a2, 13) ^ m(a3, 9),
              m(a0, 9) ^ m(a1, 14) ^ m(a2, 11) ^ m(a3, 13),
              m(a0, 13) ^ m(a1, 9) ^ m(a2, 14) ^ m(a3, 11),
              m(a0, 11) ^ m(a1, 13) ^ m(a2, 9) ^ m(a3, 14));
}

aes_status check_schedule(const aes_key_schedule* ks) {
  if (ks == nullptr) return AES_ERR_ARG;
  const bool ok = (ks->key_bits == 128 && ks->nr == 10) || (ks->key_bits == 192 && ks->nr == 12) ||
                  (ks->key_bits == 256 && ks->nr == 14);
  return ok ? AES_OK : AES_ERR_KEYSIZE;
}

// Whether the current device reads and writes pageable host memory
// coherently through the host's page tables (cudaDevAttrPageableMemoryAccess,
// as on Grace-Blackwell over NVLink-C2C), looked up once per device ordinal.
bool pageable_access() {
  static std::atomic<int> cache[64];  // 0 unknown, 1 no, 2 yes
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (dev >= 0 && dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c != 0) return c == 2;
  }
  int v = 0;
  const bool yes = cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, dev) == cudaSuccess && v == 1;
  if (dev >= 0 && dev < 64) cache[dev].store(yes ? 2 : 1, std::memory_order_relaxed);
  return yes;
}

// Resolve a caller pointer to one the current device can dereference.
// Pageable host memory only with `pageable_ok` (the library's own file
// mappings) on a device that reaches it through the host's page tables.
aes_status device_view(const void* p, const void** dev, bool pageable_ok) {
  cudaPointerAttributes attr{};
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) return cuda_failure(e);
  int cur = 0;
  e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return cuda_failure(e);
  switch (attr.type) {
    case cudaMemoryTypeDevice:
      if (attr.device != cur) return AES_ERR_ARG;  // another GPU's memory
      *dev = p;
      return AES_OK;
    case cudaMemoryTypeManaged:
      *dev = p;
      return AES_OK;
    case cudaMemoryTypeHost:  // pinned host memory, mapped into the device's address space
      if (attr.devicePointer == nullptr) return AES_ERR_ARG;
      *dev = attr.devicePointer;
      return AES_OK;
    default:  // pageable host memory: not accepted from callers
      if (pageable_ok && attr.type == cudaMemoryTypeUnregistered && pageable_access()) {
        *dev = p;
        return AES_OK;
      }
      return AES_ERR_ARG;
  }
}

aes_status check_buffers(const void* in, void* out, size_t nbytes, const void** din, void** dout,
                         bool pageable_ok = false) {
  if (in == nullptr || out == nullptr) return AES_ERR_ARG;
  const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
  if ((a | b) & 15u) return AES_ERR_ALIGN;
  if (a != b && a < b + nbytes && b < a + nbytes) return AES_ERR_OVERLAP;
  aes_status s = device_view(in, din, pageable_ok);
  if (s != AES_OK) return s;
  const void* o = nullptr;
  s = device_view(out, &o, pageable_ok);
  if (s != AES_OK) return s;
  *dout = const_cast<void*>(o);
  return AES_OK;
}

// SM count of the current device, looked up once per device ordinal.
int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < 64 && (n = cache[dev].load(std::memory_order_relaxed)) > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
  if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Default launch shapes (measured on GB300; see the bench's autotune output).
struct Defaults {
  int cta_threads, blocks_per_thread;
};
// blocks_per_thread 0 selects the run-cached CTR kernel (two cached rounds).
Defaults default_shape(Op op, int nr) {
  switch (op) {
    case Op::kCtr: return {1024, 0};
    case Op::kEcbEncrypt:
    case Op::kEcbDecrypt: return {1024, nr == 10 ? 4 : 1};
  }
  return {1024, 1};
}

aes_status resolve_shape(Op op, int nr, uint64_t nblocks, const aes_launch_config* cfg,
                         LaunchShape* shape) {
  const Defaults d = default_shape(op, nr);
  int variant = cfg ? cfg->variant : AES_VARIANT_AUTO;
  if (variant == AES_VARIANT_BITSLICE) {
    // fixed CTA shape (16 blocks per thread); grid 0 = as many CTAs as fit per SM
    const int grid = cfg ? cfg->grid_ctas : 0;
    if (grid < 0) return AES_ERR_ARG;
    *shape = LaunchShape{kBitsliceThreads, 16, grid};
    return AES_OK;
  }
  if (variant == AES_VARIANT_TTABLE_BULK) {
    // CTR only, the run-cached layout (blocks_per_thread 0); any CTA size
    if (op != Op::kCtr || (cfg && cfg->blocks_per_thread != 0)) return AES_ERR_ARG;
    const int cta = (cfg && cfg->cta_threads) ? cfg->cta_threads : 1024;
    const int grid = (cfg && cfg->grid_ctas) ? cfg->grid_ctas : sm_count();
    if (cta < 128 || cta > 1024 || cta % 32 != 0 || grid < 0) return AES_ERR_ARG;
    *shape = LaunchShape{cta, 0, grid};
    return AES_OK;
  }
  if (variant != AES_VARIANT_AUTO && variant != AES_VARIANT_TTABLE) return AES_ERR_ARG;
  int cta = (cfg && cfg->cta_threads) ? cfg->cta_threads : d.cta_threads;
  int bpt = (cfg && cfg->blocks_per_thread) ? cfg->blocks_per_thread : d.blocks_per_thread;
  if (cta < 128 || cta > 1024 || cta % 32 != 0) return AES_ERR_ARG;
  if (bpt != 1 && bpt != 2 && bpt != 4 && !(bpt == 0 && op == Op::kCtr)) return AES_ERR_ARG;
  int grid = (cfg && cfg->grid_ctas) ? cfg->grid_ctas : sm_count();
  if (grid < 0) return AES_ERR_ARG;
  if (bpt == 0) {  // the cached CTR kernel sizes its own grid from the runs
    *shape = LaunchShape{cta, 0, grid};
    return AES_OK;
  }
  // No more CTAs than there is work for (at least one, for a tail-only call).
  const uint64_t per_cta = static_cast<uint64_t>(cta) * bpt;
  const uint64_t needed = nblocks == 0 ? 1 : (nblocks + per_cta - 1) / per_cta;
  if (static_cast<uint64_t>(grid) > needed) grid = static_cast<int>(needed);
  *shape = LaunchShape{cta, bpt, grid};
  return AES_OK;
}

void copy_round_keys(const uint32_t* src, int nr, RoundKeys* rk) {
  std::memset(rk, 0, sizeof(*rk));
  std::memcpy(rk->w, src, sizeof(uint32_t) * 4 * (nr + 1));
}

// Host-side T-table word: Ti[x] = te0[x] rotated left by 8i.
uint32_t te(int i, uint32_t x) { return i == 0 ? H.te0[x] : rotl32(H.te0[x], 8 * i); }

// CTR launch constants (see CtrParams): columns 0..2 of the state after the
// initial AddRoundKey do not depend on the counter, so their contributions to
// each round-1 column are summed here once.
CtrParams make_ctr_params(const aes_key_schedule* ks, const uint8_t iv[16]) {
  CtrParams cp{};
  for (int c = 0; c < 4; ++c) cp.iv_w[c] = load_le32(iv + 4 * c);
  cp.ctr0 = ((uint32_t)iv[12] << 24) | ((uint32_t)iv[13] << 16) | ((uint32_t)iv[14] << 8) | iv[15];
  const uint32_t* rk = ks->rk_enc;
  uint32_t s[3];
  for (int c = 0; c < 3; ++c) s[c] = cp.iv_w[c] ^ rk[c];
  cp.rk0w3 = rk[3];
  for (int j = 0; j < 4; ++j) {
    uint32_t acc = rk[4 + j];
    for (int i = 0; i < 4; ++i) {
      const int col = (j + i) & 3;  // ShiftRows: row i of output column j comes from column j+i
      if (col == 3) continue;       // the counter column, looked up on the device
      acc ^= te(i, (s[col] >> (8 * i)) & 0xFF);
    }
    cp.c1[j] = acc;
  }
  return cp;
}

aes_status run(Op op, const aes_key_schedule* ks, const uint8_t* iv, const void* in, void* out,
               size_t nbytes, void* stream, const aes_launch_config* cfg, bool pageable_ok = false) {
  aes_status s = check_schedule(ks);
  if (s != AES_OK) return s;
  if (op == Op::kCtr && iv == nullptr) return AES_ERR_ARG;
  if (op != Op::kCtr && nbytes % 16 != 0) return AES_ERR_LENGTH;
  if (cfg && cfg->variant != AES_VARIANT_AUTO && cfg->variant != AES_VARIANT_TTABLE &&
      cfg->variant != AES_VARIANT_BITSLICE && cfg->variant != AES_VARIANT_TTABLE_BULK)
    return AES_ERR_ARG;
  if (nbytes == 0) return AES_OK;
  const void* din = nullptr;
  void* dout = nullptr;
  s = check_buffers(in, out, nbytes, &din, &dout, pageable_ok);
  if (s != AES_OK) return s;
  const uint64_t nblocks = nbytes / 16;
  const uint32_t tail = static_cast<uint32_t>(nbytes % 16);
  LaunchShape shape{};
  s = resolve_shape(op, static_cast<int>(ks->nr), nblocks, cfg, &shape);
  if (s != AES_OK) return s;
  const bool bitslice = cfg && cfg->variant == AES_VARIANT_BITSLICE;
  RoundKeys rk;
  copy_round_keys(op == Op::kEcbDecrypt && !bitslice ? ks->rk_dec : ks->rk_enc,
                  static_cast<int>(ks->nr), &rk);
  CtrParams cp{};
  if (op == Op::kCtr) cp = make_ctr_params(ks, iv);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nr = static_cast<int>(ks->nr);
  cudaError_t e = cudaSuccess;
  if (bitslice) {
    e = launch_bitslice(op, nr, din, dout, nblocks, tail, rk, cp, shape, st);
    if (e != cudaSuccess) return cuda_failure(e);
    return AES_OK;
  }
  if (cfg && cfg->variant == AES_VARIANT_TTABLE_BULK) {
    e = launch_ttable_ctr_bulk(nr, din, dout, nblocks, tail, rk, cp, shape, st);
    return e == cudaSuccess ? AES_OK : cuda_failure(e);
  }
  switch (op) {
    case Op::kEcbEncrypt: e = launch_ttable_enc(nr, din, dout, nblocks, 0, rk, cp, shape, st); break;
    case Op::kEcbDecrypt: e = launch_ttable_dec(nr, din, dout, nblocks, 0, rk, cp, shape, st); break;
    case Op::kCtr: e = launch_ttable_ctr(nr, din, dout, nblocks, tail, rk, cp, shape, st); break;
  }
  if (e != cudaSuccess) return cuda_failure(e);
  return AES_OK;
}

// CBC decryption and XTS: validation shared with the other single-buffer calls.
aes_status run_cbc_decrypt(const aes_key_schedule* ks, const uint8_t* iv, const void* in, void* out,
                           size_t nbytes, void* stream) {
  aes_status s = check_schedule(ks);
  if (s != AES_OK) return s;
  if (iv == nullptr) return AES_ERR_ARG;
  if (nbytes % 16 != 0) return AES_ERR_LENGTH;
  if (nbytes == 0) return AES_OK;
  if (in == out && in != nullptr) return AES_ERR_OVERLAP;  // a predecessor must still be ciphertext
  const void* din = nullptr;
  void* dout = nullptr;
  s = check_buffers(in, out, nbytes, &din, &dout);
  if (s != AES_OK) return s;
  RoundKeys rk;
  copy_round_keys(ks->rk_dec, static_cast<int>(ks->nr), &rk);
  CtrParams cp{};
  for (int c = 0; c < 4; ++c) cp.iv_w[c] = load_le32(iv + 4 * c);
  const LaunchShape shape{1024, 1, sm_count()};
  const cudaError_t e = launch_cbc_decrypt(static_cast<int>(ks->nr), din, dout, nbytes / 16, rk, cp, shape,
                                           static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? AES_OK : cuda_failure(e);
}

aes_status run_xts(bool decrypt, const aes_key_schedule* data_ks, const aes_key_schedule* tweak_ks,
                   uint64_t first_sector, size_t sector_bytes, const void* in, void* out, size_t nbytes,
                   void* stream) {
  aes_status s = check_schedule(data_ks);
  if (s != AES_OK) return s;
  s = check_schedule(tweak_ks);
  if (s != AES_OK) return s;
  // IEEE 1619 / SP 800-38E define XTS-AES-128 and XTS-AES-256 only: two
  // 128-bit or two 256-bit halves of the XTS key.
  if (data_ks->key_bits != tweak_ks->key_bits || data_ks->key_bits == 192) return AES_ERR_KEYSIZE;
  if (sector_bytes == 0 || sector_bytes % 512 != 0 || sector_bytes / 16 > 0xFFFFFFFFull ||
      nbytes % sector_bytes != 0)
    return AES_ERR_LENGTH;
  if (nbytes == 0) return AES_OK;
  const void* din = nullptr;
  void* dout = nullptr;
  s = check_buffers(in, out, nbytes, &din, &dout);
  if (s != AES_OK) return s;
  RoundKeys rk1, rk2;
  copy_round_keys(decrypt ? data_ks->rk_dec : data_ks->rk_enc, static_cast<int>(data_ks->nr), &rk1);
  copy_round_keys(tweak_ks->rk_enc, static_cast<int>(tweak_ks->nr), &rk2);
  const LaunchShape shape{1024, 1, sm_count()};
  const cudaError_t e = launch_xts_mode(decrypt, static_cast<int>(data_ks->nr), static_cast<int>(tweak_ks->nr),
                                        din, dout, nbytes / 16, rk1, rk2, first_sector,
                                        static_cast<uint32_t>(sector_bytes / 16), shape,
                                        static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? AES_OK : cuda_failure(e);
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

aes_status batch_submit(const aes_batch* b, void* ws, size_t ws_bytes, void* stream,
                        const aes_batch_config* cfg) {
  if (b == nullptr) return AES_ERR_ARG;
  if (b->op > AES_BATCH_ECB_PKCS7_DECRYPT) return AES_ERR_ARG;
  if (b->flags & ~(AES_BATCH_IN_PADDED | AES_BATCH_OUT_PADDED)) return AES_ERR_ARG;
  if (b->n_msgs == 0) return AES_OK;
  if (!b->in || !b->out || !b->in_off || !b->in_len || !b->out_off) return AES_ERR_ARG;
  const bool raw_keys = b->keys != nullptr;
  if (raw_keys ? b->key_bits == nullptr
               : (b->schedules == nullptr || b->sched_idx == nullptr || b->n_schedules == 0))
    return AES_ERR_ARG;
  if (b->op == AES_BATCH_CTR && b->iv == nullptr) return AES_ERR_ARG;
  if (ws == nullptr) return AES_ERR_ARG;
  if (!aligned(b->in, 16) || !aligned(b->out, 16) || !aligned(ws, 256)) return AES_ERR_ALIGN;
  if (raw_keys && !aligned(b->keys, 16)) return AES_ERR_ALIGN;
  if (!raw_keys && !aligned(b->schedules, 4)) return AES_ERR_ALIGN;
  if (b->iv && !aligned(b->iv, 16)) return AES_ERR_ALIGN;
  if (ws_bytes < batch_workspace_bytes(b->n_msgs)) return AES_ERR_NOMEM;
  int cta = (cfg && cfg->cta_threads) ? cfg->cta_threads : 1024;
  int tile = (cfg && cfg->tile_blocks) ? cfg->tile_blocks : 0;  // 0: sized by the kernel
  int grid = (cfg && cfg->grid_ctas) ? cfg->grid_ctas : sm_count();
  const int short_path = cfg ? cfg->short_path : AES_BATCH_SHORT_AUTO;
  if (cta < 256 || cta > 1024 || cta % 32) return AES_ERR_ARG;
  if (tile != 0 && (tile < cta || tile > (1 << 20) || tile % cta)) return AES_ERR_ARG;
  if (grid < 1) return AES_ERR_ARG;
  if (short_path < AES_BATCH_SHORT_AUTO || short_path > AES_BATCH_SHORT_LANES) return AES_ERR_ARG;
  if (short_path == AES_BATCH_SHORT_LANES && b->op != AES_BATCH_CTR) return AES_ERR_ARG;
  // The lane path needs enough short messages to keep every warp busy for
  // several chunks: on packet-sized CTR batches it ran slower than the
  // per-warp groups at 131,072 messages and faster from 262,144 on.
  constexpr uint32_t kLaneAutoMsgs = 1u << 18;
  const bool lanes = short_path == AES_BATCH_SHORT_LANES ||
                     (short_path == AES_BATCH_SHORT_AUTO && b->op == AES_BATCH_CTR && b->n_msgs >= kLaneAutoMsgs);
  const void* din = nullptr;
  void* dout = nullptr;
  aes_status st = device_view(b->in, &din, false);
  if (st != AES_OK) return st;
  const void* o = nullptr;
  st = device_view(b->out, &o, false);
  if (st != AES_OK) return st;
  dout = const_cast<void*>(o);
  BatchArgs a{};
  a.n = b->n_msgs;
  a.op = b->op;
  a.in = static_cast<const uint8_t*>(din);
  a.out = static_cast<uint8_t*>(dout);
  a.in_off = b->in_off;
  a.in_len = b->in_len;
  a.out_off = b->out_off;
  a.keys = b->keys;
  a.key_bits = b->key_bits;
  a.schedules = raw_keys ? nullptr : b->schedules;
  a.sched_idx = raw_keys ? nullptr : b->sched_idx;
  a.n_sched = raw_keys ? 0 : b->n_schedules;
  a.tile_blocks = static_cast<uint32_t>(tile);
  a.flags = b->flags;
  a.iv = b->iv;
  a.out_len = b->out_len;
  a.status = b->status;
  batch_bind_workspace(&a, ws, lanes);
  const cudaError_t e = launch_batch(a, cta, grid, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_failure(e);
  return AES_OK;
}

}  // namespace

// Records a CUDA failure for aes_last_cuda_error() from other translation units.
aes_status record_cuda_failure(cudaError_t e) { return cuda_failure(e); }

// For aes_file_crypt's direct path: whether the current device can run the
// cipher on mapped files, and the single-buffer cipher (mode as
// aes_file_mode) on host memory the library mapped itself.
bool host_pageable_access() { return pageable_access(); }

aes_status crypt_mapped(int mode, const aes_key_schedule* ks, const uint8_t* iv, const void* in, void* out,
                        size_t nbytes, cudaStream_t stream) {
  const Op op = mode == AES_FILE_CTR ? Op::kCtr : mode == AES_FILE_ECB_ENCRYPT ? Op::kEcbEncrypt : Op::kEcbDecrypt;
  return run(op, ks, iv, in, out, nbytes, stream, nullptr, true);
}

}  // namespace aesgpu

using namespace aesgpu;

extern "C" {

aes_status aes_expand_key(const uint8_t* key, int key_bits, aes_key_schedule* ks) {
  if (key == nullptr || ks == nullptr) return AES_ERR_ARG;
  int nk = 0;
  switch (key_bits) {
    case 128: nk = 4; break;
    case 192: nk = 6; break;
    case 256: nk = 8; break;
    default: return AES_ERR_KEYSIZE;
  }
  std::memset(ks, 0, sizeof(*ks));
  const int nr = nk + 6, nwords = 4 * (nr + 1);
  ks->key_bits = static_cast<uint32_t>(key_bits);
  ks->nr = static_cast<uint32_t>(nr);
  uint32_t* w = ks->rk_enc;
  for (int i = 0; i < nk; ++i) w[i] = load_le32(key + 4 * i);
  uint8_t rcon = 1;
  for (int i = nk; i < nwords; ++i) {
    uint32_t t = w[i - 1];
    if (i % nk == 0) {
      t = sub_word((t >> 8) | (t << 24)) ^ rcon;  // RotWord on a little-endian word
      rcon = gf_xtime(rcon);
    } else if (nk == 8 && i % nk == 4) {
      t = sub_word(t);
    }
    w[i] = w[i - nk] ^ t;
  }
  // Equivalent inverse cipher (FIPS-197 §5.3.5): reversed rounds, InvMixColumns
  // on the middle ones.
  for (int r = 0; r <= nr; ++r)
    for (int c = 0; c < 4; ++c) {
      const uint32_t v = w[4 * (nr - r) + c];
      ks->rk_dec[4 * r + c] = (r == 0 || r == nr) ? v : inv_mix_word(v);
    }
  return AES_OK;
}

// SP 800-38A §6.5: counter block T_{first_block} of a buffer whose block 0
// uses `iv`; only the 32-bit big-endian counter in bytes 12..15 moves.
aes_status aes_ctr_iv_advance(const uint8_t iv[16], uint64_t first_block, uint8_t out_iv[16]) {
  if (iv == nullptr || out_iv == nullptr) return AES_ERR_ARG;
  uint8_t v[16];
  std::memcpy(v, iv, 16);  // iv and out_iv may be the same array
  const uint32_t c0 = ((uint32_t)v[12] << 24) | ((uint32_t)v[13] << 16) | ((uint32_t)v[14] << 8) | v[15];
  const uint32_t c = c0 + static_cast<uint32_t>(first_block);  // modulo 2^32, no carry into the nonce
  v[12] = static_cast<uint8_t>(c >> 24);
  v[13] = static_cast<uint8_t>(c >> 16);
  v[14] = static_cast<uint8_t>(c >> 8);
  v[15] = static_cast<uint8_t>(c);
  std::memcpy(out_iv, v, 16);
  return AES_OK;
}

aes_status aes_ecb_encrypt_ex(const aes_key_schedule* ks, const void* d_in, void* d_out,
                              size_t nbytes, void* stream, const aes_launch_config* cfg) {
  return run(Op::kEcbEncrypt, ks, nullptr, d_in, d_out, nbytes, stream, cfg);
}

aes_status aes_ecb_decrypt_ex(const aes_key_schedule* ks, const void* d_in, void* d_out,
                              size_t nbytes, void* stream, const aes_launch_config* cfg) {
  return run(Op::kEcbDecrypt, ks, nullptr, d_in, d_out, nbytes, stream, cfg);
}

aes_status aes_ctr_xcrypt_ex(const aes_key_schedule* ks, const uint8_t iv[16], const void* d_in,
                             void* d_out, size_t nbytes, void* stream,
                             const aes_launch_config* cfg) {
  return run(Op::kCtr, ks, iv, d_in, d_out, nbytes, stream, cfg);
}

aes_status aes_ecb_encrypt(const aes_key_schedule* ks, const void* d_in, void* d_out,
                           size_t nbytes, void* stream) {
  return aes_ecb_encrypt_ex(ks, d_in, d_out, nbytes, stream, nullptr);
}

aes_status aes_ecb_decrypt(const aes_key_schedule* ks, const void* d_in, void* d_out,
                           size_t nbytes, void* stream) {
  return aes_ecb_decrypt_ex(ks, d_in, d_out, nbytes, stream, nullptr);
}

aes_status aes_ctr_xcrypt(const aes_key_schedule* ks, const uint8_t iv[16], const void* d_in,
                          void* d_out, size_t nbytes, void* stream) {
  return aes_ctr_xcrypt_ex(ks, iv, d_in, d_out, nbytes, stream, nullptr);
}

aes_status aes_cbc_decrypt(const aes_key_schedule* ks, const uint8_t iv[16], const void* d_in, void* d_out,
                           size_t nbytes, void* stream) {
  return run_cbc_decrypt(ks, iv, d_in, d_out, nbytes, stream);
}

aes_status aes_xts_encrypt(const aes_key_schedule* data_ks, const aes_key_schedule* tweak_ks,
                           uint64_t first_sector, size_t sector_bytes, const void* d_in, void* d_out,
                           size_t nbytes, void* stream) {
  return run_xts(false, data_ks, tweak_ks, first_sector, sector_bytes, d_in, d_out, nbytes, stream);
}

aes_status aes_xts_decrypt(const aes_key_schedule* data_ks, const aes_key_schedule* tweak_ks,
                           uint64_t first_sector, size_t sector_bytes, const void* d_in, void* d_out,
                           size_t nbytes, void* stream) {
  return run_xts(true, data_ks, tweak_ks, first_sector, sector_bytes, d_in, d_out, nbytes, stream);
}

size_t aes_batch_workspace_size(uint32_t n_msgs) { return batch_workspace_bytes(n_msgs); }

aes_status aes_batch_submit_ex(const aes_batch* b, void* d_workspace, size_t workspace_bytes,
                               void* stream, const aes_batch_config* cfg) {
  return batch_submit(b, d_workspace, workspace_bytes, stream, cfg);
}

aes_status aes_batch_submit(const aes_batch* b, void* d_workspace, size_t workspace_bytes,
                            void* stream) {
  return batch_submit(b, d_workspace, workspace_bytes, stream, nullptr);
}

aes_status aes_take_wait_timeouts(uint32_t* count) {
  if (count == nullptr) return AES_ERR_ARG;
  unsigned int v = 0, w = 0;
  cudaError_t e = take_bulk_timeouts(&v);
  if (e != cudaSuccess) return cuda_failure(e);
  e = take_lane_timeouts(&w);
  if (e != cudaSuccess) return cuda_failure(e);
  *count = v + w;
  return v + w ? AES_ERR_TIMEOUT : AES_OK;
}

int aes_last_cuda_error(void) { return g_last_cuda_error; }

const char* aes_status_string(aes_status s) {
  switch (s) {
    case AES_OK: return "ok";
    case AES_ERR_ARG: return "invalid argument";
    case AES_ERR_KEYSIZE: return "key size must be 128, 192 or 256 bits";
    case AES_ERR_LENGTH: return "length must be a multiple of 16 bytes";
    case AES_ERR_ALIGN: return "data pointers must be 16-byte aligned";
    case AES_ERR_OVERLAP: return "input and output overlap";
    case AES_ERR_PADDING: return "malformed PKCS#7 padding";
    case AES_ERR_NOMEM: return "workspace too small";
    case AES_ERR_CUDA: return "CUDA error";
    case AES_ERR_TIMEOUT: return "device wait timed out";
    case AES_ERR_BUSY: return "busy";
    case AES_ERR_IO: return "file open, read or write failed";
  }
  return "unknown status";
}

}  // extern "C"
