/*
 * aesgpu.h — C ABI of the GB300 bulk-AES library (libaesgpu.so).
 *
 * The operation is the one the paper parallelises across CPU cores (§IV,
 * Figs. 2-3): encrypt or decrypt a large buffer whose 16-byte blocks are
 * independent, with the AES steps of its Fig. 1 (§III.A) — key expansion, an
 * initial AddRoundKey, Nr-1 full rounds, a final round without MixColumns —
 * whose arithmetic is FIPS-197.  The paper names no mode; the library offers
 * the two block-independent ones of NIST SP 800-38A, ECB (§6.1) and CTR
 * (§6.5), and PKCS#7 padding for the batched ECB path.
 *
 * General rules for every call below:
 *  - Data pointers marked "device" must be readable (and, for outputs,
 *    writable) by the current CUDA device: cudaMalloc memory, managed memory,
 *    or mapped pinned host memory.  The caller owns every buffer; the library
 *    never frees or retains caller pointers after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  GPU work is enqueued on it and the call returns without
 *    waiting; results are valid once the stream reaches that point.  The
 *    calls allocate nothing and synchronise nothing, so they may be captured
 *    into a CUDA graph.
 *  - Arguments are validated on the host before anything is enqueued; a
 *    failed check returns its status and enqueues nothing.  A launch failure
 *    returns AES_ERR_CUDA; aes_last_cuda_error() then gives the CUDA code.
 *    No exception or abort crosses this interface.
 *  - Key material is never logged or copied anywhere but the kernel
 *    parameters of the launches it feeds.
 */
#ifndef AESGPU_H
#define AESGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum aes_status {
    AES_OK = 0,
    AES_ERR_ARG = 1,      /* null pointer, unknown enum value, bad struct */
    AES_ERR_KEYSIZE = 2,  /* key_bits not in {128, 192, 256} */
    AES_ERR_LENGTH = 3,   /* ECB length not a multiple of 16 */
    AES_ERR_ALIGN = 4,    /* a data pointer not 16-byte aligned */
    AES_ERR_OVERLAP = 5,  /* input and output overlap without being equal */
    AES_ERR_PADDING = 6,  /* PKCS#7 padding malformed (per-message status) */
    AES_ERR_NOMEM = 7,    /* workspace too small */
    AES_ERR_CUDA = 8,     /* a CUDA call failed; see aes_last_cuda_error() */
    AES_ERR_TIMEOUT = 9,  /* a bounded device wait gave up */
    AES_ERR_BUSY = 10,    /* resource in use */
    AES_ERR_IO = 11       /* a file could not be opened, read or written (aes_file_crypt) */
} aes_status;

/* Expanded key (FIPS-197 §5.2, paper Fig. 1 step 1).  Plain data, owned by
 * the caller, safe to copy.  Word i holds bytes 4i..4i+3 of the expanded key
 * in little-endian order (byte 4i in bits 0..7).  rk_enc has 4*(nr+1) words
 * of the cipher's schedule; rk_dec has the schedule of the equivalent inverse
 * cipher (FIPS-197 §5.3.5): rk_enc's round keys in reverse round order, with
 * InvMixColumns applied to rounds 1..nr-1. */
typedef struct aes_key_schedule {
    uint32_t key_bits; /* 128, 192 or 256 */
    uint32_t nr;       /* 10, 12 or 14 */
    uint32_t rk_enc[60];
    uint32_t rk_dec[60];
} aes_key_schedule;

/* Round implementation of the single-buffer kernels. */
typedef enum aes_variant {
    AES_VARIANT_AUTO = 0,     /* the library's measured choice per call */
    AES_VARIANT_TTABLE = 1,   /* shared-memory T-tables, replicated per bank */
    AES_VARIANT_BITSLICE = 2, /* bitsliced S-box / MixColumns on LOP3 */
    AES_VARIANT_TTABLE_BULK = 3 /* CTR only: the run-cached T-table kernel with each half run of
                                   input (2 KiB) staged into shared memory by a TMA bulk copy that
                                   overlaps the rounds; kept as the measured alternative to the
                                   default's plain 128-bit loads (other modes: AES_ERR_ARG) */
} aes_variant;

/* Optional launch shape for the _ex calls; a zero field means "choose". */
typedef struct aes_launch_config {
    int32_t variant;           /* aes_variant */
    int32_t cta_threads;       /* threads per CTA: 128..1024, multiple of 32 */
    int32_t blocks_per_thread; /* 16-byte blocks per thread per iteration: 1, 2 or 4; 0 = the
                                  library choice (for CTR: the run-cached kernel, which walks
                                  256 consecutive counters per warp and caches two rounds) */
    int32_t grid_ctas;         /* CTAs in the grid; 0 = one per SM */
} aes_launch_config;

/* Key expansion on the host (FIPS-197 §5.2; paper Fig. 1 step 1).
 * key: host, key_bits/8 bytes.  ks: host output.  Synchronous, touches no
 * GPU.  Returns AES_ERR_ARG for null pointers, AES_ERR_KEYSIZE for a bad size. */
aes_status aes_expand_key(const uint8_t *key, int key_bits, aes_key_schedule *ks);

/* ECB encryption (SP 800-38A §6.1) of nbytes bytes: block j of d_out is the
 * Cipher (paper Fig. 1; FIPS-197 §5.1) of block j of d_in.
 * ks: host.  d_in, d_out: device, 16-byte aligned; d_in == d_out is allowed
 * (in place), any other overlap returns AES_ERR_OVERLAP.  nbytes must be a
 * multiple of 16 (AES_ERR_LENGTH); 0 is a no-op. */
aes_status aes_ecb_encrypt(const aes_key_schedule *ks, const void *d_in, void *d_out,
                           size_t nbytes, void *stream);

/* ECB decryption: the inverse cipher (FIPS-197 §5.3) of every block.  Same
 * arguments and rules as aes_ecb_encrypt. */
aes_status aes_ecb_decrypt(const aes_key_schedule *ks, const void *d_in, void *d_out,
                           size_t nbytes, void *stream);

/* CTR (SP 800-38A §6.5), encryption and decryption alike: byte k of d_out is
 * byte k of d_in XOR byte k mod 16 of Cipher(T_{k/16}), where T_j is iv[0..11]
 * followed by (c0 + j) mod 2^32 in big-endian, c0 being iv[12..15] read
 * big-endian.  The counter wraps without carrying into the nonce.
 * iv: host, 16 bytes.  Any nbytes; a partial last block uses the leading
 * keystream bytes.  Pointer rules as aes_ecb_encrypt. */
aes_status aes_ctr_xcrypt(const aes_key_schedule *ks, const uint8_t iv[16], const void *d_in,
                          void *d_out, size_t nbytes, void *stream);

/* The IV of a CTR range that starts `first_block` 16-byte blocks into a
 * buffer (SP 800-38A §6.5, the counter blocks T_j): out_iv[0..11] = iv[0..11]
 * and out_iv[12..15] = BE32((c0 + first_block) mod 2^32), c0 being
 * iv[12..15] read big-endian; the counter wraps without carrying into the
 * nonce, as in aes_ctr_xcrypt.  aes_ctr_xcrypt(out_iv, ...) on the bytes from
 * 16 * first_block on therefore equals the same bytes of one call with `iv`
 * on the whole buffer: the paper's chunk split (§IV.B) of a CTR buffer across
 * calls, streams or GPUs.  iv, out_iv: host, 16 bytes each (may be the same
 * array).  Synchronous, touches no GPU.  AES_ERR_ARG for a null pointer. */
aes_status aes_ctr_iv_advance(const uint8_t iv[16], uint64_t first_block, uint8_t out_iv[16]);

/* The same three calls with an explicit launch shape (cfg may be NULL, which
 * equals the plain call).  Every shape computes identical bytes. */
aes_status aes_ecb_encrypt_ex(const aes_key_schedule *ks, const void *d_in, void *d_out,
                              size_t nbytes, void *stream, const aes_launch_config *cfg);
aes_status aes_ecb_decrypt_ex(const aes_key_schedule *ks, const void *d_in, void *d_out,
                              size_t nbytes, void *stream, const aes_launch_config *cfg);
aes_status aes_ctr_xcrypt_ex(const aes_key_schedule *ks, const uint8_t iv[16], const void *d_in,
                             void *d_out, size_t nbytes, void *stream,
                             const aes_launch_config *cfg);

/* ---- Two more block-parallel modes -------------------------------------
 * Not in the paper (it names no mode); they reuse the same round kernels. */

/* CBC decryption (SP 800-38A §6.2): block j of d_out is InvCipher(C_j) XOR
 * C_{j-1}, C_{-1} = iv (host, 16 bytes).  CBC encryption is sequential and
 * is not offered.  nbytes a multiple of 16 (AES_ERR_LENGTH).  d_in == d_out is
 * refused (AES_ERR_OVERLAP): each block's predecessor must still be
 * ciphertext when it is read.  Other pointer rules as aes_ecb_encrypt. */
aes_status aes_cbc_decrypt(const aes_key_schedule *ks, const uint8_t iv[16], const void *d_in,
                           void *d_out, size_t nbytes, void *stream);

/* XTS-AES (IEEE 1619 / SP 800-38E) over data units of sector_bytes bytes,
 * for the two key sizes those standards define: data_ks and tweak_ks both
 * AES-128 or both AES-256 (any other pair, 192-bit keys included, returns
 * AES_ERR_KEYSIZE),
 * without ciphertext stealing: sector_bytes a positive multiple of 512 and
 * nbytes a multiple of sector_bytes (AES_ERR_LENGTH).  Unit u (counted from
 * the start of d_in) uses the tweak value first_sector + u as a 128-bit
 * little-endian integer: T = Cipher_tweak_ks(value), block j of the unit is
 * Cipher_data_ks(P ^ T a^j) ^ T a^j with a the generator of GF(2^128) mod
 * x^128 + x^7 + x^2 + x + 1 (decryption: the inverse cipher in the middle).
 * data_ks and tweak_ks are the schedules of the two halves of the XTS key.
 * In place is allowed.  Other pointer rules as aes_ecb_encrypt. */
aes_status aes_xts_encrypt(const aes_key_schedule *data_ks, const aes_key_schedule *tweak_ks,
                           uint64_t first_sector, size_t sector_bytes, const void *d_in,
                           void *d_out, size_t nbytes, void *stream);
aes_status aes_xts_decrypt(const aes_key_schedule *data_ks, const aes_key_schedule *tweak_ks,
                           uint64_t first_sector, size_t sector_bytes, const void *d_in,
                           void *d_out, size_t nbytes, void *stream);

/* ---- Batched messages (one persistent launch) --------------------------
 *
 * Many independent messages of uneven byte lengths, each with its own key
 * and IV, processed by one call: the paper's chunk-per-thread scheme (§IV.B)
 * with chunks = messages.  A device prefix sum over per-message block
 * counts maps 16-byte blocks to messages; a persistent kernel claims tiles
 * of blocks, expands each message's key on the device (FIPS-197 §5.2) and
 * runs the same rounds as the single-buffer calls.  One operation per call:
 *   AES_BATCH_CTR              CTR (SP 800-38A §6.5), any length; output
 *                              length = input length.
 *   AES_BATCH_ECB_PKCS7_ENCRYPT  PKCS#7-pad (1..16 bytes) then ECB;
 *                              output length = 16*floor(len/16) + 16.
 *   AES_BATCH_ECB_PKCS7_DECRYPT  ECB-decrypt (len a positive multiple of
 *                              16), check the padding; the whole padded
 *                              plaintext is written and out_len gives the
 *                              unpadded length.
 */
typedef enum aes_batch_op {
    AES_BATCH_CTR = 0,
    AES_BATCH_ECB_PKCS7_ENCRYPT = 1,
    AES_BATCH_ECB_PKCS7_DECRYPT = 2
} aes_batch_op;

/* Description of one batch.  The struct itself is read on the host during
 * the call; every array it points to is device memory, owned by the caller,
 * and must stay valid until the stream has executed the work. */
/* aes_batch.flags: promises that let the kernel treat a message's last,
 * ragged block as a whole 16-byte block (one vector load / store instead of
 * byte-exact ones).  Offsets are multiples of 16, so the bytes concerned lie
 * between a message's end and the next 16-byte boundary. */
#define AES_BATCH_IN_PADDED 1u  /* each input may be read up to the next 16-byte boundary */
#define AES_BATCH_OUT_PADDED 2u /* output bytes up to the next 16-byte boundary after each message's
                                   output may be overwritten (their values are unspecified) */

typedef struct aes_batch {
    uint32_t n_msgs;
    uint32_t op;                  /* aes_batch_op */
    const uint8_t *in;            /* input arena (device) */
    uint8_t *out;                 /* output arena (device); outputs must not overlap inputs
                                     of other messages or each other (in == out per message is
                                     allowed for CTR) */
    const uint64_t *in_off;       /* [n_msgs] byte offset of message m in `in`, multiple of 16 */
    const uint64_t *in_len;       /* [n_msgs] byte length of message m */
    const uint64_t *out_off;      /* [n_msgs] byte offset of m's output in `out`, multiple of 16 */
    /* Key source: raw keys expanded on the device, or pre-expanded schedules. */
    const uint8_t *keys;          /* [n_msgs][32] raw keys (first key_bits/8 bytes used), 16-B aligned, or NULL */
    const uint32_t *key_bits;     /* [n_msgs] 128, 192 or 256 (with keys) */
    const aes_key_schedule *schedules; /* [n_schedules] device table (when keys == NULL) */
    const uint32_t *sched_idx;    /* [n_msgs] index into schedules */
    uint32_t n_schedules;
    uint32_t flags;               /* 0 (every read and write exact to the byte), or
                                     AES_BATCH_IN_PADDED | AES_BATCH_OUT_PADDED */
    const uint8_t *iv;            /* [n_msgs][16] IVs, 16-B aligned (CTR only; else NULL) */
    uint64_t *out_len;            /* [n_msgs] out: output bytes per message (may be NULL) */
    int32_t *status;              /* [n_msgs] out: aes_status per message (may be NULL) */
} aes_batch;

/* aes_batch_config.short_path: how the messages of fewer than 512 blocks run. */
#define AES_BATCH_SHORT_AUTO 0   /* the library's measured choice: LANES for CTR batches of 262,144
                                    messages or more, GROUPS otherwise */
#define AES_BATCH_SHORT_GROUPS 1 /* every op: each warp of the persistent kernel takes groups of
                                    consecutive messages, their round keys in shared memory */
#define AES_BATCH_SHORT_LANES 2  /* CTR only: one lane per message of fewer than 128 blocks, its
                                    round keys in registers; those messages are first sorted by key
                                    size and length (one more launch), then a kernel of
                                    their own runs them after the persistent kernel, which keeps the
                                    longer short messages (other ops: AES_ERR_ARG).  Faster on large
                                    batches of packet-sized messages, slower on small batches: a lane
                                    walks its message's blocks one after another */

/* Optional launch shape of the persistent kernel; zero fields = default. */
typedef struct aes_batch_config {
    int32_t cta_threads;  /* 256..1024, multiple of 32; up to 512 selects the build with 128
                             registers per thread, which keeps a long message's round keys in
                             registers across a span */
    int32_t tile_blocks;  /* 16-byte blocks a CTA claims at a time: multiple of cta_threads, <= 2^20;
                             0 = sized from the batch: ~4 tiles per CTA of the long messages' blocks,
                             at most 65536 */
    int32_t grid_ctas;    /* 0 = one per SM (also the lane kernel's grid) */
    int32_t short_path;   /* AES_BATCH_SHORT_* */
} aes_batch_config;

/* Bytes of device workspace aes_batch_submit needs for n_msgs messages. */
size_t aes_batch_workspace_size(uint32_t n_msgs);

/* Enqueue one batch on `stream` (a memset of the work counters and 2 kernel
 * launches: count + scan, persistent cipher kernel; on the lane path of short
 * CTR messages also the scatter into bin order and the lane kernel; no
 * allocation, no host sync, so the call can be captured into a CUDA graph
 * and replayed).  d_workspace: device,
 * 256-byte aligned, at least aes_batch_workspace_size(n_msgs) bytes; its
 * contents need no initialisation.  Per-message failures (bad key size,
 * unaligned offset, bad ECB length or padding) are reported in status[m]
 * with zero output bytes; the rest of the batch proceeds.  Returns
 * AES_ERR_ARG for missing arrays, an unknown op or unknown flags, AES_ERR_NOMEM for a
 * short workspace, AES_ERR_ALIGN for a misaligned arena, key or IV base.
 * Messages are not checked against each other for overlap. */
aes_status aes_batch_submit(const aes_batch *b, void *d_workspace, size_t workspace_bytes,
                            void *stream);
aes_status aes_batch_submit_ex(const aes_batch *b, void *d_workspace, size_t workspace_bytes,
                               void *stream, const aes_batch_config *cfg);

/* aes_batch_submit without a workspace argument, for callers that cannot
 * allocate device memory at all: code that runs where cudaMalloc is not
 * allowed or not wanted (inside a host callback, on a latency-critical path
 * where cudaMalloc's implicit device synchronisation would stall other
 * streams, or inside a framework that owns every device allocation).  The
 * paper has no counterpart; this is a deployment convenience.
 *
 * The workspace is one file-scope device array of the library, sized for
 * AES_BATCH_NOALLOC_MAX_MSGS messages (about 909 KiB); every GPU that loads
 * libaesgpu.so holds it until the process exits.  The call allocates nothing
 * and calls no allocating routine; inputs and outputs are the caller's as in
 * aes_batch_submit, with the same rules and per-message status.
 *  - n_msgs above AES_BATCH_NOALLOC_MAX_MSGS returns AES_ERR_NOMEM and
 *    enqueues nothing.
 *  - The first call in a CUDA context looks up the array's device address
 *    there (cudaGetSymbolAddress, which may load the library's GPU code) and
 *    keeps it with that context's ID; a new context on the device (after
 *    cudaDeviceReset, say) gets a fresh lookup.  Make the first call in a
 *    context before any stream capture in it.
 *  - All calls on a device share the one array, and it keeps the last call's
 *    contents; the pipeline rewrites every part it reads (the first kernel
 *    resets the tile counter and rewrites the offsets) before use.  Two calls
 *    whose work overlaps on the GPU (different streams without ordering, or
 *    host threads racing) corrupt each other's results: order them on one
 *    stream or synchronise between them. */
#define AES_BATCH_NOALLOC_MAX_MSGS 65536u
aes_status aes_batch_submit_noalloc(const aes_batch *b, void *stream);

/* ------------------------------------------------------------------------
 * File in, encrypted file out: the paper's workload (§IV, Figs. 2-3: a large
 * file is split into as many chunks as parallel instances, the chunks are
 * encrypted in parallel and the results concatenated into the output file).
 *
 * Here the chunks are fixed-size pieces of the file handed to `threads`
 * worker threads, on one of two paths:
 *  - staged (the default): each worker owns one pinned
 *    host buffer and one CUDA stream and repeats: read its next chunk at the
 *    chunk's file offset, run the cipher on the pinned buffer in place (the
 *    kernel reads and writes host memory over the CPU-GPU link; no device
 *    copy), wait for that stream, copy the chunk to the same offset of dst
 *    (through a shared mapping of dst, or pwrite when dst cannot be mapped).
 *    The GPU only ever touches the library's own pinned buffers.
 *  - direct (opt-in with AES_FILE_DIRECT, taken when the current device reads
 *    and writes pageable host memory through the host's page tables,
 *    cudaDevAttrPageableMemoryAccess, as on Grace-Blackwell over NVLink-C2C;
 *    otherwise the staged path runs): both files are mapped and the kernel
 *    reads the source chunk and writes the destination chunk in place in
 *    the mappings, no host copy.  Each worker first faults in its chunk's
 *    pages of both mappings, so the device never meets a missing page:
 *    MADV_POPULATE_READ for src; for dst a store of 0 into each page's first
 *    byte inside the chunk (bytes the kernel then overwrites), or, in place,
 *    MADV_POPULATE_WRITE (one access per page on kernels without
 *    MADV_POPULATE_*).  It then launches the cipher on its own stream and
 *    takes the next chunk; each worker waits for its stream at the end.
 *    Hazard: if another process truncates src or dst while a chunk is in
 *    flight, the kernel touches a page that no longer exists, which faults
 *    the CUDA context (a host access would get SIGBUS).  Use this path only
 *    for files that nothing else changes during the call.
 * Reads, writes and GPU work of different chunks overlap.  On the staged
 * path a truncation by another process during the call reaches only host
 * code (SIGBUS on the shared mapping of dst), as with any mapped file.  CTR chunks use the IV whose 32-bit
 * counter is advanced by the chunk's first block (mod 2^32), so the output is
 * byte-identical to one call on the whole file; ECB needs a file length that
 * is a multiple of 16 (no padding here).
 *
 * src_path / dst_path: NUL-terminated paths.  dst is created (mode 0644) or
 * truncated to the source length; when dst names the same file as src the
 * file is encrypted in place (each chunk is read before it is rewritten).
 * ks: expanded key (the caller's, read during the call).  iv: 16 bytes,
 * CTR only (NULL otherwise).  cfg may be NULL (defaults).  stats may be NULL.
 * Runs on the calling thread's current CUDA device and returns when dst is
 * complete (or on the first failure: AES_ERR_IO with stats->os_errno set,
 * AES_ERR_CUDA, AES_ERR_LENGTH for a ragged ECB file, AES_ERR_ARG for a bad
 * argument; dst is then incomplete).  Pinned memory (staged path only):
 * threads buffers of chunk_bytes rounded up to whole MiB; the call returns
 * them to a process-wide pool (at most 64 buffers) that later calls reuse,
 * since pinning host memory costs about as much as a few GB of file traffic;
 * aes_file_trim() frees the pool. */
typedef enum aes_file_mode {
    AES_FILE_CTR = 0,
    AES_FILE_ECB_ENCRYPT = 1,
    AES_FILE_ECB_DECRYPT = 2
} aes_file_mode;

#define AES_FILE_STAGED 1u  /* the staged path (the default; the flag only makes it explicit) */
#define AES_FILE_DIRECT 2u  /* opt in to the direct path where the device allows it (else staged);
                               the caller promises that neither file changes length during the call */

typedef struct aes_file_config {
    uint64_t chunk_bytes;  /* bytes per chunk: a multiple of 16; 0 = 64 MiB direct, 4 MiB staged */
    int32_t threads;       /* worker threads, 1..64; 0 = min(16, hardware threads) */
    uint32_t flags;        /* 0, AES_FILE_STAGED or AES_FILE_DIRECT; both or other bits: AES_ERR_ARG */
} aes_file_config;

typedef struct aes_file_stats {
    uint64_t bytes;         /* file length */
    uint64_t chunks;        /* chunks processed */
    double seconds;         /* wall time of the call */
    double setup_seconds;   /* of which: mappings, pinned buffers and streams */
    int32_t threads;        /* workers used */
    int32_t os_errno;       /* errno of the failing file operation (AES_ERR_IO), else 0 */
    int32_t direct;         /* 1: the direct path ran, 0: the staged one */
    int32_t reserved;       /* 0 */
} aes_file_stats;

aes_status aes_file_crypt(const char *src_path, const char *dst_path, aes_file_mode mode,
                          const aes_key_schedule *ks, const uint8_t iv[16],
                          const aes_file_config *cfg, aes_file_stats *stats);

/* Free the pinned buffers that aes_file_crypt keeps between calls.  Safe at
 * any time, from any thread; buffers in use by a running call are not in the
 * pool and stay with that call. */
void aes_file_trim(void);

/* ------------------------------------------------------------------------
 * Continuous-batching AES-CTR server.  The paper has no counterpart: its
 * chunks become requests that arrive over time, each run through the batch
 * kernels with its tenant's resident key schedule.
 *
 * aes_server_progress runs one pass of the loop:
 *  1. frees the output ranges and budget of the completions it handed out in
 *     the previous call (a completion's output stays readable until then);
 *  2. admits waiting requests in arrival order while the budget allows: each
 *     is charged its input and output bytes rounded up to 16, its output range
 *     comes from a ring arena of the budget's size, and it takes the tenant's
 *     next counter range (IV = tenant nonce || 32-bit counter, the counter
 *     advanced by the request's blocks, so no keystream block repeats within
 *     a tenant until 2^32 blocks);
 *  3. launches every admitted request into the next batch as soon as one of
 *     the n_streams x slots_per_stream slots is free (continuous batching);
 *  4. reports the requests of batches whose event fired.  A batch not
 *     complete after batch_timeout_s is declared lost: its requests are
 *     reported with AES_ERR_TIMEOUT, its slot and output ranges are never
 *     reused, and the server stops admitting (aes_server_healthy returns 0).
 *
 * A server is used from one thread at a time.  d_pool (device, 16-byte
 * aligned, pool_bytes long) holds every request's input at a 16-byte aligned
 * offset; the caller keeps it alive and unchanged while requests are in
 * flight.  schedules (host, n_tenants) and nonces (host, 12 bytes per tenant)
 * are copied at creation.  Device memory held: the output arena
 * (budget_bytes), the schedule table and per slot max_batch_msgs descriptors
 * plus a batch workspace; pinned host memory: the descriptor staging of each
 * slot.  aes_server_destroy waits for the server's streams. */
typedef struct aes_server aes_server;

typedef struct aes_server_config {
    uint64_t budget_bytes;      /* bytes admitted at once (input + output per request); 0 = 8 GiB */
    uint32_t n_streams;         /* 0 = 2 (at most 64) */
    uint32_t slots_per_stream;  /* batches in flight per stream; 0 = 2 (at most 64) */
    uint32_t max_batch_msgs;    /* 0 = 8192 */
    int32_t grid_ctas;          /* persistent-kernel CTAs; 0 = one per SM */
    double batch_timeout_s;     /* 0 = 10 s */
    uint64_t inject_lost_batch; /* test hook: the k-th launched batch (1-based) is treated as never
                                   completing, on the host (its GPU work runs normally); 0 = none */
} aes_server_config;

typedef struct aes_server_completion {
    uint64_t id;            /* the caller's request id */
    int32_t status;         /* AES_OK, or AES_ERR_TIMEOUT (its batch was declared lost) */
    uint32_t tenant;
    uint64_t out_off;       /* offset of the output in aes_server_output(), readable until the next progress call */
    uint64_t length;
    uint32_t counter;       /* CTR counter of the request's first block */
    uint32_t reserved;
    double t_arrival, t_admitted, t_done;  /* seconds on the server's clock (t_done -2 when lost) */
} aes_server_completion;

typedef struct aes_server_stats {
    uint64_t submitted, completed, timed_out;
    uint64_t batches;             /* launched */
    uint64_t batches_overlapped;  /* launched while earlier batches were still on the GPU */
    uint64_t bytes;               /* completed request bytes */
    uint64_t max_charged;         /* peak budget in use */
    double mean_batch_msgs;
} aes_server_stats;

aes_status aes_server_create(const aes_server_config *cfg, const void *d_pool, uint64_t pool_bytes,
                             const aes_key_schedule *schedules, const uint8_t *nonces, uint32_t n_tenants,
                             aes_server **out);
void aes_server_destroy(aes_server *s);
/* Queue one request (arrival = now).  AES_ERR_ARG for a bad tenant, offset or
 * range; AES_ERR_NOMEM when its input and output bytes exceed the budget. */
aes_status aes_server_submit(aes_server *s, uint64_t id, uint32_t tenant, uint64_t in_off, uint64_t length);
/* One pass of the loop; writes up to max_done completions to done and returns
 * their count (the rest come with later calls).  *status (may be NULL) gets
 * the pass's status: a failed launch or CUDA error. */
uint32_t aes_server_progress(aes_server *s, aes_server_completion *done, uint32_t max_done, aes_status *status);
int aes_server_healthy(const aes_server *s);  /* 0 once a batch was declared lost */
int aes_server_idle(const aes_server *s);     /* 1: nothing waiting, queued, on the GPU or unreported */
void *aes_server_output(aes_server *s);       /* device base of the output arena */
double aes_server_now(const aes_server *s);   /* the server's clock, seconds */
void aes_server_get_stats(const aes_server *s, aes_server_stats *stats);
/* Replay an arrival schedule in real time on the calling thread: request i
 * (id i) arrives arrival_s[i] seconds after the call starts (non-decreasing),
 * for tenants[i], input at in_offs[i], lengths[i] bytes.  Runs until every
 * request is reported, a batch is lost and nothing else is in flight, or
 * time_limit_s passes.  Per request (arrays may be NULL): latency_s (done -
 * arrival; -1 not completed, -2 lost), wait_s (admission - arrival),
 * counters (its first CTR counter).  capture (device) with capture_off: the
 * output of each request whose capture_off is not UINT64_MAX is copied to
 * capture + capture_off[i] when it completes. */
aes_status aes_server_replay(aes_server *s, uint64_t n, const double *arrival_s, const uint32_t *tenants,
                             const uint64_t *in_offs, const uint64_t *lengths, double time_limit_s,
                             double *latency_s, double *wait_s, uint32_t *counters, void *capture,
                             const uint64_t *capture_off);

/* Device waits that gave up: the TMA-staged CTR variant (AES_VARIANT_TTABLE_BULK)
 * and the batch's lane kernel (AES_BATCH_SHORT_LANES) bound each wait for a
 * staged copy to about a second of SM clock; a warp whose copy has not landed
 * by then counts one timeout, leaves its remaining blocks unwritten and stops.  *count gets the timeouts counted on the current
 * device since the last call, and the count restarts at 0.  Synchronous (it
 * reads a device word): call it once the work it covers has completed.
 * Returns AES_OK, AES_ERR_TIMEOUT when *count > 0, AES_ERR_ARG for a null
 * pointer or AES_ERR_CUDA. */
aes_status aes_take_wait_timeouts(uint32_t *count);

/* The CUDA error code behind the calling thread's last AES_ERR_CUDA (0 if none). */
int aes_last_cuda_error(void);

/* A static, human-readable name for a status value. */
const char *aes_status_string(aes_status s);

#ifdef __cplusplus
}
#endif
#endif /* AESGPU_H */
