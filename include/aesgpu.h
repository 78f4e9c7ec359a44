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
    AES_ERR_BUSY = 10     /* resource in use */
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
    AES_VARIANT_BITSLICE = 2  /* bitsliced S-box / MixColumns on LOP3 */
} aes_variant;

/* Optional launch shape for the _ex calls; a zero field means "choose". */
typedef struct aes_launch_config {
    int32_t variant;           /* aes_variant */
    int32_t cta_threads;       /* threads per CTA: 128..1024, multiple of 32 */
    int32_t blocks_per_thread; /* 16-byte blocks per thread per iteration: 1, 2 or 4 */
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

/* The same three calls with an explicit launch shape (cfg may be NULL, which
 * equals the plain call).  Every shape computes identical bytes. */
aes_status aes_ecb_encrypt_ex(const aes_key_schedule *ks, const void *d_in, void *d_out,
                              size_t nbytes, void *stream, const aes_launch_config *cfg);
aes_status aes_ecb_decrypt_ex(const aes_key_schedule *ks, const void *d_in, void *d_out,
                              size_t nbytes, void *stream, const aes_launch_config *cfg);
aes_status aes_ctr_xcrypt_ex(const aes_key_schedule *ks, const uint8_t iv[16], const void *d_in,
                             void *d_out, size_t nbytes, void *stream,
                             const aes_launch_config *cfg);

/* The CUDA error code behind the calling thread's last AES_ERR_CUDA (0 if none). */
int aes_last_cuda_error(void);

/* A static, human-readable name for a status value. */
const char *aes_status_string(aes_status s);

#ifdef __cplusplus
}
#endif
#endif /* AESGPU_H */
