/*
 * aes_ref.h — the CPU oracle for bulk AES (test infrastructure only).
 *
 * This is a plain, slow, single-threaded C99 restatement of AES as the
 * paper's Fig. 1 lists it (§III.A: key expansion, an initial AddRoundKey,
 * Nr-1 rounds of SubBytes / ShiftRows / MixColumns / AddRoundKey, a final
 * round without MixColumns), with the arithmetic taken from FIPS-197 (the
 * standard the paper's AES is), the ECB and CTR modes of NIST SP 800-38A, and
 * PKCS#7 padding.  The paper's own parallel scheme (§IV.B: split the input into
 * N contiguous chunks, one pthread per chunk, outputs concatenated in place) is
 * the `_mt` family.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline leg may load
 * this code.  It shares no code, table or header with the GPU library.
 *
 * Byte conventions: keys, IVs and data are byte strings.  A round-key "word"
 * is 4 consecutive bytes of the expanded key, w[4i..4i+3] (FIPS-197 §5.2).
 */
#ifndef AES_REF_H
#define AES_REF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    REF_OK = 0,
    REF_ERR_KEYSIZE = -1, /* key_bits not 128, 192 or 256 */
    REF_ERR_LENGTH = -2,  /* ECB length not a multiple of 16 */
    REF_ERR_PADDING = -3, /* PKCS#7 padding malformed on decrypt */
    REF_ERR_THREAD = -4   /* pthread_create / join failed */
};

/* GF(2^8) with the AES polynomial x^8+x^4+x^3+x+1 (FIPS-197 §4.2). */
uint8_t ref_gf_mul(uint8_t a, uint8_t b);
uint8_t ref_gf_inv(uint8_t a); /* a^254; 0 maps to 0 */

/* SubBytes table and its inverse (FIPS-197 §5.1.1, §5.3.2). */
void ref_sbox(uint8_t out[256]);
void ref_inv_sbox(uint8_t out[256]);

/* One column through MixColumns / InvMixColumns, in place (§5.1.3, §5.3.3). */
void ref_mix_column(uint8_t col[4]);
void ref_inv_mix_column(uint8_t col[4]);

/* KeyExpansion (§5.2).  Writes 4*(Nr+1) words (16*(Nr+1) bytes, at most 240)
 * into w and Nr into *nr.  Returns the word count or REF_ERR_KEYSIZE. */
int ref_key_expansion(const uint8_t *key, int key_bits, uint8_t w[240], int *nr);

/* Cipher (§5.1) and InvCipher (§5.3) of one 16-byte block. */
void ref_cipher(const uint8_t in[16], uint8_t out[16], const uint8_t *w, int nr);
void ref_inv_cipher(const uint8_t in[16], uint8_t out[16], const uint8_t *w, int nr);

/* ECB (SP 800-38A §6.1): n must be a multiple of 16.  in == out allowed. */
int ref_ecb_encrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out, uint64_t n);
int ref_ecb_decrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out, uint64_t n);

/* CTR (SP 800-38A §6.5) with a 96-bit nonce and a 32-bit big-endian counter
 * in IV bytes 12..15 that wraps modulo 2^32.  Data byte 0 belongs to counter
 * block number first_block; any n, the last partial block uses the leading
 * keystream bytes.  Encryption and decryption are the same call. */
int ref_ctr_xcrypt(const uint8_t *key, int key_bits, const uint8_t iv[16], uint64_t first_block,
                   const uint8_t *in, uint8_t *out, uint64_t n);

/* CTR on a sample: block k of in/out (16 bytes each) is counter block idx[k]. */
int ref_ctr_xcrypt_blocks(const uint8_t *key, int key_bits, const uint8_t iv[16],
                          const uint64_t *idx, const uint8_t *in, uint8_t *out, uint64_t nblocks);

/* PKCS#7 over ECB.  Encrypt writes ref_pkcs7_padded_len(n) bytes.  Decrypt
 * (n a positive multiple of 16) writes the unpadded plaintext and its length,
 * or returns REF_ERR_PADDING when the last block's pad is malformed. */
uint64_t ref_pkcs7_padded_len(uint64_t n);
int ref_ecb_pkcs7_encrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint64_t n,
                          uint8_t *out, uint64_t *out_len);
int ref_ecb_pkcs7_decrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint64_t n,
                          uint8_t *out, uint64_t *out_len);

/* CBC (SP 800-38A §6.2): C_j = CIPH(P_j ^ C_{j-1}), C_0 = IV; n a multiple
 * of 16.  Decryption P_j = CIPH^-1(C_j) ^ C_{j-1}.  in == out allowed. */
int ref_cbc_encrypt(const uint8_t *key, int key_bits, const uint8_t iv[16], const uint8_t *in,
                    uint8_t *out, uint64_t n);
int ref_cbc_decrypt(const uint8_t *key, int key_bits, const uint8_t iv[16], const uint8_t *in,
                    uint8_t *out, uint64_t n);

/* XTS-AES (IEEE 1619 / SP 800-38E) without ciphertext stealing: the buffer
 * is n / sector_bytes data units (n a multiple of sector_bytes, sector_bytes
 * a positive multiple of 16); unit u has the tweak value first_sector + u as a
 * 128-bit little-endian integer; T = CIPH_K2(tweak), then for each block
 * C = CIPH_K1(P ^ T) ^ T and T = T * alpha in GF(2^128) (shift left by one
 * bit of the little-endian value, 0x87 folded into byte 0 on carry out).
 * key1 encrypts the data, key2 the tweak; both key_bits. */
int ref_xts_encrypt(const uint8_t *key1, const uint8_t *key2, int key_bits, uint64_t sector_bytes,
                    uint64_t first_sector, const uint8_t *in, uint8_t *out, uint64_t n);
int ref_xts_decrypt(const uint8_t *key1, const uint8_t *key2, int key_bits, uint64_t sector_bytes,
                    uint64_t first_sector, const uint8_t *in, uint8_t *out, uint64_t n);

/* The paper's pthreads scheme (§IV.B): nthreads contiguous chunks of whole
 * blocks, the remainder (and any partial CTR block) in the last chunk, one
 * thread per chunk running the single-threaded routine, joined.  nthreads < 1
 * means 1.  Output bytes are identical to the single-threaded call. */
int ref_ecb_encrypt_mt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out,
                       uint64_t n, int nthreads);
int ref_ecb_decrypt_mt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out,
                       uint64_t n, int nthreads);
int ref_ctr_xcrypt_mt(const uint8_t *key, int key_bits, const uint8_t iv[16], uint64_t first_block,
                      const uint8_t *in, uint8_t *out, uint64_t n, int nthreads);

/* A list of independent messages, each with its own key (and IV): message m
 * is in[in_off[m] .. in_off[m] + in_len[m]), its key the first key_bits[m]/8
 * bytes of keys + 32m, its IV (CTR) ivs + 16m.  op 0: CTR
 * (ref_ctr_xcrypt, output in_len[m] bytes); op 1: PKCS#7 then ECB
 * (ref_ecb_pkcs7_encrypt); op 2: ECB decryption then the PKCS#7 check
 * (ref_ecb_pkcs7_decrypt, the whole decrypted length written, out_len[m] the
 * unpadded one).  Output m goes to out + out_off[m]; status[m] gets the
 * message's REF_* code and out_len[m] its output length (0 on failure).  The
 * messages are shared out to nthreads threads, each taking the next unclaimed
 * message in turn (the paper's chunk-per-thread scheme with chunks =
 * messages); every message runs the single-threaded routine on its own.
 * Returns REF_OK, or REF_ERR_THREAD / REF_ERR_LENGTH (unknown op). */
int ref_batch_mt(int op, uint64_t n_msgs, const uint8_t *in, const uint64_t *in_off,
                 const uint64_t *in_len, uint8_t *out, const uint64_t *out_off, const uint8_t *keys,
                 const uint32_t *key_bits, const uint8_t *ivs, uint64_t *out_len, int32_t *status,
                 int nthreads);

#ifdef __cplusplus
}
#endif
#endif
