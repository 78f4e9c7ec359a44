/*
 * aes_ref.c — CPU oracle for bulk AES.  TEST INFRASTRUCTURE: only the tests,
 * the smoke check and the bench's CPU-baseline leg load it; the GPU library
 * never does, and the two share no code or tables.
 *
 * Everything here follows the definitions step by step, with no table fusion,
 * no word tricks and no reordering:
 *   - the step list of the paper's Fig. 1 (§III.A): KeyExpansion, initial
 *     AddRoundKey, Nr-1 full rounds (SubBytes, ShiftRows, MixColumns,
 *     AddRoundKey), a final round without MixColumns;
 *   - the arithmetic of FIPS-197 (§4.2 GF(2^8), §5.1 Cipher, §5.2
 *     KeyExpansion, §5.3 InvCipher);
 *   - SP 800-38A §6.1 (ECB) and §6.5 (CTR), with the counter read as a
 *     32-bit big-endian integer in IV bytes 12..15 that wraps modulo 2^32;
 *   - PKCS#7 padding (1..16 bytes, each equal to the pad length).
 * Every pin that ties this file to something other than itself lives in
 * tests/test_oracle_pins.py.
 */
#include "aes_ref.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---- GF(2^8), FIPS-197 §4.2 ------------------------------------------- */

/* Multiply by x (§4.2.1): shift left, reduce by m(x) = 0x11B if bit 8 is set. */
static uint8_t xtime(uint8_t a) {
    unsigned v = (unsigned)a << 1;
    if (v & 0x100u) v ^= 0x11Bu;
    return (uint8_t)v;
}

/* Shift-and-add multiplication: sum of a*x^i over the set bits i of b. */
uint8_t ref_gf_mul(uint8_t a, uint8_t b) {
    uint8_t p = 0;
    while (b) {
        if (b & 1u) p ^= a;
        a = xtime(a);
        b >>= 1;
    }
    return p;
}

/* Multiplicative inverse as a^254 (a^255 = 1 for a != 0), square-and-multiply;
 * 0 maps to 0 as §5.1.1 prescribes. */
uint8_t ref_gf_inv(uint8_t a) {
    uint8_t result = 1, base = a;
    unsigned e = 254;
    if (a == 0) return 0;
    while (e) {
        if (e & 1u) result = ref_gf_mul(result, base);
        base = ref_gf_mul(base, base);
        e >>= 1;
    }
    return result;
}

/* ---- S-box, FIPS-197 §5.1.1 -------------------------------------------- */

static uint8_t rotl8(uint8_t v, int k) { return (uint8_t)((v << k) | (v >> (8 - k))); }

/* SubBytes of one byte: inverse in GF(2^8), then the affine map
 * s = b ^ rotl(b,1) ^ rotl(b,2) ^ rotl(b,3) ^ rotl(b,4) ^ 0x63 (eq. 5.1). */
static uint8_t sub_byte(uint8_t x) {
    uint8_t b = ref_gf_inv(x);
    return (uint8_t)(b ^ rotl8(b, 1) ^ rotl8(b, 2) ^ rotl8(b, 3) ^ rotl8(b, 4) ^ 0x63u);
}

static uint8_t g_sbox[256], g_inv_sbox[256];
static pthread_once_t g_sbox_once = PTHREAD_ONCE_INIT;

static void build_sbox(void) {
    for (int x = 0; x < 256; ++x) g_sbox[x] = sub_byte((uint8_t)x);
    /* InvSubBytes (§5.3.2) is the inverse permutation. */
    for (int x = 0; x < 256; ++x) g_inv_sbox[g_sbox[x]] = (uint8_t)x;
}

static void ensure_sbox(void) { pthread_once(&g_sbox_once, build_sbox); }

void ref_sbox(uint8_t out[256]) { ensure_sbox(); memcpy(out, g_sbox, 256); }
void ref_inv_sbox(uint8_t out[256]) { ensure_sbox(); memcpy(out, g_inv_sbox, 256); }

/* ---- MixColumns / InvMixColumns, §5.1.3 and §5.3.3 ---------------------- */

/* Column times the circulant matrix whose first row is (02 03 01 01). */
static const uint8_t MIX[4][4] = {
    {2, 3, 1, 1}, {1, 2, 3, 1}, {1, 1, 2, 3}, {3, 1, 1, 2}};
/* and its inverse, first row (0e 0b 0d 09). */
static const uint8_t INV_MIX[4][4] = {
    {14, 11, 13, 9}, {9, 14, 11, 13}, {13, 9, 14, 11}, {11, 13, 9, 14}};

static void mat_column(const uint8_t m[4][4], uint8_t col[4]) {
    uint8_t out[4];
    for (int r = 0; r < 4; ++r) {
        uint8_t acc = 0;
        for (int i = 0; i < 4; ++i) acc ^= ref_gf_mul(m[r][i], col[i]);
        out[r] = acc;
    }
    memcpy(col, out, 4);
}

void ref_mix_column(uint8_t col[4]) { mat_column(MIX, col); }
void ref_inv_mix_column(uint8_t col[4]) { mat_column(INV_MIX, col); }

/* ---- KeyExpansion, §5.2 (paper Fig. 1 step 1) -------------------------- */

int ref_key_expansion(const uint8_t *key, int key_bits, uint8_t w[240], int *nr) {
    int nk, rounds;
    switch (key_bits) {
    case 128: nk = 4; rounds = 10; break;
    case 192: nk = 6; rounds = 12; break;
    case 256: nk = 8; rounds = 14; break;
    default: return REF_ERR_KEYSIZE;
    }
    ensure_sbox();
    const int nwords = 4 * (rounds + 1);
    memcpy(w, key, (size_t)(4 * nk)); /* w[0..Nk-1] are the key's words */
    uint8_t rcon = 1;                 /* Rcon[i/Nk] = (x^(i/Nk - 1), 0, 0, 0) */
    for (int i = nk; i < nwords; ++i) {
        uint8_t t[4];
        memcpy(t, &w[4 * (i - 1)], 4);
        if (i % nk == 0) {
            /* RotWord: [a0,a1,a2,a3] -> [a1,a2,a3,a0]; then SubWord; then Rcon. */
            uint8_t a0 = t[0];
            t[0] = t[1]; t[1] = t[2]; t[2] = t[3]; t[3] = a0;
            for (int k = 0; k < 4; ++k) t[k] = g_sbox[t[k]];
            t[0] ^= rcon;
            rcon = xtime(rcon);
        } else if (nk > 6 && i % nk == 4) {
            for (int k = 0; k < 4; ++k) t[k] = g_sbox[t[k]];
        }
        for (int k = 0; k < 4; ++k) w[4 * i + k] = (uint8_t)(w[4 * (i - nk) + k] ^ t[k]);
    }
    *nr = rounds;
    return nwords;
}

/* ---- Cipher, §5.1 (paper Fig. 1 steps 2-4) ----------------------------- */

/* The state is s[r][c] = block byte r + 4c (§3.4). */
typedef uint8_t state_t[4][4];

static void load_state(state_t s, const uint8_t in[16]) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) s[r][c] = in[r + 4 * c];
}

static void store_state(uint8_t out[16], state_t s) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) out[r + 4 * c] = s[r][c];
}

/* AddRoundKey (§5.1.4): column c ^= w[4*round + c]. */
static void add_round_key(state_t s, const uint8_t *w, int round) {
    for (int c = 0; c < 4; ++c)
        for (int r = 0; r < 4; ++r) s[r][c] ^= w[16 * round + 4 * c + r];
}

static void sub_bytes(state_t s) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) s[r][c] = g_sbox[s[r][c]];
}

static void inv_sub_bytes(state_t s) {
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) s[r][c] = g_inv_sbox[s[r][c]];
}

/* ShiftRows (§5.1.2): row r moves left by r, s'[r][c] = s[r][(c + r) mod 4]. */
static void shift_rows(state_t s) {
    for (int r = 1; r < 4; ++r) {
        uint8_t row[4];
        for (int c = 0; c < 4; ++c) row[c] = s[r][(c + r) % 4];
        for (int c = 0; c < 4; ++c) s[r][c] = row[c];
    }
}

/* InvShiftRows (§5.3.1): s'[r][(c + r) mod 4] = s[r][c]. */
static void inv_shift_rows(state_t s) {
    for (int r = 1; r < 4; ++r) {
        uint8_t row[4];
        for (int c = 0; c < 4; ++c) row[(c + r) % 4] = s[r][c];
        for (int c = 0; c < 4; ++c) s[r][c] = row[c];
    }
}

static void mix_columns(state_t s) {
    for (int c = 0; c < 4; ++c) {
        uint8_t col[4] = {s[0][c], s[1][c], s[2][c], s[3][c]};
        ref_mix_column(col);
        for (int r = 0; r < 4; ++r) s[r][c] = col[r];
    }
}

static void inv_mix_columns(state_t s) {
    for (int c = 0; c < 4; ++c) {
        uint8_t col[4] = {s[0][c], s[1][c], s[2][c], s[3][c]};
        ref_inv_mix_column(col);
        for (int r = 0; r < 4; ++r) s[r][c] = col[r];
    }
}

void ref_cipher(const uint8_t in[16], uint8_t out[16], const uint8_t *w, int nr) {
    state_t s;
    ensure_sbox();
    load_state(s, in);
    add_round_key(s, w, 0);              /* initial round */
    for (int round = 1; round < nr; ++round) {
        sub_bytes(s);
        shift_rows(s);
        mix_columns(s);
        add_round_key(s, w, round);
    }
    sub_bytes(s);                        /* final round: no MixColumns */
    shift_rows(s);
    add_round_key(s, w, nr);
    store_state(out, s);
}

/* InvCipher in the plain order of §5.3 (Fig. 12), not the equivalent form. */
void ref_inv_cipher(const uint8_t in[16], uint8_t out[16], const uint8_t *w, int nr) {
    state_t s;
    ensure_sbox();
    load_state(s, in);
    add_round_key(s, w, nr);
    for (int round = nr - 1; round >= 1; --round) {
        inv_shift_rows(s);
        inv_sub_bytes(s);
        add_round_key(s, w, round);
        inv_mix_columns(s);
    }
    inv_shift_rows(s);
    inv_sub_bytes(s);
    add_round_key(s, w, 0);
    store_state(out, s);
}

/* ---- ECB, SP 800-38A §6.1 ---------------------------------------------- */

int ref_ecb_encrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out, uint64_t n) {
    uint8_t w[240];
    int nr;
    if (ref_key_expansion(key, key_bits, w, &nr) < 0) return REF_ERR_KEYSIZE;
    if (n % 16) return REF_ERR_LENGTH;
    for (uint64_t off = 0; off < n; off += 16) ref_cipher(in + off, out + off, w, nr);
    return REF_OK;
}

int ref_ecb_decrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out, uint64_t n) {
    uint8_t w[240];
    int nr;
    if (ref_key_expansion(key, key_bits, w, &nr) < 0) return REF_ERR_KEYSIZE;
    if (n % 16) return REF_ERR_LENGTH;
    for (uint64_t off = 0; off < n; off += 16) ref_inv_cipher(in + off, out + off, w, nr);
    return REF_OK;
}

/* ---- CTR, SP 800-38A §6.5 ---------------------------------------------- */

/* Counter block j: the IV's first 12 bytes, then (c0 + j) mod 2^32 big-endian,
 * where c0 is IV bytes 12..15 read big-endian. */
static void counter_block(const uint8_t iv[16], uint64_t j, uint8_t t[16]) {
    uint32_t c0 = ((uint32_t)iv[12] << 24) | ((uint32_t)iv[13] << 16) |
                  ((uint32_t)iv[14] << 8) | (uint32_t)iv[15];
    uint32_t c = (uint32_t)(c0 + (uint32_t)j); /* modulo 2^32 */
    memcpy(t, iv, 12);
    t[12] = (uint8_t)(c >> 24);
    t[13] = (uint8_t)(c >> 16);
    t[14] = (uint8_t)(c >> 8);
    t[15] = (uint8_t)c;
}

int ref_ctr_xcrypt(const uint8_t *key, int key_bits, const uint8_t iv[16], uint64_t first_block,
                   const uint8_t *in, uint8_t *out, uint64_t n) {
    uint8_t w[240], t[16], o[16];
    int nr;
    if (ref_key_expansion(key, key_bits, w, &nr) < 0) return REF_ERR_KEYSIZE;
    for (uint64_t off = 0, j = first_block; off < n; off += 16, ++j) {
        counter_block(iv, j, t);
        ref_cipher(t, o, w, nr);            /* O_j = CIPH_K(T_j) */
        uint64_t len = n - off < 16 ? n - off : 16;
        for (uint64_t k = 0; k < len; ++k) out[off + k] = (uint8_t)(in[off + k] ^ o[k]);
    }
    return REF_OK;
}

int ref_ctr_xcrypt_blocks(const uint8_t *key, int key_bits, const uint8_t iv[16],
                          const uint64_t *idx, const uint8_t *in, uint8_t *out, uint64_t nblocks) {
    uint8_t w[240], t[16], o[16];
    int nr;
    if (ref_key_expansion(key, key_bits, w, &nr) < 0) return REF_ERR_KEYSIZE;
    for (uint64_t k = 0; k < nblocks; ++k) {
        counter_block(iv, idx[k], t);
        ref_cipher(t, o, w, nr);
        for (int b = 0; b < 16; ++b) out[16 * k + b] = (uint8_t)(in[16 * k + b] ^ o[b]);
    }
    return REF_OK;
}

/* ---- PKCS#7 over ECB --------------------------------------------------- */

uint64_t ref_pkcs7_padded_len(uint64_t n) { return n - n % 16 + 16; }

int ref_ecb_pkcs7_encrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint64_t n,
                          uint8_t *out, uint64_t *out_len) {
    uint64_t total = ref_pkcs7_padded_len(n);
    uint8_t p = (uint8_t)(total - n); /* 1..16 */
    memmove(out, in, (size_t)n);
    for (uint64_t k = n; k < total; ++k) out[k] = p;
    *out_len = total;
    return ref_ecb_encrypt(key, key_bits, out, out, total);
}

int ref_ecb_pkcs7_decrypt(const uint8_t *key, int key_bits, const uint8_t *in, uint64_t n,
                          uint8_t *out, uint64_t *out_len) {
    if (n == 0 || n % 16) return REF_ERR_LENGTH;
    int rc = ref_ecb_decrypt(key, key_bits, in, out, n);
    if (rc) return rc;
    uint8_t p = out[n - 1];
    if (p < 1 || p > 16) return REF_ERR_PADDING;
    for (uint64_t k = n - p; k < n; ++k)
        if (out[k] != p) return REF_ERR_PADDING;
    *out_len = n - p;
    return REF_OK;
}

/* ---- CBC, SP 800-38A §6.2 ---------------------------------------------- */

int ref_cbc_encrypt(const uint8_t *key, int key_bits, const uint8_t iv[16], const uint8_t *in,
                    uint8_t *out, uint64_t n) {
    uint8_t w[240], chain[16], x[16];
    int nr;
    if (ref_key_expansion(key, key_bits, w, &nr) < 0) return REF_ERR_KEYSIZE;
    if (n % 16) return REF_ERR_LENGTH;
    memcpy(chain, iv, 16);
    for (uint64_t off = 0; off < n; off += 16) {
        for (int b = 0; b < 16; ++b) x[b] = (uint8_t)(in[off + b] ^ chain[b]);
        ref_cipher(x, out + off, w, nr);
        memcpy(chain, out + off, 16);
    }
    return REF_OK;
}

int ref_cbc_decrypt(const uint8_t *key, int key_bits, const uint8_t iv[16], const uint8_t *in,
                    uint8_t *out, uint64_t n) {
    uint8_t w[240], prev[16], cur[16], x[16];
    int nr;
    if (ref_key_expansion(key, key_bits, w, &nr) < 0) return REF_ERR_KEYSIZE;
    if (n % 16) return REF_ERR_LENGTH;
    memcpy(prev, iv, 16);
    for (uint64_t off = 0; off < n; off += 16) {
        memcpy(cur, in + off, 16); /* kept before `out` may overwrite it in place */
        ref_inv_cipher(cur, x, w, nr);
        for (int b = 0; b < 16; ++b) out[off + b] = (uint8_t)(x[b] ^ prev[b]);
        memcpy(prev, cur, 16);
    }
    return REF_OK;
}

/* ---- XTS, IEEE 1619 (no ciphertext stealing) --------------------------- */

/* T * alpha: the 16 bytes as a little-endian 128-bit integer shifted left by
 * one, the bit shifted out of byte 15 folded back as 0x87 into byte 0. */
static void xts_double(uint8_t t[16]) {
    unsigned carry = 0;
    for (int i = 0; i < 16; ++i) {
        unsigned v = ((unsigned)t[i] << 1) | carry;
        carry = (t[i] >> 7) & 1u;
        t[i] = (uint8_t)v;
    }
    if (carry) t[0] ^= 0x87u;
}

static int xts_run(int decrypt, const uint8_t *key1, const uint8_t *key2, int key_bits,
                   uint64_t sector_bytes, uint64_t first_sector, const uint8_t *in, uint8_t *out,
                   uint64_t n) {
    uint8_t w1[240], w2[240], t[16], x[16], y[16];
    int nr1, nr2;
    if (ref_key_expansion(key1, key_bits, w1, &nr1) < 0) return REF_ERR_KEYSIZE;
    if (ref_key_expansion(key2, key_bits, w2, &nr2) < 0) return REF_ERR_KEYSIZE;
    if (sector_bytes == 0 || sector_bytes % 16 || n % sector_bytes) return REF_ERR_LENGTH;
    for (uint64_t u = 0; u < n / sector_bytes; ++u) {
        uint64_t sector = first_sector + u;
        uint8_t tv[16] = {0};
        for (int i = 0; i < 8; ++i) tv[i] = (uint8_t)(sector >> (8 * i));
        ref_cipher(tv, t, w2, nr2); /* T = CIPH_K2(tweak value) */
        for (uint64_t j = 0; j < sector_bytes / 16; ++j) {
            const uint64_t off = u * sector_bytes + 16 * j;
            for (int b = 0; b < 16; ++b) x[b] = (uint8_t)(in[off + b] ^ t[b]);
            if (decrypt) ref_inv_cipher(x, y, w1, nr1);
            else ref_cipher(x, y, w1, nr1);
            for (int b = 0; b < 16; ++b) out[off + b] = (uint8_t)(y[b] ^ t[b]);
            xts_double(t);
        }
    }
    return REF_OK;
}

int ref_xts_encrypt(const uint8_t *key1, const uint8_t *key2, int key_bits, uint64_t sector_bytes,
                    uint64_t first_sector, const uint8_t *in, uint8_t *out, uint64_t n) {
    return xts_run(0, key1, key2, key_bits, sector_bytes, first_sector, in, out, n);
}

int ref_xts_decrypt(const uint8_t *key1, const uint8_t *key2, int key_bits, uint64_t sector_bytes,
                    uint64_t first_sector, const uint8_t *in, uint8_t *out, uint64_t n) {
    return xts_run(1, key1, key2, key_bits, sector_bytes, first_sector, in, out, n);
}

/* ---- The paper's pthreads scheme, §IV.B -------------------------------- */

typedef struct {
    int op; /* 0 ECB encrypt, 1 ECB decrypt, 2 CTR */
    const uint8_t *key;
    int key_bits;
    const uint8_t *iv;
    uint64_t first_block;
    const uint8_t *in;
    uint8_t *out;
    uint64_t n;
    int rc;
} chunk_t;

static void *chunk_main(void *arg) {
    chunk_t *c = (chunk_t *)arg;
    switch (c->op) {
    case 0: c->rc = ref_ecb_encrypt(c->key, c->key_bits, c->in, c->out, c->n); break;
    case 1: c->rc = ref_ecb_decrypt(c->key, c->key_bits, c->in, c->out, c->n); break;
    default:
        c->rc = ref_ctr_xcrypt(c->key, c->key_bits, c->iv, c->first_block, c->in, c->out, c->n);
    }
    return NULL;
}

static int run_chunks(int op, const uint8_t *key, int key_bits, const uint8_t *iv,
                      uint64_t first_block, const uint8_t *in, uint8_t *out, uint64_t n,
                      int nthreads) {
    if (key_bits != 128 && key_bits != 192 && key_bits != 256) return REF_ERR_KEYSIZE;
    if (op != 2 && n % 16) return REF_ERR_LENGTH;
    if (nthreads < 1) nthreads = 1;
    ensure_sbox(); /* build the shared table before any thread reads it */
    const uint64_t nblocks = n / 16, per = nblocks / (uint64_t)nthreads;
    chunk_t *cs = (chunk_t *)calloc((size_t)nthreads, sizeof(chunk_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)nthreads, sizeof(int));
    int rc = REF_OK;
    if (!cs || !th || !started) { rc = REF_ERR_THREAD; goto done; }
    for (int t = 0; t < nthreads; ++t) {
        uint64_t b0 = per * (uint64_t)t;
        uint64_t len = (t == nthreads - 1) ? n - 16 * b0 : 16 * per;
        cs[t] = (chunk_t){op, key, key_bits, iv, first_block + b0, in + 16 * b0, out + 16 * b0, len, 0};
        if (pthread_create(&th[t], NULL, chunk_main, &cs[t]) != 0) { rc = REF_ERR_THREAD; break; }
        started[t] = 1;
    }
    for (int t = 0; t < nthreads; ++t) {
        if (!started[t]) continue;
        if (pthread_join(th[t], NULL) != 0) rc = REF_ERR_THREAD;
        if (rc == REF_OK && cs[t].rc) rc = cs[t].rc;
    }
done:
    free(cs);
    free(th);
    free(started);
    return rc;
}

int ref_ecb_encrypt_mt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out,
                       uint64_t n, int nthreads) {
    return run_chunks(0, key, key_bits, NULL, 0, in, out, n, nthreads);
}

int ref_ecb_decrypt_mt(const uint8_t *key, int key_bits, const uint8_t *in, uint8_t *out,
                       uint64_t n, int nthreads) {
    return run_chunks(1, key, key_bits, NULL, 0, in, out, n, nthreads);
}

int ref_ctr_xcrypt_mt(const uint8_t *key, int key_bits, const uint8_t iv[16], uint64_t first_block,
                      const uint8_t *in, uint8_t *out, uint64_t n, int nthreads) {
    return run_chunks(2, key, key_bits, iv, first_block, in, out, n, nthreads);
}

/* ---- A list of messages over threads (the batched workloads) ----------- */

typedef struct {
    int op;
    uint64_t n_msgs;
    const uint8_t *in;
    const uint64_t *in_off, *in_len, *out_off;
    uint8_t *out;
    const uint8_t *keys, *ivs;
    const uint32_t *key_bits;
    uint64_t *out_len;
    int32_t *status;
    uint64_t next; /* next unclaimed message, under mu */
    pthread_mutex_t mu;
} batch_t;

static void batch_one(batch_t *b, uint64_t m) {
    const uint8_t *key = b->keys + 32 * m;
    const int bits = (int)b->key_bits[m];
    const uint8_t *src = b->in + b->in_off[m];
    uint8_t *dst = b->out + b->out_off[m];
    const uint64_t n = b->in_len[m];
    uint64_t olen = 0;
    int rc;
    if (b->op == 0) {
        rc = ref_ctr_xcrypt(key, bits, b->ivs + 16 * m, 0, src, dst, n);
        olen = n;
    } else if (b->op == 1) {
        rc = ref_ecb_pkcs7_encrypt(key, bits, src, n, dst, &olen);
    } else {
        rc = ref_ecb_pkcs7_decrypt(key, bits, src, n, dst, &olen);
    }
    b->status[m] = rc;
    b->out_len[m] = rc == REF_OK ? olen : 0;
}

static void *batch_main(void *arg) {
    batch_t *b = (batch_t *)arg;
    for (;;) {
        pthread_mutex_lock(&b->mu);
        const uint64_t m = b->next;
        if (m < b->n_msgs) b->next = m + 1;
        pthread_mutex_unlock(&b->mu);
        if (m >= b->n_msgs) return NULL;
        batch_one(b, m);
    }
}

int ref_batch_mt(int op, uint64_t n_msgs, const uint8_t *in, const uint64_t *in_off,
                 const uint64_t *in_len, uint8_t *out, const uint64_t *out_off, const uint8_t *keys,
                 const uint32_t *key_bits, const uint8_t *ivs, uint64_t *out_len, int32_t *status,
                 int nthreads) {
    if (op < 0 || op > 2) return REF_ERR_LENGTH;
    if (nthreads < 1) nthreads = 1;
    ensure_sbox(); /* build the shared table before any thread reads it */
    batch_t b = {op, n_msgs, in, in_off, in_len, out_off, out, keys, ivs, key_bits, out_len, status, 0,
                 PTHREAD_MUTEX_INITIALIZER};
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!th) return REF_ERR_THREAD;
    int started = 0, rc = REF_OK;
    for (; started < nthreads; ++started)
        if (pthread_create(&th[started], NULL, batch_main, &b) != 0) { rc = REF_ERR_THREAD; break; }
    if (started == 0) batch_main(&b); /* no thread could start: run the list here */
    for (int t = 0; t < started; ++t)
        if (pthread_join(th[t], NULL) != 0) rc = REF_ERR_THREAD;
    free(th);
    pthread_mutex_destroy(&b.mu);
    return rc;
}
