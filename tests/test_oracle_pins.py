"""Pins for the CPU oracle: each ties it to something other than itself.

The paper prints no key, plaintext or ciphertext (its only algorithmic text is
the step list of Fig. 1, §III.A), and the FIPS-197 / SP 800-38A example
vectors are not available offline here, so the oracle is pinned by:

* exhaustive / brute-force routes that differ from the oracle's own route
  (polynomial long division vs. its shift-and-reduce multiply, exhaustive
  inverse search vs. its x^254 exponentiation, the bit-matrix form of the
  affine map vs. its rotation form, MixColumns as polynomial multiplication
  modulo x^4+1 vs. its matrix form);
* structural facts of the definitions (S-box bijective with no fixed points,
  the key-schedule recurrence, InvMixColumns o MixColumns = id, D(E(x)) = x,
  CTR self-inverse and equal to ECB of the counter blocks, counter wrap);
* an independent library implementation: OpenSSL through the `cryptography`
  package (ECB, CTR, PKCS#7), on seeded random keys, IVs and data for every
  key size;
* the paper's chunked scheme (§IV.B) giving the same bytes as one pass.

A plausible mistake anywhere in the oracle fails at least one of these; the
mutation test at the end plants such mistakes in a copy of the oracle and
checks that the battery catches each one.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import synth
from oracle import Oracle
from oracle import oracle as oracle_mod

KEY_BITS = (128, 192, 256)


# ---------------------------------------------------------------------------
# independent GF(2^8) route: carry-less product, then polynomial long division
# ---------------------------------------------------------------------------

def clmul(a: int, b: int) -> int:
    r = 0
    for i in range(8):
        if (b >> i) & 1:
            r ^= a << i
    return r


def poly_mod(p: int, m: int = 0x11B) -> int:
    for deg in range(14, 7, -1):
        if (p >> deg) & 1:
            p ^= m << (deg - 8)
    return p


def gmul(a: int, b: int) -> int:
    return poly_mod(clmul(a, b))


def test_gf_mul_exhaustive(oracle):
    for a in range(256):
        for b in range(256):
            assert oracle.gf_mul(a, b) == gmul(a, b), (a, b)


def test_gf_inv_exhaustive_search(oracle):
    assert oracle.gf_inv(0) == 0
    for a in range(1, 256):
        inv = [b for b in range(1, 256) if gmul(a, b) == 1]
        assert len(inv) == 1
        assert oracle.gf_inv(a) == inv[0]


def affine_bitwise(b: int) -> int:
    # FIPS-197 eq. (5.1) in bit form: b'_i = b_i ^ b_{i+4} ^ b_{i+5} ^ b_{i+6} ^ b_{i+7} ^ c_i
    c = 0x63
    out = 0
    for i in range(8):
        bit = ((b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8)) ^ (b >> ((i + 6) % 8))
               ^ (b >> ((i + 7) % 8)) ^ (c >> i)) & 1
        out |= bit << i
    return out


def test_sbox_from_exhaustive_inverse_and_bit_affine(oracle):
    s = oracle.sbox()
    for x in range(256):
        inv = 0 if x == 0 else next(b for b in range(1, 256) if gmul(x, b) == 1)
        assert s[x] == affine_bitwise(inv), x


def test_sbox_structure(oracle):
    s, si = oracle.sbox(), oracle.inv_sbox()
    assert sorted(s.tolist()) == list(range(256)), "S-box must be a bijection"
    assert all(si[s[x]] == x for x in range(256))
    assert all(s[x] != x for x in range(256)), "AES S-box has no fixed points"
    assert all(s[x] != (x ^ 0xFF) for x in range(256)), "nor opposite fixed points"
    # 0 has no inverse and maps to 0, so S(0) is the affine constant; 1 is its own inverse.
    assert s[0] == 0x63 and s[1] == affine_bitwise(1)


def poly4_mul(a, b):
    """Product of two polynomials with GF(2^8) coefficients modulo x^4 + 1."""
    out = [0, 0, 0, 0]
    for i in range(4):
        for j in range(4):
            out[(i + j) % 4] ^= gmul(a[i], b[j])
    return out


def test_mix_column_is_poly_product(oracle):
    # FIPS-197 §5.1.3: column(x) * a(x), a(x) = {03}x^3 + {01}x^2 + {01}x + {02} mod x^4+1;
    # §5.3.3: a^-1(x) = {0b}x^3 + {0d}x^2 + {09}x + {0e}.
    a = [0x02, 0x01, 0x01, 0x03]
    ainv = [0x0E, 0x09, 0x0D, 0x0B]
    assert poly4_mul(a, ainv) == [1, 0, 0, 0]
    rng = np.random.default_rng(7)
    for _ in range(300):
        col = rng.integers(0, 256, 4).tolist()
        assert oracle.mix_column(col).tolist() == poly4_mul(col, a)
        assert oracle.inv_mix_column(col).tolist() == poly4_mul(col, ainv)
        assert oracle.inv_mix_column(oracle.mix_column(col)).tolist() == col


@pytest.mark.parametrize("bits", KEY_BITS)
def test_key_expansion_recurrence(oracle, bits):
    nk = bits // 32
    for seed in range(20):
        key = synth.key_bytes(seed, bits)
        w, nr = oracle.key_expansion(key, bits)
        assert nr == {128: 10, 192: 12, 256: 14}[bits]
        assert w.size == 16 * (nr + 1)
        words = w.reshape(-1, 4)
        assert np.array_equal(words[:nk].reshape(-1), key)
        for i in range(nk, words.shape[0]):
            if i % nk == 0 or (nk == 8 and i % nk == 4):
                continue
            assert np.array_equal(words[i], words[i - nk] ^ words[i - 1])


def test_key_size_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.key_expansion(np.zeros(32, np.uint8), 64)
    with pytest.raises(ValueError):
        oracle.ecb_encrypt(np.zeros(16, np.uint8), 160, np.zeros(16, np.uint8))


# ---------------------------------------------------------------------------
# independent library: OpenSSL through `cryptography`
# ---------------------------------------------------------------------------

def _openssl():
    return pytest.importorskip("cryptography.hazmat.primitives.ciphers")


def openssl_ecb(key, data, decrypt=False):
    c = _openssl()
    ctx = c.Cipher(c.algorithms.AES(bytes(key)), c.modes.ECB())
    op = ctx.decryptor() if decrypt else ctx.encryptor()
    return np.frombuffer(op.update(bytes(data)) + op.finalize(), np.uint8)


def openssl_ctr(key, iv, data):
    # OpenSSL increments the whole 128-bit block; identical to the 32-bit
    # counter as long as the low word does not wrap, which the callers ensure.
    c = _openssl()
    op = c.Cipher(c.algorithms.AES(bytes(key)), c.modes.CTR(bytes(iv))).encryptor()
    return np.frombuffer(op.update(bytes(data)) + op.finalize(), np.uint8)


@pytest.mark.parametrize("bits", KEY_BITS)
def test_cipher_matches_openssl_random(oracle, bits):
    # 10^4 seeded (key, block) pairs per key size, 100 keys x 100 blocks.
    for seed in range(100):
        key = synth.key_bytes(1000 + seed, bits)
        data = synth.bytes_np(1000 + seed, synth.STREAM_DATA, 1600)
        ct = oracle.ecb_encrypt(key, bits, data)
        assert np.array_equal(ct, openssl_ecb(key, data)), seed
        assert np.array_equal(oracle.ecb_decrypt(key, bits, ct), data)


@pytest.mark.parametrize("bits", KEY_BITS)
def test_single_block_cipher_matches_openssl(oracle, bits):
    key = synth.key_bytes(5, bits)
    blk = synth.bytes_np(5, synth.STREAM_DATA, 16)
    ct = oracle.cipher_block(key, bits, blk)
    assert np.array_equal(ct, openssl_ecb(key, blk))
    assert np.array_equal(oracle.inv_cipher_block(key, bits, ct), blk)


@pytest.mark.parametrize("bits", KEY_BITS)
@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 31, 255, 4096 + 5])
def test_ctr_matches_openssl(oracle, bits, n):
    key = synth.key_bytes(n, bits)
    iv = synth.iv_bytes(n, counter0=7)
    data = synth.bytes_np(n, synth.STREAM_DATA, n)
    out = oracle.ctr_xcrypt(key, bits, iv, data)
    assert np.array_equal(out, openssl_ctr(key, iv, data))
    assert np.array_equal(oracle.ctr_xcrypt(key, bits, iv, out), data), "CTR is self-inverse"


def counter_blocks(iv, nblocks, first=0):
    c0 = int.from_bytes(bytes(iv[12:16]), "big")
    rows = []
    for j in range(first, first + nblocks):
        rows.append(bytes(iv[:12]) + ((c0 + j) % (1 << 32)).to_bytes(4, "big"))
    return np.frombuffer(b"".join(rows), np.uint8)


@pytest.mark.parametrize("bits", KEY_BITS)
def test_ctr_is_ecb_of_counter_blocks_with_wrap(oracle, bits):
    # SP 800-38A §6.5: O_j = CIPH(T_j); the 32-bit counter wraps without a carry
    # into the nonce (start 2^32 - 16, so the run crosses the wrap).
    key = synth.key_bytes(3, bits)
    iv = synth.iv_bytes(3, counter0=0xFFFFFFF0)
    n = 32 * 16 + 9
    data = synth.bytes_np(3, synth.STREAM_DATA, n)
    ks = oracle.ecb_encrypt(key, bits, counter_blocks(iv, 33))
    expect = data ^ ks[:n]
    assert np.array_equal(oracle.ctr_xcrypt(key, bits, iv, data), expect)
    # the library increments 128 bits, so it must differ after the wrap
    lib = openssl_ctr(key, iv, data)
    assert np.array_equal(lib[: 16 * 16], expect[: 16 * 16])
    assert not np.array_equal(lib[16 * 16:], expect[16 * 16:])


def test_ctr_first_block_and_sampled_blocks(oracle):
    key = synth.key_bytes(9, 128)
    iv = synth.iv_bytes(9, counter0=123456)
    data = synth.bytes_np(9, synth.STREAM_DATA, 16 * 500)
    full = oracle.ctr_xcrypt(key, 128, iv, data)
    part = oracle.ctr_xcrypt(key, 128, iv, data[16 * 77:], first_block=77)
    assert np.array_equal(full[16 * 77:], part)
    idx = np.array([0, 5, 77, 499, 300], np.uint64)
    blocks = data.reshape(-1, 16)[idx.astype(np.int64)]
    got = oracle.ctr_xcrypt_blocks(key, 128, iv, idx, blocks)
    assert np.array_equal(got.reshape(-1, 16), full.reshape(-1, 16)[idx.astype(np.int64)])


# ---------------------------------------------------------------------------
# CBC and XTS
# ---------------------------------------------------------------------------

def openssl_cbc(key, iv, data, decrypt=False):
    c = _openssl()
    ctx = c.Cipher(c.algorithms.AES(bytes(key)), c.modes.CBC(bytes(iv)))
    op = ctx.decryptor() if decrypt else ctx.encryptor()
    return np.frombuffer(op.update(bytes(data)) + op.finalize(), np.uint8)


def openssl_xts(key1, key2, sector_bytes, first_sector, data, decrypt=False):
    c = _openssl()
    out = []
    for u in range(len(data) // sector_bytes):
        tweak = (first_sector + u).to_bytes(16, "little")
        ctx = c.Cipher(c.algorithms.AES(bytes(key1) + bytes(key2)), c.modes.XTS(tweak))
        op = ctx.decryptor() if decrypt else ctx.encryptor()
        out.append(op.update(bytes(data[u * sector_bytes:(u + 1) * sector_bytes])) + op.finalize())
    return np.frombuffer(b"".join(out), np.uint8)


@pytest.mark.parametrize("bits", KEY_BITS)
def test_cbc_matches_openssl_and_ecb(oracle, bits):
    key = synth.key_bytes(61, bits)
    iv = synth.bytes_np(61, synth.STREAM_NONCE, 16)
    data = synth.bytes_np(61, synth.STREAM_DATA, 16 * 333)
    ct = oracle.cbc_encrypt(key, bits, iv, data)
    assert np.array_equal(ct, openssl_cbc(key, iv, data))
    assert np.array_equal(oracle.cbc_decrypt(key, bits, iv, ct), data)
    # P_j = InvCipher(C_j) ^ C_{j-1}: CBC decryption is ECB decryption XOR the shifted ciphertext
    chain = np.concatenate([iv, ct[:-16]])
    assert np.array_equal(oracle.ecb_decrypt(key, bits, ct) ^ chain, data)


@pytest.mark.parametrize("bits", (128, 256))
@pytest.mark.parametrize("sector_bytes,first_sector", [(16, 0), (512, 7), (4096, (1 << 40) + 3)])
def test_xts_matches_openssl(oracle, bits, sector_bytes, first_sector):
    key1 = synth.key_bytes(62, bits)
    key2 = synth.key_bytes(63, bits)
    data = synth.bytes_np(62, synth.STREAM_DATA, 3 * sector_bytes)
    ct = oracle.xts(False, key1, key2, bits, sector_bytes, first_sector, data)
    assert np.array_equal(ct, openssl_xts(key1, key2, sector_bytes, first_sector, data))
    assert np.array_equal(oracle.xts(True, key1, key2, bits, sector_bytes, first_sector, ct), data)


def test_xts_rejects_bad_lengths(oracle):
    k = np.zeros(16, np.uint8)
    with pytest.raises(ValueError):
        oracle.xts(False, k, k, 128, 512, 0, np.zeros(513, np.uint8))
    with pytest.raises(ValueError):
        oracle.xts(False, k, k, 128, 24, 0, np.zeros(48, np.uint8))


# ---------------------------------------------------------------------------
# PKCS#7
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 32, 100])
def test_pkcs7_matches_library(oracle, n):
    padding = pytest.importorskip("cryptography.hazmat.primitives.padding")
    key = synth.key_bytes(n, 192)
    data = synth.bytes_np(n, synth.STREAM_DATA, n)
    assert oracle.pkcs7_padded_len(n) == 16 * (n // 16) + 16
    p = padding.PKCS7(128).padder()
    padded = np.frombuffer(p.update(bytes(data)) + p.finalize(), np.uint8)
    ct = oracle.ecb_pkcs7_encrypt(key, 192, data)
    assert np.array_equal(ct, openssl_ecb(key, padded))
    rc, pt = oracle.ecb_pkcs7_decrypt(key, 192, ct)
    assert rc == 0 and np.array_equal(pt, data)


def test_pkcs7_rejects_bad_padding(oracle):
    key = synth.key_bytes(1, 128)
    for last in (bytes(16), bytes(15) + b"\x11", bytes(14) + b"\x01\x02", bytes(12) + b"\x03\x04\x04\x04"):
        ct = openssl_ecb(key, np.frombuffer(b"A" * 16 + last, np.uint8))
        rc, _ = oracle.ecb_pkcs7_decrypt(key, 128, ct)
        assert rc == oracle_mod.REF_ERR_PADDING, last
    rc, _ = oracle.ecb_pkcs7_decrypt(key, 128, np.zeros(17, np.uint8))
    assert rc == oracle_mod.REF_ERR_LENGTH


# ---------------------------------------------------------------------------
# round trips and the paper's chunked scheme (§IV.B)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bits", KEY_BITS)
def test_round_trip(oracle, bits):
    key = synth.key_bytes(11, bits)
    data = synth.bytes_np(11, synth.STREAM_DATA, 16 * 64)
    assert np.array_equal(oracle.ecb_decrypt(key, bits, oracle.ecb_encrypt(key, bits, data)), data)


@pytest.mark.parametrize("threads", [1, 2, 3, 7, 64])
@pytest.mark.parametrize("n", [0, 16, 16 * 5, 16 * 1000 + 0, 16 * 1001 + 11])
def test_chunked_equals_single_pass(oracle, threads, n):
    key = synth.key_bytes(n, 256)
    iv = synth.iv_bytes(n, counter0=0xFFFFFF00)
    data = synth.bytes_np(n, synth.STREAM_DATA, n)
    assert np.array_equal(oracle.ctr_xcrypt(key, 256, iv, data, nthreads=threads),
                          oracle.ctr_xcrypt(key, 256, iv, data))
    if n % 16 == 0:
        e1 = oracle.ecb_encrypt(key, 256, data, nthreads=threads)
        assert np.array_equal(e1, oracle.ecb_encrypt(key, 256, data))
        assert np.array_equal(oracle.ecb_decrypt(key, 256, e1, nthreads=threads), data)


@pytest.mark.parametrize("threads", [1, 7])
def test_message_list_matches_openssl_per_message(oracle, threads):
    """ref_batch_mt (a list of messages over threads, the batched workloads'
    checker) against OpenSSL message by message: CTR and PKCS#7 + ECB, every
    key size, empty and ragged lengths, then decryption back with the padding
    checked, a corrupted pad and a bad key size reported per message."""
    padding = pytest.importorskip("cryptography.hazmat.primitives.padding")
    n = 60
    lengths = np.array([0, 1, 15, 16, 17, 31, 32, 33] + [int(x) for x in
                       synth.uniform01(3, synth.STREAM_LENGTH, n - 8) * 700], np.uint64)
    kb = np.array([128, 192, 256], np.uint32)[np.arange(n) % 3]
    keys = synth.bytes_np(3, synth.STREAM_KEY, 32 * n).reshape(n, 32)
    ivs = synth.bytes_np(3, synth.STREAM_NONCE, 16 * n).reshape(n, 16).copy()
    ivs[:, 12:] = 0  # OpenSSL carries into the nonce on a wrap; start low
    in_off = np.concatenate([[0], np.cumsum((lengths + np.uint64(15)) // np.uint64(16) * np.uint64(16))[:-1]])
    in_off = in_off.astype(np.uint64)
    total = int(in_off[-1] + lengths[-1] + np.uint64(16))
    data = synth.bytes_np(3, synth.STREAM_DATA, total)
    ct_len = lengths - lengths % np.uint64(16) + np.uint64(16)
    out_off = np.concatenate([[0], np.cumsum(ct_len)[:-1]]).astype(np.uint64)
    out_size = int(ct_len.sum())
    ctr, ctr_len, st = oracle.batch(0, data, in_off, lengths, out_size, out_off, keys, kb, ivs, nthreads=threads)
    assert np.all(st == 0) and np.array_equal(ctr_len, lengths)
    enc, enc_len, st = oracle.batch(1, data, in_off, lengths, out_size, out_off, keys, kb, nthreads=threads)
    assert np.all(st == 0) and np.array_equal(enc_len, ct_len)
    for m in range(n):
        key, ln = keys[m][: kb[m] // 8], int(lengths[m])
        msg = data[int(in_off[m]): int(in_off[m]) + ln]
        o = int(out_off[m])
        assert np.array_equal(ctr[o: o + ln], openssl_ctr(key, ivs[m], msg)), m
        p = padding.PKCS7(128).padder()
        padded = p.update(bytes(msg)) + p.finalize()
        assert np.array_equal(enc[o: o + int(ct_len[m])], openssl_ecb(key, padded)), m
    enc[int(out_off[5]) + int(ct_len[5]) - 1] ^= 0x5A  # corrupt message 5's last ciphertext byte
    kb2 = kb.copy()
    kb2[7] = 100
    dec, dec_len, st = oracle.batch(2, enc, out_off, ct_len, out_size, out_off, keys, kb2, nthreads=threads)
    for m in range(n):
        if m == 7:
            assert st[m] == -1 and dec_len[m] == 0   # REF_ERR_KEYSIZE
        elif m == 5:
            assert st[m] == -3 and dec_len[m] == 0   # REF_ERR_PADDING (a random last block passes ~2^-8 of the time; this seeded one fails)
        else:
            o, ln = int(out_off[m]), int(lengths[m])
            assert st[m] == 0 and dec_len[m] == ln
            assert np.array_equal(dec[o: o + ln], data[int(in_off[m]): int(in_off[m]) + ln]), m


def test_ecb_length_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.ecb_encrypt(np.zeros(16, np.uint8), 128, np.zeros(17, np.uint8))


# ---------------------------------------------------------------------------
# planted mistakes: each mutant of the oracle must fail the battery
# ---------------------------------------------------------------------------

MUTANTS = {
    "gf_poly": ("if (v & 0x100u) v ^= 0x11Bu;", "if (v & 0x100u) v ^= 0x11Du;"),
    "affine_const": ("^ rotl8(b, 4) ^ 0x63u", "^ rotl8(b, 4) ^ 0x62u"),
    "affine_term": ("^ rotl8(b, 3) ^ rotl8(b, 4)", "^ rotl8(b, 4)"),
    "inverse_exp": ("unsigned e = 254;", "unsigned e = 253;"),
    "mix_row": ("{2, 3, 1, 1}, {1, 2, 3, 1}", "{2, 3, 1, 1}, {1, 3, 2, 1}"),
    "shift_dir": ("row[c] = s[r][(c + r) % 4];", "row[c] = s[r][(c + 4 - r) % 4];"),
    "rcon": ("uint8_t rcon = 1;", "uint8_t rcon = 2;"),
    "rotword": ("t[0] = t[1]; t[1] = t[2]; t[2] = t[3]; t[3] = a0;",
                "t[0] = t[3]; t[3] = t[2]; t[2] = t[1]; t[1] = a0;"),
    "nk8_subword": ("} else if (nk > 6 && i % nk == 4) {", "} else if (nk > 8 && i % nk == 4) {"),
    "round_count": ("for (int round = 1; round < nr; ++round) {",
                    "for (int round = 1; round < nr - 1; ++round) {"),
    "state_transpose": ("s[r][c] = in[r + 4 * c];", "s[r][c] = in[c + 4 * r];"),
    "ark_index": ("s[r][c] ^= w[16 * round + 4 * c + r];", "s[r][c] ^= w[16 * round + 4 * r + c];"),
    "ctr_endian": ("t[12] = (uint8_t)(c >> 24);\n    t[13] = (uint8_t)(c >> 16);\n"
                   "    t[14] = (uint8_t)(c >> 8);\n    t[15] = (uint8_t)c;",
                   "t[15] = (uint8_t)(c >> 24);\n    t[14] = (uint8_t)(c >> 16);\n"
                   "    t[13] = (uint8_t)(c >> 8);\n    t[12] = (uint8_t)c;"),
    "ctr_carry": ("memcpy(t, iv, 12);", "memcpy(t, iv, 12);\n    if ((uint64_t)c0 + j > 0xFFFFFFFFu) t[11]++;"),
    "inv_mix_coef": ("{14, 11, 13, 9}, {9, 14, 11, 13}", "{14, 11, 13, 9}, {9, 14, 13, 11}"),
    "pkcs7_check": ("if (out[k] != p) return REF_ERR_PADDING;", "if (out[k] != p) break;"),
    "chunk_offset": ("first_block + b0, in + 16 * b0", "first_block, in + 16 * b0"),
    "cbc_chain": ("        memcpy(prev, cur, 16);", "        memcpy(prev, out + off, 16);"),
    "xts_poly": ("if (carry) t[0] ^= 0x87u;", "if (carry) t[0] ^= 0x86u;"),
    "xts_tweak_order": ("tv[i] = (uint8_t)(sector >> (8 * i));", "tv[15 - i] = (uint8_t)(sector >> (8 * i));"),
}


def battery(o: Oracle) -> list:
    """A quick subset of the pins above; returns the names of the ones that fail."""
    fails = []

    def check(name, fn):
        try:
            if not fn():
                fails.append(name)
        except Exception:  # a crash or a refused call also counts as caught
            fails.append(name)

    s = o.sbox()
    check("sbox_bijective", lambda: sorted(s.tolist()) == list(range(256)))
    check("sbox_def", lambda: all(s[x] == affine_bitwise(
        0 if x == 0 else next(b for b in range(1, 256) if gmul(x, b) == 1)) for x in range(0, 256, 5)))
    check("gf", lambda: all(o.gf_mul(a, b) == gmul(a, b) for a in range(0, 256, 7) for b in range(0, 256, 11)))
    col = [0x12, 0x9A, 0x33, 0xF0]
    check("mix", lambda: o.mix_column(col).tolist() == poly4_mul(col, [2, 1, 1, 3]))
    check("invmix", lambda: o.inv_mix_column(col).tolist() == poly4_mul(col, [0x0E, 0x09, 0x0D, 0x0B]))
    for bits in KEY_BITS:
        key = synth.key_bytes(42, bits)
        data = synth.bytes_np(42, synth.STREAM_DATA, 16 * 8)
        check(f"ecb{bits}", lambda: np.array_equal(o.ecb_encrypt(key, bits, data), openssl_ecb(key, data)))
        check(f"dec{bits}", lambda: np.array_equal(o.ecb_decrypt(key, bits, openssl_ecb(key, data)), data))
    key = synth.key_bytes(43, 128)
    iv = synth.iv_bytes(43, counter0=0xFFFFFFFE)
    data = synth.bytes_np(43, synth.STREAM_DATA, 16 * 4 + 3)
    exp = data ^ openssl_ecb(key, counter_blocks(iv, 5))[: data.size]
    check("ctr_wrap", lambda: np.array_equal(o.ctr_xcrypt(key, 128, iv, data), exp))
    big = synth.bytes_np(44, synth.STREAM_DATA, 16 * 40 + 5)
    check("chunked", lambda: np.array_equal(o.ctr_xcrypt(key, 128, iv, big, nthreads=3),
                                            o.ctr_xcrypt(key, 128, iv, big)))
    bad = openssl_ecb(key, np.frombuffer(b"B" * 16 + bytes(14) + b"\x02\x03", np.uint8))
    check("pkcs7_reject", lambda: o.ecb_pkcs7_decrypt(key, 128, bad)[0] != 0)
    civ = synth.bytes_np(45, synth.STREAM_NONCE, 16)
    cdat = synth.bytes_np(45, synth.STREAM_DATA, 16 * 6)
    check("cbc", lambda: np.array_equal(o.cbc_decrypt(key, 128, civ, openssl_cbc(key, civ, cdat)), cdat))
    k2 = synth.key_bytes(46, 128)
    xdat = synth.bytes_np(46, synth.STREAM_DATA, 16 * 24)
    check("xts", lambda: np.array_equal(o.xts(False, key, k2, 128, 16 * 12, 5, xdat),
                                        openssl_xts(key, k2, 16 * 12, 5, xdat)))
    return fails


def test_battery_passes_on_the_oracle(oracle):
    _openssl()
    assert battery(oracle) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    _openssl()
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    old, new = MUTANTS[name]
    src = open(os.path.join(oracle_mod.HERE, "aes_ref.c")).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique in aes_ref.c"
    with tempfile.TemporaryDirectory() as d:
        with open(os.path.join(d, "aes_ref.c"), "w") as f:
            f.write(src.replace(old, new))
        shutil.copy(os.path.join(oracle_mod.HERE, "aes_ref.h"), d)
        lib_path = os.path.join(d, "libmut.so")
        try:
            oracle_mod.build(force=True, src_dir=d, out_path=lib_path, extra_flags=("-w",))
        except subprocess.CalledProcessError:
            return  # a mutant that does not compile is caught trivially
        fails = battery(Oracle(oracle_mod.load(lib_path)))
    assert fails, f"mutant {name} slipped through every pin"
