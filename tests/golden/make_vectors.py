#!/usr/bin/env python3
"""Write tests/golden/aes_vectors.txt from the CPU oracle only.

Seeded keys, IVs and data (synth) through every mode the library offers:
ECB encrypt, CTR (with a counter wrap), CBC decrypt (ciphertext from the
oracle's CBC encrypt), XTS encrypt (512-byte units), PKCS#7 ECB, for all key
sizes.  The CPU tests check that the oracle still reproduces the file and
that OpenSSL agrees; the GPU tests check the GPU against it.

    python tests/golden/make_vectors.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import Oracle  # noqa: E402


def vectors():
    o = Oracle()
    rows = []
    for bits in (128, 192, 256):
        for n in (16, 48, 1024):
            seed = bits * 1000 + n
            key = synth.key_bytes(seed, bits)
            data = synth.bytes_np(seed, synth.STREAM_DATA, n)
            rows.append(("ecb_enc", bits, key, b"", data, o.ecb_encrypt(key, bits, data)))
            iv = synth.iv_bytes(seed, counter0=0xFFFFFFFE)
            rows.append(("ctr", bits, key, iv, data, o.ctr_xcrypt(key, bits, iv, data)))
            civ = synth.bytes_np(seed, synth.STREAM_NONCE, 16)
            ct = o.cbc_encrypt(key, bits, civ, data)
            rows.append(("cbc_dec", bits, key, civ, ct, o.cbc_decrypt(key, bits, civ, ct)))
        for n in (5, 33):
            seed = bits * 1000 + n
            key = synth.key_bytes(seed, bits)
            data = synth.bytes_np(seed, synth.STREAM_DATA, n)
            iv = synth.iv_bytes(seed, counter0=3)
            rows.append(("ctr", bits, key, iv, data, o.ctr_xcrypt(key, bits, iv, data)))
            rows.append(("ecb_pkcs7_enc", bits, key, b"", data, o.ecb_pkcs7_encrypt(key, bits, data)))
        if bits == 192:
            continue  # XTS is defined for AES-128 and AES-256 key pairs only (IEEE 1619)
        key1 = synth.key_bytes(bits + 7, bits)
        key2 = synth.key_bytes(bits + 8, bits)
        data = synth.bytes_np(bits + 7, synth.STREAM_DATA, 1024)
        # XTS: key is key1 || key2, iv field = first sector (8-byte little-endian), units of 512 bytes
        first = 7
        rows.append(("xts_enc_512", bits, bytes(key1) + bytes(key2), first.to_bytes(8, "little"), data,
                     o.xts(False, key1, key2, bits, 512, first, data)))
    return rows


def main():
    path = os.path.join(HERE, "aes_vectors.txt")
    with open(path, "w") as f:
        f.write("# Written by tests/golden/make_vectors.py from the CPU oracle (oracle/aes_ref.c).\n")
        f.write("# mode bits key_hex iv_hex input_hex output_hex   ('-' = empty field)\n")
        for mode, bits, key, iv, data, out in vectors():
            f.write(" ".join([mode, str(bits), bytes(key).hex(), bytes(iv).hex() or "-",
                              bytes(data).hex() or "-", bytes(out).hex() or "-"]) + "\n")
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
