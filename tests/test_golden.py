"""The golden fixtures (tests/golden/): the oracle-written vectors are still
what the oracle computes and what OpenSSL computes; the paper's Table I is
transcribed consistently and the bench quotes it correctly."""
import numpy as np
import pytest

from tests.golden_util import aes_vectors, paper_table1


def test_oracle_reproduces_vectors(oracle):
    vs = aes_vectors()
    assert len(vs) >= 40
    for v in vs:
        m, b, k, iv, d = v["mode"], v["bits"], v["key"], v["iv"], v["data"]
        if m == "ecb_enc":
            got = oracle.ecb_encrypt(k, b, d)
        elif m == "ctr":
            got = oracle.ctr_xcrypt(k, b, iv, d)
        elif m == "cbc_dec":
            got = oracle.cbc_decrypt(k, b, iv, d)
        elif m == "ecb_pkcs7_enc":
            got = oracle.ecb_pkcs7_encrypt(k, b, d)
        else:
            half = k.size // 2
            got = oracle.xts(False, k[:half], k[half:], b, 512, int.from_bytes(bytes(iv), "little"), d)
        assert np.array_equal(got, v["out"]), m


def test_openssl_reproduces_vectors():
    c = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    padding = pytest.importorskip("cryptography.hazmat.primitives.padding")

    def run(mode, key, data, decrypt=False):
        ctx = c.Cipher(c.algorithms.AES(bytes(key)), mode)
        op = ctx.decryptor() if decrypt else ctx.encryptor()
        return np.frombuffer(op.update(bytes(data)) + op.finalize(), np.uint8)

    for v in aes_vectors():
        m, k, iv, d = v["mode"], v["key"], v["iv"], v["data"]
        if m == "ecb_enc":
            got = run(c.modes.ECB(), k, d)
        elif m == "ctr":
            if int.from_bytes(bytes(iv[12:]), "big") + (d.size + 15) // 16 > 1 << 32:
                continue  # OpenSSL carries into the nonce; the wrap is pinned against ECB instead
            got = run(c.modes.CTR(bytes(iv)), k, d)
        elif m == "cbc_dec":
            got = run(c.modes.CBC(bytes(iv)), k, d, decrypt=True)
        elif m == "ecb_pkcs7_enc":
            p = padding.PKCS7(128).padder()
            got = run(c.modes.ECB(), k, np.frombuffer(p.update(bytes(d)) + p.finalize(), np.uint8))
        else:
            assert v["bits"] in (128, 256)  # the XTS-AES key sizes (IEEE 1619)
            first = int.from_bytes(bytes(iv), "little")
            got = np.concatenate([run(c.modes.XTS((first + u).to_bytes(16, "little")), k, d[512 * u: 512 * (u + 1)])
                                  for u in range(d.size // 512)])
        assert np.array_equal(got, v["out"]), m


def test_paper_table1_is_consistent_and_quoted():
    rows = paper_table1()
    cores = {"core2duo": 2, "corei3": 2, "xeon_x7560_32core": 32}
    assert len(rows) == 6
    for method, proc, best, per_core in rows:
        assert abs(best / cores[proc] - per_core) <= 1, (method, proc)  # the per-core column (§VI)
    best = max(r[2] for r in rows)
    assert best == 6637 and [r for r in rows if r[2] == best][0][:2] == ("pthread", "xeon_x7560_32core")
    import bench

    assert abs(bench.PAPER_BEST_GBPS - best * 1e6 / 8 / 1e9) < 1e-12
