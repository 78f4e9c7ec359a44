"""Host-side checks of libaesgpu.so that need no GPU.

* the library builds for sm_103a, loads, and exports every entry point that
  include/*.h declares;
* host key expansion equals the oracle's (FIPS-197 §5.2), and the decryption
  schedule is the equivalent inverse cipher's (§5.3.5);
* argument validation that happens before any CUDA call returns the
  documented status codes.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synth
from paper_1403_7295_gb300 import aes as A
from paper_1403_7295_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return A.lib()


def declared_entry_points(header="aesgpu.h"):
    names = set()
    for h in [os.path.join(ROOT, "include", header)]:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(aes\w*)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    headers = sorted(os.path.basename(h) for h in glob.glob(os.path.join(ROOT, "include", "*.h")))
    assert headers == ["aesgpu.h", "aesgpu_probe.h"]
    names = declared_entry_points("aesgpu.h")
    assert "aes_ctr_xcrypt" in names and "aes_expand_key" in names
    for n in names:
        assert hasattr(lib, n), f"libaesgpu.so does not export {n}"
    probe = ctypes.CDLL(B.PROBE_LIB_PATH)
    pnames = declared_entry_points("aesgpu_probe.h")
    assert "aesgpu_probe_pipe" in pnames
    for n in pnames:
        assert hasattr(probe, n), f"libaesgpu_probe.so does not export {n}"


def test_build_targets_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.ARCH)
    assert os.path.dirname(B.LIB_PATH).startswith(ROOT), "the library is built in-tree"


@pytest.mark.parametrize("bits", [128, 192, 256])
def test_expand_key_matches_oracle(lib, oracle, bits):
    for seed in range(10):
        key = synth.key_bytes(100 + seed, bits)
        ks = A.aes_expand_key(key, bits)
        w, nr = oracle.key_expansion(key, bits)
        assert ks.nr == nr and ks.key_bits == bits
        nwords = 4 * (nr + 1)
        enc = np.array(ks.rk_enc[:nwords], dtype="<u4").view(np.uint8)
        assert np.array_equal(enc, w)
        assert all(v == 0 for v in ks.rk_enc[nwords:])
        # equivalent inverse cipher: round r uses InvMixColumns(round key nr - r)
        dec = np.array(ks.rk_dec[:nwords], dtype="<u4").view(np.uint8).reshape(nr + 1, 4, 4)
        rounds = w.reshape(nr + 1, 4, 4)
        for r in range(nr + 1):
            src = rounds[nr - r]
            want = src if r in (0, nr) else np.stack([oracle.inv_mix_column(c) for c in src])
            assert np.array_equal(dec[r], want), (seed, r)


def test_expand_key_rejects_bad_sizes(lib):
    for bits in (0, 64, 129, 512):
        with pytest.raises(A.AesError) as e:
            A.aes_expand_key(np.zeros(64, np.uint8), bits)
        assert e.value.status == 2
    ks = A.KeySchedule()
    assert lib.aes_expand_key(None, 128, ctypes.byref(ks)) == 1


def _call(lib, fn, ks, inp, out, n, iv=None, cfg=None):
    if fn == "ctr":
        ivb = (ctypes.c_uint8 * 16)() if iv is None else iv
        return lib.aes_ctr_xcrypt_ex(ctypes.byref(ks) if ks is not None else None, ivb, inp, out, n,
                                     None, cfg)
    f = lib.aes_ecb_encrypt_ex if fn == "enc" else lib.aes_ecb_decrypt_ex
    return f(ctypes.byref(ks) if ks is not None else None, inp, out, n, None, cfg)


def test_validation_before_any_cuda_call(lib):
    ks = A.aes_expand_key(synth.key_bytes(0, 128))
    base = 1 << 20  # never dereferenced: every case below fails validation first
    for fn in ("enc", "dec", "ctr"):
        assert _call(lib, fn, None, base, base, 16) == 1            # null schedule
        bad = A.KeySchedule()
        ctypes.memmove(ctypes.byref(bad), ctypes.byref(ks), ctypes.sizeof(ks))
        bad.nr = 11
        assert _call(lib, fn, bad, base, base, 16) == 2             # inconsistent schedule
        assert _call(lib, fn, ks, 0, base, 16) == 1                 # null input
        assert _call(lib, fn, ks, base + 8, base + 4096, 32) == 4   # misaligned
        assert _call(lib, fn, ks, base, base + 16, 64) == 5         # partial overlap
        assert _call(lib, fn, ks, base, base + 16, 0) == 0          # empty is a no-op
        cfg = A.LaunchConfig(variant=7)
        assert _call(lib, fn, ks, base, base + 4096, 16, cfg=ctypes.byref(cfg)) == 1
    assert _call(lib, "enc", ks, base, base + 4096, 17) == 3        # ECB needs whole blocks
    assert _call(lib, "dec", ks, base, base + 4096, 8) == 3
    assert lib.aes_ctr_xcrypt(ctypes.byref(ks), None, base, base, 16, None) == 1  # null IV


def test_status_strings(lib):
    for s in range(12):
        assert lib.aes_status_string(s)
    assert lib.aes_status_string(99) == b"unknown status"


def test_cbc_and_xts_validation(lib):
    ks = A.aes_expand_key(synth.key_bytes(0, 128))
    kr = ctypes.byref(ks)
    ivb = (ctypes.c_uint8 * 16)()
    base = 1 << 20
    assert lib.aes_cbc_decrypt(kr, ivb, base, base, 64, None) == 5           # in place refused
    assert lib.aes_cbc_decrypt(kr, ivb, base, base + 4096, 17, None) == 3    # whole blocks only
    assert lib.aes_cbc_decrypt(kr, None, base, base + 4096, 16, None) == 1   # IV required
    assert lib.aes_cbc_decrypt(kr, ivb, base, base + 4096, 0, None) == 0
    for fn in (lib.aes_xts_encrypt, lib.aes_xts_decrypt):
        assert fn(kr, kr, 0, 496, base, base, 496, None) == 3                # unit not a multiple of 512
        assert fn(kr, kr, 0, 512, base, base, 1000, None) == 3               # not whole units
        assert fn(kr, None, 0, 512, base, base, 512, None) == 1
        assert fn(kr, kr, 0, 512, base + 8, base + 8, 512, None) == 4        # misaligned
        assert fn(kr, kr, 0, 512, base, base, 0, None) == 0


def test_file_crypt_validation_and_empty_file(lib, tmp_path):
    """aes_file_crypt: argument checks, a missing source (AES_ERR_IO with
    errno), a ragged ECB file (AES_ERR_LENGTH before dst is created), and an
    empty file (done without a GPU: dst created empty)."""
    import errno

    from paper_1403_7295_gb300 import filecrypt as F

    L = F._declare()
    ks = A.aes_expand_key(synth.key_bytes(0, 128))
    kr = ctypes.byref(ks)
    ivb = ctypes.create_string_buffer(16)
    src, dst = tmp_path / "src", tmp_path / "dst"
    src.write_bytes(b"")
    s, d = os.fsencode(src), os.fsencode(dst)
    st = F.FileStats()
    assert L.aes_file_crypt(None, d, 0, kr, ivb, None, None) == 1
    assert L.aes_file_crypt(s, d, 3, kr, ivb, None, None) == 1                     # unknown mode
    assert L.aes_file_crypt(s, d, 0, kr, None, None, None) == 1                    # CTR without IV
    assert L.aes_file_crypt(s, d, 0, None, ivb, None, None) == 1                   # no key
    for cfg in (F.FileConfig(17, 0, 0), F.FileConfig(0, 65, 0), F.FileConfig(0, -1, 0), F.FileConfig(0, 0, 4),
                F.FileConfig(0, 0, F.STAGED | F.DIRECT)):
        assert L.aes_file_crypt(s, d, 0, kr, ivb, ctypes.byref(cfg), None) == 1
    missing = os.fsencode(tmp_path / "missing")
    assert L.aes_file_crypt(missing, d, 0, kr, ivb, None, ctypes.byref(st)) == 11
    assert st.os_errno == errno.ENOENT
    src.write_bytes(b"x" * 33)
    assert L.aes_file_crypt(s, d, 1, kr, None, None, None) == 3                    # ECB of 33 bytes
    assert not dst.exists()
    src.write_bytes(b"")
    assert L.aes_file_crypt(s, d, 0, kr, ivb, None, ctypes.byref(st)) == 0
    assert dst.exists() and dst.stat().st_size == 0 and st.bytes == 0 and st.chunks == 0 and st.direct == 0
    for flag in (F.STAGED, F.DIRECT):  # the known flags, one at a time: accepted
        cfg = F.FileConfig(0, 0, flag)
        assert L.aes_file_crypt(s, d, 0, kr, ivb, ctypes.byref(cfg), None) == 0
    L.aes_file_trim()  # nothing pinned yet: a no-op without a GPU


def test_server_validation_without_a_gpu(lib):
    """aes_server_*: argument checks that fail before any CUDA call, and the
    null-handle behaviour of the query calls."""
    from paper_1403_7295_gb300 import serve as S

    L = S._declare()
    ks = A.aes_expand_key(synth.key_bytes(0, 128))
    nonces = (ctypes.c_uint8 * 12)()
    h = ctypes.c_void_p()
    base = 1 << 20  # never dereferenced
    assert L.aes_server_create(None, base, 4096, ctypes.byref(ks), nonces, 0, ctypes.byref(h)) == 1  # no tenants
    assert L.aes_server_create(None, None, 4096, ctypes.byref(ks), nonces, 1, ctypes.byref(h)) == 1  # no pool
    assert L.aes_server_create(None, base, 4096, None, nonces, 1, ctypes.byref(h)) == 1             # no schedules
    cfg = S.ServerConfig(1 << 20, 65, 2, 16, 0, 1.0, 0)                                          # too many streams
    assert L.aes_server_create(ctypes.byref(cfg), base, 4096, ctypes.byref(ks), nonces, 1, ctypes.byref(h)) == 1
    assert L.aes_server_submit(None, 0, 0, 0, 16) == 1
    st = ctypes.c_int(0)
    assert L.aes_server_progress(None, None, 0, ctypes.byref(st)) == 0 and st.value == 1
    assert L.aes_server_healthy(None) == 0 and L.aes_server_idle(None) == 0
    assert L.aes_server_output(None) is None
    L.aes_server_destroy(None)


def test_ctr_iv_advance_is_the_counter_block_function(lib):
    """aes_ctr_iv_advance: SP 800-38A §6.5 counter blocks, the 32-bit
    big-endian counter in bytes 12..15 advanced modulo 2^32, the nonce bytes
    untouched (written out here from the definition), in place too."""
    rng = np.random.default_rng(1403)
    cases = [(bytes(12) + b"\xff\xff\xff\xff", 1), (bytes(range(16)), 0), (b"\xaa" * 12 + b"\xff\xff\xff\xf0", 17),
             (bytes(16), (1 << 32) + 5), (bytes(16), (1 << 64) - 1)]
    cases += [(rng.integers(0, 256, 16, dtype=np.uint8).tobytes(), int(rng.integers(0, 1 << 62))) for _ in range(200)]
    for iv, b in cases:
        c0 = int.from_bytes(iv[12:], "big")
        want = iv[:12] + ((c0 + b) % (1 << 32)).to_bytes(4, "big")
        assert A.aes_ctr_iv_advance(iv, b) == want, (iv.hex(), b)
        buf = (ctypes.c_uint8 * 16).from_buffer_copy(iv)
        assert lib.aes_ctr_iv_advance(buf, b, buf) == 0  # the same array in and out
        assert bytes(buf) == want
    out = (ctypes.c_uint8 * 16)()
    assert lib.aes_ctr_iv_advance(None, 1, out) == 1
    assert lib.aes_ctr_iv_advance(out, 1, None) == 1


def test_xts_key_sizes_refused_before_any_gpu_work(lib):
    """XTS is defined for AES-128 and AES-256 key pairs (IEEE 1619); a 192-bit
    or mixed pair is refused on the host (the pointers are never touched)."""
    ks = {b: A.aes_expand_key(synth.key_bytes(3, b)) for b in (128, 192, 256)}
    p = 1 << 20  # never dereferenced
    for d, t in ((192, 192), (128, 256), (256, 128), (192, 128), (128, 192)):
        for fn in (lib.aes_xts_encrypt, lib.aes_xts_decrypt):
            assert fn(ctypes.byref(ks[d]), ctypes.byref(ks[t]), 0, 512, p, p, 4096, None) == 2


def test_batch_workspace_layout_and_short_path_refusals(lib):
    """aes_batch_workspace_size is the sum of its parts, each rounded up to
    256 bytes: block offsets (n + 1 words), chunk totals (one per 4096
    messages), the work counters, the lane path's bin counts and cursors
    (2 x 1536 + 1 words), its bins (n halfwords) and order (n + 96 words); the
    allocation-free call's scratch is that size at its cap of 65,536
    messages.  A short_path outside AES_BATCH_SHORT_*, or the lane path for
    an ECB batch, is refused before any CUDA call."""
    from paper_1403_7295_gb300 import batch as BT

    L = BT._declare()
    up = lambda x: (x + 255) // 256 * 256  # noqa: E731
    for n in (1, 4095, 4096, 4097, 65536, 1_000_000):
        want = (up(8 * (n + 1)) + up(8 * -(-n // 4096)) + 256 + up(8 * 1536 + 4) + up(2 * n)
                + up(4 * (n + 96)))
        assert L.aes_batch_workspace_size(n) == want, n
    assert L.aes_batch_workspace_size(65536) == 931_328
    base = 1 << 20  # never dereferenced: every case below fails validation first
    d = BT.AesBatch()
    d.n_msgs, d.in_, d.out = 4, base, base + (1 << 16)
    d.in_off, d.in_len, d.out_off = base + 4096, base + 8192, base + 12288
    d.keys, d.key_bits, d.iv = base + 16384, base + 20480, base + 24576
    ws = base + (1 << 17)
    for op, path in ((BT.BATCH_CTR, 3), (BT.BATCH_CTR, -1), (BT.BATCH_ECB_PKCS7_ENCRYPT, BT.SHORT_LANES),
                     (BT.BATCH_ECB_PKCS7_DECRYPT, BT.SHORT_LANES)):
        d.op = op
        cfg = BT.AesBatchConfig(1024, 0, 152, path)
        assert L.aes_batch_submit_ex(ctypes.byref(d), ws, 1 << 30, None, ctypes.byref(cfg)) == 1, (op, path)
