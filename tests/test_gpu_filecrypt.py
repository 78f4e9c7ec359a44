"""File encryption pipeline: file in, encrypted file out, byte-identical to
one library call on the whole buffer (and to the oracle), across several
chunks with a ragged end, for CTR and ECB, and back again."""
import os
import tempfile

import numpy as np
import pytest

import synth
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def test_ctr_file_round_trip(torch, oracle):
    from paper_1403_7295_gb300 import aes as A
    from paper_1403_7295_gb300.filecrypt import crypt_file

    n = (24 << 20) + 5
    data = synth.bytes_np(71, synth.STREAM_DATA, n)
    key = synth.key_bytes(71, 192)
    iv = bytes(synth.iv_bytes(71, counter0=0xFFFFF000))  # the counter wraps inside the file
    with tempfile.TemporaryDirectory() as d:
        src, enc, dec = (os.path.join(d, f) for f in ("p", "c", "q"))
        data.tofile(src)
        r = crypt_file(src, enc, key, "ctr", iv, chunk_bytes=4 << 20, depth=3)
        assert r["bytes"] == n
        got = np.fromfile(enc, np.uint8)
        whole = A.aes_ctr_xcrypt(A.aes_expand_key(key), iv, torch.from_numpy(data).cuda()).cpu().numpy()
        assert np.array_equal(got, whole)
        assert np.array_equal(got[: 1 << 20], oracle.ctr_xcrypt(key, 192, np.frombuffer(iv, np.uint8), data[: 1 << 20]))
        crypt_file(enc, dec, key, "ctr", iv, chunk_bytes=8 << 20, depth=2)
        assert np.array_equal(np.fromfile(dec, np.uint8), data)


def test_ecb_file_round_trip(torch, oracle):
    from paper_1403_7295_gb300.filecrypt import crypt_file

    n = 12 << 20
    data = synth.bytes_np(72, synth.STREAM_DATA, n)
    key = synth.key_bytes(72, 128)
    with tempfile.TemporaryDirectory() as d:
        src, enc, dec = (os.path.join(d, f) for f in ("p", "c", "q"))
        data.tofile(src)
        crypt_file(src, enc, key, "ecb-enc", chunk_bytes=5 << 20)
        got = np.fromfile(enc, np.uint8)
        assert np.array_equal(got[: 1 << 16], oracle.ecb_encrypt(key, 128, data[: 1 << 16]))
        crypt_file(enc, dec, key, "ecb-dec", chunk_bytes=3 << 20)
        assert np.array_equal(np.fromfile(dec, np.uint8), data)
        open(src, "ab").write(b"x")
        with pytest.raises(ValueError):
            crypt_file(src, enc, key, "ecb-enc")
