"""File encryption pipeline (aes_file_crypt): file in, encrypted file out,
byte-identical to one library call on the whole buffer and to the oracle,
across many chunks with a ragged end, for CTR and ECB, any number of worker
threads, in place on the same file, and back again; on both paths (staged
through pinned buffers, the default, or, opted in, files mapped and
processed by the kernel directly)."""
import os
import tempfile

import numpy as np
import pytest

import synth
from tests.gpu_util import pageable_memory_access, require_cuda

pytestmark = pytest.mark.gpu
PATHS = pytest.mark.parametrize("direct", [True, False], ids=["direct", "staged"])


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@PATHS
def test_ctr_file_round_trip(torch, oracle, direct):
    from paper_1403_7295_gb300 import aes as A
    from paper_1403_7295_gb300.filecrypt import crypt_file

    n = (24 << 20) + 5
    data = synth.bytes_np(71, synth.STREAM_DATA, n)
    key = synth.key_bytes(71, 192)
    iv = bytes(synth.iv_bytes(71, counter0=0xFFFFF000))  # the counter wraps inside the file
    with tempfile.TemporaryDirectory() as d:
        src, enc, dec = (os.path.join(d, f) for f in ("p", "c", "q"))
        data.tofile(src)
        r = crypt_file(src, enc, key, "ctr", iv, chunk_bytes=4 << 20, threads=3, direct=direct)
        assert r["bytes"] == n and r["chunks"] == 7 and r["threads"] == 3
        assert r["direct"] == (direct and bool(pageable_memory_access()))
        got = np.fromfile(enc, np.uint8)
        whole = A.aes_ctr_xcrypt(A.aes_expand_key(key), iv, torch.from_numpy(data).cuda()).cpu().numpy()
        assert np.array_equal(got, whole)
        assert np.array_equal(got[: 1 << 20], oracle.ctr_xcrypt(key, 192, np.frombuffer(iv, np.uint8), data[: 1 << 20]))
        crypt_file(enc, dec, key, "ctr", iv, chunk_bytes=8 << 20, threads=2, direct=direct)
        assert np.array_equal(np.fromfile(dec, np.uint8), data)


@PATHS
@pytest.mark.parametrize("n", [1, 15, 16, 17, 1000, 4096 + 3, (1 << 16) + 48])
def test_ctr_small_files_tiny_chunks(torch, oracle, n, direct):
    """Files shorter than a block and chunks of one block: every chunk is its
    own launch with its own advanced IV."""
    from paper_1403_7295_gb300.filecrypt import crypt_file

    data = synth.bytes_np(73 + n, synth.STREAM_DATA, n)
    key = synth.key_bytes(73, 256)
    iv = synth.iv_bytes(73, counter0=0xFFFFFFFE)
    want = oracle.ctr_xcrypt(key, 256, iv, data)
    with tempfile.TemporaryDirectory() as d:
        src, enc = os.path.join(d, "p"), os.path.join(d, "c")
        data.tofile(src)
        for chunk, threads in ((16, 8), (64, 1), (1 << 20, 0), (4096 + 16, 5)):
            crypt_file(src, enc, key, "ctr", bytes(iv), chunk_bytes=chunk, threads=threads, direct=direct)
            assert np.array_equal(np.fromfile(enc, np.uint8), want), (chunk, threads)


@PATHS
def test_ctr_in_place_same_file(torch, oracle, direct):
    from paper_1403_7295_gb300.filecrypt import crypt_file, trim

    n = (3 << 20) + 77
    data = synth.bytes_np(74, synth.STREAM_DATA, n)
    key = synth.key_bytes(74, 128)
    iv = synth.iv_bytes(74)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "f")
        data.tofile(path)
        crypt_file(path, path, key, "ctr", bytes(iv), chunk_bytes=1 << 20, threads=4, direct=direct)
        assert os.path.getsize(path) == n
        assert np.array_equal(np.fromfile(path, np.uint8), oracle.ctr_xcrypt(key, 128, iv, data))
        trim()  # the next call pins fresh buffers
        crypt_file(path, path, key, "ctr", bytes(iv), chunk_bytes=(1 << 18) + 16, threads=7, direct=direct)
        assert np.array_equal(np.fromfile(path, np.uint8), data)


@PATHS
def test_ecb_file_round_trip(torch, oracle, direct):
    from paper_1403_7295_gb300.filecrypt import crypt_file

    n = 12 << 20
    data = synth.bytes_np(72, synth.STREAM_DATA, n)
    key = synth.key_bytes(72, 128)
    with tempfile.TemporaryDirectory() as d:
        src, enc, dec = (os.path.join(d, f) for f in ("p", "c", "q"))
        data.tofile(src)
        crypt_file(src, enc, key, "ecb-enc", chunk_bytes=5 << 20, direct=direct)
        got = np.fromfile(enc, np.uint8)
        assert np.array_equal(got[: 1 << 16], oracle.ecb_encrypt(key, 128, data[: 1 << 16]))
        assert np.array_equal(got[-(1 << 16):], oracle.ecb_encrypt(key, 128, data[-(1 << 16):]))
        crypt_file(enc, dec, key, "ecb-dec", chunk_bytes=3 << 20, threads=5, direct=direct)
        assert np.array_equal(np.fromfile(dec, np.uint8), data)
        open(src, "ab").write(b"x")
        with pytest.raises(ValueError):
            crypt_file(src, enc, key, "ecb-enc")


@PATHS
def test_existing_longer_destination_is_replaced(torch, oracle, direct):
    """dst already holds other, longer content: afterwards it has exactly the
    source length and the cipher bytes (nothing stale past the end, nothing
    stale inside), on both paths."""
    from paper_1403_7295_gb300.filecrypt import crypt_file

    n = (5 << 20) + 333
    data = synth.bytes_np(75, synth.STREAM_DATA, n)
    key = synth.key_bytes(75, 256)
    iv = synth.iv_bytes(75, counter0=0x7FFFFFF0)
    with tempfile.TemporaryDirectory() as d:
        src, enc = os.path.join(d, "p"), os.path.join(d, "c")
        data.tofile(src)
        synth.bytes_np(76, synth.STREAM_DATA, 2 * n + 4096).tofile(enc)
        r = crypt_file(src, enc, key, "ctr", bytes(iv), chunk_bytes=(1 << 20) + 16, threads=6, direct=direct)
        assert r["bytes"] == n and os.path.getsize(enc) == n
        assert np.array_equal(np.fromfile(enc, np.uint8), oracle.ctr_xcrypt(key, 256, iv, data))
