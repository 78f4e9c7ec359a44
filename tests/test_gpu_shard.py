"""The multi-GPU split run through the CUDA path, on one GPU.

A buffer split into the contiguous whole-block ranges of ``shard_ranges``
(the paper's N-chunk scheme, §IV.B, at device granularity) and processed one
library call per range, each CTR range with the IV that
``aes_ctr_iv_advance`` gives for its first block, must equal one oracle pass
over the whole buffer byte for byte: for 1, 2, 3 and 8 ranks, a ragged end,
and a counter that wraps modulo 2^32 inside the buffer (and, for some splits,
exactly at a range boundary).  On a multi-GPU node each range would be one
rank's call on its own device; here the calls run one after another.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import Guarded, host_threads, require_cuda, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def A(torch):
    from paper_1403_7295_gb300 import aes

    aes.lib()
    return aes


@pytest.mark.parametrize("world", [1, 2, 3, 8])
@pytest.mark.parametrize("nbytes,counter0", [(16 * 100_003 + 7, 0xFFFFF000),
                                             (64 << 20, 0xFFFFFFFF - (2 << 20)),
                                             (16 * 24, 0xFFFFFFF4)])
def test_ctr_shards_equal_one_pass(A, torch, oracle, world, nbytes, counter0):
    from paper_1403_7295_gb300.shard import ctr_iv_at, shard_ranges

    bits = 256
    key = synth.key_bytes(world, bits)
    iv = synth.iv_bytes(world, counter0=counter0)
    x = synth.bytes_np(world, synth.STREAM_DATA, nbytes)
    ks = A.aes_expand_key(key)
    xd = to_dev(x)
    g = Guarded(nbytes)
    for sh in shard_ranges(nbytes, world):
        if sh.byte_len == 0:
            continue
        riv = ctr_iv_at(iv, sh.first_block)
        A.aes_ctr_xcrypt(ks, riv, xd[sh.byte_off: sh.byte_off + sh.byte_len],
                         g.view[sh.byte_off: sh.byte_off + sh.byte_len])
    torch.cuda.synchronize()
    assert np.array_equal(g.numpy(), oracle.ctr_xcrypt(key, bits, iv, x, nthreads=host_threads()))
    assert g.intact()


@pytest.mark.parametrize("world", [2, 3, 8])
def test_ecb_shards_equal_one_pass(A, torch, oracle, world):
    from paper_1403_7295_gb300.shard import shard_ranges

    nbytes = 16 * 300_001
    key = synth.key_bytes(10 + world, 128)
    x = synth.bytes_np(10 + world, synth.STREAM_DATA, nbytes)
    ks = A.aes_expand_key(key)
    xd = to_dev(x)
    enc, dec = Guarded(nbytes), Guarded(nbytes)
    for sh in shard_ranges(nbytes, world):
        sl = slice(sh.byte_off, sh.byte_off + sh.byte_len)
        A.aes_ecb_encrypt(ks, xd[sl], enc.view[sl])
        A.aes_ecb_decrypt(ks, enc.view[sl], dec.view[sl])
    torch.cuda.synchronize()
    assert np.array_equal(enc.numpy(), oracle.ecb_encrypt(key, 128, x, nthreads=host_threads()))
    assert np.array_equal(dec.numpy(), x)
    assert enc.intact() and dec.intact()
