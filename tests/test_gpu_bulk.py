"""GPU parity of the TMA-staged CTR variant (AES_VARIANT_TTABLE_BULK).

The variant stages each half run of input into shared memory with a bulk
copy before XORing the keystream; every byte must equal the oracle's: whole
runs (the staged path), partial first and last runs and split tail pieces
(plain loads), a ragged last block, in place, the counter wrap, every key
size, small and large grids and CTA sizes, and a 64 MiB buffer (several
whole waves of staged runs).  No bounded wait may have given up.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import Guarded, host_threads, require_cuda, to_dev

pytestmark = pytest.mark.gpu

BULK = 3  # AES_VARIANT_TTABLE_BULK


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def A(torch):
    from paper_1403_7295_gb300 import aes

    aes.lib()
    aes.aes_take_wait_timeouts()  # start the count from zero
    return aes


@pytest.mark.parametrize("bits", (128, 192, 256))
def test_bulk_variant_matches_oracle(A, torch, oracle, bits):
    key = synth.key_bytes(300 + bits, bits)
    ks = A.aes_expand_key(key)
    shapes = [dict(variant=BULK, cta_threads=0, blocks_per_thread=0, grid_ctas=0),
              dict(variant=BULK, cta_threads=256, blocks_per_thread=0, grid_ctas=3),
              dict(variant=BULK, cta_threads=1024, blocks_per_thread=0, grid_ctas=1)]
    for c0 in (0, 0x00000011, 0xFFFFF0F0):  # run-aligned start, a partial first run, the 2^32 wrap
        iv = synth.iv_bytes(bits, counter0=c0)
        for n in (16 * 256, 16 * 257 + 3, 16 * (1024 * 40 + 5) + 9, (4 << 20) + 7):
            x = synth.bytes_np(n, synth.STREAM_DATA, n)
            want = oracle.ctr_xcrypt(key, bits, iv, x, nthreads=host_threads())
            xd = to_dev(x)
            for shape in shapes:
                g = Guarded(n)
                A.aes_ctr_xcrypt(ks, iv, xd, g.view, config=shape)
                torch.cuda.synchronize()
                assert np.array_equal(g.numpy(), want), (c0, n, shape)
                assert g.intact(), (c0, n, shape)
    assert A.aes_take_wait_timeouts() == 0


def test_bulk_variant_in_place_and_64MiB(A, torch, oracle):
    n = 64 << 20
    key = synth.key_bytes(310, 128)
    iv = synth.iv_bytes(310, counter0=0x00123400)
    ks = A.aes_expand_key(key)
    x = synth.bytes_np(310, synth.STREAM_DATA, n)
    buf = to_dev(x)
    A.aes_ctr_xcrypt(ks, iv, buf, buf, config=dict(variant=BULK, cta_threads=0, blocks_per_thread=0,
                                                   grid_ctas=0))
    torch.cuda.synchronize()
    assert np.array_equal(buf.cpu().numpy(), oracle.ctr_xcrypt(key, 128, iv, x, nthreads=host_threads()))
    assert A.aes_take_wait_timeouts() == 0


def test_bulk_variant_is_ctr_only(A, torch):
    ks = A.aes_expand_key(synth.key_bytes(311, 128))
    x = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    for fn in (A.aes_ecb_encrypt, A.aes_ecb_decrypt):
        with pytest.raises(A.AesError) as e:
            fn(ks, x, config=dict(variant=BULK, cta_threads=0, blocks_per_thread=0, grid_ctas=0))
        assert e.value.status == 1
    with pytest.raises(A.AesError):
        A.aes_ctr_xcrypt(ks, bytes(16), x, config=dict(variant=BULK, cta_threads=0, blocks_per_thread=2,
                                                       grid_ctas=0))
