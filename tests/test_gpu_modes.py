"""GPU parity of CBC decryption and XTS against the oracle (bit-exact).

CBC: every key size, sizes spanning several CTAs with a ragged block count,
canary bands, in-place refused.  XTS: AES-128 and AES-256 key pairs (the
two sizes IEEE 1619 defines; 192-bit and mixed pairs are refused), data units
of 512 B, 4 KiB and 64 KiB (a unit longer than one warp's 1024 blocks, so a
warp starts in the middle of a unit), first sector 0, 7 and 2^40 + 3, encrypt
against the oracle, decrypt back, in place.
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


@pytest.mark.parametrize("bits", (128, 192, 256))
def test_cbc_decrypt_matches_oracle(A, torch, oracle, bits):
    key = synth.key_bytes(80 + bits, bits)
    iv = synth.bytes_np(80, synth.STREAM_NONCE, 16)
    ks = A.aes_expand_key(key)
    for nblocks in (1, 37, 1024 * 3 + 77, 152 * 1024 + 5):
        pt = synth.bytes_np(nblocks, synth.STREAM_DATA, 16 * nblocks)
        ct = oracle.cbc_encrypt(key, bits, iv, pt)
        g = Guarded(ct.size)
        A.aes_cbc_decrypt(ks, iv, to_dev(ct), g.view)
        torch.cuda.synchronize()
        assert np.array_equal(g.numpy(), pt), nblocks
        assert g.intact()
    x = to_dev(ct)
    with pytest.raises(A.AesError):
        A.aes_cbc_decrypt(ks, iv, x, x)


@pytest.mark.parametrize("bits", (128, 256))
@pytest.mark.parametrize("sector_bytes,first_sector", [(512, 0), (4096, 7), (65536, (1 << 40) + 3)])
def test_xts_matches_oracle(A, torch, oracle, bits, sector_bytes, first_sector):
    key1, key2 = synth.key_bytes(90 + bits, bits), synth.key_bytes(91 + bits, bits)
    k1, k2 = A.aes_expand_key(key1), A.aes_expand_key(key2)
    units = max(3, (2 << 20) // sector_bytes) + 1
    pt = synth.bytes_np(units, synth.STREAM_DATA, units * sector_bytes)
    want = oracle.xts(False, key1, key2, bits, sector_bytes, first_sector, pt)
    g = Guarded(pt.size)
    A.aes_xts_encrypt(k1, k2, first_sector, sector_bytes, to_dev(pt), g.view)
    torch.cuda.synchronize()
    assert np.array_equal(g.numpy(), want)
    assert g.intact()
    buf = g.view.clone()
    A.aes_xts_decrypt(k1, k2, first_sector, sector_bytes, buf, buf)  # in place
    torch.cuda.synchronize()
    assert np.array_equal(buf.cpu().numpy(), pt)


def test_xts_refuses_key_sizes_outside_the_standard(A, torch):
    """IEEE 1619 / SP 800-38E define XTS-AES-128 and XTS-AES-256 only."""
    x = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    k128, k192, k256 = (A.aes_expand_key(synth.key_bytes(97, b)) for b in (128, 192, 256))
    for d, t in ((k192, k192), (k128, k256), (k256, k128), (k192, k128)):
        for fn in (A.aes_xts_encrypt, A.aes_xts_decrypt):
            with pytest.raises(A.AesError) as e:
                fn(d, t, 0, 512, x)
            assert e.value.status == 2  # AES_ERR_KEYSIZE


def test_xts_large_buffer_sampled(A, torch, oracle):
    """256 MiB of 4 KiB units: sampled units against the oracle, round trip on the device."""
    n, su = 256 << 20, 4096
    key1, key2 = synth.key_bytes(95, 256), synth.key_bytes(96, 256)
    k1, k2 = A.aes_expand_key(key1), A.aes_expand_key(key2)
    x = synth.bytes_torch(95, synth.STREAM_DATA, n, device="cuda")
    y = A.aes_xts_encrypt(k1, k2, 1000, su, x)
    units = n // su
    for u in np.unique((synth.uniform01(95, synth.STREAM_MISC, 64) * units).astype(np.int64)).tolist() + [0, units - 1]:
        src = x[u * su: (u + 1) * su].cpu().numpy()
        got = y[u * su: (u + 1) * su].cpu().numpy()
        assert np.array_equal(got, oracle.xts(False, key1, key2, 256, su, 1000 + u, src)), u
    z = A.aes_xts_decrypt(k1, k2, 1000, su, y)
    assert torch.equal(z, x)
