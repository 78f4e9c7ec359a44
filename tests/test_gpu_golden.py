"""The GPU library reproduces every stored oracle vector (tests/golden/)."""
import numpy as np
import pytest

from tests.golden_util import aes_vectors
from tests.gpu_util import require_cuda, to_dev

pytestmark = pytest.mark.gpu


def test_gpu_reproduces_golden_vectors():
    torch = require_cuda()
    from paper_1403_7295_gb300 import aes as A
    from paper_1403_7295_gb300 import batch as B

    for v in aes_vectors():
        m, b, k, iv, d = v["mode"], v["bits"], v["key"], v["iv"], v["data"]
        if m == "xts_enc_512":
            half = k.size // 2
            got = A.aes_xts_encrypt(A.aes_expand_key(k[:half], b), A.aes_expand_key(k[half:], b),
                                    int.from_bytes(bytes(iv), "little"), 512, to_dev(d))
        elif m == "ecb_pkcs7_enc":
            in_off, total = B.pack_offsets(np.array([d.size], np.uint64))
            arena = torch.zeros(max(total, 16), dtype=torch.uint8, device="cuda")
            arena[: d.size] = to_dev(d)
            keys = np.zeros((1, 32), np.uint8)
            keys[0, : k.size] = k
            bt = B.Batch(B.BATCH_ECB_PKCS7_ENCRYPT, arena, in_off, np.array([d.size], np.uint64),
                         keys=keys, key_bits=np.array([b], np.uint32)).submit()
            got = bt.out[: int(bt.out_len[0].item())]
        else:
            ks = A.aes_expand_key(k, b)
            x = to_dev(d)
            if m == "ecb_enc":
                got = A.aes_ecb_encrypt(ks, x)
            elif m == "ctr":
                got = A.aes_ctr_xcrypt(ks, iv, x)
            else:
                got = A.aes_cbc_decrypt(ks, iv, x)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), v["out"]), (m, b, d.size)
