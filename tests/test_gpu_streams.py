"""The single-buffer entry points inside a CUDA graph and from several host threads.

Graph: each single-buffer call is a set of kernel launches with the round keys
and counter parameters passed by value, so after one warm-up call (which sets
the kernels' shared-memory attribute) a sequence of calls captures into one
graph.  Replays with new contents in the captured input buffers must give the
oracle's bytes for those contents.

Threads: eight host threads, each on its own stream with its own key, call the
library at the same time (ctypes releases the GIL around each call); every
output must equal the oracle's.  This covers the process-wide caches (SM count,
the shared-memory opt-in per kernel and device) under concurrent first use.

Chain: dependent in-place calls back to back on one stream, with torch
kernels in between and no synchronisation (the single-buffer launches use
programmatic dependent launch, so this checks every wait is in place).
"""
import threading

import numpy as np
import pytest

import synth
from tests.gpu_util import require_cuda, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def A(torch):
    from paper_1403_7295_gb300 import aes

    aes.lib()
    return aes


def test_single_buffer_calls_replay_in_a_graph(A, torch, oracle):
    bits = 256
    key, k2 = synth.key_bytes(301, bits), synth.key_bytes(302, bits)
    ks, ks2 = A.aes_expand_key(key), A.aes_expand_key(k2)
    iv = synth.iv_bytes(303, counter0=0xFFFFFF00)
    n = 152 * 1024 * 16 * 3 + 4096  # several waves of CTAs, whole 4 KiB sectors
    x = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ctr_out, ecb_out, cbc_out, xts_out = (torch.empty_like(x) for _ in range(4))
    cbc_in = torch.zeros_like(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        # warm-up outside capture: first use of each kernel sets its attributes
        A.aes_ctr_xcrypt(ks, iv, x, ctr_out)
        A.aes_ecb_encrypt(ks, x, ecb_out)
        A.aes_cbc_decrypt(ks, iv, cbc_in, cbc_out)
        A.aes_xts_encrypt(ks, ks2, 5, 4096, x, xts_out)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        A.aes_ctr_xcrypt(ks, iv, x, ctr_out)
        A.aes_ecb_encrypt(ks, x, ecb_out)
        A.aes_cbc_decrypt(ks, iv, cbc_in, cbc_out)
        A.aes_xts_encrypt(ks, ks2, 5, 4096, x, xts_out)
    for rep in range(3):
        pt = synth.bytes_np(310 + rep, synth.STREAM_DATA, n)
        ct = oracle.cbc_encrypt(key, bits, iv, pt)
        x.copy_(to_dev(pt))
        cbc_in.copy_(to_dev(ct))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(ctr_out.cpu().numpy(), oracle.ctr_xcrypt(key, bits, iv, pt)), rep
        assert np.array_equal(ecb_out.cpu().numpy(), oracle.ecb_encrypt(key, bits, pt)), rep
        assert np.array_equal(cbc_out.cpu().numpy(), pt), rep
        assert np.array_equal(xts_out.cpu().numpy(), oracle.xts(False, key, k2, bits, 4096, 5, pt)), rep


def test_concurrent_calls_from_host_threads(A, torch, oracle):
    n_threads, reps = 8, 6
    sizes = [(1 << 20) * (t + 1) + 16 * t + (t % 3) for t in range(n_threads)]
    cases = []
    for t in range(n_threads):
        bits = (128, 192, 256)[t % 3]
        key = synth.key_bytes(400 + t, bits)
        iv = synth.iv_bytes(420 + t)
        pt = synth.bytes_np(440 + t, synth.STREAM_DATA, sizes[t])
        ecb_len = sizes[t] - sizes[t] % 16
        cases.append((bits, key, iv, pt, oracle.ctr_xcrypt(key, bits, iv, pt),
                      oracle.ecb_encrypt(key, bits, pt[:ecb_len])))
    results = [None] * n_threads
    errors = []
    start = threading.Barrier(n_threads)

    def worker(t):
        try:
            bits, key, iv, pt, _, _ = cases[t]
            stream = torch.cuda.Stream()
            ecb_len = pt.size - pt.size % 16
            with torch.cuda.stream(stream):
                x = to_dev(pt)
                ks = A.aes_expand_key(key)
                outs = []
                start.wait()
                for _ in range(reps):
                    c = A.aes_ctr_xcrypt(ks, iv, x)
                    e = A.aes_ecb_encrypt(ks, x[:ecb_len])
                    d = A.aes_ecb_decrypt(ks, e)
                    outs = [c, e, d]
                stream.synchronize()
                results[t] = [o.cpu().numpy() for o in outs]
        except Exception as exc:  # reported on the main thread
            errors.append((t, repr(exc)))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(n_threads)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert not errors, errors
    for t in range(n_threads):
        _, _, _, pt, want_ctr, want_ecb = cases[t]
        c, e, d = results[t]
        assert np.array_equal(c, want_ctr), t
        assert np.array_equal(e, want_ecb), t
        assert np.array_equal(d, pt[:want_ecb.size]), t


def test_dependent_calls_back_to_back_without_sync(A, torch, oracle):
    """Single-buffer launches may start (and fill their tables) while the
    previous kernel in the stream finishes; each waits for that grid before
    it touches memory.  A chain of in-place calls that each read the previous
    call's output, with torch kernels in between and no synchronisation, must
    give exactly the oracle's chain."""
    bits = 128
    k1, k2 = synth.key_bytes(501, bits), synth.key_bytes(502, bits)
    ks1, ks2 = A.aes_expand_key(k1), A.aes_expand_key(k2)
    iv = synth.iv_bytes(503, counter0=0xFFFFFF00)
    n = (3 << 20) + 4096
    pt = synth.bytes_np(504, synth.STREAM_DATA, n)
    x = to_dev(pt)
    other = torch.empty_like(x)
    want = pt.copy()
    for rep in range(6):
        A.aes_ctr_xcrypt(ks1, iv, x, x)                # in place
        A.aes_ecb_encrypt(ks2, x, x)                   # reads the CTR output
        x.add_(rep)                                    # a torch kernel in between (uint8 wraps)
        A.aes_ecb_decrypt(ks1, x, other)               # another buffer
        A.aes_xts_encrypt(ks1, ks2, rep, 4096, other, x)
        want = oracle.ctr_xcrypt(k1, bits, iv, want)
        want = oracle.ecb_encrypt(k2, bits, want)
        want = (want.astype(np.uint16) + rep).astype(np.uint8)
        want = oracle.ecb_decrypt(k1, bits, want)
        want = oracle.xts(False, k1, k2, bits, 4096, rep, want)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), want)
