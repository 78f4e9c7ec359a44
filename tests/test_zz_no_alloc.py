"""The allocation-free batch call computes exactly what aes_batch_submit does.

Some callers cannot allocate device memory: code running in a host callback,
on a latency-critical path where cudaMalloc's implicit synchronisation would
stall other streams, or inside a framework that owns every device
allocation.  ``aes_batch_submit_noalloc`` serves them by keeping the batch
workspace in a fixed device array of the library.  These tests call it
through the C ABI for two different batches in a row (then the first one
again, over the array the second left behind), for a batch of exactly the
message cap twice, and across CUDA contexts, and compare every output byte,
status and output length with the workspace-taking ``aes_batch_submit`` (AES
is exact, so the tolerance is zero), and check the size limit.

This file sorts last so a run that stops at the first failure has already run
everything else; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth
from synth import workloads as W
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def lib(torch):
    from paper_1403_7295_gb300 import batch

    L = batch._declare()
    L.aes_batch_submit_noalloc.argtypes = [ctypes.POINTER(batch.AesBatch), ctypes.c_void_p]
    L.aes_batch_submit_noalloc.restype = ctypes.c_int
    return L


def make(torch, op, n, seed):
    from paper_1403_7295_gb300 import batch as B

    lengths = W.uniform_lengths(seed, n, 0, 3000)
    lengths[:6] = [0, 1, 15, 16, 17, 4096]
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(seed, synth.STREAM_DATA, max(total, 16), device="cuda")
    ivs = W.message_ivs(seed, n, counter0=0xFFFFFFFE) if op == B.BATCH_CTR else None
    b = B.Batch(op, data, in_off, lengths, keys=W.message_keys(seed, n),
                key_bits=W.key_sizes(seed, n), ivs=ivs)
    return b


def snapshot(b):
    return b.out.clone(), b.status.clone(), b.out_len.clone()


def reset(b):
    b.out.fill_(0)
    b.status.fill_(-1)
    b.out_len.fill_(-1)


def test_noalloc_matches_workspace_call_two_calls_in_a_row(torch, lib):
    from paper_1403_7295_gb300 import batch as B

    b1 = make(torch, B.BATCH_CTR, 300, 1)
    b2 = make(torch, B.BATCH_ECB_PKCS7_ENCRYPT, 5000, 2)  # > 4096: the chunked scan
    refs = []
    for b in (b1, b2):
        reset(b)
        b.submit()
        torch.cuda.synchronize()
        refs.append(snapshot(b))
    for b in (b1, b2):
        reset(b)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.aes_batch_submit_noalloc(ctypes.byref(b1.desc), stream) == 0
    assert lib.aes_batch_submit_noalloc(ctypes.byref(b2.desc), stream) == 0
    torch.cuda.synchronize()
    for b, ref in zip((b1, b2), refs):
        got = snapshot(b)
        for g, r in zip(got, ref):
            assert torch.equal(g, r)
    assert int((b2.status != 0).sum()) == 0
    # the first batch again, over the scratch contents the larger batch left
    reset(b1)
    assert lib.aes_batch_submit_noalloc(ctypes.byref(b1.desc), stream) == 0
    torch.cuda.synchronize()
    for g, r in zip(snapshot(b1), refs[0]):
        assert torch.equal(g, r)


def test_noalloc_at_the_message_cap(torch, lib):
    """Exactly AES_BATCH_NOALLOC_MAX_MSGS (65,536) messages, so the scratch
    array is used to its last byte (offsets, 16 scan chunks, counters): two
    calls in a row equal aes_batch_submit."""
    from paper_1403_7295_gb300 import batch as B

    n = 65536
    lengths = W.uniform_lengths(4, n, 0, 600)
    lengths[:4] = [0, 1, 16, 8192]  # empty, one byte, one block, a tile-phase message
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(4, synth.STREAM_DATA, max(total, 16), device="cuda")
    b = B.Batch(B.BATCH_CTR, data, in_off, lengths, keys=W.message_keys(4, n),
                key_bits=W.key_sizes(4, n), ivs=W.message_ivs(4, n, counter0=0xFFFFFF80))
    reset(b)
    b.submit()
    torch.cuda.synchronize()
    ref = snapshot(b)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        reset(b)
        assert lib.aes_batch_submit_noalloc(ctypes.byref(b.desc), stream) == 0
        torch.cuda.synchronize()
        for g, r in zip(snapshot(b), ref):
            assert torch.equal(g, r)
    assert int((b.status != 0).sum()) == 0


def test_noalloc_follows_the_current_context(torch):
    """The scratch address is kept per CUDA context: in a child process (driver
    API only) the call runs in the device's primary context, in a second
    context made with cuCtxCreate, and in the primary one again, each time
    equal to aes_batch_submit byte for byte (tests/noalloc_context_child.py)."""
    import os
    import subprocess
    import sys

    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "noalloc_context_child.py")
    r = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), (r.returncode, r.stdout[-2000:], r.stderr[-2000:])


def test_noalloc_size_limit_and_arguments(torch, lib):
    from paper_1403_7295_gb300 import batch as B

    b = make(torch, B.BATCH_CTR, 8, 3)
    d = B.AesBatch.from_buffer_copy(b.desc)
    d.n_msgs = 65536 + 1
    assert lib.aes_batch_submit_noalloc(ctypes.byref(d), None) == 7  # AES_ERR_NOMEM, nothing enqueued
    assert lib.aes_batch_submit_noalloc(None, None) == 1              # AES_ERR_ARG
    d.n_msgs = 0
    assert lib.aes_batch_submit_noalloc(ctypes.byref(d), None) == 0   # empty batch: no-op
