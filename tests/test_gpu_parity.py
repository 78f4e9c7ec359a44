"""GPU parity: every byte the CUDA path writes equals the CPU oracle's.

AES is exact integer work with one correct output per (key, input), so the
bar is bit-exact equality.  Cases span several CTAs and a ragged tail, every
launch shape the library accepts, all three key sizes, ECB encrypt/decrypt
and CTR, the 16 MiB ECB round trip, counter wrap, in-place operation, and
canary bands around every output.  Whole buffers of 64 MiB (every key size
and op: past the 19 MiB where the default CTR kernel starts walking whole
waves of counter runs) and 1 GiB are compared with the threaded oracle byte
for byte at the default launch shape the bench times; 8 GiB is checked on
sampled blocks the oracle computes one by one, plus whole-buffer round trips.
"""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_util import Guarded, host_threads, library_mapped, require_cuda, to_dev

pytestmark = pytest.mark.gpu

KEY_BITS = (128, 192, 256)
SHAPES = [
    None,  # library default (what the bench times)
    dict(variant=1, cta_threads=128, blocks_per_thread=1, grid_ctas=0),
    dict(variant=1, cta_threads=256, blocks_per_thread=2, grid_ctas=3),
    dict(variant=1, cta_threads=512, blocks_per_thread=4, grid_ctas=7),
    dict(variant=1, cta_threads=1024, blocks_per_thread=4, grid_ctas=0),
    dict(variant=1, cta_threads=1024, blocks_per_thread=1, grid_ctas=1),
    dict(variant=2, cta_threads=0, blocks_per_thread=0, grid_ctas=0),  # bitsliced
    dict(variant=2, cta_threads=0, blocks_per_thread=0, grid_ctas=3),
]


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def A(torch):
    from paper_1403_7295_gb300 import aes

    aes.lib()
    return aes


def run_op(A, op, ks, iv, x_dev, out=None, config=None):
    if op == "ecb_enc":
        return A.aes_ecb_encrypt(ks, x_dev, out, config=config)
    if op == "ecb_dec":
        return A.aes_ecb_decrypt(ks, x_dev, out, config=config)
    return A.aes_ctr_xcrypt(ks, iv, x_dev, out, config=config)


def oracle_op(oracle, op, key, bits, iv, x, nthreads=0):
    if op == "ecb_enc":
        return oracle.ecb_encrypt(key, bits, x, nthreads=nthreads)
    if op == "ecb_dec":
        return oracle.ecb_decrypt(key, bits, x, nthreads=nthreads)
    return oracle.ctr_xcrypt(key, bits, iv, x, nthreads=nthreads)


def test_native_library_is_loaded(A, torch):
    assert library_mapped()


def test_config1_ecb_16MiB_round_trip(A, torch, oracle):
    """AES-128 ECB encrypt then decrypt of 16 MiB of seed-0 bytes, full compare."""
    n = 16 << 20
    key = synth.key_bytes(0, 128)
    pt = synth.bytes_np(0, synth.STREAM_DATA, n)
    ks = A.aes_expand_key(key)
    ct_buf, back_buf = Guarded(n), Guarded(n)
    A.aes_ecb_encrypt(ks, to_dev(pt), ct_buf.view)
    A.aes_ecb_decrypt(ks, ct_buf.view, back_buf.view)
    torch.cuda.synchronize()
    ct = ct_buf.numpy()
    assert np.array_equal(ct, oracle.ecb_encrypt(key, 128, pt, nthreads=host_threads()))
    assert np.array_equal(back_buf.numpy(), pt)
    assert ct_buf.intact() and back_buf.intact()


@pytest.mark.parametrize("bits", KEY_BITS)
@pytest.mark.parametrize("op", ["ecb_enc", "ecb_dec", "ctr"])
def test_parity_every_shape(A, torch, oracle, bits, op):
    # 1 block, a few warps' worth, and several CTAs' worth plus a ragged end.
    sizes = [16, 16 * 37, 16 * (1024 * 4 * 3 + 77)]
    if op == "ctr":
        sizes += [16 * (1024 * 2 * 5 + 3) + 11]
    key = synth.key_bytes(bits + len(op), bits)
    iv = synth.iv_bytes(bits, counter0=0x7FFFFF00)
    ks = A.aes_expand_key(key)
    for n in sizes:
        x = synth.bytes_np(n, synth.STREAM_DATA, n)
        want = oracle_op(oracle, op, key, bits, iv, x)
        xd = to_dev(x)
        for shape in SHAPES:
            g = Guarded(n)
            run_op(A, op, ks, iv, xd, g.view, config=shape)
            torch.cuda.synchronize()
            assert np.array_equal(g.numpy(), want), (n, shape)
            assert g.intact(), (n, shape)


@pytest.mark.parametrize("bits", KEY_BITS)
def test_ctr_edge_lengths_and_wrap(A, torch, oracle, bits):
    key = synth.key_bytes(7, bits)
    ks = A.aes_expand_key(key)
    lengths = sorted({0, 1, 15, 16, 17, 31, 33} | {(1 << k) + d for k in range(4, 21, 2) for d in (-1, 1)})
    for c0 in (0, 0xFFFFFFF0):  # the second crosses the 2^32 counter wrap
        iv = synth.iv_bytes(bits, counter0=c0)
        for n in lengths:
            x = synth.bytes_np(n + 1, synth.STREAM_DATA, n)
            want = oracle.ctr_xcrypt(key, bits, iv, x)
            g = Guarded(max(n, 1))
            out = g.view[:n]
            A.aes_ctr_xcrypt(ks, iv, to_dev(x), out)
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), want), (c0, n)
            assert g.intact(), (c0, n)


@pytest.mark.parametrize("op", ["ecb_enc", "ecb_dec", "ctr"])
def test_in_place(A, torch, oracle, op):
    n = 16 * 50_001 + (5 if op == "ctr" else 0)
    key = synth.key_bytes(21, 256)
    iv = synth.iv_bytes(21)
    x = synth.bytes_np(21, synth.STREAM_DATA, n)
    ks = A.aes_expand_key(key)
    buf = to_dev(x)
    run_op(A, op, ks, iv, buf, buf)
    torch.cuda.synchronize()
    assert np.array_equal(buf.cpu().numpy(), oracle_op(oracle, op, key, 256, iv, x))


@pytest.mark.parametrize("bits", KEY_BITS)
def test_multi_tile_4MiB_ragged(A, torch, oracle, bits):
    n = (4 << 20) + 5
    key = synth.key_bytes(31, bits)
    iv = synth.iv_bytes(31, counter0=12345)
    x = synth.bytes_np(31, synth.STREAM_DATA, n)
    ks = A.aes_expand_key(key)
    g = Guarded(n)
    A.aes_ctr_xcrypt(ks, iv, to_dev(x), g.view)
    torch.cuda.synchronize()
    assert np.array_equal(g.numpy(), oracle.ctr_xcrypt(key, bits, iv, x, nthreads=host_threads()))
    assert g.intact()
    m = n - 5
    g2 = Guarded(m)
    A.aes_ecb_encrypt(ks, to_dev(x[:m]), g2.view)
    torch.cuda.synchronize()
    assert np.array_equal(g2.numpy(), oracle.ecb_encrypt(key, bits, x[:m], nthreads=host_threads()))


def sample_indices(nblocks: int, count: int, seed: int) -> np.ndarray:
    u = synth.uniform01(seed, synth.STREAM_MISC, count)
    idx = np.unique((u * nblocks).astype(np.uint64))
    return np.unique(np.concatenate([idx, np.array([0, nblocks - 1], np.uint64)]))


@pytest.mark.parametrize("bits", KEY_BITS)
@pytest.mark.parametrize("op", ["ctr", "ecb_enc", "ecb_dec"])
def test_whole_buffer_64MiB(A, torch, oracle, bits, op):
    """64 MiB (2^22 blocks = 16,384 counter runs, over three whole waves of
    the default CTR kernel's 4,864 warps plus a split tail) at the default
    launch shape, every byte against the threaded oracle; the counter start
    is not run-aligned, so the first and last runs are partial."""
    n = 64 << 20
    seed = 61 + bits + len(op)
    key = synth.key_bytes(seed, bits)
    iv = synth.iv_bytes(seed, counter0=0x00ABCD37)
    x = synth.bytes_np(seed, synth.STREAM_DATA, n)
    ks = A.aes_expand_key(key)
    g = Guarded(n)
    run_op(A, op, ks, iv, to_dev(x), g.view)
    torch.cuda.synchronize()
    assert np.array_equal(g.numpy(), oracle_op(oracle, op, key, bits, iv, x, nthreads=host_threads()))
    assert g.intact()


@pytest.mark.parametrize("mib,bits", [(2, 128), (4, 256), (16, 256), (32, 128), (48, 256), (128, 128),
                                      (256, 256)])
def test_ctr_every_tail_split_whole_buffer(A, torch, oracle, mib, bits):
    """The default CTR kernel splits the runs of its last, partial wave into
    1, 2, 4 or 8 pieces, chosen from the run count and the grid: with 4,864
    warps, 2 MiB takes 8 pieces and 4 MiB 4 on a shrunk grid, 16 MiB keeps
    its 4,096 runs whole on 128 CTAs, and after whole waves 32 and 128 MiB
    take 4 pieces, 48 MiB 8 and 256 MiB 2.  Every byte against the threaded
    oracle, with a counter start inside a run and a ragged last block."""
    n = (mib << 20) + 11
    seed = 70 + mib
    key = synth.key_bytes(seed, bits)
    iv = synth.iv_bytes(seed, counter0=0x0001F0C5)
    x = synth.bytes_np(seed, synth.STREAM_DATA, n)
    ks = A.aes_expand_key(key)
    g = Guarded(n)
    A.aes_ctr_xcrypt(ks, iv, to_dev(x), g.view)
    torch.cuda.synchronize()
    assert np.array_equal(g.numpy(), oracle.ctr_xcrypt(key, bits, iv, x, nthreads=host_threads()))
    assert g.intact()


@pytest.mark.parametrize("bits,op", [(128, "ctr"), (256, "ctr"), (128, "ecb_enc"), (128, "ecb_dec")])
def test_whole_buffer_1GiB(A, torch, oracle, bits, op):
    """1 GiB at the bench's launch shape, every byte against the threaded
    oracle (AES-128 CTR is the bench's headline kernel; the other key size and
    both ECB directions take the other kernels)."""
    n = 1 << 30
    seed = 41 + bits
    key = synth.key_bytes(seed, bits)
    iv = synth.iv_bytes(seed)
    ks = A.aes_expand_key(key)
    x = synth.bytes_torch(seed, synth.STREAM_DATA, n, device="cuda")
    y = run_op(A, op, ks, iv, x)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    del y
    want = oracle_op(oracle, op, key, bits, iv, x.cpu().numpy(), nthreads=host_threads())
    mism = np.flatnonzero(got != want)
    assert mism.size == 0, f"{mism.size} bytes differ, first at {mism[:4]}"


def test_full_size_sampled_8GiB(A, torch, oracle):
    """8 GiB (the bench's buffer) at its launch shape: 4,096 sampled blocks vs
    the oracle (one by one), whole-buffer round trips on the device."""
    gib = 8
    n = gib << 30
    nblocks = n // 16
    seed = 40 + gib
    x = synth.bytes_torch(seed, synth.STREAM_DATA, n, device="cuda")
    idx = sample_indices(nblocks, 4096, seed)
    tix = torch.from_numpy(idx.astype(np.int64)).cuda()
    xs = x.view(-1, 16)[tix].cpu().numpy()
    for bits in (128, 256):
        key = synth.key_bytes(seed, bits)
        iv = synth.iv_bytes(seed)
        ks = A.aes_expand_key(key)
        y = torch.empty_like(x)
        A.aes_ctr_xcrypt(ks, iv, x, y)
        ys = y.view(-1, 16)[tix].cpu().numpy()
        assert np.array_equal(ys.reshape(-1), oracle.ctr_xcrypt_blocks(key, bits, iv, idx, xs))
        A.aes_ctr_xcrypt(ks, iv, y, y)  # CTR is its own inverse, in place
        assert torch.equal(y, x)
        A.aes_ecb_encrypt(ks, x, y)
        ys = y.view(-1, 16)[tix].cpu().numpy()
        assert np.array_equal(ys.reshape(-1), oracle.ecb_encrypt(key, bits, xs.reshape(-1)))
        A.aes_ecb_decrypt(ks, y, y)
        assert torch.equal(y, x)
        del y
    torch.cuda.empty_cache()


def test_pinned_host_buffers(A, torch, oracle):
    n = 16 * 4099 + 9
    key = synth.key_bytes(50, 192)
    iv = synth.iv_bytes(50)
    x = synth.bytes_np(50, synth.STREAM_DATA, n)
    ks = A.aes_expand_key(key)
    h_in = torch.from_numpy(x).pin_memory()
    h_out = torch.empty(n, dtype=torch.uint8).pin_memory()
    A.aes_ctr_xcrypt(ks, iv, h_in, h_out, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy(), oracle.ctr_xcrypt(key, 192, iv, x))


def test_pageable_host_pointer_is_refused(A, torch):
    lib = A.lib()
    ks = A.aes_expand_key(synth.key_bytes(1, 128))
    buf = (ctypes.c_uint8 * 4096)()
    p = (ctypes.addressof(buf) + 15) & ~15
    rc = lib.aes_ecb_encrypt(ctypes.byref(ks), p, p, 1024, None)
    assert rc == 1  # AES_ERR_ARG: pageable memory is never handed to a kernel


def test_shapes_agree_at_bench_size(A, torch):
    """Every accepted launch shape computes the same bytes on a 64 MiB buffer."""
    n = 64 << 20
    x = synth.bytes_torch(60, synth.STREAM_DATA, n, device="cuda")
    key = synth.key_bytes(60, 128)
    iv = synth.iv_bytes(60)
    ks = A.aes_expand_key(key)
    ref = A.aes_ctr_xcrypt(ks, iv, x)
    for shape in SHAPES[1:]:
        assert torch.equal(A.aes_ctr_xcrypt(ks, iv, x, config=shape), ref), shape
