"""GPU parity of the batched path: every message equals the oracle run on that
message alone, bit for bit.

Covers CTR, ECB+PKCS#7 encrypt and decrypt; mixed key sizes; raw keys
expanded on the device and pre-expanded schedule tables; empty, 1-byte,
block-sized and ragged messages; batches large enough for the chunked scan
(> 4096 messages) and for many key windows per tile (thousands of one-block
messages per tile); per-message failures (bad key size, misaligned offset,
bad ECB length, bad padding) that leave the rest of the batch intact;
CUDA-graph replay; and the full-size batched workloads: all 1,000,000
packet-sized messages compared whole, and of the 16,384 log-uniform messages
(64 B .. 4 MiB) every message up to 1 MiB compared whole and the larger ones
on sampled blocks, for CTR and for ECB+PKCS#7 encryption and decryption.
The whole-message compares run the oracle's message list over all host
threads.
"""
import ctypes

import numpy as np
import pytest

import synth
from synth import workloads as W
from tests.gpu_util import host_threads, require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def B(torch):
    from paper_1403_7295_gb300 import batch

    return batch


def build(B, torch, op, lengths, key_bits, keys, ivs, seed, **kw):
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(seed, synth.STREAM_DATA, max(total, 16), device="cuda")
    return B.Batch(op, data, in_off, lengths, keys=keys, key_bits=key_bits, ivs=ivs, **kw)


def oracle_check(B, oracle, batch, key_bits, keys, ivs, idx=None, check_status=True):
    data = batch.data.cpu().numpy()
    out = batch.out.cpu().numpy()
    out_len = batch.out_len.cpu().numpy()
    status = batch.status.cpu().numpy()
    in_off = batch.in_off.cpu().numpy()
    ms = range(batch.n) if idx is None else idx
    for m in ms:
        ln = int(batch.lengths_np[m])
        bits = int(key_bits[m])
        key = keys[m][: bits // 8]
        io = int(in_off[m])
        msg = data[io: io + ln]
        oo = int(batch.out_off_np[m])
        if batch.op == B.BATCH_CTR:
            want = oracle.ctr_xcrypt(key, bits, ivs[m], msg)
            assert status[m] == 0 and out_len[m] == ln, m
            assert np.array_equal(out[oo: oo + ln], want), m
        elif batch.op == B.BATCH_ECB_PKCS7_ENCRYPT:
            want = oracle.ecb_pkcs7_encrypt(key, bits, msg)
            assert status[m] == 0 and out_len[m] == want.size, m
            assert np.array_equal(out[oo: oo + want.size], want), m
        else:
            rc, pt = oracle.ecb_pkcs7_decrypt(key, bits, msg)
            if rc == 0:
                assert status[m] == 0 and out_len[m] == pt.size, m
                assert np.array_equal(out[oo: oo + pt.size], pt), m
            else:
                assert status[m] == 6 and out_len[m] == 0, m


# Messages below 512 blocks take the per-warp short phase, the others the tile
# phase: these lengths sit on both sides of that split for every op (ECB
# encryption adds a padding block, so 8175 / 8176 bytes fall on either side).
SPLIT = [8175, 8176, 8177, 8191, 8192, 8193, 8208, 20000, 70001]


def mixed_lengths(seed, n):
    special = np.array([0, 1, 15, 16, 17, 31, 32, 33, 255, 256, 4095, 4096, 4097] + SPLIT, np.uint64)
    rest = W.uniform_lengths(seed, n - special.size, 0, 5000)
    return np.concatenate([special, rest])


@pytest.mark.parametrize("op", [0, 1])
def test_batch_small_messages_all_key_sizes(torch, B, oracle, op):
    n = 400
    lengths = mixed_lengths(1 + op, n)
    kb = W.key_sizes(1, n)
    keys = W.message_keys(1, n)
    ivs = W.message_ivs(1, n, counter0=0xFFFFFFF0)  # every message with > 16 blocks wraps
    b = build(B, torch, op, lengths, kb, keys, ivs if op == 0 else None, seed=11).submit()
    torch.cuda.synchronize()
    oracle_check(B, oracle, b, kb, keys, ivs)


@pytest.mark.parametrize("op", [0, 1])
def test_batch_writes_nothing_outside_messages(torch, B, oracle, op):
    """Output bytes between messages (the 16-byte alignment gaps after ragged
    CTR messages) keep their canary value; ECB output fills its padded length."""
    n = 600
    lengths = mixed_lengths(31 + op, n)
    kb = W.key_sizes(31, n)
    keys = W.message_keys(31, n)
    ivs = W.message_ivs(31, n)
    b = build(B, torch, op, lengths, kb, keys, ivs if op == 0 else None, seed=32, padded=False)
    assert b.flags == 0
    b.out.fill_(0xA5)
    b.submit()
    torch.cuda.synchronize()
    oracle_check(B, oracle, b, kb, keys, ivs)
    out = b.out.cpu().numpy()
    written = np.zeros(out.size, bool)
    ol = b.out_len.cpu().numpy()
    for m in range(n):
        o = int(b.out_off_np[m])
        written[o: o + int(ol[m])] = True
    assert np.all(out[~written] == 0xA5)


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("padded", [False, True])
def test_batch_exact_and_padded_last_blocks(torch, B, oracle, op, padded):
    """The ragged last block read and written byte-exactly (flags 0) or as a
    whole block (AES_BATCH_IN_PADDED | AES_BATCH_OUT_PADDED): identical
    message bytes, short and long messages, every key size."""
    n = 500
    lengths = mixed_lengths(35 + op, n)
    kb = W.key_sizes(35, n)
    keys = W.message_keys(35, n)
    ivs = W.message_ivs(35, n, counter0=0xFFFFFF00)
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(36, synth.STREAM_DATA, total, device="cuda")  # exactly the packed size
    b = B.Batch(op, data, in_off, lengths, keys=keys, key_bits=kb, ivs=ivs if op == 0 else None,
                padded=None if padded else False)
    assert b.flags == (3 if padded else 0)
    b.submit()
    torch.cuda.synchronize()
    oracle_check(B, oracle, b, kb, keys, ivs)


def test_batch_decrypt_round_trip_and_bad_padding(torch, B, oracle):
    n = 300
    lengths = mixed_lengths(5, n)
    kb = W.key_sizes(5, n)
    keys = W.message_keys(5, n)
    enc = build(B, torch, B.BATCH_ECB_PKCS7_ENCRYPT, lengths, kb, keys, None, seed=12).submit()
    torch.cuda.synchronize()
    ct_len = enc.out_len.cpu().numpy().astype(np.uint64)
    # corrupt the last byte of a few ciphertexts: their padding check must fail (almost surely)
    bad = [3, 50, 299]
    out = enc.out.clone()
    for m in bad:
        pos = int(enc.out_off_np[m] + ct_len[m] - 1)
        out[pos] ^= 0x5A
    dec = B.Batch(B.BATCH_ECB_PKCS7_DECRYPT, out, enc.out_off_np, ct_len, keys=keys, key_bits=kb).submit()
    torch.cuda.synchronize()
    oracle_check(B, oracle, dec, kb, keys, None)
    st = dec.status.cpu().numpy()
    ol = dec.out_len.cpu().numpy()
    src = enc.data.cpu().numpy()
    res = dec.out.cpu().numpy()
    in_off = enc.in_off.cpu().numpy()
    for m in range(n):
        if m in bad:
            continue
        assert st[m] == 0 and ol[m] == lengths[m]
        o, i, ln = int(dec.out_off_np[m]), int(in_off[m]), int(lengths[m])
        assert np.array_equal(res[o: o + ln], src[i: i + ln])


def test_batch_schedule_table_matches_raw_keys(torch, B, oracle):
    from paper_1403_7295_gb300 import aes as A

    n = 257
    lengths = mixed_lengths(7, n)
    kb = W.key_sizes(7, n)
    keys = W.message_keys(7, n)
    ivs = W.message_ivs(7, n)
    n_tenants = 37
    tid = (np.arange(n) * 7) % n_tenants
    tkeys = W.message_keys(70, n_tenants)
    tbits = W.key_sizes(70, n_tenants)
    table = b"".join(bytes(A.aes_expand_key(tkeys[t][: tbits[t] // 8], int(tbits[t]))) for t in range(n_tenants))
    sched = torch.frombuffer(bytearray(table), dtype=torch.uint8).cuda()
    # both builds of the persistent kernel (1024 and 512 threads per CTA)
    configs = (None, B.AesBatchConfig(512, 0, 0, 0))
    for op in (0, 1):
        b = build(B, torch, op, lengths, None, None, ivs if op == 0 else None, seed=13,
                  schedules=sched, n_schedules=n_tenants, sched_idx=tid)
        for cfg in configs:
            b.out.fill_(0)
            b.submit(config=cfg)
            torch.cuda.synchronize()
            oracle_check(B, oracle, b, tbits[tid], tkeys[tid], ivs)
    enc = b  # op 1 output: decrypt it through the schedule table too
    ct_len = enc.out_len.cpu().numpy().astype(np.uint64)
    src = enc.data.cpu().numpy()
    in_off = enc.in_off.cpu().numpy()
    dec = B.Batch(B.BATCH_ECB_PKCS7_DECRYPT, enc.out, enc.out_off_np, ct_len, schedules=sched,
                  n_schedules=n_tenants, sched_idx=tid)
    for cfg in configs:
        dec.out.fill_(0)
        dec.submit(config=cfg)
        torch.cuda.synchronize()
        assert np.array_equal(dec.out_len.cpu().numpy(), lengths.astype(np.int64))
        res = dec.out.cpu().numpy()
        for m in range(n):
            o, i, ln = int(dec.out_off_np[m]), int(in_off[m]), int(lengths[m])
            assert np.array_equal(res[o: o + ln], src[i: i + ln]), (cfg, m)


def test_batch_many_tiny_messages_multi_window(torch, B, oracle):
    """20,000 one-block messages: > 4096 (chunked scan) and thousands per tile."""
    n = 20000
    lengths = W.uniform_lengths(9, n, 1, 16)
    kb = W.key_sizes(9, n)
    keys = W.message_keys(9, n)
    ivs = W.message_ivs(9, n)
    b = build(B, torch, 0, lengths, kb, keys, ivs, seed=14)
    for cfg in (None, B.AesBatchConfig(256, 256, 0, 0), B.AesBatchConfig(1024, 32768, 3, 0)):
        b.out.fill_(0)
        b.submit(config=cfg)
        torch.cuda.synchronize()
        oracle_check(B, oracle, b, kb, keys, ivs)


@pytest.mark.parametrize("op", [0, 1, 2])
def test_batch_long_messages_among_many_short(torch, B, oracle, op):
    """Long messages (>= 512 blocks) each followed by 300 short ones: a tile's
    message range then spans several key windows (most slots empty), and the
    short phase runs beside the tile phase."""
    n_long, gap = 12, 300
    longs = W.uniform_lengths(41, n_long, 8192, 40000)
    shorts = W.uniform_lengths(42, n_long * gap, 0, 600)
    lengths = np.concatenate([np.concatenate([[longs[i]], shorts[i * gap:(i + 1) * gap]])
                              for i in range(n_long)]).astype(np.uint64)
    if op == 2:
        lengths = np.maximum((lengths // np.uint64(16)) * np.uint64(16), np.uint64(16))
    n = lengths.size
    kb = W.key_sizes(41, n)
    keys = W.message_keys(41, n)
    ivs = W.message_ivs(41, n, counter0=0xFFFFFF80)
    b = build(B, torch, op, lengths, kb, keys, ivs if op == 0 else None, seed=43)
    for cfg in (None, B.AesBatchConfig(1024, 65536, 0, 0), B.AesBatchConfig(512, 1024, 5, 0)):
        b.out.fill_(0)
        b.submit(config=cfg)
        torch.cuda.synchronize()
        oracle_check(B, oracle, b, kb, keys, ivs)


def test_batch_short_ctr_random_counters(torch, B, oracle):
    """Short CTR messages whose counters start anywhere: many cross a run of
    256 counters (and some wrap the 32-bit counter) inside the message."""
    n = 3000
    lengths = W.uniform_lengths(51, n, 1, 8000)
    kb = W.key_sizes(51, n)
    keys = W.message_keys(51, n)
    ivs = synth.bytes_np(51, synth.STREAM_NONCE, 16 * n).reshape(n, 16)
    ivs[::7, 12:16] = 0xFF  # counter 2^32 - 1: wraps after the first block
    b = build(B, torch, 0, lengths, kb, keys, ivs, seed=52).submit()
    torch.cuda.synchronize()
    oracle_check(B, oracle, b, kb, keys, ivs)


def test_batch_modes_in_flight_together(torch, B, oracle):
    """Mixed-mode run: a CTR batch and an ECB+PKCS#7 batch of the same
    messages, submitted alternately on two streams so both are in flight at
    once, three times; every message of both equals the oracle."""
    n = 700
    lengths = mixed_lengths(61, n)
    kb = W.key_sizes(61, n)
    keys = W.message_keys(61, n)
    ivs = W.message_ivs(61, n)
    ctr = build(B, torch, 0, lengths, kb, keys, ivs, seed=62)
    ecb = build(B, torch, 1, lengths, kb, keys, None, seed=62)
    torch.cuda.synchronize()  # inputs and descriptors were written on the default stream
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):
        ctr.submit(stream=s1)
        ecb.submit(stream=s2)
    torch.cuda.synchronize()
    oracle_check(B, oracle, ctr, kb, keys, ivs)
    oracle_check(B, oracle, ecb, kb, keys, None)


@pytest.mark.parametrize("op", [0, 1, 2])
@pytest.mark.parametrize("cta", [512, 256, 1024])
def test_batch_all_phases_at_once(torch, B, oracle, op, cta):
    """Short (1..511 blocks) and long (>= 512) messages in one batch, mixed
    key sizes and counters, in both builds of the persistent kernel: the
    tile and per-warp phases run, warps in different phases at the same
    time; ECB+PKCS#7 lengths of whole blocks exercise the padding block that
    is never read."""
    n = 900
    u = W.uniform_lengths(81 + op, n, 0, 2)
    lengths = np.where(u == 0, W.uniform_lengths(82, n, 1, 2040),
                       np.where(u == 1, W.uniform_lengths(83, n, 2100, 8100), W.uniform_lengths(84, n, 8200, 60000)))
    lengths = lengths.astype(np.uint64)
    if op == 2:
        lengths = np.maximum((lengths // np.uint64(16)) * np.uint64(16), np.uint64(16))
    kb = W.key_sizes(81, n)
    keys = W.message_keys(81, n)
    ivs = synth.bytes_np(85, synth.STREAM_NONCE, 16 * n).reshape(n, 16)
    b = build(B, torch, op, lengths, kb, keys, ivs if op == 0 else None, seed=86)
    b.submit(config=B.AesBatchConfig(cta, 0, 0, 0))
    torch.cuda.synchronize()
    oracle_check(B, oracle, b, kb, keys, ivs)


def test_batch_per_message_errors(torch, B, oracle):
    n = 64
    lengths = mixed_lengths(10, n)
    kb = W.key_sizes(10, n).copy()
    keys = W.message_keys(10, n)
    ivs = W.message_ivs(10, n)
    in_off, total = B.pack_offsets(lengths + np.uint64(16))
    in_off = in_off.copy()
    kb[5] = 100          # bad key size
    in_off[9] += 8       # misaligned message
    data = synth.bytes_torch(15, synth.STREAM_DATA, total + 32, device="cuda")
    b = B.Batch(0, data, in_off, lengths, keys=keys, key_bits=kb, ivs=ivs).submit()
    torch.cuda.synchronize()
    st = b.status.cpu().numpy()
    assert st[5] == 2 and st[9] == 4
    ok = [m for m in range(n) if m not in (5, 9)]
    oracle_check(B, oracle, b, kb, keys, ivs, idx=ok)
    # ECB decrypt with a length that is not a positive multiple of 16
    lens = np.array([32, 17, 0, 48], np.uint64)
    b2 = build(B, torch, 2, lens, np.full(4, 128, np.uint32), W.message_keys(11, 4), None, seed=16).submit()
    torch.cuda.synchronize()
    st = b2.status.cpu().numpy()
    assert st[1] == 3 and st[2] == 3


def test_batch_host_validation(torch, B):
    from paper_1403_7295_gb300 import aes as A

    lengths = np.array([16, 32], np.uint64)
    b = build(B, torch, 0, lengths, np.array([128, 128], np.uint32), W.message_keys(1, 2),
              W.message_ivs(1, 2), seed=17)
    L = B._declare()
    ws = b.workspace
    assert L.aes_batch_submit(ctypes.byref(b.desc), ws.data_ptr(), 8, None) == 7  # short workspace
    d = B.AesBatch.from_buffer_copy(b.desc)
    d.op = 9
    assert L.aes_batch_submit(ctypes.byref(d), ws.data_ptr(), ws.numel(), None) == 1
    d = B.AesBatch.from_buffer_copy(b.desc)
    d.iv = None
    assert L.aes_batch_submit(ctypes.byref(d), ws.data_ptr(), ws.numel(), None) == 1
    d = B.AesBatch.from_buffer_copy(b.desc)
    d.in_ = b.data.data_ptr() + 4
    assert L.aes_batch_submit(ctypes.byref(d), ws.data_ptr(), ws.numel(), None) == 4
    cfg = B.AesBatchConfig(1024, 1000, 0, 0)  # tile not a multiple of the CTA
    with pytest.raises(A.AesError):
        b.submit(config=cfg)
    d = B.AesBatch.from_buffer_copy(b.desc)
    d.flags = 4  # unknown flag bit
    assert L.aes_batch_submit(ctypes.byref(d), ws.data_ptr(), ws.numel(), None) == 1
    d = B.AesBatch.from_buffer_copy(b.desc)
    d.n_msgs = 0
    assert L.aes_batch_submit(ctypes.byref(d), None, 0, None) == 0


def test_batch_graph_replay_is_deterministic(torch, B, oracle):
    n = 1000
    lengths = W.log_uniform_lengths(21, n, 16, 1 << 16)
    kb = W.key_sizes(21, n)
    keys = W.message_keys(21, n)
    ivs = W.message_ivs(21, n)
    b = build(B, torch, 0, lengths, kb, keys, ivs, seed=18)
    b.out.fill_(0)  # slot padding is never written: start from a known arena
    b.submit()
    torch.cuda.synchronize()
    first = b.out.clone()
    b.capture()
    for _ in range(2):
        b.out.fill_(0)
        b.replay()
        torch.cuda.synchronize()
        assert torch.equal(b.out, first)
    oracle_check(B, oracle, b, kb, keys, ivs, idx=range(0, n, 7))


def sampled_check_large(B, oracle, b, key_bits, keys, ivs, ms, max_full=1 << 20):
    """Messages up to max_full bytes compared whole; larger ones on 256 sampled blocks."""
    import torch

    for m in ms:
        ln = int(b.lengths_np[m])
        bits = int(key_bits[m])
        key = keys[m][: bits // 8]
        io = int(b.in_off[m].item())
        oo = int(b.out_off_np[m])
        if ln <= max_full:
            msg = b.data[io: io + ln].cpu().numpy()
            got = b.out[oo: oo + ln].cpu().numpy()
            assert np.array_equal(got, oracle.ctr_xcrypt(key, bits, ivs[m], msg)), m
        else:
            nb = ln // 16
            idx = np.unique((synth.uniform01(m, synth.STREAM_MISC, 256) * nb).astype(np.uint64))
            t = torch.from_numpy(idx.astype(np.int64)).cuda()
            blocks = b.data[io: io + 16 * nb].view(-1, 16)[t].cpu().numpy()
            got = b.out[oo: oo + 16 * nb].view(-1, 16)[t].cpu().numpy()
            want = oracle.ctr_xcrypt_blocks(key, bits, ivs[m], idx, blocks)
            assert np.array_equal(got.reshape(-1), want), m


def oracle_list_check(B, oracle, b, key_bits, keys, ivs, ms):
    """Messages `ms` of batch `b` against the oracle's message list (one
    oracle call per message, all host threads): output bytes, status and
    output length.  The oracle writes its outputs over a copy of the GPU's
    output arena, so the two arenas are equal exactly when every checked
    message is."""
    ms = np.asarray(ms, np.int64)
    data = b.data.cpu().numpy()
    got = b.out.cpu().numpy()
    status = b.status.cpu().numpy()[ms]
    out_len = b.out_len.cpu().numpy()[ms]
    in_off = b.in_off.cpu().numpy().astype(np.uint64)[ms]
    ivs_m = np.asarray(ivs)[ms] if ivs is not None else None
    want, want_len, want_st = oracle.batch(b.op, data, in_off, b.lengths_np[ms], got.size, b.out_off_np[ms],
                                           np.asarray(keys)[ms], np.asarray(key_bits)[ms], ivs_m,
                                           nthreads=host_threads(), out=got.copy())
    # the library's status codes: 0 ok, 6 AES_ERR_PADDING (the oracle's -3)
    assert np.array_equal(status, np.where(want_st == 0, 0, np.where(want_st == -3, 6, -100)))
    assert np.array_equal(out_len.astype(np.uint64), want_len)
    mism = np.flatnonzero(got != want)
    assert mism.size == 0, f"{mism.size} output bytes differ, first at {mism[:4]}"


def sampled_check_large_ecb(B, oracle, b, key_bits, keys, ms, decrypt):
    """ECB messages compared on 256 sampled whole blocks each (block j of the
    output is the cipher, or inverse cipher, of block j of the input; the
    padded last block is covered by the whole-message compares)."""
    import torch

    for m in ms:
        ln = int(b.lengths_np[m])
        bits = int(key_bits[m])
        key = keys[m][: bits // 8]
        io = int(b.in_off[m].item())
        oo = int(b.out_off_np[m])
        nb = ln // 16
        idx = np.unique((synth.uniform01(m, synth.STREAM_MISC, 256) * nb).astype(np.int64))
        t = torch.from_numpy(idx).cuda()
        blocks = b.data[io: io + 16 * nb].view(-1, 16)[t].cpu().numpy().reshape(-1)
        got = b.out[oo: oo + 16 * nb].view(-1, 16)[t].cpu().numpy().reshape(-1)
        want = oracle.ecb_decrypt(key, bits, blocks) if decrypt else oracle.ecb_encrypt(key, bits, blocks)
        assert np.array_equal(got, want), m


def test_full_size_batched_varlen_16384(torch, B, oracle):
    """16,384 messages, log-uniform 64 B .. 4 MiB, mixed key sizes (about
    6 GB), at the autotuned shape in a CUDA graph: every message up to 1 MiB
    compared whole with the oracle (about 1.5 GB), the larger ones on 256
    sampled blocks each; then the same for ECB+PKCS#7 encryption, and for
    decryption of that ciphertext (padding checked, lengths restored)."""
    wl = W.batched_varlen(3, 16384)
    lengths, kb, keys, ivs = wl["lengths"], wl["key_bits"], wl["keys"], wl["ivs"]
    small = np.flatnonzero(lengths <= (1 << 20))
    large = np.flatnonzero(lengths > (1 << 20))
    assert small.size > 14000 and large.size > 1000
    b = build(B, torch, 0, lengths, kb, keys, ivs, seed=19)
    b.capture(B.autotune(b))
    b.replay()
    torch.cuda.synchronize()
    assert int((b.status != 0).sum()) == 0
    oracle_list_check(B, oracle, b, kb, keys, ivs, small)
    sampled_check_large(B, oracle, b, kb, keys, ivs, large)
    del b
    torch.cuda.empty_cache()
    enc = build(B, torch, 1, lengths, kb, keys, None, seed=20)
    enc.capture(B.autotune(enc))
    enc.replay()
    torch.cuda.synchronize()
    assert int((enc.status != 0).sum()) == 0
    oracle_list_check(B, oracle, enc, kb, keys, None, small)
    sampled_check_large_ecb(B, oracle, enc, kb, keys, large, decrypt=False)
    ct_len = enc.out_len.cpu().numpy().astype(np.uint64)
    assert np.array_equal(ct_len, lengths - lengths % np.uint64(16) + np.uint64(16))
    dec = B.Batch(2, enc.out, enc.out_off_np, ct_len, keys=keys, key_bits=kb)
    dec.capture(B.autotune(dec))
    dec.replay()
    torch.cuda.synchronize()
    assert int((dec.status != 0).sum()) == 0
    assert np.array_equal(dec.out_len.cpu().numpy(), lengths.astype(np.int64))
    oracle_list_check(B, oracle, dec, kb, keys, None, small)
    sampled_check_large_ecb(B, oracle, dec, kb, keys, large, decrypt=True)
    # and the plaintext back, message by message on the device (offsets differ only by padding)
    src_off = enc.in_off.cpu().numpy()
    for m in large:
        ln, o, i = int(lengths[m]), int(dec.out_off_np[m]), int(src_off[m])
        assert torch.equal(dec.out[o: o + ln], enc.data[i: i + ln]), m


def test_full_size_small_messages_1M(torch, B, oracle):
    """1,000,000 messages of 16..1500 bytes, AES-128 CTR, keys expanded on the
    device, at the autotuned shape in a CUDA graph: every message compared
    whole with the oracle."""
    wl = W.small_messages(4, 1_000_000)
    lengths, kb, keys, ivs = wl["lengths"], wl["key_bits"], wl["keys"], wl["ivs"]
    b = build(B, torch, 0, lengths, kb, keys, ivs, seed=21)
    b.capture(B.autotune(b))
    b.replay()
    torch.cuda.synchronize()
    assert int((b.status != 0).sum()) == 0
    oracle_list_check(B, oracle, b, kb, keys, ivs, np.arange(b.n))


def test_batch_randomized_shapes(torch, B, oracle):
    """Seeded random trials over everything a caller controls: message count,
    length mix (empty to 70 KB, so every phase and tile boundary shows up),
    op, key sizes, counter starts, CTA size (both builds), tile size (kernel-
    sized or explicit), grid size and the padded flags.  Every message of
    every trial equals the oracle."""
    rng = np.random.default_rng(20261204)
    for trial in range(16):
        op = int(rng.integers(0, 3))
        n = int(rng.integers(1, 700))
        kind = rng.integers(0, 4, n)
        lengths = np.where(kind == 0, rng.integers(0, 64, n),
                           np.where(kind == 1, rng.integers(64, 2048, n),
                                    np.where(kind == 2, rng.integers(2048, 8192, n), rng.integers(8192, 70000, n))))
        lengths = lengths.astype(np.uint64)
        if op == 2:
            lengths = np.maximum((lengths // np.uint64(16)) * np.uint64(16), np.uint64(16))
        kb = np.array([128, 192, 256], np.uint32)[rng.integers(0, 3, n)]
        keys = rng.integers(0, 256, (n, 32)).astype(np.uint8)
        ivs = rng.integers(0, 256, (n, 16)).astype(np.uint8)
        cta = int(rng.choice([256, 384, 512, 640, 1024]))
        tile = int(rng.choice([0, cta, 4 * cta, 32 * cta]))
        grid = int(rng.choice([0, 1, 7, 152, 300]))
        padded = bool(rng.integers(0, 2))
        in_off, total = B.pack_offsets(lengths)
        data = synth.bytes_torch(900 + trial, synth.STREAM_DATA, max(total, 16), device="cuda")
        b = B.Batch(op, data, in_off, lengths, keys=keys, key_bits=kb, ivs=ivs if op == 0 else None,
                    padded=None if padded else False)
        b.submit(config=B.AesBatchConfig(cta, tile, grid, 0))
        torch.cuda.synchronize()
        oracle_check(B, oracle, b, kb, keys, ivs)
