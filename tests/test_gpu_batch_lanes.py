"""GPU parity of the batch's lane path for short CTR messages
(AES_BATCH_SHORT_LANES: one lane per message, round keys in registers, data
staged through shared memory by TMA bulk copies): every message equals the
oracle run on that message alone, bit for bit.

Covers mixed key sizes (the three key-size classes of the sort); short and
long messages in one batch (the persistent kernel's tile phase and its
per-warp groups beside the lane kernel); lengths on every stage boundary of
8 blocks and on both sides of the 128-block limit of the lane path and of the
512-block split; ragged last blocks read and written byte-exactly
and as whole blocks; nothing written outside the messages; counters that
cross runs of 256 and wrap at 2^32; pre-expanded schedule tables; in-place
operation; one CTA and odd grid sizes; CUDA-graph replay; equality with the
per-warp group path on the same batch; the refusal of the lane path for
ECB; and no bounded wait giving up.
"""
import ctypes

import numpy as np
import pytest

import synth
from synth import workloads as W
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu

LANES = 2  # AES_BATCH_SHORT_LANES
GROUPS = 1


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.fixture(scope="module")
def B(torch):
    from paper_1403_7295_gb300 import batch

    return batch


def cfg(B, cta=1024, tile=0, grid=0, path=LANES):
    return B.AesBatchConfig(cta, tile, grid, path)


def build(B, op, lengths, key_bits, keys, ivs, seed, **kw):
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(seed, synth.STREAM_DATA, max(total, 16), device="cuda")
    return B.Batch(op, data, in_off, lengths, keys=keys, key_bits=key_bits, ivs=ivs, **kw)


def check(B, oracle, b, key_bits, keys, ivs, idx=None):
    data = b.data.cpu().numpy()
    out = b.out.cpu().numpy()
    out_len = b.out_len.cpu().numpy()
    status = b.status.cpu().numpy()
    in_off = b.in_off.cpu().numpy()
    for m in (range(b.n) if idx is None else idx):
        ln = int(b.lengths_np[m])
        bits = int(key_bits[m])
        io, oo = int(in_off[m]), int(b.out_off_np[m])
        want = oracle.ctr_xcrypt(keys[m][: bits // 8], bits, ivs[m], data[io: io + ln])
        assert status[m] == 0 and out_len[m] == ln, m
        assert np.array_equal(out[oo: oo + ln], want), m


def no_timeouts():
    from paper_1403_7295_gb300 import aes as A

    assert A.aes_take_wait_timeouts() == 0


# every stage boundary of 8 blocks up to 40 blocks, the 128-block limit of
# the lane path (longer short messages stay with the per-warp groups), the
# 511/512-block split, and a few long messages for the tile phase
EDGES = sorted({b * 16 + d for b in range(0, 41) for d in (-1, 0, 1) if b * 16 + d >= 0}
               | {127 * 16 - 1, 127 * 16, 127 * 16 + 1, 128 * 16, 128 * 16 + 1}
               | {511 * 16 - 1, 511 * 16, 511 * 16 + 1, 512 * 16, 512 * 16 + 1, 20000, 70001})


def edge_lengths(seed, n):
    rest = W.uniform_lengths(seed, max(n - len(EDGES), 0), 0, 8200)
    return np.concatenate([np.array(EDGES, np.uint64), rest]).astype(np.uint64)


@pytest.mark.parametrize("cta", [1024, 512])
def test_lanes_mixed_key_sizes_and_edges(torch, B, oracle, cta):
    n = 1500
    lengths = edge_lengths(3, n)
    kb = W.key_sizes(3, n)
    keys = W.message_keys(3, n)
    ivs = W.message_ivs(3, n)
    b = build(B, 0, lengths, kb, keys, ivs, seed=4).submit(config=cfg(B, cta))
    torch.cuda.synchronize()
    check(B, oracle, b, kb, keys, ivs)
    no_timeouts()


@pytest.mark.parametrize("padded", [False, True])
def test_lanes_exact_and_padded_last_blocks(torch, B, oracle, padded):
    """Flags 0: the ragged last block is read and written byte by byte and the
    16-byte gaps after the messages keep their canary; with both padded flags
    the same message bytes come out."""
    n = 900
    lengths = edge_lengths(5, n)
    kb = W.key_sizes(5, n)
    keys = W.message_keys(5, n)
    ivs = W.message_ivs(5, n, counter0=0xFFFFFF00)
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(6, synth.STREAM_DATA, total, device="cuda")  # exactly the packed size
    b = B.Batch(0, data, in_off, lengths, keys=keys, key_bits=kb, ivs=ivs, padded=None if padded else False)
    assert b.flags == (3 if padded else 0)
    b.out.fill_(0xA5)
    b.submit(config=cfg(B))
    torch.cuda.synchronize()
    check(B, oracle, b, kb, keys, ivs)
    if not padded:
        out = b.out.cpu().numpy()
        written = np.zeros(out.size, bool)
        for m in range(n):
            o = int(b.out_off_np[m])
            written[o: o + int(lengths[m])] = True
        assert np.all(out[~written] == 0xA5)


def test_lanes_counter_runs_and_wrap(torch, B, oracle):
    """Counters starting anywhere: messages cross runs of 256 counters at
    every position of a stage, and every 7th wraps at 2^32 after one block."""
    n = 4000
    lengths = W.uniform_lengths(7, n, 1, 8000)
    kb = W.key_sizes(7, n)
    keys = W.message_keys(7, n)
    ivs = synth.bytes_np(7, synth.STREAM_NONCE, 16 * n).reshape(n, 16)
    ivs[::7, 12:16] = 0xFF
    ivs[1::7, 12:16] = [0, 0, 0, 0xF9]  # run boundary after 7 blocks, inside the first stage
    b = build(B, 0, lengths, kb, keys, ivs, seed=8).submit(config=cfg(B))
    torch.cuda.synchronize()
    check(B, oracle, b, kb, keys, ivs)


def test_lanes_schedule_table(torch, B, oracle):
    """Pre-expanded schedules (keys == NULL): each lane loads its message's
    schedule from the device table."""
    from paper_1403_7295_gb300 import aes as A

    n = 800
    lengths = edge_lengths(9, n)
    kb = W.key_sizes(9, n)
    keys = W.message_keys(9, n)
    ivs = W.message_ivs(9, n)
    table = b"".join(bytes(A.aes_expand_key(keys[m][: int(kb[m]) // 8], int(kb[m]))) for m in range(n))
    table = torch.frombuffer(bytearray(table), dtype=torch.uint8).cuda()
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(10, synth.STREAM_DATA, max(total, 16), device="cuda")
    b = B.Batch(0, data, in_off, lengths, schedules=table, n_schedules=n, sched_idx=np.arange(n), ivs=ivs)
    b.submit(config=cfg(B))
    torch.cuda.synchronize()
    check(B, oracle, b, kb, keys, ivs)


def test_lanes_in_place(torch, B, oracle):
    """Output arena = input arena, same offsets: each stage's bulk store
    overwrites the blocks its bulk copy has already brought in."""
    n = 600
    lengths = edge_lengths(11, n)
    kb = W.key_sizes(11, n)
    keys = W.message_keys(11, n)
    ivs = W.message_ivs(11, n)
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(12, synth.STREAM_DATA, max(total, 16), device="cuda")
    src = data.cpu().numpy().copy()
    b = B.Batch(0, data, in_off, lengths, keys=keys, key_bits=kb, ivs=ivs, out=data, out_off=in_off)
    b.submit(config=cfg(B))
    torch.cuda.synchronize()
    out = data.cpu().numpy()
    for m in range(n):
        ln, o, bits = int(lengths[m]), int(in_off[m]), int(kb[m])
        assert np.array_equal(out[o: o + ln], oracle.ctr_xcrypt(keys[m][: bits // 8], bits, ivs[m], src[o: o + ln])), m


@pytest.mark.parametrize("grid", [1, 7, 300])
def test_lanes_grid_sizes(torch, B, oracle, grid):
    n = 700
    lengths = edge_lengths(13, n)
    kb = W.key_sizes(13, n)
    keys = W.message_keys(13, n)
    ivs = W.message_ivs(13, n)
    b = build(B, 0, lengths, kb, keys, ivs, seed=14).submit(config=cfg(B, grid=grid))
    torch.cuda.synchronize()
    check(B, oracle, b, kb, keys, ivs)


def test_lanes_single_and_degenerate_batches(torch, B, oracle):
    """One message; only empty messages; one short message among long ones;
    one key size only (two empty classes)."""
    cases = [np.array([37], np.uint64), np.array([0, 0, 0], np.uint64),
             np.array([9000, 100000, 33, 70000], np.uint64), np.full(64, 1500, np.uint64)]
    for i, lengths in enumerate(cases):
        n = lengths.size
        kb = np.full(n, 256, np.uint32) if i == 3 else W.key_sizes(20 + i, n)
        keys = W.message_keys(20 + i, n)
        ivs = W.message_ivs(20 + i, n)
        b = build(B, 0, lengths, kb, keys, ivs, seed=30 + i).submit(config=cfg(B))
        torch.cuda.synchronize()
        check(B, oracle, b, kb, keys, ivs)


def test_lanes_equal_groups_and_graph_replay(torch, B, oracle):
    """The lane path and the per-warp group path write the same arena on a
    20,000-message batch of packet-sized and longer messages; a CUDA graph of
    the lane path replays it identically."""
    n = 20000
    lengths = np.concatenate([W.uniform_lengths(40, n - 100, 16, 1500), W.uniform_lengths(41, 100, 2000, 40000)])
    kb = W.key_sizes(40, n)
    keys = W.message_keys(40, n)
    ivs = synth.bytes_np(40, synth.STREAM_NONCE, 16 * n).reshape(n, 16)
    b = build(B, 0, lengths, kb, keys, ivs, seed=42)
    b.out.fill_(0)
    b.submit(config=cfg(B, path=GROUPS))
    torch.cuda.synchronize()
    groups = b.out.clone()
    b.out.fill_(0)
    b.submit(config=cfg(B, path=LANES))
    torch.cuda.synchronize()
    assert torch.equal(b.out, groups)
    b.capture(cfg(B, path=LANES))
    for _ in range(2):
        b.out.fill_(0)
        b.replay()
        torch.cuda.synchronize()
        assert torch.equal(b.out, groups)
    check(B, oracle, b, kb, keys, ivs, idx=range(0, n, 37))
    no_timeouts()


def test_lanes_refused_for_ecb(torch, B):
    lengths = np.array([16, 32], np.uint64)
    b = build(B, 1, lengths, np.array([128, 128], np.uint32), W.message_keys(1, 2), None, seed=17)
    L = B._declare()
    c = cfg(B)
    assert L.aes_batch_submit_ex(ctypes.byref(b.desc), b.workspace.data_ptr(), b.workspace.numel(), None,
                                 ctypes.byref(c)) == 1
    c = cfg(B, path=3)
    assert L.aes_batch_submit_ex(ctypes.byref(b.desc), b.workspace.data_ptr(), b.workspace.numel(), None,
                                 ctypes.byref(c)) == 1


def test_lanes_by_default_on_large_ctr_batches(torch, B, oracle):
    """A CTR batch of 300,000 packet-sized messages submitted without a
    config (the library's choice: the lane path from 262,144 messages on)
    writes the same arena as the per-warp groups, and every message equals
    the oracle (the oracle's message list over all host threads)."""
    from tests.gpu_util import host_threads

    n = 300_000
    wl = W.small_messages(60, n)
    lengths, kb, keys, ivs = wl["lengths"], wl["key_bits"], wl["keys"], wl["ivs"]
    b = build(B, 0, lengths, kb, keys, ivs, seed=61)
    b.out.fill_(0)
    b.submit()
    torch.cuda.synchronize()
    auto = b.out.clone()
    b.out.fill_(0)
    b.submit(config=cfg(B, path=GROUPS))
    torch.cuda.synchronize()
    assert torch.equal(b.out, auto)
    in_off = b.in_off.cpu().numpy().astype(np.uint64)
    want = auto.cpu().numpy().copy()
    status = np.zeros(n, np.int32)
    oracle.batch(0, b.data.cpu().numpy(), in_off, lengths.astype(np.uint64), want.size,
                 b.out_off_np.astype(np.uint64), keys, kb.astype(np.uint32), ivs, nthreads=host_threads(), out=want)
    assert np.array_equal(want, auto.cpu().numpy())
    assert int((b.status != 0).sum()) == 0
    no_timeouts()

