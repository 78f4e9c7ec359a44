"""The multi-GPU path on CPU: world_size-2 `gloo` process groups.

Every GPU machine here has one GPU, so the N > 1 logic is tested on host ranks:
the shard planner (contiguous whole-block ranges, CTR IV advanced by the
range's first block) must make the union of per-rank results equal the
single-pass result, with no data exchange between ranks; the bench's
timing reduction (barrier, max over ranks) must pick the slowest rank.
Each rank computes its shard with the CPU oracle (test infrastructure).
"""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1403_7295_gb300.shard import ctr_iv_at, shard_ranges

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


@pytest.fixture(scope="module", autouse=True)
def library():
    """The shard IVs come from the library's aes_ctr_iv_advance (a host call:
    no GPU needed); build it once here, before the ranks start."""
    from paper_1403_7295_gb300 import build

    build.build()


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nbytes, results):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import Oracle

        o = Oracle()
        key = synth.key_bytes(5, 256)
        iv = synth.iv_bytes(5, counter0=0xFFFFFFF0)  # the counter wraps inside the buffer
        data = synth.bytes_np(5, synth.STREAM_DATA, nbytes)
        sh = shard_ranges(nbytes, world)[rank]
        mine = data[sh.byte_off: sh.byte_off + sh.byte_len]
        ctr = o.ctr_xcrypt(key, 256, np.frombuffer(ctr_iv_at(iv, sh.first_block), np.uint8), mine)
        whole_blocks = sh.byte_len - sh.byte_len % 16
        ecb = o.ecb_encrypt(key, 256, mine[:whole_blocks])
        # gather to every rank (the test's check; the data path itself exchanges nothing)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([ctr.size], dtype=torch.int64))
        maxn = int(max(s.item() for s in sizes))
        buf = torch.zeros(maxn, dtype=torch.uint8)
        buf[: ctr.size] = torch.from_numpy(ctr)
        bufs = [torch.zeros(maxn, dtype=torch.uint8) for _ in range(world)]
        dist.all_gather(bufs, buf)
        ebuf = torch.zeros(maxn, dtype=torch.uint8)
        ebuf[: ecb.size] = torch.from_numpy(ecb)
        ebufs = [torch.zeros(maxn, dtype=torch.uint8) for _ in range(world)]
        dist.all_gather(ebufs, ebuf)
        # the bench's timing reduction: barrier, then max over ranks
        elapsed = torch.tensor([10.0 + rank])
        dist.barrier()
        dist.all_reduce(elapsed, op=dist.ReduceOp.MAX)
        if rank == 0:
            parts = [bufs[r][: int(sizes[r].item())].numpy() for r in range(world)]
            eparts = []
            for r in range(world):
                s = shard_ranges(nbytes, world)[r]
                eparts.append(ebufs[r][: s.byte_len - s.byte_len % 16].numpy())
            results["ctr"] = np.concatenate(parts)
            results["ecb"] = np.concatenate(eparts)
            results["max_elapsed"] = float(elapsed.item())
    finally:
        dist.destroy_process_group()


def _run(world, nbytes):
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_worker, args=(world, port, nbytes, results), nprocs=world, join=True)
        return dict(results)


@pytest.mark.parametrize("nbytes", [16 * 4099 + 7, 16 * 64])
def test_two_rank_shards_equal_single_pass(oracle, nbytes):
    res = _run(2, nbytes)
    key = synth.key_bytes(5, 256)
    iv = synth.iv_bytes(5, counter0=0xFFFFFFF0)
    data = synth.bytes_np(5, synth.STREAM_DATA, nbytes)
    assert np.array_equal(res["ctr"], oracle.ctr_xcrypt(key, 256, iv, data))
    whole = nbytes - nbytes % 16
    assert np.array_equal(res["ecb"], oracle.ecb_encrypt(key, 256, data[:whole]))
    assert res["max_elapsed"] == 11.0


def test_shard_ranges_cover_the_buffer():
    for nbytes in (0, 15, 16, 17, 16 * 1000 + 3, 1 << 20):
        for world in (1, 2, 3, 8):
            sh = shard_ranges(nbytes, world)
            assert len(sh) == world
            pos = 0
            for s in sh:
                assert s.byte_off == pos and s.byte_off % 16 == 0 and s.first_block * 16 == s.byte_off
                pos += s.byte_len
            assert pos == nbytes
    assert ctr_iv_at(bytes(12) + b"\xff\xff\xff\xff", 2)[12:] == b"\x00\x00\x00\x01"
    with pytest.raises(ValueError):
        shard_ranges(16, 0)
