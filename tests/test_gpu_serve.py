"""GPU tests of the native continuous-batching server (aes_server_*).

* each request's output, captured when its batch completes, equals the same
  request run alone through the single-buffer CTR call (and, for small ones,
  the CPU oracle): exact, 0 differing bytes;
* requests that arrive while batches are on the GPU are admitted and launched
  before those batches finish (continuous batching, several batches in
  flight);
* admission never charges more than the device-memory budget, and a budget
  much smaller than the offered load still completes every request;
* tenant counters never reuse a keystream block; a lost batch (injected on
  the host) times out without hanging and stops admission;
* the online submit / progress API reports every request with its output.
"""
import numpy as np
import pytest

import synth
from synth import workloads as W
from tests.gpu_util import require_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


def setup_server(torch, n_tenants, pool_bytes, budget, seed=50, **kw):
    from paper_1403_7295_gb300.serve import Server

    pool = synth.bytes_torch(seed, synth.STREAM_DATA, pool_bytes, device="cuda")
    keys = W.message_keys(seed + 1, n_tenants)
    bits = W.key_sizes(seed + 1, n_tenants)
    bits[: n_tenants // 2] = 256
    nonces = synth.bytes_np(seed + 2, synth.STREAM_NONCE, 12 * n_tenants).reshape(n_tenants, 12)
    srv = Server(pool, keys, bits, nonces, budget_bytes=budget, **kw)
    return srv, pool, keys, bits


def workload(seed, n, pool_bytes, max_len, rate):
    arr = W.poisson_arrivals(seed, rate, n / rate * 1.5)[:n]
    n = arr.size
    lengths = np.minimum(W.serving_sizes(seed, n), max_len).astype(np.uint64)
    u = synth.uniform01(seed, synth.STREAM_MISC + 3, n)
    offs = (np.floor(u * (pool_bytes - lengths.astype(np.float64))).astype(np.uint64) // 16) * 16
    return arr, offs, lengths


def check_alone(torch, oracle, srv, pool, keys, bits, captured, tenants, offs, lengths, n_oracle=6):
    from paper_1403_7295_gb300 import aes as A

    assert captured
    checked = 0
    for rid, (out, iv) in captured.items():
        t = int(tenants[rid])
        ks = A.aes_expand_key(keys[t][: bits[t] // 8], int(bits[t]))
        o, ln = int(offs[rid]), int(lengths[rid])
        alone = A.aes_ctr_xcrypt(ks, iv, pool[o: o + ln])
        torch.cuda.synchronize()
        assert torch.equal(alone, out), rid
        if checked < n_oracle and ln <= 64 << 10:
            want = oracle.ctr_xcrypt(keys[t][: bits[t] // 8], int(bits[t]), np.frombuffer(iv, np.uint8),
                                     pool[o: o + ln].cpu().numpy())
            assert np.array_equal(out.cpu().numpy(), want), rid
            checked += 1
    assert checked > 0


def test_serving_results_equal_alone_and_batches_overlap(torch, oracle):
    pool_bytes = 256 << 20
    srv, pool, keys, bits = setup_server(torch, 64, pool_bytes, 1 << 30, n_streams=2,
                                         slots_per_stream=2, max_batch_msgs=128)
    n = 3000
    arr, offs, lengths = workload(7, n, pool_bytes, 4 << 20, rate=20000.0)
    tenants = W.tenants(7, arr.size, 64)
    rep = srv.run(arr, tenants, offs, lengths, time_limit=60.0, capture=range(0, arr.size, 25))
    assert rep["completed"] == arr.size
    assert rep["p50_ms"] is not None and rep["p99_ms"] >= rep["p50_ms"]
    assert rep["batches"] > 1
    assert rep["batches_launched_while_previous_in_flight"] > 0
    check_alone(torch, oracle, srv, pool, keys, bits, rep["captured"], tenants, offs, lengths)


def test_admission_respects_a_tight_budget(torch, oracle):
    pool_bytes = 64 << 20
    budget = 4 << 20
    srv, pool, keys, bits = setup_server(torch, 8, pool_bytes, budget, seed=60, n_streams=2,
                                         slots_per_stream=2, max_batch_msgs=16)
    n = 400
    arr, offs, lengths = workload(8, n, pool_bytes, 1 << 20, rate=50000.0)
    tenants = W.tenants(8, arr.size, 8)
    rep = srv.run(arr, tenants, offs, lengths, time_limit=60.0, capture=range(0, arr.size, 20))
    assert rep["completed"] == arr.size
    assert rep["max_budget_charged"] <= budget
    check_alone(torch, oracle, srv, pool, keys, bits, rep["captured"], tenants, offs, lengths)


def test_tenant_counters_never_reuse_a_keystream_block(torch):
    srv, pool, keys, bits = setup_server(torch, 4, 16 << 20, 64 << 20, seed=70)
    arr = np.linspace(0, 0.01, 200)
    lengths = W.uniform_lengths(9, 200, 1, 5000)
    offs = np.zeros(200, dtype=np.uint64)
    tenants = np.arange(200) % 4
    rep = srv.run(arr, tenants, offs, lengths, time_limit=30.0)
    assert rep["completed"] == 200
    ctr = rep["counters"]
    for t in range(4):
        ranges = sorted((int(ctr[i]), int(ctr[i]) + (int(lengths[i]) + 15) // 16) for i in range(200) if tenants[i] == t)
        assert ranges[0][0] == 0
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0  # consecutive, never overlapping


def test_lost_batch_times_out_without_hanging(torch):
    """The first batch is declared lost on the host (its GPU work runs; the
    server is told its completion never comes): after the bounded wait its
    request fails with a timeout, admission stops, and the replay returns."""
    import time

    srv, pool, keys, bits = setup_server(torch, 4, 16 << 20, 64 << 20, seed=80, batch_timeout_s=0.2,
                                         inject_lost_batch=1)
    t0 = time.perf_counter()
    arr = np.array([0.0, 0.5])  # the second request arrives after the first batch was declared lost
    rep = srv.run(arr, np.array([0, 1]), np.zeros(2, np.uint64), np.array([4096, 32], np.uint64), time_limit=5.0)
    assert time.perf_counter() - t0 < 5.0
    assert rep["completed"] == 0 and rep["timed_out"] == 1
    assert not srv.healthy()


def test_online_submit_and_progress(torch, oracle):
    from paper_1403_7295_gb300 import aes as A

    srv, pool, keys, bits = setup_server(torch, 3, 8 << 20, 32 << 20, seed=90, max_batch_msgs=4)
    lengths = [1, 15, 16, 17, 4096, 100000, 7, 65536, 3, 12345]
    offs = [(i * 700000) // 16 * 16 for i in range(len(lengths))]
    for i, (o, ln) in enumerate(zip(offs, lengths)):
        srv.submit(1000 + i, i % 3, o, ln)
    seen = {}
    for _ in range(100000):
        for c in srv.progress(max_done=3):
            assert c.status == 0
            out = srv.output()[c.out_off: c.out_off + c.length].clone()
            seen[c.id] = (out, srv.iv(c.tenant, c.counter), c.t_done >= c.t_admitted >= c.t_arrival)
        if srv.idle():
            break
    assert sorted(seen) == [1000 + i for i in range(len(lengths))]
    torch.cuda.synchronize()
    for i, (o, ln) in enumerate(zip(offs, lengths)):
        out, iv, ordered = seen[1000 + i]
        t = i % 3
        assert ordered
        ks = A.aes_expand_key(keys[t][: bits[t] // 8], int(bits[t]))
        assert torch.equal(out, A.aes_ctr_xcrypt(ks, iv, pool[o: o + ln])), i
    st = srv.stats()
    assert st["completed"] == len(lengths) and st["batches"] >= 3
