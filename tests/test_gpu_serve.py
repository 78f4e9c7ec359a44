"""GPU tests of the continuous-batching server.

* each request's output, captured when its batch completes, equals the same
  request run alone through the single-buffer CTR call (and, for small ones,
  the CPU oracle): exact, 0 differing bytes;
* requests that arrive while batches are on the GPU are admitted and launched
  before those batches finish (continuous batching, several batches in
  flight);
* admission never charges more than the device-memory budget, and a budget
  much smaller than the offered load still completes every request.
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
    captured = {}

    def grab(r, view):
        if r.rid % 25 == 0:
            captured[r.rid] = (view.clone(), r.iv)

    srv.on_complete = grab
    rep = srv.run(arr, tenants, offs, lengths, time_limit=60.0)
    assert rep["completed"] == arr.size
    assert rep["p50_ms"] is not None and rep["p99_ms"] >= rep["p50_ms"]
    assert rep["batches"] > 1
    assert rep["batches_launched_while_previous_in_flight"] > 0
    check_alone(torch, oracle, srv, pool, keys, bits, captured, tenants, offs, lengths)


def test_admission_respects_a_tight_budget(torch, oracle):
    pool_bytes = 64 << 20
    budget = 4 << 20
    srv, pool, keys, bits = setup_server(torch, 8, pool_bytes, budget, seed=60, n_streams=2,
                                         slots_per_stream=2, max_batch_msgs=16)
    n = 400
    arr, offs, lengths = workload(8, n, pool_bytes, 1 << 20, rate=50000.0)
    tenants = W.tenants(8, arr.size, 8)
    captured = {}

    def grab(r, view):
        if r.rid % 20 == 0:
            captured[r.rid] = (view.clone(), r.iv)

    srv.on_complete = grab
    rep = srv.run(arr, tenants, offs, lengths, time_limit=60.0)
    assert rep["completed"] == arr.size
    assert rep["max_budget_charged"] <= budget
    check_alone(torch, oracle, srv, pool, keys, bits, captured, tenants, offs, lengths)


def test_tenant_counters_never_reuse_a_keystream_block(torch):
    srv, pool, keys, bits = setup_server(torch, 4, 16 << 20, 64 << 20, seed=70)
    arr = np.linspace(0, 0.01, 200)
    lengths = W.uniform_lengths(9, 200, 1, 5000)
    offs = np.zeros(200, dtype=np.uint64)
    tenants = np.arange(200) % 4
    ivs = {}

    def grab(r, view):
        ivs[r.rid] = (r.tenant, int.from_bytes(r.iv[12:], "big"), (r.length + 15) // 16)

    srv.on_complete = grab
    srv.run(arr, tenants, offs, lengths, time_limit=30.0)
    for t in range(4):
        ranges = sorted((c, c + nb) for (tt, c, nb) in ivs.values() if tt == t)
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 <= b0


class _NeverDone:
    """A completion event that never fires: a lost batch, injected on the host."""

    def query(self):
        return False


def test_lost_batch_times_out_without_hanging(torch):
    import time

    from paper_1403_7295_gb300.serve import Request

    srv, pool, keys, bits = setup_server(torch, 4, 16 << 20, 64 << 20, seed=80, batch_timeout_s=0.2)
    srv.arrive(Request(0, 1, 0, 4096, 0.0))
    srv.admit(0.0)
    assert srv.launch(0.0)
    slot = srv.inflight[0]
    torch.cuda.synchronize()
    slot.event = _NeverDone()  # the real work finished; the host never hears of it
    t0 = time.perf_counter()
    while srv.inflight and time.perf_counter() - t0 < 5.0:
        srv.poll(lambda: time.perf_counter() - t0 + 0.0)
    assert not srv.inflight and len(srv.timed_out) == 1 and not srv.healthy()
    assert srv.quarantined and srv.quarantined[0] is slot
    # the run loop stops admitting and returns instead of waiting forever
    arr = np.array([0.0, 0.001])
    rep = srv.run(arr, np.array([0, 1]), np.zeros(2, np.uint64), np.array([32, 32], np.uint64), time_limit=5.0)
    assert rep["completed"] == 0 and rep["timed_out"] == 1
