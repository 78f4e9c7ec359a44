"""Continuous-batching AES server over ``aes_batch_submit``.

Requests (tenant, input slice, length) arrive over time.  The loop:

1. **admits** arrived requests in arrival order while the device-memory
   budget allows (each request is charged its input and output bytes; its
   output slot comes from a ring arena of the budget's size).  A request that
   does not fit waits; nothing is ever allocated past the budget;
2. **batches** every admitted, not yet launched request into the next batch
   as soon as an in-flight slot is free, so requests that arrive while other
   batches are on the GPU join the next launch (continuous batching, not a
   queue drained one batch at a time);
3. **launches** the batch on one of several streams: descriptor arrays go
   through a pinned staging buffer with one async copy, then the batch call
   (tenant key schedules and per-tenant counters stay resident; each batch
   uses part of the GPU, so consecutive batches run concurrently);
4. **completes** batches whose event has fired, stamps each request's
   completion time and frees its budget.

CTR counters: each tenant has a fixed random nonce and a running 32-bit
block counter; a request gets IV = nonce || counter and advances the counter
by its block count, so no keystream block repeats within a tenant until
2^32 blocks.

Every AES step runs in the library's kernels; this module is scheduling,
bookkeeping and argument marshalling.
"""
from __future__ import annotations

import collections
import gc
import time
from dataclasses import dataclass

import numpy as np

from . import aes as _aes
from . import batch as _batch

ALIGN = 16


def _up16(x: int) -> int:
    return (x + 15) & ~15


class RingArena:
    """Byte ranges of one device buffer handed out in FIFO order.

    ``alloc`` returns an offset or None when the bytes are not free;
    ``free`` may come out of order (batches on different streams), the tail
    advances over every freed range at the front.
    """

    def __init__(self, size: int):
        self.size = size
        self.head = 0
        self.live = collections.deque()  # [start, size, freed]
        self.used = 0

    def _tail(self) -> int:
        return self.live[0][0] if self.live else self.head

    def alloc(self, nbytes: int):
        n = max(_up16(nbytes), ALIGN)
        if n > self.size:
            return None
        tail = self._tail()
        if not self.live:
            self.head = 0
            tail = 0
        if self.head >= tail and self.live:
            if self.head + n <= self.size:
                start = self.head
            elif n < tail:  # wrap; strict so head != tail while live
                start = 0
            else:
                return None
        elif self.live:
            if self.head + n < tail:
                start = self.head
            else:
                return None
        else:
            start = 0
        entry = [start, n, False]
        self.live.append(entry)
        self.head = start + n
        self.used += n
        return entry

    def free(self, entry):
        entry[2] = True
        self.used -= entry[1]
        while self.live and self.live[0][2]:
            self.live.popleft()


@dataclass
class Request:
    rid: int
    tenant: int
    in_off: int
    length: int
    arrival: float
    admitted: float = -1.0
    done: float = -1.0
    out_entry: list | None = None
    iv: bytes = b""


class _Slot:
    """Per in-flight batch: pinned + device descriptor buffers, workspace, event."""

    FIELDS = (("in_off", 8), ("in_len", 8), ("out_off", 8), ("out_len", 8), ("sched_idx", 4),
              ("status", 4), ("iv", 16))

    def __init__(self, torch, max_msgs: int, device):
        self.max = max_msgs
        self.offsets = {}
        off = 0
        for name, width in self.FIELDS:
            self.offsets[name] = off
            off = _up16(off + width * max_msgs)
        self.nbytes = off
        self.host = torch.empty(off, dtype=torch.uint8).pin_memory()
        self.host_np = self.host.numpy()
        self.dev = torch.empty(off, dtype=torch.uint8, device=device)
        self.ws = torch.empty(_batch.aes_batch_workspace_size(max_msgs), dtype=torch.uint8, device=device)
        self.event = torch.cuda.Event()
        self.reqs: list[Request] = []
        self.stream = None
        self.t_launch = 0.0

    def view(self, name, dtype, n):
        o = self.offsets[name]
        w = np.dtype(dtype).itemsize
        return self.host_np[o: o + w * n].view(dtype)

    def dptr(self, name) -> int:
        return self.dev.data_ptr() + self.offsets[name]


class Server:
    """AES-CTR serving loop with resident tenant key schedules."""

    def __init__(self, pool, tenant_keys: np.ndarray, tenant_bits: np.ndarray, tenant_nonces: np.ndarray,
                 budget_bytes: int = 8 << 30, n_streams: int = 2, slots_per_stream: int = 2,
                 max_batch_msgs: int = 8192, grid_ctas: int = 0, batch_timeout_s: float = 10.0,
                 device="cuda"):
        import torch

        self.torch = torch
        self.pool = pool  # device uint8 tensor holding every request's input
        n_t = tenant_keys.shape[0]
        table = bytearray()
        for t in range(n_t):
            bits = int(tenant_bits[t])
            table += bytes(_aes.aes_expand_key(tenant_keys[t][: bits // 8], bits))
        self.schedules = torch.frombuffer(table, dtype=torch.uint8).to(device)
        self.n_tenants = n_t
        self.nonces = np.asarray(tenant_nonces, dtype=np.uint8).reshape(n_t, 12)
        self.counters = np.zeros(n_t, dtype=np.uint64)
        self.budget = budget_bytes
        self.charged = 0
        self.max_charged = 0
        self.arena = RingArena(budget_bytes)
        self.out = torch.empty(budget_bytes, dtype=torch.uint8, device=device)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_streams)]
        self.free_slots = collections.deque(
            _Slot(torch, max_batch_msgs, device) for _ in range(n_streams * slots_per_stream))
        self.inflight: collections.deque[_Slot] = collections.deque()
        self.waiting: collections.deque[Request] = collections.deque()   # arrived, not admitted
        self.admitted: collections.deque[Request] = collections.deque()  # admitted, not launched
        self.completed: list[Request] = []
        self.grid = grid_ctas
        self.next_stream = 0
        self.batches = []  # (t_launch, t_done, n_reqs, bytes, stream index)
        self.on_complete = None  # optional callback(request, out_view) at completion
        # Bounded wait: a batch not complete after batch_timeout_s is declared
        # lost; its requests fail with a timeout and its slot and output bytes
        # are quarantined (never reused: the GPU might still write them).
        self.batch_timeout_s = batch_timeout_s
        self.timed_out: list[Request] = []
        self.quarantined: list[_Slot] = []

    # ---- request flow ----
    def arrive(self, req: Request):
        self.waiting.append(req)

    def admit(self, now: float):
        while self.waiting:
            r = self.waiting[0]
            cost = 2 * _up16(r.length)  # input + output bytes
            if self.charged + cost > self.budget:
                break
            entry = self.arena.alloc(r.length)
            if entry is None:
                break
            self.waiting.popleft()
            self.charged += cost
            self.max_charged = max(self.max_charged, self.charged)
            r.out_entry = entry
            r.admitted = now
            nb = (r.length + 15) // 16
            c = int(self.counters[r.tenant])
            r.iv = bytes(self.nonces[r.tenant]) + (c % (1 << 32)).to_bytes(4, "big")
            self.counters[r.tenant] = c + nb
            self.admitted.append(r)

    def launch(self, now: float) -> bool:
        if not self.admitted or not self.free_slots:
            return False
        slot = self.free_slots.popleft()
        reqs = []
        while self.admitted and len(reqs) < slot.max:
            reqs.append(self.admitted.popleft())
        n = len(reqs)
        slot.view("in_off", np.uint64, n)[:] = [r.in_off for r in reqs]
        slot.view("in_len", np.uint64, n)[:] = [r.length for r in reqs]
        slot.view("out_off", np.uint64, n)[:] = [r.out_entry[0] for r in reqs]
        slot.view("sched_idx", np.uint32, n)[:] = [r.tenant for r in reqs]
        slot.view("iv", np.uint8, 16 * n)[:] = np.frombuffer(b"".join(r.iv for r in reqs), np.uint8)
        torch = self.torch
        s = self.streams[self.next_stream]
        self.next_stream = (self.next_stream + 1) % len(self.streams)
        with torch.cuda.stream(s):
            # one async copy of the used part of the staging buffer (the iv field is last)
            end = slot.offsets["iv"] + 16 * n
            slot.dev[:end].copy_(slot.host[:end], non_blocking=True)
            d = _batch.AesBatch()
            d.n_msgs = n
            d.op = _batch.BATCH_CTR
            d.in_ = self.pool.data_ptr()
            d.out = self.out.data_ptr()
            d.in_off, d.in_len = slot.dptr("in_off"), slot.dptr("in_len")
            d.out_off = slot.dptr("out_off")
            d.schedules = self.schedules.data_ptr()
            d.sched_idx = slot.dptr("sched_idx")
            d.n_schedules = self.n_tenants
            # outputs sit in 16-byte-rounded ring allocations; inputs may be read
            # to their next 16-byte boundary when the pool holds it
            pool_bytes = self.pool.numel()
            d.flags = _batch.OUT_PADDED | (_batch.IN_PADDED if all(
                (r.in_off + r.length + 15) // 16 * 16 <= pool_bytes for r in reqs) else 0)
            d.iv = slot.dptr("iv")
            d.out_len, d.status = slot.dptr("out_len"), slot.dptr("status")
            cfg = _batch.AesBatchConfig(0, 0, self.grid, 0) if self.grid else None
            _batch.aes_batch_submit(d, slot.ws, s, cfg)
            slot.event.record(s)
        slot.reqs = reqs
        slot.stream = self.streams.index(s)
        slot.t_launch = now
        self.inflight.append(slot)
        return True

    def poll(self, now_fn) -> int:
        done = 0
        for slot in list(self.inflight):
            if not slot.event.query():
                t = now_fn()
                if t - slot.t_launch > self.batch_timeout_s:
                    self.inflight.remove(slot)
                    self.quarantined.append(slot)
                    for r in slot.reqs:
                        r.done = -2.0  # timed out
                        self.timed_out.append(r)
                continue
            t = now_fn()
            self.inflight.remove(slot)
            nbytes = 0
            for r in slot.reqs:
                r.done = t
                if self.on_complete is not None:
                    self.on_complete(r, self.out[r.out_entry[0]: r.out_entry[0] + r.length])
                self.arena.free(r.out_entry)
                self.charged -= 2 * _up16(r.length)
                nbytes += r.length
                self.completed.append(r)
            self.batches.append((slot.t_launch, t, len(slot.reqs), nbytes, slot.stream))
            slot.reqs = []
            self.free_slots.append(slot)
            done += 1
        return done

    def idle(self) -> bool:
        return not (self.waiting or self.admitted or self.inflight)

    def healthy(self) -> bool:
        """False once a batch has timed out: stop admitting and report."""
        return not self.quarantined

    # ---- driving a recorded workload in real time ----
    def run(self, arrivals: np.ndarray, tenants: np.ndarray, in_offs: np.ndarray, lengths: np.ndarray,
            time_limit: float | None = None) -> dict:
        """Replay an arrival schedule (seconds from start) in real time."""
        n = arrivals.size
        reqs = [Request(i, int(tenants[i]), int(in_offs[i]), int(lengths[i]), float(arrivals[i]))
                for i in range(n)]
        # The loop allocates many small objects; a generational collection in
        # the middle of it would stall admission and completion for tens of ms.
        gc_was_enabled = gc.isenabled()
        gc.collect()
        gc.disable()
        t0 = time.perf_counter()
        now_fn = lambda: time.perf_counter() - t0  # noqa: E731
        i = 0
        limit = time_limit if time_limit is not None else float(arrivals[-1]) + 60.0 if n else 1.0
        while True:
            now = now_fn()
            while i < n and reqs[i].arrival <= now:
                self.arrive(reqs[i])
                i += 1
            if self.healthy():
                self.admit(now)
                while self.launch(now):
                    pass
            self.poll(now_fn)
            if i >= n and self.idle():
                break
            if not self.healthy() and not self.inflight:
                break  # a batch was lost: report instead of waiting forever
            if now > limit:
                break
        self.torch.cuda.synchronize()
        wall = now_fn()
        if gc_was_enabled:
            gc.enable()
        return self.report(reqs, wall)

    def report(self, reqs, wall: float) -> dict:
        lat = np.array([r.done - r.arrival for r in reqs if r.done >= 0])
        wait = np.array([r.admitted - r.arrival for r in reqs if r.done >= 0])
        nbytes = sum(r.length for r in reqs if r.done >= 0)
        overlap = 0
        b = sorted(self.batches)
        for k in range(1, len(b)):
            if b[k][0] < b[k - 1][1]:  # launched before the previous batch completed
                overlap += 1
        return {
            "requests": len(reqs), "completed": int(lat.size), "bytes": int(nbytes), "wall_s": wall,
            "gbps": nbytes / wall / 1e9 if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat, 50) * 1e3) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99) * 1e3) if lat.size else None,
            "max_ms": float(lat.max() * 1e3) if lat.size else None,
            "admission_wait_p99_ms": float(np.percentile(wait, 99) * 1e3) if wait.size else None,
            "batches": len(self.batches),
            "mean_batch_msgs": float(np.mean([x[2] for x in self.batches])) if self.batches else 0.0,
            "batches_launched_while_previous_in_flight": overlap,
            "max_budget_charged": int(self.max_charged), "budget": int(self.budget),
            "timed_out": len(self.timed_out),
        }
