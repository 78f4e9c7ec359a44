"""Continuous-batching AES-CTR server: Python binding of the library's native
serving engine (``aes_server_*`` in include/aesgpu.h, csrc/aes_serve.cu).

Requests (tenant, input slice of a device pool, length) arrive over time.
The engine admits them in arrival order against a device-memory budget
(input + output bytes; outputs in a ring arena), launches every admitted
request into the next batch as soon as one of its in-flight slots is free
(continuous batching over several streams), reports completions by event,
and declares a batch lost after a bounded wait (its requests fail with a
timeout, its slot and output bytes are quarantined, admission stops).  Each
tenant has a resident key schedule, a fixed nonce and a running 32-bit block
counter, so no keystream block repeats within a tenant.

This module only marshals arguments: the loop itself (admission, batching,
launch, completion, timeouts) runs in the library, and every AES step in its
batch kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import aes as _aes


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("n_streams", ctypes.c_uint32),
                ("slots_per_stream", ctypes.c_uint32), ("max_batch_msgs", ctypes.c_uint32),
                ("grid_ctas", ctypes.c_int32), ("batch_timeout_s", ctypes.c_double),
                ("inject_lost_batch", ctypes.c_uint64)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("tenant", ctypes.c_uint32),
                ("out_off", ctypes.c_uint64), ("length", ctypes.c_uint64), ("counter", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("t_arrival", ctypes.c_double), ("t_admitted", ctypes.c_double),
                ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("timed_out", ctypes.c_uint64),
                ("batches", ctypes.c_uint64), ("batches_overlapped", ctypes.c_uint64), ("bytes", ctypes.c_uint64),
                ("max_charged", ctypes.c_uint64), ("mean_batch_msgs", ctypes.c_double)]


def _declare():
    L = _aes.lib()
    if not getattr(L, "_serve_declared", False):
        vp, u64, u32, dp = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)
        L.aes_server_create.argtypes = [ctypes.POINTER(ServerConfig), vp, u64, vp, vp, u32, ctypes.POINTER(vp)]
        L.aes_server_create.restype = ctypes.c_int
        L.aes_server_destroy.argtypes = [vp]
        L.aes_server_destroy.restype = None
        L.aes_server_submit.argtypes = [vp, u64, u32, u64, u64]
        L.aes_server_submit.restype = ctypes.c_int
        L.aes_server_progress.argtypes = [vp, ctypes.POINTER(Completion), u32, ctypes.POINTER(ctypes.c_int)]
        L.aes_server_progress.restype = u32
        L.aes_server_healthy.argtypes = [vp]
        L.aes_server_healthy.restype = ctypes.c_int
        L.aes_server_idle.argtypes = [vp]
        L.aes_server_idle.restype = ctypes.c_int
        L.aes_server_output.argtypes = [vp]
        L.aes_server_output.restype = vp
        L.aes_server_now.argtypes = [vp]
        L.aes_server_now.restype = ctypes.c_double
        L.aes_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.aes_server_get_stats.restype = None
        L.aes_server_replay.argtypes = [vp, u64, dp, vp, vp, vp, ctypes.c_double, dp, dp, vp, vp, vp]
        L.aes_server_replay.restype = ctypes.c_int
        L._serve_declared = True
    return L


class Server:
    """AES-CTR serving engine with resident tenant key schedules."""

    def __init__(self, pool, tenant_keys: np.ndarray, tenant_bits: np.ndarray, tenant_nonces: np.ndarray,
                 budget_bytes: int = 8 << 30, n_streams: int = 2, slots_per_stream: int = 2,
                 max_batch_msgs: int = 8192, grid_ctas: int = 0, batch_timeout_s: float = 10.0,
                 inject_lost_batch: int = 0, device="cuda"):
        import torch

        self.torch = torch
        self.pool = pool  # device uint8 tensor holding every request's input
        n_t = tenant_keys.shape[0]
        table = bytearray()
        for t in range(n_t):
            bits = int(tenant_bits[t])
            table += bytes(_aes.aes_expand_key(tenant_keys[t][: bits // 8], bits))
        self._table = (ctypes.c_uint8 * len(table)).from_buffer(table)
        self.nonces = np.ascontiguousarray(np.asarray(tenant_nonces, dtype=np.uint8).reshape(n_t, 12))
        self.n_tenants = n_t
        self.budget = budget_bytes
        cfg = ServerConfig(budget_bytes, n_streams, slots_per_stream, max_batch_msgs, grid_ctas,
                           batch_timeout_s, inject_lost_batch)
        self._L = _declare()
        h = ctypes.c_void_p()
        rc = self._L.aes_server_create(ctypes.byref(cfg), pool.data_ptr(), pool.numel(), ctypes.addressof(self._table),
                                       self.nonces.ctypes.data, n_t, ctypes.byref(h))
        _aes._check(rc, "aes_server_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.aes_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # ---- online use ----
    def submit(self, rid: int, tenant: int, in_off: int, length: int) -> None:
        _aes._check(self._L.aes_server_submit(self._h, rid, tenant, in_off, length), "aes_server_submit")

    def progress(self, max_done: int = 4096) -> list:
        """One pass of the loop; the completions it reports (their outputs stay
        readable through output() until the next call)."""
        buf = (Completion * max_done)()
        st = ctypes.c_int(0)
        k = self._L.aes_server_progress(self._h, buf, max_done, ctypes.byref(st))
        _aes._check(st.value, "aes_server_progress")
        return [buf[i] for i in range(k)]

    def output(self):
        """The output arena as a device uint8 tensor (budget bytes)."""
        ptr = self._L.aes_server_output(self._h)

        class _Arena:
            __cuda_array_interface__ = {"shape": (self.budget,), "typestr": "|u1", "data": (ptr, False),
                                        "version": 3}

        return self.torch.as_tensor(_Arena(), device="cuda")

    def healthy(self) -> bool:
        """False once a batch was declared lost: admission has stopped."""
        return bool(self._L.aes_server_healthy(self._h))

    def idle(self) -> bool:
        return bool(self._L.aes_server_idle(self._h))

    def stats(self) -> dict:
        st = ServerStats()
        self._L.aes_server_get_stats(self._h, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def iv(self, tenant: int, counter: int) -> bytes:
        return bytes(self.nonces[tenant]) + int(counter).to_bytes(4, "big")

    # ---- driving a recorded workload in real time ----
    def run(self, arrivals: np.ndarray, tenants: np.ndarray, in_offs: np.ndarray, lengths: np.ndarray,
            time_limit: float | None = None, capture=None) -> dict:
        """Replay an arrival schedule (seconds from start) in real time in the
        library.  ``capture``: request indices whose outputs are copied out as
        they complete (returned under "captured" as rid -> (tensor, iv))."""
        torch = self.torch
        n = int(np.asarray(arrivals).size)
        arr = np.ascontiguousarray(arrivals, dtype=np.float64)
        ten = np.ascontiguousarray(tenants, dtype=np.uint32)
        offs = np.ascontiguousarray(in_offs, dtype=np.uint64)
        lens = np.ascontiguousarray(lengths, dtype=np.uint64)
        lat = np.full(n, -1.0)
        wait = np.full(n, -1.0)
        ctrs = np.zeros(n, dtype=np.uint32)
        cap_buf, cap_off = None, None
        capture = sorted(set(int(i) for i in capture)) if capture is not None else []
        if capture:
            cap_off = np.full(n, np.iinfo(np.uint64).max, dtype=np.uint64)
            pos = 0
            for i in capture:
                cap_off[i] = pos
                pos += (int(lens[i]) + 15) // 16 * 16
            cap_buf = torch.empty(max(pos, 16), dtype=torch.uint8, device="cuda")
        limit = time_limit if time_limit is not None else (float(arr[-1]) + 60.0 if n else 1.0)
        dptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
        t0 = self._L.aes_server_now(self._h)
        rc = self._L.aes_server_replay(self._h, n, dptr(arr), ten.ctypes.data, offs.ctypes.data, lens.ctypes.data,
                                       limit, dptr(lat), dptr(wait), ctrs.ctypes.data,
                                       cap_buf.data_ptr() if cap_buf is not None else None,
                                       cap_off.ctypes.data if cap_off is not None else None)
        wall = self._L.aes_server_now(self._h) - t0
        _aes._check(rc, "aes_server_replay")
        st = self.stats()
        ok = lat >= 0
        rep = {
            "requests": n, "completed": int(ok.sum()), "bytes": int(lens[ok].sum()), "wall_s": wall,
            "gbps": float(lens[ok].sum()) / wall / 1e9 if wall > 0 else 0.0,
            "p50_ms": float(np.percentile(lat[ok], 50) * 1e3) if ok.any() else None,
            "p99_ms": float(np.percentile(lat[ok], 99) * 1e3) if ok.any() else None,
            "max_ms": float(lat[ok].max() * 1e3) if ok.any() else None,
            "admission_wait_p99_ms": float(np.percentile(wait[ok], 99) * 1e3) if ok.any() else None,
            "admission_wait_mean_ms": float(wait[ok].mean() * 1e3) if ok.any() else None,
            "admission_wait_max_ms": float(wait[ok].max() * 1e3) if ok.any() else None,
            "batches": st["batches"], "mean_batch_msgs": st["mean_batch_msgs"],
            "batches_launched_while_previous_in_flight": st["batches_overlapped"],
            "max_budget_charged": st["max_charged"], "budget": self.budget,
            "timed_out": int((lat == -2.0).sum()),
            "counters": ctrs,
        }
        if capture:
            rep["captured"] = {i: (cap_buf[int(cap_off[i]): int(cap_off[i]) + int(lens[i])],
                                   self.iv(int(ten[i]), int(ctrs[i])))
                               for i in capture if lat[i] >= 0}
        return rep
