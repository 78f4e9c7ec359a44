"""Batched messages: marshalling for ``aes_batch_submit``, CUDA-graph replay
and the launch-shape autotuner.

Every AES step runs in the library's kernels; this module only lays out the
caller's messages in device arenas (16-byte aligned offsets), fills the
``aes_batch`` descriptor, captures the submit call into a CUDA graph, and
times candidate launch shapes.
"""
from __future__ import annotations

import ctypes
import json
import os
import time

import numpy as np

from . import aes as _aes

BATCH_CTR = 0
BATCH_ECB_PKCS7_ENCRYPT = 1
BATCH_ECB_PKCS7_DECRYPT = 2
IN_PADDED = 1   # AES_BATCH_IN_PADDED
OUT_PADDED = 2  # AES_BATCH_OUT_PADDED


class AesBatch(ctypes.Structure):
    """Mirror of ``aes_batch``."""
    _fields_ = [
        ("n_msgs", ctypes.c_uint32), ("op", ctypes.c_uint32),
        ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
        ("in_off", ctypes.c_void_p), ("in_len", ctypes.c_void_p), ("out_off", ctypes.c_void_p),
        ("keys", ctypes.c_void_p), ("key_bits", ctypes.c_void_p),
        ("schedules", ctypes.c_void_p), ("sched_idx", ctypes.c_void_p),
        ("n_schedules", ctypes.c_uint32), ("flags", ctypes.c_uint32),
        ("iv", ctypes.c_void_p), ("out_len", ctypes.c_void_p), ("status", ctypes.c_void_p),
    ]


SHORT_AUTO, SHORT_GROUPS, SHORT_LANES = 0, 1, 2  # AES_BATCH_SHORT_*


class AesBatchConfig(ctypes.Structure):
    """Mirror of ``aes_batch_config``; zero fields mean "library default"."""
    _fields_ = [("cta_threads", ctypes.c_int32), ("tile_blocks", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("short_path", ctypes.c_int32)]


def _declare():
    L = _aes.lib()
    if not getattr(L, "_batch_declared", False):
        L.aes_batch_workspace_size.argtypes = [ctypes.c_uint32]
        L.aes_batch_workspace_size.restype = ctypes.c_size_t
        L.aes_batch_submit.argtypes = [ctypes.POINTER(AesBatch), ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_void_p]
        L.aes_batch_submit.restype = ctypes.c_int
        L.aes_batch_submit_ex.argtypes = [ctypes.POINTER(AesBatch), ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p, ctypes.POINTER(AesBatchConfig)]
        L.aes_batch_submit_ex.restype = ctypes.c_int
        L._batch_declared = True
    return L


def aes_batch_workspace_size(n_msgs: int) -> int:
    return int(_declare().aes_batch_workspace_size(n_msgs))


def aes_batch_submit(desc: AesBatch, workspace, stream=None, config: AesBatchConfig | None = None):
    """Enqueue one batch (``workspace``: a device uint8 tensor)."""
    import torch

    L = _declare()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = L.aes_batch_submit_ex(ctypes.byref(desc), ctypes.c_void_p(workspace.data_ptr()),
                               workspace.numel(), ctypes.c_void_p(s.cuda_stream),
                               ctypes.byref(config) if config is not None else None)
    _aes._check(rc, "aes_batch_submit")


def output_capacity(op: int, lengths: np.ndarray) -> np.ndarray:
    """Bytes each message's output slot must hold."""
    lengths = np.asarray(lengths, dtype=np.uint64)
    if op == BATCH_ECB_PKCS7_ENCRYPT:
        return (lengths // np.uint64(16) + np.uint64(1)) * np.uint64(16)
    return lengths


def pack_offsets(sizes: np.ndarray) -> tuple[np.ndarray, int]:
    """16-byte aligned offsets for consecutive slots of the given sizes."""
    sizes = np.asarray(sizes, dtype=np.uint64)
    padded = (sizes + np.uint64(15)) // np.uint64(16) * np.uint64(16)
    offs = np.zeros(sizes.size, dtype=np.uint64)
    if sizes.size:
        offs[1:] = np.cumsum(padded)[:-1]
    total = int(padded.sum()) if sizes.size else 0
    return offs, total


class Batch:
    """Device-resident batch of messages plus its descriptor and workspace.

    ``data``: device uint8 arena holding the inputs at ``in_off``; ``lengths``
    per message; keys either raw (``keys`` [n,32] + ``key_bits``) or as
    indices into a device table of ``aes_key_schedule`` (``schedules`` +
    ``sched_idx``); ``ivs`` [n,16] for CTR.  The output arena is allocated
    here unless ``out`` is given.

    ``padded``: None (default) sets ``AES_BATCH_IN_PADDED`` when ``data``
    holds every message up to its next 16-byte boundary, and
    ``AES_BATCH_OUT_PADDED`` when the output arena is allocated here (its
    gaps belong to no one); False keeps every read and write exact to the
    byte; True asserts both for caller-given arenas.
    """

    def __init__(self, op: int, data, in_off, lengths, *, keys=None, key_bits=None,
                 schedules=None, n_schedules: int = 0, sched_idx=None, ivs=None, out=None,
                 out_off=None, device="cuda", padded: bool | None = None):
        import torch

        self.op = op
        self.n = int(np.asarray(lengths).size)
        dev = torch.device(device)

        def to_dev(a, dtype):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                return a.to(device=dev, dtype=dtype).contiguous()
            return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev, dtype=dtype)

        self.lengths_np = np.asarray(lengths, dtype=np.uint64)
        self.data = data
        self.in_off = to_dev(np.asarray(in_off, dtype=np.uint64).view(np.int64), torch.int64)
        self.in_len = to_dev(self.lengths_np.view(np.int64), torch.int64)
        cap = output_capacity(op, self.lengths_np)
        if out_off is None:
            out_off_np, total = pack_offsets(cap)
        else:
            out_off_np = np.asarray(out_off, dtype=np.uint64)
            total = int((out_off_np + cap).max()) if self.n else 0
        self.out_off_np = out_off_np
        self.out_off = to_dev(out_off_np.view(np.int64), torch.int64)
        self.out = out if out is not None else torch.empty(max(total, 16), dtype=torch.uint8, device=dev)
        self.keys = to_dev(keys, torch.uint8) if keys is not None else None
        self.key_bits = to_dev(np.asarray(key_bits, dtype=np.uint32).view(np.int32), torch.int32) \
            if key_bits is not None else None
        self.schedules = schedules
        self.n_schedules = n_schedules
        self.sched_idx = to_dev(np.asarray(sched_idx, dtype=np.uint32).view(np.int32), torch.int32) \
            if sched_idx is not None else None
        self.ivs = to_dev(ivs, torch.uint8) if ivs is not None else None
        self.out_len = torch.zeros(max(self.n, 1), dtype=torch.int64, device=dev)
        self.status = torch.zeros(max(self.n, 1), dtype=torch.int32, device=dev)
        self.workspace = torch.empty(aes_batch_workspace_size(self.n), dtype=torch.uint8, device=dev)
        if padded is None:
            in_off_np = np.asarray(in_off, dtype=np.uint64)
            ends = (in_off_np + self.lengths_np + np.uint64(15)) // np.uint64(16) * np.uint64(16)
            fits = self.n == 0 or int(ends.max()) <= data.numel() * data.element_size()
            self.flags = (IN_PADDED if fits else 0) | (OUT_PADDED if out is None else 0)
        else:
            self.flags = IN_PADDED | OUT_PADDED if padded else 0
        self.desc = self._descriptor()
        self.graph = None

    def _descriptor(self) -> AesBatch:
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        d = AesBatch()
        d.n_msgs = self.n
        d.op = self.op
        d.in_ = p(self.data)
        d.out = p(self.out)
        d.in_off, d.in_len, d.out_off = p(self.in_off), p(self.in_len), p(self.out_off)
        d.keys, d.key_bits = p(self.keys), p(self.key_bits)
        d.schedules = p(self.schedules)
        d.sched_idx = p(self.sched_idx)
        d.n_schedules = self.n_schedules
        d.flags = self.flags
        d.iv = p(self.ivs)
        d.out_len, d.status = p(self.out_len), p(self.status)
        return d

    def submit(self, stream=None, config: AesBatchConfig | None = None):
        aes_batch_submit(self.desc, self.workspace, stream, config)
        return self

    # -- CUDA graph: the memset and launches of one submit, captured once, replayed
    def capture(self, config: AesBatchConfig | None = None):
        import torch

        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.submit(s, config)  # warm-up outside the graph (lazy module load, smem opt-in)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.submit(torch.cuda.current_stream(), config)
        self.graph = g
        return self

    def replay(self):
        self.graph.replay()
        return self

    def total_input_bytes(self) -> int:
        return int(self.lengths_np.sum())


# ---------------------------------------------------------------------------
# autotuner: launch shapes of the persistent kernel, timed on the batch itself
# ---------------------------------------------------------------------------

CANDIDATES = [(cta, tile) for cta in (512, 1024) for tile in (0, 8192, 16384, 32768, 65536, 131072)
              if tile % cta == 0]  # tile 0: sized by the kernel from the batch
_CACHE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "batch_tune.json")


def _bucket(batch: Batch) -> str:
    import torch

    name = torch.cuda.get_device_name()
    n = batch.n
    mean = batch.total_input_bytes() / max(1, n)
    keys = "keys" if batch.keys is not None else "schedules"  # device expansion or resident schedules
    return f"{name}|op{batch.op}|{keys}|n2^{int(np.log2(max(n, 1)))}|mean2^{int(np.log2(max(mean, 1)))}"


def autotune(batch: Batch, reps: int = 3, use_cache: bool = True) -> AesBatchConfig:
    """Pick (cta_threads, tile_blocks, short_path) for this batch shape by
    CUDA-event timing (the short-message path only for CTR, the one op with
    two); the choice is cached per (GPU, op, message-count and mean-size
    bucket)."""
    import torch

    key = _bucket(batch)
    cache = {}
    if use_cache and os.path.exists(_CACHE_PATH):
        try:
            cache = json.load(open(_CACHE_PATH))
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache and len(cache[key]) == 3:
        cta, tile, path = cache[key]
        return AesBatchConfig(cta, tile, 0, path)
    paths = (SHORT_GROUPS, SHORT_LANES) if batch.op == BATCH_CTR else (SHORT_AUTO,)
    best, best_t = None, float("inf")
    for (cta, tile), path in [(c, p) for c in CANDIDATES for p in paths]:
        cfg = AesBatchConfig(cta, tile, 0, path)
        batch.submit(config=cfg)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            batch.submit(config=cfg)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        if t < best_t:
            best, best_t = (cta, tile, path), t
    cache[key] = list(best)
    try:
        os.makedirs(os.path.dirname(_CACHE_PATH), exist_ok=True)
        tmp = _CACHE_PATH + f".{os.getpid()}.{time.time_ns()}"
        json.dump(cache, open(tmp, "w"))
        os.replace(tmp, _CACHE_PATH)
    except OSError:
        pass
    return AesBatchConfig(best[0], best[1], 0, best[2])
