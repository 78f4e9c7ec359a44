"""Seeded workload recipes (sizes, length mixes, keys, IVs, arrivals).

No AES arithmetic here: only which messages exist, how long they are and
which key and IV each carries, drawn from the SplitMix64 streams of
``synth``.
"""
from __future__ import annotations

import numpy as np

from . import STREAM_KEY, STREAM_LENGTH, STREAM_MISC, STREAM_NONCE, bytes_np, uniform01, words_np


def log_uniform_lengths(seed: int, n: int, lo: int = 64, hi: int = 4 << 20) -> np.ndarray:
    """len = floor(lo * (hi/lo)^u), u ~ U[0,1), clamped to [lo, hi] (byte-granular)."""
    u = uniform01(seed, STREAM_LENGTH, n)
    ln = np.floor(lo * np.exp(u * np.log(hi / lo)))
    return np.clip(ln, lo, hi).astype(np.uint64)


def uniform_lengths(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    """len ~ U{lo..hi} (inclusive)."""
    u = uniform01(seed, STREAM_LENGTH, n)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.uint64)


def key_sizes(seed: int, n: int, choices=(128, 192, 256)) -> np.ndarray:
    u = uniform01(seed, STREAM_MISC, n)
    idx = np.minimum((u * len(choices)).astype(np.int64), len(choices) - 1)
    return np.asarray(choices, dtype=np.uint32)[idx]


def message_keys(seed: int, n: int) -> np.ndarray:
    """[n, 32] raw key slots (a 128/192-bit key uses the leading bytes)."""
    return bytes_np(seed, STREAM_KEY, 32 * n).reshape(n, 32)


def message_ivs(seed: int, n: int, counter0: int = 0) -> np.ndarray:
    """[n, 16] IVs: 12 random nonce bytes, then counter0 big-endian."""
    iv = bytes_np(seed, STREAM_NONCE, 16 * n).reshape(n, 16)
    iv[:, 12:16] = np.frombuffer(int(counter0).to_bytes(4, "big"), np.uint8)
    return iv


def batched_varlen(seed: int = 3, n: int = 16384):
    """Batched varlen workload: n messages, lengths log-uniform over
    64 B .. 4 MiB, key sizes uniform over {128, 192, 256}, own key and nonce."""
    return dict(lengths=log_uniform_lengths(seed, n), key_bits=key_sizes(seed, n),
                keys=message_keys(seed, n), ivs=message_ivs(seed, n))


def small_messages(seed: int = 4, n: int = 1_000_000):
    """Packet-sized batch: n messages of U{16..1500} bytes, AES-128, own key and nonce."""
    return dict(lengths=uniform_lengths(seed, n, 16, 1500),
                key_bits=np.full(n, 128, dtype=np.uint32),
                keys=message_keys(seed, n), ivs=message_ivs(seed, n))


def serving_sizes(seed: int, n: int) -> np.ndarray:
    """Request sizes: 70 % U[1,16] KiB, 25 % U[16 KiB, 1 MiB], 5 % U[1, 64] MiB
    (uniform within each bucket, byte-granular)."""
    u = uniform01(seed, STREAM_LENGTH, n)
    v = uniform01(seed, STREAM_MISC, n)
    lo = np.where(u < 0.70, 1 << 10, np.where(u < 0.95, 16 << 10, 1 << 20)).astype(np.float64)
    hi = np.where(u < 0.70, 16 << 10, np.where(u < 0.95, 1 << 20, 64 << 20)).astype(np.float64)
    return np.floor(lo + v * (hi - lo + 1)).astype(np.uint64)


def poisson_arrivals(seed: int, rate_per_s: float, duration_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps of mean 1/rate."""
    n_max = int(rate_per_s * duration_s * 1.2 + 100)
    u = uniform01(seed, STREAM_NONCE + 16, n_max)
    gaps = -np.log1p(-u) / rate_per_s
    t = np.cumsum(gaps)
    return t[t < duration_s]


def tenants(seed: int, n: int, n_tenants: int = 1024) -> np.ndarray:
    w = words_np(seed, STREAM_MISC + 8, n)
    return (w % np.uint64(n_tenants)).astype(np.uint32)
