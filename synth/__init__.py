"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no AES arithmetic.  It is one counter-based generator,
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; the finaliser constants as Vigna publishes them),
computed identically with numpy on the host and with torch int64 ops on any
device, so both sides can regenerate the same bytes without a transfer:

    word i of (seed, stream) = mix(base + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64)
    base = seed * 2^40 + stream * 2^32
    mix(z): z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
            z *= 0x94D049BB133111EB; z ^= z >> 31

Bytes are the little-endian bytes of consecutive words.  The workload recipes
(buffer sizes, message-length mixes, arrivals) are in ``synth.workloads``.
"""
from __future__ import annotations

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

STREAM_DATA = 0
STREAM_KEY = 1
STREAM_NONCE = 2
STREAM_LENGTH = 3
STREAM_MISC = 4


def _base(seed: int, stream: int) -> int:
    return ((int(seed) << 40) + (int(stream) << 32)) & MASK64


def words_np(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` uint64 words of (seed, stream) starting at word ``start``."""
    i = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(_base(seed, stream)) + i * np.uint64(GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        z = z ^ (z >> np.uint64(31))
    return z


def bytes_np(seed: int, stream: int, nbytes: int) -> np.ndarray:
    """``nbytes`` bytes of (seed, stream) as a uint8 numpy array."""
    w = words_np(seed, stream, (nbytes + 7) // 8)
    return w.astype("<u8").view(np.uint8)[:nbytes].copy()


def _signed(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def bytes_torch(seed: int, stream: int, nbytes: int, device="cpu", chunk_words: int = 1 << 25):
    """Same bytes as ``bytes_np`` built with torch int64 ops on ``device``.

    int64 multiplication wraps modulo 2^64 and a logical right shift is an
    arithmetic shift followed by a mask, so the words match ``words_np``.
    """
    import torch

    nwords = (nbytes + 7) // 8
    out = torch.empty(nwords * 8, dtype=torch.uint8, device=device)
    ow = out.view(torch.int64)
    base = _signed(_base(seed, stream))
    g, m1, m2 = _signed(GOLDEN), _signed(M1), _signed(M2)
    masks = {k: (1 << (64 - k)) - 1 for k in (27, 30, 31)}
    for s in range(0, nwords, chunk_words):
        e = min(nwords, s + chunk_words)
        z = torch.arange(s + 1, e + 1, dtype=torch.int64, device=device)
        z.mul_(g).add_(base)
        z = (z ^ ((z >> 30) & masks[30])) * m1
        z = (z ^ ((z >> 27) & masks[27])) * m2
        z = z ^ ((z >> 31) & masks[31])
        ow[s:e] = z
    return out[:nbytes]


def key_bytes(seed: int, key_bits: int) -> np.ndarray:
    """A random key of ``key_bits`` bits for run ``seed``."""
    return bytes_np(seed, STREAM_KEY, key_bits // 8)


def iv_bytes(seed: int, counter0: int = 0) -> np.ndarray:
    """A 16-byte CTR IV: 12 random nonce bytes, then ``counter0`` big-endian."""
    iv = bytes_np(seed, STREAM_NONCE, 16)
    iv[12:16] = np.frombuffer(int(counter0).to_bytes(4, "big"), np.uint8)
    return iv


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from the top 53 bits of each word."""
    w = words_np(seed, stream, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
