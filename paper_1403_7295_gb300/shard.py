"""Splitting one buffer across GPUs (the paper's N-chunk scheme, §IV, at
device granularity).

ECB and CTR blocks are independent, so a buffer splits into contiguous
ranges of whole 16-byte blocks, one per rank, with no exchange between
ranks: each rank encrypts its range in place and the outputs sit at the same
offsets (the paper's concatenation step disappears).  The remainder blocks
and any partial CTR tail go to the last rank, as the paper's last chunk
takes the remainder.  For CTR a range starting at block b uses the IV whose
32-bit big-endian counter is advanced by b (modulo 2^32, no carry into the
nonce, computed by the library's ``aes_ctr_iv_advance``), so every rank
produces exactly the bytes of the single-pass call.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Shard:
    rank: int
    byte_off: int
    byte_len: int
    first_block: int


def shard_ranges(nbytes: int, world: int) -> list[Shard]:
    """Contiguous whole-block ranges for `world` ranks covering nbytes."""
    if world < 1:
        raise ValueError("world must be >= 1")
    nblocks = nbytes // 16
    per = nblocks // world
    out = []
    for r in range(world):
        b0 = per * r
        length = (nbytes - 16 * b0) if r == world - 1 else 16 * per
        out.append(Shard(r, 16 * b0, length, b0))
    return out


def ctr_iv_at(iv, first_block: int) -> bytes:
    """IV of a CTR range that starts at block `first_block` of the buffer:
    the library's ``aes_ctr_iv_advance`` (the counter arithmetic stays behind
    the C ABI; this only marshals)."""
    from .aes import aes_ctr_iv_advance

    return aes_ctr_iv_advance(iv, first_block)
