"""Encrypt or decrypt a file on the GPU: the paper's workload (a file in, the
encrypted file out, §IV) with the chunk split done by a pipeline instead of
processes.

Three stages overlap through a ring of `depth` pinned buffer pairs:

  reader thread   file -> pinned input buffer (sequential reads)
  GPU             the library call on the pinned buffers (the kernel reads
                  and writes host memory over NVLink-C2C; CTR chunks use the
                  IV advanced by the chunk's first block, so the result is
                  byte-identical to one call on the whole file)
  writer thread   pinned output buffer -> file, once the chunk's event fired

ECB needs a file length that is a multiple of 16 (no padding here).

    python -m paper_1403_7295_gb300.filecrypt {ctr,ecb-enc,ecb-dec} SRC DST --key HEX [--iv HEX]
"""
from __future__ import annotations

import argparse
import os
import queue
import threading
import time

import numpy as np

from . import aes as _aes
from .shard import ctr_iv_at


def crypt_file(src: str, dst: str, key, mode: str = "ctr", iv=None, chunk_bytes: int = 64 << 20,
               depth: int = 3) -> dict:
    """Process `src` into `dst`; returns bytes, seconds and GB/s (file to file)."""
    import torch

    if mode not in ("ctr", "ecb-enc", "ecb-dec"):
        raise ValueError(f"unknown mode {mode}")
    if chunk_bytes % 16:
        raise ValueError("chunk_bytes must be a multiple of 16")
    ks = _aes.aes_expand_key(key)
    size = os.path.getsize(src)
    if mode != "ctr" and size % 16:
        raise ValueError("ECB needs a file length that is a multiple of 16")
    if mode == "ctr" and (iv is None or len(bytes(iv)) != 16):
        raise ValueError("CTR needs a 16-byte IV")
    chunk_bytes = max(16, min(chunk_bytes, (size + 15) // 16 * 16 or 16))
    bufs_in = [torch.empty(chunk_bytes, dtype=torch.uint8).pin_memory() for _ in range(depth)]
    bufs_out = [torch.empty(chunk_bytes, dtype=torch.uint8).pin_memory() for _ in range(depth)]
    free: queue.Queue = queue.Queue()
    for k in range(depth):
        free.put(k)
    filled: queue.Queue = queue.Queue()
    done: queue.Queue = queue.Queue()
    errors: list = []
    stream = torch.cuda.Stream()

    def reader():
        try:
            with open(src, "rb", buffering=0) as f:
                off = 0
                while off < size:
                    k = free.get()
                    n = min(chunk_bytes, size - off)
                    view = memoryview(bufs_in[k].numpy())[:n]
                    got = 0
                    while got < n:
                        r = f.readinto(view[got:])
                        if not r:
                            raise IOError("short read")
                        got += r
                    filled.put((k, off, n))
                    off += n
        except BaseException as e:  # surfaced by the caller
            errors.append(e)
        filled.put(None)

    def writer():
        try:
            with open(dst, "wb", buffering=0) as f:
                while True:
                    item = done.get()
                    if item is None:
                        break
                    k, n, ev = item
                    ev.synchronize()
                    mv = memoryview(bufs_out[k].numpy())[:n]
                    w = 0
                    while w < n:
                        w += f.write(mv[w:])
                    free.put(k)
        except BaseException as e:
            errors.append(e)
            for _ in range(depth):
                free.put(0)  # unblock the reader

    t0 = time.perf_counter()
    tr = threading.Thread(target=reader, daemon=True)
    tw = threading.Thread(target=writer, daemon=True)
    tr.start()
    tw.start()
    while True:
        item = filled.get()
        if item is None or errors:
            break
        k, off, n = item
        x, y = bufs_in[k][:n], bufs_out[k][:n]
        if mode == "ctr":
            _aes.aes_ctr_xcrypt(ks, ctr_iv_at(iv, off // 16), x, y, stream=stream)
        elif mode == "ecb-enc":
            _aes.aes_ecb_encrypt(ks, x, y, stream=stream)
        else:
            _aes.aes_ecb_decrypt(ks, x, y, stream=stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        done.put((k, n, ev))
    done.put(None)
    tr.join()
    tw.join()
    if errors:
        raise errors[0]
    dt = time.perf_counter() - t0
    return {"bytes": size, "seconds": dt, "gbps": size / dt / 1e9 if dt > 0 else 0.0,
            "chunk_bytes": chunk_bytes, "depth": depth}


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("mode", choices=["ctr", "ecb-enc", "ecb-dec"])
    p.add_argument("src")
    p.add_argument("dst")
    p.add_argument("--key", required=True, help="hex, 16/24/32 bytes")
    p.add_argument("--iv", default=None, help="hex, 16 bytes (CTR)")
    p.add_argument("--chunk-mib", type=int, default=64)
    a = p.parse_args()
    iv = bytes.fromhex(a.iv) if a.iv else None
    r = crypt_file(a.src, a.dst, np.frombuffer(bytes.fromhex(a.key), np.uint8), a.mode, iv,
                   a.chunk_mib << 20)
    print(r)


if __name__ == "__main__":
    main()
