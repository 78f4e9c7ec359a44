"""Encrypt or decrypt a file on the GPU: the paper's workload (a file in, the
encrypted file out, §IV), through the library's native pipeline
``aes_file_crypt`` (include/aesgpu.h).  Worker threads take fixed-size
chunks.  By default each worker reads its chunk into a pinned buffer, runs
the cipher on it in place and copies it into the output (the staged path).
With ``direct=True`` (``--direct``), where the device reaches pageable host
memory through the host's page tables (Grace-Blackwell over NVLink-C2C),
both files are mapped and the kernel reads and writes the mapped chunks
directly (no host copy); the files must then keep their length during the
call, since a page truncated away under a running kernel faults the GPU.  CTR
chunks use the IV advanced by the chunk's first block, so the result is
byte-identical to one call on the whole file.  ECB needs a file length that
is a multiple of 16 (no padding here).

    python -m paper_1403_7295_gb300.filecrypt {ctr,ecb-enc,ecb-dec} SRC DST --key HEX [--iv HEX]
"""
from __future__ import annotations

import argparse
import ctypes
import os

import numpy as np

from . import aes as _aes

MODES = {"ctr": 0, "ecb-enc": 1, "ecb-dec": 2}


STAGED = 1  # AES_FILE_STAGED: the staged path (the default)
DIRECT = 2  # AES_FILE_DIRECT: opt in to the direct path where the device allows it


class FileConfig(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_uint64), ("threads", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class FileStats(ctypes.Structure):
    _fields_ = [("bytes", ctypes.c_uint64), ("chunks", ctypes.c_uint64), ("seconds", ctypes.c_double),
                ("setup_seconds", ctypes.c_double), ("threads", ctypes.c_int32), ("os_errno", ctypes.c_int32),
                ("direct", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _declare():
    L = _aes.lib()
    if not getattr(L, "_file_declared", False):
        L.aes_file_crypt.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int,
                                     ctypes.POINTER(_aes.KeySchedule), ctypes.c_void_p,
                                     ctypes.POINTER(FileConfig), ctypes.POINTER(FileStats)]
        L.aes_file_crypt.restype = ctypes.c_int
        L.aes_file_trim.argtypes = []
        L.aes_file_trim.restype = None
        L._file_declared = True
    return L


def crypt_file(src: str, dst: str, key, mode: str = "ctr", iv=None, chunk_bytes: int = 0,
               threads: int = 0, direct: bool = False) -> dict:
    """Process `src` into `dst` (the same path encrypts in place); returns
    bytes, chunks, seconds (of which setup), worker threads, whether the
    direct path ran, and GB/s file to file.  chunk_bytes 0 takes the path's
    default (64 MiB direct, 4 MiB staged); `direct` opts in to the direct path
    (taken where the device reaches pageable memory; else staged).
    Raises ValueError for a bad mode, IV or ragged ECB length, and OSError /
    AesError when the native call fails."""
    if mode not in MODES:
        raise ValueError(f"unknown mode {mode}")
    if chunk_bytes % 16:
        raise ValueError("chunk_bytes must be a multiple of 16")
    if mode == "ctr" and (iv is None or len(bytes(iv)) != 16):
        raise ValueError("CTR needs a 16-byte IV")
    if mode != "ctr" and os.path.getsize(src) % 16:
        raise ValueError("ECB needs a file length that is a multiple of 16")
    ks = _aes.aes_expand_key(key)
    ivb = ctypes.create_string_buffer(bytes(iv), 16) if mode == "ctr" else None
    cfg = FileConfig(chunk_bytes, threads, DIRECT if direct else 0)
    st = FileStats()
    rc = _declare().aes_file_crypt(os.fsencode(src), os.fsencode(dst), MODES[mode], ctypes.byref(ks),
                                   ivb, ctypes.byref(cfg), ctypes.byref(st))
    if rc == 11:  # AES_ERR_IO
        raise OSError(st.os_errno, os.strerror(st.os_errno) if st.os_errno else "file I/O failed", src)
    _aes._check(rc, "aes_file_crypt")
    return {"bytes": st.bytes, "chunks": st.chunks, "seconds": st.seconds, "setup_seconds": st.setup_seconds,
            "threads": st.threads, "chunk_bytes": chunk_bytes, "direct": bool(st.direct),
            "gbps": st.bytes / st.seconds / 1e9 if st.seconds > 0 else 0.0}


def trim() -> None:
    """Free the pinned chunk buffers the staged path keeps between calls."""
    _declare().aes_file_trim()


def main():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("mode", choices=sorted(MODES))
    p.add_argument("src")
    p.add_argument("dst")
    p.add_argument("--key", required=True, help="hex, 16/24/32 bytes")
    p.add_argument("--iv", default=None, help="hex, 16 bytes (CTR)")
    p.add_argument("--chunk-mib", type=int, default=0, help="0: the path's default")
    p.add_argument("--threads", type=int, default=0)
    p.add_argument("--direct", action="store_true",
                   help="run the kernel on the mapped files (the files must not change length meanwhile)")
    a = p.parse_args()
    iv = bytes.fromhex(a.iv) if a.iv else None
    r = crypt_file(a.src, a.dst, np.frombuffer(bytes.fromhex(a.key), np.uint8), a.mode, iv,
                   a.chunk_mib << 20, a.threads, a.direct)
    print(r)


if __name__ == "__main__":
    main()
