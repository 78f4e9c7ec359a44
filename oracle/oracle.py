"""ctypes binding of the CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  It compiles ``aes_ref.c`` with the system C
compiler into ``oracle/_build/liboracle.so`` on first use (plain ``-O2``, no
target-specific flags, so the same source builds on x86-64 and on aarch64) and
exposes numpy-facing wrappers.  Every function here only marshals arguments;
the arithmetic is in ``aes_ref.c``, which cites FIPS-197 / SP 800-38A and the
paper's §III.A (Fig. 1) and §IV.B.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ("aes_ref.c",)
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

REF_OK = 0
REF_ERR_KEYSIZE = -1
REF_ERR_LENGTH = -2
REF_ERR_PADDING = -3
REF_ERR_THREAD = -4

_lock = threading.Lock()
_lib = None


def build(force: bool = False, src_dir: str = HERE, out_path: str = LIB_PATH,
          extra_flags: tuple = ()) -> str:
    """Compile the oracle into a shared library and return its path."""
    srcs = [os.path.join(src_dir, s) for s in SOURCES]
    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    if not force and os.path.exists(out_path):
        newest = max(os.path.getmtime(p) for p in srcs + [os.path.join(HERE, "aes_ref.h")])
        if os.path.getmtime(out_path) >= newest:
            return out_path
    tmp = out_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-pthread", "-Wall", "-Wextra",
           "-D_POSIX_C_SOURCE=200809L", f"-I{HERE}", *extra_flags, *srcs, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out_path)
    return out_path


def _declare(lib):
    u8p = ctypes.c_void_p
    lib.ref_gf_mul.argtypes = [ctypes.c_uint8, ctypes.c_uint8]
    lib.ref_gf_mul.restype = ctypes.c_uint8
    lib.ref_gf_inv.argtypes = [ctypes.c_uint8]
    lib.ref_gf_inv.restype = ctypes.c_uint8
    lib.ref_sbox.argtypes = [u8p]
    lib.ref_inv_sbox.argtypes = [u8p]
    lib.ref_mix_column.argtypes = [u8p]
    lib.ref_inv_mix_column.argtypes = [u8p]
    lib.ref_key_expansion.argtypes = [u8p, ctypes.c_int, u8p, ctypes.POINTER(ctypes.c_int)]
    lib.ref_key_expansion.restype = ctypes.c_int
    lib.ref_cipher.argtypes = [u8p, u8p, u8p, ctypes.c_int]
    lib.ref_inv_cipher.argtypes = [u8p, u8p, u8p, ctypes.c_int]
    for name in ("ref_ecb_encrypt", "ref_ecb_decrypt"):
        getattr(lib, name).argtypes = [u8p, ctypes.c_int, u8p, u8p, ctypes.c_uint64]
        getattr(lib, name).restype = ctypes.c_int
    for name in ("ref_ecb_encrypt_mt", "ref_ecb_decrypt_mt"):
        getattr(lib, name).argtypes = [u8p, ctypes.c_int, u8p, u8p, ctypes.c_uint64, ctypes.c_int]
        getattr(lib, name).restype = ctypes.c_int
    lib.ref_ctr_xcrypt.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_uint64, u8p, u8p, ctypes.c_uint64]
    lib.ref_ctr_xcrypt.restype = ctypes.c_int
    lib.ref_ctr_xcrypt_mt.argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_uint64, u8p, u8p,
                                      ctypes.c_uint64, ctypes.c_int]
    lib.ref_ctr_xcrypt_mt.restype = ctypes.c_int
    lib.ref_ctr_xcrypt_blocks.argtypes = [u8p, ctypes.c_int, u8p, u8p, u8p, u8p, ctypes.c_uint64]
    lib.ref_ctr_xcrypt_blocks.restype = ctypes.c_int
    for name in ("ref_cbc_encrypt", "ref_cbc_decrypt"):
        getattr(lib, name).argtypes = [u8p, ctypes.c_int, u8p, u8p, u8p, ctypes.c_uint64]
        getattr(lib, name).restype = ctypes.c_int
    for name in ("ref_xts_encrypt", "ref_xts_decrypt"):
        getattr(lib, name).argtypes = [u8p, u8p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, u8p, u8p,
                                       ctypes.c_uint64]
        getattr(lib, name).restype = ctypes.c_int
    lib.ref_batch_mt.argtypes = [ctypes.c_int, ctypes.c_uint64, u8p, u8p, u8p, u8p, u8p, u8p, u8p, u8p, u8p,
                                 u8p, ctypes.c_int]
    lib.ref_batch_mt.restype = ctypes.c_int
    lib.ref_pkcs7_padded_len.argtypes = [ctypes.c_uint64]
    lib.ref_pkcs7_padded_len.restype = ctypes.c_uint64
    for name in ("ref_ecb_pkcs7_encrypt", "ref_ecb_pkcs7_decrypt"):
        getattr(lib, name).argtypes = [u8p, ctypes.c_int, u8p, ctypes.c_uint64, u8p,
                                       ctypes.POINTER(ctypes.c_uint64)]
        getattr(lib, name).restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; cached for the default path."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _declare(ctypes.CDLL(build()))
        return _lib


# ---- numpy helpers -------------------------------------------------------

def _u8(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint8).reshape(-1))
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc != REF_OK:
        raise ValueError(f"oracle {what} failed with status {rc}")


class Oracle:
    """Numpy front end over one loaded copy of the oracle library."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    # GF(2^8) and table pieces
    def gf_mul(self, a: int, b: int) -> int:
        return int(self.lib.ref_gf_mul(a, b))

    def gf_inv(self, a: int) -> int:
        return int(self.lib.ref_gf_inv(a))

    def sbox(self) -> np.ndarray:
        out = np.zeros(256, np.uint8)
        self.lib.ref_sbox(_ptr(out))
        return out

    def inv_sbox(self) -> np.ndarray:
        out = np.zeros(256, np.uint8)
        self.lib.ref_inv_sbox(_ptr(out))
        return out

    def mix_column(self, col) -> np.ndarray:
        c = _u8(col).copy()
        self.lib.ref_mix_column(_ptr(c))
        return c

    def inv_mix_column(self, col) -> np.ndarray:
        c = _u8(col).copy()
        self.lib.ref_inv_mix_column(_ptr(c))
        return c

    def key_expansion(self, key, key_bits: int):
        k = _u8(key)
        w = np.zeros(240, np.uint8)
        nr = ctypes.c_int(0)
        n = self.lib.ref_key_expansion(_ptr(k), key_bits, _ptr(w), ctypes.byref(nr))
        if n < 0:
            raise ValueError(f"bad key size {key_bits}")
        return w[: 4 * n].copy(), nr.value

    def cipher_block(self, key, key_bits: int, block) -> np.ndarray:
        w, nr = self.key_expansion(key, key_bits)
        b = _u8(block)
        out = np.zeros(16, np.uint8)
        self.lib.ref_cipher(_ptr(b), _ptr(out), _ptr(w), nr)
        return out

    def inv_cipher_block(self, key, key_bits: int, block) -> np.ndarray:
        w, nr = self.key_expansion(key, key_bits)
        b = _u8(block)
        out = np.zeros(16, np.uint8)
        self.lib.ref_inv_cipher(_ptr(b), _ptr(out), _ptr(w), nr)
        return out

    # modes
    def ecb_encrypt(self, key, key_bits: int, data, nthreads: int = 0) -> np.ndarray:
        k, d = _u8(key), _u8(data)
        out = np.empty_like(d)
        if nthreads:
            rc = self.lib.ref_ecb_encrypt_mt(_ptr(k), key_bits, _ptr(d), _ptr(out), d.size, nthreads)
        else:
            rc = self.lib.ref_ecb_encrypt(_ptr(k), key_bits, _ptr(d), _ptr(out), d.size)
        _check(rc, "ecb_encrypt")
        return out

    def ecb_decrypt(self, key, key_bits: int, data, nthreads: int = 0) -> np.ndarray:
        k, d = _u8(key), _u8(data)
        out = np.empty_like(d)
        if nthreads:
            rc = self.lib.ref_ecb_decrypt_mt(_ptr(k), key_bits, _ptr(d), _ptr(out), d.size, nthreads)
        else:
            rc = self.lib.ref_ecb_decrypt(_ptr(k), key_bits, _ptr(d), _ptr(out), d.size)
        _check(rc, "ecb_decrypt")
        return out

    def ctr_xcrypt(self, key, key_bits: int, iv, data, first_block: int = 0,
                   nthreads: int = 0) -> np.ndarray:
        k, v, d = _u8(key), _u8(iv), _u8(data)
        assert v.size == 16
        out = np.empty_like(d)
        if nthreads:
            rc = self.lib.ref_ctr_xcrypt_mt(_ptr(k), key_bits, _ptr(v), first_block, _ptr(d),
                                            _ptr(out), d.size, nthreads)
        else:
            rc = self.lib.ref_ctr_xcrypt(_ptr(k), key_bits, _ptr(v), first_block, _ptr(d),
                                         _ptr(out), d.size)
        _check(rc, "ctr_xcrypt")
        return out

    def ctr_xcrypt_blocks(self, key, key_bits: int, iv, idx, blocks) -> np.ndarray:
        """CTR on sampled blocks: row k of ``blocks`` (16 bytes) is counter block idx[k]."""
        k, v = _u8(key), _u8(iv)
        ix = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64).reshape(-1))
        b = _u8(blocks)
        assert b.size == 16 * ix.size
        out = np.empty_like(b)
        rc = self.lib.ref_ctr_xcrypt_blocks(_ptr(k), key_bits, _ptr(v), _ptr(ix), _ptr(b),
                                            _ptr(out), ix.size)
        _check(rc, "ctr_xcrypt_blocks")
        return out

    def batch(self, op: int, data, in_off, in_len, out_size: int, out_off, keys, key_bits, ivs=None,
              nthreads: int = 1, out=None):
        """A list of messages (op 0 CTR, 1 PKCS#7 + ECB encrypt, 2 ECB decrypt
        + PKCS#7 check), each with its own key and IV, one oracle call per
        message.  Returns (out arena of out_size bytes, out_len, status);
        ``out`` (optional) is an arena to write into, whose bytes outside the
        messages' outputs are left as they are."""
        d = _u8(data)
        io = np.ascontiguousarray(np.asarray(in_off, np.uint64).reshape(-1))
        il = np.ascontiguousarray(np.asarray(in_len, np.uint64).reshape(-1))
        oo = np.ascontiguousarray(np.asarray(out_off, np.uint64).reshape(-1))
        n = io.size
        assert il.size == n and oo.size == n
        k = np.ascontiguousarray(np.asarray(keys, np.uint8).reshape(n, 32))
        kb = np.ascontiguousarray(np.asarray(key_bits, np.uint32).reshape(-1))
        assert kb.size == n
        if op == 0:
            v = np.ascontiguousarray(np.asarray(ivs, np.uint8).reshape(n, 16))
        else:
            v = np.zeros((max(n, 1), 16), np.uint8)
        # every message must lie inside the arenas it reads and writes
        if n:
            assert int((io + il).max()) <= d.size
            span = il if op != 1 else (il - il % np.uint64(16) + np.uint64(16))
            assert int((oo + span).max()) <= out_size
        o = np.zeros(out_size, np.uint8) if out is None else out
        assert o.dtype == np.uint8 and o.flags.c_contiguous and o.size == out_size
        out_len = np.zeros(max(n, 1), np.uint64)
        status = np.zeros(max(n, 1), np.int32)
        rc = self.lib.ref_batch_mt(op, n, _ptr(d), _ptr(io), _ptr(il), _ptr(o), _ptr(oo), _ptr(k), _ptr(kb),
                                   _ptr(v), _ptr(out_len), _ptr(status), nthreads)
        _check(rc, "batch")
        return o, out_len[:n], status[:n]

    def pkcs7_padded_len(self, n: int) -> int:
        return int(self.lib.ref_pkcs7_padded_len(n))

    def ecb_pkcs7_encrypt(self, key, key_bits: int, data) -> np.ndarray:
        k, d = _u8(key), _u8(data)
        out = np.zeros(self.pkcs7_padded_len(d.size), np.uint8)
        n = ctypes.c_uint64(0)
        rc = self.lib.ref_ecb_pkcs7_encrypt(_ptr(k), key_bits, _ptr(d), d.size, _ptr(out),
                                            ctypes.byref(n))
        _check(rc, "ecb_pkcs7_encrypt")
        return out[: n.value]

    def ecb_pkcs7_decrypt(self, key, key_bits: int, data):
        """Returns (status, plaintext); status is REF_OK or REF_ERR_PADDING/LENGTH."""
        k, d = _u8(key), _u8(data)
        out = np.zeros(max(d.size, 1), np.uint8)
        n = ctypes.c_uint64(0)
        rc = self.lib.ref_ecb_pkcs7_decrypt(_ptr(k), key_bits, _ptr(d), d.size, _ptr(out),
                                            ctypes.byref(n))
        if rc != REF_OK:
            return rc, None
        return rc, out[: n.value].copy()

    def cbc_encrypt(self, key, key_bits: int, iv, data) -> np.ndarray:
        k, v, d = _u8(key), _u8(iv), _u8(data)
        out = np.empty_like(d)
        _check(self.lib.ref_cbc_encrypt(_ptr(k), key_bits, _ptr(v), _ptr(d), _ptr(out), d.size), "cbc_encrypt")
        return out

    def cbc_decrypt(self, key, key_bits: int, iv, data) -> np.ndarray:
        k, v, d = _u8(key), _u8(iv), _u8(data)
        out = np.empty_like(d)
        _check(self.lib.ref_cbc_decrypt(_ptr(k), key_bits, _ptr(v), _ptr(d), _ptr(out), d.size), "cbc_decrypt")
        return out

    def xts(self, decrypt: bool, key1, key2, key_bits: int, sector_bytes: int, first_sector: int,
            data) -> np.ndarray:
        k1, k2, d = _u8(key1), _u8(key2), _u8(data)
        out = np.empty_like(d)
        fn = self.lib.ref_xts_decrypt if decrypt else self.lib.ref_xts_encrypt
        _check(fn(_ptr(k1), _ptr(k2), key_bits, sector_bytes, first_sector, _ptr(d), _ptr(out), d.size), "xts")
        return out
