"""Python binding of libaesgpu.so: argument marshalling only.

Each function has the name of the C entry point it calls (``include/aesgpu.h``)
and does no arithmetic of its own: it turns torch tensors into device
pointers and byte counts, passes the current torch CUDA stream, and raises
``AesError`` on a non-zero status.  There is no CPU path: without the built
library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

AES_OK = 0
STATUS_NAMES = {
    0: "AES_OK", 1: "AES_ERR_ARG", 2: "AES_ERR_KEYSIZE", 3: "AES_ERR_LENGTH", 4: "AES_ERR_ALIGN",
    5: "AES_ERR_OVERLAP", 6: "AES_ERR_PADDING", 7: "AES_ERR_NOMEM", 8: "AES_ERR_CUDA",
    9: "AES_ERR_TIMEOUT", 10: "AES_ERR_BUSY",
}
VARIANT_AUTO, VARIANT_TTABLE, VARIANT_BITSLICE, VARIANT_TTABLE_BULK = 0, 1, 2, 3


class AesError(RuntimeError):
    def __init__(self, status: int, what: str, cuda_error: int = 0):
        self.status = status
        self.cuda_error = cuda_error
        name = STATUS_NAMES.get(status, str(status))
        extra = f" (cuda error {cuda_error})" if status == 8 else ""
        super().__init__(f"{what}: {name}{extra}")


class KeySchedule(ctypes.Structure):
    """Mirror of ``aes_key_schedule``."""
    _fields_ = [("key_bits", ctypes.c_uint32), ("nr", ctypes.c_uint32),
                ("rk_enc", ctypes.c_uint32 * 60), ("rk_dec", ctypes.c_uint32 * 60)]


class LaunchConfig(ctypes.Structure):
    """Mirror of ``aes_launch_config``; zero fields mean "library default"."""
    _fields_ = [("variant", ctypes.c_int32), ("cta_threads", ctypes.c_int32),
                ("blocks_per_thread", ctypes.c_int32), ("grid_ctas", ctypes.c_int32)]


_LIB = None


def library_path() -> str:
    return _build.LIB_PATH


def lib():
    """The loaded libaesgpu.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        ksp = ctypes.POINTER(KeySchedule)
        cfgp = ctypes.POINTER(LaunchConfig)
        L.aes_expand_key.argtypes = [vp, ctypes.c_int, ksp]
        for name in ("aes_ecb_encrypt", "aes_ecb_decrypt"):
            getattr(L, name).argtypes = [ksp, vp, vp, sz, vp]
            getattr(L, name + "_ex").argtypes = [ksp, vp, vp, sz, vp, cfgp]
        L.aes_ctr_xcrypt.argtypes = [ksp, vp, vp, vp, sz, vp]
        L.aes_ctr_xcrypt_ex.argtypes = [ksp, vp, vp, vp, sz, vp, cfgp]
        L.aes_ctr_iv_advance.argtypes = [vp, ctypes.c_uint64, vp]
        L.aes_ctr_iv_advance.restype = ctypes.c_int
        L.aes_cbc_decrypt.argtypes = [ksp, vp, vp, vp, sz, vp]
        for name in ("aes_xts_encrypt", "aes_xts_decrypt"):
            getattr(L, name).argtypes = [ksp, ksp, ctypes.c_uint64, sz, vp, vp, sz, vp]
            getattr(L, name).restype = ctypes.c_int
        L.aes_cbc_decrypt.restype = ctypes.c_int
        L.aes_take_wait_timeouts.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
        L.aes_take_wait_timeouts.restype = ctypes.c_int
        L.aes_last_cuda_error.argtypes = []
        L.aes_status_string.argtypes = [ctypes.c_int]
        L.aes_status_string.restype = ctypes.c_char_p
        for name in ("aes_expand_key", "aes_ecb_encrypt", "aes_ecb_decrypt", "aes_ctr_xcrypt",
                     "aes_ecb_encrypt_ex", "aes_ecb_decrypt_ex", "aes_ctr_xcrypt_ex",
                     "aes_last_cuda_error"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(status: int, what: str):
    if status != AES_OK:
        raise AesError(status, what, lib().aes_last_cuda_error() if status == 8 else 0)


def _host_bytes(x) -> np.ndarray:
    if hasattr(x, "detach"):  # torch tensor
        x = x.detach().cpu().numpy()
    if isinstance(x, (bytes, bytearray)):
        x = np.frombuffer(bytes(x), np.uint8)
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8).reshape(-1))


def aes_expand_key(key, key_bits: int | None = None) -> KeySchedule:
    """Host key expansion (FIPS-197 §5.2) into an ``aes_key_schedule``."""
    k = _host_bytes(key)
    bits = key_bits if key_bits is not None else 8 * k.size
    ks = KeySchedule()
    buf = (ctypes.c_uint8 * max(1, k.size)).from_buffer_copy(k.tobytes() or b"\0")
    _check(lib().aes_expand_key(ctypes.cast(buf, ctypes.c_void_p), bits, ctypes.byref(ks)),
           "aes_expand_key")
    return ks


def _stream_handle(stream, tensor):
    import torch

    if stream is None:
        # host (pinned) tensors run on the current device's stream
        stream = torch.cuda.current_stream(tensor.device if tensor.is_cuda else None)
    return ctypes.c_void_p(stream.cuda_stream)


def _prepare(inp, out):
    import torch

    if not isinstance(inp, torch.Tensor) or inp.dtype != torch.uint8:
        raise TypeError("input must be a torch.uint8 tensor")
    if not inp.is_contiguous():
        raise ValueError("input must be contiguous")
    if out is None:
        out = torch.empty_like(inp)
    if out.dtype != torch.uint8 or not out.is_contiguous() or out.numel() < inp.numel():
        raise ValueError("output must be a contiguous uint8 tensor at least as large as the input")
    return inp, out


def _cfg(config):
    if config is None:
        return None
    if isinstance(config, LaunchConfig):
        return ctypes.byref(config)
    c = LaunchConfig(**config)
    return ctypes.byref(c)


def aes_ecb_encrypt(ks: KeySchedule, inp, out=None, stream=None, config=None):
    """ECB encryption of a device uint8 tensor; returns ``out``."""
    inp, out = _prepare(inp, out)
    _check(lib().aes_ecb_encrypt_ex(ctypes.byref(ks), inp.data_ptr(), out.data_ptr(), inp.numel(),
                                    _stream_handle(stream, inp), _cfg(config)), "aes_ecb_encrypt")
    return out


def aes_ecb_decrypt(ks: KeySchedule, inp, out=None, stream=None, config=None):
    """ECB decryption of a device uint8 tensor; returns ``out``."""
    inp, out = _prepare(inp, out)
    _check(lib().aes_ecb_decrypt_ex(ctypes.byref(ks), inp.data_ptr(), out.data_ptr(), inp.numel(),
                                    _stream_handle(stream, inp), _cfg(config)), "aes_ecb_decrypt")
    return out


def aes_ctr_xcrypt(ks: KeySchedule, iv, inp, out=None, stream=None, config=None):
    """CTR encryption/decryption of a device uint8 tensor; returns ``out``."""
    inp, out = _prepare(inp, out)
    v = _host_bytes(iv)
    if v.size != 16:
        raise ValueError("iv must be 16 bytes")
    vb = (ctypes.c_uint8 * 16).from_buffer_copy(v.tobytes())
    _check(lib().aes_ctr_xcrypt_ex(ctypes.byref(ks), ctypes.cast(vb, ctypes.c_void_p), inp.data_ptr(),
                                   out.data_ptr(), inp.numel(), _stream_handle(stream, inp),
                                   _cfg(config)), "aes_ctr_xcrypt")
    return out


def aes_ctr_iv_advance(iv, first_block: int) -> bytes:
    """The IV of a CTR range starting ``first_block`` blocks into a buffer
    (the library's counter advance, modulo 2^32, nonce unchanged)."""
    v = _host_bytes(iv)
    if v.size != 16:
        raise ValueError("iv must be 16 bytes")
    if first_block < 0:
        raise ValueError("first_block must be >= 0")
    vb = (ctypes.c_uint8 * 16).from_buffer_copy(v.tobytes())
    out = (ctypes.c_uint8 * 16)()
    _check(lib().aes_ctr_iv_advance(ctypes.cast(vb, ctypes.c_void_p), first_block,
                                    ctypes.cast(out, ctypes.c_void_p)), "aes_ctr_iv_advance")
    return bytes(out)


def aes_take_wait_timeouts() -> int:
    """Bounded device waits (of the TMA-staged CTR variant and the batch's
    lane kernel) that gave up on the current device since the last call; the
    count restarts at 0."""
    n = ctypes.c_uint32(0)
    rc = lib().aes_take_wait_timeouts(ctypes.byref(n))
    if rc not in (AES_OK, 9):  # 9: AES_ERR_TIMEOUT, reported through the count
        _check(rc, "aes_take_wait_timeouts")
    return int(n.value)


def aes_cbc_decrypt(ks: KeySchedule, iv, inp, out=None, stream=None):
    """CBC decryption of a device uint8 tensor (not in place); returns ``out``."""
    inp, out = _prepare(inp, out)
    v = _host_bytes(iv)
    if v.size != 16:
        raise ValueError("iv must be 16 bytes")
    vb = (ctypes.c_uint8 * 16).from_buffer_copy(v.tobytes())
    _check(lib().aes_cbc_decrypt(ctypes.byref(ks), ctypes.cast(vb, ctypes.c_void_p), inp.data_ptr(),
                                 out.data_ptr(), inp.numel(), _stream_handle(stream, inp)), "aes_cbc_decrypt")
    return out


def aes_xts_encrypt(data_ks: KeySchedule, tweak_ks: KeySchedule, first_sector: int, sector_bytes: int,
                    inp, out=None, stream=None):
    """XTS encryption of a device uint8 tensor of whole data units; returns ``out``."""
    inp, out = _prepare(inp, out)
    _check(lib().aes_xts_encrypt(ctypes.byref(data_ks), ctypes.byref(tweak_ks), first_sector, sector_bytes,
                                 inp.data_ptr(), out.data_ptr(), inp.numel(), _stream_handle(stream, inp)),
           "aes_xts_encrypt")
    return out


def aes_xts_decrypt(data_ks: KeySchedule, tweak_ks: KeySchedule, first_sector: int, sector_bytes: int,
                    inp, out=None, stream=None):
    """XTS decryption of a device uint8 tensor of whole data units; returns ``out``."""
    inp, out = _prepare(inp, out)
    _check(lib().aes_xts_decrypt(ctypes.byref(data_ks), ctypes.byref(tweak_ks), first_sector, sector_bytes,
                                 inp.data_ptr(), out.data_ptr(), inp.numel(), _stream_handle(stream, inp)),
           "aes_xts_decrypt")
    return out
