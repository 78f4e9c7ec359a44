"""Helpers shared by the GPU tests (device buffers with guard bands, oracle calls)."""
import os

import numpy as np
import pytest

GUARD = 4096  # bytes of canary on each side of every output buffer
CANARY = 0xA5


def require_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1403_7295_gb300 import build

    build.build()
    return torch


def to_dev(a: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class Guarded:
    """A device byte buffer of n bytes with canary bands on both sides."""

    def __init__(self, n: int):
        import torch

        self.n = n
        self.raw = torch.full((n + 2 * GUARD,), CANARY, dtype=torch.uint8, device="cuda")
        self.view = self.raw[GUARD:GUARD + n]

    def intact(self) -> bool:
        import torch

        return bool(torch.all(self.raw[:GUARD] == CANARY)) and bool(torch.all(self.raw[GUARD + self.n:] == CANARY))

    def numpy(self) -> np.ndarray:
        return self.view.cpu().numpy()


def host_threads() -> int:
    return max(1, os.cpu_count() or 1)


def library_mapped() -> bool:
    """True once libaesgpu.so is mapped into this process."""
    with open("/proc/self/maps") as f:
        return any("libaesgpu.so" in line for line in f)


def pageable_memory_access():
    """cudaDevAttrPageableMemoryAccess of device 0 from the CUDA runtime, or
    None when no runtime library is found."""
    import ctypes
    import glob

    libs = sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    if not libs:
        return None
    rt = ctypes.CDLL(libs[0])
    v = ctypes.c_int(0)
    if rt.cudaDeviceGetAttribute(ctypes.byref(v), 88, 0) != 0:  # 88: cudaDevAttrPageableMemoryAccess
        return None
    return v.value == 1

