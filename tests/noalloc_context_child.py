"""Child process of test_zz_no_alloc.py: aes_batch_submit_noalloc across CUDA contexts.

The allocation-free batch call keeps the device address of its scratch
array per CUDA context.  This program switches the current context under
the library, using the driver API only (no torch, so nothing else holds
state in the contexts): the device's primary context, then a second context
on the same device made with cuCtxCreate, then the primary one again.  In
each it builds one CTR batch in that context's memory and checks that the
allocation-free call writes exactly what aes_batch_submit (with a workspace
from cuMemAlloc) writes: output bytes, statuses and output lengths.  Prints
OK and exits 0 on success; any mismatch or failed call exits non-zero.
"""
import ctypes
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_1403_7295_gb300 import batch as B  # noqa: E402
from synth import workloads as W  # noqa: E402

cu = ctypes.CDLL("libcuda.so.1")
vp = ctypes.c_void_p


def check(rc, what):
    if rc != 0:
        print(f"{what} failed: {rc}")
        sys.exit(2)


def dev_alloc(nbytes):
    p = ctypes.c_uint64(0)
    check(cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(max(int(nbytes), 16))), "cuMemAlloc")
    return p.value


def to_dev(a):
    a = np.ascontiguousarray(a)
    p = dev_alloc(a.nbytes)
    check(cu.cuMemcpyHtoD_v2(ctypes.c_uint64(p), a.ctypes.data_as(vp), ctypes.c_size_t(a.nbytes)), "cuMemcpyHtoD")
    return p


def from_dev(p, nbytes, dtype=np.uint8):
    out = np.zeros(nbytes // np.dtype(dtype).itemsize, dtype)
    check(cu.cuMemcpyDtoH_v2(out.ctypes.data_as(vp), ctypes.c_uint64(p), ctypes.c_size_t(nbytes)), "cuMemcpyDtoH")
    return out


def run_once(L, seed):
    n = 700
    lengths = W.uniform_lengths(seed, n, 0, 3000)
    lengths[:5] = [0, 1, 16, 17, 9000]  # empty, one byte, one block, ragged, a tile-phase message
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_np(seed, synth.STREAM_DATA, max(total, 16))
    out_off, out_total = B.pack_offsets(lengths)
    keys = W.message_keys(seed, n)
    kb = W.key_sizes(seed, n)
    ivs = W.message_ivs(seed, n, counter0=0xFFFFFF00)
    d = B.AesBatch()
    d.n_msgs, d.op = n, B.BATCH_CTR
    d.in_ = to_dev(data)
    d.in_off = to_dev(in_off.astype(np.uint64))
    d.in_len = to_dev(lengths.astype(np.uint64))
    d.out_off = to_dev(out_off.astype(np.uint64))
    d.keys = to_dev(keys)
    d.key_bits = to_dev(kb.astype(np.uint32))
    d.iv = to_dev(ivs)
    results = []
    for noalloc in (False, True):
        d.out = dev_alloc(out_total + 16)
        d.out_len = dev_alloc(8 * n)
        d.status = dev_alloc(4 * n)
        if noalloc:
            check(L.aes_batch_submit_noalloc(ctypes.byref(d), None), "aes_batch_submit_noalloc")
        else:
            ws_bytes = L.aes_batch_workspace_size(n)
            check(L.aes_batch_submit(ctypes.byref(d), vp(dev_alloc(ws_bytes)), ws_bytes, None), "aes_batch_submit")
        check(cu.cuCtxSynchronize(), "cuCtxSynchronize")
        results.append((from_dev(d.out, out_total), from_dev(d.out_len, 8 * n, np.uint64),
                        from_dev(d.status, 4 * n, np.int32)))
    (o1, l1, s1), (o2, l2, s2) = results
    if not (np.array_equal(o1, o2) and np.array_equal(l1, l2) and np.array_equal(s1, s2)):
        print(f"mismatch (seed {seed})")
        sys.exit(3)
    if int((s1 != 0).sum()) != 0 or not np.array_equal(l1, lengths.astype(np.uint64)):
        print(f"unexpected status or length (seed {seed})")
        sys.exit(4)


def main():
    L = B._declare()
    L.aes_batch_submit_noalloc.argtypes = [ctypes.POINTER(B.AesBatch), vp]
    L.aes_batch_submit_noalloc.restype = ctypes.c_int
    check(cu.cuInit(0), "cuInit")
    dev = ctypes.c_int(0)
    check(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
    primary = vp()
    check(cu.cuDevicePrimaryCtxRetain(ctypes.byref(primary), dev), "cuDevicePrimaryCtxRetain")
    check(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent")
    run_once(L, 1)
    second = vp()
    if hasattr(cu, "cuCtxCreate_v4"):
        check(cu.cuCtxCreate_v4(ctypes.byref(second), None, 0, dev), "cuCtxCreate")
    else:
        check(cu.cuCtxCreate_v2(ctypes.byref(second), 0, dev), "cuCtxCreate")
    check(cu.cuCtxSetCurrent(second), "cuCtxSetCurrent")
    run_once(L, 2)
    check(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent")
    run_once(L, 3)
    check(cu.cuCtxSynchronize(), "cuCtxSynchronize")
    check(cu.cuCtxDestroy_v2(second), "cuCtxDestroy")
    print("OK")


if __name__ == "__main__":
    main()
