"""Readers for the fixtures in tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _hex(s):
    return np.frombuffer(bytes.fromhex(s), np.uint8) if s != "-" else np.zeros(0, np.uint8)


def aes_vectors():
    out = []
    for ln in open(os.path.join(GOLDEN, "aes_vectors.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        mode, bits, key, iv, data, res = ln.split()
        out.append(dict(mode=mode, bits=int(bits), key=_hex(key), iv=_hex(iv), data=_hex(data), out=_hex(res)))
    return out


def paper_table1():
    rows = []
    for ln in open(os.path.join(GOLDEN, "paper_table1.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        method, proc, best, per_core = ln.split()
        rows.append((method, proc, int(best), int(per_core)))
    return rows
