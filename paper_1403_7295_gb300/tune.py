"""Launch-shape autotuner for the single-buffer calls.

Times every (variant, CTA size, blocks per thread) candidate for each
(mode, key size) on a device-resident buffer with CUDA events and reports
the fastest.  The library's compiled-in defaults (``default_shape`` in
``csrc/aes_api.cu``) are set from this table as measured on GB300; callers
can also pass the tuned shape per call through the ``_ex`` entry points.

    python -m paper_1403_7295_gb300.tune [--size-mib 1024] [--reps 10] [--json out.json]
"""
from __future__ import annotations

import argparse
import json

CTAS = (256, 512, 768, 1024)
BPTS = (1, 2, 4)
MODES = ("ctr", "ecb_enc", "ecb_dec")
BITS = (128, 192, 256)


def _call(A, mode, ks, iv, x, y, cfg):
    if mode == "ctr":
        return A.aes_ctr_xcrypt(ks, iv, x, y, config=cfg)
    if mode == "ecb_enc":
        return A.aes_ecb_encrypt(ks, x, y, config=cfg)
    return A.aes_ecb_decrypt(ks, x, y, config=cfg)


def candidates(mode: str = "ctr"):
    for cta in CTAS:
        for bpt in ((0,) + BPTS if mode == "ctr" else BPTS):  # 0: the run-cached CTR kernel
            yield dict(variant=1, cta_threads=cta, blocks_per_thread=bpt, grid_ctas=0)
    yield dict(variant=2, cta_threads=0, blocks_per_thread=0, grid_ctas=0)


def autotune_single(size_mib: int = 1024, reps: int = 10, modes=MODES, bits_list=BITS) -> dict:
    import torch

    import synth

    from . import aes as A

    n = size_mib << 20
    x = synth.bytes_torch(11, synth.STREAM_DATA, n, device="cuda")
    y = torch.empty_like(x)
    iv = synth.iv_bytes(11)
    table = {}
    for bits in bits_list:
        ks = A.aes_expand_key(synth.key_bytes(11, bits))
        for mode in modes:
            results = []
            for cfg in candidates(mode):
                _call(A, mode, ks, iv, x, y, cfg)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    _call(A, mode, ks, iv, x, y, cfg)
                e1.record()
                torch.cuda.synchronize()
                gbps = n * reps / (e0.elapsed_time(e1) / 1e3) / 1e9
                results.append((gbps, cfg))
            results.sort(key=lambda r: -r[0])
            best_gbps, best = results[0]
            table[f"{mode}/{bits}"] = {"best": best, "gbps": round(best_gbps, 1),
                                       "all": [(round(g, 1), c) for g, c in results]}
    return table


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--size-mib", type=int, default=1024)
    p.add_argument("--reps", type=int, default=10)
    p.add_argument("--json", default=None)
    a = p.parse_args()
    t = autotune_single(a.size_mib, a.reps)
    for k, v in t.items():
        print(k, v["gbps"], v["best"])
    if a.json:
        json.dump(t, open(a.json, "w"), indent=1)


if __name__ == "__main__":
    main()
