#!/usr/bin/env python3
"""Throughput bench for GB300 bulk AES (one JSON line on rank 0).

Default workload: AES-128 CTR encryption of one 8 GiB buffer of seeded
uniform random bytes (the largest buffer of the single-buffer sweep, 64 MiB /
1 GiB / 8 GiB), data resident in HBM, one library call per step.  The input
is larger than L2 (129 MB), so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--bits 128|192|256] [--mode ctr|ecb_enc|ecb_dec] [--size-mib M]
                  [--sweep] [--no-e2e] [--no-cpu] [--no-probes]

Under torchrun (N > 1) every rank encrypts its own buffer (weak scaling, no
data-path collective: the blocks are independent); the barrier and the
max-over-ranks of the elapsed time are the only collectives.

`--impl reference` times the CPU oracle (test infrastructure, the one other
place this file runs it) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "AES-128/256 ECB/CTR GB/s on 1 GB300 vs roofline; batched-vs-plain; p50/p99"
PAPER_BEST_GBPS = 6637e6 / 8 / 1e9  # Table I: 6637 Mb/s, pthreads on 32 cores (context only)
SM_MAX_MHZ_FALLBACK = 2070.0
HBM_FALLBACK_GBPS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    p.add_argument("--bits", type=int, default=128, choices=[128, 192, 256])
    p.add_argument("--mode", default="ctr", choices=["ctr", "ecb_enc", "ecb_dec"])
    p.add_argument("--size-mib", type=int, default=8192)
    p.add_argument("--variant", type=int, default=0, help="0 auto, 1 T-table, 2 bitsliced, 3 T-table with TMA-staged input (CTR)")
    p.add_argument("--cta", type=int, default=0)
    p.add_argument("--bpt", type=int, default=0)
    p.add_argument("--sweep", action="store_true", help="also time the 36-run key/mode/size sweep")
    p.add_argument("--file-pipeline", action="store_true",
                   help="also time file -> encrypted file (4 GiB in /dev/shm), direct (mapped files) and staged paths")
    p.add_argument("--no-scaling", action="store_true",
                   help="skip the compact scaling study (throughput vs buffer size and vs CTAs, the paper's "
                        "Figs. 4-9 on GPU, plus the CTR size sweep at 64 MiB / 1 GiB / 8 GiB)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-probes", action="store_true")
    p.add_argument("--no-variants", action="store_true", help="skip the T-table vs bitsliced comparison")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-message workloads")
    p.add_argument("--only", choices=["all", "batched", "small"], default="all",
                   help="'batched': time only the batched varlen workload; 'small': only the "
                        "1,000,000 packet-sized messages (profiling entries)")
    p.add_argument("--batch-msgs", type=int, default=16384, help="messages in the batched varlen workload")
    p.add_argument("--short-path", choices=["auto", "groups", "lanes"], default="auto",
                   help="with --only: the batch's short-message path (aes_batch_config.short_path)")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="duration of the serving leg (Poisson 50k req/s, the configured 60 s); 0 skips it "
                        "and the loaded point")
    p.add_argument("--serve-loaded-seconds", type=float, default=10.0,
                   help="duration of the loaded serving point (Poisson 250k req/s, 1 GiB budget); 0 skips it")
    return p.parse_args()


# ---------------------------------------------------------------------------
# environment: ranks, peaks, clocks
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d.get("hbm_gbs", HBM_FALLBACK_GBPS), d.get("sm_max_mhz", SM_MAX_MHZ_FALLBACK), "measured"
    return HBM_FALLBACK_GBPS, SM_MAX_MHZ_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str, period_ms: int = 25):
        self.gpu_id = gpu_id
        self.period_ms = period_ms
        self.proc = None
        self.lines: list[str] = []
        self.stamps: list[float] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms), "-i", self.gpu_id], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL,
                text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.stamps.append(time.perf_counter())
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        return self.summary()

    def summary(self, t0: float | None = None, t1: float | None = None) -> dict:
        """Median SM clock, max clock, power and throttle reasons of the
        samples read between perf_counter times t0 and t1 (all if None)."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, ln in zip(list(self.stamps), list(self.lines)):
            if (t0 is not None and ts < t0) or (t1 is not None and ts > t1):
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm),
            "reasons": sorted(reasons),
        }


# ---------------------------------------------------------------------------
# probes: the roofline's on-chip denominators
# ---------------------------------------------------------------------------

PROBE_NAMES = ["lop3", "prmt", "iadd", "shf", "imad", "lds32", "lop3+imad", "lop3+lds32",
               "prmt+lds32", "lop3+prmt"]


def run_probes() -> dict:
    from paper_1403_7295_gb300 import build as B

    L = ctypes.CDLL(B.PROBE_LIB_PATH)
    L.aesgpu_probe_pipe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    out = {}
    for kind, name in enumerate(PROBE_NAMES):
        r, s = ctypes.c_double(), ctypes.c_double()
        rc = L.aesgpu_probe_pipe(kind, 1024, 2000, ctypes.byref(r), ctypes.byref(s))
        out[name] = round(r.value, 2) if rc == 0 else None
    return out


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

# Algorithmic table lookups per 16-byte block: one per state byte per round
# (paper Fig. 1: Nr rounds of SubBytes over 16 bytes).
def lookups_per_block(bits: int) -> int:
    return 16 * {128: 10, 192: 12, 256: 14}[bits]


def launch(A, mode, ks, iv, x, y, cfg, stream=None):
    if mode == "ctr":
        return A.aes_ctr_xcrypt(ks, iv, x, y, stream=stream, config=cfg)
    if mode == "ecb_enc":
        return A.aes_ecb_encrypt(ks, x, y, stream=stream, config=cfg)
    return A.aes_ecb_decrypt(ks, x, y, stream=stream, config=cfg)


def per_step_stats(torch, fn, n):
    """Per-call CUDA-event times of n calls (after the timed region): median,
    p99, and the paper's averaging (repeat, drop the runs that deviate most,
    average the rest), read as: drop samples more than 3 median absolute
    deviations from the median."""
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    t = np.array([a.elapsed_time(b) for a, b in ev])
    med = float(np.median(t))
    mad = float(np.median(np.abs(t - med)))
    keep = t[np.abs(t - med) <= 3 * mad] if mad > 0 else t
    return {"n": n, "median_ms": round(med, 5), "p99_ms": round(float(np.percentile(t, 99)), 5),
            "paper_mean_ms": round(float(keep.mean()), 5), "paper_mean_kept": int(keep.size),
            "min_ms": round(float(t.min()), 5), "max_ms": round(float(t.max()), 5)}


def time_device(torch, fn, steps, warmup, barrier=None):
    """CUDA-event time of `steps` calls of fn() on the current stream (ms total)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return e0.elapsed_time(e1)


def gpu_arm(args):
    import torch

    if args.only in ("batched", "small"):
        return batched_only(args)

    from paper_1403_7295_gb300 import aes as A
    from paper_1403_7295_gb300 import build as B

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    barrier = (lambda: dist.barrier()) if dist else None

    B.build()
    A.lib()
    nbytes = args.size_mib << 20
    seed = rank
    bits = args.bits
    # Every rank holds one shard of a logical world x size buffer under one key:
    # rank r's counter starts at its first block (the paper's chunk split, no
    # exchange); the library's aes_ctr_iv_advance gives that IV.
    key = synth.key_bytes(0, bits)
    iv = np.frombuffer(A.aes_ctr_iv_advance(synth.iv_bytes(0), rank * (nbytes // 16)), np.uint8)
    ks = A.aes_expand_key(key)
    x = synth.bytes_torch(seed, synth.STREAM_DATA, nbytes, device="cuda")
    y = torch.empty_like(x)
    cfg = None
    if args.variant or args.cta or args.bpt:
        cfg = dict(variant=args.variant, cta_threads=args.cta, blocks_per_thread=args.bpt, grid_ctas=0)

    hbm_peak, sm_max_mhz, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    gpu_id = str(getattr(props, "uuid", local))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) == 36:
        gpu_id = "GPU-" + gpu_id

    probes = run_probes() if (rank == 0 and not args.no_probes) else None

    sampler = ClockSampler(gpu_id) if rank == 0 else None
    if sampler:
        sampler.start()
    ms = time_device(torch, lambda: launch(A, args.mode, ks, iv, x, y, cfg), args.steps, args.warmup,
                     barrier)
    clocks = sampler.summary() if sampler else None
    dist_steps = per_step_stats(torch, lambda: launch(A, args.mode, ks, iv, x, y, cfg), min(args.steps, 200))
    t = torch.tensor([ms], device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    per_launch_s = ms / 1e3 / args.steps  # this rank's kernel, one launch per step
    value = world * nbytes * args.steps / (ms_max / 1e3) / 1e9

    result = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic: SplitMix64-seeded uniform random bytes",
        "config": {
            "workload": f"AES-{bits} {args.mode.upper()} of one {args.size_mib} MiB buffer per GPU, "
                        "device-resident (single-buffer sweep 64 MiB / 1 GiB / 8 GiB; "
                        + ("its largest buffer)" if args.size_mib == 8192 else "not its largest buffer)"),
            "key_bits": bits, "mode": args.mode, "buffer_bytes": nbytes,
            "l2": "input larger than L2 (129 MB); no flush",
            "launch": cfg or "library default",
            "parallelism": f"{world} contiguous shards of one {world * args.size_mib} MiB buffer "
                           "(one key, counter offset per shard, no data exchange)",
        },
        "gpu_launches": args.steps,
    }
    if rank == 0:
        blocks = nbytes / 16
        result["roofline"] = roofline(args, bits, nbytes, per_launch_s, probes, sms, sm_max_mhz,
                                      hbm_peak, peak_src)
        dist_steps["gbps_at_median"] = round(nbytes / (dist_steps["median_ms"] / 1e3) / 1e9, 2)
        dist_steps["how"] = ("one event pair per launch, after the timed region (rank 0); the timed "
                             "value above is the event span over all steps")
        result["per_step"] = dist_steps
        result["probes_ops_per_clk_per_sm"] = probes
        result["clocks"] = clocks
        result["context"] = {"paper_best_cpu_gbps": round(PAPER_BEST_GBPS, 3),
                             "paper_best_cpu": "6637 Mb/s, pthreads, 4x Xeon X7560 (Table I)"}
        del blocks
        if not args.no_variants:
            result["variants"] = variant_arm(torch, A, args, ks, iv, x, y, value)
            result["other_modes"] = modes_arm(torch, A, x[: 1 << 30], y[: 1 << 30])
        if not args.no_scaling:
            result["scaling_study"] = scaling_study(torch, A, x, y, sampler)
        if sampler:
            sampler.stop()
        if args.sweep:
            result["sweep"] = sweep(torch, A)
        if args.file_pipeline:
            result["file_pipeline"] = file_pipeline(torch)
        del x, y
        torch.cuda.empty_cache()
        x = y = None
        if not args.no_e2e:
            result["e2e"] = e2e_arm(torch, A, args, ks, iv, nbytes, cfg)
        if not args.no_batch:
            result["batched"] = batched_arm(torch, A)
        if args.serve_seconds > 0:
            torch.cuda.empty_cache()
            result["serving"] = serving_arm(torch, args.serve_seconds)
            if args.serve_loaded_seconds > 0:
                result["serving_loaded"] = serving_arm(torch, args.serve_loaded_seconds, rate=250_000.0,
                                                       budget_bytes=1 << 30)
        torch.cuda.empty_cache()
        if not args.no_cpu:
            result["cpu_baseline"] = cpu_baseline(args.bits, args.mode, budget_s=10.0)
        print(json.dumps(result), flush=True)
    else:
        del x, y
        torch.cuda.empty_cache()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def roofline(args, bits, nbytes, per_launch_s, probes, sms, clock_mhz, hbm_peak, peak_src):
    """The headline kernel against its three ceilings, each as GB/s of
    plaintext: HBM (2 bytes moved per plaintext byte at the measured copy
    bandwidth), the shared-memory pipe (the kernel's executed table lookups
    per block at the probe's conflict-free LDS.32 rate) and the integer ALU
    pipe (the kernel's ALU thread-instructions per block, from its ncu
    summary, at the probe's LOP3 rate: the INT32 term).  The roofline is the
    slowest of the three; `achieved`/`peak`/`frac` are the binding
    shared-memory pipe's executed lookups per second against its peak."""
    blocks = nbytes / 16
    nr = {128: 10, 192: 12, 256: 14}[bits]
    value_gbps = nbytes / per_launch_s / 1e9
    hbm_ceiling = hbm_peak / 2
    rl = {"hbm_gbps_moved": round(2 * nbytes / per_launch_s / 1e9, 1), "hbm_peak_gbps": hbm_peak,
          "hbm_frac": round(2 * value_gbps / hbm_peak, 4),
          "hbm_peak_source": f"{peak_src} (MEASURED_PEAKS.json copy bandwidth)" if peak_src == "measured"
          else "fallback 6.8 TB/s", "traffic": read_traffic(args)}
    if args.variant == 2:
        # bitsliced rounds: no lookups; bound by the ALU pipe (LOP3 / PRMT / SHF)
        ops = read_profile_field(args, "thread_instructions_per_block_measured:")
        rl.update({"bound": "alu", "unit": "Gop/s", "achieved": None, "peak": None, "frac": None,
                   "ops_per_block": ops, "pipe": "64-lane ALU pipe (LOP3, PRMT, SHF of the bitsliced circuit)"})
        if ops and probes and probes.get("lop3"):
            peak = probes["lop3"] * sms * clock_mhz * 1e6 / 1e9
            rl["achieved"] = round(ops * blocks / per_launch_s / 1e9, 1)
            rl["peak"] = round(peak, 1)
            rl["frac"] = round(rl["achieved"] / peak, 4)
            rl["peak_source"] = (f"measured probe: {probes['lop3']} LOP3 per clock per SM x {sms} SMs "
                                 f"x {clock_mhz:.0f} MHz (max SM clock), of measured")
        return rl
    lk = read_profile_field(args, "lookups_per_block_measured:")
    lk_src = "ncu (committed summary of this kernel source)"
    if lk is None:
        lk = executed_lookups_per_block(args, bits, nbytes, sms)
        lk_src = "the kernel's own lookup count, derived from its structure (no current ncu summary)"
    alu = read_profile_field(args, "alu_instructions_per_block_measured:")
    rl.update({"bound": "alu", "unit": "Glookup/s", "achieved": None, "peak": None, "frac": None,
               "pipe": "shared-memory (LSU) pipe: replicated T-table lookups, 32-bit conflict-free",
               "lookups_per_block_executed": lk, "lookups_source": lk_src,
               "analytic_ops_per_block": 16 * nr,
               "analytic_ops": "one table lookup per state byte per round (paper Fig. 1: SubBytes over "
                               "16 bytes in each of Nr rounds) = 16*Nr; the run-cached CTR kernel executes fewer"})
    terms = {"hbm": round(hbm_ceiling, 1)}
    if probes and probes.get("lds32") and lk:
        peak = probes["lds32"] * sms * clock_mhz * 1e6 / 1e9
        rl["achieved"] = round(lk * blocks / per_launch_s / 1e9, 1)
        rl["peak"] = round(peak, 1)
        rl["frac"] = round(rl["achieved"] / peak, 4)
        rl["achieved_analytic"] = round(16 * nr * blocks / per_launch_s / 1e9, 1)
        rl["peak_source"] = (f"measured probe: {probes['lds32']} conflict-free LDS.32 per clock per SM x {sms} "
                             f"SMs x {clock_mhz:.0f} MHz (max SM clock), of measured")
        terms["lds"] = round(peak * 1e9 / lk * 16 / 1e9, 1)
    if probes and probes.get("lop3") and alu:
        ipeak = probes["lop3"] * sms * clock_mhz * 1e6 / 1e9
        rl["int32"] = {"alu_instructions_per_block": alu, "unit": "Gop/s",
                       "achieved": round(alu * blocks / per_launch_s / 1e9, 1), "peak": round(ipeak, 1),
                       "frac": round(alu * blocks / per_launch_s / 1e9 / ipeak, 4),
                       "peak_source": f"measured probe: {probes['lop3']} LOP3 per clock per SM (the 64-lane "
                                      f"integer ALU pipe that LOP3, PRMT and SHF share) x {sms} SMs x "
                                      f"{clock_mhz:.0f} MHz, of measured",
                       "count_source": "ncu sm__inst_executed_pipe_alu of the committed summary"}
        terms["alu"] = round(ipeak * 1e9 / alu * 16 / 1e9, 1)
    rl["ceilings_gbps_plaintext"] = terms
    binding = min(terms, key=terms.get)
    rl["binding"] = binding
    rl["roofline_gbps_plaintext"] = terms[binding]
    rl["frac_of_roofline"] = round(value_gbps / terms[binding], 4)
    return rl


def executed_lookups_per_block(args, bits, nbytes, sms):
    """Table lookups the default CTR kernel executes per block, from its
    structure: 16 per full round from round 3 on and in the final round, 5
    for rounds 1-2 (the counter byte's round-1 lookup and its four round-2
    lookups), and 15 per counter-run piece for the run's constants.  Other
    modes and launch shapes execute the full 16*Nr."""
    nr = {128: 10, 192: 12, 256: 14}[bits]
    if args.mode != "ctr" or args.bpt or args.variant not in (0, 1):
        return 16 * nr
    units = nbytes // 16 + (1 if nbytes % 16 else 0)
    runs = (units + 255) // 256
    warps = sms * 32  # one 1024-thread CTA per SM
    whole = runs - runs % warps
    tail = runs - whole
    # the kernel's split of the last partial wave: P pieces of 8 / P steps per run,
    # P minimising the busiest warp's cost there in quarter steps (4 per step, 1 per
    # piece's setup), the fewest pieces on a tie
    split = min((1, 2, 4, 8), key=lambda p: (-(-tail * p // warps) * (32 // p + 1), p)) if tail else 1
    pieces = whole + tail * split
    return round(16 * (nr - 2) + 5 + 15 * pieces / (nbytes / 16), 3)


# The committed ncu summary of each round implementation's AES-128 CTR kernel,
# with the sources whose hash it records (numbers from a stale summary are
# not used).
PROFILE_OF_VARIANT = {
    0: ("ttable_ctr_aes128_8GiB.md", ["aes_ttable.cuh"]),
    1: ("ttable_ctr_aes128_8GiB.md", ["aes_ttable.cuh"]),
    2: ("bitslice_ctr_aes128_256MiB.md", ["aes_bitslice.cu", "aes_bitslice_circuit.cuh"]),
}


def read_profile_field(args, key):
    """A number from the committed ncu summary of the kernel this run uses
    (AES-128 CTR only), if the summary still matches the kernel's source."""
    import hashlib

    if args.mode != "ctr" or args.bits != 128 or args.bpt or args.variant not in PROFILE_OF_VARIANT:
        return None
    name, sources = PROFILE_OF_VARIANT[args.variant]
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    h = hashlib.sha256()
    for src in sources:
        h.update(open(os.path.join(ROOT, "paper_1403_7295_gb300", "csrc", src), "rb").read())
    text = open(path).read()
    if f"source_sha256_16: {h.hexdigest()[:16]}" not in text:
        return None
    for ln in text.splitlines():
        if ln.startswith(key):
            return float(ln.split()[1])
    return None


def read_traffic(args):
    """dram bytes per launch from the committed ncu summary (scaled from its
    per-GiB figure to this buffer), if it still matches the kernel source;
    else null."""
    per_gib = read_profile_field(args, "traffic_bytes_per_GiB_launch:")
    return None if per_gib is None else per_gib * (args.size_mib / 1024)


def modes_arm(torch, A, x, y):
    """CBC decryption and XTS (4 KiB units) on the same 1 GiB buffer, AES-128 and AES-256."""
    out = {}
    iv = synth.iv_bytes(13)
    for bits in (128, 256):
        k1 = A.aes_expand_key(synth.key_bytes(13, bits))
        k2 = A.aes_expand_key(synth.key_bytes(14, bits))
        n = x.numel()
        for name, fn in (("cbc_decrypt", lambda: A.aes_cbc_decrypt(k1, iv, x, y)),
                         ("xts_encrypt", lambda: A.aes_xts_encrypt(k1, k2, 0, 4096, x, y)),
                         ("xts_decrypt", lambda: A.aes_xts_decrypt(k1, k2, 0, 4096, x, y))):
            ms = time_device(torch, fn, 50, 3)
            out[f"{name}_{bits}_gbps"] = round(n * 50 / (ms / 1e3) / 1e9, 1)
    return out


def variant_arm(torch, A, args, ks, iv, x, y, ttable_gbps):
    """The round implementations on the headline workload: the library's
    choice (T-tables) against the bitsliced circuit; for CTR also the
    T-table kernel with TMA-staged input against the default's plain loads,
    at the headline size and at 1 GiB, timed back to back."""
    cfg = dict(variant=2, cta_threads=0, blocks_per_thread=0, grid_ctas=0)
    steps = max(10, args.steps // 10)
    ms = time_device(torch, lambda: launch(A, args.mode, ks, iv, x, y, cfg), steps, 3)
    bs = x.numel() * steps / (ms / 1e3) / 1e9
    out = {"ttable_gbps": round(ttable_gbps, 1), "bitslice_gbps": round(bs, 1),
           "chosen": "ttable" if ttable_gbps >= bs else "bitslice"}
    if args.mode == "ctr" and not args.variant and not args.cta and not args.bpt:
        bulk = dict(variant=3, cta_threads=0, blocks_per_thread=0, grid_ctas=0)
        tma = {}
        for n in sorted({x.numel(), min(1 << 30, x.numel())}):
            xs, ys = x[:n], y[:n]
            k = max(10, int(20 * (8 << 30) / n) // 10)
            g = {}
            for name, c in (("default_plain_loads", None), ("tma_bulk_staged", bulk),
                            ("default_plain_loads_again", None)):
                t = time_device(torch, lambda: A.aes_ctr_xcrypt(ks, iv, xs, ys, config=c), k, 3)
                g[name] = round(n * k / (t / 1e3) / 1e9, 1)
            tma[f"{n >> 20}_MiB"] = g
        out["tma_staging"] = tma
        out["tma_wait_timeouts"] = A.aes_take_wait_timeouts()
    return out


def e2e_arm(torch, A, args, ks, iv, nbytes, cfg):
    """Same call with pinned HOST buffers: the kernel reads the input from
    host memory and writes the result back to host memory (NVLink-C2C), so
    both transfers are inside the timed call."""
    h_in = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_in.copy_(synth.bytes_torch(0, synth.STREAM_DATA, nbytes, device="cuda").cpu())
    h_out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    steps = max(20, min(50, args.steps // 5))
    ms = time_device(torch, lambda: launch(A, args.mode, ks, iv, h_in, h_out, cfg), steps, 3)
    val = nbytes * steps / (ms / 1e3) / 1e9
    # The ceiling: the host link moving bytes both ways at once (copy engines,
    # H2D and D2H on two streams), on 1 GiB of the same pinned buffers (the
    # copy engines run slower on single multi-GiB pinned copies).
    lk = min(nbytes, 1 << 30)
    d_a = torch.empty(lk, dtype=torch.uint8, device="cuda")
    d_b = torch.empty_like(d_a)
    h_in_l, h_out_l = h_in[:lk], h_out[:lk]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def both_ways():
        cur = torch.cuda.current_stream()
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            d_a.copy_(h_in_l, non_blocking=True)
        with torch.cuda.stream(s2):
            h_out_l.copy_(d_b, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    # the link's capacity: best of three short samples (one sample can land on a
    # disturbed moment of the host's memory system)
    link = max(lk * 5 / (time_device(torch, both_ways, 5, 2) / 1e3) / 1e9 for _ in range(3))
    del d_a, d_b, h_in, h_out, h_in_l, h_out_l
    return {"value": round(val, 2), "unit": "GB/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": steps,
            "how": "aes call on pinned host input/output buffers (the kernel reads and writes host "
                   "memory over NVLink-C2C)",
            "link_gbps_each_way": round(link, 1), "link_how": f"copy engines, H2D and D2H at once, {lk >> 20} MiB",
            "frac_of_link": round(val / link, 3)}


def time_graph(torch, b, steps):
    """CUDA-event time (ms) of `steps` replays of a captured batch graph."""
    return time_device(torch, b.replay, steps, 3)


def batched_only(args):
    """Just one batched CTR workload: the varlen one at --batch-msgs messages
    (tile 32768), or with --only small the 1,000,000 packet-sized AES-128
    messages (tile 8192); --cta picks the CTA size (default 1024); --warmup
    then --steps graph replays (the profiling entries for the batch kernel)."""
    import torch

    from paper_1403_7295_gb300 import aes as A
    from paper_1403_7295_gb300 import batch as B
    from paper_1403_7295_gb300 import build as BLD
    from synth import workloads as W

    BLD.build()
    A.lib()
    small = args.only == "small"
    wl = W.small_messages(4, 1_000_000) if small else W.batched_varlen(3, args.batch_msgs)
    lengths = wl["lengths"]
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(3, synth.STREAM_DATA, total, device="cuda")
    b = B.Batch(B.BATCH_CTR, data, in_off, lengths, keys=wl["keys"], key_bits=wl["key_bits"], ivs=wl["ivs"])
    path = {"auto": B.SHORT_AUTO, "groups": B.SHORT_GROUPS, "lanes": B.SHORT_LANES}[args.short_path]
    b.capture(B.AesBatchConfig(args.cta or 1024, 8192 if small else 32768, 0, path))
    ms = time_graph(torch, b, args.steps) if args.warmup >= 3 else time_device(torch, b.replay, args.steps, args.warmup)
    gbps = b.total_input_bytes() * args.steps / (ms / 1e3) / 1e9
    name = "1,000,000 packet-sized messages" if small else f"{args.batch_msgs} messages"
    print(json.dumps({"workload": f"batched varlen CTR, {name}", "bytes": b.total_input_bytes(),
                      "short_path": args.short_path,
                      "gbps": round(gbps, 1), "ms_per_batch": round(ms / args.steps, 3)}), flush=True)


# aes_batch_config.short_path values, as reported in the batched results
SHORT_PATH_NAMES = {0: "auto", 1: "groups (per-warp message groups, keys in shared memory)",
                    2: "lanes (one lane per message, keys in registers)"}


def batched_arm(torch, A):
    """Batched workloads: (a) 16,384 messages, log-uniform 64 B .. 4 MiB, mixed
    key sizes, CTR, one persistent launch in a CUDA graph with an autotuned
    shape, against the byte-weighted harmonic mix of single-buffer 1 GiB CTR
    rates; (b) 1,000,000 packet-sized AES-128 CTR messages with keys expanded
    on the device vs pre-expanded schedules.  The autotuner picks the launch
    shape and, for CTR, the short-message path (per-warp groups or one lane
    per message) by timing both on the batch itself."""
    from paper_1403_7295_gb300 import batch as B
    from synth import workloads as W

    out = {}
    # single-buffer 1 GiB CTR rates per key size, measured here beside the batches
    rates = {}
    n = 1 << 30
    x = synth.bytes_torch(7, synth.STREAM_DATA, n, device="cuda")
    y = torch.empty_like(x)
    for bits in (128, 192, 256):
        ks = A.aes_expand_key(synth.key_bytes(7, bits))
        iv = synth.iv_bytes(7)
        ms = time_device(torch, lambda: A.aes_ctr_xcrypt(ks, iv, x, y), 100, 5)
        rates[bits] = n * 100 / (ms / 1e3) / 1e9
    del x, y
    torch.cuda.empty_cache()

    wl = W.batched_varlen(3, 16384)
    lengths, kb = wl["lengths"], wl["key_bits"]
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(3, synth.STREAM_DATA, total, device="cuda")
    b = B.Batch(B.BATCH_CTR, data, in_off, lengths, keys=wl["keys"], key_bits=kb, ivs=wl["ivs"])
    cfg = B.autotune(b)
    b.capture(cfg)
    steps = 50
    ms = time_graph(torch, b, steps)
    nbytes = b.total_input_bytes()
    gbps = nbytes * steps / (ms / 1e3) / 1e9
    by_bits = {bits: float(lengths[kb == bits].sum()) for bits in (128, 192, 256)}
    mix = sum(by_bits.values()) / sum(by_bits[k] / rates[k] for k in by_bits)
    st = per_step_stats(torch, b.replay, 20)
    out["varlen_16384"] = {
        "gbps": round(gbps, 1), "bytes": nbytes, "ms_per_batch": round(ms / steps, 3),
        "per_batch": {k: st[k] for k in ("median_ms", "p99_ms", "paper_mean_ms")},
        "plain_ctr_1GiB_gbps": {str(k): round(v, 1) for k, v in rates.items()},
        "plain_mix_gbps": round(mix, 1), "ratio_vs_plain": round(gbps / mix, 4),
        "launch": {"cta_threads": cfg.cta_threads, "tile_blocks": cfg.tile_blocks,
                   "short_path": SHORT_PATH_NAMES[cfg.short_path]},
        "kernels_per_batch": 2 if cfg.short_path != B.SHORT_LANES else 4, "graph": True,
    }
    # the same messages as ECB + PKCS#7, encrypt then decrypt, against the ECB mix
    ecb_rates = {}
    x = synth.bytes_torch(7, synth.STREAM_DATA, 1 << 30, device="cuda")
    y = torch.empty_like(x)
    for bits in (128, 192, 256):
        kse = A.aes_expand_key(synth.key_bytes(7, bits))
        ms_e = time_device(torch, lambda: A.aes_ecb_encrypt(kse, x, y), 50, 3)
        ms_d = time_device(torch, lambda: A.aes_ecb_decrypt(kse, x, y), 50, 3)
        ecb_rates[bits] = ((1 << 30) * 50 / (ms_e / 1e3) / 1e9, (1 << 30) * 50 / (ms_d / 1e3) / 1e9)
    del x, y
    del b
    torch.cuda.empty_cache()
    enc = B.Batch(B.BATCH_ECB_PKCS7_ENCRYPT, data, in_off, lengths, keys=wl["keys"], key_bits=kb)
    enc.capture(B.autotune(enc))
    ms_enc = time_graph(torch, enc, 20)
    ct_len = (lengths // np.uint64(16) + np.uint64(1)) * np.uint64(16)
    dec = B.Batch(B.BATCH_ECB_PKCS7_DECRYPT, enc.out, enc.out_off_np, ct_len, keys=wl["keys"], key_bits=kb)
    dec.capture(B.autotune(dec))
    ms_dec = time_graph(torch, dec, 20)
    ok = int((dec.status != 0).sum()) == 0 and bool(torch.equal(dec.out_len.cpu(), torch.from_numpy(lengths.astype(np.int64))))
    mix_e = sum(by_bits.values()) / sum(by_bits[k] / ecb_rates[k][0] for k in by_bits)
    mix_d = sum(by_bits.values()) / sum(by_bits[k] / ecb_rates[k][1] for k in by_bits)
    g_e = nbytes * 20 / (ms_enc / 1e3) / 1e9
    g_d = float(ct_len.sum()) * 20 / (ms_dec / 1e3) / 1e9
    out["varlen_16384_ecb_pkcs7"] = {
        "encrypt_gbps": round(g_e, 1), "decrypt_gbps": round(g_d, 1),
        "plain_ecb_mix_gbps": {"encrypt": round(mix_e, 1), "decrypt": round(mix_d, 1)},
        "ratio_vs_plain": {"encrypt": round(g_e / mix_e, 4), "decrypt": round(g_d / mix_d, 4)},
        "decrypt_restored_every_length": ok,
    }
    del enc, dec, data
    torch.cuda.empty_cache()

    wl = W.small_messages(4, 1_000_000)
    lengths = wl["lengths"]
    in_off, total = B.pack_offsets(lengths)
    data = synth.bytes_torch(4, synth.STREAM_DATA, total, device="cuda")
    b = B.Batch(B.BATCH_CTR, data, in_off, lengths, keys=wl["keys"], key_bits=wl["key_bits"], ivs=wl["ivs"])
    cfg = B.autotune(b)
    b.capture(cfg)
    ms_dev = time_graph(torch, b, steps)
    st_small = per_step_stats(torch, b.replay, 30)
    nbytes = b.total_input_bytes()
    # the same batch with pre-expanded schedules (one per message)
    table = bytearray()
    keys = wl["keys"]
    for m in range(b.n):
        table += bytes(A.aes_expand_key(keys[m][:16], 128))
    sched = torch.frombuffer(table, dtype=torch.uint8).cuda()
    b2 = B.Batch(B.BATCH_CTR, data, in_off, lengths, schedules=sched, n_schedules=b.n,
                 sched_idx=np.arange(b.n, dtype=np.uint32), ivs=wl["ivs"], out=b.out)
    cfg2 = B.autotune(b2)  # its own choice: resident schedules load differently
    b2.capture(cfg2)
    ms_pre = time_graph(torch, b2, steps)
    g_dev = nbytes * steps / (ms_dev / 1e3) / 1e9
    out["small_1M"] = {
        "gbps_device_key_expansion": round(g_dev, 1),
        "single_buffer_ctr128_1GiB_gbps": round(rates[128], 1),
        "ratio_vs_single_buffer": round(g_dev / rates[128], 4),
        "gbps_preexpanded": round(nbytes * steps / (ms_pre / 1e3) / 1e9, 1),
        "bytes": nbytes, "ms_per_batch_device_keys": round(ms_dev / steps, 3),
        "ms_per_batch_preexpanded": round(ms_pre / steps, 3),
        "per_batch_device_keys": {k: st_small[k] for k in ("median_ms", "p99_ms", "paper_mean_ms")},
        "launch": {"cta_threads": cfg.cta_threads, "tile_blocks": cfg.tile_blocks,
                   "short_path": SHORT_PATH_NAMES[cfg.short_path]},
        "kernels_per_batch": 2 if cfg.short_path != B.SHORT_LANES else 4,
        "launch_preexpanded": {"cta_threads": cfg2.cta_threads, "tile_blocks": cfg2.tile_blocks,
                               "short_path": SHORT_PATH_NAMES[cfg2.short_path]},
    }
    return out


def serving_arm(torch, seconds: float, rate: float = 50_000.0, budget_bytes: int = 8 << 30) -> dict:
    """Continuous-batching server: Poisson arrivals at `rate`/s for `seconds`,
    sizes 70 % 1-16 KiB / 25 % 16 KiB-1 MiB / 5 % 1-64 MiB, AES-256 CTR with
    1,024 resident tenant schedules, admission under `budget_bytes` (the
    configured 8 GiB by default), inputs sliced from a 2 GiB device pool;
    p50/p99 of arrival -> completion."""
    from paper_1403_7295_gb300.serve import Server
    from synth import workloads as W

    pool_bytes = 2 << 30
    pool = synth.bytes_torch(5, synth.STREAM_DATA, pool_bytes, device="cuda")
    n_t = 1024
    keys = W.message_keys(5, n_t)
    bits = np.full(n_t, 256, dtype=np.uint32)
    nonces = synth.bytes_np(5, synth.STREAM_NONCE, 12 * n_t).reshape(n_t, 12)
    arr = W.poisson_arrivals(5, rate, seconds)
    n = arr.size
    lengths = W.serving_sizes(5, n)
    u = synth.uniform01(5, synth.STREAM_MISC + 3, n)
    offs = (np.floor(u * (pool_bytes - lengths.astype(np.float64))).astype(np.uint64) // 16) * 16
    tenants = W.tenants(5, n, n_t)
    srv = Server(pool, keys, bits, nonces, budget_bytes=budget_bytes, n_streams=2, slots_per_stream=2,
                 max_batch_msgs=8192)
    rep = srv.run(arr, tenants, offs, lengths, time_limit=seconds + 120.0)
    rep.pop("counters", None)
    rep["engine"] = "native aes_server_replay (admission, batching, launch and completion in the library)"
    rep.update({"rate_per_s": rate, "seconds": seconds, "key_bits": 256, "tenants": n_t,
                "budget_bytes": budget_bytes, "offered_gbps": float(lengths.sum()) / seconds / 1e9})
    for k in ("p50_ms", "p99_ms", "max_ms", "gbps", "wall_s", "mean_batch_msgs", "offered_gbps",
              "admission_wait_p99_ms", "admission_wait_mean_ms", "admission_wait_max_ms"):
        if rep.get(k) is not None:
            rep[k] = round(rep[k], 3)
    srv.close()
    del srv, pool
    torch.cuda.empty_cache()
    return rep


def file_pipeline(torch, nbytes: int = 4 << 30) -> dict:
    """The paper's workload end to end: a file of seeded bytes encrypted into
    another file (AES-128 CTR) through the native pipeline; the files live in
    /dev/shm when it exists, so the figure is not disk-bound."""
    import tempfile

    from paper_1403_7295_gb300.filecrypt import crypt_file

    base = "/dev/shm" if os.path.isdir("/dev/shm") else None
    with tempfile.TemporaryDirectory(dir=base) as d:
        src, dst = os.path.join(d, "plain"), os.path.join(d, "cipher")
        x = synth.bytes_torch(12, synth.STREAM_DATA, nbytes, device="cuda")
        x.cpu().numpy().tofile(src)
        del x
        key, iv = synth.key_bytes(12, 128), bytes(synth.iv_bytes(12))
        cold = crypt_file(src, dst, key, "ctr", iv)  # the default path: staged (pins its buffers)
        r = crypt_file(src, dst, key, "ctr", iv)
        r["where"] = base or tempfile.gettempdir()
        r["first_call_gbps"] = round(cold["gbps"], 3)
        r["first_call_setup_seconds"] = round(cold["setup_seconds"], 4)
        for k in ("seconds", "gbps", "setup_seconds"):
            r[k] = round(r[k], 4)
        r["how"] = ("native aes_file_crypt, default (staged) path, second call on the same files: workers "
                    "pread chunks into pinned buffers, the kernel encrypts them in place over NVLink-C2C, the "
                    "chunks are copied into a shared mapping of the output file")
        crypt_file(src, dst, key, "ctr", iv, direct=True)
        d = crypt_file(src, dst, key, "ctr", iv, direct=True)
        r["direct_gbps"] = round(d["gbps"], 3) if d["direct"] else None
        r["direct_how"] = ("opt-in direct path (AES_FILE_DIRECT): both files mapped, workers fault in each "
                           "chunk's pages and the kernel reads and writes the mappings over NVLink-C2C")
        return r


def scaling_study(torch, A, big, dst, sampler=None) -> dict:
    """The paper's throughput-vs-data-size and throughput-vs-parallel-instances
    curves (its Figs. 4-9, on CPUs) restated for one GB300, compact enough for
    every bench run: AES-128 CTR GB/s for buffers of 64 KiB .. the headline
    buffer, AES-128 and AES-256 CTR at the single-buffer sweep's 64 MiB, 1 GiB
    and 8 GiB, and AES-128 CTR on 1 GiB with 1 .. all SMs' worth of CTAs (one
    CTA per SM).  Every point carries the clocks sampled while it ran."""
    out = {"size_bytes": [], "size_gbps": [], "size_clocks_mhz": [],
           "ctr_sweep": [], "ctas": [], "ctas_gbps": [], "ctas_clocks_mhz": []}
    iv = synth.iv_bytes(9)
    n_big = big.numel()

    def point(fn, nbytes, target_s=0.15, max_steps=2000):
        one = time_device(torch, fn, 1, 2) / 1e3
        steps = int(min(max_steps, max(5, target_s / max(one, 1e-6))))
        t0 = time.perf_counter()
        ms = time_device(torch, fn, steps, 1)
        t1 = time.perf_counter()
        clk = sampler.summary(t0, t1) if sampler else {}
        return round(nbytes * steps / (ms / 1e3) / 1e9, 2), clk

    ks128 = A.aes_expand_key(synth.key_bytes(9, 128))
    for n in (64 << 10, 1 << 20, 16 << 20, 64 << 20, 256 << 20, 1 << 30, 8 << 30):
        if n > n_big:
            break
        x, y = big[:n], dst[:n]
        g, clk = point(lambda: A.aes_ctr_xcrypt(ks128, iv, x, y), n)
        out["size_bytes"].append(n)
        out["size_gbps"].append(g)
        out["size_clocks_mhz"].append(clk.get("sm_mhz"))
    for bits in (128, 256):
        ks = A.aes_expand_key(synth.key_bytes(9, bits))
        for n in (64 << 20, 1 << 30, 8 << 30):
            if n > n_big:
                continue
            x, y = big[:n], dst[:n]
            g, clk = point(lambda: A.aes_ctr_xcrypt(ks, iv, x, y), n, target_s=0.25)
            out["ctr_sweep"].append({"bits": bits, "size_mib": n >> 20, "gbps": g, "clocks": clk})
    n = min(1 << 30, n_big)
    x, y = big[:n], dst[:n]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for ctas in sorted({1, sms // 4, sms // 2, sms}):
        cfg = dict(variant=1, cta_threads=0, blocks_per_thread=0, grid_ctas=ctas)
        g, clk = point(lambda: A.aes_ctr_xcrypt(ks128, iv, x, y, config=cfg), n, target_s=0.3, max_steps=50)
        out["ctas"].append(ctas)
        out["ctas_gbps"].append(g)
        out["ctas_clocks_mhz"].append(clk.get("sm_mhz"))
    return out


def sweep(torch, A):
    """The 36-run size sweep: {128,192,256} x {ECB,CTR} x {enc,dec} x {64 MiB, 1 GiB, 8 GiB}."""
    out = []
    run = 0
    for size_mib in (64, 1024, 8192):
        n = size_mib << 20
        x = synth.bytes_torch(100 + size_mib, synth.STREAM_DATA, n, device="cuda")
        y = torch.empty_like(x)
        steps = max(20, int(2 * 2**30 / n * 10))
        for bits in (128, 192, 256):
            for mode in ("ecb_enc", "ecb_dec", "ctr_enc", "ctr_dec"):
                ks = A.aes_expand_key(synth.key_bytes(run, bits))
                iv = synth.iv_bytes(run)
                m = "ctr" if mode.startswith("ctr") else mode
                fn = lambda: launch(A, m, ks, iv, x, y, None)  # noqa: E731
                ms = time_device(torch, fn, steps, 3)
                st = per_step_stats(torch, fn, min(steps, 50))
                out.append({"bits": bits, "mode": mode, "size_mib": size_mib,
                            "gbps": round(n * steps / (ms / 1e3) / 1e9, 1),
                            "median_ms": st["median_ms"], "p99_ms": st["p99_ms"],
                            "paper_mean_ms": st["paper_mean_ms"]})
                run += 1
        del x, y
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# CPU baseline / reference arm: the oracle as it stands
# ---------------------------------------------------------------------------

def _oracle_call(o, bits, mode, key, iv, data, nthreads):
    if mode == "ctr":
        return o.ctr_xcrypt(key, bits, iv, data, nthreads=nthreads)
    if mode == "ecb_enc":
        return o.ecb_encrypt(key, bits, data, nthreads=nthreads)
    return o.ecb_decrypt(key, bits, data, nthreads=nthreads)


def cpu_baseline(bits, mode, budget_s=10.0) -> dict:
    from oracle import Oracle

    o = Oracle()
    cores = os.cpu_count() or 1
    key = synth.key_bytes(0, bits)
    iv = synth.iv_bytes(0)
    cal = synth.bytes_np(0, synth.STREAM_DATA, 1 << 20)
    t0 = time.perf_counter()
    _oracle_call(o, bits, mode, key, iv, cal, cores)
    rate = (1 << 20) / max(time.perf_counter() - t0, 1e-6)
    nbytes = int(max(1 << 20, min(1 << 30, rate * budget_s)) // (1 << 20)) << 20
    data = synth.bytes_np(1, synth.STREAM_DATA, nbytes)
    t0 = time.perf_counter()
    _oracle_call(o, bits, mode, key, iv, data, cores)
    dt = time.perf_counter() - t0
    single = synth.bytes_np(2, synth.STREAM_DATA, 1 << 20)
    t1 = time.perf_counter()
    _oracle_call(o, bits, mode, key, iv, single, 0)
    dt1 = time.perf_counter() - t1
    return {"value": round(nbytes / dt / 1e9, 5), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"AES-{bits} {mode} of {nbytes >> 20} MiB, pthreads over {cores} threads "
                      "(the paper's contiguous chunk split)",
            "single_thread_gbps": round((1 << 20) / dt1 / 1e9, 5)}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import Oracle

    o = Oracle()
    cores = os.cpu_count() or 1
    bits, mode = args.bits, args.mode
    key = synth.key_bytes(0, bits)
    iv = synth.iv_bytes(0)
    cal = synth.bytes_np(0, synth.STREAM_DATA, 1 << 20)
    t0 = time.perf_counter()
    _oracle_call(o, bits, mode, key, iv, cal, cores)
    rate = (1 << 20) / max(time.perf_counter() - t0, 1e-6)
    total_budget = 120.0  # seconds for warmup + steps
    per_step = max(1 << 16, int(rate * total_budget / max(1, args.steps + args.warmup)) // 16 * 16)
    per_step = min(per_step, 1 << 30)
    data = synth.bytes_np(1, synth.STREAM_DATA, per_step)
    for _ in range(args.warmup):
        _oracle_call(o, bits, mode, key, iv, data, cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_call(o, bits, mode, key, iv, data, cores)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic: SplitMix64-seeded uniform random bytes",
        "config": {"workload": f"AES-{bits} {mode.upper()} of one {args.size_mib} MiB buffer per GPU, "
                               "device-resident (single-buffer sweep 64 MiB / 1 GiB / 8 GiB; "
                               + ("its largest buffer)" if args.size_mib == 8192 else "not its largest buffer)"),
                   "key_bits": bits, "mode": mode, "buffer_bytes": args.size_mib << 20},
        "cpu_baseline": {"value": round(value, 5), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} bytes per step of the same workload, pthreads over {cores} threads"},
        "e2e": {"value": round(value, 5), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
