"""In-tree build of libaesgpu.so for sm_103a (GB300).

Each ``csrc/*.cu`` compiles to an object in parallel (one ``-gencode``, no
cmake), then the objects link into ``_build/libaesgpu.so`` beside this file.
A rebuild happens only when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_NAME = "libaesgpu.so"
LIB_PATH = os.path.join(BUILD_DIR, LIB_NAME)
PROBE_LIB_PATH = os.path.join(BUILD_DIR, "libaesgpu_probe.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
              "--expt-relaxed-constexpr", f"-I{INCLUDE}", f"-I{CSRC}"]


# Per-file extra nvcc flags (none at present).  nvcc's -split-compile was
# tried on the batch kernel and dropped: its output is not deterministic
# (the same source compiled five times gave two different register
# allocations), so it cannot be measured once and relied on.
EXTRA_FLAGS: dict[str, list[str]] = {}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaesgpu.so")


def sources(subdir: str = "") -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, subdir, "*.cu")))


def _inputs(subdir: str = "") -> list[str]:
    d = os.path.join(CSRC, subdir)
    return (sources(subdir) + glob.glob(os.path.join(d, "*.cuh")) + glob.glob(os.path.join(d, "*.h"))
            + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
            + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)])


def up_to_date(lib_path: str = LIB_PATH, subdir: str = "") -> bool:
    if not os.path.exists(lib_path):
        return False
    lib_t = os.path.getmtime(lib_path)
    return all(os.path.getmtime(p) <= lib_t for p in _inputs(subdir))


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile every CUDA source for sm_103a and link libaesgpu.so and the
    bench-only libaesgpu_probe.so.  Returns the path of libaesgpu.so."""
    _build_lib(LIB_PATH, "", force, verbose, jobs)
    _build_lib(PROBE_LIB_PATH, "probe", force, verbose, jobs)
    return LIB_PATH


def _build_lib(lib_path: str, subdir: str, force: bool, verbose: bool, jobs: int | None) -> str:
    if not force and up_to_date(lib_path, subdir):
        return lib_path
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    srcs = sources(subdir)
    objs = [os.path.join(BUILD_DIR, (subdir + "_" if subdir else "") + os.path.basename(s)[:-3] + ".o")
            for s in srcs]

    def compile_one(pair):
        src, obj = pair
        cmd = [cc, *ARCH, *NVCC_FLAGS, *EXTRA_FLAGS.get(os.path.basename(src), []), "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    jobs = jobs or min(len(srcs), max(1, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose:
        for src, log in zip(srcs, logs):
            print(f"== {os.path.basename(src)}\n{log}")
    tmp = lib_path + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
