"""The boundary used from C (no Python, no torch): tests/c_abi_example.c
links libaesgpu.so through include/aesgpu.h and the CUDA runtime only.

CPU: the program compiles and links against the header and the library.
GPU: it runs and every byte equals the oracle's (linked into the program as
the checker)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EXE = os.path.join(ROOT, "tests", "_build", "c_abi_example")


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def build_example() -> str:
    from paper_1403_7295_gb300 import build as B

    lib = B.build()
    cuda = _cuda_home()
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    cmd = ["gcc", "-std=c99", "-O1", "-D_POSIX_C_SOURCE=200809L", f"-I{ROOT}/include", f"-I{ROOT}/oracle",
           f"-I{cuda}/include", os.path.join(ROOT, "tests", "c_abi_example.c"), os.path.join(ROOT, "oracle", "aes_ref.c"),
           "-o", EXE, f"-L{os.path.dirname(lib)}", "-laesgpu", f"-L{cuda}/lib64", f"-L{cuda}/targets/sbsa-linux/lib",
           "-lcudart", "-pthread", f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath,{cuda}/lib64"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return EXE


def test_c_program_builds_against_the_header():
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    assert os.path.exists(build_example())


@pytest.mark.gpu
def test_c_program_runs_and_matches_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = build_example()
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "c abi ok" in r.stdout, r.stdout + r.stderr
