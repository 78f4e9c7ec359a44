"""Host logic of the serving engine (no GPU): its ring arena
(paper_1403_7295_gb300/csrc/aes_ring.h) never hands out overlapping or
out-of-range bytes, accounts every byte, frees out of order and refuses what
does not fit.  The checks are a C++ program (tests/ring_test.cpp) compiled
against the engine's own header and run here."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_ring_arena_random_sequences_and_limits(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "ring_test"
    subprocess.run([cxx, "-O1", "-std=c++17", f"-I{ROOT}/paper_1403_7295_gb300/csrc",
                    os.path.join(ROOT, "tests", "ring_test.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "ring ok" in r.stdout, r.stdout + r.stderr
