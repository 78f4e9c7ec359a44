"""The generated S-box circuits (bitsliced variant) against the oracle, on CPU.

gen_bitslice.py derives SubBytes / InvSubBytes as Boolean circuits from
inversion in a tower field and checks them itself; here the committed header
is compiled for the host with g++ and evaluated on all 256 inputs (eight
words of 32 lanes), then compared with the oracle's tables, and the header
is checked to be exactly what the generator writes.
"""
import os
import shutil
import subprocess
import sys
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1403_7295_gb300", "csrc")

HARNESS = r"""
#include <cstdint>
#include <cstdio>
#include "aes_bitslice_circuit.cuh"
int main() {
  for (int inv = 0; inv < 2; ++inv) {
    for (int base = 0; base < 256; base += 32) {
      uint32_t x[8] = {0};
      for (int k = 0; k < 32; ++k)
        for (int b = 0; b < 8; ++b) x[b] |= (uint32_t)(((base + k) >> b) & 1) << k;
      if (inv) aesgpu::bs_inv_sbox(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
      else aesgpu::bs_sbox(x[0], x[1], x[2], x[3], x[4], x[5], x[6], x[7]);
      for (int k = 0; k < 32; ++k) {
        int y = 0;
        for (int b = 0; b < 8; ++b) y |= (int)((x[b] >> k) & 1) << b;
        std::printf("%d\n", y);
      }
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def circuit_tables():
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "h.cpp")
        exe = os.path.join(d, "h")
        open(src, "w").write(HARNESS)
        subprocess.run(["g++", "-std=c++17", "-O1", f"-I{CSRC}", src, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()]
    return np.array(vals[:256], np.uint8), np.array(vals[256:], np.uint8)


def test_sbox_circuit_equals_oracle(circuit_tables, oracle):
    sbox, inv = circuit_tables
    assert np.array_equal(sbox, oracle.sbox())
    assert np.array_equal(inv, oracle.inv_sbox())


def test_committed_header_matches_generator():
    with tempfile.TemporaryDirectory() as d:
        shutil.copy(os.path.join(CSRC, "gen_bitslice.py"), d)
        subprocess.run([sys.executable, os.path.join(d, "gen_bitslice.py")], check=True, capture_output=True)
        fresh = open(os.path.join(d, "aes_bitslice_circuit.cuh")).read()
    assert fresh == open(os.path.join(CSRC, "aes_bitslice_circuit.cuh")).read()
