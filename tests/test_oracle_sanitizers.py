"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (host).

compute-sanitizer is closed on this machine, so memory safety of the host code
is checked with the compiler's sanitizers: a C driver links aes_ref.c built
with -fsanitize=address,undefined and calls every entry point on edge
lengths (0, 1, 15, 16, 17, 4097), in place, with malformed padding, and
through the pthreads chunk split with more threads than blocks.  Any
sanitizer report fails the run.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

DRIVER = r"""
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "aes_ref.h"

static int fail(const char *what) { fprintf(stderr, "FAIL %s\n", what); return 1; }

int main(void) {
  const int bits[3] = {128, 192, 256};
  const uint64_t lens[] = {0, 1, 15, 16, 17, 31, 4097, 16 * 257};
  uint8_t key[32], iv[16];
  for (int i = 0; i < 32; ++i) key[i] = (uint8_t)(i * 37 + 1);
  for (int i = 0; i < 16; ++i) iv[i] = (uint8_t)(0xF0 + i);
  for (int b = 0; b < 3; ++b) {
    for (size_t li = 0; li < sizeof lens / sizeof lens[0]; ++li) {
      const uint64_t n = lens[li];
      uint8_t *in = malloc(n + 1), *out = malloc(n + 1), *back = malloc(n + 1);
      uint8_t *pad = malloc(n + 32), *dec = malloc(n + 32);
      for (uint64_t i = 0; i < n; ++i) in[i] = (uint8_t)(i * 131 + 7);
      if (ref_ctr_xcrypt(key, bits[b], iv, 0, in, out, n)) return fail("ctr");
      if (ref_ctr_xcrypt_mt(key, bits[b], iv, 0, out, back, n, 7)) return fail("ctr_mt");
      if (n && memcmp(in, back, n)) return fail("ctr round trip");
      memcpy(back, in, n);
      if (ref_ctr_xcrypt(key, bits[b], iv, 3, back, back, n)) return fail("ctr in place");
      if (n % 16 == 0) {
        if (ref_ecb_encrypt_mt(key, bits[b], in, out, n, 64)) return fail("ecb_mt");
        if (ref_ecb_decrypt(key, bits[b], out, out, n)) return fail("ecb in place");
        if (n && memcmp(in, out, n)) return fail("ecb round trip");
      } else if (ref_ecb_encrypt(key, bits[b], in, out, n) != REF_ERR_LENGTH) {
        return fail("ecb length");
      }
      uint64_t pl = 0, dl = 0;
      if (ref_ecb_pkcs7_encrypt(key, bits[b], in, n, pad, &pl)) return fail("pkcs7 enc");
      if (pl != ref_pkcs7_padded_len(n)) return fail("pkcs7 len");
      if (ref_ecb_pkcs7_decrypt(key, bits[b], pad, pl, dec, &dl) || dl != n) return fail("pkcs7 dec");
      pad[pl - 1] ^= 0x40;
      int rc = ref_ecb_pkcs7_decrypt(key, bits[b], pad, pl, dec, &dl);
      if (rc != REF_OK && rc != REF_ERR_PADDING) return fail("pkcs7 bad");
      uint64_t idx[3] = {0, 5, 1u << 20};
      uint8_t blk[48] = {0}, ob[48];
      if (ref_ctr_xcrypt_blocks(key, bits[b], iv, idx, blk, ob, 3)) return fail("blocks");
      free(in); free(out); free(back); free(pad); free(dec);
    }
  }
  uint8_t w[240]; int nr;
  if (ref_key_expansion(key, 100, w, &nr) != REF_ERR_KEYSIZE) return fail("keysize");
  puts("ok");
  return 0;
}
"""


def test_oracle_clean_under_asan_and_ubsan():
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    with tempfile.TemporaryDirectory() as d:
        drv = os.path.join(d, "drv.c")
        exe = os.path.join(d, "drv")
        open(drv, "w").write(DRIVER)
        cmd = ["gcc", "-std=c99", "-O1", "-g", "-fsanitize=address,undefined", "-fno-omit-frame-pointer",
               "-fno-sanitize-recover=undefined", "-pthread", "-D_POSIX_C_SOURCE=200809L", f"-I{ORACLE}",
               drv, os.path.join(ORACLE, "aes_ref.c"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 and "asan" in (r.stderr + r.stdout).lower():
            pytest.skip("sanitizer runtime unavailable: " + r.stderr[-200:])
        assert r.returncode == 0, r.stderr
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
        run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
        assert run.returncode == 0 and run.stdout.strip() == "ok", run.stdout + run.stderr
        assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr
