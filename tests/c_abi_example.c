/* A C caller of libaesgpu.so: only include/aesgpu.h and the CUDA runtime.
 * Encrypts a buffer with AES-256 CTR and AES-128 ECB on the GPU and compares
 * the bytes with the CPU oracle (test infrastructure, linked in for the check).
 * Exit status 0 = every byte equal. */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "aes_ref.h"
#include "aesgpu.h"

#define CHECK(x) do { if (!(x)) { fprintf(stderr, "check failed: %s (line %d)\n", #x, __LINE__); return 1; } } while (0)

int main(void) {
  const size_t n = (1u << 22) + 7; /* 4 MiB + a ragged tail */
  uint8_t *h_in = malloc(n), *h_out = malloc(n), *h_ref = malloc(n);
  uint8_t key[32], iv[16];
  for (size_t i = 0; i < n; ++i) h_in[i] = (uint8_t)(i * 2654435761u >> 13);
  for (int i = 0; i < 32; ++i) key[i] = (uint8_t)(7 * i + 3);
  for (int i = 0; i < 16; ++i) iv[i] = (uint8_t)(0xA0 + i);
  iv[12] = iv[13] = iv[14] = 0xFF; /* the counter wraps inside the buffer */

  aes_key_schedule ks;
  CHECK(aes_expand_key(key, 256, &ks) == AES_OK);
  void *d_in = NULL, *d_out = NULL;
  CHECK(cudaMalloc(&d_in, n) == cudaSuccess && cudaMalloc(&d_out, n) == cudaSuccess);
  CHECK(cudaMemcpy(d_in, h_in, n, cudaMemcpyHostToDevice) == cudaSuccess);
  cudaStream_t s;
  CHECK(cudaStreamCreate(&s) == cudaSuccess);

  CHECK(aes_ctr_xcrypt(&ks, iv, d_in, d_out, n, s) == AES_OK);
  CHECK(cudaStreamSynchronize(s) == cudaSuccess);
  CHECK(cudaMemcpy(h_out, d_out, n, cudaMemcpyDeviceToHost) == cudaSuccess);
  CHECK(ref_ctr_xcrypt(key, 256, iv, 0, h_in, h_ref, n) == REF_OK);
  CHECK(memcmp(h_out, h_ref, n) == 0);

  aes_key_schedule k128;
  CHECK(aes_expand_key(key, 128, &k128) == AES_OK);
  const size_t m = n - n % 16;
  CHECK(aes_ecb_encrypt(&k128, d_in, d_out, m, s) == AES_OK);
  CHECK(aes_ecb_decrypt(&k128, d_out, d_out, m, s) == AES_OK); /* in place */
  CHECK(cudaStreamSynchronize(s) == cudaSuccess);
  CHECK(cudaMemcpy(h_out, d_out, m, cudaMemcpyDeviceToHost) == cudaSuccess);
  CHECK(memcmp(h_out, h_in, m) == 0);
  CHECK(aes_ecb_encrypt(&k128, d_in, d_out, m + 1, s) == AES_ERR_LENGTH);
  CHECK(aes_ctr_xcrypt(&ks, iv, h_in, d_out, 64, s) == AES_ERR_ARG); /* pageable host memory */
  printf("c abi ok: %s\n", aes_status_string(AES_OK));
  cudaFree(d_in);
  cudaFree(d_out);
  cudaStreamDestroy(s);
  free(h_in);
  free(h_out);
  free(h_ref);
  return 0;
}
