// aes_probe.cu — micro-benchmarks for the roofline's denominators (bench only;
// built into libaesgpu_probe.so, never linked into libaesgpu.so).
//
// Each probe keeps one CTA per SM busy with 8 independent dependency chains
// per thread of one instruction kind and reads the SM clock around the loop,
// giving thread-operations per clock per SM for:
//   LOP3, PRMT, 32-bit add, funnel shift, IMAD, conflict-free 32-bit shared
//   loads, and mixes of them (to see which pipes co-issue),
// and a streaming 128-bit copy for the achievable HBM bandwidth.
#include <cuda_runtime.h>

#include <cstdint>

#include "aesgpu_probe.h"

namespace {

enum Kind {
  kLop3 = 0,
  kPrmt = 1,
  kIadd = 2,
  kShf = 3,
  kImad = 4,
  kLds = 5,
  kLop3Imad = 6,  // one LOP3 chain step and one IMAD chain step per unit
  kLop3Lds = 7,   // one LOP3 and one LDS per unit
  kPrmtLds = 8,   // one PRMT and one LDS per unit
  kLop3Prmt = 9,  // one LOP3 and one PRMT per unit
  kNumKinds = 10
};

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t op_prmt(uint32_t a, uint32_t b, uint32_t s) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(s));
  return d;
}
__device__ __forceinline__ uint32_t op_add(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("add.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t op_shf(uint32_t a, uint32_t s) {
  uint32_t d;
  asm("shf.l.wrap.b32 %0, %1, %1, %2;" : "=r"(d) : "r"(a), "r"(s));
  return d;
}
__device__ __forceinline__ uint32_t op_imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t op_lds(uint32_t addr) {
  uint32_t d;
  asm("ld.shared.u32 %0, [%1];" : "=r"(d) : "r"(addr));
  return d;
}

template <int KIND>
__global__ void __launch_bounds__(1024, 1)
    pipe_probe(uint32_t* sink, unsigned long long* cycles, int iters) {
  extern __shared__ uint32_t sm[];  // 256 rows x 32 lanes
  const uint32_t lane = threadIdx.x & 31;
  // Row r of lane l holds the byte address of row (5r+1) mod 256 of lane l,
  // so a chase stays in the lane's bank: conflict-free by construction.
  const uint32_t smem_base = static_cast<uint32_t>(__cvta_generic_to_shared(sm));
  for (uint32_t i = threadIdx.x; i < 256 * 32; i += blockDim.x) {
    const uint32_t r = i / 32, l = i % 32;
    sm[i] = smem_base + (((5 * r + 1) & 255) * 32 + l) * 4;
  }
  __syncthreads();
  uint32_t a[kChains], p[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = threadIdx.x * 2654435761u + c;
    p[c] = smem_base + ((c * 29 + threadIdx.x / 32) % 256) * 128 + lane * 4;
  }
  const uint32_t b = blockIdx.x | 0x9E3779B9u, k = threadIdx.x ^ 0x7F4A7C15u;
  const uint32_t sel = 0x1032u, sh = 7u;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if (KIND == kLop3) a[c] = op_lop3(a[c], b, k);
        if (KIND == kPrmt) a[c] = op_prmt(a[c], b, sel);
        if (KIND == kIadd) a[c] = op_add(a[c], b);
        if (KIND == kShf) a[c] = op_shf(a[c], sh);
        if (KIND == kImad) a[c] = op_imad(a[c], b, k);
        if (KIND == kLds) p[c] = op_lds(p[c]);
        if (KIND == kLop3Imad) {
          a[c] = op_lop3(a[c], b, k);
          p[c] = op_imad(p[c], b, k);
        }
        if (KIND == kLop3Lds) {
          a[c] = op_lop3(a[c], b, k);
          p[c] = op_lds(p[c]);
        }
        if (KIND == kPrmtLds) {
          a[c] = op_prmt(a[c], b, sel);
          p[c] = op_lds(p[c]);
        }
        if (KIND == kLop3Prmt) {
          a[c] = op_lop3(a[c], b, k);
          p[c] = op_prmt(p[c], b, sel);
        }
      }
    }
  }
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= a[c] ^ p[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(t1 - t0);
}

__global__ void stream_copy(const uint4* in, uint4* out, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    __stcs(out + i, __ldcs(in + i));
}

template <int KIND>
cudaError_t launch_probe(int ctas, int threads, int iters, uint32_t* sink,
                         unsigned long long* cyc, cudaStream_t s) {
  const int smem = 256 * 32 * 4;
  pipe_probe<KIND><<<ctas, threads, smem, s>>>(sink, cyc, iters);
  return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int ctas, int threads, int iters, uint32_t* sink,
                        unsigned long long* cyc, cudaStream_t s) {
  switch (kind) {
    case kLop3: return launch_probe<kLop3>(ctas, threads, iters, sink, cyc, s);
    case kPrmt: return launch_probe<kPrmt>(ctas, threads, iters, sink, cyc, s);
    case kIadd: return launch_probe<kIadd>(ctas, threads, iters, sink, cyc, s);
    case kShf: return launch_probe<kShf>(ctas, threads, iters, sink, cyc, s);
    case kImad: return launch_probe<kImad>(ctas, threads, iters, sink, cyc, s);
    case kLds: return launch_probe<kLds>(ctas, threads, iters, sink, cyc, s);
    case kLop3Imad: return launch_probe<kLop3Imad>(ctas, threads, iters, sink, cyc, s);
    case kLop3Lds: return launch_probe<kLop3Lds>(ctas, threads, iters, sink, cyc, s);
    case kPrmtLds: return launch_probe<kPrmtLds>(ctas, threads, iters, sink, cyc, s);
    case kLop3Prmt: return launch_probe<kLop3Prmt>(ctas, threads, iters, sink, cyc, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

extern "C" {

int aesgpu_probe_num_kinds(void) { return kNumKinds; }

int aesgpu_probe_ops_per_unit(int kind) { return (kind >= kLop3Imad) ? 2 : 1; }

// Runs one pipe probe on every SM (one CTA of `threads` threads each).
// Outputs: thread-operations per clock per SM (median over CTAs of
// ops / cycles) and the wall time of the launch in seconds.
int aesgpu_probe_pipe(int kind, int threads, int iters, double* ops_per_clk_per_sm,
                      double* seconds) {
  if (kind < 0 || kind >= kNumKinds || threads < 32 || threads > 1024 || iters < 1) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  uint32_t* sink = nullptr;
  unsigned long long* cyc = nullptr;
  if (cudaMalloc(&sink, sizeof(uint32_t) * sms * threads) != cudaSuccess) return 2;
  if (cudaMalloc(&cyc, sizeof(unsigned long long) * sms) != cudaSuccess) {
    cudaFree(sink);
    return 2;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = 0;
  // warm-up launch, then the timed one
  if (launch_kind(kind, sms, threads, iters / 4 + 1, sink, cyc, 0) != cudaSuccess) rc = 3;
  cudaEventRecord(e0, 0);
  if (!rc && launch_kind(kind, sms, threads, iters, sink, cyc, 0) != cudaSuccess) rc = 3;
  cudaEventRecord(e1, 0);
  if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = 4;
  if (!rc) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long* host = new unsigned long long[sms];
    cudaMemcpy(host, cyc, sizeof(unsigned long long) * sms, cudaMemcpyDeviceToHost);
    // median cycles over SMs
    for (int i = 1; i < sms; ++i)
      for (int j = i; j > 0 && host[j - 1] > host[j]; --j) {
        unsigned long long t = host[j];
        host[j] = host[j - 1];
        host[j - 1] = t;
      }
    const double med = static_cast<double>(host[sms / 2]);
    delete[] host;
    const double ops = static_cast<double>(threads) * iters * kUnroll * kChains *
                       aesgpu_probe_ops_per_unit(kind);
    *ops_per_clk_per_sm = ops / med;
    *seconds = ms * 1e-3;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(cyc);
  return rc;
}

// Streaming 128-bit copy of nbytes (multiple of 16) between two device
// buffers, `reps` timed launches after one warm-up; returns the best
// read+write bandwidth in GB/s.
int aesgpu_probe_copy(const void* d_in, void* d_out, size_t nbytes, int ctas_per_sm, int threads,
                      int reps, double* gbps) {
  if (nbytes % 16 || reps < 1) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const uint64_t n = nbytes / 16;
  const int grid = sms * ctas_per_sm;
  stream_copy<<<grid, threads>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out), n);
  double best = 0;
  int rc = 0;
  for (int r = 0; r < reps && !rc; ++r) {
    cudaEventRecord(e0, 0);
    stream_copy<<<grid, threads>>>(static_cast<const uint4*>(d_in), static_cast<uint4*>(d_out), n);
    cudaEventRecord(e1, 0);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = 4;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    const double bw = 2.0 * nbytes / (ms * 1e-3) / 1e9;
    if (bw > best) best = bw;
  }
  *gbps = best;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // extern "C"
