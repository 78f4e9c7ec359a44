// aes_ttable_ctr.cu — instantiates the T-table kernels for Op::kCtr, and the
// TMA-staged CTR variant with its device counter of given-up waits.
#include "aes_ttable_launch.cuh"

namespace aesgpu {
namespace {
// Bounded mbarrier waits of the TMA-staged kernel that gave up (each warp
// that gives up adds one); read and cleared by take_bulk_timeouts().
__device__ unsigned int g_bulk_timeouts = 0;
}  // namespace

cudaError_t launch_ttable_ctr(int nr, const void* in, void* out, uint64_t nblocks, uint32_t tail,
                            const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                            cudaStream_t stream) {
  return dispatch_nr<Op::kCtr>(nr, in, out, nblocks, tail, rk, cp, shape, stream);
}

cudaError_t launch_ttable_ctr_bulk(int nr, const void* in, void* out, uint64_t nblocks, uint32_t tail,
                                   const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                                   cudaStream_t stream) {
  unsigned int* counter = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&counter), g_bulk_timeouts);
  if (e != cudaSuccess) return e;
  switch (nr) {
    case 10: return launch_ctr_bulk<10>(in, out, nblocks, tail, rk, cp, shape, counter, stream);
    case 12: return launch_ctr_bulk<12>(in, out, nblocks, tail, rk, cp, shape, counter, stream);
    case 14: return launch_ctr_bulk<14>(in, out, nblocks, tail, rk, cp, shape, counter, stream);
    default: return cudaErrorInvalidValue;
  }
}

// The given-up waits counted on the current device so far, reset to 0.
// Synchronises with the device (a symbol copy).
cudaError_t take_bulk_timeouts(unsigned int* out) {
  unsigned int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_bulk_timeouts, sizeof(v));
  if (e != cudaSuccess) return e;
  if (v != 0) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(g_bulk_timeouts, &zero, sizeof(zero));
    if (e != cudaSuccess) return e;
  }
  *out = v;
  return cudaSuccess;
}

}  // namespace aesgpu
