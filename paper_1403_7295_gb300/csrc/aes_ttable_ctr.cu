// aes_ttable_ctr.cu — instantiates the T-table kernels for Op::kCtr.
#include "aes_ttable_launch.cuh"

namespace aesgpu {

cudaError_t launch_ttable_ctr(int nr, const void* in, void* out, uint64_t nblocks, uint32_t tail,
                            const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                            cudaStream_t stream) {
  return dispatch_nr<Op::kCtr>(nr, in, out, nblocks, tail, rk, cp, shape, stream);
}

}  // namespace aesgpu
