// aes_ttable_enc.cu — instantiates the T-table kernels for Op::kEcbEncrypt.
#include "aes_ttable_launch.cuh"

namespace aesgpu {

cudaError_t launch_ttable_enc(int nr, const void* in, void* out, uint64_t nblocks, uint32_t tail,
                            const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                            cudaStream_t stream) {
  return dispatch_nr<Op::kEcbEncrypt>(nr, in, out, nblocks, tail, rk, cp, shape, stream);
}

}  // namespace aesgpu
