// aes_ttable_launch.cuh — host-side launch helpers of the T-table kernels:
// shape checks, the one-time shared-memory opt-in per device, dispatch over
// (operation, rounds, blocks per thread).
#pragma once
#include "aes_smem_attr.h"
#include "aes_ttable.cuh"

namespace aesgpu {
namespace {

// The grid of the run-cached CTR kernels and their run split (CtrParams).
inline uint64_t ctr_cached_grid(uint64_t nblocks, uint32_t tail, const LaunchShape& shape, CtrParams* p) {
  // one warp per run of 256 blocks, or per piece of a run when the runs do
  // not fill the grid's warps: no more CTAs than those work units need
  const uint64_t runs = (nblocks + (tail ? 1 : 0) + (p->ctr0 & 255u) + 255) / 256;
  const uint64_t warps_per_cta = shape.cta_threads / 32;
  uint64_t grid = shape.grid_ctas;
  const uint64_t max_warps = grid * warps_per_cta;
  const uint64_t work = runs >= max_warps ? max_warps : runs * ctr_tail_pieces(runs, max_warps);
  const uint64_t needed = (work + warps_per_cta - 1) / warps_per_cta;
  if (grid > needed) grid = needed > 0 ? needed : 1;
  const uint64_t warps = grid * warps_per_cta;
  const uint32_t pieces = ctr_tail_pieces(runs % warps, warps);
  // a last wave left unsplit runs through the (unrolled) loop of the whole waves
  p->whole_runs = pieces == 1 ? runs : runs - runs % warps;
  p->tail_shift = pieces == 8 ? 3 : pieces == 4 ? 2 : pieces == 2 ? 1 : 0;
  return grid;
}

template <int NR>
cudaError_t launch_ctr_cached(const void* in, void* out, uint64_t nblocks, uint32_t tail,
                              const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                              cudaStream_t stream) {
  auto kern = ttable_ctr_cached_kernel<NR>;
  cudaError_t e = ensure_dynamic_smem(kern, kTtableSmemEnc);
  if (e != cudaSuccess) return e;
  CtrParams p = cp;
  const uint64_t grid = ctr_cached_grid(nblocks, tail, shape, &p);
  return launch_pdl(kern, static_cast<unsigned>(grid), shape.cta_threads, kTtableSmemEnc, stream,
                    static_cast<const uint4*>(in), static_cast<uint4*>(out), nblocks, tail, rk, p);
}

// The TMA-staged variant (timeouts: the device counter of given-up waits).
template <int NR>
cudaError_t launch_ctr_bulk(const void* in, void* out, uint64_t nblocks, uint32_t tail, const RoundKeys& rk,
                            const CtrParams& cp, const LaunchShape& shape, unsigned int* timeouts,
                            cudaStream_t stream) {
  auto kern = ttable_ctr_bulk_kernel<NR>;
  const int smem = bulk_smem_bytes(shape.cta_threads / 32);
  // opt in once to the largest size any CTA shape needs (the opt-in is cached per kernel)
  cudaError_t e = ensure_dynamic_smem(kern, bulk_smem_bytes(32));
  if (e != cudaSuccess) return e;
  CtrParams p = cp;
  const uint64_t grid = ctr_cached_grid(nblocks, tail, shape, &p);
  return launch_pdl(kern, static_cast<unsigned>(grid), shape.cta_threads, smem, stream,
                    static_cast<const uint4*>(in), static_cast<uint4*>(out), nblocks, tail, rk, p, timeouts);
}

template <Op OP, int NR, int BPT>
cudaError_t launch_one(const void* in, void* out, uint64_t nblocks, uint32_t tail,
                       const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                       cudaStream_t stream) {
  auto kern = ttable_kernel<OP, NR, BPT>;
  const int smem = OP == Op::kEcbDecrypt ? kTtableSmemDec : kTtableSmemEnc;
  cudaError_t e = ensure_dynamic_smem(kern, smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, shape.grid_ctas, shape.cta_threads, smem, stream, static_cast<const uint4*>(in),
                    static_cast<uint4*>(out), nblocks, tail, rk, cp);
}

template <Op OP, int NR>
cudaError_t dispatch_bpt(const void* in, void* out, uint64_t nblocks, uint32_t tail,
                         const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                         cudaStream_t stream) {
  if constexpr (OP == Op::kCtr) {
    if (shape.blocks_per_thread == 0)  // the run-cached CTR kernel
      return launch_ctr_cached<NR>(in, out, nblocks, tail, rk, cp, shape, stream);
  }
  switch (shape.blocks_per_thread) {
    case 1: return launch_one<OP, NR, 1>(in, out, nblocks, tail, rk, cp, shape, stream);
    case 2: return launch_one<OP, NR, 2>(in, out, nblocks, tail, rk, cp, shape, stream);
    case 4: return launch_one<OP, NR, 4>(in, out, nblocks, tail, rk, cp, shape, stream);
    default: return cudaErrorInvalidValue;
  }
}

template <Op OP>
inline cudaError_t dispatch_nr(int nr, const void* in, void* out, uint64_t nblocks, uint32_t tail,
                        const RoundKeys& rk, const CtrParams& cp, const LaunchShape& shape,
                        cudaStream_t stream) {
  switch (nr) {
    case 10: return dispatch_bpt<OP, 10>(in, out, nblocks, tail, rk, cp, shape, stream);
    case 12: return dispatch_bpt<OP, 12>(in, out, nblocks, tail, rk, cp, shape, stream);
    case 14: return dispatch_bpt<OP, 14>(in, out, nblocks, tail, rk, cp, shape, stream);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace aesgpu
