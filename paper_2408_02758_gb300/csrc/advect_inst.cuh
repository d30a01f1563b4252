// Instantiation helper for the advection kernels of one flow kind.
#pragma once
#include "advect.cuh"

namespace ftle {

template <int KIND, int DIM, typename CT>
int launch_advect_typed(int prec, int out, const AdvArgs& args, int grid, int block, size_t smem,
                        cudaStream_t stream) {
  if (prec == P64 && out == O64) {
    k_advect<KIND, DIM, P64, O64, CT><<<grid, block, smem, stream>>>(args);
  } else if (prec == P32 && out == O32) {
    k_advect<KIND, DIM, P32, O32, CT><<<grid, block, smem, stream>>>(args);
  } else if (prec == P32C && out == O32PAIR) {
    constexpr bool kAbc = KIND == FTLE_FLOW_ABC;
    if (kAbc && args.rot_safe && args.abc_refresh > 1)
      k_advect<KIND, DIM, P32C, O32PAIR, CT, kAbc, kAbc><<<grid, block, smem, stream>>>(args);
    else if (kAbc && args.rot_safe)
      k_advect<KIND, DIM, P32C, O32PAIR, CT, kAbc><<<grid, block, smem, stream>>>(args);
    else
      k_advect<KIND, DIM, P32C, O32PAIR, CT><<<grid, block, smem, stream>>>(args);
  } else if (prec == P64 && out == O32PAIR) {
    k_advect<KIND, DIM, P64, O32PAIR, CT><<<grid, block, smem, stream>>>(args);
  } else {
    return fail(FTLE_EUNSUPPORTED, "advection: unsupported precision/output pair %d/%d", prec, out);
  }
  FTLE_LAUNCH_CHECK("k_advect launch");
  return FTLE_OK;
}

template <int KIND, int DIM>
int launch_advect_kind(int prec, int out, bool coord64, const AdvArgs& args, int grid, int block,
                       size_t smem, cudaStream_t stream) {
  return coord64 ? launch_advect_typed<KIND, DIM, double>(prec, out, args, grid, block, smem, stream)
                 : launch_advect_typed<KIND, DIM, float>(prec, out, args, grid, block, smem, stream);
}

int launch_advect_dg(int prec, int out, bool coord64, const AdvArgs& args, int grid, int block,
                     size_t smem, cudaStream_t stream);
int launch_advect_abc(int prec, int out, bool coord64, const AdvArgs& args, int grid, int block,
                      size_t smem, cudaStream_t stream);
int launch_advect_misc(int kind, int dim, int prec, int out, bool coord64, const AdvArgs& args,
                       int grid, int block, size_t smem, cudaStream_t stream);

}  // namespace ftle
