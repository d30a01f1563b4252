// Double-gyre advection instantiations (2D).
#include "advect_inst.cuh"

namespace ftle {
int launch_advect_dg(int prec, int out, bool coord64, const AdvArgs& args, int grid, int block,
                     size_t smem, cudaStream_t stream) {
  return launch_advect_kind<FTLE_FLOW_DOUBLE_GYRE, 2>(prec, out, coord64, args, grid, block, smem, stream);
}
}  // namespace ftle
