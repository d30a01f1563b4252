// Linear and saddle-flow advection instantiations (2D and 3D); their flowmaps have closed forms,
// which the tests use to pin the kernels.
#include "advect_inst.cuh"

namespace ftle {
int launch_advect_misc(int kind, int dim, int prec, int out, bool coord64, const AdvArgs& args,
                       int grid, int block, size_t smem, cudaStream_t stream) {
  if (kind == FTLE_FLOW_LINEAR && dim == 2)
    return launch_advect_kind<FTLE_FLOW_LINEAR, 2>(prec, out, coord64, args, grid, block, smem, stream);
  if (kind == FTLE_FLOW_LINEAR && dim == 3)
    return launch_advect_kind<FTLE_FLOW_LINEAR, 3>(prec, out, coord64, args, grid, block, smem, stream);
  if (kind == FTLE_FLOW_SADDLE && dim == 2)
    return launch_advect_kind<FTLE_FLOW_SADDLE, 2>(prec, out, coord64, args, grid, block, smem, stream);
  if (kind == FTLE_FLOW_SADDLE && dim == 3)
    return launch_advect_kind<FTLE_FLOW_SADDLE, 3>(prec, out, coord64, args, grid, block, smem, stream);
  return fail(FTLE_EUNSUPPORTED, "advection: flow kind %d not available in %dD", kind, dim);
}
}  // namespace ftle
