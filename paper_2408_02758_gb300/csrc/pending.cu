// Entry points whose kernels are not in this build yet: they validate nothing and report
// FTLE_EUNSUPPORTED, so every symbol of ftle.h is exported.
#include "capi_internal.cuh"

using namespace ftle;

extern "C" {

size_t ftle_backward_workspace_bytes(int64_t, int32_t) { return 0; }

int ftle_backward(const ftle_mesh*, const ftle_flow*, double, double, double, int32_t, const void*,
                  const void*, int32_t, const float*, double*, void*, size_t, const ftle_options*, void*) {
  return fail(FTLE_EUNSUPPORTED, "ftle_backward is not available in this build");
}

}  // extern "C"
