// Entry points whose kernels are not in this build yet: they validate nothing and report
// FTLE_EUNSUPPORTED, so every symbol of ftle.h is exported.
#include "capi_internal.cuh"

using namespace ftle;

extern "C" {

size_t ftle_batch_workspace_bytes(int32_t, const ftle_mesh*, int32_t) { return 0; }

int ftle_batch(int32_t, const ftle_mesh*, const ftle_flow*, const double*, double, int32_t, void* const*,
               void*, size_t, const ftle_options*, void*) {
  return fail(FTLE_EUNSUPPORTED, "ftle_batch is not available in this build");
}

int ftle_batch_plan_create(int32_t, const ftle_mesh*, const ftle_flow*, const double*, double, int32_t,
                           void* const*, void*, size_t, const ftle_options*, void*, ftle_batch_plan** plan) {
  if (plan) *plan = nullptr;
  return fail(FTLE_EUNSUPPORTED, "ftle_batch_plan_create is not available in this build");
}

int ftle_batch_plan_launch(ftle_batch_plan*, void*) {
  return fail(FTLE_EUNSUPPORTED, "ftle_batch_plan_launch is not available in this build");
}

int ftle_batch_plan_destroy(ftle_batch_plan*) { return FTLE_OK; }

size_t ftle_backward_workspace_bytes(int64_t, int32_t) { return 0; }

int ftle_backward(const ftle_mesh*, const ftle_flow*, double, double, double, int32_t, const void*,
                  const void*, int32_t, const float*, double*, void*, size_t, const ftle_options*, void*) {
  return fail(FTLE_EUNSUPPORTED, "ftle_backward is not available in this build");
}

}  // extern "C"
