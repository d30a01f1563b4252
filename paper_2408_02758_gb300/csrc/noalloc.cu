// ftle_gradient_eig_noalloc: the FTLE core with its scratch in a file-scope device array, for
// callers that may not allocate device memory (see include/ftle.h).  The paper has no
// counterpart; the kernels are the ones ftle_gradient_eig launches.
#include <mutex>

#include "capi_internal.cuh"

namespace ftle {
namespace {

// Scratch: ftle_counters header (256 B) followed by the FP64-path node list, int32 per node.
// Laid out exactly as the head of a ftle_workspace_bytes workspace (header, then flag list), so
// the same kernels run on it; the refinement's mark list and bitmap are not needed here.
constexpr size_t kNoallocBytes = 256 + sizeof(int32_t) * (size_t)FTLE_NOALLOC_MAX_NODES;
static_assert(sizeof(ftle_counters) <= 256, "counters must fit the header");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the array's name is
// only a host-side stand-in, never a device address.  Outside stream capture the address is looked
// up afresh on every call (cheap), so a module reloaded after cudaDeviceReset is never reached
// through a stale pointer; while `s` is capturing, the address from the last call on this device
// outside capture is used (a first call made inside a capture is refused).
int scratch_address(cudaStream_t s, void** out) {
  int dev = -1;
  FTLE_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(FTLE_ERANGE, "device ordinal %d beyond %d", dev, kMaxDevices);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t qe = cudaStreamIsCapturing(s, &cap);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (qe == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_addr[dev] = p;
  } else {
    if (qe != cudaSuccess) (void)cudaGetLastError();  // clear the refused query's error
    if (!g_scratch_addr[dev])
      return fail(FTLE_EINVAL, "ftle_gradient_eig_noalloc: the first call on device %d must come before stream "
                  "capture begins", dev);
  }
  *out = g_scratch_addr[dev];
  return FTLE_OK;
}

}  // namespace
}  // namespace ftle

using namespace ftle;

extern "C" int ftle_gradient_eig_noalloc(const ftle_mesh* mesh, const void* flowmap, int32_t precision, double T,
                                         void* ftle_out, double* lambda_out, const ftle_options* opt,
                                         void* stream) {
  int rc;
  if ((rc = check_mesh(mesh)) || (rc = check_prec(precision))) return rc;
  if (mesh->n_nodes > FTLE_NOALLOC_MAX_NODES)
    return fail(FTLE_ERANGE, "n_nodes %lld beyond the static scratch limit %d", (long long)mesh->n_nodes,
                FTLE_NOALLOC_MAX_NODES);
  if (!isfinite(T) || T == 0.0) return fail(FTLE_EINVAL, "T must be finite and non-zero");
  if (mesh->n_nodes > 0 && (!flowmap || !ftle_out)) return fail(FTLE_EINVAL, "flowmap / ftle_out is NULL");
  const Launch L = resolve_launch(opt);
  if ((rc = check_launch(L))) return rc;
  // the deferred FP64 pass belongs to an ftle_refine on a caller workspace, which cannot see the
  // flag list kept here
  if (L.defer_fp64) return fail(FTLE_EINVAL, "ftle_gradient_eig_noalloc: defer_fp64 is not supported");
  cudaStream_t s = (cudaStream_t)stream;
  void* scratch = nullptr;
  if ((rc = scratch_address(s, &scratch))) return rc;
  // the layout run_gradient expects: header at 0, flag list at the next 256-byte boundary
  if (ws_layout(mesh->n_nodes).flag_list != 256) return fail(FTLE_EINVAL, "unexpected workspace layout");
  if (L.validate_mesh && (rc = validate_mesh_sync(mesh, scratch, s, nullptr))) return rc;
  FTLE_CUDA_CHECK(cudaMemsetAsync(scratch, 0, sizeof(ftle_counters), s));
  return run_gradient(mesh, flowmap, precision, T, ftle_out, lambda_out, scratch, L, s, true);
}
