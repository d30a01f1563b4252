// Mesh validation: the contract of the precomputed neighbour lists (Section 2.2 of the paper:
// the host prepares, per point, the indices of its neighbours, and the FTLE core only gathers
// through them).  Every gradient, refinement and adjoint kernel indexes coordinates and flowmaps
// by these values, so a value outside [0, n_nodes) would make them read out of bounds.  This
// pass reads the index arrays themselves and never dereferences a value it reads:
//   row_ptr: row_ptr[0] = 0, non-decreasing, row_ptr[n_nodes] = nnz;
//   col_idx: every entry in [0, n_nodes);
//   ell_idx: every entry in [-1, n_nodes) (-1 marks an absent neighbour).
#include "capi_internal.cuh"

namespace ftle {

// One grid-stride pass over the three arrays as one index space [rows | col_idx | ell_idx]; the
// counts are summed per block in shared memory and added with one atomic per block and array.
// Positions of the first bad entries are kept as unsigned minima, "none" being the largest value.
__global__ void __launch_bounds__(256) k_validate_mesh(int64_t n, int64_t nnz, const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col_idx,
                                                       const int32_t* __restrict__ ell, int64_t ell_len,
                                                       MeshCheck* out) {
  constexpr unsigned long long kNone = ~0ull;
  __shared__ unsigned long long s_cnt[3], s_first[3];
  if (threadIdx.x < 3) {
    s_cnt[threadIdx.x] = 0ull;
    s_first[threadIdx.x] = kNone;
  }
  __syncthreads();
  unsigned long long cnt[3] = {0ull, 0ull, 0ull}, first[3] = {kNone, kNone, kNone};
  const int64_t total = n + nnz + ell_len;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    int which = -1;
    unsigned long long pos = 0;
    if (t < n) {
      const int32_t a = row_ptr[t], b = row_ptr[t + 1];
      if (b < a || (t == 0 && a != 0) || (t == n - 1 && (int64_t)b != nnz)) which = 0, pos = (unsigned long long)t;
    } else if (t < n + nnz) {
      const int64_t e = t - n;
      const int32_t j = col_idx[e];
      if (j < 0 || (int64_t)j >= n) which = 1, pos = (unsigned long long)e;
    } else {
      const int64_t e = t - n - nnz;
      const int32_t j = ell[e];
      if (j < -1 || (int64_t)j >= n) which = 2, pos = (unsigned long long)e;
    }
    if (which >= 0) {
      ++cnt[which];
      if (pos < first[which]) first[which] = pos;
    }
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (cnt[q]) {
      atomicAdd(&s_cnt[q], cnt[q]);
      atomicMin(&s_first[q], first[q]);
    }
  }
  __syncthreads();
  if (threadIdx.x < 3 && s_cnt[threadIdx.x]) {
    atomicAdd(&out->count[threadIdx.x], s_cnt[threadIdx.x]);
    atomicMin(&out->first[threadIdx.x], s_first[threadIdx.x]);
  }
}

int launch_validate_mesh(const ftle_mesh* m, MeshCheck* dev_out, cudaStream_t s) {
  const int64_t n = m->n_nodes;
  FTLE_CUDA_CHECK(cudaMemsetAsync(dev_out->count, 0, sizeof dev_out->count, s));
  FTLE_CUDA_CHECK(cudaMemsetAsync(dev_out->first, 0xFF, sizeof dev_out->first, s));
  if (n == 0) return FTLE_OK;
  const int64_t ell_len = (m->ell_width > 0 && m->ell_idx) ? (int64_t)m->ell_width * n : 0;
  const int64_t total = n + m->nnz + ell_len;
  const int grid = grid_for(total, 256, 8);
  k_validate_mesh<<<grid, 256, 0, s>>>(n, m->nnz, m->row_ptr, m->col_idx, m->ell_idx, ell_len, dev_out);
  FTLE_LAUNCH_CHECK("k_validate_mesh launch");
  return FTLE_OK;
}

// Host side: reads the counters back (synchronising `s`), fills the report and turns any bad
// entry into FTLE_EINVAL with a message naming the first one.
int finish_validate_mesh(const MeshCheck* dev_out, cudaStream_t s, ftle_mesh_report* report) {
  MeshCheck h;
  FTLE_CUDA_CHECK(cudaMemcpyAsync(&h, dev_out, sizeof h, cudaMemcpyDeviceToHost, s));
  FTLE_CUDA_CHECK(cudaStreamSynchronize(s));
  ftle_mesh_report r;
  r.bad_row_ptr = (int64_t)h.count[0];
  r.bad_col_idx = (int64_t)h.count[1];
  r.bad_ell_idx = (int64_t)h.count[2];
  r.first_bad_row = h.count[0] ? (int64_t)h.first[0] : -1;
  r.first_bad_col = h.count[1] ? (int64_t)h.first[1] : -1;
  r.first_bad_ell = h.count[2] ? (int64_t)h.first[2] : -1;
  if (report) *report = r;
  if (r.bad_row_ptr)
    return fail(FTLE_EINVAL, "mesh: %lld bad row_ptr rows (first at row %lld: row_ptr[0] != 0, a decrease, or "
                "row_ptr[n_nodes] != nnz)", (long long)r.bad_row_ptr, (long long)r.first_bad_row);
  if (r.bad_col_idx)
    return fail(FTLE_EINVAL, "mesh: %lld col_idx entries outside [0, n_nodes) (first at entry %lld)",
                (long long)r.bad_col_idx, (long long)r.first_bad_col);
  if (r.bad_ell_idx)
    return fail(FTLE_EINVAL, "mesh: %lld ell_idx entries outside [-1, n_nodes) (first at entry %lld)",
                (long long)r.bad_ell_idx, (long long)r.first_bad_ell);
  return FTLE_OK;
}

int validate_mesh_sync(const ftle_mesh* m, void* ws, cudaStream_t s, ftle_mesh_report* report) {
  MeshCheck* c = mesh_check_ptr(ws);
  int rc = launch_validate_mesh(m, c, s);
  if (rc) return rc;
  return finish_validate_mesh(c, s, report);
}

}  // namespace ftle

using namespace ftle;

extern "C" int ftle_validate_mesh(const ftle_mesh* mesh, ftle_mesh_report* report, void* workspace,
                                  size_t workspace_bytes, void* stream) {
  int rc;
  if ((rc = check_mesh(mesh))) return rc;
  if ((rc = check_workspace(workspace, workspace_bytes, 256))) return rc;
  return validate_mesh_sync(mesh, workspace, (cudaStream_t)stream, report);
}
