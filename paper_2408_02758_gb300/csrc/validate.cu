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

// Block shape of the pass: 16 blocks of 128 threads per SM (every warp slot), each thread keeping
// two 16-byte loads in flight.  On its own the pass reads the 3D workload's 1 GB of lists in
// 0.24 ms; the host-buffer entry point runs it on a side stream beside the advection, where it
// adds about 0.16 ms to the call (on the caller's stream after the advection: 0.33 ms; one block
// per SM beside the advection's blocks for the whole advection: 1.4 ms, taking issue slots from
// the FP32-bound advection).
constexpr int kValBlock = 128;
constexpr int kValBlocksPerSm = 16;

// Adds a block's count and first bad position (threads that found something, through shared
// memory) to the output: one atomic pair per block.
__device__ __forceinline__ void block_report(uint32_t cnt, unsigned long long first, unsigned long long* out_cnt,
                                             unsigned long long* out_first) {
  __shared__ unsigned long long s_cnt, s_first;
  if (threadIdx.x == 0) {
    s_cnt = 0ull;
    s_first = ~0ull;
  }
  __syncthreads();
  if (cnt) {
    atomicAdd(&s_cnt, (unsigned long long)cnt);
    atomicMin(&s_first, first);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_cnt) {
    atomicAdd(out_cnt, s_cnt);
    atomicMin(out_first, s_first);
  }
}

// Rows [0, n): row_ptr[0] = 0, no decrease, row_ptr[n] = nnz.
__global__ void __launch_bounds__(kValBlock, kValBlocksPerSm)
    k_validate_rows(const int32_t* __restrict__ row_ptr, int64_t n, int64_t nnz, MeshCheck* out) {
  uint32_t cnt = 0;
  unsigned long long first = ~0ull;
#pragma unroll 1
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = __ldg(row_ptr + t), b = __ldg(row_ptr + t + 1);
    if (b < a || (t == 0 && a != 0) || (t == n - 1 && (int64_t)b != nnz)) {
      ++cnt;
      if ((unsigned long long)t < first) first = (unsigned long long)t;
    }
  }
  block_report(cnt, first, &out->count[0], &out->first[0]);
}

// The entries j of p[0, len) outside the range given by (uint32)j + shift < lim: one thread every
// gridDim.x * blockDim.x int4 of the 16-byte-aligned body, the unaligned head and tail entry by
// entry.  The values are read and compared, never used.  q selects the output slot.
__global__ void __launch_bounds__(kValBlock, kValBlocksPerSm)
    k_validate_range(const int32_t* __restrict__ p, int64_t len, uint32_t shift, uint32_t lim, int q, MeshCheck* out) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  uint32_t cnt = 0;
  unsigned long long first = ~0ull;
  auto test = [&](int32_t j, int64_t pos) {
    if ((uint32_t)j + shift >= lim) {
      ++cnt;
      if ((unsigned long long)pos < first) first = (unsigned long long)pos;
    }
  };
  const int64_t head = min(len, (int64_t)(((16u - ((uint32_t)(uintptr_t)p & 15u)) & 15u) >> 2));
  if (tid < head) test(__ldg(p + tid), tid);
  const int64_t nv = (len - head) >> 2;
  const int4* v = reinterpret_cast<const int4*>(p + head);
#pragma unroll 2
  for (int64_t k = tid; k < nv; k += stride) {
    const int4 x = __ldg(v + k);
    if (((uint32_t)x.x + shift >= lim) | ((uint32_t)x.y + shift >= lim) | ((uint32_t)x.z + shift >= lim) |
        ((uint32_t)x.w + shift >= lim)) {  // rare: find which
      const int64_t b = head + 4 * k;
      test(x.x, b);
      test(x.y, b + 1);
      test(x.z, b + 2);
      test(x.w, b + 3);
    }
  }
  const int64_t t0 = head + 4 * nv;
  if (tid < len - t0) test(__ldg(p + t0 + tid), t0 + tid);
  block_report(cnt, first, &out->count[q], &out->first[q]);
}

int launch_validate_mesh(const ftle_mesh* m, MeshCheck* dev_out, cudaStream_t s) {
  PhaseRange range("ftle.validate_mesh");
  const int64_t n = m->n_nodes;
  FTLE_CUDA_CHECK(cudaMemsetAsync(dev_out->count, 0, sizeof dev_out->count, s));
  FTLE_CUDA_CHECK(cudaMemsetAsync(dev_out->first, 0xFF, sizeof dev_out->first, s));
  if (n == 0) return FTLE_OK;
  const int per_sm = kValBlocksPerSm;
  // the range tests take n capped at 2^31 (no int32 value reaches past that): col_idx in [0, n)
  // is (uint32)j < n, ell_idx in [-1, n) is (uint32)j + 1 < n + 1
  const uint32_t nlim = n < (int64_t)0x80000000LL ? (uint32_t)n : 0x80000000u;
  k_validate_rows<<<grid_for(n, kValBlock, per_sm), kValBlock, 0, s>>>(m->row_ptr, n, m->nnz, dev_out);
  FTLE_LAUNCH_CHECK("k_validate_rows launch");
  if (m->nnz > 0) {
    k_validate_range<<<grid_for((m->nnz + 3) / 4, kValBlock, per_sm), kValBlock, 0, s>>>(m->col_idx, m->nnz, 0u, nlim,
                                                                                       1, dev_out);
    FTLE_LAUNCH_CHECK("k_validate_range launch");
  }
  const int64_t ell_len = (m->ell_width > 0 && m->ell_idx) ? (int64_t)m->ell_width * n : 0;
  if (ell_len > 0) {
    k_validate_range<<<grid_for((ell_len + 3) / 4, kValBlock, per_sm), kValBlock, 0, s>>>(m->ell_idx, ell_len, 1u,
                                                                                        nlim + 1u, 2, dev_out);
    FTLE_LAUNCH_CHECK("k_validate_range launch");
  }
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
