// Neighbour lists on the GPU from element connectivity: the node adjacency of a triangle or
// tetrahedral mesh (two nodes are neighbours when an element contains both), as the sorted,
// symmetric CSR rows the FTLE kernels read.  The paper computes the neighbour list on the host
// and names accelerating it as future work (Section 2.2, Conclusions); this moves that
// preparation step onto the device for meshes that arrive without adjacency.
//
// 1. every element appends its ordered vertex pairs (a, b), a != b, to a bounded slot list of
//    node a (raw entries, duplicates included; a full list sets an overflow flag, never writes
//    past its slots; an out-of-range vertex is counted and its element skipped);
// 2. each row is sorted (insertion sort) and deduplicated in place;
// 3. an exclusive scan of the row lengths gives row_ptr; 4. the rows are compacted into col_idx.
#include <stdint.h>
#include <string.h>

#include "capi_internal.cuh"

namespace ftle {
namespace {

constexpr int kScanBlock = 1024;

struct CsrBuildFlags {
  unsigned int overflow;
  unsigned int bad_vertex;
  unsigned long long nnz;
};

__global__ void k_elem_pairs(int64_t n_elem, int v, const int32_t* __restrict__ elems, int64_t n_nodes, int cap,
                             int32_t* __restrict__ slots, int32_t* __restrict__ raw, CsrBuildFlags* flags) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t vert[4];
    bool ok = true;
    for (int q = 0; q < v; ++q) {
      vert[q] = elems[e * v + q];
      if (vert[q] < 0 || vert[q] >= n_nodes) ok = false;
    }
    if (!ok) {
      atomicAdd(&flags->bad_vertex, 1u);
      continue;
    }
    for (int p = 0; p < v; ++p)
      for (int q = 0; q < v; ++q) {
        if (p == q || vert[p] == vert[q]) continue;
        const int s = atomicAdd(raw + vert[p], 1);
        if (s < cap)
          slots[(int64_t)vert[p] * cap + s] = vert[q];
        else
          atomicOr(&flags->overflow, 1u);
      }
  }
}

// Sort and deduplicate each node's slots in place; the unique count replaces the raw count.
__global__ void k_row_unique(int64_t n_nodes, int cap, int32_t* __restrict__ slots, int32_t* __restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t* row = slots + i * cap;
    const int k = min(cnt[i], cap);
    for (int a = 1; a < k; ++a) {
      const int32_t x = row[a];
      int b = a - 1;
      while (b >= 0 && row[b] > x) {
        row[b + 1] = row[b];
        --b;
      }
      row[b + 1] = x;
    }
    int u = 0;
    for (int a = 0; a < k; ++a)
      if (u == 0 || row[a] != row[u - 1]) row[u++] = row[a];
    cnt[i] = u;
  }
}

// Exclusive scan of cnt[0..n) into out[0..n], out[n] = total: per-block scans, a scan of the
// block totals by one block, then the block offsets added.
__global__ void k_scan_blocks(int64_t n, const int32_t* __restrict__ cnt, int32_t* __restrict__ out,
                              int64_t* __restrict__ block_sum) {
  __shared__ int64_t s[kScanBlock];
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  s[threadIdx.x] = i < n ? cnt[i] : 0;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    const int64_t t = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = (int32_t)(s[threadIdx.x] - (i < n ? cnt[i] : 0));  // exclusive within the block
  if (threadIdx.x == kScanBlock - 1) block_sum[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_sums(int64_t nb, int64_t* __restrict__ block_sum, CsrBuildFlags* flags) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
      const int64_t t = block_sum[b];
      block_sum[b] = run;
      run += t;
    }
    flags->nnz = (unsigned long long)run;
  }
}

__global__ void k_scan_add(int64_t n, int32_t* __restrict__ out, const int64_t* __restrict__ block_sum,
                           const CsrBuildFlags* flags) {
  const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] = (int32_t)(out[i] + block_sum[blockIdx.x]);
  if (i == n) out[n] = (int32_t)flags->nnz;
}

__global__ void k_compact(int64_t n_nodes, int cap, const int32_t* __restrict__ slots, const int32_t* __restrict__ cnt,
                          const int32_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx, int64_t nnz_cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t base = row_ptr[i];
    for (int a = 0; a < cnt[i]; ++a)
      if (base + a >= 0 && base + a < nnz_cap) col_idx[base + a] = slots[i * cap + a];
  }
}

struct CsrLayout {
  size_t flags = 0, raw = 0, slots = 0, block_sum = 0, total = 0;
  int64_t nb = 0;
};

CsrLayout csr_layout(int64_t n_nodes, int cap) {
  CsrLayout L;
  size_t off = 0;
  L.flags = off;
  off += align256(sizeof(CsrBuildFlags));
  L.raw = off;
  off += align256(sizeof(int32_t) * (size_t)(n_nodes > 0 ? n_nodes : 1));
  L.slots = off;
  off += align256(sizeof(int32_t) * (size_t)(n_nodes > 0 ? n_nodes : 1) * (size_t)cap);
  L.nb = (n_nodes + 1 + kScanBlock - 1) / kScanBlock;
  L.block_sum = off;
  off += align256(sizeof(int64_t) * (size_t)(L.nb > 0 ? L.nb : 1));
  L.total = off;
  return L;
}

}  // namespace
}  // namespace ftle

using namespace ftle;

extern "C" {

size_t ftle_csr_workspace_bytes(int64_t n_nodes, int32_t max_row) {
  if (n_nodes < 0 || max_row < 1) return 0;
  return csr_layout(n_nodes, max_row).total;
}

int ftle_csr_from_elements(int64_t n_nodes, int64_t n_elem, int32_t verts_per_elem, const int32_t* elems,
                           int32_t max_row, int32_t* row_ptr, int32_t* col_idx, int64_t nnz_cap, int64_t* nnz_out,
                           void* workspace, size_t workspace_bytes, void* stream) {
  int rc;
  if (n_nodes < 0 || n_nodes >= (int64_t)INT32_MAX || n_elem < 0)
    return fail(FTLE_ERANGE, "n_nodes must be in [0, 2^31 - 1) and n_elem >= 0");
  if (verts_per_elem < 2 || verts_per_elem > 4) return fail(FTLE_EINVAL, "verts_per_elem must be 2, 3 or 4");
  if (max_row < 1 || max_row > 4096) return fail(FTLE_EINVAL, "max_row must be in [1, 4096]");
  if (!row_ptr || !nnz_out || (n_elem > 0 && !elems) || (nnz_cap > 0 && !col_idx))
    return fail(FTLE_EINVAL, "NULL pointer argument");
  const CsrLayout L = csr_layout(n_nodes, max_row);
  if ((rc = check_workspace(workspace, workspace_bytes, L.total))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = reinterpret_cast<char*>(workspace);
  CsrBuildFlags* flags = reinterpret_cast<CsrBuildFlags*>(w + L.flags);
  int32_t* raw = reinterpret_cast<int32_t*>(w + L.raw);
  int32_t* slots = reinterpret_cast<int32_t*>(w + L.slots);
  int64_t* bsum = reinterpret_cast<int64_t*>(w + L.block_sum);
  FTLE_CUDA_CHECK(cudaMemsetAsync(flags, 0, sizeof(CsrBuildFlags), s));
  FTLE_CUDA_CHECK(cudaMemsetAsync(raw, 0, sizeof(int32_t) * (size_t)(n_nodes > 0 ? n_nodes : 1), s));
  const int grid = grid_for(n_elem > n_nodes ? n_elem : n_nodes, 256, 8);
  if (n_elem > 0) {
    k_elem_pairs<<<grid, 256, 0, s>>>(n_elem, verts_per_elem, elems, n_nodes, max_row, slots, raw, flags);
    FTLE_LAUNCH_CHECK("k_elem_pairs launch");
  }
  if (n_nodes > 0) {
    k_row_unique<<<grid, 256, 0, s>>>(n_nodes, max_row, slots, raw);
    FTLE_LAUNCH_CHECK("k_row_unique launch");
  }
  k_scan_blocks<<<(unsigned)L.nb, kScanBlock, 0, s>>>(n_nodes, raw, row_ptr, bsum);
  FTLE_LAUNCH_CHECK("k_scan_blocks launch");
  k_scan_sums<<<1, 32, 0, s>>>(L.nb, bsum, flags);
  FTLE_LAUNCH_CHECK("k_scan_sums launch");
  k_scan_add<<<(unsigned)L.nb, kScanBlock, 0, s>>>(n_nodes, row_ptr, bsum, flags);
  FTLE_LAUNCH_CHECK("k_scan_add launch");
  if (n_nodes > 0) {
    k_compact<<<grid, 256, 0, s>>>(n_nodes, max_row, slots, raw, row_ptr, col_idx, nnz_cap);
    FTLE_LAUNCH_CHECK("k_compact launch");
  }
  CsrBuildFlags h;
  FTLE_CUDA_CHECK(cudaMemcpyAsync(&h, flags, sizeof h, cudaMemcpyDeviceToHost, s));
  FTLE_CUDA_CHECK(cudaStreamSynchronize(s));
  *nnz_out = (int64_t)h.nnz;
  if (h.bad_vertex) return fail(FTLE_EINVAL, "%u elements reference a vertex outside [0, n_nodes)", h.bad_vertex);
  if (h.overflow) return fail(FTLE_ERANGE, "a node has more than max_row = %d element pair entries", max_row);
  if (h.nnz > (unsigned long long)INT32_MAX) return fail(FTLE_ERANGE, "nnz %llu beyond int32", h.nnz);
  if ((int64_t)h.nnz > nnz_cap) return fail(FTLE_ERANGE, "nnz %llu exceeds col_idx capacity %lld", h.nnz, (long long)nnz_cap);
  return FTLE_OK;
}

}  // extern "C"
