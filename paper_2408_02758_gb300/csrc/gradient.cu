// FTLE core kernels (arXiv 2408.02758, Section 2.1 / Table 1 core; Section 2.2 neighbour lists).
//
// Float kernel, one thread per node:
//   M = sum dx dx^T, B = sum dphi dx^T over the node's CSR row (dx from the stored coordinates,
//   dphi = (hi_j - hi_i) + (lo_j - lo_i) for compensated flowmaps), F = B adj(M) / det(M),
//   C = F^T F, lambda_max in closed form (2D: the quadratic's larger root; 3D: the
//   trigonometric form of the symmetric 3x3 eigenvalues, Smith 1961), FTLE = log1p(mu)/(2|T|)
//   with mu = lambda_max - 1.
// It flags a node for the double kernel when float cannot be trusted there: fewer than d
// neighbours or det(M) <= kCondFlag (tr M/d)^d (ill-conditioned fit); mu < kMuFloor
// (lambda_max - 1 cancels); ln(lambda_max) h_i < refine_kappa with h_i the RMS neighbour
// distance (a float flowmap error e shifts F by ~e/h_i, hence the FTLE by ~e/(h_i ln sigma) in
// relative terms, so these nodes need the float-float re-advection); or in 3D the two largest
// eigenvalues nearly coincide (1 + r <= kNearDoubleTop, where the trigonometric form loses
// accuracy).  Flagged nodes are appended to a list with one atomic per warp.
//
// Double kernel: the same fit in double for every node (FTLE_PREC_FP64) or for a node list
// (the fix-up).  mu is the largest eigenvalue of E = F^T F - I formed in double, so it keeps
// its relative accuracy as lambda_max -> 1.  A neighbourhood is rank-deficient when it has
// fewer than d nodes or det(M) <= kRankTol (tr M/d)^d: FTLE = NaN and n_degenerate counts it.
#include <math.h>

#include "gradient_node.cuh"

namespace ftle {

// ----------------------------------------------------------------------------- float kernel

template <int DIM, int PL, typename CT, bool REC>
__global__ void __launch_bounds__(256) k_grad_f32(GradArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n = a.n;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool flag = false;
    if (i < n) {
      if constexpr (REC)
        flag = grad_node_f32_rec<DIM>(a, i);
      else
        flag = grad_node_f32<DIM, PL, CT>(a, i);
    }
    // warp-aggregated append of flagged nodes (the loop is uniform per block)
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long basepos = 0;
      if (lane == leader) basepos = atomicAdd(&a.hdr->n_flagged, (unsigned long long)__popc(mask));
      basepos = __shfl_sync(0xffffffffu, basepos, leader);
      if (flag) a.flag_list[basepos + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
}

// Float kernel over the fixed-width neighbour list (W = 0: width read at run time).
template <int DIM, int PL, typename CT, int W, bool REC>
__global__ void __launch_bounds__(256) k_grad_f32_ell(GradArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n = a.n;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool flag = false;
    if (i < n) {
      if constexpr (REC)
        flag = grad_node_f32_ell_rec<DIM, W>(a, i);
      else if constexpr (W > 0)
        flag = grad_node_f32_ell<DIM, PL, CT, W>(a, i);
      else
        flag = grad_node_f32_ell_any<DIM, PL, CT>(a, i);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long basepos = 0;
      if (lane == leader) basepos = atomicAdd(&a.hdr->n_flagged, (unsigned long long)__popc(mask));
      basepos = __shfl_sync(0xffffffffu, basepos, leader);
      if (flag) a.flag_list[basepos + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
}

// Float kernel over the fixed-width list with each tile's index slices staged in shared memory.
// A block takes tiles of 256 consecutive nodes (one per thread); for every tile, thread 0 issues
// W bulk copies (one per slot: the tile's contiguous slice of that slot's indices) that complete
// on the stage's "full" mbarrier, one tile ahead of the one being computed (two stages).  The
// index stream then arrives from DRAM without occupying the warps' registers or issue slots, and
// a node reads its indices from shared memory at fixed offsets; the neighbour records are
// gathered and the node computed exactly as in grad_node_f32_ell_rec (same results bit for bit).
// Every thread releases a stage on its "empty" mbarrier once its indices are in registers, and
// thread 0 refills the stage only after all 256 releases, so no block-wide barrier holds the
// warps together: a warp runs up to a tile ahead of the slowest.  Requirements (checked by the
// launcher): n_nodes a multiple of 4 and ell_idx 16-byte aligned (every slice then starts and
// ends on 16-byte boundaries), compensated flowmap records.  Every wait is bounded
// (kStageWaitPolls polls); a warp whose wait runs out counts in ftle_counters.n_wait_timeouts and
// stops, thread 0 first waiting, again bounded, for the copy it still has in flight.
constexpr int kStageTile = 256;
constexpr uint32_t kStageWaitPolls = 1u << 22;

template <int DIM, int W>
__global__ void __launch_bounds__(kStageTile) k_grad_f32_ell_staged(GradArgs a) {
  constexpr int T = kStageTile;
  __shared__ __align__(128) int32_t s_idx[2][W][T];
  __shared__ __align__(8) uint64_t s_full[2], s_empty[2];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t n = a.n;
  const int64_t ntiles = (n + T - 1) / T;
  if ((int64_t)blockIdx.x >= ntiles) return;  // the same for every thread of the block
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      mbar_init(&s_full[st], 1);
      mbar_init(&s_empty[st], T);
    }
    mbar_init_fence();
  }
  __syncthreads();
  auto issue = [&](int64_t tile, int stage) {  // thread 0
    const int64_t t0 = tile * T;
    const uint32_t bytes = (uint32_t)(n - t0 < T ? n - t0 : T) * 4u;
    mbar_arrive_expect_tx(&s_full[stage], bytes * W);
#pragma unroll
    for (int s = 0; s < W; ++s) bulk_g2s(&s_idx[stage][s][0], a.ell + (int64_t)s * n + t0, bytes, &s_full[stage]);
  };
  if (tid == 0) issue(blockIdx.x, 0);
  int k = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int stage = k & 1;
    const int64_t next = tile + gridDim.x;
    bool ok = true, issued = false;
    if (tid == 0 && next < ntiles) {
      // the other stage was read in iteration k - 1: refill it once every thread released it
      if (k >= 1) ok = mbar_wait_bounded(&s_empty[stage ^ 1], (uint32_t)((k - 1) >> 1) & 1u, kStageWaitPolls);
      if (ok) {
        fence_proxy_async_smem();
        issue(next, stage ^ 1);
        issued = true;
      }
    }
    if (ok) ok = mbar_wait_bounded(&s_full[stage], (uint32_t)(k >> 1) & 1u, kStageWaitPolls);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicAdd(&a.hdr->n_wait_timeouts, 1ull);
      if (tid == 0) {
        // the copies this block still has in flight land in its shared memory: wait for them
        mbar_wait_bounded(&s_full[stage], (uint32_t)(k >> 1) & 1u, kStageWaitPolls);
        if (issued) mbar_wait_bounded(&s_full[stage ^ 1], (uint32_t)((k + 1) >> 1) & 1u, kStageWaitPolls);
      }
      break;
    }
    const int64_t i = tile * T + tid;
    int js[W];
#pragma unroll
    for (int s = 0; s < W; ++s) js[s] = s_idx[stage][s][tid];
    mbar_arrive(&s_empty[stage]);
    const bool flag = i < n && grad_node_f32_rec_slots<DIM, W>(a, i, js);
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long basepos = 0;
      if (lane == leader) basepos = atomicAdd(&a.hdr->n_flagged, (unsigned long long)__popc(mask));
      basepos = __shfl_sync(0xffffffffu, basepos, leader);
      if (flag) a.flag_list[basepos + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
}

// Float kernel over CSR rows with each tile's stretch of col_idx staged in shared memory.  The
// rows of a tile of 256 consecutive nodes are one contiguous stretch [row_ptr[t0],
// row_ptr[t0 + 256]) of col_idx; thread 0 brings it into shared memory with one bulk copy a tile
// ahead (two stages, mbarriers as in k_grad_f32_ell_staged), taking the row_ptr bounds it needs
// from loads issued one tile earlier still, so that nothing waits on them.  The copy covers the
// stretch from its start rounded down to a 16-byte boundary to its end rounded down likewise; a
// node reads the few indices past that end (and every index of a stretch longer than a stage) from
// global memory.  The per-node arithmetic and the neighbour order are grad_node_f32_rec's (same
// results bit for bit).  The copy stays inside [0, nnz) whatever row_ptr holds; the gathers trust
// the indices as the plain kernel does.
constexpr int kCsrStageInts = 16 * kStageTile;  // indices per stage: 16 per node of a full tile

template <int DIM>
__global__ void __launch_bounds__(kStageTile) k_grad_f32_csr_staged(GradArgs a) {
  constexpr int T = kStageTile;
  __shared__ __align__(128) int32_t s_idx[2][kCsrStageInts];
  __shared__ __align__(8) uint64_t s_full[2], s_empty[2];
  __shared__ int64_t s_lo[2], s_hi[2];  // positions [lo, hi) of col_idx held by the stage
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t n = a.n;
  const int64_t ntiles = (n + T - 1) / T;
  if ((int64_t)blockIdx.x >= ntiles) return;  // the same for every thread of the block
  if (tid == 0) {
    for (int st = 0; st < 2; ++st) {
      mbar_init(&s_full[st], 1);
      mbar_init(&s_empty[st], T);
    }
    mbar_init_fence();
  }
  __syncthreads();
  // thread 0: the row_ptr bounds of a tile, loaded ahead of its copy
  auto bounds = [&](int64_t tile, int64_t& lo, int64_t& hi) {
    const int64_t t0 = tile * T, t1 = t0 + T < n ? t0 + T : n;
    lo = __ldg(a.row_ptr + t0);
    hi = __ldg(a.row_ptr + t1);
  };
  auto issue = [&](int stage, int64_t lo, int64_t hi) {  // thread 0
    int64_t lo0 = lo & ~(int64_t)3, hi0 = hi & ~(int64_t)3;
    if (lo0 < 0 || hi0 > a.nnz || hi0 <= lo0 || hi0 - lo0 > kCsrStageInts) hi0 = lo0 = lo;  // nothing staged
    s_lo[stage] = lo0;
    s_hi[stage] = hi0;
    if (hi0 > lo0) {
      const uint32_t bytes = (uint32_t)(hi0 - lo0) * 4u;
      mbar_arrive_expect_tx(&s_full[stage], bytes);
      bulk_g2s(&s_idx[stage][0], a.col_idx + lo0, bytes, &s_full[stage]);
    } else {
      mbar_arrive(&s_full[stage]);
    }
  };
  int64_t plo = 0, phi = 0;  // thread 0: bounds of the next tile to issue
  if (tid == 0) {
    int64_t lo, hi;
    bounds(blockIdx.x, lo, hi);
    issue(0, lo, hi);
    if ((int64_t)blockIdx.x + gridDim.x < ntiles) bounds(blockIdx.x + gridDim.x, plo, phi);
  }
  int k = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
    const int stage = k & 1;
    const int64_t next = tile + gridDim.x;
    bool ok = true, issued = false;
    if (tid == 0 && next < ntiles) {
      if (k >= 1) ok = mbar_wait_bounded(&s_empty[stage ^ 1], (uint32_t)((k - 1) >> 1) & 1u, kStageWaitPolls);
      if (ok) {
        fence_proxy_async_smem();
        issue(stage ^ 1, plo, phi);
        issued = true;
        if (next + gridDim.x < ntiles) bounds(next + gridDim.x, plo, phi);
      }
    }
    if (ok) ok = mbar_wait_bounded(&s_full[stage], (uint32_t)(k >> 1) & 1u, kStageWaitPolls);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) atomicAdd(&a.hdr->n_wait_timeouts, 1ull);
      if (tid == 0) {
        mbar_wait_bounded(&s_full[stage], (uint32_t)(k >> 1) & 1u, kStageWaitPolls);
        if (issued) mbar_wait_bounded(&s_full[stage ^ 1], (uint32_t)((k + 1) >> 1) & 1u, kStageWaitPolls);
      }
      break;
    }
    const int64_t lo = s_lo[stage], hi = s_hi[stage];
    const int64_t i = tile * T + tid;
    int rs = 0, re = 0;
    if (i < n) {
      rs = __ldg(a.row_ptr + i);
      re = __ldg(a.row_ptr + i + 1);
    }
    bool flag = false;
    if (i < n) {
      float xi[DIM], hi_[DIM], li[DIM];
      float m[DIM * (DIM + 1) / 2] = {}, b[DIM * DIM] = {};
      load_record<DIM>(a.rec, i, xi, hi_, li);
      for (int e = rs; e < re; ++e) {
        const int j = (e >= lo && e < hi) ? s_idx[stage][e - lo] : ld_index(a.col_idx + e);
        grad_accumulate_rec<DIM>(a.rec, j, xi, hi_, li, m, b);
      }
      mbar_arrive(&s_empty[stage]);
      flag = grad_finish_f32<DIM>(a, i, re - rs, m, b);
    } else {
      mbar_arrive(&s_empty[stage]);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long basepos = 0;
      if (lane == leader) basepos = atomicAdd(&a.hdr->n_flagged, (unsigned long long)__popc(mask));
      basepos = __shfl_sync(0xffffffffu, basepos, leader);
      if (flag) a.flag_list[basepos + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
}

// Float kernel over the implicit neighbours of a lattice stencil.
template <int DIM, int ST, bool REC, int PL, typename CT>
__global__ void __launch_bounds__(256) k_grad_f32_stencil(GradArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n = a.n;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool flag = i < n && grad_node_f32_stencil<DIM, ST, REC, PL, CT>(a, i);
    const unsigned mask = __ballot_sync(0xffffffffu, flag);
    if (mask) {
      const int leader = __ffs(mask) - 1;
      unsigned long long basepos = 0;
      if (lane == leader) basepos = atomicAdd(&a.hdr->n_flagged, (unsigned long long)__popc(mask));
      basepos = __shfl_sync(0xffffffffu, basepos, leader);
      if (flag) a.flag_list[basepos + __popc(mask & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
}

// ----------------------------------------------------------------------------- double kernel

// Every node (FTLE_PREC_FP64) or the nodes of a list, with lanes per node as the list's length
// allows (grad_list_f64).
template <int DIM, int PL, typename CT, typename OT>
__global__ void __launch_bounds__(128) k_grad_f64(GradArgs a) {
  const int64_t count = a.list ? (int64_t)*a.list_count : a.n;
  grad_list_f64<DIM>(
      count, kF64Lanes<DIM>,
      [=](int64_t slot, int sub, int L, double* m, double* b) {
        const int64_t i = a.list ? (int64_t)a.list[slot] : slot;
        const int rs = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
        grad_moments_f64<DIM, PL, CT>(a, i, rs + sub, re, L, m, b);
        return re - rs;
      },
      [=](int64_t slot, int k, const double* m, const double* b) {
        grad_finish_f64<DIM, OT>(a, a.list ? (int64_t)a.list[slot] : slot, k, m, b);
      });
}

// ----------------------------------------------------------------------------- refine marks

__global__ void k_refine_mark(GradArgs a, int32_t* mark_list, uint32_t* bitmap) {
  const int64_t count = (int64_t)*a.list_count;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < count;
       slot += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = a.list[slot];
    mark_node(i, bitmap, mark_list, &a.hdr->n_readvected);
    const int rs = a.row_ptr[i], re = a.row_ptr[i + 1];
    for (int e = rs; e < re; ++e) mark_node(a.col_idx[e], bitmap, mark_list, &a.hdr->n_readvected);
  }
}

// ----------------------------------------------------------------------------- ELL from CSR

__global__ void k_ell_from_csr(int64_t n, const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                               int width, int32_t* __restrict__ ell) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int rs = row_ptr[i], re = row_ptr[i + 1];
    for (int s = 0; s < width; ++s) ell[(int64_t)s * n + i] = (rs + s < re) ? col_idx[rs + s] : -1;
  }
}

int launch_ell_from_csr(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, int width, int32_t* ell, int grid,
                        cudaStream_t s) {
  k_ell_from_csr<<<grid, 256, 0, s>>>(n, row_ptr, col_idx, width, ell);
  FTLE_LAUNCH_CHECK("k_ell_from_csr launch");
  return FTLE_OK;
}

// ----------------------------------------------------------------------------- launchers

// The staged kernel applies to records with the widths of the triangle (6) and Kuhn (14) lists.
template <int DIM>
static bool grad_f32_ell_staged(const GradArgs& a, cudaStream_t s) {
  constexpr int W = DIM == 2 ? 6 : 14;
  if (!a.staged || a.ell_width != W || (a.n & 3) || ((uintptr_t)a.ell & 15)) return false;
  const int64_t tiles = (a.n + kStageTile - 1) / kStageTile;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grad_f32_ell_staged<DIM, W>, kStageTile, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  const int64_t cap = (int64_t)sms * per_sm;
  k_grad_f32_ell_staged<DIM, W><<<(int)(tiles < cap ? tiles : cap), kStageTile, 0, s>>>(a);
  return true;
}

// The staged CSR kernel applies to records over any rows (col_idx 16-byte aligned).
template <int DIM>
static bool grad_f32_csr_staged(const GradArgs& a, cudaStream_t s) {
  if (!a.staged || a.nnz <= 0 || ((uintptr_t)a.col_idx & 15)) return false;
  const int64_t tiles = (a.n + kStageTile - 1) / kStageTile;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_grad_f32_csr_staged<DIM>, kStageTile, 0) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  const int64_t cap = (int64_t)sms * per_sm;
  k_grad_f32_csr_staged<DIM><<<(int)(tiles < cap ? tiles : cap), kStageTile, 0, s>>>(a);
  return true;
}

template <int DIM, int PL, typename CT, bool REC>
static void grad_f32_ell_dispatch(const GradArgs& a, int grid, int block, cudaStream_t s) {
  if constexpr (REC) {
    if (grad_f32_ell_staged<DIM>(a, s)) return;
  }
  switch (a.ell_width) {
    case 4: k_grad_f32_ell<DIM, PL, CT, 4, REC><<<grid, block, 0, s>>>(a); break;
    case 6: k_grad_f32_ell<DIM, PL, CT, 6, REC><<<grid, block, 0, s>>>(a); break;
    case 8: k_grad_f32_ell<DIM, PL, CT, 8, REC><<<grid, block, 0, s>>>(a); break;
    case 14: k_grad_f32_ell<DIM, PL, CT, 14, REC><<<grid, block, 0, s>>>(a); break;
    case 16: k_grad_f32_ell<DIM, PL, CT, 16, REC><<<grid, block, 0, s>>>(a); break;
    default: k_grad_f32_ell<DIM, PL, CT, 0, REC><<<grid, block, 0, s>>>(a); break;
  }
}

template <int DIM, int ST, int PL>
static void grad_f32_stencil_dispatch(bool rec, bool coord64, const GradArgs& a, int grid, int block, cudaStream_t s) {
  if constexpr (PL == PHI32PAIR) {
    if (rec) {
      k_grad_f32_stencil<DIM, ST, true, PL, float><<<grid, block, 0, s>>>(a);
      return;
    }
  }
  if (coord64)
    k_grad_f32_stencil<DIM, ST, false, PL, double><<<grid, block, 0, s>>>(a);
  else
    k_grad_f32_stencil<DIM, ST, false, PL, float><<<grid, block, 0, s>>>(a);
}

template <int DIM, int PL>
static void grad_f32_dispatch(bool coord64, const GradArgs& a, int grid, int block, cudaStream_t s) {
  // gradient records exist for compensated flowmaps; they carry float coordinates
  const bool rec = PL == PHI32PAIR && a.rec && !coord64;
  if (a.stencil == FTLE_STENCIL_AXIS) {
    grad_f32_stencil_dispatch<DIM, FTLE_STENCIL_AXIS, PL>(rec, coord64, a, grid, block, s);
  } else if (a.stencil != FTLE_STENCIL_NONE) {  // TRI in 2D, KUHN in 3D (checked by the C-ABI)
    grad_f32_stencil_dispatch<DIM, DIM == 2 ? FTLE_STENCIL_TRI : FTLE_STENCIL_KUHN, PL>(rec, coord64, a, grid, block, s);
  } else if (a.ell) {
    if (rec)
      grad_f32_ell_dispatch<DIM, PL, float, true>(a, grid, block, s);
    else if (coord64)
      grad_f32_ell_dispatch<DIM, PL, double, false>(a, grid, block, s);
    else
      grad_f32_ell_dispatch<DIM, PL, float, false>(a, grid, block, s);
  } else if (rec) {
    if constexpr (PL == PHI32PAIR) {
      if (grad_f32_csr_staged<DIM>(a, s)) return;
    }
    k_grad_f32<DIM, PL, float, true><<<grid, block, 0, s>>>(a);
  } else if (coord64) {
    k_grad_f32<DIM, PL, double, false><<<grid, block, 0, s>>>(a);
  } else {
    k_grad_f32<DIM, PL, float, false><<<grid, block, 0, s>>>(a);
  }
}

int launch_grad_f32(int dim, int phi_layout, bool coord64, const GradArgs& a, int grid, int block,
                    cudaStream_t stream) {
  if (dim == 2 && phi_layout == PHI32) grad_f32_dispatch<2, PHI32>(coord64, a, grid, block, stream);
  else if (dim == 2 && phi_layout == PHI32PAIR) grad_f32_dispatch<2, PHI32PAIR>(coord64, a, grid, block, stream);
  else if (dim == 3 && phi_layout == PHI32) grad_f32_dispatch<3, PHI32>(coord64, a, grid, block, stream);
  else if (dim == 3 && phi_layout == PHI32PAIR) grad_f32_dispatch<3, PHI32PAIR>(coord64, a, grid, block, stream);
  else return fail(FTLE_EUNSUPPORTED, "gradient: float kernel for dim %d layout %d", dim, phi_layout);
  FTLE_LAUNCH_CHECK("k_grad_f32 launch");
  return FTLE_OK;
}

template <int DIM, int PL>
static void grad_f64_dispatch(bool coord64, bool out64, const GradArgs& a, int grid, int block,
                              cudaStream_t s) {
  if (coord64) {
    if (out64) k_grad_f64<DIM, PL, double, double><<<grid, block, 0, s>>>(a);
    else k_grad_f64<DIM, PL, double, float><<<grid, block, 0, s>>>(a);
  } else {
    if (out64) k_grad_f64<DIM, PL, float, double><<<grid, block, 0, s>>>(a);
    else k_grad_f64<DIM, PL, float, float><<<grid, block, 0, s>>>(a);
  }
}

int launch_grad_f64(int dim, int phi_layout, bool coord64, bool out64, const GradArgs& a, int grid,
                    int block, cudaStream_t stream) {
  if (dim == 2) {
    if (phi_layout == PHI64) grad_f64_dispatch<2, PHI64>(coord64, out64, a, grid, block, stream);
    else if (phi_layout == PHI32) grad_f64_dispatch<2, PHI32>(coord64, out64, a, grid, block, stream);
    else grad_f64_dispatch<2, PHI32PAIR>(coord64, out64, a, grid, block, stream);
  } else if (dim == 3) {
    if (phi_layout == PHI64) grad_f64_dispatch<3, PHI64>(coord64, out64, a, grid, block, stream);
    else if (phi_layout == PHI32) grad_f64_dispatch<3, PHI32>(coord64, out64, a, grid, block, stream);
    else grad_f64_dispatch<3, PHI32PAIR>(coord64, out64, a, grid, block, stream);
  } else {
    return fail(FTLE_EUNSUPPORTED, "gradient: double kernel for dim %d", dim);
  }
  FTLE_LAUNCH_CHECK("k_grad_f64 launch");
  return FTLE_OK;
}

int launch_refine_mark(const GradArgs& a, int32_t* mark_list, uint32_t* bitmap, int grid, int block,
                       cudaStream_t stream) {
  k_refine_mark<<<grid, block, 0, stream>>>(a, mark_list, bitmap);
  FTLE_LAUNCH_CHECK("k_refine_mark launch");
  return FTLE_OK;
}

}  // namespace ftle
