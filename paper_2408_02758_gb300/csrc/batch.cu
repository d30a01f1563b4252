// Batched FTLE: many independent problems of uneven mesh size and horizon in one launch
// sequence.  The host plans a queue of (instance, node range) items ordered longest-first (LPT:
// cost = nodes x RK4 steps), persistent blocks pull items with one atomic per item, and the per
// node arithmetic is the single-problem kernels' (rk4_step, grad_node_f32, grad_node_f64), so
// every instance's FTLE equals its single-problem result.  Nodes that need the FP64 path are kept
// as (instance, node) pairs; their re-advection runs in float-float with per-lane time
// coefficients (lanes of one warp may belong to different instances).  The sequence can be
// captured once into a CUDA graph (ftle_batch_plan_*) and replayed.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include <type_traits>

#include "batch.cuh"
#include "capi_internal.cuh"
#include "gradient_node.cuh"

namespace ftle {

// ------------------------------------------------------------------------------- kernels

// Compensated kernels held to four 256-thread blocks per SM (64 registers): 155.0 -> 158.1 M
// points/s on the 64-instance batch, against 72 registers and three blocks.
template <int KIND, int DIM, int PREC, int OUT>
__global__ void __launch_bounds__(256, PREC == P32C ? 4 : 1) k_batch_advect(const BatchInst* __restrict__ insts,
                                                      const BatchItem* __restrict__ items, int n_items,
                                                      unsigned int* next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kTable = (KIND == FTLE_FLOW_DOUBLE_GYRE);
  float2* tab32 = reinterpret_cast<float2*>(smem_raw);
  double* tab64 = reinterpret_cast<double*>(smem_raw);
  __shared__ int s_item, s_tab_inst;
  if (threadIdx.x == 0) s_tab_inst = -1;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const AdvArgs a = insts[item.inst].adv;
    const int64_t i = (int64_t)item.lo + threadIdx.x;
    const bool active = i < item.hi;
    float xh[DIM], xl[DIM], x0[DIM];
    double xd[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double c = active ? (double)__ldg(reinterpret_cast<const float*>(a.coords) + d * a.n_mesh + i) : 0.0;
      xd[d] = c;
      xh[d] = (float)c;
      xl[d] = 0.f;
      x0[d] = xh[d];
    }
    bool safe = false;
    if constexpr (PREC == P32C && KIND == FTLE_FLOW_DOUBLE_GYRE) safe = dg_node_safe(a, xd[0], xd[1]);
    if constexpr (PREC == P32C && KIND == FTLE_FLOW_ABC) safe = a.rot_safe != 0;
    const int nchunks = (a.nsteps + kAdvChunk - 1) / kAdvChunk;
    // run-boundary states of compensated 2D flowmaps (as k_advect stores them)
    constexpr bool kSegs = PREC == P32C && OUT == O32PAIR && DIM == 2;
    int seg_slot = 0, next_seg = a.seg_len;
    AbcCarry carry;  // as k_advect: the same steps, the same bits
    for (int ch = 0; ch < nchunks; ++ch) {
      const int k0 = ch * kAdvChunk;
      const int k1 = min(a.nsteps, k0 + kAdvChunk);
      if constexpr (kTable) {
        if (!(s_tab_inst == item.inst && nchunks == 1)) {
          __syncthreads();
          build_table<KIND, PREC>(a, tab32, tab64, k0, k1);
          __syncthreads();
          if (threadIdx.x == 0) s_tab_inst = nchunks == 1 ? item.inst : -1;
        }
      }
      if (!active) continue;
      for (int k = k0; k < k1;) {
        const int stop = (kSegs && a.seg) ? min(k1, next_seg) : k1;
        auto steps = [&](auto safe, auto carried) {
          if constexpr (KIND == FTLE_FLOW_ABC && PREC == P32C && decltype(safe)::value && decltype(carried)::value) {
            abc_steps_carried(a, k, stop, xh, xl, carry);
            return;
          }
          for (; k < stop; ++k) {
            const int m = 2 * (k - k0);
            const Coef c0 = coef_at<KIND, PREC>(tab32, tab64, m);
            const Coef c1 = coef_at<KIND, PREC>(tab32, tab64, m + 1);
            const Coef c2 = coef_at<KIND, PREC>(tab32, tab64, m + 2);
            if constexpr (KIND == FTLE_FLOW_ABC && PREC == P32C && decltype(safe)::value && decltype(carried)::value)
              abc_step_carried(a, k, xh, xl, carry);
            else
              rk4_step<KIND, DIM, PREC, decltype(safe)::value>(a, c0, c1, c2, xh, xl, xd);
          }
        };
        // the unchecked steps exactly where k_advect takes them (dg_node_safe; ABC: rot_safe),
        // stage one carried as k_advect carries it
        if (safe && a.abc_refresh > 1)
          steps(std::true_type{}, std::true_type{});
        else if (safe)
          steps(std::true_type{}, std::false_type{});
        else
          steps(std::false_type{}, std::false_type{});
        if constexpr (kSegs) {
          if (a.seg && k == next_seg) {
            if (seg_slot < kSegments - 1)
              store_state<OUT, DIM>(a.seg + (int64_t)seg_slot * a.seg_stride, a.n_mesh, i, xh, xl, xd);
            ++seg_slot;
            next_seg += a.seg_len;
          }
        }
      }
    }
    if constexpr (kSegs) {
      if (a.seg && active)
        for (; seg_slot < kSegments - 1; ++seg_slot)
          store_state<OUT, DIM>(a.seg + (int64_t)seg_slot * a.seg_stride, a.n_mesh, i, xh, xl, xd);
    }
    if (active) {
      split_state<PREC, DIM>(xh, xl, xd);
      store_state<OUT, DIM>(a.out, a.n_mesh, i, xh, xl, xd);
      if constexpr (OUT == O32PAIR) {
        if (a.rec) store_record<DIM>(a.rec, i, x0, xh, xl);
      }
    }
  }
}

template <int DIM, int PL>
__global__ void __launch_bounds__(256) k_batch_grad(const BatchInst* __restrict__ insts,
                                                    const BatchItem* __restrict__ items, int n_items,
                                                    unsigned int* next, ftle_counters* hdr, int2* flags) {
  __shared__ int s_item;
  const int lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    const GradArgs g = insts[item.inst].grad;
    for (int base = item.lo; base < item.hi; base += blockDim.x) {
      const int i = base + threadIdx.x;
      bool flag = false;
      if (i < item.hi) {
        if constexpr (PL == PHI32PAIR)
          flag = grad_node_f32_rec<DIM>(g, i);
        else
          flag = grad_node_f32<DIM, PL, float>(g, i);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, flag);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        unsigned long long pos = 0;
        if (lane == leader) pos = atomicAdd(&hdr->n_flagged, (unsigned long long)__popc(mask));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (flag) flags[pos + __popc(mask & ((1u << lane) - 1u))] = make_int2(item.inst, i);
      }
    }
  }
}

template <int DIM, int PL>
__global__ void __launch_bounds__(128) k_batch_grad_f64(const BatchInst* __restrict__ insts, const int2* pairs,
                                                        const unsigned long long* count) {
  grad_list_f64<DIM>(
      (int64_t)*count, kF64Lanes<DIM>,
      [=](int64_t slot, int sub, int L, double* m, double* b) {
        const int2 p = pairs[slot];
        const GradArgs& a = insts[p.x].grad;
        const int rs = __ldg(a.row_ptr + p.y), re = __ldg(a.row_ptr + p.y + 1);
        grad_moments_f64<DIM, PL, float>(a, p.y, rs + sub, re, L, m, b);
        return re - rs;
      },
      [=](int64_t slot, int k, const double* m, const double* b) {
        const int2 p = pairs[slot];
        grad_finish_f64<DIM, float>(insts[p.x].grad, p.y, k, m, b);
      });
}

__device__ __forceinline__ void batch_mark_node(int inst, int j, int64_t off, uint32_t* bitmap, int2* marks,
                                                unsigned long long* n_marks) {
  const int64_t g = off + j;
  const uint32_t bit = 1u << (g & 31);
  const uint32_t old = atomicOr(bitmap + (g >> 5), bit);
  if (!(old & bit)) marks[atomicAdd(n_marks, 1ULL)] = make_int2(inst, j);
}

__global__ void k_batch_mark(const BatchInst* __restrict__ insts, const int2* flags, const unsigned long long* n_flags,
                             int2* marks, unsigned long long* n_marks, uint32_t* bitmap) {
  const int64_t cnt = (int64_t)*n_flags;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < cnt; s += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = flags[s];
    const GradArgs& g = insts[p.x].grad;
    const int64_t off = insts[p.x].off;
    batch_mark_node(p.x, p.y, off, bitmap, marks, n_marks);
    const int rs = g.row_ptr[p.y], re = g.row_ptr[p.y + 1];
    for (int e = rs; e < re; ++e) batch_mark_node(p.x, g.col_idx[e], off, bitmap, marks, n_marks);
  }
}

// ------------------------------------------------------------------------------- launchers

template <int KIND, int DIM>
static void batch_advect_prec(int prec, const BatchInst* insts, const BatchItem* items, int n_items,
                              unsigned int* next, int grid, int block, size_t smem, cudaStream_t s) {
  if (prec == P32C)
    k_batch_advect<KIND, DIM, P32C, O32PAIR><<<grid, block, smem, s>>>(insts, items, n_items, next);
  else
    k_batch_advect<KIND, DIM, P32, O32><<<grid, block, smem, s>>>(insts, items, n_items, next);
}

int launch_batch_advect(int kind, int dim, int prec, const BatchInst* insts, const BatchItem* items, int n_items,
                        unsigned int* next, int grid, int block, size_t smem, cudaStream_t s) {
  if (kind == FTLE_FLOW_DOUBLE_GYRE && dim == 2) batch_advect_prec<FTLE_FLOW_DOUBLE_GYRE, 2>(prec, insts, items, n_items, next, grid, block, smem, s);
  else if (kind == FTLE_FLOW_ABC && dim == 3) batch_advect_prec<FTLE_FLOW_ABC, 3>(prec, insts, items, n_items, next, grid, block, smem, s);
  else if (kind == FTLE_FLOW_LINEAR && dim == 2) batch_advect_prec<FTLE_FLOW_LINEAR, 2>(prec, insts, items, n_items, next, grid, block, smem, s);
  else if (kind == FTLE_FLOW_LINEAR && dim == 3) batch_advect_prec<FTLE_FLOW_LINEAR, 3>(prec, insts, items, n_items, next, grid, block, smem, s);
  else if (kind == FTLE_FLOW_SADDLE && dim == 2) batch_advect_prec<FTLE_FLOW_SADDLE, 2>(prec, insts, items, n_items, next, grid, block, smem, s);
  else if (kind == FTLE_FLOW_SADDLE && dim == 3) batch_advect_prec<FTLE_FLOW_SADDLE, 3>(prec, insts, items, n_items, next, grid, block, smem, s);
  else return fail(FTLE_EUNSUPPORTED, "batch: flow %d in %dD", kind, dim);
  FTLE_LAUNCH_CHECK("k_batch_advect launch");
  return FTLE_OK;
}

int launch_batch_grad(int dim, int phi_layout, const BatchInst* insts, const BatchItem* items, int n_items,
                      unsigned int* next, ftle_counters* hdr, int2* flags, int grid, int block, cudaStream_t s) {
  if (dim == 2 && phi_layout == PHI32PAIR) k_batch_grad<2, PHI32PAIR><<<grid, block, 0, s>>>(insts, items, n_items, next, hdr, flags);
  else if (dim == 2) k_batch_grad<2, PHI32><<<grid, block, 0, s>>>(insts, items, n_items, next, hdr, flags);
  else if (phi_layout == PHI32PAIR) k_batch_grad<3, PHI32PAIR><<<grid, block, 0, s>>>(insts, items, n_items, next, hdr, flags);
  else k_batch_grad<3, PHI32><<<grid, block, 0, s>>>(insts, items, n_items, next, hdr, flags);
  FTLE_LAUNCH_CHECK("k_batch_grad launch");
  return FTLE_OK;
}

int launch_batch_grad_f64(int dim, int phi_layout, const BatchInst* insts, const int2* pairs,
                          const unsigned long long* count, int grid, int block, cudaStream_t s) {
  if (dim == 2 && phi_layout == PHI32PAIR) k_batch_grad_f64<2, PHI32PAIR><<<grid, block, 0, s>>>(insts, pairs, count);
  else if (dim == 2) k_batch_grad_f64<2, PHI32><<<grid, block, 0, s>>>(insts, pairs, count);
  else if (phi_layout == PHI32PAIR) k_batch_grad_f64<3, PHI32PAIR><<<grid, block, 0, s>>>(insts, pairs, count);
  else k_batch_grad_f64<3, PHI32><<<grid, block, 0, s>>>(insts, pairs, count);
  FTLE_LAUNCH_CHECK("k_batch_grad_f64 launch");
  return FTLE_OK;
}

int launch_batch_mark(const BatchInst* insts, const int2* flags, const unsigned long long* n_flags, int2* marks,
                      unsigned long long* n_marks, uint32_t* bitmap, int grid, int block, cudaStream_t s) {
  k_batch_mark<<<grid, block, 0, s>>>(insts, flags, n_flags, marks, n_marks, bitmap);
  FTLE_LAUNCH_CHECK("k_batch_mark launch");
  return FTLE_OK;
}

// ------------------------------------------------------------------------------- planning

namespace {

struct BatchLayout {
  size_t header = 0, insts = 0, adv_items = 0, grad_items = 0, phi = 0, flags = 0, marks = 0, bitmap = 0, total = 0;
  std::vector<size_t> phi_off;
  int64_t total_nodes = 0;
  int max_items = 0;
};

BatchLayout batch_layout(int n_inst, const ftle_mesh* meshes, int precision) {
  BatchLayout L;
  size_t off = 0;
  int64_t tot = 0;
  int64_t items = 0;
  for (int q = 0; q < n_inst; ++q) {
    tot += meshes[q].n_nodes;
    items += (meshes[q].n_nodes + 31) / 32;
  }
  L.total_nodes = tot;
  L.max_items = (int)items;
  L.header = off;
  off += align256(sizeof(ftle_counters));
  L.insts = off;
  off += align256(sizeof(BatchInst) * (size_t)(n_inst > 0 ? n_inst : 1));
  L.adv_items = off;
  off += align256(sizeof(BatchItem) * (size_t)(items > 0 ? items : 1));
  L.grad_items = off;
  off += align256(sizeof(BatchItem) * (size_t)(items > 0 ? items : 1));
  L.phi = off;
  for (int q = 0; q < n_inst; ++q) {
    L.phi_off.push_back(off);
    off += align256(ftle_flowmap_bytes(meshes[q].dim, meshes[q].n_nodes, precision));
  }
  L.flags = off;
  off += align256(sizeof(int2) * (size_t)(tot > 0 ? tot : 1));
  L.marks = off;
  off += align256(sizeof(int2) * (size_t)(tot > 0 ? tot : 1));
  L.bitmap = off;
  off += align256(sizeof(uint32_t) * (size_t)((tot + 31) / 32 + 1));
  L.total = off;
  return L;
}

struct BatchPlanHost {
  int n_inst = 0, dim = 0, kind = 0, precision = 0, max_steps = 0;
  int adv_block = 256, grad_block = 256, grad_tile = 256, adv_grid = 1, grad_grid = 1;
  bool refine = true;
  bool validate = false;
  char* ws = nullptr;
  BatchLayout L;
  std::vector<BatchInst> insts;
  std::vector<BatchItem> adv_items, grad_items;
};

int plan_batch(int32_t n_inst, const ftle_mesh* meshes, const ftle_flow* flows, const double* T, double dt,
               int32_t precision, void* const* ftle_out, void* workspace, size_t workspace_bytes,
               const ftle_options* opt, BatchPlanHost& P) {
  int rc;
  if (n_inst <= 0 || !meshes || !flows || !T || !ftle_out) return fail(FTLE_EINVAL, "batch: empty batch or NULL arrays");
  if (precision != FTLE_PREC_FP32 && precision != FTLE_PREC_FP32C)
    return fail(FTLE_EINVAL, "batch: precision must be FP32 or FP32C");
  const Launch Lc = resolve_launch(opt);
  if ((rc = check_launch(Lc))) return rc;
  P.n_inst = n_inst;
  P.dim = meshes[0].dim;
  P.kind = flows[0].kind;
  P.precision = precision;
  P.refine = precision == FTLE_PREC_FP32C && Lc.refine_kappa >= 0;
  for (int q = 0; q < n_inst; ++q) {
    if ((rc = check_mesh(&meshes[q])) || (rc = check_flow(&flows[q], meshes[q].dim))) return rc;
    if (meshes[q].dim != P.dim || flows[q].kind != P.kind)
      return fail(FTLE_EINVAL, "batch: instances must share the dimension and the flow kind");
    if (meshes[q].coord_fp64) return fail(FTLE_EUNSUPPORTED, "batch: coordinates must be float");
    if (meshes[q].n_nodes > 0 && !ftle_out[q]) return fail(FTLE_EINVAL, "batch: ftle_out[%d] is NULL", q);
  }
  P.L = batch_layout(n_inst, meshes, precision);
  if ((rc = check_workspace(workspace, workspace_bytes, P.L.total))) return rc;
  P.ws = reinterpret_cast<char*>(workspace);
  // launch shapes (tile of the gradient queue: opt->grad_tile, a multiple of the block)
  P.adv_block = Lc.advect_block;
  P.grad_block = Lc.grad_block;
  P.grad_tile = (opt && opt->grad_tile > 0) ? opt->grad_tile : Lc.grad_block;
  if (P.grad_tile % P.grad_block) return fail(FTLE_EINVAL, "batch: grad_tile must be a multiple of grad_block");
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  P.adv_grid = sms * (Lc.advect_bps > 0 ? Lc.advect_bps : 2048 / P.adv_block);
  P.grad_grid = sms * std::max(1, 2048 / P.grad_block);

  ftle_counters* hdr = reinterpret_cast<ftle_counters*>(P.ws + P.L.header);
  P.insts.resize(n_inst);
  int64_t off = 0;
  std::vector<int> steps(n_inst);
  for (int q = 0; q < n_inst; ++q) {
    int nsteps = 0;
    if ((rc = check_time(T[q], dt, &nsteps))) return rc;
    steps[q] = nsteps;
    P.max_steps = std::max(P.max_steps, nsteps);
    BatchInst& bi = P.insts[q];
    memset(&bi, 0, sizeof bi);
    void* phi = P.ws + P.L.phi_off[q];
    bi.adv = make_adv_args(&meshes[q], &flows[q], 0.0, T[q], dt, nsteps);
    bi.adv.abc_refresh = bi.adv.carry_ok ? Lc.abc_refresh : 1;
    bi.adv.out = phi;
    if (precision == FTLE_PREC_FP32C && meshes[q].dim == 2) {
      bi.adv.seg = reinterpret_cast<float2*>(reinterpret_cast<char*>(phi) + seg_offset(2, meshes[q].n_nodes));
      bi.adv.seg_stride = (int64_t)(seg_slot_bytes(meshes[q].n_nodes) / sizeof(float2));
      bi.adv.seg_len = seg_len(nsteps);
    }
    float4* rec = precision == FTLE_PREC_FP32C
                      ? reinterpret_cast<float4*>(reinterpret_cast<char*>(phi) + rec_offset(meshes[q].dim, meshes[q].n_nodes))
                      : nullptr;
    bi.adv.rec = rec;
    Launch Lq = Lc;
    bi.grad = make_grad_args(&meshes[q], phi, T[q], ftle_out[q], nullptr, workspace, Lq);
    bi.grad.rec = rec;
    bi.grad.hdr = hdr;        // batch-wide counters
    bi.grad.flag_list = nullptr;
    bi.off = off;
    off += meshes[q].n_nodes;
  }
  // advection queue: items of one block of nodes, longest (steps x nodes) first
  for (int q = 0; q < n_inst; ++q)
    for (int64_t lo = 0; lo < meshes[q].n_nodes; lo += P.adv_block)
      P.adv_items.push_back({q, (int32_t)lo, (int32_t)std::min<int64_t>(meshes[q].n_nodes, lo + P.adv_block), 0});
  std::stable_sort(P.adv_items.begin(), P.adv_items.end(), [&](const BatchItem& x, const BatchItem& y) {
    return (int64_t)steps[x.inst] * (x.hi - x.lo) > (int64_t)steps[y.inst] * (y.hi - y.lo);
  });
  for (int q = 0; q < n_inst; ++q)
    for (int64_t lo = 0; lo < meshes[q].n_nodes; lo += P.grad_tile)
      P.grad_items.push_back({q, (int32_t)lo, (int32_t)std::min<int64_t>(meshes[q].n_nodes, lo + P.grad_tile), 0});
  if ((int)P.adv_items.size() > P.L.max_items || (int)P.grad_items.size() > P.L.max_items)
    return fail(FTLE_EINVAL, "batch: blocks narrower than 32 nodes are not supported");
  P.validate = Lc.validate_mesh;
  return FTLE_OK;
}

// ftle_options.validate_mesh: every instance's lists checked before anything else runs
// (synchronises `s` once per instance).
int validate_batch(const BatchPlanHost& P, const ftle_mesh* meshes, cudaStream_t s) {
  if (!P.validate) return FTLE_OK;
  for (int q = 0; q < P.n_inst; ++q) {
    const int rc = validate_mesh_sync(&meshes[q], P.ws + P.L.header, s, nullptr);
    if (rc) {
      char msg[400];
      snprintf(msg, sizeof msg, "%s", ftle_last_error());
      return fail(rc, "batch instance %d: %s", q, msg);
    }
  }
  return FTLE_OK;
}

int upload_batch(const BatchPlanHost& P, cudaStream_t s) {
  FTLE_CUDA_CHECK(cudaMemcpyAsync(P.ws + P.L.insts, P.insts.data(), sizeof(BatchInst) * P.insts.size(),
                                  cudaMemcpyHostToDevice, s));
  FTLE_CUDA_CHECK(cudaMemcpyAsync(P.ws + P.L.adv_items, P.adv_items.data(), sizeof(BatchItem) * P.adv_items.size(),
                                  cudaMemcpyHostToDevice, s));
  FTLE_CUDA_CHECK(cudaMemcpyAsync(P.ws + P.L.grad_items, P.grad_items.data(),
                                  sizeof(BatchItem) * P.grad_items.size(), cudaMemcpyHostToDevice, s));
  return FTLE_OK;
}

// The launch sequence of one batch (capturable: memsets and kernels only).
int enqueue_batch(const BatchPlanHost& P, cudaStream_t s) {
  int rc;
  char* w = P.ws;
  ftle_counters* hdr = reinterpret_cast<ftle_counters*>(w + P.L.header);
  const BatchInst* insts = reinterpret_cast<const BatchInst*>(w + P.L.insts);
  unsigned int* adv_next = reinterpret_cast<unsigned int*>(&hdr->reserved[0]);
  unsigned int* grad_next = reinterpret_cast<unsigned int*>(&hdr->reserved[1]);
  int2* flags = reinterpret_cast<int2*>(w + P.L.flags);
  int2* marks = reinterpret_cast<int2*>(w + P.L.marks);
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  const int prec = P.precision == FTLE_PREC_FP32C ? P32C : P32;
  const int pl = P.precision == FTLE_PREC_FP32C ? PHI32PAIR : PHI32;
  FTLE_CUDA_CHECK(cudaMemsetAsync(hdr, 0, sizeof(ftle_counters), s));
  const size_t smem = advect_smem_bytes(P.kind, prec, P.max_steps);
  if ((rc = launch_batch_advect(P.kind, P.dim, prec, insts, reinterpret_cast<const BatchItem*>(w + P.L.adv_items),
                                (int)P.adv_items.size(), adv_next, P.adv_grid, P.adv_block, smem, s)))
    return rc;
  if ((rc = launch_batch_grad(P.dim, pl, insts, reinterpret_cast<const BatchItem*>(w + P.L.grad_items),
                              (int)P.grad_items.size(), grad_next, hdr, flags, P.grad_grid, P.grad_block, s)))
    return rc;
  // with the refinement on, the flagged nodes get their FP64 pass after the re-advection (which
  // overwrites whatever a pass here would write), so only a batch without it runs one now
  if (!P.refine) return launch_batch_grad_f64(P.dim, pl, insts, flags, &hdr->n_flagged, sms * 4, 128, s);
  FTLE_CUDA_CHECK(cudaMemsetAsync(w + P.L.bitmap, 0, sizeof(uint32_t) * (size_t)((P.L.total_nodes + 31) / 32 + 1), s));
  FTLE_CUDA_CHECK(cudaMemsetAsync(&hdr->n_degenerate, 0, sizeof(unsigned long long), s));
  if ((rc = launch_batch_mark(insts, flags, &hdr->n_flagged, marks, &hdr->n_readvected,
                              reinterpret_cast<uint32_t*>(w + P.L.bitmap), sms * 4, 128, s)))
    return rc;
  if (P.kind == FTLE_FLOW_DOUBLE_GYRE && P.dim == 2 && P.precision == FTLE_PREC_FP32C)
    rc = launch_batch_refine_runs_dg(insts, marks, &hdr->n_readvected, sms * 8, s);
  else
    rc = launch_batch_advect_ds(P.kind, P.dim, insts, marks, &hdr->n_readvected, sms * 8, 32, s);
  if (rc) return rc;
  return launch_batch_grad_f64(P.dim, pl, insts, flags, &hdr->n_flagged, sms * 4, 128, s);
}

}  // namespace
}  // namespace ftle

using namespace ftle;

struct ftle_batch_plan {
  BatchPlanHost host;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

size_t ftle_batch_workspace_bytes(int32_t n_inst, const ftle_mesh* meshes, int32_t precision) {
  if (n_inst <= 0 || !meshes) return 0;
  for (int q = 0; q < n_inst; ++q)
    if (meshes[q].n_nodes < 0 || (meshes[q].dim != 2 && meshes[q].dim != 3)) return 0;
  return batch_layout(n_inst, meshes, precision).total;
}

int ftle_batch(int32_t n_inst, const ftle_mesh* meshes, const ftle_flow* flows, const double* T, double dt,
               int32_t precision, void* const* ftle_out, void* workspace, size_t workspace_bytes,
               const ftle_options* opt, void* stream) {
  PhaseRange range("ftle.batch");
  BatchPlanHost P;
  int rc = plan_batch(n_inst, meshes, flows, T, dt, precision, ftle_out, workspace, workspace_bytes, opt, P);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = validate_batch(P, meshes, s))) return rc;
  if ((rc = upload_batch(P, s))) return rc;
  // the host vectors are released on return: wait for the uploads (pageable sources)
  FTLE_CUDA_CHECK(cudaStreamSynchronize(s));
  return enqueue_batch(P, s);
}

int ftle_batch_plan_create(int32_t n_inst, const ftle_mesh* meshes, const ftle_flow* flows, const double* T,
                           double dt, int32_t precision, void* const* ftle_out, void* workspace,
                           size_t workspace_bytes, const ftle_options* opt, void* stream, ftle_batch_plan** plan) {
  if (!plan) return fail(FTLE_EINVAL, "plan is NULL");
  *plan = nullptr;
  ftle_batch_plan* p = new (std::nothrow) ftle_batch_plan();
  if (!p) return fail(FTLE_ENOMEM, "host allocation failed");
  int rc = plan_batch(n_inst, meshes, flows, T, dt, precision, ftle_out, workspace, workspace_bytes, opt, p->host);
  cudaStream_t s = (cudaStream_t)stream;
  if (!rc) rc = validate_batch(p->host, meshes, s);
  if (!rc) rc = upload_batch(p->host, s);
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  }
  if (!rc) {
    // capture on a private stream so the caller's stream is never left in capture mode
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreateWithFlags");
    if (!rc) {
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamBeginCapture");
      const int rc2 = rc ? rc : enqueue_batch(p->host, cs);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cs, &g);
      if (!rc) rc = rc2;
      if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
      p->graph = g;
      if (!rc) {
        e = cudaGraphInstantiate(&p->exec, g, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
      }
      cudaStreamDestroy(cs);
    }
  }
  if (rc) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    delete p;
    return rc;
  }
  *plan = p;
  return FTLE_OK;
}

int ftle_batch_plan_launch(ftle_batch_plan* plan, void* stream) {
  if (!plan || !plan->exec) return fail(FTLE_EINVAL, "plan is NULL or not instantiated");
  PhaseRange range("ftle.batch_plan_launch");
  FTLE_CUDA_CHECK(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
  return FTLE_OK;
}

int ftle_batch_plan_destroy(ftle_batch_plan* plan) {
  if (!plan) return FTLE_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
  return FTLE_OK;
}

}  // extern "C"
