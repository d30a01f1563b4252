// Float-float RK4 re-advection of a short node list (the nodes the float gradient kernel flagged
// and their neighbours).  Same scheme and stage times as k_advect, every operation in
// float-float (~48-bit) arithmetic on the FP32 pipes; one node per lane (two for the 2D double
// gyre, three for the ABC flow), 32-thread blocks so the few warps spread over the SMs.  The double-gyre coefficient a(t) is tabulated
// per block in double and split into float-float.
#include "advect.cuh"
#include "batch.cuh"
#include "capi_internal.cuh"
#include "dsfloat.cuh"

namespace ftle {

struct DsFlow {
  dsf c[9];
};

template <int KIND, int DIM>
__device__ __forceinline__ void vel_ds(const DsFlow& F, const dsf* x, dsf a, dsf* u) {
  if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
    const dsf b = ds_add_f(ds_make(-2.0f * a.h, -2.0f * a.l), 1.0f);  // b = 1 - 2a
    const dsf t1 = ds_mul(a, x[0]);
    const dsf f = ds_mul(ds_add(t1, b), x[0]);                        // a x^2 + b x
    const dsf fx = ds_add(ds_make(2.0f * t1.h, 2.0f * t1.l), b);      // 2 a x + b
    dsf sf, cf, sy, cy;
    ds_sincospi(f, sf, cf);
    ds_sincospi(x[1], sy, cy);
    u[0] = ds_neg(ds_mul(ds_mul(F.c[0], sf), cy));
    u[1] = ds_mul(ds_mul(ds_mul(F.c[0], cf), sy), fx);
  } else if constexpr (KIND == FTLE_FLOW_ABC) {
    dsf sx, cx, sy, cy, sz, cz;
    ds_sincos(x[0], sx, cx);
    ds_sincos(x[1], sy, cy);
    ds_sincos(x[2], sz, cz);
    u[0] = ds_add(ds_mul_u(F.c[0], sz), ds_mul_u(F.c[2], cy));
    u[1] = ds_add(ds_mul_u(F.c[1], sx), ds_mul_u(F.c[0], cz));
    u[2] = ds_add(ds_mul_u(F.c[2], sy), ds_mul_u(F.c[1], cx));
  } else if constexpr (KIND == FTLE_FLOW_LINEAR) {
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      dsf s = ds_mul(F.c[r * DIM], x[0]);
#pragma unroll
      for (int c = 1; c < DIM; ++c) s = ds_add(s, ds_mul(F.c[r * DIM + c], x[c]));
      u[r] = s;
    }
  } else {
    u[0] = x[0];
    u[1] = ds_neg(x[1]);
    if constexpr (DIM == 3) u[2] = ds_make(0.f, 0.f);
  }
}

template <int DIM>
__device__ __forceinline__ void ds_axpy(const dsf* x, dsf h, const dsf* k, dsf* y) {
#pragma unroll
  for (int d = 0; d < DIM; ++d) y[d] = ds_add(x[d], ds_mul_u(h, k[d]));
}

template <int KIND, int DIM, typename CT>
__global__ void __launch_bounds__(32) k_advect_ds(AdvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dsf* tab = reinterpret_cast<dsf*>(smem_raw);
  constexpr bool kTable = (KIND == FTLE_FLOW_DOUBLE_GYRE);

  const int64_t count = a.list ? (int64_t)*a.list_count : a.n;
  const int nchunks = (a.nsteps + kAdvChunk - 1) / kAdvChunk;
  DsFlow F;
  if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
    F.c[0] = ds_from_double(kPi * a.p[0]);
  } else {
#pragma unroll
    for (int q = 0; q < 9; ++q) F.c[q] = ds_from_double(a.p[q]);
  }
  const dsf h = ds_from_double(a.h), h2 = ds_from_double(0.5 * a.h), h6 = ds_from_double(a.h / 6.0);
  bool table_valid = false;

  const int lanes = (a.lanes > 0 && a.lanes < (int)blockDim.x) ? a.lanes : (int)blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * lanes; base < count; base += (int64_t)gridDim.x * lanes) {
    const int64_t slot = base + threadIdx.x;
    const bool active = (int)threadIdx.x < lanes && slot < count;
    const int64_t i = active ? (a.list ? (int64_t)a.list[slot] : slot) : 0;
    dsf x[DIM];
    float x0[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      x[d] = ds_from_double(active ? (double)__ldg(reinterpret_cast<const CT*>(a.coords) + d * a.n_mesh + i) : 0.0);
      x0[d] = x[d].h;
    }

    for (int ch = 0; ch < nchunks; ++ch) {
      const int k0 = ch * kAdvChunk;
      const int k1 = min(a.nsteps, k0 + kAdvChunk);
      if constexpr (kTable) {
        if (!(table_valid && nchunks == 1)) {
          __syncthreads();
          for (int m = threadIdx.x; m <= 2 * (k1 - k0); m += blockDim.x)
            tab[m] = ds_from_double(a.p[1] * sin(a.p[2] * (a.t0 + 0.5 * a.h * (double)(2 * k0 + m))));
          __syncthreads();
          table_valid = true;
        }
      }
      if (!active) continue;
      for (int k = k0; k < k1; ++k) {
        const int m = 2 * (k - k0);
        dsf c0 = ds_make(0.f, 0.f), c1 = c0, c2 = c0;
        if constexpr (kTable) {
          c0 = tab[m];
          c1 = tab[m + 1];
          c2 = tab[m + 2];
        }
        dsf k1v[DIM], k2v[DIM], k3v[DIM], k4v[DIM], y[DIM];
        vel_ds<KIND, DIM>(F, x, c0, k1v);
        ds_axpy<DIM>(x, h2, k1v, y);
        vel_ds<KIND, DIM>(F, y, c1, k2v);
        ds_axpy<DIM>(x, h2, k2v, y);
        vel_ds<KIND, DIM>(F, y, c1, k3v);
        ds_axpy<DIM>(x, h, k3v, y);
        vel_ds<KIND, DIM>(F, y, c2, k4v);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          const dsf s23 = ds_add(k2v[d], k3v[d]);
          const dsf s = ds_add(ds_add(k1v[d], k4v[d]), ds_make(2.0f * s23.h, 2.0f * s23.l));
          x[d] = ds_add(x[d], ds_mul_u(h6, s));
        }
      }
    }
    if (active) {
      float2* o = reinterpret_cast<float2*>(a.out);
      float ph[DIM], pl[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        o[d * a.n_mesh + i] = make_float2(x[d].h, x[d].l);
        ph[d] = x[d].h;
        pl[d] = x[d].l;
      }
      if (a.rec) store_record<DIM>(a.rec, i, x0, ph, pl);
    }
  }
}

// Double gyre in 2D with two lanes per node: lane p = 0 carries x and evaluates sin/cos(pi f),
// lane p = 1 carries y and evaluates sin/cos(pi y).  Both lanes run one instruction stream: the
// argument is f = (a_p x + b_p) x with (a_p, b_p) = (a, 1 - 2a) for p = 0 and (0, 1) for p = 1,
// so lane 1's argument is y and its slope is 1.  Each lane then needs only the partner's cosine
// and slope (four floats by shuffle):
//   u = -pi A sin(pi f) cos(pi y),  v = pi A sin(pi y) cos(pi f) f_x,
// and updates its own coordinate.  The node's two float-float chains run on two lanes instead of
// interleaving in one, which halves the instructions a lane issues per stage; the arithmetic is
// the single-lane kernel's up to the order of the velocity product and of the final sum.
struct DsPairConst {
  dsf piA;              // -pi A on lane 0, pi A on lane 1
  dsf h, h2, h6, third;
  unsigned int mask;    // the two lanes of this pair
  int p;
};

// whole_warp: every lane of the warp reaches each shuffle together (the single-problem kernel);
// otherwise the shuffles name only the pair's two lanes.
__device__ __forceinline__ DsPairConst ds_pair_const(const AdvArgs& a, bool whole_warp) {
  DsPairConst K;
  K.p = threadIdx.x & 1;
  K.mask = whole_warp ? 0xffffffffu : 3u << (threadIdx.x & 30);
  K.piA = ds_from_double((K.p ? kPi : -kPi) * a.p[0]);
  K.h = ds_from_double(a.h);
  K.h2 = ds_from_double(0.5 * a.h);
  K.h6 = ds_from_double(a.h / 6.0);
  K.third = ds_from_double(1.0 / 3.0);
  return K;
}

// hc times this lane's velocity component at y, with a(t) = ca: the scale (a stage's step
// fraction times -pi A or pi A times the partner's slope) is formed while the sine and cosine
// evaluate, so two products follow them on the dependency chain.
__device__ __forceinline__ dsf ds_pair_dg_vel(const DsPairConst& K, const dsf& y, const dsf& ca, const dsf& hc) {
  const dsf ap = K.p ? ds_make(0.f, 0.f) : ca;
  const dsf bp = K.p ? ds_make(1.0f, 0.0f) : ds_add_f(ds_make(-2.0f * ca.h, -2.0f * ca.l), 1.0f);
  const dsf t1 = ds_mul_u(ap, y);
  const dsf f = ds_mul(ds_add_u(t1, bp), y);  // normalized: its high part is reduced by rint
  const dsf fx = ds_add(ds_make(2.0f * t1.h, 2.0f * t1.l), bp);
  const dsf fq = ds_make(__shfl_xor_sync(K.mask, fx.h, 1), __shfl_xor_sync(K.mask, fx.l, 1));
  const dsf g = ds_make(K.p ? fq.h : 1.0f, K.p ? fq.l : 0.0f);
  const dsf scale = ds_mul(ds_mul(K.piA, g), hc);
  dsf sn, cs;
  ds_sincospi(f, sn, cs);
  const dsf cq = ds_make(__shfl_xor_sync(K.mask, cs.h, 1), __shfl_xor_sync(K.mask, cs.l, 1));
  return ds_mul_u(ds_mul_u(sn, cq), scale);
}

// One RK4 step of this lane's coordinate, with a(t) at the step's start, middle and end:
// d1 = h/2 k1, d2 = h/2 k2, d3 = h k3, e4 = h/6 k4, and x + (d1 + 2 d2 + d3) / 3 + e4.
__device__ __forceinline__ dsf ds_pair_dg_step(const DsPairConst& K, const dsf& x, const dsf& c0, const dsf& c1,
                                               const dsf& c2) {
  const dsf d1 = ds_pair_dg_vel(K, x, c0, K.h2);
  const dsf d2 = ds_pair_dg_vel(K, ds_add_u(x, d1), c1, K.h2);
  const dsf d3 = ds_pair_dg_vel(K, ds_add_u(x, d2), c1, K.h);
  const dsf e4 = ds_pair_dg_vel(K, ds_add_u(x, d3), c2, K.h6);
  const dsf sum = ds_add(ds_add(d1, d3), ds_make(2.0f * d2.h, 2.0f * d2.l));
  return ds_add(x, ds_add(ds_mul(sum, K.third), e4));
}

// Lane 0 of a pair writes the node's gradient record (both coordinates, from the partner).
__device__ __forceinline__ void ds_pair_store(const AdvArgs& a, const DsPairConst& K, int64_t i, bool active, float x0,
                                              const dsf& x) {
  const float q0 = __shfl_xor_sync(K.mask, x0, 1);
  const float qh = __shfl_xor_sync(K.mask, x.h, 1), ql = __shfl_xor_sync(K.mask, x.l, 1);
  if (!active) return;
  reinterpret_cast<float2*>(a.out)[K.p * a.n_mesh + i] = make_float2(x.h, x.l);
  if (a.rec && K.p == 0) {
    const float xs[2] = {x0, q0}, ph[2] = {x.h, qh}, pl[2] = {x.l, ql};
    store_record<2>(a.rec, i, xs, ph, pl);
  }
}

template <typename CT>
__global__ void __launch_bounds__(32) k_advect_ds_dg_pair(AdvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dsf* tab = reinterpret_cast<dsf*>(smem_raw);
  const int64_t count = a.list ? (int64_t)*a.list_count : a.n;
  const int nchunks = (a.nsteps + kAdvChunk - 1) / kAdvChunk;
  const DsPairConst K = ds_pair_const(a, true);
  bool table_valid = false;

  const int lanes = (a.lanes > 0 && a.lanes < (int)blockDim.x) ? max(2, a.lanes & ~1) : (int)blockDim.x;
  const int per_block = lanes / 2;
  for (int64_t base = (int64_t)blockIdx.x * per_block; base < count; base += (int64_t)gridDim.x * per_block) {
    const int64_t slot = base + (threadIdx.x >> 1);
    // both lanes of a pair are active or idle together; idle pairs integrate a dummy node
    const bool active = (int)threadIdx.x < lanes && slot < count;
    const int64_t i = active ? (a.list ? (int64_t)a.list[slot] : slot) : 0;
    dsf x = ds_from_double(active ? (double)__ldg(reinterpret_cast<const CT*>(a.coords) + K.p * a.n_mesh + i) : 0.0);
    const float x0 = x.h;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int k0 = ch * kAdvChunk;
      const int k1 = min(a.nsteps, k0 + kAdvChunk);
      if (!(table_valid && nchunks == 1)) {
        __syncthreads();
        for (int m = threadIdx.x; m <= 2 * (k1 - k0); m += blockDim.x)
          tab[m] = ds_from_double(a.p[1] * sin(a.p[2] * (a.t0 + 0.5 * a.h * (double)(2 * k0 + m))));
        __syncthreads();
        table_valid = true;
      }
      for (int k = k0; k < k1; ++k) {
        const int m = 2 * (k - k0);
        x = ds_pair_dg_step(K, x, tab[m], tab[m + 1], tab[m + 2]);
      }
    }
    ds_pair_store(a, K, i, active, x0, x);
  }
}

// ABC flow with three lanes per node: lane d carries coordinate x_d and evaluates sin and cos
// of it, and takes from its group the two values its velocity component needs,
//   u_d = P_d sin x_{d+2} + Q_d cos x_{d+1}   (indices mod 3; (P, Q) = (A, C), (B, A), (C, B)),
// four floats by shuffle.  A stage's step fraction is folded into (P, Q).  The node's three
// float-float sines run on three lanes instead of interleaving in one, which cuts the chain a
// lane issues per stage about threefold.  Ten nodes share a warp; lanes 30 and 31 integrate a
// dummy group.
struct DsTriConst {
  dsf ph2, qh2, ph, qh, ph6, qh6;  // P and Q times h/2, h, h/6
  dsf third;
  int d, src_s, src_c;             // this lane's coordinate; lanes holding sin x_{d+2}, cos x_{d+1}
};

__device__ __forceinline__ DsTriConst ds_tri_const(const AdvArgs& a) {
  DsTriConst K;
  const int lane = threadIdx.x & 31, g = lane / 3;
  K.d = lane - 3 * g;
  K.src_s = 3 * g + (K.d + 2) % 3;  // lanes 30, 31 read lanes 32, 33, that is 0, 1 (shuffles wrap)
  K.src_c = 3 * g + (K.d + 1) % 3;
  const double P = a.p[K.d], Q = a.p[(K.d + 2) % 3];
  K.ph2 = ds_from_double(P * 0.5 * a.h);
  K.qh2 = ds_from_double(Q * 0.5 * a.h);
  K.ph = ds_from_double(P * a.h);
  K.qh = ds_from_double(Q * a.h);
  K.ph6 = ds_from_double(P * a.h / 6.0);
  K.qh6 = ds_from_double(Q * a.h / 6.0);
  K.third = ds_from_double(1.0 / 3.0);
  return K;
}

// This lane's velocity component at y (its own coordinate of the stage point) times a step
// fraction, given as (P, Q) already scaled.
__device__ __forceinline__ dsf ds_tri_abc_vel(const DsTriConst& K, const dsf& y, const dsf& p, const dsf& q) {
  dsf sn, cs;
  ds_sincos(y, sn, cs);
  const dsf so = ds_make(__shfl_sync(0xffffffffu, sn.h, K.src_s), __shfl_sync(0xffffffffu, sn.l, K.src_s));
  const dsf co = ds_make(__shfl_sync(0xffffffffu, cs.h, K.src_c), __shfl_sync(0xffffffffu, cs.l, K.src_c));
  return ds_add(ds_mul_u(p, so), ds_mul_u(q, co));
}

// d1 = h/2 k1, d2 = h/2 k2, d3 = h k3, e4 = h/6 k4, and x + (d1 + 2 d2 + d3) / 3 + e4.
__device__ __forceinline__ dsf ds_tri_abc_step(const DsTriConst& K, const dsf& x) {
  const dsf d1 = ds_tri_abc_vel(K, x, K.ph2, K.qh2);
  const dsf d2 = ds_tri_abc_vel(K, ds_add_u(x, d1), K.ph2, K.qh2);
  const dsf d3 = ds_tri_abc_vel(K, ds_add_u(x, d2), K.ph, K.qh);
  const dsf e4 = ds_tri_abc_vel(K, ds_add_u(x, d3), K.ph6, K.qh6);
  const dsf sum = ds_add(ds_add(d1, d3), ds_make(2.0f * d2.h, 2.0f * d2.l));
  return ds_add(x, ds_add(ds_mul(sum, K.third), e4));
}

template <typename CT>
__global__ void __launch_bounds__(32) k_advect_ds_abc_tri(AdvArgs a) {
  const int64_t count = a.list ? (int64_t)*a.list_count : a.n;
  const DsTriConst K = ds_tri_const(a);
  const int g = (int)(threadIdx.x & 31) / 3;
  // a.lanes (when set) caps the lanes of a block, as for the one-lane kernel: lanes / 3 nodes
  const int cap = (a.lanes > 0 && a.lanes < (int)blockDim.x) ? a.lanes : (int)blockDim.x;
  const int per_block = max(1, min(10, cap / 3));
  for (int64_t base = (int64_t)blockIdx.x * per_block; base < count; base += (int64_t)gridDim.x * per_block) {
    const int64_t slot = base + g;
    const bool active = g < per_block && slot < count;
    const int64_t i = active ? (a.list ? (int64_t)a.list[slot] : slot) : 0;
    dsf x = ds_from_double(active ? (double)__ldg(reinterpret_cast<const CT*>(a.coords) + K.d * a.n_mesh + i) : 0.0);
    const float x0 = x.h;
    for (int k = 0; k < a.nsteps; ++k) x = ds_tri_abc_step(K, x);
    // lane d = 0 of a group gathers the node's record from its two partners
    const int lane = threadIdx.x & 31;
    const float q0a = __shfl_sync(0xffffffffu, x0, lane + 1), q0b = __shfl_sync(0xffffffffu, x0, lane + 2);
    const float qha = __shfl_sync(0xffffffffu, x.h, lane + 1), qhb = __shfl_sync(0xffffffffu, x.h, lane + 2);
    const float qla = __shfl_sync(0xffffffffu, x.l, lane + 1), qlb = __shfl_sync(0xffffffffu, x.l, lane + 2);
    if (!active) continue;
    reinterpret_cast<float2*>(a.out)[K.d * a.n_mesh + i] = make_float2(x.h, x.l);
    if (a.rec && K.d == 0) {
      const float xs[3] = {x0, q0a, q0b}, ph[3] = {x.h, qha, qhb}, pl[3] = {x.l, qla, qlb};
      store_record<3>(a.rec, i, xs, ph, pl);
    }
  }
}

// ------------------------------------------------------- run-parallel re-advection (3D ABC)
//
// One warp per node: lane 3j + d integrates coordinate d over run j of kAbcRuns runs of
// L = ceil(nsteps / kAbcRuns) steps, with the three-lane float-float step above (lanes 30 and 31
// integrate a dummy group).  The runs start from boundary states that lane 0 first computes with
// the compensated float step (the main advection's, stage one carried where the host bounds the
// angles; one lane, short dependent chains), each run carries its RK4 tangent in float, and the
// runs are joined as the 2D gyre's are (below): delta_0 = 0, delta_{j+1} = J_j delta_j + (F_j -
// x_{j+1}), x(T) = F_last + J_last delta_last.  At 256^3 (803 nodes, 500 steps) the boundary pass
// takes ~0.07 ms and the runs ~0.06 ms, against 0.36 ms for all 500 steps on one lane group.
// Lane d holds row d of its run's tangent.  The ABC Jacobian has a zero diagonal:
// row d is (d u_d / d x_{d+1}, d u_d / d x_{d+2}) = (-Q_d sin x_{d+1}, P_d cos x_{d+2}) at the
// columns d + 1 and d + 2, so a stage's tangent row takes the sine and cosine from the two partner
// lanes and their rows of the stage matrix, all by shuffle.
constexpr int kAbcRunWarps = 4;  // nodes per block

// This lane's velocity component at y times a step fraction (as ds_tri_abc_vel), and this lane's
// row of J(y) M for the stage matrix M whose rows the lanes hold (Pf, Qf: P_d, Q_d).
__device__ __forceinline__ dsf ds_tri_abc_vel_tan(const DsTriConst& K, const dsf& y, const dsf& p, const dsf& q,
                                                  float Pf, float Qf, const float* M, float* T) {
  dsf sn, cs;
  ds_sincos(y, sn, cs);
  const dsf so = ds_make(__shfl_sync(0xffffffffu, sn.h, K.src_s), __shfl_sync(0xffffffffu, sn.l, K.src_s));
  const dsf co = ds_make(__shfl_sync(0xffffffffu, cs.h, K.src_c), __shfl_sync(0xffffffffu, cs.l, K.src_c));
  const float a1 = -Qf * __shfl_sync(0xffffffffu, sn.h, K.src_c);  // d u_d / d x_{d+1}
  const float a2 = Pf * __shfl_sync(0xffffffffu, cs.h, K.src_s);   // d u_d / d x_{d+2}
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float m1 = __shfl_sync(0xffffffffu, M[c], K.src_c), m2 = __shfl_sync(0xffffffffu, M[c], K.src_s);
    T[c] = fmaf(a1, m1, a2 * m2);
  }
  return ds_add(ds_mul_u(p, so), ds_mul_u(q, co));
}

// ds_tri_abc_step with this lane's tangent row carried along (RK4 of J' = grad(v) J, in float).
__device__ __forceinline__ dsf ds_tri_abc_step_tan(const DsTriConst& K, const dsf& x, float* row, float Pf, float Qf,
                                                   float h) {
  float M[3], T1[3], T2[3], T3[3], T4[3];
  const dsf d1 = ds_tri_abc_vel_tan(K, x, K.ph2, K.qh2, Pf, Qf, row, T1);
#pragma unroll
  for (int c = 0; c < 3; ++c) M[c] = fmaf(0.5f * h, T1[c], row[c]);
  const dsf d2 = ds_tri_abc_vel_tan(K, ds_add_u(x, d1), K.ph2, K.qh2, Pf, Qf, M, T2);
#pragma unroll
  for (int c = 0; c < 3; ++c) M[c] = fmaf(0.5f * h, T2[c], row[c]);
  const dsf d3 = ds_tri_abc_vel_tan(K, ds_add_u(x, d2), K.ph, K.qh, Pf, Qf, M, T3);
#pragma unroll
  for (int c = 0; c < 3; ++c) M[c] = fmaf(h, T3[c], row[c]);
  const dsf e4 = ds_tri_abc_vel_tan(K, ds_add_u(x, d3), K.ph6, K.qh6, Pf, Qf, M, T4);
#pragma unroll
  for (int c = 0; c < 3; ++c) row[c] = fmaf(h * (1.0f / 6.0f), fmaf(2.0f, T2[c] + T3[c], T1[c] + T4[c]), row[c]);
  const dsf sum = ds_add(ds_add(d1, d3), ds_make(2.0f * d2.h, 2.0f * d2.l));
  return ds_add(x, ds_add(ds_mul(sum, K.third), e4));
}

template <typename CT>
__global__ void __launch_bounds__(32 * kAbcRunWarps) k_refine_runs_abc(AdvArgs a) {
  __shared__ float2 s_bnd[kAbcRunWarps][kAbcRuns][3];  // boundary states (hi, lo) of runs 1 ..
  const DsTriConst K = ds_tri_const(a);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int g = lane / 3;  // this lane's run; 10 for the idle lanes 30, 31
  const bool run_lane = g < kAbcRuns;
  const float Pf = (float)a.p[K.d], Qf = (float)a.p[(K.d + 2) % 3], hf = (float)a.h;
  const int L = (a.nsteps + kAbcRuns - 1) / kAbcRuns;
  const int64_t count = (int64_t)*a.list_count;
  for (int64_t slot = (int64_t)blockIdx.x * kAbcRunWarps + wib; slot < count;
       slot += (int64_t)gridDim.x * kAbcRunWarps) {  // the same slot on every lane of the warp
    const int64_t i = (int64_t)a.list[slot];
    if (lane == 0) {  // boundary states by the compensated float step
      float xh[3], xl[3];
      double xd[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        xd[q] = load_coord<CT>(a.coords, q * a.n_mesh + i);
        xh[q] = (float)xd[q];
        xl[q] = (float)(xd[q] - (double)xh[q]);
      }
      const Coef c0{0.f, 0.f, 0.f, 0.0};  // the ABC flow is autonomous
      AbcCarry carry;  // the unchecked step carries stage one's pairs, as the main advection does
      int k = 0;
      for (int j = 1; j < kAbcRuns; ++j) {
        const int kend = min(j * L, a.nsteps);
        if (a.rot_safe)
          abc_steps_carried(a, k, kend, xh, xl, carry);
        else
          for (; k < kend; ++k) rk4_step<FTLE_FLOW_ABC, 3, P32C, false>(a, c0, c0, c0, xh, xl, xd);
#pragma unroll
        for (int q = 0; q < 3; ++q) s_bnd[wib][j][q] = make_float2(xh[q], xl[q]);
      }
    }
    __syncwarp();
    const double xd0 = load_coord<CT>(a.coords, K.d * a.n_mesh + i);
    const float x0 = (float)xd0;
    dsf x = ds_from_double(xd0);
    if (run_lane && g > 0) {
      const float2 b = s_bnd[wib][g][K.d];
      x = ds_make(b.x, b.y);
    }
    float row[3] = {K.d == 0 ? 1.0f : 0.0f, K.d == 1 ? 1.0f : 0.0f, K.d == 2 ? 1.0f : 0.0f};
    const int k0 = g * L;
    for (int s = 0; s < L; ++s) {  // the same count on every lane; steps past nsteps are discarded
      float rn[3] = {row[0], row[1], row[2]};
      const dsf xn = ds_tri_abc_step_tan(K, x, rn, Pf, Qf, hf);
      if (run_lane && k0 + s < a.nsteps) {
        x = xn;
        row[0] = rn[0];
        row[1] = rn[1];
        row[2] = rn[2];
      }
    }
    // join: r_j = F_j - x_{j+1} on run j's lanes, delta carried through the runs on every lane
    float r = 0.f;
    if (run_lane && g < kAbcRuns - 1) {
      const float2 b = s_bnd[wib][g + 1][K.d];
      const dsf dr = ds_add(x, ds_neg(ds_make(b.x, b.y)));
      r = dr.h + dr.l;
    }
    float dl[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < kAbcRuns - 1; ++j) {
      float nd[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int src = 3 * j + q;
        const float f0 = __shfl_sync(0xffffffffu, row[0], src), f1 = __shfl_sync(0xffffffffu, row[1], src);
        const float f2 = __shfl_sync(0xffffffffu, row[2], src), rq = __shfl_sync(0xffffffffu, r, src);
        nd[q] = fmaf(f0, dl[0], fmaf(f1, dl[1], fmaf(f2, dl[2], rq)));
      }
      dl[0] = nd[0];
      dl[1] = nd[1];
      dl[2] = nd[2];
    }
    x = ds_add_f(x, fmaf(row[0], dl[0], fmaf(row[1], dl[1], row[2] * dl[2])));  // the last run's lanes
    const float q0a = __shfl_sync(0xffffffffu, x0, lane + 1), q0b = __shfl_sync(0xffffffffu, x0, lane + 2);
    const float qha = __shfl_sync(0xffffffffu, x.h, lane + 1), qhb = __shfl_sync(0xffffffffu, x.h, lane + 2);
    const float qla = __shfl_sync(0xffffffffu, x.l, lane + 1), qlb = __shfl_sync(0xffffffffu, x.l, lane + 2);
    if (g == kAbcRuns - 1) {
      reinterpret_cast<float2*>(a.out)[K.d * a.n_mesh + i] = make_float2(x.h, x.l);
      if (a.rec && K.d == 0) {
        const float xs[3] = {x0, q0a, q0b}, ph[3] = {x.h, qha, qhb}, pl[3] = {x.l, qla, qlb};
        store_record<3>(a.rec, i, xs, ph, pl);
      }
    }
    __syncwarp();  // every lane has read the boundary states before lane 0 writes the next node's
  }
}

int launch_refine_runs_abc(bool coord64, const AdvArgs& args, int grid, cudaStream_t s) {
  if (coord64)
    k_refine_runs_abc<double><<<grid, 32 * kAbcRunWarps, 0, s>>>(args);
  else
    k_refine_runs_abc<float><<<grid, 32 * kAbcRunWarps, 0, s>>>(args);
  FTLE_LAUNCH_CHECK("k_refine_runs_abc launch");
  return FTLE_OK;
}

// ------------------------------------------------------- run-parallel re-advection (2D gyre)
//
// The compensated advection leaves each node's (hi, lo) state at the boundaries of kSegments runs
// of seg_len steps.  Here the runs of a node are integrated side by side in float-float, each
// from its boundary state x_j (run 0 from the exact initial point), and each also carries the
// tangent of the RK4 map over the run, J_j = d(run end)/d(run start), in float.  The boundary
// states are the compensated flowmap's, off the float-float trajectory by delta_j ~ 1e-8, so
// with F_j the float-float end of run j and x_{j+1} the next boundary state,
//   delta_0 = 0,   delta_{j+1} = J_j delta_j + (F_j - x_{j+1}),   x(T) = F_last + J_last delta_last,
// to first order in delta; the second-order term, ~|delta|^2 |d^2 Phi|, is near 1e-15, below the
// float-float accuracy these nodes need.  The chain of dependent steps is one run long instead
// of the whole horizon.  RK4 applied to the variational equation J' = grad(v) J alongside the
// state gives exactly the derivative of the RK4 map.

// a(t_m) = eps sin(omega t_m) at the half steps t_m = t0 + m h/2, m = 0 .. 2 nsteps, float-float
__global__ void k_ds_coef_table(double t0, double h, double eps, double omega, int nsteps, dsf* tab) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m <= 2 * nsteps) tab[m] = ds_from_double(eps * sin(omega * (t0 + 0.5 * h * (double)m)));
}

// ds_pair_dg_vel plus this lane's row of the velocity gradient in float (piA = pi A):
//   lane 0, u = -pi A sin(pi f) cos(pi y):  du/dx = -pi^2 A f_x cos(pi f) cos(pi y),
//                                          du/dy =  pi^2 A sin(pi f) sin(pi y);
//   lane 1, v = pi A cos(pi f) sin(pi y) f_x:  dv/dx = pi A sin(pi y) (2 a cos(pi f) - pi f_x^2 sin(pi f)),
//                                              dv/dy = pi^2 A cos(pi f) cos(pi y) f_x.
__device__ __forceinline__ dsf ds_pair_dg_vel_tan(const DsPairConst& K, const dsf& y, const dsf& ca, const dsf& hc,
                                                  float piA, float& gx, float& gy) {
  const float kPiF = 3.14159265358979323846f;
  const dsf ap = K.p ? ds_make(0.f, 0.f) : ca;
  const dsf bp = K.p ? ds_make(1.0f, 0.0f) : ds_add_f(ds_make(-2.0f * ca.h, -2.0f * ca.l), 1.0f);
  const dsf t1 = ds_mul_u(ap, y);
  const dsf f = ds_mul(ds_add_u(t1, bp), y);
  const dsf fx = ds_add(ds_make(2.0f * t1.h, 2.0f * t1.l), bp);
  const dsf fq = ds_make(__shfl_xor_sync(K.mask, fx.h, 1), __shfl_xor_sync(K.mask, fx.l, 1));
  const dsf g = ds_make(K.p ? fq.h : 1.0f, K.p ? fq.l : 0.0f);
  const dsf scale = ds_mul(ds_mul(K.piA, g), hc);
  dsf sn, cs;
  ds_sincospi(f, sn, cs);
  const dsf cq = ds_make(__shfl_xor_sync(K.mask, cs.h, 1), __shfl_xor_sync(K.mask, cs.l, 1));
  const float sq = __shfl_xor_sync(K.mask, sn.h, 1);
  const float S = sn.h, C = cs.h, Cq = cq.h, fo = fx.h, fp = fq.h;
  const float gx0 = -kPiF * piA * fo * C * Cq, gy0 = kPiF * piA * S * sq;
  const float gx1 = piA * S * fmaf(2.0f * ca.h, Cq, -kPiF * fp * fp * sq), gy1 = kPiF * piA * Cq * C * fp;
  gx = K.p ? gx1 : gx0;
  gy = K.p ? gy1 : gy0;
  return ds_mul_u(ds_mul_u(sn, cq), scale);
}

// This lane's tangent row times the stage gradient: (g . J)_p with J's rows on lanes 0 and 1.
__device__ __forceinline__ float2 ds_pair_tan_row(const DsPairConst& K, float gx, float gy, float2 jr) {
  const float2 jq = make_float2(__shfl_xor_sync(K.mask, jr.x, 1), __shfl_xor_sync(K.mask, jr.y, 1));
  const float2 r0 = K.p ? jq : jr, r1 = K.p ? jr : jq;
  return make_float2(fmaf(gx, r0.x, gy * r1.x), fmaf(gx, r0.y, gy * r1.y));
}

// ds_pair_dg_step with the tangent row jr (row p of J) advanced by the same RK4 step.
__device__ __forceinline__ dsf ds_pair_dg_step_tan(const DsPairConst& K, const dsf& x, float2& jr, const dsf& c0,
                                                   const dsf& c1, const dsf& c2, float piA, float h) {
  float gx, gy;
  const dsf d1 = ds_pair_dg_vel_tan(K, x, c0, K.h2, piA, gx, gy);
  const float2 k1 = ds_pair_tan_row(K, gx, gy, jr);
  const dsf d2 = ds_pair_dg_vel_tan(K, ds_add_u(x, d1), c1, K.h2, piA, gx, gy);
  const float2 k2 = ds_pair_tan_row(K, gx, gy, make_float2(fmaf(0.5f * h, k1.x, jr.x), fmaf(0.5f * h, k1.y, jr.y)));
  const dsf d3 = ds_pair_dg_vel_tan(K, ds_add_u(x, d2), c1, K.h, piA, gx, gy);
  const float2 k3 = ds_pair_tan_row(K, gx, gy, make_float2(fmaf(0.5f * h, k2.x, jr.x), fmaf(0.5f * h, k2.y, jr.y)));
  const dsf e4 = ds_pair_dg_vel_tan(K, ds_add_u(x, d3), c2, K.h6, piA, gx, gy);
  const float2 k4 = ds_pair_tan_row(K, gx, gy, make_float2(fmaf(h, k3.x, jr.x), fmaf(h, k3.y, jr.y)));
  const float h6 = h * (1.0f / 6.0f);
  jr.x = fmaf(h6, fmaf(2.0f, k2.x + k3.x, k1.x + k4.x), jr.x);
  jr.y = fmaf(h6, fmaf(2.0f, k2.y + k3.y, k1.y + k4.y), jr.y);
  const dsf sum = ds_add(ds_add(d1, d3), ds_make(2.0f * d2.h, 2.0f * d2.l));
  return ds_add(x, ds_add(ds_mul(sum, K.third), e4));
}

// The join of a node's runs (lanes grp .. grp + 2 kSegments - 1, K.mask covering them): with x the
// end of this lane's run (component p) and jr its tangent row, r_j = F_j - x_{j+1} (float), then
// delta_{j+1} = J_j delta_j + r_j broadcast from each run's lanes, and the last run's end
// corrected by J_last delta_last; the last run's lanes store the node's state and record.
__device__ __forceinline__ void ds_runs_join_store(const AdvArgs& a, const DsPairConst& K, int grp, int run,
                                                   bool active, int64_t i, float xc, dsf x, float2 jr) {
  float r = 0.f;
  if (run < kSegments - 1) {
    const float2 c = active ? a.seg[(int64_t)run * a.seg_stride + K.p * a.n_mesh + i] : make_float2(0.f, 0.f);
    const dsf dr = ds_add(x, ds_neg(ds_make(c.x, c.y)));
    r = dr.h + dr.l;
  }
  float d0 = 0.f, d1 = 0.f;
#pragma unroll
  for (int j = 0; j < kSegments - 1; ++j) {
    const int l0 = grp + 2 * j, l1 = l0 + 1;
    const float a00 = __shfl_sync(K.mask, jr.x, l0), a01 = __shfl_sync(K.mask, jr.y, l0);
    const float a10 = __shfl_sync(K.mask, jr.x, l1), a11 = __shfl_sync(K.mask, jr.y, l1);
    const float r0 = __shfl_sync(K.mask, r, l0), r1 = __shfl_sync(K.mask, r, l1);
    const float n0 = fmaf(a00, d0, fmaf(a01, d1, r0));
    const float n1 = fmaf(a10, d0, fmaf(a11, d1, r1));
    d0 = n0;
    d1 = n1;
  }
  x = ds_add_f(x, fmaf(jr.x, d0, jr.y * d1));  // meaningful on the last run's lanes
  const float qc = __shfl_xor_sync(K.mask, xc, 1);
  const float qh = __shfl_xor_sync(K.mask, x.h, 1), ql = __shfl_xor_sync(K.mask, x.l, 1);
  if (active && run == kSegments - 1) {
    reinterpret_cast<float2*>(a.out)[K.p * a.n_mesh + i] = make_float2(x.h, x.l);
    if (a.rec && K.p == 0) {
      const float xs[2] = {xc, qc}, ph[2] = {x.h, qh}, pl[2] = {x.l, ql};
      store_record<2>(a.rec, i, xs, ph, pl);
    }
  }
}

// Persistent blocks of 128 threads; a node takes 2 kSegments lanes of one warp: run j on lanes
// 2j (x) and 2j + 1 (y).  `coef` holds the coefficient table (k_ds_coef_table).  Held to eight
// 128-thread blocks per SM (64 registers): 1.017 -> 0.977 ms on the 2D workload's 11,222 nodes,
// against 72 registers and seven blocks.
template <typename CT>
__global__ void __launch_bounds__(128, 8) k_refine_runs_dg(AdvArgs a, const dsf* __restrict__ coef) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dsf* tab = reinterpret_cast<dsf*>(smem_raw);
  for (int m = threadIdx.x; m <= 2 * a.nsteps; m += blockDim.x) tab[m] = coef[m];
  __syncthreads();
  constexpr int kLanes = 2 * kSegments;  // lanes per node
  static_assert(32 % kLanes == 0, "a node's runs fit in one warp");
  const int lane = threadIdx.x & 31;
  const int run = (lane >> 1) & (kSegments - 1);
  const int grp = lane & (32 - kLanes);  // first lane of this node's group
  const DsPairConst K = ds_pair_const(a, true);
  const float piA = (float)(kPi * a.p[0]);
  const float h = (float)a.h;
  const int L = a.seg_len;
  const int64_t count = (int64_t)*a.list_count;
  const int per_block = blockDim.x / kLanes;
  for (int64_t base = (int64_t)blockIdx.x * per_block; base < count; base += (int64_t)gridDim.x * per_block) {
    const int64_t slot = base + (threadIdx.x / kLanes);
    const bool active = slot < count;
    const int64_t i = active ? (int64_t)a.list[slot] : 0;
    const float xc = active ? (float)__ldg(reinterpret_cast<const CT*>(a.coords) + K.p * a.n_mesh + i) : 0.f;
    dsf x;
    if (run == 0) {
      x = ds_from_double(active ? (double)__ldg(reinterpret_cast<const CT*>(a.coords) + K.p * a.n_mesh + i) : 0.0);
    } else {
      const float2 c = active ? a.seg[(int64_t)(run - 1) * a.seg_stride + K.p * a.n_mesh + i] : make_float2(0.f, 0.f);
      x = ds_make(c.x, c.y);
    }
    float2 jr = make_float2(K.p == 0 ? 1.0f : 0.0f, K.p == 0 ? 0.0f : 1.0f);
    const int k0 = run * L;
    for (int s = 0; s < L; ++s) {  // the same count on every lane; steps past nsteps are discarded
      const int k = k0 + s;
      const bool live = k < a.nsteps;
      const int m = live ? 2 * k : 0;
      float2 jn = jr;
      const dsf xn = ds_pair_dg_step_tan(K, x, jn, tab[m], tab[m + 1], tab[m + 2], piA, h);
      if (live) {
        x = xn;
        jr = jn;
      }
    }
    ds_runs_join_store(a, K, grp, run, active, i, xc, x, jr);
  }
}

int launch_refine_runs_dg(bool coord64, const AdvArgs& args, void* coef_ws, int grid, cudaStream_t s) {
  dsf* coef = reinterpret_cast<dsf*>(coef_ws);
  const int entries = 2 * args.nsteps + 1;
  k_ds_coef_table<<<(entries + 255) / 256, 256, 0, s>>>(args.t0, args.h, args.p[1], args.p[2], args.nsteps, coef);
  FTLE_LAUNCH_CHECK("k_ds_coef_table launch");
  const size_t smem = sizeof(dsf) * (size_t)entries;
  if (coord64)
    k_refine_runs_dg<double><<<grid, 128, smem, s>>>(args, coef);
  else
    k_refine_runs_dg<float><<<grid, 128, smem, s>>>(args, coef);
  FTLE_LAUNCH_CHECK("k_refine_runs_dg launch");
  return FTLE_OK;
}

// Batched re-advection: the list holds (instance, node) pairs, so lanes of one warp may belong
// to different instances; each lane forms its own double-gyre coefficient a(t_m) =
// eps sin(omega t_m) in float-float (t_m = t0 + m h/2) instead of reading a shared table.
template <int KIND, int DIM>
__global__ void __launch_bounds__(32) k_batch_advect_ds(const BatchInst* __restrict__ insts, const int2* pairs,
                                                        const unsigned long long* count) {
  const int64_t cnt = (int64_t)*count;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < cnt;
       slot += (int64_t)gridDim.x * blockDim.x) {
    const int2 pr = pairs[slot];
    const AdvArgs a = insts[pr.x].adv;
    const int64_t i = pr.y;
    DsFlow F;
    if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
      F.c[0] = ds_from_double(kPi * a.p[0]);
    } else {
#pragma unroll
      for (int q = 0; q < 9; ++q) F.c[q] = ds_from_double(a.p[q]);
    }
    const dsf h = ds_from_double(a.h), h2 = ds_from_double(0.5 * a.h), h6 = ds_from_double(a.h / 6.0);
    const dsf eps = ds_from_double(a.p[1]), omega = ds_from_double(a.p[2]);
    auto coef = [&](int m) -> dsf {
      if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
        dsf s, c;
        ds_sincos(ds_mul(omega, ds_from_double(a.t0 + 0.5 * a.h * (double)m)), s, c);
        return ds_mul(eps, s);
      } else {
        return ds_make(0.f, 0.f);
      }
    };
    dsf x[DIM];
    float x0[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      x[d] = ds_from_double((double)__ldg(reinterpret_cast<const float*>(a.coords) + d * a.n_mesh + i));
      x0[d] = x[d].h;
    }
    dsf c2 = coef(0);
    for (int k = 0; k < a.nsteps; ++k) {
      const dsf c0 = c2, c1 = coef(2 * k + 1);
      c2 = coef(2 * k + 2);
      dsf k1v[DIM], k2v[DIM], k3v[DIM], k4v[DIM], y[DIM];
      vel_ds<KIND, DIM>(F, x, c0, k1v);
      ds_axpy<DIM>(x, h2, k1v, y);
      vel_ds<KIND, DIM>(F, y, c1, k2v);
      ds_axpy<DIM>(x, h2, k2v, y);
      vel_ds<KIND, DIM>(F, y, c1, k3v);
      ds_axpy<DIM>(x, h, k3v, y);
      vel_ds<KIND, DIM>(F, y, c2, k4v);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const dsf s23 = ds_add(k2v[d], k3v[d]);
        const dsf s = ds_add(ds_add(k1v[d], k4v[d]), ds_make(2.0f * s23.h, 2.0f * s23.l));
        x[d] = ds_add(x[d], ds_mul_u(h6, s));
      }
    }
    float2* o = reinterpret_cast<float2*>(a.out);
    float ph[DIM], pl[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      o[d * a.n_mesh + i] = make_float2(x[d].h, x[d].l);
      ph[d] = x[d].h;
      pl[d] = x[d].l;
    }
    if (a.rec) store_record<DIM>(a.rec, i, x0, ph, pl);
  }
}

// Batched run-parallel re-advection (2D double gyre, compensated flowmaps with run-boundary
// states): a half-warp per (instance, node) pair, run j on its lanes 2j and 2j + 1.  The two
// halves of a warp may belong to instances with different steps, so every shuffle names only its
// half.  Each run forms its time coefficients a(t) = eps sin(omega t) by turning
// (sin, cos)(omega t) from its own first half step through omega h/2 per half step.
__global__ void __launch_bounds__(128) k_batch_refine_runs_dg(const BatchInst* __restrict__ insts, const int2* pairs,
                                                              const unsigned long long* count) {
  const int lane = threadIdx.x & 31;
  const int run = (lane >> 1) & (kSegments - 1);
  const int grp = lane & 16;
  const int64_t cnt = (int64_t)*count;
  const int64_t stride = (int64_t)gridDim.x * (blockDim.x >> 4);
  for (int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> 4) + (threadIdx.x >> 4); slot < cnt; slot += stride) {
    const int2 pr = pairs[slot];
    const AdvArgs& a = insts[pr.x].adv;
    const int64_t i = pr.y;
    DsPairConst K = ds_pair_const(a, false);
    K.mask = 0xFFFFu << grp;
    const float piA = (float)(kPi * a.p[0]);
    const float h = (float)a.h;
    const int L = a.seg_len;
    const float xc = __ldg(reinterpret_cast<const float*>(a.coords) + K.p * a.n_mesh + i);
    dsf x;
    if (run == 0) {
      x = ds_from_double((double)xc);
    } else {
      const float2 c = a.seg[(int64_t)(run - 1) * a.seg_stride + K.p * a.n_mesh + i];
      x = ds_make(c.x, c.y);
    }
    const dsf eps = ds_from_double(a.p[1]);
    const dsf rs = ds_from_double(sin(0.5 * a.p[2] * a.h)), rc = ds_from_double(cos(0.5 * a.p[2] * a.h));
    const double t_start = a.t0 + a.h * (double)(run * L);
    dsf sw = ds_from_double(sin(a.p[2] * t_start)), cw = ds_from_double(cos(a.p[2] * t_start));
    auto advance = [&]() {
      const dsf s2 = ds_add(ds_mul(sw, rc), ds_mul(cw, rs));
      cw = ds_add(ds_mul(cw, rc), ds_neg(ds_mul(sw, rs)));
      sw = s2;
    };
    float2 jr = make_float2(K.p == 0 ? 1.0f : 0.0f, K.p == 0 ? 0.0f : 1.0f);
    dsf c2 = ds_mul(eps, sw);
    for (int s = 0; s < L; ++s) {  // every lane of the half-warp runs L steps; past nsteps discarded
      const bool live = run * L + s < a.nsteps;
      const dsf c0 = c2;
      advance();
      const dsf c1 = ds_mul(eps, sw);
      advance();
      c2 = ds_mul(eps, sw);
      float2 jn = jr;
      const dsf xn = ds_pair_dg_step_tan(K, x, jn, c0, c1, c2, piA, h);
      if (live) {
        x = xn;
        jr = jn;
      }
    }
    ds_runs_join_store(a, K, grp, run, true, i, xc, x, jr);
  }
}

int launch_batch_refine_runs_dg(const BatchInst* insts, const int2* pairs, const unsigned long long* count, int grid,
                                cudaStream_t s) {
  k_batch_refine_runs_dg<<<grid, 128, 0, s>>>(insts, pairs, count);
  FTLE_LAUNCH_CHECK("k_batch_refine_runs_dg launch");
  return FTLE_OK;
}

int launch_batch_advect_ds(int kind, int dim, const BatchInst* insts, const int2* pairs,
                           const unsigned long long* count, int grid, int block, cudaStream_t s) {
  if (kind == FTLE_FLOW_DOUBLE_GYRE && dim == 2) k_batch_advect_ds<FTLE_FLOW_DOUBLE_GYRE, 2><<<grid, block, 0, s>>>(insts, pairs, count);
  else if (kind == FTLE_FLOW_ABC && dim == 3) k_batch_advect_ds<FTLE_FLOW_ABC, 3><<<grid, block, 0, s>>>(insts, pairs, count);
  else if (kind == FTLE_FLOW_LINEAR && dim == 2) k_batch_advect_ds<FTLE_FLOW_LINEAR, 2><<<grid, block, 0, s>>>(insts, pairs, count);
  else if (kind == FTLE_FLOW_LINEAR && dim == 3) k_batch_advect_ds<FTLE_FLOW_LINEAR, 3><<<grid, block, 0, s>>>(insts, pairs, count);
  else if (kind == FTLE_FLOW_SADDLE && dim == 2) k_batch_advect_ds<FTLE_FLOW_SADDLE, 2><<<grid, block, 0, s>>>(insts, pairs, count);
  else if (kind == FTLE_FLOW_SADDLE && dim == 3) k_batch_advect_ds<FTLE_FLOW_SADDLE, 3><<<grid, block, 0, s>>>(insts, pairs, count);
  else return fail(FTLE_EUNSUPPORTED, "batched float-float advection: flow %d in %dD", kind, dim);
  FTLE_LAUNCH_CHECK("k_batch_advect_ds launch");
  return FTLE_OK;
}

template <int KIND, int DIM>
static void ds_dispatch(bool coord64, const AdvArgs& args, int grid, int block, size_t smem, cudaStream_t s) {
  if (coord64)
    k_advect_ds<KIND, DIM, double><<<grid, block, smem, s>>>(args);
  else
    k_advect_ds<KIND, DIM, float><<<grid, block, smem, s>>>(args);
}

int launch_advect_ds(int kind, int dim, bool coord64, const AdvArgs& args, int grid, int block,
                     cudaStream_t stream) {
  const size_t smem = advect_smem_bytes(kind, P32, args.nsteps);  // one float pair per half step
  if (kind == FTLE_FLOW_DOUBLE_GYRE && dim == 2) {
    if (coord64)
      k_advect_ds_dg_pair<double><<<2 * grid, block, smem, stream>>>(args);
    else
      k_advect_ds_dg_pair<float><<<2 * grid, block, smem, stream>>>(args);
  } else if (kind == FTLE_FLOW_ABC && dim == 3) {
    if (coord64)
      k_advect_ds_abc_tri<double><<<3 * grid, block, 0, stream>>>(args);
    else
      k_advect_ds_abc_tri<float><<<3 * grid, block, 0, stream>>>(args);
  }
  else if (kind == FTLE_FLOW_LINEAR && dim == 2) ds_dispatch<FTLE_FLOW_LINEAR, 2>(coord64, args, grid, block, smem, stream);
  else if (kind == FTLE_FLOW_LINEAR && dim == 3) ds_dispatch<FTLE_FLOW_LINEAR, 3>(coord64, args, grid, block, smem, stream);
  else if (kind == FTLE_FLOW_SADDLE && dim == 2) ds_dispatch<FTLE_FLOW_SADDLE, 2>(coord64, args, grid, block, smem, stream);
  else if (kind == FTLE_FLOW_SADDLE && dim == 3) ds_dispatch<FTLE_FLOW_SADDLE, 3>(coord64, args, grid, block, smem, stream);
  else return fail(FTLE_EUNSUPPORTED, "float-float advection: flow %d in %dD", kind, dim);
  FTLE_LAUNCH_CHECK("k_advect_ds launch");
  return FTLE_OK;
}

}  // namespace ftle
