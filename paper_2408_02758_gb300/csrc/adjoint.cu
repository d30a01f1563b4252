// Reverse-mode derivative of L = sum_i w_i FTLE_i with respect to the double-gyre parameters
// theta = (A, eps, omega) (row: differentiation of the FTLE path).
//
// 1. FTLE-map adjoint (double, per node i): F, C = F^T F, lambda and its unit eigenvector v;
//    with p_i = M_i^-1 v_i and a_i = w_i F_i v_i / (|T| lambda_i), the derivative of L with
//    respect to the flowmap is
//        dL/dphi_j = sum_{i : j in N(i)} ((x_j - x_i) . p_i) a_i  -  (sum_k dx_jk . p_j) a_j,
//    from d lambda = 2 (F v) . (dF v) and dF v = sum_k d(dphi_k) (dx_k . p).  The first sum is a
//    gather over j's own row, which needs a symmetric adjacency (i in N(j) <=> j in N(i)).
// 2. Discrete adjoint of the RK4 steps (float), backward segment by segment: each segment's
//    states are recomputed from its checkpoint with the forward kernel's own step (so they equal
//    the forward states bit for bit) into shared memory, then each step is reversed:
//        kb4 = h/6 l, kb3 = h/3 l, kb2 = h/3 l, kb1 = h/6 l, xb = l
//        stage 4: yb = J(y4)^T kb4, thb += P(y4)^T kb4, xb += yb, kb3 += h yb
//        stage 3: yb = J(y3)^T kb3, thb += P(y3)^T kb3, xb += yb, kb2 += h/2 yb
//        stage 2: yb = J(y2)^T kb2, thb += P(y2)^T kb2, xb += yb, kb1 += h/2 yb
//        stage 1: yb = J(y1)^T kb1, thb += P(y1)^T kb1, xb += yb;   l <- xb
//    with J = du/dx and P = du/dtheta of the double gyre at the stage point and time.
// 3. Parameter terms: float per segment, double across segments; per-block partial sums in a
//    fixed order, then one block sums the partials in order (deterministic).
#include <math.h>
#include <string.h>

#include <type_traits>

#include "advect.cuh"
#include "capi_internal.cuh"
#include "gradient_node.cuh"

namespace ftle {

constexpr int kAdjBlock = 64;

// ------------------------------------------------------------------- 1. FTLE-map adjoint

template <typename CT, int PL>
__global__ void __launch_bounds__(128) k_ftle_adjoint_node(GradArgs g, const float* __restrict__ w,
                                                           double* __restrict__ pa) {
  const int64_t n = g.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double p0 = 0, p1 = 0, a0 = 0, a1 = 0, s = 0;
    const float wi = w[i];
    const int rs = g.row_ptr[i], re = g.row_ptr[i + 1];
    if (wi != 0.f && re - rs >= 2) {
      const double xi0 = (double)ldc<CT>(g.coords, i), xi1 = (double)ldc<CT>(g.coords, n + i);
      const double fi0 = ld_phi64<PL>(g.phi, i), fi1 = ld_phi64<PL>(g.phi, n + i);
      double m0 = 0, m1 = 0, m2 = 0, b00 = 0, b01 = 0, b10 = 0, b11 = 0, sx0 = 0, sx1 = 0;
      for (int e = rs; e < re; ++e) {
        const int j = g.col_idx[e];
        const double dx0 = (double)ldc<CT>(g.coords, j) - xi0, dx1 = (double)ldc<CT>(g.coords, n + j) - xi1;
        const double dp0 = ld_phi64<PL>(g.phi, j) - fi0, dp1 = ld_phi64<PL>(g.phi, n + j) - fi1;
        m0 += dx0 * dx0; m1 += dx0 * dx1; m2 += dx1 * dx1;
        b00 += dp0 * dx0; b01 += dp0 * dx1; b10 += dp1 * dx0; b11 += dp1 * dx1;
        sx0 += dx0; sx1 += dx1;
      }
      const double det = m0 * m2 - m1 * m1;
      const double tr = m0 + m2;
      if (det > kRankTol * 0.25 * tr * tr) {
        const double i00 = m2 / det, i01 = -m1 / det, i11 = m0 / det;  // M^-1
        const double F00 = b00 * i00 + b01 * i01, F01 = b00 * i01 + b01 * i11;
        const double F10 = b10 * i00 + b11 * i01, F11 = b10 * i01 + b11 * i11;
        const double c00 = F00 * F00 + F10 * F10, c01 = F00 * F01 + F10 * F11, c11 = F01 * F01 + F11 * F11;
        const double hd = 0.5 * (c00 - c11);
        const double lam = 0.5 * (c00 + c11) + sqrt(hd * hd + c01 * c01);
        // unit eigenvector of lam: the better conditioned of (c01, lam - c00) and (lam - c11, c01)
        double v0 = c01, v1 = lam - c00;
        const double u0 = lam - c11, u1 = c01;
        if (u0 * u0 + u1 * u1 > v0 * v0 + v1 * v1) { v0 = u0; v1 = u1; }
        const double nv = sqrt(v0 * v0 + v1 * v1);
        if (nv > 0) { v0 /= nv; v1 /= nv; } else { v0 = 1; v1 = 0; }
        const double coef = (double)wi * 2.0 * g.inv_2absT / lam;  // w / (|T| lambda)
        a0 = coef * (F00 * v0 + F01 * v1);
        a1 = coef * (F10 * v0 + F11 * v1);
        p0 = i00 * v0 + i01 * v1;
        p1 = i01 * v0 + i11 * v1;
        s = sx0 * p0 + sx1 * p1;
      }
    }
    pa[i] = p0; pa[n + i] = p1; pa[2 * n + i] = a0; pa[3 * n + i] = a1; pa[4 * n + i] = s;
  }
}

template <typename CT>
__global__ void __launch_bounds__(128) k_ftle_adjoint_gather(GradArgs g, const double* __restrict__ pa,
                                                             float* __restrict__ phibar) {
  const int64_t n = g.n;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double xj0 = (double)ldc<CT>(g.coords, j), xj1 = (double)ldc<CT>(g.coords, n + j);
    double g0 = -pa[4 * n + j] * pa[2 * n + j], g1 = -pa[4 * n + j] * pa[3 * n + j];
    const int rs = g.row_ptr[j], re = g.row_ptr[j + 1];
    for (int e = rs; e < re; ++e) {
      const int i = g.col_idx[e];
      const double c = (xj0 - (double)ldc<CT>(g.coords, i)) * pa[i] + (xj1 - (double)ldc<CT>(g.coords, n + i)) * pa[n + i];
      g0 += c * pa[2 * n + i];
      g1 += c * pa[3 * n + i];
    }
    phibar[j] = (float)g0;
    phibar[n + j] = (float)g1;
  }
}

// ---------------------------------------------------------------- 2. RK4 discrete adjoint

struct DgDer {
  float u0, u1;              // velocity
  float j01, j10, j11;       // du/dx (j00 = -j11: the flow is divergence-free)
  float pA0, pA1;            // du/dA / pi
  float q0, q1;              // du/deps = s q, du/domega = eps t c q
};

// Double-gyre velocity and derivatives at a point with abscissa x, from the slope f_x of the
// stream function's argument and (sin, cos) of pi f and of pi y there; coefficient a = eps s.
// The four products of the sines and cosines are formed once and shared.
__device__ __forceinline__ DgDer dg_derivs_sc(float piA, float a, float fx, float x, float sf, float cf, float sy,
                                              float cy) {
  const float kPiF = 3.14159265358979323846f;
  DgDer d;
  const float scy = sf * cy, ccy = cf * cy, csy = cf * sy, ssy = sf * sy;
  const float t1 = csy * fx;
  const float pi2A = kPiF * piA;
  d.u0 = -piA * scy;
  d.u1 = piA * t1;
  d.j01 = pi2A * ssy;
  d.j10 = piA * fmaf(-kPiF * ssy, fx * fx, csy * 2.0f * a);
  d.j11 = pi2A * (ccy * fx);
  d.pA0 = -scy;
  d.pA1 = t1;
  const float g1 = fmaf(x, x, -2.0f * x), g2 = fmaf(2.0f, x, -2.0f);
  d.q0 = -pi2A * (ccy * g1);
  d.q1 = piA * fmaf(-kPiF * ssy * g1, fx, csy * g2);
  return d;
}

// ... at (x, y) with coefficients a, b = 1 - 2a, evaluating the sines and cosines.
__device__ __forceinline__ DgDer dg_derivs32(float piA, float a, float b, float x, float y) {
  const float f = fmaf(a, x, b) * x;
  float sf, cf, sy, cy;
  fsincospi(f, sf, cf);
  fsincospi(y, sy, cy);
  return dg_derivs_sc(piA, a, fmaf(2.0f * a, x, b), x, sf, cf, sy, cy);
}

// ... at the stage point (xk + dx, yk + dy) of a step whose first stage point is (xk, yk), with
// (sin, cos) of pi f and pi y there turned from stage one's pairs by the small angles, as the
// forward step does (e1 = 2 (xk - 1), dg = (a_s - a_0) xk (xk - 2)).  `mx` collects the larger
// angle; past kRotMax the caller evaluates the stage in full.
__device__ __forceinline__ DgDer dg_derivs32_rot(float piA, float as, float e1, float dg, float dx, float dy,
                                                 float sf0, float cf0, float sy0, float cy0, float xs, float& mx) {
  const float kPiF = 3.14159265358979323846f;
  const float w = fmaf(as, e1 + dx, 1.0f);
  const float tf = kPiF * fmaf(dx, w, dg), ty = kPiF * dy;
  mx = fmaxf(mx, fmaxf(fabsf(tf), fabsf(ty)));
  float2 s, c;  // lanes: pi f, pi y
  rotate_small2(make_float2(sf0, sy0), make_float2(cf0, cy0), make_float2(tf, ty), s, c);
  return dg_derivs_sc(piA, as, fmaf(as, dx, w), xs, s.x, c.x, s.y, c.y);
}

// Segment table per half step: (a, b_l) of the forward kernel, sin(omega t), t cos(omega t).
// The sine and cosine take dg_coef's reduction: u = omega t / pi in double, then sinpi and cospi
// of u - rint(u) in float, so no double transcendental runs (GB300's FP64 rate is low, and every
// block rebuilds the table for every segment).
__device__ __forceinline__ void build_adj_table(const AdvArgs& a, float4* tab, int k0, int k1) {
  const double nu = a.p[2] / kPi;
  for (int m = threadIdx.x; m <= 2 * (k1 - k0); m += blockDim.x) {
    const int mm = 2 * k0 + m;
    const float2 c = dg_coef(a.p[1], nu, a.t0, 0.5 * a.h, mm);
    const double t = a.t0 + 0.5 * a.h * (double)mm;
    const double u = nu * t, k = rint(u);
    float sr, cr;
    sincospif((float)(u - k), &sr, &cr);
    if (((long long)k) & 1) {  // sin, cos(pi (k + r)) = (-1)^k sin, cos(pi r)
      sr = -sr;
      cr = -cr;
    }
    tab[m] = make_float4(c.x, c.y, sr, (float)t * cr);
  }
}

template <int PREC, int OUT>
__global__ void __launch_bounds__(kAdjBlock) k_adjoint_rk4(AdvArgs a, const float* __restrict__ phibar,
                                                           double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ce = a.ckpt_every;
  float4* tab = reinterpret_cast<float4*>(smem_raw);
  float2* states = reinterpret_cast<float2*>(smem_raw + sizeof(float4) * (size_t)(2 * ce + 1));
  __shared__ double red[3][kAdjBlock];

  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < a.n;
  const float piA = (float)(kPi * a.p[0]);
  const float eps = (float)a.p[1];
  float lam0 = active ? phibar[i] : 0.f, lam1 = active ? phibar[a.n_mesh + i] : 0.f;
  // the forward kernel's choice between the checked and the unchecked step (dg_node_safe), so
  // the recomputed states are the forward's
  const bool safe = PREC == P32C && active &&
                    dg_node_safe(a, (double)reinterpret_cast<const float*>(a.coords)[i],
                                 (double)reinterpret_cast<const float*>(a.coords)[a.n_mesh + i]);
  double th0 = 0, th1 = 0, th2 = 0;
  const int nseg = (a.nsteps + ce - 1) / ce;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int k0 = seg * ce, k1 = min(a.nsteps, k0 + ce);
    __syncthreads();
    build_adj_table(a, tab, k0, k1);
    __syncthreads();
    // recompute the segment's states from its checkpoint with the forward step
    float xh[2] = {0.f, 0.f}, xl[2] = {0.f, 0.f};
    double xd[2] = {0.0, 0.0};
    if (active) {
      const char* slot = reinterpret_cast<const char*>(a.ckpt) + (int64_t)seg * a.ckpt_stride_bytes;
      if constexpr (OUT == O32PAIR) {
        const float2* c = reinterpret_cast<const float2*>(slot);
        const float2 c0 = c[i], c1 = c[a.n_mesh + i];
        xh[0] = c0.x; xl[0] = c0.y; xh[1] = c1.x; xl[1] = c1.y;
      } else {
        const float* c = reinterpret_cast<const float*>(slot);
        xh[0] = c[i]; xh[1] = c[a.n_mesh + i];
      }
      auto recompute = [&](auto unchecked) {
        for (int k = k0; k < k1; ++k) {
          states[(k - k0) * blockDim.x + threadIdx.x] = make_float2(xh[0], xh[1]);
          const int m = 2 * (k - k0);
          Coef c0{tab[m].x, fmaf(-2.f, tab[m].x, 1.f), tab[m].y, 0.0};
          Coef c1{tab[m + 1].x, fmaf(-2.f, tab[m + 1].x, 1.f), tab[m + 1].y, 0.0};
          Coef c2{tab[m + 2].x, fmaf(-2.f, tab[m + 2].x, 1.f), tab[m + 2].y, 0.0};
          rk4_step<FTLE_FLOW_DOUBLE_GYRE, 2, PREC, decltype(unchecked)::value>(a, c0, c1, c2, xh, xl, xd);
        }
      };
      if (safe)
        recompute(std::true_type{});
      else
        recompute(std::false_type{});
      // reverse the segment's steps
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
      const float h = a.h32, h2 = a.h2_32, h6 = a.h6_32, h3 = 2.0f * a.h6_32;
      for (int k = k1 - 1; k >= k0; --k) {
        const float2 xk = states[(k - k0) * blockDim.x + threadIdx.x];
        const int m = 2 * (k - k0);
        const float4 t0 = tab[m], t1 = tab[m + 1], t2 = tab[m + 2];
        const float b0 = fmaf(-2.f, t0.x, 1.f), b1 = fmaf(-2.f, t1.x, 1.f), b2 = fmaf(-2.f, t2.x, 1.f);
        // stage points (float); stages two to four turn stage one's sines and cosines
        float sf0, cf0, sy0, cy0;
        fsincospi(fmaf(t0.x, xk.x, b0) * xk.x, sf0, cf0);
        fsincospi(xk.y, sy0, cy0);
        const DgDer d1 = dg_derivs_sc(piA, t0.x, fmaf(2.0f * t0.x, xk.x, b0), xk.x, sf0, cf0, sy0, cy0);
        const float e1 = fmaf(2.0f, xk.x, -2.0f), g0 = xk.x * (xk.x - 2.0f);
        const float dg1 = (t1.x - t0.x) * g0, dg2 = (t2.x - t0.x) * g0;
        float mx = 0.0f;
        const float y2x = fmaf(h2, d1.u0, xk.x), y2y = fmaf(h2, d1.u1, xk.y);
        DgDer d2 = dg_derivs32_rot(piA, t1.x, e1, dg1, y2x - xk.x, y2y - xk.y, sf0, cf0, sy0, cy0, y2x, mx);
        const float y3x = fmaf(h2, d2.u0, xk.x), y3y = fmaf(h2, d2.u1, xk.y);
        DgDer d3 = dg_derivs32_rot(piA, t1.x, e1, dg1, y3x - xk.x, y3y - xk.y, sf0, cf0, sy0, cy0, y3x, mx);
        const float y4x = fmaf(h, d3.u0, xk.x), y4y = fmaf(h, d3.u1, xk.y);
        DgDer d4 = dg_derivs32_rot(piA, t2.x, e1, dg2, y4x - xk.x, y4y - xk.y, sf0, cf0, sy0, cy0, y4x, mx);
        if (!(mx <= kRotMax)) {  // a step too long for the small-angle turns
          d2 = dg_derivs32(piA, t1.x, b1, y2x, y2y);
          const float z3x = fmaf(h2, d2.u0, xk.x), z3y = fmaf(h2, d2.u1, xk.y);
          d3 = dg_derivs32(piA, t1.x, b1, z3x, z3y);
          d4 = dg_derivs32(piA, t2.x, b2, fmaf(h, d3.u0, xk.x), fmaf(h, d3.u1, xk.y));
        }
        // the stage adjoints kb, the accumulated xb and lambda carry (x, y) as paired lanes
        const float2 lam = make_float2(lam0, lam1);
        float2 kb1 = mul2(f2(h6), lam), kb2 = mul2(f2(h3), lam), kb3 = kb2;
        const float2 kb4 = kb1;
        float2 xb = lam;
        auto stage = [&](const DgDer& d, float2 kb, const float4& tc) -> float2 {
          const float2 yb = make_float2(fmaf(-d.j11, kb.x, d.j10 * kb.y), fmaf(d.j01, kb.x, d.j11 * kb.y));
          const float qk = fmaf(d.q0, kb.x, d.q1 * kb.y);
          s0 = fmaf(d.pA0, kb.x, fmaf(d.pA1, kb.y, s0));
          s1 = fmaf(tc.z, qk, s1);
          s2 = fmaf(eps * tc.w, qk, s2);
          return yb;
        };
        float2 yb = stage(d4, kb4, t2);
        xb = add2(xb, yb); kb3 = fma2(f2(h), yb, kb3);
        yb = stage(d3, kb3, t1);
        xb = add2(xb, yb); kb2 = fma2(f2(h2), yb, kb2);
        yb = stage(d2, kb2, t1);
        xb = add2(xb, yb); kb1 = fma2(f2(h2), yb, kb1);
        yb = stage(d1, kb1, t0);
        const float2 ln = add2(xb, yb);
        lam0 = ln.x;
        lam1 = ln.y;
      }
      th0 += kPi * (double)s0;  // the pA terms are du/dA / pi
      th1 += (double)s1;
      th2 += (double)s2;
    }
  }
  // block sum in a fixed order
  red[0][threadIdx.x] = th0;
  red[1][threadIdx.x] = th1;
  red[2][threadIdx.x] = th2;
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) partial[(int64_t)q * gridDim.x + blockIdx.x] = red[q][0];
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  __shared__ double red[3][256];
  for (int q = 0; q < 3; ++q) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(int64_t)q * nb + b];
    red[q][threadIdx.x] = s;
  }
  __syncthreads();
  for (int stride = blockDim.x / 2; stride > 0; stride >>= 1) {
    if ((int)threadIdx.x < stride)
      for (int q = 0; q < 3; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + stride];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) out[q] = red[q][0];
}

}  // namespace ftle

using namespace ftle;

namespace {

struct BwLayout {
  size_t pa = 0, phibar = 0, partial = 0, total = 0;
  int nblocks = 0;
};

BwLayout bw_layout(int64_t n) {
  BwLayout L;
  size_t off = 0;
  L.pa = off;
  off += align256(sizeof(double) * 5 * (size_t)(n > 0 ? n : 1));
  L.phibar = off;
  off += align256(sizeof(float) * 2 * (size_t)(n > 0 ? n : 1));
  L.nblocks = (int)((n + kAdjBlock - 1) / kAdjBlock);
  L.partial = off;
  off += align256(sizeof(double) * 3 * (size_t)(L.nblocks > 0 ? L.nblocks : 1));
  L.total = off;
  return L;
}

template <int PREC, int OUT>
int launch_adjoint_rk4(const AdvArgs& a, const float* phibar, double* partial, int nblocks, size_t smem,
                       cudaStream_t s) {
  if (smem > 48 * 1024)
    FTLE_CUDA_CHECK(cudaFuncSetAttribute(k_adjoint_rk4<PREC, OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
  k_adjoint_rk4<PREC, OUT><<<nblocks, kAdjBlock, smem, s>>>(a, phibar, partial);
  FTLE_LAUNCH_CHECK("k_adjoint_rk4 launch");
  return FTLE_OK;
}

}  // namespace

extern "C" {

size_t ftle_backward_workspace_bytes(int64_t n_nodes, int32_t dim) {
  if (n_nodes < 0 || dim != 2) return 0;
  return bw_layout(n_nodes).total;
}

int ftle_backward(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt, int32_t precision,
                  const void* flowmap, const void* checkpoints, int32_t ckpt_every, const float* dL_dftle,
                  double* dL_dparams, void* workspace, size_t workspace_bytes, const ftle_options* opt,
                  void* stream) {
  PhaseRange range("ftle.backward");
  int rc, nsteps = 0;
  if ((rc = check_mesh(mesh)) || (rc = check_flow(flow, mesh->dim)) || (rc = check_prec(precision)) ||
      (rc = check_time(T, dt, &nsteps)))
    return rc;
  if (mesh->dim != 2 || flow->kind != FTLE_FLOW_DOUBLE_GYRE)
    return fail(FTLE_EUNSUPPORTED, "ftle_backward: the parameter derivative is defined for the 2D double gyre");
  if (precision == FTLE_PREC_FP64) return fail(FTLE_EUNSUPPORTED, "ftle_backward: FP32 or FP32C forward only");
  if (mesh->coord_fp64) return fail(FTLE_EUNSUPPORTED, "ftle_backward: coordinates must be float");
  if (!isfinite(t0)) return fail(FTLE_EINVAL, "t0 must be finite");
  if (ckpt_every < 1 || ckpt_every > 256) return fail(FTLE_EINVAL, "ckpt_every must be in [1, 256]");
  if (!dL_dparams) return fail(FTLE_EINVAL, "dL_dparams is NULL");
  if (mesh->n_nodes > 0 && (!flowmap || !checkpoints || !dL_dftle))
    return fail(FTLE_EINVAL, "flowmap / checkpoints / dL_dftle is NULL");
  const BwLayout W = bw_layout(mesh->n_nodes);
  if ((rc = check_workspace(workspace, workspace_bytes, W.total))) return rc;
  const Launch L = resolve_launch(opt);
  if ((rc = check_launch(L))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (mesh->n_nodes == 0) {
    FTLE_CUDA_CHECK(cudaMemsetAsync(dL_dparams, 0, 3 * sizeof(double), s));
    return FTLE_OK;
  }
  char* w = reinterpret_cast<char*>(workspace);
  double* pa = reinterpret_cast<double*>(w + W.pa);
  float* phibar = reinterpret_cast<float*>(w + W.phibar);
  double* partial = reinterpret_cast<double*>(w + W.partial);
  GradArgs g;
  memset(&g, 0, sizeof g);
  g.n = mesh->n_nodes;
  g.coords = mesh->coords;
  g.row_ptr = mesh->row_ptr;
  g.col_idx = mesh->col_idx;
  g.phi = flowmap;
  g.inv_2absT = 1.0 / (2.0 * fabs(T));
  g.inv_2absT32 = (float)g.inv_2absT;
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  if (precision == FTLE_PREC_FP32C)
    k_ftle_adjoint_node<float, PHI32PAIR><<<sms * 8, 128, 0, s>>>(g, dL_dftle, pa);
  else
    k_ftle_adjoint_node<float, PHI32><<<sms * 8, 128, 0, s>>>(g, dL_dftle, pa);
  FTLE_LAUNCH_CHECK("k_ftle_adjoint_node launch");
  k_ftle_adjoint_gather<float><<<sms * 8, 128, 0, s>>>(g, pa, phibar);
  FTLE_LAUNCH_CHECK("k_ftle_adjoint_gather launch");
  AdvArgs a = make_adv_args(mesh, flow, t0, T, dt, nsteps);
  a.ckpt = const_cast<void*>(checkpoints);
  a.ckpt_every = ckpt_every;
  a.ckpt_stride_bytes = (int64_t)ftle_checkpoint_bytes(mesh->dim, mesh->n_nodes, precision);
  const size_t smem = sizeof(float4) * (size_t)(2 * ckpt_every + 1) + sizeof(float2) * (size_t)ckpt_every * kAdjBlock;
  if (precision == FTLE_PREC_FP32C)
    rc = launch_adjoint_rk4<P32C, O32PAIR>(a, phibar, partial, W.nblocks, smem, s);
  else
    rc = launch_adjoint_rk4<P32, O32>(a, phibar, partial, W.nblocks, smem, s);
  if (rc) return rc;
  k_sum_partials<<<1, 256, 0, s>>>(partial, W.nblocks, dL_dparams);
  FTLE_LAUNCH_CHECK("k_sum_partials launch");
  return FTLE_OK;
}

}  // extern "C"
