// Per-node bodies of the FTLE core (least-squares gradient, Cauchy-Green, lambda_max, FTLE) in
// float and in double, shared by the single-mesh kernels (gradient.cu) and the batched ones
// (batch.cu).  See gradient.cu for the method and the flagging rules.
#pragma once

#include <math.h>

#include "gradient.cuh"

namespace ftle {

template <typename CT>
__device__ __forceinline__ CT ldc(const void* p, int64_t idx) {
  return __ldg(reinterpret_cast<const CT*>(p) + idx);
}

template <int PL>
__device__ __forceinline__ float2 ld_phi32(const void* phi, int64_t idx) {
  if constexpr (PL == PHI32PAIR) {
    return __ldg(reinterpret_cast<const float2*>(phi) + idx);
  } else {
    return make_float2(__ldg(reinterpret_cast<const float*>(phi) + idx), 0.f);
  }
}

template <int PL>
__device__ __forceinline__ double ld_phi64(const void* phi, int64_t idx) {
  if constexpr (PL == PHI32PAIR) {
    float2 v = __ldg(reinterpret_cast<const float2*>(phi) + idx);
    return (double)v.x + (double)v.y;
  } else if constexpr (PL == PHI32) {
    return (double)__ldg(reinterpret_cast<const float*>(phi) + idx);
  } else {
    return __ldg(reinterpret_cast<const double*>(phi) + idx);
  }
}

// Largest eigenvalue of a symmetric 3x3 matrix [[a00,a01,a02],[.,a11,a12],[.,.,a22]] by the
// trigonometric closed form; r_out gets det(B)/2 with B = (A - q I)/p (r -> -1 when the two
// largest eigenvalues coincide).
template <typename T>
__device__ __forceinline__ T sym3_lmax(T a00, T a01, T a02, T a11, T a12, T a22, T& r_out) {
  const T q = (a00 + a11 + a22) / T(3);
  const T p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const T d0 = a00 - q, d1 = a11 - q, d2 = a22 - q;
  const T p2 = d0 * d0 + d1 * d1 + d2 * d2 + T(2) * p1;
  if (!(p2 > T(0))) {
    r_out = T(1);
    return q;
  }
  const T p = sqrt(p2 / T(6));
  const T det = d0 * (d1 * d2 - a12 * a12) - a01 * (a01 * d2 - a12 * a02) + a02 * (a01 * a12 - d1 * a02);
  T r = det / (T(2) * p * p * p);
  r = r < T(-1) ? T(-1) : (r > T(1) ? T(1) : r);
  r_out = r;
  return q + T(2) * p * cos(acos(r) / T(3));
}

// Float variant of sym3_lmax for the float kernel: constant reciprocals and a reciprocal square
// root instead of divisions, and c = cos(acos(r)/3) as the largest root of 4c^3 - 3c = r (the
// triple-angle identity) by two Newton steps from c0 = 1/2 + sqrt(u/6) g(u), u = 1 + r.  The
// factor g(u) = 1 - 0.16115366 u + 0.05104364 u^2 is a least-squares fit of the exact
// (c - 1/2)/sqrt(u/6) over u in [0, 2] (g(0) = 1 keeps the leading term at the double root), so
// c0 is within 1e-2 and two steps reach 2e-8 in exact arithmetic, below float rounding.  Near
// r = -1 the root is double and the steps slow down; such nodes (1 + r <= kNearDoubleTop) take
// the FP64 path anyway.
__device__ __forceinline__ float sym3_lmax_f32(float a00, float a01, float a02, float a11, float a12, float a22,
                                               float& r_out) {
  const float q = (a00 + a11 + a22) * (1.0f / 3.0f);
  const float p1 = fmaf(a01, a01, fmaf(a02, a02, a12 * a12));
  const float d0 = a00 - q, d1 = a11 - q, d2 = a22 - q;
  const float p2 = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, 2.0f * p1)));
  if (!(p2 > 0.0f)) {
    r_out = 1.0f;
    return q;
  }
  const float pp = p2 * (1.0f / 6.0f);  // p^2
  const float rp = rsqrtf(pp);          // 1 / p
  const float p = pp * rp;
  const float det = d0 * (d1 * d2 - a12 * a12) - a01 * (a01 * d2 - a12 * a02) + a02 * (a01 * a12 - d1 * a02);
  float r = 0.5f * det * (rp * rp * rp);
  r = fminf(fmaxf(r, -1.0f), 1.0f);
  r_out = r;
  const float u = 1.0f + r;
  float c = fmaf(sqrtf(u * (1.0f / 6.0f)), fmaf(u, fmaf(u, 0.05104364f, -0.16115366f), 1.0f), 0.5f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float c2 = c * c;
    const float g = fmaf(c, fmaf(4.0f, c2, -3.0f), -r);
    c -= __fdividef(g, fmaf(12.0f, c2, -3.0f));
  }
  return fmaf(2.0f * p, c, q);
}

// M += dx dx^T (upper triangle), B += dphi dx^T.
template <int DIM>
__device__ __forceinline__ void grad_moments(const float* dx, const float* dp, float* m, float* b) {
  int q = 0;
#pragma unroll
  for (int r = 0; r < DIM; ++r)
#pragma unroll
    for (int c = r; c < DIM; ++c, ++q) m[q] = fmaf(dx[r], dx[c], m[q]);
#pragma unroll
  for (int r = 0; r < DIM; ++r)
#pragma unroll
    for (int c = 0; c < DIM; ++c) b[r * DIM + c] = fmaf(dp[r], dx[c], b[r * DIM + c]);
}

// Float moments of one neighbour j read from the coordinate and flowmap arrays.
template <int DIM, int PL, typename CT>
__device__ __forceinline__ void grad_accumulate(const GradArgs& a, int64_t j, const CT* xi, const float2* pi,
                                                float* m, float* b) {
  const int64_t n = a.n;
  float dx[DIM], dp[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    dx[d] = (float)(ldc<CT>(a.coords, d * n + j) - xi[d]);
    const float2 pj = ld_phi32<PL>(a.phi, d * n + j);
    dp[d] = (pj.x - pi[d].x) + (pj.y - pi[d].y);
  }
  grad_moments<DIM>(dx, dp, m, b);
}

// Float moments of one neighbour j read from its gradient record.
template <int DIM>
__device__ __forceinline__ void grad_accumulate_rec(const float4* rec, int64_t j, const float* xi, const float* hi,
                                                    const float* li, float* m, float* b) {
  float xj[DIM], hj[DIM], lj[DIM], dx[DIM], dp[DIM];
  load_record<DIM>(rec, j, xj, hj, lj);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    dx[d] = xj[d] - xi[d];
    dp[d] = (hj[d] - hi[d]) + (lj[d] - li[d]);
  }
  grad_moments<DIM>(dx, dp, m, b);
}

template <int DIM, int PL, typename CT>
__device__ __forceinline__ void grad_load_self(const GradArgs& a, int64_t i, CT* xi, float2* pi, float* m, float* b) {
  const int64_t n = a.n;
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    xi[d] = ldc<CT>(a.coords, d * n + i);
    pi[d] = ld_phi32<PL>(a.phi, d * n + i);
  }
#pragma unroll
  for (int q = 0; q < DIM * (DIM + 1) / 2; ++q) m[q] = 0.f;
#pragma unroll
  for (int q = 0; q < DIM * DIM; ++q) b[q] = 0.f;
}

// From the float moments of k neighbours: F, C = F^T F, lambda_max, FTLE (NaN when flagged) and
// lambda_max to the outputs; returns whether the node needs the FP64 path.
template <int DIM>
__device__ __forceinline__ bool grad_finish_f32(const GradArgs& a, int64_t i, int k, const float* m, const float* b) {
  bool flag = false;
  float lam = NAN, mu = NAN;
  const float trm = DIM == 2 ? m[0] + m[2] : m[0] + m[3] + m[5];
  if (k < DIM) {
    flag = true;
  } else if constexpr (DIM == 2) {
    const float det = m[0] * m[2] - m[1] * m[1];
    const float tr = m[0] + m[2];
    if (!(det > kCondFlag * 0.25f * tr * tr)) {
      flag = true;
    } else {
      const float inv = 1.0f / det;
      const float F00 = (b[0] * m[2] - b[1] * m[1]) * inv, F01 = (b[1] * m[0] - b[0] * m[1]) * inv;
      const float F10 = (b[2] * m[2] - b[3] * m[1]) * inv, F11 = (b[3] * m[0] - b[2] * m[1]) * inv;
      const float c00 = fmaf(F00, F00, F10 * F10), c11 = fmaf(F01, F01, F11 * F11);
      const float c01 = fmaf(F00, F01, F10 * F11);
      const float hd = 0.5f * (c00 - c11);
      lam = 0.5f * (c00 + c11) + sqrtf(fmaf(hd, hd, c01 * c01));
    }
  } else {
    // m = {m00, m01, m02, m11, m12, m22}
    const float a00 = m[3] * m[5] - m[4] * m[4], a01 = m[2] * m[4] - m[1] * m[5];
    const float a02 = m[1] * m[4] - m[2] * m[3], a11 = m[0] * m[5] - m[2] * m[2];
    const float a12 = m[1] * m[2] - m[0] * m[4], a22 = m[0] * m[3] - m[1] * m[1];
    const float det = m[0] * a00 + m[1] * a01 + m[2] * a02;
    const float tr3 = (m[0] + m[3] + m[5]) * (1.0f / 3.0f);
    if (!(det > kCondFlag * tr3 * tr3 * tr3)) {
      flag = true;
    } else {
      const float inv = __fdividef(1.0f, det);  // det > 0 here; a reciprocal to ~2 ulp
      float F[9];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const float b0 = b[r * 3 + 0], b1 = b[r * 3 + 1], b2 = b[r * 3 + 2];
        F[r * 3 + 0] = (b0 * a00 + b1 * a01 + b2 * a02) * inv;
        F[r * 3 + 1] = (b0 * a01 + b1 * a11 + b2 * a12) * inv;
        F[r * 3 + 2] = (b0 * a02 + b1 * a12 + b2 * a22) * inv;
      }
      float c[6];
      int q = 0;
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = r; s < 3; ++s)
          c[q++] = fmaf(F[r], F[s], fmaf(F[3 + r], F[3 + s], F[6 + r] * F[6 + s]));
      float rr;
      lam = sym3_lmax_f32(c[0], c[1], c[2], c[3], c[4], c[5], rr);
      if (rr <= -1.0f + kNearDoubleTop) flag = true;
    }
  }
  mu = lam - 1.0f;
  // ln(lambda_max) h_i < kappa with h_i = sqrt(tr M / k), compared squared (mu < kMuFloor, where
  // the log could be negative, is flagged anyway)
  const float lg = log1pf(mu);
  const bool sensitive =
      (a.refine_kappa >= 0.f) && !(lg * lg * trm >= a.refine_kappa * a.refine_kappa * (float)k);
  flag = flag || !(mu >= kMuFloor) || sensitive || !(lam == lam);
  const float ftle = flag ? NAN : lg * a.inv_2absT32;
  reinterpret_cast<float*>(a.ftle_out)[i] = ftle;
  if (a.lam_out) a.lam_out[i] = (double)(flag ? NAN : lam);
  return flag;
}

// One node of the float kernel over its CSR row.
template <int DIM, int PL, typename CT>
__device__ __forceinline__ bool grad_node_f32(const GradArgs& a, int64_t i) {
  const int rs = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
  CT xi[DIM];
  float2 pi[DIM];
  float m[DIM * (DIM + 1) / 2], b[DIM * DIM];
  grad_load_self<DIM, PL, CT>(a, i, xi, pi, m, b);
  for (int e = rs; e < re; ++e) grad_accumulate<DIM, PL, CT>(a, __ldg(a.col_idx + e), xi, pi, m, b);
  return grad_finish_f32<DIM>(a, i, re - rs, m, b);
}

// One node over the fixed-width neighbour list of the paper's decoupled layout (Section 2.2):
// W slots stored slot-major (ell[s * n + i]), -1 marking an absent neighbour.  All W indices are
// independent coalesced loads, and the unrolled gathers can all be in flight at once.
template <int DIM, int PL, typename CT, int W>
__device__ __forceinline__ bool grad_node_f32_ell(const GradArgs& a, int64_t i) {
  const int64_t n = a.n;
  int js[W];
#pragma unroll
  for (int s = 0; s < W; ++s) js[s] = __ldg(a.ell + (int64_t)s * n + i);
  CT xi[DIM];
  float2 pi[DIM];
  float m[DIM * (DIM + 1) / 2], b[DIM * DIM];
  grad_load_self<DIM, PL, CT>(a, i, xi, pi, m, b);
  int k = 0;
#pragma unroll
  for (int s = 0; s < W; ++s) {
    if (js[s] >= 0) {
      grad_accumulate<DIM, PL, CT>(a, js[s], xi, pi, m, b);
      ++k;
    }
  }
  return grad_finish_f32<DIM>(a, i, k, m, b);
}

// Record-reading variants (compensated flowmaps with float coordinates): a neighbour is one
// address and two 16-byte loads instead of 2 * DIM scattered loads.
template <int DIM>
__device__ __forceinline__ bool grad_node_f32_rec(const GradArgs& a, int64_t i) {
  const int rs = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
  float xi[DIM], hi[DIM], li[DIM];
  float m[DIM * (DIM + 1) / 2] = {}, b[DIM * DIM] = {};
  load_record<DIM>(a.rec, i, xi, hi, li);
  for (int e = rs; e < re; ++e) grad_accumulate_rec<DIM>(a.rec, ld_index(a.col_idx + e), xi, hi, li, m, b);
  return grad_finish_f32<DIM>(a, i, re - rs, m, b);
}

// One node over W neighbour indices already in registers (-1: absent).
template <int DIM, int W>
__device__ __forceinline__ bool grad_node_f32_rec_slots(const GradArgs& a, int64_t i, const int* js) {
  float xi[DIM], hi[DIM], li[DIM];
  float m[DIM * (DIM + 1) / 2] = {}, b[DIM * DIM] = {};
  load_record<DIM>(a.rec, i, xi, hi, li);
  int k = 0;
  // an absent neighbour (-1) reads the node's own record: dx = dphi = 0 leaves the sums
  // unchanged exactly, and the loop has no branch
#pragma unroll
  for (int s = 0; s < W; ++s) {
    const bool ok = js[s] >= 0;
    grad_accumulate_rec<DIM>(a.rec, (uint32_t)(ok ? js[s] : (int)i), xi, hi, li, m, b);
    k += ok;
  }
  return grad_finish_f32<DIM>(a, i, k, m, b);
}

template <int DIM, int W>
__device__ __forceinline__ bool grad_node_f32_ell_rec(const GradArgs& a, int64_t i) {
  const int64_t n = a.n;
  int js[W > 0 ? W : 1];
  if constexpr (W > 0) {
#pragma unroll
    for (int s = 0; s < W; ++s) js[s] = ld_index(a.ell + (int64_t)s * n + i);
    return grad_node_f32_rec_slots<DIM, W>(a, i, js);
  }
  // a width without its own instantiation: the width read at run time
  float xi[DIM], hi[DIM], li[DIM];
  float m[DIM * (DIM + 1) / 2] = {}, b[DIM * DIM] = {};
  load_record<DIM>(a.rec, i, xi, hi, li);
  int k = 0;
  for (int s = 0; s < a.ell_width; ++s) {
    const int j = ld_index(a.ell + (int64_t)s * n + i);
    if (j >= 0) {
      grad_accumulate_rec<DIM>(a.rec, j, xi, hi, li, m, b);
      ++k;
    }
  }
  return grad_finish_f32<DIM>(a, i, k, m, b);
}

// Implicit neighbours of a lattice node (ftle_stencil): W offsets in ascending node order, which
// is the order of the sorted CSR rows of the same mesh for lattices at least 2 nodes wide.
template <int DIM, int ST>
__device__ __forceinline__ constexpr int stencil_width() {
  return ST == FTLE_STENCIL_AXIS ? 2 * DIM : (ST == FTLE_STENCIL_TRI ? 6 : 14);
}

template <int DIM, int ST>
__device__ __forceinline__ void stencil_offset(int s, int& ox, int& oy, int& oz) {
  if constexpr (DIM == 2 && ST == FTLE_STENCIL_AXIS) {
    constexpr int t[4][2] = {{0, -1}, {-1, 0}, {1, 0}, {0, 1}};
    ox = t[s][0], oy = t[s][1], oz = 0;
  } else if constexpr (DIM == 2) {  // TRI
    constexpr int t[6][2] = {{-1, -1}, {0, -1}, {-1, 0}, {1, 0}, {0, 1}, {1, 1}};
    ox = t[s][0], oy = t[s][1], oz = 0;
  } else if constexpr (ST == FTLE_STENCIL_AXIS) {
    constexpr int t[6][3] = {{0, 0, -1}, {0, -1, 0}, {-1, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    ox = t[s][0], oy = t[s][1], oz = t[s][2];
  } else {  // KUHN
    constexpr int t[14][3] = {{-1, -1, -1}, {0, -1, -1}, {-1, 0, -1}, {0, 0, -1}, {-1, -1, 0},
                              {0, -1, 0},   {-1, 0, 0},  {1, 0, 0},   {0, 1, 0},  {1, 1, 0},
                              {0, 0, 1},    {1, 0, 1},   {0, 1, 1},   {1, 1, 1}};
    ox = t[s][0], oy = t[s][1], oz = t[s][2];
  }
}

// One node over the implicit neighbours of a lattice stencil: no neighbour index is read.  A
// neighbour outside the lattice reads the node itself (dx = dphi = 0 adds exact zeros), as the
// fixed-width list's padding does, so the unrolled loop has no branch and the accumulation order
// over the real neighbours is the sorted CSR row's.
template <int DIM, int ST, bool REC, int PL, typename CT>
__device__ __forceinline__ bool grad_node_f32_stencil(const GradArgs& a, int64_t i) {
  const uint32_t nx = a.grid[0], ny = a.grid[1], nz = a.grid[2];
  const uint32_t u = (uint32_t)i, t = u / nx;
  const uint32_t ix = u - t * nx, iy = DIM == 3 ? t % ny : t, iz = DIM == 3 ? t / ny : 0u;
  const bool xm = ix > 0, xp = ix + 1 < nx, ym = iy > 0, yp = iy + 1 < ny, zm = iz > 0, zp = iz + 1 < nz;
  const int sy = (int)nx, sz = (int)(nx * ny);
  float m[DIM * (DIM + 1) / 2] = {}, b[DIM * DIM] = {};
  float xr[DIM], hr[DIM], lr[DIM];  // record path: the node's coordinates and (hi, lo) flowmap
  CT xc[DIM];
  float2 pc[DIM];
  if constexpr (REC)
    load_record<DIM>(a.rec, i, xr, hr, lr);
  else
    grad_load_self<DIM, PL, CT>(a, i, xc, pc, m, b);
  constexpr int W = stencil_width<DIM, ST>();
  int k = 0;
#pragma unroll
  for (int s = 0; s < W; ++s) {
    int ox, oy, oz;
    stencil_offset<DIM, ST>(s, ox, oy, oz);
    const bool ok = (ox < 0 ? xm : (ox > 0 ? xp : true)) && (oy < 0 ? ym : (oy > 0 ? yp : true)) &&
                    (oz < 0 ? zm : (oz > 0 ? zp : true));
    const int64_t j = ok ? i + (ox + oy * sy + oz * sz) : i;
    if constexpr (REC)
      grad_accumulate_rec<DIM>(a.rec, j, xr, hr, lr, m, b);
    else
      grad_accumulate<DIM, PL, CT>(a, j, xc, pc, m, b);
    k += ok;
  }
  return grad_finish_f32<DIM>(a, i, k, m, b);
}

// Fixed-width list of a width without its own instantiation.
template <int DIM, int PL, typename CT>
__device__ __forceinline__ bool grad_node_f32_ell_any(const GradArgs& a, int64_t i) {
  const int64_t n = a.n;
  CT xi[DIM];
  float2 pi[DIM];
  float m[DIM * (DIM + 1) / 2], b[DIM * DIM];
  grad_load_self<DIM, PL, CT>(a, i, xi, pi, m, b);
  int k = 0;
  for (int s = 0; s < a.ell_width; ++s) {
    const int j = __ldg(a.ell + (int64_t)s * n + i);
    if (j >= 0) {
      grad_accumulate<DIM, PL, CT>(a, j, xi, pi, m, b);
      ++k;
    }
  }
  return grad_finish_f32<DIM>(a, i, k, m, b);
}

// Double moments M = sum dx dx^T (upper triangle), B = sum dphi dx^T of node i over the CSR
// entries e0, e0 + step, ... < e1: the whole row (step 1) or one lane's share of it.
template <int DIM, int PL, typename CT>
__device__ __forceinline__ void grad_moments_f64(const GradArgs& a, int64_t i, int e0, int e1, int step, double* m,
                                                 double* b) {
  const int64_t n = a.n;
  double xi[DIM], pi[DIM], pil[DIM];  // node i: coordinates, flowmap (hi and lo parts of a pair)
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    xi[d] = (double)ldc<CT>(a.coords, d * n + i);
    if constexpr (PL == PHI32PAIR) {
      const float2 pv = __ldg(reinterpret_cast<const float2*>(a.phi) + d * n + i);
      pi[d] = (double)pv.x;
      pil[d] = (double)pv.y;
    } else {
      pi[d] = ld_phi64<PL>(a.phi, d * n + i);
      pil[d] = 0.0;
    }
  }
#pragma unroll
  for (int q = 0; q < DIM * (DIM + 1) / 2; ++q) m[q] = 0.0;
#pragma unroll
  for (int q = 0; q < DIM * DIM; ++q) b[q] = 0.0;
  for (int e = e0; e < e1; e += step) {
    const int j = __ldg(a.col_idx + e);
    double dx[DIM], dp[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      dx[d] = (double)ldc<CT>(a.coords, d * n + j) - xi[d];
      if constexpr (PL == PHI32PAIR) {
        const float2 pj = __ldg(reinterpret_cast<const float2*>(a.phi) + d * n + j);
        dp[d] = ((double)pj.x - pi[d]) + ((double)pj.y - pil[d]);
      } else {
        dp[d] = ld_phi64<PL>(a.phi, d * n + j) - pi[d];
      }
    }
    int q = 0;
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int c = r; c < DIM; ++c, ++q) m[q] = fma(dx[r], dx[c], m[q]);
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int c = 0; c < DIM; ++c) b[r * DIM + c] = fma(dp[r], dx[c], b[r * DIM + c]);
  }
}

// From the double moments of k neighbours: F = B M^-1, mu = lambda_max(F^T F - I), FTLE and
// lambda_max to the outputs; counts and NaNs rank-deficient neighbourhoods.
template <int DIM, typename OT>
__device__ __forceinline__ void grad_finish_f64(const GradArgs& a, int64_t i, int k, const double* m, const double* b) {
  double mu = NAN;
  bool degenerate = (k < DIM);
  if (!degenerate) {
    if constexpr (DIM == 2) {
      const double det = m[0] * m[2] - m[1] * m[1];
      const double tr = m[0] + m[2];
      if (!(det > kRankTol * 0.25 * tr * tr)) {
        degenerate = true;
      } else {
        const double inv = 1.0 / det;
        const double F00 = (b[0] * m[2] - b[1] * m[1]) * inv, F01 = (b[1] * m[0] - b[0] * m[1]) * inv;
        const double F10 = (b[2] * m[2] - b[3] * m[1]) * inv, F11 = (b[3] * m[0] - b[2] * m[1]) * inv;
        const double e00 = fma(F00, F00, fma(F10, F10, -1.0));
        const double e11 = fma(F01, F01, fma(F11, F11, -1.0));
        const double e01 = fma(F00, F01, F10 * F11);
        const double hd = 0.5 * (e00 - e11);
        mu = 0.5 * (e00 + e11) + sqrt(fma(hd, hd, e01 * e01));
      }
    } else {
      const double a00 = m[3] * m[5] - m[4] * m[4], a01 = m[2] * m[4] - m[1] * m[5];
      const double a02 = m[1] * m[4] - m[2] * m[3], a11 = m[0] * m[5] - m[2] * m[2];
      const double a12 = m[1] * m[2] - m[0] * m[4], a22 = m[0] * m[3] - m[1] * m[1];
      const double det = m[0] * a00 + m[1] * a01 + m[2] * a02;
      const double tr3 = (m[0] + m[3] + m[5]) / 3.0;
      if (!(det > kRankTol * tr3 * tr3 * tr3)) {
        degenerate = true;
      } else {
        const double inv = 1.0 / det;
        double F[9];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const double b0 = b[r * 3 + 0], b1 = b[r * 3 + 1], b2 = b[r * 3 + 2];
          F[r * 3 + 0] = (b0 * a00 + b1 * a01 + b2 * a02) * inv;
          F[r * 3 + 1] = (b0 * a01 + b1 * a11 + b2 * a12) * inv;
          F[r * 3 + 2] = (b0 * a02 + b1 * a12 + b2 * a22) * inv;
        }
        double e[6];
        int q = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int s = r; s < 3; ++s)
            e[q++] = fma(F[r], F[s], fma(F[3 + r], F[3 + s], fma(F[6 + r], F[6 + s], r == s ? -1.0 : 0.0)));
        double rr;
        mu = sym3_lmax<double>(e[0], e[1], e[2], e[3], e[4], e[5], rr);
      }
    }
  }
  if (degenerate) atomicAdd(&a.hdr->n_degenerate, 1ULL);
  // mu carries the double precision (lambda_max - 1 without cancellation); for a float output
  // the logarithm of the rounded mu is as good as the double one rounded, at a fraction of the
  // cost of double log1p on GB300
  double lg;
  if constexpr (sizeof(OT) == sizeof(float))
    lg = (double)log1pf((float)mu);
  else
    lg = log1p(mu);
  const double ftle = degenerate ? (double)NAN : lg * a.inv_2absT;
  reinterpret_cast<OT*>(a.ftle_out)[i] = (OT)ftle;
  if (a.lam_out) a.lam_out[i] = degenerate ? (double)NAN : 1.0 + mu;
}

// One node in double over its whole CSR row.
template <int DIM, int PL, typename CT, typename OT>
__device__ __forceinline__ void grad_node_f64(const GradArgs& a, int64_t i) {
  const int rs = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
  double m[DIM * (DIM + 1) / 2], b[DIM * DIM];
  grad_moments_f64<DIM, PL, CT>(a, i, rs, re, 1, m, b);
  grad_finish_f64<DIM, OT>(a, i, re - rs, m, b);
}

// Double work over a list of nodes with L lanes per node.  GB300 runs a warp's double
// instruction for about the same time whatever its active lanes, so the cost is the number of
// warps that carry double work, spread over as many SMs as possible.  A long list therefore runs
// one node per lane (L = 1); a short one (tens of flagged nodes) gives each node up to `lmax`
// lanes (about a row's length), as many as keep the groups within an eighth of the grid's lanes,
// to cut the latency of its row.  The lanes of a group split the node's row, a butterfly over the
// group sums the moments, and the group's first lane finishes the node.  Warps are numbered
// block-fastest, so consecutive warps go to different blocks (and SMs).  moments(slot, sub, L, m, b) fills one lane's share and returns
// the neighbour count; finish(slot, k, m, b) writes the node.
template <int DIM, class Moments, class Finish>
__device__ __forceinline__ void grad_list_f64(int64_t count, int lmax, Moments moments, Finish finish) {
  constexpr int NM = DIM * (DIM + 1) / 2;
  const int64_t threads = (int64_t)gridDim.x * blockDim.x;
  int L = lmax;
  while (L > 1 && count * L * 8 > threads) L >>= 1;
  const int groups_per_warp = 32 / L;
  const int64_t warp = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const int64_t nwarps = threads >> 5;
  const int lane = threadIdx.x & 31, sub = lane & (L - 1);
  for (int64_t w0 = warp * groups_per_warp; w0 < count; w0 += nwarps * groups_per_warp) {
    const int64_t slot = w0 + lane / L;
    const bool active = slot < count;
    double m[NM], b[DIM * DIM];
    int k = 0;
    if (active) {
      k = moments(slot, sub, L, m, b);
    } else {
#pragma unroll
      for (int q = 0; q < NM; ++q) m[q] = 0.0;
#pragma unroll
      for (int q = 0; q < DIM * DIM; ++q) b[q] = 0.0;
    }
    for (int off = L >> 1; off > 0; off >>= 1) {
#pragma unroll
      for (int q = 0; q < NM; ++q) m[q] += __shfl_xor_sync(0xffffffffu, m[q], off);
#pragma unroll
      for (int q = 0; q < DIM * DIM; ++q) b[q] += __shfl_xor_sync(0xffffffffu, b[q], off);
    }
    if (active && sub == 0) finish(slot, k, m, b);
  }
}

// Largest lanes per node of the double list kernels (a 2D triangle row has ~6 entries, a 3D
// tetrahedral row ~14).
template <int DIM>
constexpr int kF64Lanes = DIM == 2 ? 8 : 16;

__device__ __forceinline__ void mark_node(int32_t j, uint32_t* bitmap, int32_t* mark_list,
                                          unsigned long long* counter) {
  const uint32_t bit = 1u << (j & 31);
  const uint32_t old = atomicOr(bitmap + (j >> 5), bit);
  if (!(old & bit)) mark_list[atomicAdd(counter, 1ULL)] = j;
}

}  // namespace ftle
