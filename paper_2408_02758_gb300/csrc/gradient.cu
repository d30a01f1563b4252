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

// ----------------------------------------------------------------------------- float kernel

template <int DIM, int PL, typename CT>
__global__ void __launch_bounds__(256) k_grad_f32(GradArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t n = a.n;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    bool flag = false;
    if (i < n) {
      const int rs = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
      CT xi[DIM];
      float2 pi[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        xi[d] = ldc<CT>(a.coords, d * n + i);
        pi[d] = ld_phi32<PL>(a.phi, d * n + i);
      }
      constexpr int NM = DIM * (DIM + 1) / 2;
      float m[NM], b[DIM * DIM];
#pragma unroll
      for (int q = 0; q < NM; ++q) m[q] = 0.f;
#pragma unroll
      for (int q = 0; q < DIM * DIM; ++q) b[q] = 0.f;
      for (int e = rs; e < re; ++e) {
        const int j = __ldg(a.col_idx + e);
        float dx[DIM], dp[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
          dx[d] = (float)(ldc<CT>(a.coords, d * n + j) - xi[d]);
          const float2 pj = ld_phi32<PL>(a.phi, d * n + j);
          dp[d] = (pj.x - pi[d].x) + (pj.y - pi[d].y);
        }
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
      float lam = NAN, mu = NAN;
      const float trm = DIM == 2 ? m[0] + m[2] : m[0] + m[3] + m[5];
      if (re - rs < DIM) {
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
          const float inv = 1.0f / det;
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
          lam = sym3_lmax<float>(c[0], c[1], c[2], c[3], c[4], c[5], rr);
          if (rr <= -1.0f + kNearDoubleTop) flag = true;
        }
      }
      mu = lam - 1.0f;
      const float h_i = sqrtf(trm / (float)(re - rs > 0 ? re - rs : 1));
      const bool sensitive = (a.refine_kappa >= 0.f) && !(log1pf(mu) * h_i >= a.refine_kappa);
      flag = flag || !(mu >= kMuFloor) || sensitive || !(lam == lam);
      const float ftle = flag ? NAN : log1pf(mu) * (float)a.inv_2absT;
      reinterpret_cast<float*>(a.ftle_out)[i] = ftle;
      if (a.lam_out) a.lam_out[i] = flag ? NAN : (double)lam;
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

// ----------------------------------------------------------------------------- double kernel

template <int DIM, int PL, typename CT, typename OT>
__global__ void __launch_bounds__(128) k_grad_f64(GradArgs a) {
  const int64_t n = a.n;
  const int64_t count = a.list ? (int64_t)*a.list_count : n;
  for (int64_t slot = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; slot < count;
       slot += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = a.list ? (int64_t)a.list[slot] : slot;
    const int rs = __ldg(a.row_ptr + i), re = __ldg(a.row_ptr + i + 1);
    double xi[DIM], pi[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      xi[d] = (double)ldc<CT>(a.coords, d * n + i);
      pi[d] = 0.0;
    }
    constexpr int NM = DIM * (DIM + 1) / 2;
    double m[NM], b[DIM * DIM];
#pragma unroll
    for (int q = 0; q < NM; ++q) m[q] = 0.0;
#pragma unroll
    for (int q = 0; q < DIM * DIM; ++q) b[q] = 0.0;
    for (int e = rs; e < re; ++e) {
      const int j = __ldg(a.col_idx + e);
      double dx[DIM], dp[DIM];
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        dx[d] = (double)ldc<CT>(a.coords, d * n + j) - xi[d];
        if constexpr (PL == PHI32PAIR) {
          const float2 pj = __ldg(reinterpret_cast<const float2*>(a.phi) + d * n + j);
          const float2 pv = __ldg(reinterpret_cast<const float2*>(a.phi) + d * n + i);
          dp[d] = ((double)pj.x - (double)pv.x) + ((double)pj.y - (double)pv.y);
        } else {
          dp[d] = ld_phi64<PL>(a.phi, d * n + j) - ld_phi64<PL>(a.phi, d * n + i);
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
    (void)pi;
    double mu = NAN;
    bool degenerate = (re - rs < DIM);
    if (!degenerate) {
      if constexpr (DIM == 2) {
        const double det = m[0] * m[2] - m[1] * m[1];
        const double tr = m[0] + m[2];
        if (!(det > kRankTol * 0.25 * tr * tr)) {
          degenerate = true;
        } else {
          const double F00 = (b[0] * m[2] - b[1] * m[1]) / det, F01 = (b[1] * m[0] - b[0] * m[1]) / det;
          const double F10 = (b[2] * m[2] - b[3] * m[1]) / det, F11 = (b[3] * m[0] - b[2] * m[1]) / det;
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
          double F[9];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            const double b0 = b[r * 3 + 0], b1 = b[r * 3 + 1], b2 = b[r * 3 + 2];
            F[r * 3 + 0] = (b0 * a00 + b1 * a01 + b2 * a02) / det;
            F[r * 3 + 1] = (b0 * a01 + b1 * a11 + b2 * a12) / det;
            F[r * 3 + 2] = (b0 * a02 + b1 * a12 + b2 * a22) / det;
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
    const double ftle = degenerate ? (double)NAN : log1p(mu) * a.inv_2absT;
    reinterpret_cast<OT*>(a.ftle_out)[i] = (OT)ftle;
    if (a.lam_out) a.lam_out[i] = degenerate ? (double)NAN : 1.0 + mu;
  }
}

// ----------------------------------------------------------------------------- refine marks

__device__ __forceinline__ void mark_node(int32_t j, uint32_t* bitmap, int32_t* mark_list,
                                          unsigned long long* counter) {
  const uint32_t bit = 1u << (j & 31);
  const uint32_t old = atomicOr(bitmap + (j >> 5), bit);
  if (!(old & bit)) mark_list[atomicAdd(counter, 1ULL)] = j;
}

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

// ----------------------------------------------------------------------------- launchers

template <int DIM, int PL>
static void grad_f32_dispatch(bool coord64, const GradArgs& a, int grid, int block, cudaStream_t s) {
  if (coord64)
    k_grad_f32<DIM, PL, double><<<grid, block, 0, s>>>(a);
  else
    k_grad_f32<DIM, PL, float><<<grid, block, 0, s>>>(a);
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
