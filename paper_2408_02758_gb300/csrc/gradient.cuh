// FTLE core kernels: least-squares flowmap gradient over each node's CSR neighbour list, the
// Cauchy-Green tensor, its largest eigenvalue and the FTLE (arXiv 2408.02758, Section 2.1 and
// Table 1: the per-point core; Section 2.2: precomputed neighbour lists and the branch-reduced
// gradient).  The float kernel handles every node; the nodes where float cancels are listed
// and recomputed by the double kernel.
#pragma once

#include "common.cuh"

namespace ftle {

enum PhiLayout { PHI64 = 0, PHI32 = 1, PHI32PAIR = 2 };

struct GradArgs {
  int64_t n;                   // nodes of the mesh
  const void* coords;          // SoA [dim][n], float or double
  const int32_t* row_ptr;
  const int32_t* col_idx;
  int64_t nnz;                 // entries of col_idx
  const void* phi;             // flowmap, layout per PhiLayout
  void* ftle_out;              // float [n] (double [n] when out64)
  double* lam_out;             // nullable
  double inv_2absT;            // 1 / (2 |T|)
  float inv_2absT32;           // the same in float (a double-to-float conversion per node would
                               // take GB300's narrow FP64 pipe)
  float refine_kappa;          // float kernel: flag nodes with ln(lambda_max) * h_i < refine_kappa
  ftle_counters* hdr;
  int32_t* flag_list;          // float kernel appends here
  const float4* rec;           // nullable: gradient records of a compensated flowmap (float coords)
  const int32_t* ell;          // nullable: fixed-width neighbour list [ell_width][n], -1 = none
  int ell_width;
  bool staged;                 // neighbour indices staged in shared memory by bulk copies where
                               // the layout allows (k_grad_f32_ell_staged for the fixed-width
                               // list, k_grad_f32_csr_staged for CSR rows)
  int stencil;                 // ftle_stencil: implicit lattice neighbours (0: from the lists)
  uint32_t grid[3];            // lattice nodes per axis when stencil != 0
  const int32_t* list;         // double kernel: nullable node list ...
  const unsigned long long* list_count;  // ... and its device-side length
};

// Conditioning and cancellation thresholds of the float kernel (see gradient.cu).
constexpr float kCondFlag = 0.02f;       // det(M) <= kCondFlag (tr M / d)^d -> FP64 path
constexpr float kNearDoubleTop = 1e-3f;  // 3D: 1 + r <= this (two top eigenvalues close) -> FP64
constexpr double kRankTol = 1e-12;       // FP64: det(M) <= kRankTol (tr M / d)^d -> rank-deficient
constexpr float kMuFloor = 0.01f;        // lambda_max - 1 below this cancels in float -> FP64

int launch_grad_f32(int dim, int phi_layout, bool coord64, const GradArgs& a, int grid, int block,
                    cudaStream_t stream);
int launch_grad_f64(int dim, int phi_layout, bool coord64, bool out64, const GradArgs& a, int grid,
                    int block, cudaStream_t stream);
int launch_ell_from_csr(int64_t n, const int32_t* row_ptr, const int32_t* col_idx, int width, int32_t* ell, int grid,
                        cudaStream_t s);
int launch_refine_mark(const GradArgs& a, int32_t* mark_list, uint32_t* bitmap, int grid, int block,
                       cudaStream_t stream);

}  // namespace ftle
