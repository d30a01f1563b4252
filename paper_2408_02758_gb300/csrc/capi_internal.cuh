// Internal helpers shared by the C-ABI translation units (capi.cu, batch.cu, adjoint.cu).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "advect.cuh"
#include "common.cuh"
#include "gradient.cuh"

namespace ftle {

// A named range on the host timeline around one phase of a call (advection, gradient, the
// re-advection, the list copies and checks, a batch, the adjoint), for profilers that record
// NVTX ranges (e.g. ncu --nvtx --nvtx-include "ftle.gradient/"); without one attached the calls
// do nothing.  Header-only NVTX 3: no library to link.
struct PhaseRange {
  explicit PhaseRange(const char* name) { nvtxRangePushA(name); }
  ~PhaseRange() { nvtxRangePop(); }
  PhaseRange(const PhaseRange&) = delete;
  PhaseRange& operator=(const PhaseRange&) = delete;
};

struct Launch {
  double refine_kappa = 4e-4;
  int advect_block = 256;
  int advect_bps = 0;     // resident blocks per SM the advection grid is sized for (0: 2048/block)
  int grad_block = 256;
  int refine_lanes = 32;
  bool defer_fp64 = false;
  bool validate_mesh = false;
  int grad_staging = 0;   // 0: staged index tiles where possible, 1: direct loads
  int abc_refresh = kAbcRefreshDefault;
};

// Mesh validation counters (validate.cu), kept in the workspace header past ftle_counters (which
// the batch extends into its reserved words): [0] row_ptr, [1] col_idx, [2] ell_idx.
struct MeshCheck {
  unsigned long long count[3];
  unsigned long long first[3];
};
constexpr size_t kMeshCheckOffset = 128;
static_assert(sizeof(ftle_counters) <= kMeshCheckOffset && kMeshCheckOffset + sizeof(MeshCheck) <= 256,
              "mesh check counters live in the 256-byte workspace header");
inline MeshCheck* mesh_check_ptr(void* ws) {
  return reinterpret_cast<MeshCheck*>(reinterpret_cast<char*>(ws) + kMeshCheckOffset);
}
int launch_validate_mesh(const ftle_mesh* m, MeshCheck* dev_out, cudaStream_t s);
int finish_validate_mesh(const MeshCheck* dev_out, cudaStream_t s, ftle_mesh_report* report);
// Validation pass on `s` and its result (synchronises `s`); FTLE_EINVAL on a bad index.
int validate_mesh_sync(const ftle_mesh* m, void* ws, cudaStream_t s, ftle_mesh_report* report);

int check_mesh(const ftle_mesh* m);
int check_flow(const ftle_flow* f, int dim);
int check_prec(int precision);
int check_time(double T, double dt, int* nsteps);
int check_workspace(const void* ws, size_t bytes, size_t need);
Launch resolve_launch(const ftle_options* opt);
int check_launch(const Launch& L);
int grid_for(int64_t work, int block, int per_sm);
int phi_layout_of(int precision);

int launch_advect_dg(int prec, int out, bool coord64, const AdvArgs& args, int grid, int block,
                     size_t smem, cudaStream_t stream);
int launch_advect_abc(int prec, int out, bool coord64, const AdvArgs& args, int grid, int block,
                      size_t smem, cudaStream_t stream);
// Run-parallel float-float re-advection of a compensated 2D double-gyre flowmap (needs the run
// boundary states, args.seg, and nsteps <= kSegMaxSteps); coef_ws: the workspace's table region.
int launch_refine_runs_dg(bool coord64, const AdvArgs& args, void* coef_ws, int grid, cudaStream_t s);
// 3D ABC re-advection in kAbcRuns runs per node side by side (nsteps >= kAbcRuns).
constexpr int kAbcRuns = 10;
int launch_refine_runs_abc(bool coord64, const AdvArgs& args, int grid, cudaStream_t s);
int launch_advect_ds(int kind, int dim, bool coord64, const AdvArgs& args, int grid, int block,
                     cudaStream_t stream);
int launch_advect_misc(int kind, int dim, int prec, int out, bool coord64, const AdvArgs& args,
                       int grid, int block, size_t smem, cudaStream_t stream);

AdvArgs make_adv_args(const ftle_mesh* m, const ftle_flow* f, double t0, double T, double dt, int nsteps);
GradArgs make_grad_args(const ftle_mesh* m, const void* phi, double T, void* ftle_out, double* lam_out,
                        void* ws, const Launch& L);
int run_advect(const ftle_mesh* m, const ftle_flow* fl, double t0, double T, double dt, int nsteps,
               int precision, void* phi, void* ckpt, int ckpt_every, const Launch& L, cudaStream_t s);
float4* rec_ptr(const ftle_mesh* m, const void* phi, int precision);
// Whether run_refine re-advects and recomputes the flagged nodes for these arguments.
bool refine_runs(const ftle_mesh* m, int precision, const Launch& L);
int run_gradient(const ftle_mesh* m, const void* phi, int precision, double T, void* ftle_out,
                 double* lam_out, void* ws, const Launch& L, cudaStream_t s, bool fixup);
int run_refine(const ftle_mesh* m, const ftle_flow* fl, double t0, double T, double dt, int nsteps,
               int precision, void* phi, void* ftle_out, double* lam_out, void* ws, const Launch& L,
               cudaStream_t s);

}  // namespace ftle
