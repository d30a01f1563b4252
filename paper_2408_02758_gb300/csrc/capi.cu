// C-ABI of libftle.so (include/ftle.h): argument validation, workspace layout, launch sizing and
// the sequence of kernels behind each entry point.  No exception crosses this boundary and no
// device memory is allocated here.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "advect.cuh"
#include "capi_internal.cuh"
#include "gradient.cuh"

namespace ftle {

// ------------------------------------------------------------------------------------ status

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

int fail(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return status;
}

int cuda_fail(cudaError_t err, const char* where) {
  snprintf(g_err, sizeof g_err, "%s: %s (%s)", where, cudaGetErrorName(err), cudaGetErrorString(err));
  return FTLE_ECUDA;
}

int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
  if (dev < 64) {
    int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

WsLayout ws_layout(int64_t n) {
  WsLayout L;
  size_t off = 0;
  L.header = off;
  off += align256(sizeof(ftle_counters));
  L.flag_list = off;
  off += align256(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  L.mark_list = off;
  off += align256(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  L.bitmap = off;
  off += align256(sizeof(uint32_t) * (size_t)((n + 31) / 32 + 1));
  L.coef = off;
  off += align256(sizeof(float) * 2 * (size_t)(2 * kSegMaxSteps + 1));
  L.total = off;
  return L;
}

// ----------------------------------------------------------------------------- validation

int check_mesh(const ftle_mesh* m) {
  if (!m) return fail(FTLE_EINVAL, "mesh is NULL");
  if (m->dim != 2 && m->dim != 3) return fail(FTLE_EINVAL, "mesh dim %d not in {2, 3}", m->dim);
  if (m->n_nodes < 0 || m->n_nodes >= (int64_t)INT32_MAX)
    return fail(FTLE_ERANGE, "n_nodes %lld outside [0, 2^31 - 1)", (long long)m->n_nodes);
  if (m->nnz < 0 || m->nnz >= (int64_t)INT32_MAX)
    return fail(FTLE_ERANGE, "nnz %lld outside [0, 2^31 - 1)", (long long)m->nnz);
  if (m->coord_fp64 != 0 && m->coord_fp64 != 1) return fail(FTLE_EINVAL, "coord_fp64 must be 0 or 1");
  if (m->n_nodes > 0 && (!m->coords || !m->row_ptr)) return fail(FTLE_EINVAL, "mesh pointers are NULL");
  if (m->nnz > 0 && !m->col_idx) return fail(FTLE_EINVAL, "col_idx is NULL");
  if (m->ell_width < 0 || m->reserved != 0) return fail(FTLE_EINVAL, "ell_width < 0 or reserved != 0");
  if (m->stencil != FTLE_STENCIL_NONE) {
    if (m->stencil < FTLE_STENCIL_AXIS || m->stencil > FTLE_STENCIL_KUHN)
      return fail(FTLE_EINVAL, "unknown stencil %d", m->stencil);
    if ((m->stencil == FTLE_STENCIL_TRI && m->dim != 2) || (m->stencil == FTLE_STENCIL_KUHN && m->dim != 3))
      return fail(FTLE_EINVAL, "stencil %d does not exist in %dD", m->stencil, m->dim);
    int64_t prod = 1;
    for (int a = 0; a < 3; ++a) {
      const bool used = a < m->dim;
      if ((used && m->grid[a] < 2) || (!used && m->grid[a] != 1))
        return fail(FTLE_EINVAL, "stencil lattice: grid[%d] = %d (>= 2 on used axes, 1 otherwise)", a, m->grid[a]);
      prod *= m->grid[a];
    }
    if (prod != m->n_nodes) return fail(FTLE_EINVAL, "stencil lattice has %lld nodes, mesh %lld", (long long)prod,
                                        (long long)m->n_nodes);
  }
  if (m->ell_width > 0 && m->n_nodes > 0 && !m->ell_idx) return fail(FTLE_EINVAL, "ell_width set without ell_idx");
  return FTLE_OK;
}

int check_flow(const ftle_flow* f, int dim) {
  if (!f) return fail(FTLE_EINVAL, "flow is NULL");
  if (f->reserved != 0) return fail(FTLE_EINVAL, "flow.reserved must be 0");
  switch (f->kind) {
    case FTLE_FLOW_DOUBLE_GYRE:
      if (dim != 2) return fail(FTLE_EINVAL, "the double gyre is a 2D flow");
      break;
    case FTLE_FLOW_ABC:
      if (dim != 3) return fail(FTLE_EINVAL, "the ABC flow is a 3D flow");
      break;
    case FTLE_FLOW_LINEAR:
    case FTLE_FLOW_SADDLE:
      break;
    default:
      return fail(FTLE_EINVAL, "unknown flow kind %d", f->kind);
  }
  for (int q = 0; q < 12; ++q)
    if (!isfinite(f->p[q])) return fail(FTLE_EINVAL, "flow parameter %d is not finite", q);
  return FTLE_OK;
}

int check_prec(int precision) {
  if (precision != FTLE_PREC_FP64 && precision != FTLE_PREC_FP32 && precision != FTLE_PREC_FP32C)
    return fail(FTLE_EINVAL, "unknown precision %d", precision);
  return FTLE_OK;
}

int check_time(double T, double dt, int* nsteps) {
  if (!isfinite(T) || T == 0.0) return fail(FTLE_EINVAL, "T must be finite and non-zero");
  if (!isfinite(dt) || dt == 0.0) return fail(FTLE_EINVAL, "dt must be finite and non-zero");
  const double ns = nearbyint(fabs(T) / fabs(dt));
  if (!(ns >= 1.0)) return fail(FTLE_EINVAL, "|T| / |dt| rounds to zero steps");
  if (ns > (double)INT32_MAX) return fail(FTLE_ERANGE, "step count %.0f beyond 2^31 - 1", ns);
  *nsteps = (int)ns;
  return FTLE_OK;
}

int check_workspace(const void* ws, size_t bytes, size_t need) {
  if (!ws) return fail(FTLE_EWORKSPACE, "workspace is NULL");
  if (((uintptr_t)ws & 255u) != 0) return fail(FTLE_EWORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < need) return fail(FTLE_EWORKSPACE, "workspace holds %zu bytes, needs %zu", bytes, need);
  return FTLE_OK;
}

Launch resolve_launch(const ftle_options* opt) {
  Launch L;
  if (opt) {
    if (opt->refine_kappa != 0.0) L.refine_kappa = opt->refine_kappa;
    if (opt->advect_block > 0) L.advect_block = opt->advect_block;
    if (opt->advect_blocks_per_sm > 0) L.advect_bps = opt->advect_blocks_per_sm;
    if (opt->grad_block > 0) L.grad_block = opt->grad_block;
    if (opt->refine_lanes > 0) L.refine_lanes = opt->refine_lanes;
    L.defer_fp64 = opt->defer_fp64 != 0;
    L.validate_mesh = opt->validate_mesh != 0;
    L.grad_staging = opt->grad_staging;
    if (opt->abc_refresh != 0) L.abc_refresh = opt->abc_refresh;
  }
  return L;
}

int check_launch(const Launch& L) {
  if (L.advect_block % 32 || L.advect_block < 32 || L.advect_block > 256)
    return fail(FTLE_EINVAL, "advect_block must be a multiple of 32 in [32, 256]");
  if (L.grad_block % 32 || L.grad_block < 32 || L.grad_block > 256)
    return fail(FTLE_EINVAL, "grad_block must be a multiple of 32 in [32, 256]");
  if (L.advect_bps < 0 || L.advect_bps > 64) return fail(FTLE_EINVAL, "advect_blocks_per_sm in [0, 64]");
  if (L.refine_lanes < 1 || L.refine_lanes > 32) return fail(FTLE_EINVAL, "refine_lanes in [1, 32]");
  if (L.grad_staging != 0 && L.grad_staging != 1) return fail(FTLE_EINVAL, "grad_staging must be 0 or 1");
  if (L.abc_refresh < 1 || L.abc_refresh > 1024 || (L.abc_refresh & (L.abc_refresh - 1)))
    return fail(FTLE_EINVAL, "abc_refresh must be a power of two in [1, 1024]");
  return FTLE_OK;
}

size_t advect_smem_bytes(int kind, int prec, int nsteps) {
  if (kind != FTLE_FLOW_DOUBLE_GYRE) return 0;
  const int steps = nsteps < kAdvChunk ? nsteps : kAdvChunk;
  const size_t entries = 2 * (size_t)steps + 1;
  return entries * (prec == P64 ? sizeof(double) : sizeof(float2));
}

int launch_advect(int kind, int dim, int prec, int out, bool coord64, const AdvArgs& args, int grid,
                  int block, cudaStream_t stream) {
  const size_t smem = advect_smem_bytes(kind, prec, args.nsteps);
  if (kind == FTLE_FLOW_DOUBLE_GYRE)
    return launch_advect_dg(prec, out, coord64, args, grid, block, smem, stream);
  if (kind == FTLE_FLOW_ABC) return launch_advect_abc(prec, out, coord64, args, grid, block, smem, stream);
  return launch_advect_misc(kind, dim, prec, out, coord64, args, grid, block, smem, stream);
}

// Bounds on the stage angles of one RK4 step of size |h| (radians) and on stage three's angle
// differences, for the flows whose compensated step turns stage one's sines and cosines
// (rk4_step); returns false for the others.
//   Double gyre, nodes in [0, 2] x [0, 1] (the invariant domain their trajectories keep): the x
//   increment of a full step is at most D = |h| pi |A|, so pi f moves by at most
//   pi (D (1 + |eps| (2 + D)) + |eps| |omega| |h|) and pi y by at most
//   pi |h| pi |A| (1 + 2 |eps| (1 + D)).  Stage three turns stage two's pairs by the angle
//   differences to first order: with the half-step increment D2 = D / 2 and the stage-two angle
//   bound S2 (pi f and pi y together), |d pi f| <= pi D2 S2 (1 + |eps| (2 + 2 D2)) (dg cancels,
//   k_u moves by at most the angles) and |d pi y| <= pi D2 ((1 + 2 |eps| (1 + D2)) S2 +
//   |eps| |omega| |h| + 2 |eps| D2) (the y angle's scale is pi D2; k_v adds the slope's change).
//   ABC: a stage increment of component q is a step fraction <= |h| times P_q sin + Q_q cos, with
//   (P, Q) = (A, C), (B, A), (C, B), so at most |h| U with U the largest pair sum; stage three's
//   turn from stage two, d2 - d1 = h/2 (k2 - k1), is at most h^2/4 L U with the flow's Lipschitz
//   constant L (max-norm row sums), this same maximum pair sum for the ABC flow.
static bool rotation_bounds(const ftle_flow* f, double h_signed, double* angle, double* diff) {
  const double h = fabs(h_signed);
  if (f->kind == FTLE_FLOW_DOUBLE_GYRE) {
    const double A = fabs(f->p[0]), eps = fabs(f->p[1]), om = fabs(f->p[2]);
    const double D = h * kPi * A;
    const double tf = kPi * (D * (1.0 + eps * (2.0 + D)) + eps * om * h);
    const double ty = kPi * h * kPi * A * (1.0 + 2.0 * eps * (1.0 + D));
    const double D2 = 0.5 * D;
    const double S2 = kPi * (D2 * (1.0 + eps * (2.0 + D2)) + 0.5 * eps * om * h) +
                      kPi * D2 * (1.0 + 2.0 * eps * (1.0 + D2));
    const double df = kPi * D2 * S2 * (1.0 + eps * (2.0 + 2.0 * D2));
    const double dy = kPi * D2 * ((1.0 + 2.0 * eps * (1.0 + D2)) * S2 + eps * om * h + 2.0 * eps * D2);
    *angle = fmax(tf, ty);
    *diff = fmax(df, dy);
    return true;
  }
  if (f->kind == FTLE_FLOW_ABC) {
    const double A = fabs(f->p[0]), B = fabs(f->p[1]), C = fabs(f->p[2]);
    const double U = fmax(A + C, fmax(B + A, C + B));
    *angle = h * U;
    *diff = 0.25 * h * h * U * U;
    return true;
  }
  *angle = *diff = INFINITY;
  return false;
}

// The unchecked steps apply when both bounds sit within the turns' limits; the 1e-3 margin covers
// the float rounding of the angles and of positions a rounding off the walls.
static bool rotation_unchecked(double angle, double diff) {
  return angle <= (double)kRotMax * (1.0 - 1e-3) && diff <= (double)kTinyMax * (1.0 - 1e-3);
}

// The ABC step carries stage one's pairs (abc_refresh > 1) only while the step's angle bound stays
// within kCarryAngleMax, where its shorter stage-four turn drops less than 4.4e-8.
static bool carry_allowed(const ftle_flow* f, bool unchecked, double angle) {
  return f->kind == FTLE_FLOW_ABC && unchecked && angle <= (double)kCarryAngleMax * (1.0 - 1e-3);
}

AdvArgs make_adv_args(const ftle_mesh* m, const ftle_flow* f, double t0, double T, double dt, int nsteps) {
  AdvArgs a;
  memset(&a, 0, sizeof a);
  a.n = m->n_nodes;
  a.n_mesh = m->n_nodes;
  a.coords = m->coords;
  a.nsteps = nsteps;
  a.t0 = t0;
  a.h = (T < 0 ? -1.0 : 1.0) * fabs(dt);
  a.h32 = (float)a.h;
  a.h2_32 = (float)(0.5 * a.h);
  a.h6_32 = (float)(a.h / 6.0);
  a.h6_lo = (float)(a.h / 6.0 - (double)a.h6_32);
  memcpy(a.p, f->p, sizeof a.p);
  for (int d = 0; d < 3; ++d) {
    double scale = 1.0;  // the compensated double gyre carries u / (-pi A) and v / (pi A)
    if (f->kind == FTLE_FLOW_DOUBLE_GYRE && d < 2) scale = (d == 0 ? -kPi : kPi) * f->p[0];
    a.hs[d][0] = (float)(0.5 * a.h * scale);
    a.hs[d][1] = (float)(a.h * scale);
    a.hs[d][2] = (float)(a.h / 6.0 * scale);
    a.hs_lo[d] = (float)(a.h / 6.0 * scale - (double)a.hs[d][2]);
  }
  if (f->kind == FTLE_FLOW_DOUBLE_GYRE) {
    a.hs_pi[0] = (float)(kPi * 0.5 * a.h * kPi * f->p[0]);
    a.hs_pi[1] = (float)(kPi * a.h * kPi * f->p[0]);
  }
  const double hsc[3] = {0.5 * a.h, a.h, a.h / 6.0};
  for (int s = 0; s < 3; ++s)
    for (int q = 0; q < 3; ++q) a.habc[s][q] = (float)(hsc[s] * f->p[q]);
  double angle, diff;
  if (rotation_bounds(f, a.h, &angle, &diff)) a.rot_safe = rotation_unchecked(angle, diff) ? 1 : 0;
  a.carry_ok = carry_allowed(f, a.rot_safe != 0, angle);
  a.abc_refresh = a.carry_ok ? kAbcRefreshDefault : 1;
  return a;
}

int grid_for(int64_t work, int block, int per_sm) {
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  const int64_t need = (work + block - 1) / block;
  const int64_t cap = (int64_t)sms * per_sm;
  const int64_t g = need < cap ? need : cap;
  return (int)(g > 0 ? g : 1);
}

GradArgs make_grad_args(const ftle_mesh* m, const void* phi, double T, void* ftle_out, double* lam_out,
                        void* ws, const Launch& L) {
  GradArgs g;
  memset(&g, 0, sizeof g);
  const WsLayout W = ws_layout(m->n_nodes);
  char* w = reinterpret_cast<char*>(ws);
  g.n = m->n_nodes;
  g.coords = m->coords;
  g.row_ptr = m->row_ptr;
  g.col_idx = m->col_idx;
  g.nnz = m->nnz;
  g.staged = L.grad_staging == 0;
  g.stencil = m->stencil;
  for (int q = 0; q < 3; ++q) g.grid[q] = (uint32_t)m->grid[q];
  if (m->ell_width > 0 && m->ell_idx) {
    g.ell = m->ell_idx;
    g.ell_width = m->ell_width;
  }
  g.phi = phi;
  g.ftle_out = ftle_out;
  g.lam_out = lam_out;
  g.inv_2absT = 1.0 / (2.0 * fabs(T));
  g.inv_2absT32 = (float)g.inv_2absT;
  g.refine_kappa = (float)L.refine_kappa;
  g.hdr = reinterpret_cast<ftle_counters*>(w + W.header);
  g.flag_list = reinterpret_cast<int32_t*>(w + W.flag_list);
  return g;
}

int phi_layout_of(int precision) {
  return precision == FTLE_PREC_FP64 ? PHI64 : (precision == FTLE_PREC_FP32 ? PHI32 : PHI32PAIR);
}

// One call of the gradient stage (float kernel + FP64 fix-up, or the FP64 kernel).
float4* rec_ptr(const ftle_mesh* m, const void* phi, int precision) {
  if (precision != FTLE_PREC_FP32C) return nullptr;
  return reinterpret_cast<float4*>(reinterpret_cast<char*>(const_cast<void*>(phi)) + rec_offset(m->dim, m->n_nodes));
}

bool refine_runs(const ftle_mesh* m, int precision, const Launch& L) {
  return precision == FTLE_PREC_FP32C && m->n_nodes > 0 && L.refine_kappa >= 0;
}

// fixup: run the FP64 pass over the float kernel's flag list now.  ftle_compute leaves it to
// run_refine when that runs, since the refinement recomputes the same list in FP64 after the
// re-advection and overwrites every value a pass here would write.
int run_gradient(const ftle_mesh* m, const void* phi, int precision, double T, void* ftle_out,
                 double* lam_out, void* ws, const Launch& L, cudaStream_t s, bool fixup) {
  if (m->n_nodes == 0) return FTLE_OK;
  PhaseRange range("ftle.gradient");
  GradArgs g = make_grad_args(m, phi, T, ftle_out, lam_out, ws, L);
  g.rec = rec_ptr(m, phi, precision);
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  const bool c64 = m->coord_fp64 != 0;
  if (precision == FTLE_PREC_FP64) {
    const int grid = grid_for(m->n_nodes, 128, 16);
    return launch_grad_f64(m->dim, PHI64, c64, true, g, grid, 128, s);
  }
  const int grid = grid_for(m->n_nodes, L.grad_block, 2048 / L.grad_block);
  int rc = launch_grad_f32(m->dim, phi_layout_of(precision), c64, g, grid, L.grad_block, s);
  if (rc || !fixup) return rc;
  GradArgs f = g;
  f.list = g.flag_list;
  f.list_count = &g.hdr->n_flagged;
  return launch_grad_f64(m->dim, phi_layout_of(precision), c64, false, f, sms * 4, 128, s);
}

int run_refine(const ftle_mesh* m, const ftle_flow* fl, double t0, double T, double dt, int nsteps,
               int precision, void* phi, void* ftle_out, double* lam_out, void* ws, const Launch& L,
               cudaStream_t s) {
  if (!refine_runs(m, precision, L)) return FTLE_OK;
  PhaseRange range("ftle.refine");
  const WsLayout W = ws_layout(m->n_nodes);
  char* w = reinterpret_cast<char*>(ws);
  ftle_counters* hdr = reinterpret_cast<ftle_counters*>(w + W.header);
  const int sms = device_sm_count() > 0 ? device_sm_count() : 1;
  FTLE_CUDA_CHECK(cudaMemsetAsync(w + W.bitmap, 0, sizeof(uint32_t) * (size_t)((m->n_nodes + 31) / 32 + 1), s));
  FTLE_CUDA_CHECK(cudaMemsetAsync(&hdr->n_readvected, 0, sizeof(unsigned long long), s));
  FTLE_CUDA_CHECK(cudaMemsetAsync(&hdr->n_degenerate, 0, sizeof(unsigned long long), s));
  GradArgs g = make_grad_args(m, phi, T, ftle_out, lam_out, ws, L);
  g.list = g.flag_list;
  g.list_count = &hdr->n_flagged;
  int32_t* mark = reinterpret_cast<int32_t*>(w + W.mark_list);
  int rc = launch_refine_mark(g, mark, reinterpret_cast<uint32_t*>(w + W.bitmap), sms * 4, 128, s);
  if (rc) return rc;
  AdvArgs a = make_adv_args(m, fl, t0, T, dt, nsteps);
  a.out = phi;
  a.list = mark;
  a.list_count = &hdr->n_readvected;
  a.lanes = L.refine_lanes;
  a.rec = rec_ptr(m, phi, precision);
  if (fl->kind == FTLE_FLOW_DOUBLE_GYRE && m->dim == 2 && nsteps <= kSegMaxSteps && nsteps >= kSegments) {
    // the flowmap carries its run boundary states (ftle_advect writes them for compensated 2D)
    a.seg = reinterpret_cast<float2*>(reinterpret_cast<char*>(phi) + seg_offset(2, m->n_nodes));
    a.seg_stride = (int64_t)(seg_slot_bytes(m->n_nodes) / sizeof(float2));
    a.seg_len = seg_len(nsteps);
    rc = launch_refine_runs_dg(m->coord_fp64 != 0, a, w + W.coef, sms * 8, s);
  } else if (fl->kind == FTLE_FLOW_ABC && m->dim == 3 && nsteps >= kAbcRuns) {
    rc = launch_refine_runs_abc(m->coord_fp64 != 0, a, sms * 8, s);  // runs of a node side by side
  } else {
    rc = launch_advect_ds(fl->kind, m->dim, m->coord_fp64 != 0, a, sms * 8, 32, s);
  }
  if (rc) return rc;
  return launch_grad_f64(m->dim, PHI32PAIR, m->coord_fp64 != 0, false, g, sms * 4, 128, s);
}

int run_advect(const ftle_mesh* m, const ftle_flow* fl, double t0, double T, double dt, int nsteps,
               int precision, void* phi, void* ckpt, int ckpt_every, const Launch& L, cudaStream_t s) {
  if (m->n_nodes == 0) return FTLE_OK;
  PhaseRange range("ftle.advect");
  AdvArgs a = make_adv_args(m, fl, t0, T, dt, nsteps);
  a.abc_refresh = a.carry_ok ? L.abc_refresh : 1;  // beyond kCarryAngleMax every step is fresh
  a.out = phi;
  a.ckpt = ckpt;
  a.ckpt_every = ckpt ? ckpt_every : 0;
  a.ckpt_stride_bytes = (int64_t)ftle_checkpoint_bytes(m->dim, m->n_nodes, precision);
  a.rec = rec_ptr(m, phi, precision);
  if (precision == FTLE_PREC_FP32C && m->dim == 2) {
    a.seg = reinterpret_cast<float2*>(reinterpret_cast<char*>(phi) + seg_offset(2, m->n_nodes));
    a.seg_stride = (int64_t)(seg_slot_bytes(m->n_nodes) / sizeof(float2));
    a.seg_len = seg_len(nsteps);
  }
  const int prec = precision == FTLE_PREC_FP64 ? P64 : (precision == FTLE_PREC_FP32 ? P32 : P32C);
  const int out = precision == FTLE_PREC_FP64 ? O64 : (precision == FTLE_PREC_FP32 ? O32 : O32PAIR);
  int block = L.advect_block;
  if (prec == P64 && block > 128) block = 128;
  // by default a grid of 8192 / block blocks per SM (32 of 256 threads), more than fit at once:
  // blocks of few node tiles even out the end of the launch (measured against 8 per SM: 2D
  // 15.47 -> 15.34 ms, 3D 43.59 -> 43.43 ms)
  const int grid = grid_for(m->n_nodes, block, L.advect_bps > 0 ? L.advect_bps : 8192 / block);
  return launch_advect(fl->kind, m->dim, prec, out, m->coord_fp64 != 0, a, grid, block, s);
}

}  // namespace ftle

using namespace ftle;

// =================================================================================== C-ABI

extern "C" {

int ftle_version(void) { return FTLE_API_VERSION; }

const char* ftle_last_error(void) { return g_err; }

const char* ftle_status_string(int status) {
  switch (status) {
    case FTLE_OK: return "ok";
    case FTLE_EINVAL: return "invalid argument";
    case FTLE_ECUDA: return "CUDA error";
    case FTLE_EWORKSPACE: return "workspace missing, misaligned or too small";
    case FTLE_EUNSUPPORTED: return "unsupported combination";
    case FTLE_ERANGE: return "size beyond a fixed limit";
    case FTLE_ENOMEM: return "host allocation failed";
    default: return "unknown status";
  }
}

size_t ftle_checkpoint_bytes(int32_t dim, int64_t n_nodes, int32_t precision) {
  if ((dim != 2 && dim != 3) || n_nodes < 0) return 0;
  const size_t per = precision == FTLE_PREC_FP32 ? sizeof(float) : (precision == FTLE_PREC_FP64 ||
                                                                       precision == FTLE_PREC_FP32C)
                                                                          ? 8
                                                                          : 0;
  return per * (size_t)dim * (size_t)n_nodes;
}

size_t ftle_flowmap_bytes(int32_t dim, int64_t n_nodes, int32_t precision) {
  if ((dim != 2 && dim != 3) || n_nodes < 0) return 0;
  if (precision == FTLE_PREC_FP32C && dim == 2)
    return seg_offset(dim, n_nodes) + (size_t)(kSegments - 1) * seg_slot_bytes(n_nodes);
  if (precision == FTLE_PREC_FP32C) return rec_offset(dim, n_nodes) + 32 * (size_t)n_nodes;
  return ftle_checkpoint_bytes(dim, n_nodes, precision);
}

size_t ftle_workspace_bytes(int64_t n_nodes) {
  if (n_nodes < 0) return 0;
  return ws_layout(n_nodes).total;
}

int ftle_advect(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt,
                int32_t precision, void* flowmap, void* checkpoints, int32_t ckpt_every,
                const ftle_options* opt, void* stream) {
  int rc, nsteps = 0;
  if ((rc = check_mesh(mesh)) || (rc = check_flow(flow, mesh->dim)) || (rc = check_prec(precision)) ||
      (rc = check_time(T, dt, &nsteps)))
    return rc;
  if (!isfinite(t0)) return fail(FTLE_EINVAL, "t0 must be finite");
  if (mesh->n_nodes > 0 && !flowmap) return fail(FTLE_EINVAL, "flowmap is NULL");
  if (checkpoints && ckpt_every <= 0) return fail(FTLE_EINVAL, "ckpt_every must be > 0 with checkpoints");
  const Launch L = resolve_launch(opt);
  if ((rc = check_launch(L))) return rc;
  return run_advect(mesh, flow, t0, T, dt, nsteps, precision, flowmap, checkpoints, ckpt_every, L,
                    (cudaStream_t)stream);
}

int ftle_rotation_bounds(const ftle_flow* flow, double dt, ftle_rotation_info* out) {
  int rc;
  if ((rc = check_flow(flow, flow && flow->kind == FTLE_FLOW_ABC ? 3 : 2))) return rc;
  if (!out) return fail(FTLE_EINVAL, "out is NULL");
  if (!isfinite(dt) || dt == 0.0) return fail(FTLE_EINVAL, "dt must be finite and non-zero");
  double angle, diff;
  const bool rotated = rotation_bounds(flow, dt, &angle, &diff);
  out->unchecked = rotated && rotation_unchecked(angle, diff) ? 1 : 0;
  out->carried = carry_allowed(flow, out->unchecked != 0, angle) ? 1 : 0;
  out->angle_bound = angle;
  out->diff_bound = diff;
  out->angle_limit = (double)kRotMax * (1.0 - 1e-3);
  out->diff_limit = (double)kTinyMax * (1.0 - 1e-3);
  return FTLE_OK;
}

int ftle_gradient_eig(const ftle_mesh* mesh, const void* flowmap, int32_t precision, double T,
                      void* ftle_out, double* lambda_out, void* workspace, size_t workspace_bytes,
                      const ftle_options* opt, void* stream) {
  int rc;
  if ((rc = check_mesh(mesh)) || (rc = check_prec(precision))) return rc;
  if (!isfinite(T) || T == 0.0) return fail(FTLE_EINVAL, "T must be finite and non-zero");
  if (mesh->n_nodes > 0 && (!flowmap || !ftle_out)) return fail(FTLE_EINVAL, "flowmap / ftle_out is NULL");
  if ((rc = check_workspace(workspace, workspace_bytes, ftle_workspace_bytes(mesh->n_nodes)))) return rc;
  const Launch L = resolve_launch(opt);
  if ((rc = check_launch(L))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (L.validate_mesh && (rc = validate_mesh_sync(mesh, workspace, s, nullptr))) return rc;
  FTLE_CUDA_CHECK(cudaMemsetAsync(workspace, 0, sizeof(ftle_counters), s));
  return run_gradient(mesh, flowmap, precision, T, ftle_out, lambda_out, workspace, L, s,
                      !(L.defer_fp64 && refine_runs(mesh, precision, L)));
}

int ftle_refine(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt,
                int32_t precision, void* flowmap, void* ftle_out, double* lambda_out, void* workspace,
                size_t workspace_bytes, const ftle_options* opt, void* stream) {
  int rc, nsteps = 0;
  if ((rc = check_mesh(mesh)) || (rc = check_flow(flow, mesh->dim)) || (rc = check_prec(precision)) ||
      (rc = check_time(T, dt, &nsteps)))
    return rc;
  if (mesh->n_nodes > 0 && (!flowmap || !ftle_out)) return fail(FTLE_EINVAL, "flowmap / ftle_out is NULL");
  if ((rc = check_workspace(workspace, workspace_bytes, ftle_workspace_bytes(mesh->n_nodes)))) return rc;
  const Launch L = resolve_launch(opt);
  if ((rc = check_launch(L))) return rc;
  return run_refine(mesh, flow, t0, T, dt, nsteps, precision, flowmap, ftle_out, lambda_out, workspace, L,
                    (cudaStream_t)stream);
}

int ftle_compute(const ftle_mesh* mesh, const ftle_flow* flow, double t0, double T, double dt,
                 int32_t precision, void* flowmap, void* ftle_out, double* lambda_out, void* workspace,
                 size_t workspace_bytes, const ftle_options* opt, void* stream) {
  int rc, nsteps = 0;
  if ((rc = check_mesh(mesh)) || (rc = check_flow(flow, mesh->dim)) || (rc = check_prec(precision)) ||
      (rc = check_time(T, dt, &nsteps)))
    return rc;
  if (!isfinite(t0)) return fail(FTLE_EINVAL, "t0 must be finite");
  if (mesh->n_nodes > 0 && (!flowmap || !ftle_out)) return fail(FTLE_EINVAL, "flowmap / ftle_out is NULL");
  if ((rc = check_workspace(workspace, workspace_bytes, ftle_workspace_bytes(mesh->n_nodes)))) return rc;
  const Launch L = resolve_launch(opt);
  if ((rc = check_launch(L))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (L.validate_mesh && (rc = validate_mesh_sync(mesh, workspace, s, nullptr))) return rc;
  if ((rc = run_advect(mesh, flow, t0, T, dt, nsteps, precision, flowmap, nullptr, 0, L, s))) return rc;
  FTLE_CUDA_CHECK(cudaMemsetAsync(workspace, 0, sizeof(ftle_counters), s));
  if ((rc = run_gradient(mesh, flowmap, precision, T, ftle_out, lambda_out, workspace, L, s,
                         !refine_runs(mesh, precision, L))))
    return rc;
  return run_refine(mesh, flow, t0, T, dt, nsteps, precision, flowmap, ftle_out, lambda_out, workspace, L, s);
}

// A second stream for copies that overlap work on the caller's stream: open() makes it wait for
// what the caller's stream already holds, join() makes the caller's stream wait for it.
struct SideStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  int open(cudaStream_t main) {
    FTLE_CUDA_CHECK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    FTLE_CUDA_CHECK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    FTLE_CUDA_CHECK(cudaEventRecord(ev, main));
    FTLE_CUDA_CHECK(cudaStreamWaitEvent(stream, ev, 0));
    return FTLE_OK;
  }
  int join(cudaStream_t main) {
    FTLE_CUDA_CHECK(cudaEventRecord(ev, stream));
    FTLE_CUDA_CHECK(cudaStreamWaitEvent(main, ev, 0));
    return FTLE_OK;
  }
  ~SideStream() {  // on an early error return the copies may still be in flight: wait for them
    if (stream) cudaStreamSynchronize(stream);
    if (ev) cudaEventDestroy(ev);
    if (stream) cudaStreamDestroy(stream);
  }
};

// The device address of a host buffer the GPU can read and write in place (page-locked memory
// mapped into the device's address space, e.g. from cudaHostAlloc): the kernels then reach it
// over the host link without a staging copy.  NULL for anything else (pageable memory is
// copied as before).
static void* device_view(const void* host) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

size_t ftle_host_workspace_bytes(int32_t dim, int64_t n_nodes, int64_t nnz, int32_t precision) {
  if ((dim != 2 && dim != 3) || n_nodes < 0 || nnz < 0) return 0;
  const size_t cb = (precision == FTLE_PREC_FP64 ? sizeof(double) : sizeof(float)) * (size_t)dim * (size_t)n_nodes;
  size_t off = align256(ftle_workspace_bytes(n_nodes));
  off += align256(cb);                                               // coords
  off += align256(sizeof(int32_t) * (size_t)(n_nodes + 1));          // row_ptr
  off += align256(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));    // col_idx
  off += align256(ftle_flowmap_bytes(dim, n_nodes, precision));      // flowmap
  off += align256((precision == FTLE_PREC_FP64 ? 8 : 4) * (size_t)(n_nodes > 0 ? n_nodes : 1));  // ftle
  return off;
}

int ftle_compute_host(int32_t dim, int64_t n_nodes, int64_t nnz, const void* coords_host,
                      const int32_t* row_ptr_host, const int32_t* col_idx_host, const ftle_flow* flow,
                      double t0, double T, double dt, int32_t precision, void* ftle_host, void* device_ws,
                      size_t device_ws_bytes, const ftle_options* opt, void* stream) {
  int rc;
  if ((rc = check_prec(precision))) return rc;
  if ((dim != 2 && dim != 3) || n_nodes < 0 || nnz < 0) return fail(FTLE_EINVAL, "bad dim / sizes");
  if (n_nodes > 0 && (!coords_host || !row_ptr_host || !ftle_host)) return fail(FTLE_EINVAL, "host buffer is NULL");
  if (nnz > 0 && !col_idx_host) return fail(FTLE_EINVAL, "col_idx_host is NULL");
  const size_t need = ftle_host_workspace_bytes(dim, n_nodes, nnz, precision);
  if ((rc = check_workspace(device_ws, device_ws_bytes, need))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = reinterpret_cast<char*>(device_ws);
  const size_t cb = (precision == FTLE_PREC_FP64 ? sizeof(double) : sizeof(float)) * (size_t)dim * (size_t)n_nodes;
  size_t off = align256(ftle_workspace_bytes(n_nodes));
  char* coords = w + off;
  off += align256(cb);
  int32_t* rp = reinterpret_cast<int32_t*>(w + off);
  off += align256(sizeof(int32_t) * (size_t)(n_nodes + 1));
  int32_t* ci = reinterpret_cast<int32_t*>(w + off);
  off += align256(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  void* phi = w + off;
  off += align256(ftle_flowmap_bytes(dim, n_nodes, precision));
  void* ftle_dev = w + off;
  const size_t ob = (precision == FTLE_PREC_FP64 ? 8 : 4) * (size_t)n_nodes;
  ftle_mesh m;
  m.dim = dim;
  m.coord_fp64 = precision == FTLE_PREC_FP64 ? 1 : 0;
  m.n_nodes = n_nodes;
  m.nnz = nnz;
  m.coords = coords;
  m.row_ptr = rp;
  m.col_idx = ci;
  m.ell_width = 0;
  m.reserved = 0;
  m.ell_idx = nullptr;
  m.stencil = FTLE_STENCIL_NONE;
  m.grid[0] = m.grid[1] = m.grid[2] = 0;
  int nsteps = 0;
  if ((rc = check_mesh(&m)) || (rc = check_flow(flow, dim)) || (rc = check_time(T, dt, &nsteps))) return rc;
  if (!isfinite(t0)) return fail(FTLE_EINVAL, "t0 must be finite");
  const Launch L = resolve_launch(opt);
  if ((rc = check_launch(L))) return rc;
  // Page-locked, mapped host buffers are used in place: the advection reads each node's
  // coordinates once over the host link (compensated float mode, where the gradient reads the
  // flowmap's records and only the few FP64-path nodes read coordinates again), and the kernels
  // write the FTLE straight into the caller's buffer; anything else goes through staging copies.
  void* coords_view = precision == FTLE_PREC_FP32C && n_nodes > 0 ? device_view(coords_host) : nullptr;
  void* out_view = n_nodes > 0 ? device_view(ftle_host) : nullptr;
  if (coords_view) m.coords = coords_view;
  if (out_view) ftle_dev = out_view;
  // The neighbour lists are needed only once the flowmap is done, so they cross on a side stream
  // while the advection (which needs the coordinates alone) runs.
  PhaseRange range("ftle.compute_host");
  SideStream side;
  if ((rc = side.open(s))) return rc;
  if (n_nodes > 0) {
    if (!coords_view) FTLE_CUDA_CHECK(cudaMemcpyAsync(coords, coords_host, cb, cudaMemcpyHostToDevice, s));
    FTLE_CUDA_CHECK(cudaMemcpyAsync(rp, row_ptr_host, sizeof(int32_t) * (size_t)(n_nodes + 1),
                                    cudaMemcpyHostToDevice, side.stream));
  }
  if (nnz > 0)
    FTLE_CUDA_CHECK(
        cudaMemcpyAsync(ci, col_idx_host, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, side.stream));
  // the copied lists are checked on the side stream while the advection runs (its counters sit
  // in the workspace header, apart from the ftle_counters that the main stream clears)
  MeshCheck* chk = mesh_check_ptr(device_ws);
  if ((rc = launch_validate_mesh(&m, chk, side.stream))) return rc;
  if ((rc = run_advect(&m, flow, t0, T, dt, nsteps, precision, phi, nullptr, 0, L, s))) return rc;
  if ((rc = finish_validate_mesh(chk, side.stream, nullptr))) {
    cudaStreamSynchronize(s);  // nothing of this call stays in flight on an error return
    return rc;
  }
  if ((rc = side.join(s))) return rc;
  FTLE_CUDA_CHECK(cudaMemsetAsync(device_ws, 0, sizeof(ftle_counters), s));
  if ((rc = run_gradient(&m, phi, precision, T, ftle_dev, nullptr, device_ws, L, s, !refine_runs(&m, precision, L))))
    return rc;
  if ((rc = run_refine(&m, flow, t0, T, dt, nsteps, precision, phi, ftle_dev, nullptr, device_ws, L, s))) return rc;
  if (n_nodes > 0 && !out_view) FTLE_CUDA_CHECK(cudaMemcpyAsync(ftle_host, ftle_dev, ob, cudaMemcpyDeviceToHost, s));
  FTLE_CUDA_CHECK(cudaStreamSynchronize(s));
  return FTLE_OK;
}

int ftle_ell_from_csr(const ftle_mesh* mesh, int32_t width, int32_t* ell_idx, void* stream) {
  int rc;
  if ((rc = check_mesh(mesh))) return rc;
  if (width < 1 || width > 1024) return fail(FTLE_EINVAL, "width must be in [1, 1024]");
  if (mesh->n_nodes == 0) return FTLE_OK;
  if (!ell_idx) return fail(FTLE_EINVAL, "ell_idx is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int32_t> rp((size_t)mesh->n_nodes + 1);
  FTLE_CUDA_CHECK(cudaMemcpyAsync(rp.data(), mesh->row_ptr, sizeof(int32_t) * rp.size(), cudaMemcpyDeviceToHost, s));
  FTLE_CUDA_CHECK(cudaStreamSynchronize(s));
  int maxdeg = 0;
  for (int64_t i = 0; i < mesh->n_nodes; ++i) {
    const int d = rp[i + 1] - rp[i];
    if (d < 0) return fail(FTLE_EINVAL, "row_ptr decreases at row %lld", (long long)i);
    maxdeg = d > maxdeg ? d : maxdeg;
  }
  if (maxdeg > width) return fail(FTLE_ERANGE, "a row has %d neighbours, more than width %d", maxdeg, width);
  return launch_ell_from_csr(mesh->n_nodes, mesh->row_ptr, mesh->col_idx, width, ell_idx,
                             grid_for(mesh->n_nodes, 256, 8), s);
}

int ftle_read_counters(const void* workspace, ftle_counters* out, void* stream) {
  if (!workspace || !out) return fail(FTLE_EINVAL, "workspace / out is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  FTLE_CUDA_CHECK(cudaMemcpyAsync(out, workspace, sizeof(ftle_counters), cudaMemcpyDeviceToHost, s));
  FTLE_CUDA_CHECK(cudaStreamSynchronize(s));
  return FTLE_OK;
}

}  // extern "C"
