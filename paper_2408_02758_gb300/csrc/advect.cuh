// RK4 flowmap advection kernels (the flowmap that the FTLE core of arXiv 2408.02758 takes as
// input, Section 2.2).  One thread integrates one node; the state stays in registers for all
// steps.  Time-dependent coefficients of the double gyre are shared by every node of a step and
// live in a shared-memory table, rebuilt per chunk of steps.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace ftle {

enum Prec { P64 = 0, P32 = 1, P32C = 2 };
enum Out { O64 = 0, O32 = 1, O32PAIR = 2 };

constexpr int kAdvChunk = 2048;  // steps per coefficient-table chunk (2*chunk+1 half steps)
constexpr int kAbcRefreshDefault = 8;  // AdvArgs::abc_refresh unless ftle_options sets it

struct AdvArgs {
  int64_t n;                   // nodes (or list capacity when `list` is set)
  const void* coords;          // SoA [dim][n_mesh], float or double
  int64_t n_mesh;              // stride of coords / out
  void* out;                   // flowmap, layout per Out
  void* ckpt;                  // nullable: checkpoint slots, each one flowmap
  int64_t ckpt_stride_bytes;   // bytes per checkpoint slot
  int ckpt_every;
  int nsteps;
  double t0, h;                // h signed
  float h32, h2_32, h6_32;     // h, h/2, h/6 rounded once
  float hs[3][3];              // per component: (h/2, h, h/6) times that component's velocity
                               // scale, rounded once (compensated double gyre: -pi A, pi A; else 1)
  float hs_lo[3];              // the rounding residual of hs[d][2] (exact h/6 scale - hs[d][2]):
                               // the update carries the step's scale to ~2^-48, so no bias of
                               // its float rounding (up to 6e-8 of the velocity) builds up over
                               // the steps
  float h6_lo;                 // the same residual for h6_32
  float hs_pi[2];              // double gyre: pi (h/2, h) pi A, the y angle per unit of carried v
  float habc[3][3];            // ABC: (h/2, h, h/6) times (A, B, C), rounded once
  int abc_refresh;             // compensated ABC, unchecked steps: stage one's sines and cosines
                               // evaluated afresh every abc_refresh steps (a power of two),
                               // carried and turned by each step's increment in between
  int carry_ok;                // ABC: rot_safe and the step's angles within kCarryAngleMax, so
                               // stage one's pairs may be carried (abc_refresh > 1)
  int rot_safe;                // no stage angle can exceed kRotMax (the host's bound on the
                               // increments; for the double gyre, of nodes in [0, 2] x [0, 1]),
                               // so the steps skip the angle check
  double p[12];                // flow parameters
  const int32_t* list;         // nullable: process list[0 .. *list_count)
  const unsigned long long* list_count;
  int lanes;                   // active threads per block (0 = all): few-node lists spread wider
  float4* rec;                 // nullable: gradient records of a compensated flowmap
  float2* seg;                 // nullable: run-boundary states of a compensated 2D flowmap
  int64_t seg_stride;          // float2 per boundary slot
  int seg_len;                 // steps per run
};

// ------------------------------------------------------------------------- velocity dispatch

template <int KIND, int DIM>
__device__ __forceinline__ void vel_f32(const AdvArgs& a, const float* x, float ca, float cb, float* u) {
  if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
    dg_vel32((float)(kPi * a.p[0]), ca, cb, x[0], x[1], u[0], u[1]);
  } else if constexpr (KIND == FTLE_FLOW_ABC) {
    abc_vel32((float)a.p[0], (float)a.p[1], (float)a.p[2], x[0], x[1], x[2], u[0], u[1], u[2]);
  } else if constexpr (KIND == FTLE_FLOW_LINEAR) {
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < DIM; ++c) s = fmaf((float)a.p[r * DIM + c], x[c], s);
      u[r] = s;
    }
  } else {
    u[0] = x[0];
    u[1] = -x[1];
    if constexpr (DIM == 3) u[2] = 0.f;
  }
}

template <int KIND, int DIM>
__device__ __forceinline__ void vel_f32c(const AdvArgs& a, const float* xh, const float* xl, float ca,
                                         float cbh, float cbl, float* u) {
  if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
    dg_vel32c((float)(kPi * a.p[0]), ca, cbh, cbl, xh[0], xl[0], xh[1], xl[1], u[0], u[1]);
  } else if constexpr (KIND == FTLE_FLOW_ABC) {
    abc_vel32c((float)a.p[0], (float)a.p[1], (float)a.p[2], xh[0], xl[0], xh[1], xl[1], xh[2], xl[2],
               u[0], u[1], u[2]);
  } else if constexpr (KIND == FTLE_FLOW_LINEAR) {
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      float s = 0.f;
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        float m = (float)a.p[r * DIM + c];
        s = fmaf(m, xh[c], fmaf(m, xl[c], s));
      }
      u[r] = s;
    }
  } else {
    u[0] = xh[0] + xl[0];
    u[1] = -(xh[1] + xl[1]);
    if constexpr (DIM == 3) u[2] = 0.f;
  }
}

template <int KIND, int DIM>
__device__ __forceinline__ void vel_f64(const AdvArgs& a, const double* x, double s_om, double* u) {
  if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
    double A = a.p[0], eps = a.p[1];
    double aa = eps * s_om, bb = 1.0 - 2.0 * eps * s_om;
    double f = fma(aa, x[0], bb) * x[0];
    double fx = fma(2.0 * aa, x[0], bb);
    double sf, cf, sy, cy;
    sincospi(f, &sf, &cf);
    sincospi(x[1], &sy, &cy);
    u[0] = -kPi * A * sf * cy;
    u[1] = kPi * A * cf * sy * fx;
  } else if constexpr (KIND == FTLE_FLOW_ABC) {
    abc_vel64(a.p[0], a.p[1], a.p[2], x[0], x[1], x[2], u[0], u[1], u[2]);
  } else if constexpr (KIND == FTLE_FLOW_LINEAR) {
#pragma unroll
    for (int r = 0; r < DIM; ++r) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) s = fma(a.p[r * DIM + c], x[c], s);
      u[r] = s;
    }
  } else {
    u[0] = x[0];
    u[1] = -x[1];
    if constexpr (DIM == 3) u[2] = 0.0;
  }
}

// ----------------------------------------------------------------------------- load / store

template <typename CT>
__device__ __forceinline__ double load_coord(const void* c, int64_t idx) {
  return (double)__ldg(reinterpret_cast<const CT*>(c) + idx);
}

template <int OUT, int DIM>
__device__ __forceinline__ void store_state(void* base, int64_t n, int64_t i, const float* xh,
                                            const float* xl, const double* xd) {
  if constexpr (OUT == O64) {
    double* o = reinterpret_cast<double*>(base);
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d * n + i] = xd[d];
  } else if constexpr (OUT == O32) {
    float* o = reinterpret_cast<float*>(base);
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d * n + i] = xh[d];
  } else {
    float2* o = reinterpret_cast<float2*>(base);
#pragma unroll
    for (int d = 0; d < DIM; ++d) o[d * n + i] = make_float2(xh[d], xl[d]);
  }
}

// ----------------------------------------------------------------------------- one RK4 step

// Time coefficients of one half step: double gyre a(t), b = bh + bl (float paths) or sin(omega t)
// (double path); unused by autonomous flows.
struct Coef {
  float a, bh, bl;
  double s;
};

template <int KIND, int PREC>
__device__ __forceinline__ Coef coef_at(const float2* tab32, const double* tab64, int m) {
  Coef c{0.f, 0.f, 0.f, 0.0};
  if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
    if constexpr (PREC == P64) {
      c.s = tab64[m];
    } else {
      const float2 t = tab32[m];
      c.a = t.x;
      c.bh = fmaf(-2.f, t.x, 1.f);
      c.bl = t.y;
    }
  }
  return c;
}

// Position update x + d for the compensated state by Fast2Sum, exact when |d| <= |x| (or x = 0).
// That ordering always holds for the double gyre, saddle and linear flows, whose velocity
// vanishes linearly at the walls / origin (|d| = |h u| << |x|).  For the ABC flow it can fail
// only within |h u| <= 0.014 of a coordinate plane, where the error term is then off by at most
// an ulp of |h u| (~2e-9), far below the compensated scheme's own error at that mesh spacing.
template <int KIND>
__device__ __forceinline__ void comp_add(float xh, float d, float& s, float& e) {
  fast_two_sum(xh, d, s, e);
}

// Double gyre stage two, three or four of the compensated step.  With b = 1 - 2a the stream
// function's argument is f_t(x) = x + a(t) x (x - 2), so at the stage point x0 + dx
//   f_s(x0 + dx) - f_0(x0) = dx (1 + a_s (2 (x0 - 1) + dx)) + (a_s - a_0) x0 (x0 - 2),
// a small difference that float forms to a relative rounding (e1 = 2 (x0 - 1), dg = the last
// term).  The stage's (sin, cos)(pi f) and (sin, cos)(pi y) are stage one's pairs rotated by pi
// times the differences.  The larger angle joins `mx`; a step whose largest angle exceeds
// kRotMax is recomputed in full (rk4_step_c_full).  The y increment arrives as kv with the
// angle's scale hy_pi (pi times the increment's scale).  Returns the velocity without its
// factors -pi A and pi A.
template <bool CHECK>
__device__ __forceinline__ void dg_stage_rot(float as, float e1, float dg, float dx, float kv_prev, float hy_pi,
                                             float sf, float cf, float sy, float cy, float& mx, float& ku,
                                             float& kv) {
  const float kPiF = 3.14159265358979323846f;
  const float w = fmaf(as, e1 + dx, 1.0f);  // 1 + a_s (2 (x0 - 1) + dx)
  const float tf = kPiF * fmaf(dx, w, dg);
  const float ty = hy_pi * kv_prev;
  if constexpr (CHECK) mx = fmaxf(mx, fmaxf(fabsf(tf), fabsf(ty)));
  float2 s, c;  // lanes: pi f, pi y
  rotate_small2(make_float2(sf, sy), make_float2(cf, cy), make_float2(tf, ty), s, c);
  const float fxs = fmaf(as, dx, w);  // f_s'(x0 + dx) = 1 + 2 a_s (x0 + dx - 1)
  ku = s.x * c.y;
  kv = c.x * s.y * fxs;
}

// Largest stage-three angle difference the first-order turns of the unchecked steps take (the
// dropped term, at most kTinyMax^2 / 2 = 4.5e-8, stays at float rounding).
constexpr float kTinyMax = 3e-4f;

// Double gyre stages two and three of the unchecked step (nodes in the invariant domain).  Stage
// two turns stage one's pairs as dg_stage_rot does, without the th^4/24 term of cos th - 1 (its
// half-step angles stay within kRotMax / 2 under the host's bound, below 0.01 on the 2D
// workload, where the term is below 5e-10), but keeps the turn's corrections apart
// (sin = s0 + ds); stage three turns stage two's pairs by the angle difference (tf3 - tf2,
// ty3 - ty2, which the host bounds by kTinyMax for these steps: 1.4e-4 at dt = 0.01 on the
// default workload, so the dropped square stays below 1e-8) to first order, adding
// that to the kept correction before the one rounding onto s0.  Stage three thus costs a few
// fused operations instead of a full turn, at stage two's accuracy (measured: the same error bins
// as turning every stage from stage one).  Returns the velocities without -pi A and pi A.
__device__ __forceinline__ void dg_stages23(float as, float e1, float dg, float hs, float hy_pi, float k1u, float k1v,
                                            float sf, float cf, float sy, float cy, float& k2u, float& k2v,
                                            float& k3u, float& k3v) {
  const float kPiF = 3.14159265358979323846f;
  const float dx2 = hs * k1u;
  const float w2 = fmaf(as, e1 + dx2, 1.0f);
  const float tf2 = kPiF * fmaf(dx2, w2, dg), ty2 = hy_pi * k1v;
  float dsf, dcf, dsy, dcy;
  {
    const float t2 = tf2 * tf2, st = fmaf(tf2 * t2, -1.0f / 6.0f, tf2), cm = -0.5f * t2;
    dsf = fmaf(sf, cm, cf * st);
    dcf = fmaf(cf, cm, -(sf * st));
  }
  {
    const float t2 = ty2 * ty2, st = fmaf(ty2 * t2, -1.0f / 6.0f, ty2), cm = -0.5f * t2;
    dsy = fmaf(sy, cm, cy * st);
    dcy = fmaf(cy, cm, -(sy * st));
  }
  const float sf2 = sf + dsf, cf2 = cf + dcf, sy2 = sy + dsy, cy2 = cy + dcy;
  k2u = sf2 * cy2;
  k2v = cf2 * sy2 * fmaf(as, dx2, w2);
  const float dx3 = hs * k2u;
  const float w3 = fmaf(as, e1 + dx3, 1.0f);
  const float df = kPiF * fmaf(dx3, w3, dg) - tf2, dy = hy_pi * k2v - ty2;
  const float sf3 = sf + fmaf(cf2, df, dsf), cf3 = cf + fmaf(-sf2, df, dcf);
  const float sy3 = sy + fmaf(cy2, dy, dsy), cy3 = cy + fmaf(-sy2, dy, dcy);
  k3u = sf3 * cy3;
  k3v = cf3 * sy3 * fmaf(as, dx3, w3);
}

// The ABC velocity components times the step fractions folded into co = (A, B, C) h_s, from the
// sines s and cosines c of x, y, z.
__device__ __forceinline__ void abc_stage_k(const float* co, const float* s, const float* c, float* k) {
  k[0] = fmaf(co[0], s[2], co[2] * c[1]);
  k[1] = fmaf(co[1], s[0], co[0] * c[2]);
  k[2] = fmaf(co[2], s[1], co[1] * c[0]);
}

// rotate_small of the (sin, cos) pairs of x, y and z by the angles d, three scalar rotations.
// With stage one carried across steps the ABC step is held by the FP32 pipe, not by issue, and a
// paired f32x2 rotation of x and y (same bits) holds that pipe longer: 39.9 ms paired against
// 38.5 ms scalar at 256^3 (it paid while the step was issue-bound: 45.2 -> 43.6 ms then).
__device__ __forceinline__ void rotate_small_xyz(const float* s0, const float* c0, const float* d, float* s,
                                                 float* c) {
  const float sx = s0[0], sy = s0[1], cx = c0[0], cy = c0[1];  // s and c may alias s0 and c0
  rotate_small(sx, cx, d[0], s[0], c[0]);
  rotate_small(sy, cy, d[1], s[1], c[1]);
  rotate_small(s0[2], c0[2], d[2], s[2], c[2]);
}

// Largest step angle (|h| U, the host's bound) for which the ABC step carries stage one's pairs.
constexpr float kCarryAngleMax = 0.032f;

// rotate_small_xyz without the th^4/24 term of cos th - 1, for the unchecked ABC step's stage
// two, whose angles d1 = h/2 k1 stay within kRotMax / 2 under the host's bound (the dropped term
// below 1.6e-8, about 1e-10 at dt = 0.01 on the 3D workload), and for stage four of a carried
// step, whose angles stay within kCarryAngleMax (below 4.4e-8; about 2e-9 there).  At stage four
// the term would shrink the carried pairs' norm by that much per step until the next fresh
// evaluation; measured over the whole 256^3 field (period 8) the worst node went 8.5e-5 -> 7.4e-5
// and the p99 stayed at 2.7e-6, i.e. the shrink is below the pairs' rounding.
__device__ __forceinline__ void rotate_small_xyz_short(const float* s0, const float* c0, const float* d, float* s,
                                                       float* c) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float t2 = d[q] * d[q];
    const float st = fmaf(d[q] * t2, -1.0f / 6.0f, d[q]);
    const float cm = -0.5f * t2;
    s[q] = fmaf(s0[q], cm, fmaf(c0[q], st, s0[q]));
    c[q] = fmaf(c0[q], cm, fmaf(-s0[q], st, c0[q]));
  }
}

// ABC stage two, three or four of the compensated step: stage one's (sin, cos) of x, y, z rotated
// by the stage increments d (radians); with CHECK the largest increment joins `mx`.  co = (A, B, C) times
// the scale of the value returned (the next stage's increment, or h/6 k4).
template <bool CHECK>
__device__ __forceinline__ void abc_stage_rot(const float* co, const float* d, const float* s0, const float* c0,
                                              float& mx, float* k) {
  float s[3], c[3];
  if constexpr (CHECK) mx = fmaxf(mx, fmaxf(fabsf(d[0]), fmaxf(fabsf(d[1]), fabsf(d[2]))));
  rotate_small_xyz(s0, c0, d, s, c);
  abc_stage_k(co, s, c, k);
}

// One RK4 step of the compensated state with every stage's velocity evaluated in full at the
// compensated stage point (flows without a rotated form, and steps too long for the rotation).
template <int KIND, int DIM>
__device__ __forceinline__ void rk4_step_c_full(const AdvArgs& a, const Coef& c0, const Coef& c1, const Coef& c2,
                                                float* xh, float* xl) {
  float k1v[DIM], k2v[DIM], k3v[DIM], k4v[DIM], yh[DIM], yl[DIM];
  vel_f32c<KIND, DIM>(a, xh, xl, c0.a, c0.bh, c0.bl, k1v);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    float e;
    comp_add<KIND>(xh[d], a.h2_32 * k1v[d], yh[d], e);
    yl[d] = e + xl[d];
  }
  vel_f32c<KIND, DIM>(a, yh, yl, c1.a, c1.bh, c1.bl, k2v);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    float e;
    comp_add<KIND>(xh[d], a.h2_32 * k2v[d], yh[d], e);
    yl[d] = e + xl[d];
  }
  vel_f32c<KIND, DIM>(a, yh, yl, c1.a, c1.bh, c1.bl, k3v);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    float e;
    comp_add<KIND>(xh[d], a.h32 * k3v[d], yh[d], e);
    yl[d] = e + xl[d];
  }
  vel_f32c<KIND, DIM>(a, yh, yl, c2.a, c2.bh, c2.bl, k4v);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    float s, e;
    const float sum = fmaf(2.f, k2v[d] + k3v[d], k1v[d] + k4v[d]);
    comp_add<KIND>(xh[d], fmaf(a.h6_32, sum, fmaf(a.h6_lo, sum, xl[d])), s, e);
    xh[d] = s;
    xl[d] = e;
  }
}

// The compensated ABC step from stage one's (sin, cos) of x, y, z at the state, (s0, c0):
// stage increments d1 = h/2 k1, d2 = h/2 k2, d3 = h k3 and e4 = h/6 k4 straight from the folded
// constants; the state's increment h/6 (k1 + 2 k2 + 2 k3 + k4) = (d1 + 2 d2 + d3) / 3 + e4 goes
// to inc.  Stage two turns stage one's pairs by d1; stage three turns stage two's by d2 - d1 to
// first order (|d2 - d1| <= h^2/4 L U for a flow with Lipschitz constant L and speed bound U, so
// the dropped (d2 - d1)^2 / 2 stays near float rounding: kTinyMax); stage four turns stage one's
// by d3.  Without SAFE a stage angle beyond the turns' limits returns false (the caller then
// evaluates the step in full).  With st4 (unchecked steps only) stage four's pairs and d3 are
// handed back for the carried steps below.
struct AbcStage4 {
  float s[3], c[3], d3[3];
};

template <bool SAFE, bool KEEP4 = false>
__device__ __forceinline__ bool abc_step_from(const AdvArgs& a, const float* s0, const float* c0v, float* inc,
                                              AbcStage4* st4 = nullptr) {
  static_assert(SAFE || !KEEP4, "stage four's pairs are kept by the unchecked step only");
  float d1[3], d2[3], d3[3], e4[3], mx = 0.0f;
  d1[0] = fmaf(a.habc[0][0], s0[2], a.habc[0][2] * c0v[1]);
  d1[1] = fmaf(a.habc[0][1], s0[0], a.habc[0][0] * c0v[2]);
  d1[2] = fmaf(a.habc[0][2], s0[1], a.habc[0][1] * c0v[0]);
  float s2[3], c2v[3];
  if constexpr (SAFE)
    rotate_small_xyz_short(s0, c0v, d1, s2, c2v);
  else
    rotate_small_xyz(s0, c0v, d1, s2, c2v);
  abc_stage_k(a.habc[0], s2, c2v, d2);
  {
    float s3[3], c3[3], dmax = 0.0f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float dd = d2[q] - d1[q];
      if constexpr (!SAFE) dmax = fmaxf(dmax, fabsf(dd));
      s3[q] = fmaf(c2v[q], dd, s2[q]);
      c3[q] = fmaf(-s2[q], dd, c2v[q]);
    }
    if constexpr (!SAFE)
      mx = fmaxf(fmaxf(mx, fmaxf(fabsf(d1[0]), fmaxf(fabsf(d1[1]), fabsf(d1[2])))), dmax * (kRotMax / kTinyMax));
    abc_stage_k(a.habc[1], s3, c3, d3);
  }
  if constexpr (KEEP4) {
    rotate_small_xyz_short(s0, c0v, d3, st4->s, st4->c);  // carried steps only: |d3| <= kCarryAngleMax
    abc_stage_k(a.habc[2], st4->s, st4->c, e4);
#pragma unroll
    for (int q = 0; q < 3; ++q) st4->d3[q] = d3[q];
  } else {
    abc_stage_rot<!SAFE>(a.habc[2], d3, s0, c0v, mx, e4);
  }
  if (!(SAFE || mx <= kRotMax)) return false;
#pragma unroll
  for (int q = 0; q < 3; ++q) inc[q] = fmaf(fmaf(2.f, d2[q], d1[q] + d3[q]), 1.0f / 3.0f, e4[q]);
  return true;
}

// Stage one's (sin, cos) of the state carried from step to step by the unchecked compensated ABC
// step (AdvArgs::rot_safe): a step whose index is a multiple of AdvArgs::abc_refresh evaluates
// them afresh at the compensated state (fsincos_c); the steps between start from the previous
// step's stage-four pairs, at x + d3 with d3 = h k3, and turn them to first order by what the
// state moved beyond that point, inc - d3 = h/6 ((k1 - k3) + 2 (k2 - k3) + (k4 - k3)).  That
// difference is third order in h (about h^3 L^2 U / 12; ~2e-6 rad at h = 0.01); in any case
// |inc - d3| <= h^2 L U / 6 (1 + hL/2 + (hL)^2 / 8), below stage three's bound h^2 L U / 4
// whenever hL <= kRotMax, so the host's kTinyMax check on stage three covers it and the dropped
// (inc - d3)^2 / 2 stays below float rounding.  The increment is taken before its low part joins
// the state, which moves the angle by at most half an ulp of the increment.  The turns'
// roundings accumulate over at most abc_refresh - 1 steps before the next fresh evaluation.
struct AbcCarry {
  float s[3], c[3];
};

// One carried step from the pairs in cy: the step's increment, the compensated state update,
// and (with TURN) the next step's pairs from stage four's, turned by inc - d3 (formed exactly
// where inc and d3 agree within a factor of two, as they do unless both are tiny).
template <bool TURN>
__device__ __forceinline__ void abc_carried_one(const AdvArgs& a, float* xh, float* xl, AbcCarry& cy) {
  float inc[3];
  AbcStage4 st4;
  if constexpr (TURN)
    abc_step_from<true, true>(a, cy.s, cy.c, inc, &st4);
  else
    abc_step_from<true>(a, cy.s, cy.c, inc);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    float s, e;
    comp_add<FTLE_FLOW_ABC>(xh[q], inc[q] + xl[q], s, e);
    xh[q] = s;
    xl[q] = e;
  }
  if constexpr (TURN) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float dl = inc[q] - st4.d3[q];
      cy.s[q] = fmaf(st4.c[q], dl, st4.s[q]);
      cy.c[q] = fmaf(-st4.s[q], dl, st4.c[q]);
    }
  }
}

__device__ __forceinline__ void abc_fresh_pairs(const float* xh, const float* xl, AbcCarry& cy) {
#pragma unroll
  for (int q = 0; q < 3; ++q) fsincos_c(xh[q], xl[q], cy.s[q], cy.c[q]);
}

// Step k alone (for loops that do more per step, such as storing checkpoints).
__device__ __forceinline__ void abc_step_carried(const AdvArgs& a, int k, float* xh, float* xl, AbcCarry& cy) {
  const int mask = a.abc_refresh - 1;  // abc_refresh is a power of two
  if ((k & mask) == 0) abc_fresh_pairs(xh, xl, cy);
  if (((k + 1) & mask) != 0)
    abc_carried_one<true>(a, xh, xl, cy);
  else
    abc_carried_one<false>(a, xh, xl, cy);
}

// Steps k .. stop - 1, the same arithmetic as abc_step_carried step by step, grouped between
// refreshes so that the inner loop tests nothing but its bound (k ends at stop).
__device__ __forceinline__ void abc_steps_carried(const AdvArgs& a, int& k, int stop, float* xh, float* xl,
                                                  AbcCarry& cy) {
  const int mask = a.abc_refresh - 1;
  while (k < stop) {
    const int g = min(stop, (k | mask) + 1);  // the next step that refreshes, or stop
    if (mask == kAbcRefreshDefault - 1 && (k & mask) == 0 && g - k == kAbcRefreshDefault) {
      // a whole group of the default period, unrolled
      abc_fresh_pairs(xh, xl, cy);
#pragma unroll
      for (int q = 0; q < kAbcRefreshDefault - 1; ++q) abc_carried_one<true>(a, xh, xl, cy);
      abc_carried_one<false>(a, xh, xl, cy);
      k = g;
      continue;
    }
    if ((k & mask) == 0) abc_fresh_pairs(xh, xl, cy);
    for (; k < g - 1; ++k) abc_carried_one<true>(a, xh, xl, cy);
    if ((g & mask) != 0)  // cut short by stop: a later call carries on from these pairs
      abc_carried_one<true>(a, xh, xl, cy);
    else
      abc_carried_one<false>(a, xh, xl, cy);
    ++k;
  }
}

// Advance one node by one classic RK4 step (stages at t, t + h/2, t + h/2, t + h, with the
// coefficients c0, c1, c2 of those half steps).  P64 updates xd; P32 updates xh; P32C updates
// the compensated pair (xh, xl), evaluating the velocity at compensated stage points.  SAFE
// (AdvArgs::rot_safe, and for the double gyre a node inside its invariant domain): every stage
// angle is known to be within kRotMax, so the rotated stages run without the angle check (same
// scheme; the rounding may differ from the checked step's, see dg_node_safe).
template <int KIND, int DIM, int PREC, bool SAFE = false>
__device__ __forceinline__ void rk4_step(const AdvArgs& a, const Coef& c0, const Coef& c1, const Coef& c2,
                                         float* xh, float* xl, double* xd) {
  if constexpr (PREC == P64) {
    double k1v[DIM], k2v[DIM], k3v[DIM], k4v[DIM], y[DIM];
    vel_f64<KIND, DIM>(a, xd, c0.s, k1v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) y[d] = fma(0.5 * a.h, k1v[d], xd[d]);
    vel_f64<KIND, DIM>(a, y, c1.s, k2v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) y[d] = fma(0.5 * a.h, k2v[d], xd[d]);
    vel_f64<KIND, DIM>(a, y, c1.s, k3v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) y[d] = fma(a.h, k3v[d], xd[d]);
    vel_f64<KIND, DIM>(a, y, c2.s, k4v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) xd[d] += (a.h / 6.0) * (k1v[d] + 2.0 * (k2v[d] + k3v[d]) + k4v[d]);
  } else if constexpr (PREC == P32) {
    float k1v[DIM], k2v[DIM], k3v[DIM], k4v[DIM], y[DIM];
    vel_f32<KIND, DIM>(a, xh, c0.a, c0.bh, k1v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) y[d] = fmaf(a.h2_32, k1v[d], xh[d]);
    vel_f32<KIND, DIM>(a, y, c1.a, c1.bh, k2v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) y[d] = fmaf(a.h2_32, k2v[d], xh[d]);
    vel_f32<KIND, DIM>(a, y, c1.a, c1.bh, k3v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) y[d] = fmaf(a.h32, k3v[d], xh[d]);
    vel_f32<KIND, DIM>(a, y, c2.a, c2.bh, k4v);
#pragma unroll
    for (int d = 0; d < DIM; ++d) xh[d] = fmaf(a.h6_32, fmaf(2.f, k2v[d] + k3v[d], k1v[d] + k4v[d]), xh[d]);
  } else if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {  // P32C, stages two to four by rotation
    float sf, cf, sy, cy, fx_unused;
    dg_base32c(c0.a, c0.bh, c0.bl, xh[0], xl[0], xh[1], xl[1], sf, cf, sy, cy, fx_unused);
    const float e1 = fmaf(2.0f, xh[0], -2.0f);        // 2 (x0 - 1)
    const float fx = fmaf(c0.a, e1, 1.0f);            // f_0'(x0) = 1 + 2 a_0 (x0 - 1)
    const float k1u = sf * cy, k1v = cf * sy * fx;
    const float g0 = xh[0] * (xh[0] - 2.0f);
    const float dg1 = (c1.a - c0.a) * g0, dg2 = (c2.a - c0.a) * g0;
    float k2u, k2v, k3u, k3v, k4u, k4v, mx = 0.0f;
    if constexpr (SAFE) {
      dg_stages23(c1.a, e1, dg1, a.hs[0][0], a.hs_pi[0], k1u, k1v, sf, cf, sy, cy, k2u, k2v, k3u, k3v);
    } else {
      dg_stage_rot<!SAFE>(c1.a, e1, dg1, a.hs[0][0] * k1u, k1v, a.hs_pi[0], sf, cf, sy, cy, mx, k2u, k2v);
      dg_stage_rot<!SAFE>(c1.a, e1, dg1, a.hs[0][0] * k2u, k2v, a.hs_pi[0], sf, cf, sy, cy, mx, k3u, k3v);
    }
    dg_stage_rot<!SAFE>(c2.a, e1, dg2, a.hs[0][1] * k3u, k3v, a.hs_pi[1], sf, cf, sy, cy, mx, k4u, k4v);
    if (SAFE || mx <= kRotMax) {
      // the increment h/6 (k1 + 2 k2 + 2 k3 + k4) (its scale in two parts) and the low part
      // join in one rounding
      const float sum[2] = {fmaf(2.f, k2u + k3u, k1u + k4u), fmaf(2.f, k2v + k3v, k1v + k4v)};
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        float s, e;
        comp_add<KIND>(xh[d], fmaf(a.hs[d][2], sum[d], fmaf(a.hs_lo[d], sum[d], xl[d])), s, e);
        xh[d] = s;
        xl[d] = e;
      }
    } else {
      rk4_step_c_full<KIND, DIM>(a, c0, c1, c2, xh, xl);
    }
  } else if constexpr (KIND == FTLE_FLOW_ABC) {  // P32C, stages two to four by rotation
    float s0[3], c0v[3], inc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) fsincos_c(xh[q], xl[q], s0[q], c0v[q]);
    if (abc_step_from<SAFE>(a, s0, c0v, inc)) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        float s, e;
        comp_add<KIND>(xh[q], inc[q] + xl[q], s, e);
        xh[q] = s;
        xl[q] = e;
      }
    } else {
      rk4_step_c_full<KIND, DIM>(a, c0, c1, c2, xh, xl);
    }
  } else {  // P32C, other flows: velocity at the compensated stage points
    rk4_step_c_full<KIND, DIM>(a, c0, c1, c2, xh, xl);
  }
}

// Fill the shared table with the coefficients of half steps 2 k0 .. 2 k1 (whole block).
template <int KIND, int PREC>
__device__ __forceinline__ void build_table(const AdvArgs& a, float2* tab32, double* tab64, int k0, int k1) {
  if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE) {
    const double nu = a.p[2] / kPi;  // omega / pi
    for (int m = threadIdx.x; m <= 2 * (k1 - k0); m += blockDim.x) {
      if constexpr (PREC == P64) {
        tab64[m] = sin(a.p[2] * (a.t0 + 0.5 * a.h * (double)(2 * k0 + m)));
      } else {
        tab32[m] = dg_coef(a.p[1], nu, a.t0, 0.5 * a.h, 2 * k0 + m);
      }
    }
  }
}

template <int PREC, int DIM>
__device__ __forceinline__ void split_state(float* xh, float* xl, const double* xd) {
  if constexpr (PREC == P64) {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      xh[d] = (float)xd[d];
      xl[d] = (float)(xd[d] - (double)xh[d]);
    }
  }
}

// --------------------------------------------------------------------------------- kernel

// Whether a double-gyre node takes the unchecked steps: the host's angle bound holds (rot_safe)
// and the node starts in the invariant domain [0, 2] x [0, 1] (x, y its initial coordinates).
// The unchecked and the checked step may round differently (the compiler contracts their
// products differently), so every kernel that advances a node (k_advect, k_batch_advect, the
// adjoint's recomputation) decides by this function of the node alone, and their states agree
// bit for bit.  A warp mixing both kinds of node runs the two loops one after the other.
__device__ __forceinline__ bool dg_node_safe(const AdvArgs& a, double x, double y) {
  return a.rot_safe && x >= 0.0 && x <= 2.0 && y >= 0.0 && y <= 1.0;
}

// SAFE: the instantiation for AdvArgs::rot_safe (rk4_step's angle-check-free ABC step).  The
// compensated float kernels are held to five 256-thread blocks per SM (48 registers) for the
// double gyre (measured on the full mesh: 15.84 ms at 40 registers, six blocks; 15.47 at 48;
// 15.83 at 64, four blocks) and six for the ABC flow with stage one carried (40 registers, a
// few bytes spilled outside the step loop: 37.83 ms against 38.46 at five blocks).
// CARRY (with SAFE, the compensated ABC step): stage one's (sin, cos) carried across steps
// (abc_step_carried, AdvArgs::abc_refresh > 1).
template <int KIND, int DIM, int PREC, int OUT, typename CT, bool SAFE = false, bool CARRY = false>
__global__ void __launch_bounds__(256, PREC == P32C ? (KIND == FTLE_FLOW_ABC ? 6 : 5) : 1) k_advect(AdvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kTable = (KIND == FTLE_FLOW_DOUBLE_GYRE);
  float2* tab32 = reinterpret_cast<float2*>(smem_raw);
  double* tab64 = reinterpret_cast<double*>(smem_raw);

  const int64_t count = a.list ? (int64_t)*a.list_count : a.n;
  const int nchunks = (a.nsteps + kAdvChunk - 1) / kAdvChunk;
  bool table_valid = false;  // single-chunk tables are built once per block

  const int lanes = (a.lanes > 0 && a.lanes < (int)blockDim.x) ? a.lanes : (int)blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * lanes; base < count; base += (int64_t)gridDim.x * lanes) {
    const int64_t slot = base + threadIdx.x;
    const bool active = (int)threadIdx.x < lanes && slot < count;
    const int64_t i = active ? (a.list ? (int64_t)a.list[slot] : slot) : 0;

    float xh[DIM], xl[DIM], x0[DIM];
    double xd[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double c = active ? load_coord<CT>(a.coords, d * a.n_mesh + i) : 0.0;
      xd[d] = c;
      xh[d] = (float)c;
      xl[d] = (float)(c - (double)xh[d]);
      x0[d] = xh[d];
    }
    if (a.ckpt && active) store_state<OUT, DIM>(a.ckpt, a.n_mesh, i, xh, xl, xd);
    bool safe_node = false;
    if constexpr (KIND == FTLE_FLOW_DOUBLE_GYRE && PREC == P32C) safe_node = dg_node_safe(a, xd[0], xd[1]);
    int ck_left = a.ckpt_every;
    int ck_slot = 1;
    AbcCarry carry;  // stage one's carried (sin, cos), refreshed at step 0 and every abc_refresh
    constexpr bool kSegs = PREC == P32C && OUT == O32PAIR && DIM == 2;
    int seg_slot = 0, next_seg = a.seg_len;

    for (int ch = 0; ch < nchunks; ++ch) {
      const int k0 = ch * kAdvChunk;
      const int k1 = min(a.nsteps, k0 + kAdvChunk);
      if constexpr (kTable) {
        if (!(table_valid && nchunks == 1)) {
          __syncthreads();
          build_table<KIND, PREC>(a, tab32, tab64, k0, k1);
          __syncthreads();
          table_valid = true;
        }
      }
      if (!active) continue;
      for (int k = k0; k < k1;) {
        // steps up to the next run boundary (uniform across the block), then its state
        const int stop = (kSegs && a.seg) ? min(k1, next_seg) : k1;
        // abc_refresh = 1 takes rk4_step's unchecked ABC step (CARRY false), the same arithmetic
        // without the carried pairs' bookkeeping
        auto steps = [&](auto safe, auto carried) {
          if constexpr (KIND == FTLE_FLOW_ABC && PREC == P32C && decltype(safe)::value && decltype(carried)::value) {
            if (!a.ckpt) {
              abc_steps_carried(a, k, stop, xh, xl, carry);
              return;
            }
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
            if (a.ckpt) {
              if (--ck_left == 0) {
                ck_left = a.ckpt_every;
                split_state<PREC, DIM>(xh, xl, xd);
                store_state<OUT, DIM>(reinterpret_cast<char*>(a.ckpt) + (int64_t)ck_slot * a.ckpt_stride_bytes,
                                      a.n_mesh, i, xh, xl, xd);
                ++ck_slot;
              }
            }
          }
        };
        if (SAFE) {
          steps(std::integral_constant<bool, SAFE>{}, std::integral_constant<bool, CARRY>{});
        } else if (safe_node) {
          steps(std::true_type{}, std::false_type{});
        } else {
          steps(std::false_type{}, std::false_type{});
        }
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
      // boundaries at or past the last step hold the final state
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

// Host-side launcher (advect.cu): picks the instantiation for (kind, dim, prec, out, coord type).
int launch_advect(int kind, int dim, int prec, int out, bool coord64, const AdvArgs& args, int grid,
                  int block, cudaStream_t stream);

size_t advect_smem_bytes(int kind, int prec, int nsteps);

}  // namespace ftle
