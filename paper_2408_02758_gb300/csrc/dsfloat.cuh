// Float-float ("double-single") arithmetic: a value is an unevaluated sum h + l of two floats
// with |l| <= ulp(h)/2, about 48 significant bits, built from the error-free TwoSum, Fast2Sum and
// FMA-based TwoProduct (Dekker 1971; Knuth, TAOCP vol. 2).  It runs on the FP32 pipes, which on
// GB300 issue ~70x the FP64 rate, and serves the short re-advection lists where FP64 latency
// would dominate.
#pragma once

#include "common.cuh"
#include "poly_coef.cuh"

namespace ftle {

struct dsf {
  float h, l;
};

__device__ __forceinline__ dsf ds_make(float h, float l) { dsf r; r.h = h; r.l = l; return r; }

// Fast2Sum into a float-float, requires |a| >= |b| (or a == 0)
__device__ __forceinline__ dsf ds_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ds_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dsf ds_from_double(double x) {
  const float h = (float)x;
  return ds_make(h, (float)(x - (double)h));
}

__device__ __forceinline__ dsf ds_add(dsf a, dsf b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return ds_fast(s, e);
}

// Sum without the final renormalization, for operands of a product or of another sum whose terms
// do not cancel (|a + b| not far below |a| + |b|): the pair (s, e), |e| within a few ulps of s.
__device__ __forceinline__ dsf ds_add_u(dsf a, dsf b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return ds_make(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ dsf ds_add_f(dsf a, float b) {
  float s, e;
  two_sum(a.h, b, s, e);
  e = __fadd_rn(e, a.l);
  return ds_fast(s, e);
}

__device__ __forceinline__ dsf ds_mul(dsf a, dsf b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ds_fast(p, e);
}

// Product without the final renormalization: (p, e) with p = fl(a.h b.h) and e the rest to
// first order, |e| within a couple of ulps of p.  For operands of another product or of a sum,
// which take the pair as it is; it saves the Fast2Sum's three dependent operations on the chain.
__device__ __forceinline__ dsf ds_mul_u(dsf a, dsf b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return ds_make(p, e);
}

__device__ __forceinline__ dsf ds_mul_f(dsf a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return ds_fast(p, e);
}

__device__ __forceinline__ dsf ds_neg(dsf a) { return ds_make(-a.h, -a.l); }


// ---------------------------------------------------------------------- sine and cosine

// pi^k / k! with alternating signs, evaluated at compile time in double.
constexpr double cfact(int k) {
  double v = 1.0;
  for (int i = 2; i <= k; ++i) v *= (double)i;
  return v;
}
constexpr double cpow(double x, int k) {
  double v = 1.0;
  for (int i = 0; i < k; ++i) v *= x;
  return v;
}
constexpr double kPiD = 3.14159265358979323846;
template <int K, bool PI>
struct TaylorCoef {
  static constexpr double value = ((K / 2) % 2 ? -1.0 : 1.0) * (PI ? cpow(kPiD, K) : 1.0) / cfact(K);
  static constexpr float h = (float)value;
  static constexpr float l = (float)(value - (double)(float)value);
};

template <int K, bool PI>
__device__ __forceinline__ dsf tc() {
  return ds_make(TaylorCoef<K, PI>::h, TaylorCoef<K, PI>::l);
}

// Quarter-turn fix-up: (sin, cos) of (q * quarter + r) from (sin r, cos r), q taken mod 4: an odd
// q swaps the pair, bit 1 of q negates the sine and bit 1 of q + 1 the cosine (selects and sign
// flips, no branches).
__device__ __forceinline__ dsf ds_flip(dsf a, unsigned int m) {
  return ds_make(__uint_as_float(__float_as_uint(a.h) ^ m), __uint_as_float(__float_as_uint(a.l) ^ m));
}

__device__ __forceinline__ void ds_quadrant(int q, dsf sr, dsf cr, dsf& s, dsf& c) {
  const bool odd = q & 1;
  const dsf a = ds_make(odd ? cr.h : sr.h, odd ? cr.l : sr.l);
  const dsf b = ds_make(odd ? sr.h : cr.h, odd ? sr.l : cr.l);
  s = ds_flip(a, ((unsigned int)q << 30) & 0x80000000u);
  c = ds_flip(b, ((unsigned int)(q + 1) << 30) & 0x80000000u);
}

// sin and cos of a tiny float-float x (|x| <= 0.025): the terms that matter at float-float
// precision (x, x^3/6, x^2/2) in float-float, the small remainder of each series in float.
__device__ __forceinline__ void ds_sincos_tiny(dsf x, dsf& s, dsf& c) {
  const dsf x2 = ds_mul_u(x, x);
  // sin x = x + x^3 (-1/6 + x^2/120 - x^4/5040)
  const float q = x2.h * fmaf(-x2.h, 1.0f / 5040.0f, 1.0f / 120.0f);
  const dsf cs = ds_add_f(tc<3, false>(), q);
  s = ds_add_u(x, ds_mul_u(ds_mul_u(x2, x), cs));
  // cos x = 1 + x^2 (-1/2 + x^2/24 - x^4/720)
  const float p = x2.h * fmaf(-x2.h, 1.0f / 720.0f, 1.0f / 24.0f);
  c = ds_add_f(ds_mul_u(x2, ds_add_f(ds_make(-0.5f, 0.f), p)), 1.0f);
}

// (sin, cos)(a + u) from the tabulated (sin, cos)(a) and the tiny-argument pair of u.
__device__ __forceinline__ void ds_rotate(const float4 t, dsf su, dsf cu, dsf& s, dsf& c) {
  const dsf sa = ds_make(t.x, t.y), ca = ds_make(t.z, t.w);
  s = ds_add_u(ds_mul_u(sa, cu), ds_mul_u(ca, su));
  c = ds_add_u(ds_mul_u(ca, cu), ds_neg(ds_mul_u(sa, su)));
}

// sin(pi x), cos(pi x) of a float-float x: x = 2k + r (|r| <= 1), r = j/512 + u (|u| <= 1/1024),
// both subtractions exact; (sin, cos)(pi j/512) from a one-period table, and of t = pi u by
//   sin t = t + t^3 (-1/6 + t^2/120),   cos t = 1 - t^2/2 + t^4/24   (Taylor).
// With |t| <= pi/1024 the cubic part (< 5e-9) and t^4/24 (< 4e-12) are formed in float, whose
// rounding stays below 3e-16, and the dropped terms are below 2e-15 t and 1e-18.
__device__ __forceinline__ void ds_sincospi(dsf x, dsf& s, dsf& c) {
  const float k2 = 2.0f * rintf(0.5f * x.h);
  const dsf r = ds_fast(x.h - k2, x.l);
  const float j = rintf(512.0f * r.h);
  const dsf u = ds_fast(r.h - j * (1.0f / 512.0f), r.l);
  const dsf t = ds_mul_u(u, tc<1, true>());
  const float t2 = t.h * t.h;
  const dsf su = ds_fast(t.h, fmaf(t.h * t2, fmaf(t2, 1.0f / 120.0f, -1.0f / 6.0f), t.l));
  const dsf tt = ds_mul_u(t, t);
  const float cl = fmaf(-0.5f, tt.l, tt.h * tt.h * (1.0f / 24.0f));
  const dsf ch = ds_fast(1.0f, -0.5f * tt.h);
  const dsf cu = ds_make(ch.h, ch.l + cl);
  ds_rotate(__ldg(reinterpret_cast<const float4*>(kDS_SINPI512_TAB) + (int)j + 512), su, cu, s, c);
}

// sin(x), cos(x) of a float-float x: x = k pi/2 + r (the product in float-float), r = j/32 + u
// (|u| <= 1/64, exact), (sin, cos)(j/32) from the table, u by the tiny series.
__device__ __forceinline__ void ds_sincos(dsf x, dsf& s, dsf& c) {
  constexpr double kHalfPi = 1.57079632679489661923;
  const float k = rintf(x.h * (float)(2.0 / kPiD));
  const dsf pio2 = ds_make((float)kHalfPi, (float)(kHalfPi - (double)(float)kHalfPi));
  const dsf r = ds_add(x, ds_mul_f(pio2, -k));
  const float j = rintf(32.0f * r.h);
  const dsf u = ds_fast(r.h - j * (1.0f / 32.0f), r.l);
  dsf su, cu, sr, cr;
  ds_sincos_tiny(u, su, cu);
  ds_rotate(__ldg(reinterpret_cast<const float4*>(kDS_SIN_TAB) + (int)j + 26), su, cu, sr, cr);
  ds_quadrant((int)k, sr, cr, s, c);
}

}  // namespace ftle
