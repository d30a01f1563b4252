// Float-float ("double-single") arithmetic: a value is an unevaluated sum h + l of two floats
// with |l| <= ulp(h)/2, about 48 significant bits, built from the error-free TwoSum, Fast2Sum and
// FMA-based TwoProduct (Dekker 1971; Knuth, TAOCP vol. 2).  It runs on the FP32 pipes, which on
// GB300 issue ~70x the FP64 rate, and serves the short re-advection lists where FP64 latency
// would dominate.
#pragma once

#include "common.cuh"

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

__device__ __forceinline__ dsf ds_mul_f(dsf a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = fmaf(a.h, b, -p);
  e = fmaf(a.l, b, e);
  return ds_fast(p, e);
}

// a * b + c
__device__ __forceinline__ dsf ds_fma(dsf a, dsf b, dsf c) { return ds_add(ds_mul(a, b), c); }

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

// sin(s r) and cos(s r) for a small float-float r (|s r| <= pi/4), s = pi (PI) or 1.
// Terms whose size stays below 2^-26 of the result are summed in float, the rest in
// float-float (Horner in z = r^2).
template <bool PI>
__device__ __forceinline__ void ds_sincos_small(dsf r, dsf& s, dsf& c) {
  const dsf z = ds_mul(r, r);
  // sin: r * (c1 + z (c3 + z (c5 + z (c7 + z (c9 + z q))))), q = c11 + z (c13 + z c15) in float
  float q = fmaf(fmaf(TaylorCoef<15, PI>::h, z.h, TaylorCoef<13, PI>::h), z.h, TaylorCoef<11, PI>::h);
  dsf a = ds_add(tc<9, PI>(), ds_mul_f(z, q));
  a = ds_add(tc<7, PI>(), ds_mul(z, a));
  a = ds_add(tc<5, PI>(), ds_mul(z, a));
  a = ds_add(tc<3, PI>(), ds_mul(z, a));
  a = ds_add(tc<1, PI>(), ds_mul(z, a));
  s = ds_mul(r, a);
  // cos: 1 + z (c2 + z (c4 + z (c6 + z (c8 + z p)))), p = c10 + z (c12 + z (c14 + z c16)) in float
  float p = fmaf(fmaf(fmaf(TaylorCoef<16, PI>::h, z.h, TaylorCoef<14, PI>::h), z.h, TaylorCoef<12, PI>::h), z.h,
                 TaylorCoef<10, PI>::h);
  dsf b = ds_add(tc<8, PI>(), ds_mul_f(z, p));
  b = ds_add(tc<6, PI>(), ds_mul(z, b));
  b = ds_add(tc<4, PI>(), ds_mul(z, b));
  b = ds_add(tc<2, PI>(), ds_mul(z, b));
  c = ds_add_f(ds_mul(z, b), 1.0f);
}

// Quarter-turn fix-up: (sin, cos) of (q * quarter + r) from (sin r, cos r), q taken mod 4.
__device__ __forceinline__ void ds_quadrant(int q, dsf sr, dsf cr, dsf& s, dsf& c) {
  const int m = q & 3;
  if (m == 0) { s = sr; c = cr; }
  else if (m == 1) { s = cr; c = ds_neg(sr); }
  else if (m == 2) { s = ds_neg(sr); c = ds_neg(cr); }
  else { s = ds_neg(cr); c = sr; }
}

// sin(pi x), cos(pi x) of a float-float x: x = k/2 + r exactly, |r| <= 1/4.
__device__ __forceinline__ void ds_sincospi(dsf x, dsf& s, dsf& c) {
  const float k = rintf(2.0f * x.h);
  const dsf r = ds_fast(x.h - 0.5f * k, x.l);  // x.h - k/2 is exact
  dsf sr, cr;
  ds_sincos_small<true>(r, sr, cr);
  ds_quadrant((int)k, sr, cr, s, c);
}

// sin(x), cos(x) of a float-float x: x = k pi/2 + r, the product k pi/2 in float-float.
__device__ __forceinline__ void ds_sincos(dsf x, dsf& s, dsf& c) {
  constexpr double kHalfPi = 1.57079632679489661923;
  const float k = rintf(x.h * (float)(2.0 / kPiD));
  const dsf pio2 = ds_make((float)kHalfPi, (float)(kHalfPi - (double)(float)kHalfPi));
  const dsf r = ds_add(x, ds_mul_f(pio2, -k));
  dsf sr, cr;
  ds_sincos_small<false>(r, sr, cr);
  ds_quadrant((int)k, sr, cr, s, c);
}

}  // namespace ftle
