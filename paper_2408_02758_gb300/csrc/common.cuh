// Shared device and host helpers of libftle.so (CUDA path only; nothing here is used by the
// oracle).  Velocity fields, error-free float transformations and launch plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ftle.h"
#include "poly_coef.cuh"

namespace ftle {

// ------------------------------------------------------------------------------------ status

void set_error(const char* fmt, ...);
int fail(int status, const char* fmt, ...);
int cuda_fail(cudaError_t err, const char* where);

#define FTLE_CUDA_CHECK(expr)                                  \
  do {                                                         \
    cudaError_t _e = (expr);                                   \
    if (_e != cudaSuccess) return ::ftle::cuda_fail(_e, #expr); \
  } while (0)

#define FTLE_LAUNCH_CHECK(where)                                 \
  do {                                                           \
    cudaError_t _e = cudaGetLastError();                         \
    if (_e != cudaSuccess) return ::ftle::cuda_fail(_e, where);  \
  } while (0)

int device_sm_count();

// Workspace layout shared by gradient_eig / refine / compute (all offsets 256-aligned).
struct WsLayout {
  size_t header = 0;     // ftle_counters
  size_t flag_list = 0;  // int32 [n]
  size_t mark_list = 0;  // int32 [n]
  size_t bitmap = 0;     // uint32 [ceil(n/32)]
  size_t coef = 0;       // float-float a(t) at the half steps of a run-parallel re-advection
  size_t total = 0;
};

// Longest step count the run-parallel re-advection takes (its coefficient table of 2 n + 1
// float-float values lives in the workspace and in each block's shared memory).
constexpr int kSegMaxSteps = 2047;
WsLayout ws_layout(int64_t n);

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ------------------------------------------------------------------ error-free transformations

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest, no reassociation).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Dekker's Fast2Sum: s + e == a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// ------------------------------------------------------------------------ float sin / cos

constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23: x + magic rounds x to an integer

// (sin, cos) of q quarter turns plus the reduced argument, from the reduced pair (sr, cr); q is
// the integer held in the low bits of the magic-rounded float t.
__device__ __forceinline__ void quarter_turn(float t, float sr, float cr, float& s, float& c) {
  const int q = __float_as_int(t);
  const bool odd = q & 1;
  const float a = odd ? cr : sr, b = odd ? sr : cr;
  s = __int_as_float(__float_as_int(a) ^ ((q << 30) & 0x80000000));
  c = __int_as_float(__float_as_int(b) ^ (((q + 1) << 30) & 0x80000000));
}

// sin(pi x), cos(pi x): x = k/2 + r with k = rint(2x) and r = x - k/2 exact, |r| <= 1/4;
// minimax polynomials (gen_poly.py) on r, then k quarter turns.  Valid for |x| < 2^21.
__device__ __forceinline__ void fsincospi(float x, float& s, float& c) {
  const float t = fmaf(x, 2.0f, kRoundMagic);
  const float k = __fsub_rn(t, kRoundMagic);
  const float r = fmaf(k, -0.5f, x);
  const float z = r * r;
  const float ps = fmaf(fmaf(fmaf(kPI_S[3], z, kPI_S[2]), z, kPI_S[1]), z, kPI_S[0]) * r;
  const float pc = fmaf(fmaf(fmaf(fmaf(kPI_C[4], z, kPI_C[3]), z, kPI_C[2]), z, kPI_C[1]), z, kPI_C[0]);
  quarter_turn(t, ps, pc, s, c);
}

// ------------------------------------------------------------------ paired float arithmetic
// sm_100 and later issue two float lanes in one instruction (fma/mul/add .f32x2), each lane
// rounded exactly as the scalar instruction.  The FP32 pipe's rate stays the same, but a paired
// instruction takes one issue slot for two results, which frees slots for the integer and
// conversion work beside an FMA-bound loop.  The paired helpers below give the bits of their
// scalar counterparts lane by lane.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// pi/2 in three parts: A (8 significant bits) and B (13) make k*A and k*B exact for |k| < 2^11;
// C is the rest, rounded.
constexpr float kPio2A = 0x1.92p+0f;
constexpr float kPio2B = 0x1.fb4p-12f;
constexpr float kPio2C = (float)(1.57079632679489661923 - (double)0x1.92p+0 - (double)0x1.fb4p-12);

// sin(x), cos(x) at the compensated point xh + xl: x = k pi/2 + r, r carried as rh + rl (the
// third part of pi/2 and xl go to rl), minimax polynomials on rh, and the first-order
// correction rl * (cos, -sin).  Valid for |x| < 2^11 * pi/2.  Both reduction steps are exact:
// for k != 0 (|x| > pi/4) xh, k A and k B are multiples of 2^-24 and |xh - k A|, |xh - k A - k B|
// stay below 2, so each difference fits in a float; for k = 0 they return xh.
__device__ __forceinline__ void fsincos_c(float xh, float xl, float& s, float& c) {
  const float t = fmaf(xh, 0.636619772367581343f, kRoundMagic);
  const float k = __fsub_rn(t, kRoundMagic);
  const float rh = fmaf(-k, kPio2B, fmaf(-k, kPio2A, xh));
  const float rl = fmaf(-k, kPio2C, xl);
  const float z = rh * rh;
  const float ps = fmaf(fmaf(fmaf(kRAD_S[3], z, kRAD_S[2]), z, kRAD_S[1]), z, kRAD_S[0]) * rh;
  const float pc = fmaf(fmaf(fmaf(fmaf(kRAD_C[4], z, kRAD_C[3]), z, kRAD_C[2]), z, kRAD_C[1]), z, kRAD_C[0]);
  quarter_turn(t, fmaf(rl, pc, ps), fmaf(-rl, ps, pc), s, c);
}

__device__ __forceinline__ void fsincos(float x, float& s, float& c) { fsincos_c(x, 0.0f, s, c); }

// ------------------------------------------------------------------------- gradient records

// A compensated flowmap carries, after its (hi, lo) pairs, one 32-byte record per node for the
// float gradient kernel, so that a neighbour costs one address and two 16-byte loads:
//   2D: {x, y, phx_h, phy_h} {phx_l, phy_l, 0, 0}
//   3D: {x, y, z, phx_h} {phy_h, phz_h, phx_l, bf16(phy_l) | bf16(phz_l) << 16}
// (x the node's float coordinates).  The 3D record keeps two low parts in bfloat16: 8
// significant bits of a part below half an ulp of its high part, i.e. ~2^-33 relative to the
// position.  The full (hi, lo) pairs stay in the flowmap for the FP64 paths.
__host__ __device__ inline size_t rec_offset(int dim, int64_t n) {
  return ((size_t)8 * (size_t)dim * (size_t)n + 255) & ~size_t(255);
}

// A compensated 2D flowmap carries, after its records, the (hi, lo) state of every node at the
// kSegments - 1 interior boundaries of kSegments equal runs of steps (run length
// seg_len(nsteps), the last run shorter): the starting points from which the float-float
// re-advection integrates the runs side by side.  Slot j (j = 0 .. kSegments - 2) holds the state
// after min((j + 1) seg_len, nsteps) steps, laid out like the (hi, lo) pairs, float2 [2][n].
constexpr int kSegments = 8;

__host__ __device__ inline int seg_len(int nsteps) { return (nsteps + kSegments - 1) / kSegments; }
__host__ __device__ inline size_t seg_slot_bytes(int64_t n) { return ((size_t)16 * (size_t)n + 255) & ~size_t(255); }
__host__ __device__ inline size_t seg_offset(int dim, int64_t n) {
  return rec_offset(dim, n) + (((size_t)32 * (size_t)n + 255) & ~size_t(255));
}

__device__ __forceinline__ uint32_t bf16_bits(float v) {  // round to nearest even
  const uint32_t u = __float_as_uint(v);
  return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

template <int DIM>
__device__ __forceinline__ void store_record(float4* rec, int64_t i, const float* x, const float* ph, const float* pl) {
  if constexpr (DIM == 2) {
    rec[2 * i] = make_float4(x[0], x[1], ph[0], ph[1]);
    rec[2 * i + 1] = make_float4(pl[0], pl[1], 0.f, 0.f);
  } else {
    rec[2 * i] = make_float4(x[0], x[1], x[2], ph[0]);
    const uint32_t w = bf16_bits(pl[1]) | (bf16_bits(pl[2]) << 16);
    rec[2 * i + 1] = make_float4(ph[1], ph[2], pl[0], __uint_as_float(w));
  }
}

// One 32-byte record in one 256-bit read-only load (records start 256-byte aligned and are 32
// bytes each, so every record is 32-byte aligned): a warp reading consecutive records moves
// whole lines in one instruction.
__device__ __forceinline__ void ld_record256(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
      : "l"(p));
}

// A neighbour index, read once: kept out of L1 so that the lines there serve the records that
// neighbouring nodes share.
__device__ __forceinline__ int ld_index(const int32_t* p) {
  int v;
  asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}

template <int DIM>
__device__ __forceinline__ void load_record(const float4* rec, int64_t i, float* x, float* ph, float* pl) {
  float4 a, b;
  ld_record256(rec + 2 * i, a, b);
  if constexpr (DIM == 2) {
    x[0] = a.x; x[1] = a.y; ph[0] = a.z; ph[1] = a.w; pl[0] = b.x; pl[1] = b.y;
  } else {
    x[0] = a.x; x[1] = a.y; x[2] = a.z; ph[0] = a.w; ph[1] = b.x; ph[2] = b.y; pl[0] = b.z;
    const uint32_t w = __float_as_uint(b.w);
    pl[1] = __uint_as_float(w << 16);
    pl[2] = __uint_as_float(w & 0xFFFF0000u);
  }
}

// ------------------------------------------------------------- bulk copies into shared memory
// One-dimensional bulk copies (the TMA engine's untiled form) completed on an mbarrier, written
// from the PTX ISA: both addresses 16-byte aligned, the size a multiple of 16 bytes.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the async proxy (the bulk copies that complete on them).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Orders this thread's earlier generic-proxy accesses of shared memory before later async-proxy
// ones (a bulk copy refilling a buffer the block has just read).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Waits for the phase of `parity` to complete, giving up after `limit` polls; returns whether the
// phase completed.  Each poll blocks in hardware for a bounded, implementation-defined time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_addr(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ------------------------------------------------------------------------------ flow params

constexpr double kPi = 3.14159265358979323846;

struct FlowArgs {
  int kind;
  int dim;
  double p[12];
};

// Double gyre time coefficients at the half steps t_m = t0 + m h/2: a(t) = eps sin(omega t)
// rounded to float, and b = 1 - 2a carried as b_h + b_l with b_h = fl(1 - 2a) and b_l its exact
// residual, so that 2a + b is exactly 1 and the walls x = 0, 2 stay invariant in float
// arithmetic.  sin(omega t) = sin(pi u), u = (omega/pi) t formed and reduced to [-1/2, 1/2] in
// double, then evaluated by sinpif: the argument keeps double accuracy, the value float.
// Returns (a, b_l); b_h = fmaf(-2, a, 1).
__device__ __forceinline__ float2 dg_coef(double eps, double nu, double t0, double half_h, int m) {
  double u = nu * (t0 + half_h * (double)m);
  double k = rint(u);
  float s = sinpif((float)(u - k));
  if (((long long)k) & 1) s = -s;  // sin(pi (k + r)) = (-1)^k sin(pi r)
  float a = (float)eps * s;
  float bh, bl;
  two_sum(1.0f, -2.0f * a, bh, bl);
  return make_float2(a, bl);
}

// --- double gyre, plain float: (u, v) at (x, y) with coefficients (a, b)
__device__ __forceinline__ void dg_vel32(float piA, float a, float b, float x, float y, float& u,
                                         float& v) {
  float f = fmaf(a, x, b) * x;
  float fx = fmaf(2.0f * a, x, b);
  float sf, cf, sy, cy;
  fsincospi(f, sf, cf);
  fsincospi(y, sy, cy);
  u = -piA * sf * cy;
  v = piA * cf * sy * fx;
}

// --- double gyre at the compensated point (xh + xl, yh + yl).  f = x (a x + b) is formed with
// error-free products and sums, so its rounding does not act as a position error; sin/cos of
// pi (fh + fl) take the first-order correction pi fl cos / -pi fl sin.  b = bh + bl.
__device__ __forceinline__ void dg_base32c(float a, float bh, float bl, float xh, float xl, float yh, float yl,
                                           float& sf2, float& cf2, float& sy2, float& cy2, float& fx) {
  const float kPiF = 3.14159265358979323846f;
  float p = a * xh;
  float pe = fmaf(a, xh, -p);  // a xh = p + pe exactly
  float g, ge;
  fast_two_sum(bh, p, g, ge);  // bh + p = g + ge exactly (|bh| >= 1/2 >= |p| on the gyre domain)
  ge = ge + (bl + fmaf(a, xl, pe));  // a x + b = g + ge (to second order)
  float fh = g * xh;
  float fe = fmaf(g, xh, -fh);               // g xh = fh + fe exactly
  float fl = fe + fmaf(ge, xh, g * xl);      // f = fh + fl
  fx = fmaf(2.0f * a, xh, bh + fmaf(2.0f * a, xl, bl));
  float sf, cf, sy, cy;
  fsincospi(fh, sf, cf);
  fsincospi(yh, sy, cy);
  float df = kPiF * fl, dy = kPiF * yl;
  sf2 = fmaf(df, cf, sf);
  cf2 = fmaf(-df, sf, cf);
  sy2 = fmaf(dy, cy, sy);
  cy2 = fmaf(-dy, sy, cy);
}

__device__ __forceinline__ void dg_vel32c(float piA, float a, float bh, float bl, float xh, float xl,
                                          float yh, float yl, float& u, float& v) {
  float sf, cf, sy, cy, fx;
  dg_base32c(a, bh, bl, xh, xl, yh, yl, sf, cf, sy, cy, fx);
  u = -piA * sf * cy;
  v = piA * cf * sy * fx;
}

// (sin, cos)(phi + th) from (s0, c0) = (sin, cos)(phi) by the angle-addition formulas, with the
// small angle's sin th = th - th^3/6 and cos th - 1 = -th^2/2 + th^4/24 (Taylor).  For |th| <=
// kRotMax the dropped terms are below th^5/120 <= 2.7e-9 and th^6/720 <= 2.2e-11.  Each result
// takes two fused steps, s0 + c0 sin th and then + s0 (cos th - 1): two roundings at the
// result's scale (at most an ulp), for two FMA-pipe instructions instead of three.
constexpr float kRotMax = 0.05f;

__device__ __forceinline__ void rotate_small(float s0, float c0, float th, float& s, float& c) {
  const float t2 = th * th;
  const float st = fmaf(th * t2, -1.0f / 6.0f, th);
  const float cm = t2 * fmaf(t2, 1.0f / 24.0f, -0.5f);
  s = fmaf(s0, cm, fmaf(c0, st, s0));
  c = fmaf(c0, cm, fmaf(-s0, st, c0));
}

// rotate_small of both lanes.
__device__ __forceinline__ void rotate_small2(float2 s0, float2 c0, float2 th, float2& s, float2& c) {
  const float2 t2 = mul2(th, th);
  const float2 st = fma2(mul2(th, t2), f2(-1.0f / 6.0f), th);
  const float2 cm = mul2(t2, fma2(t2, f2(1.0f / 24.0f), f2(-0.5f)));
  s = fma2(s0, cm, fma2(c0, st, s0));
  c = fma2(c0, cm, fma2(neg2(s0), st, c0));
}

// --- ABC flow
__device__ __forceinline__ void abc_vel32(float A, float B, float C, float x, float y, float z,
                                          float& u, float& v, float& w) {
  float sx, cx, sy, cy, sz, cz;
  fsincos(x, sx, cx);
  fsincos(y, sy, cy);
  fsincos(z, sz, cz);
  u = fmaf(A, sz, C * cy);
  v = fmaf(B, sx, A * cz);
  w = fmaf(C, sy, B * cx);
}

// ABC flow at the compensated point: sin/cos take the low parts (and their own reduction
// residual) as a first-order correction.
__device__ __forceinline__ void abc_vel32c(float A, float B, float C, float xh, float xl, float yh,
                                           float yl, float zh, float zl, float& u, float& v,
                                           float& w) {
  float sx, cx, sy, cy, sz, cz;
  fsincos_c(xh, xl, sx, cx);
  fsincos_c(yh, yl, sy, cy);
  fsincos_c(zh, zl, sz, cz);
  u = fmaf(A, sz, C * cy);
  v = fmaf(B, sx, A * cz);
  w = fmaf(C, sy, B * cx);
}

__device__ __forceinline__ void abc_vel64(double A, double B, double C, double x, double y, double z,
                                          double& u, double& v, double& w) {
  double sx, cx, sy, cy, sz, cz;
  sincos(x, &sx, &cx);
  sincos(y, &sy, &cy);
  sincos(z, &sz, &cz);
  u = fma(A, sz, C * cy);
  v = fma(B, sx, A * cz);
  w = fma(C, sy, B * cx);
}

}  // namespace ftle
