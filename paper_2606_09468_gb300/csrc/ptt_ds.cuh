// Double-single arithmetic: FP64-accurate transforms on the FP32 pipe.
//
// FP64 throughput on this part is 1/64 of FP32 per warp instruction, while
// the transforms and products of the step need about 1e-14 relative accuracy
// (the FP64 path's bars against the FP64 oracle are 1e-11 after one step and
// 1e-9 after 100 steps).  A value here is the unevaluated sum h + l of two FP32
// numbers with |l| below one unit in the last place of h: 48 significant bits
// (unit roundoff about 2^-47 for these operations, ~7e-15), with FP32's
// exponent range (values between 1e-38 and 3e38, which the fields, their
// derivatives and products of this method stay inside: |c| ~ 1e4,
// derivatives ~ 1e6 at most).
//
// The building blocks are the error-free transformations of floating-point
// arithmetic: Dekker's product splitting (T. J. Dekker, "A floating-point
// technique for extending the available precision", Numer. Math. 18, 1971)
// with the product's error taken exactly by a fused multiply-add, and
// Knuth's two-sum (D. E. Knuth, TAOCP vol. 2, Sec. 4.2.2): for FP32 a, b
//   s = fl(a + b),  e = (a - (s - (s - a))) + (b - (s - a))   gives s + e = a + b,
//   p = fl(a b),    e = fma(a, b, -p)                          gives p + e = a b,
// and, when |a| >= |b|, the cheaper s = fl(a + b), e = b - (s - a).
// Sums of two double-single values add the high parts exactly, fold the
// low parts into the error and renormalise (error below ~2^-47 (|a| + |b|),
// the norm-wise bound that an FFT's error analysis needs); products add the
// cross terms h_a l_b + l_a h_b to the exact error of h_a h_b.  Every step uses
// the round-to-nearest intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn), which
// the compiler never contracts or reorders, so the transformations stay
// error-free whatever the optimisation flags.
//
// Values cross to and from FP64 arrays by integer operations on the bit
// patterns (no FP64 pipe work on loads; one FP64 addition per stored value).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "ptt_internal.h"

namespace ptt {
namespace {

struct dsf {
  float h, l;
  dsf() = default;
  __host__ __device__ constexpr dsf(float h_, float l_) : h(h_), l(l_) {}
  // small integers (|v| < 2^24) are exact in h
  __host__ __device__ constexpr dsf(int v) : h((float)v), l(0.f) {}
  // from a double: h its FP32 rounding, l the rounding of the remainder
  // (compile-time constants fold; at run time this costs FP64 work, so the
  // kernels use it only for per-block parameters)
  __host__ __device__ explicit constexpr dsf(double d)
      : h((float)d), l((float)(d - (double)(float)d)) {}
};

// complex double-single value: real part x, imaginary part y (16 bytes)
struct __align__(16) dsc {
  dsf x, y;
};

// ---------------------------------------------- error-free transformations
__device__ __forceinline__ dsf ds_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dsf(s, e);
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ dsf ds_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dsf(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// ---------------------------------------------- double-single arithmetic
__device__ __forceinline__ dsf operator-(dsf a) { return dsf(-a.h, -a.l); }
__device__ __forceinline__ dsf operator+(dsf a, dsf b) {
  const dsf s = ds_two_sum(a.h, b.h);
  return ds_quick_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }
__device__ __forceinline__ dsf operator*(dsf a, dsf b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return ds_quick_two_sum(p, e);
}
__device__ __forceinline__ dsf& operator+=(dsf& a, dsf b) { a = a + b; return a; }
__device__ __forceinline__ dsf& operator-=(dsf& a, dsf b) { a = a - b; return a; }
__device__ __forceinline__ dsf& operator*=(dsf& a, dsf b) { a = a * b; return a; }
// a b + c in one renormalisation (an overload of fma; the FP64 and FP32
// ones stay visible)
using ::fma;
__device__ __forceinline__ dsf fma(dsf a, dsf b, dsf c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const dsf s = ds_two_sum(p, c.h);
  return ds_quick_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}
// a b - c d in one renormalisation (the real part of a complex product)
__device__ __forceinline__ dsf ds_mul_sub(dsf a, dsf b, dsf c, dsf d) {
  const float p = __fmul_rn(a.h, b.h), q = __fmul_rn(c.h, d.h);
  const float ep = __fmaf_rn(a.h, b.h, -p), eq = __fmaf_rn(c.h, d.h, -q);
  const dsf s = ds_two_sum(p, -q);
  float t = __fadd_rn(s.l, __fsub_rn(ep, eq));
  t = __fmaf_rn(a.h, b.l, t);
  t = __fmaf_rn(a.l, b.h, t);
  t = __fmaf_rn(-c.h, d.l, t);
  t = __fmaf_rn(-c.l, d.h, t);
  return ds_quick_two_sum(s.h, t);
}
// a b + c d (the imaginary part of a complex product)
__device__ __forceinline__ dsf ds_mul_add(dsf a, dsf b, dsf c, dsf d) {
  return ds_mul_sub(a, b, -c, d);
}

// ---------------------------------------------- complex double-single
__device__ __forceinline__ dsc mk_dsc(dsf x, dsf y) { dsc r; r.x = x; r.y = y; return r; }
__device__ __forceinline__ dsc cadd(dsc a, dsc b) { return mk_dsc(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ dsc csub(dsc a, dsc b) { return mk_dsc(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ dsc cscl(dsc a, dsf s) { return mk_dsc(a.x * s, a.y * s); }
__device__ __forceinline__ dsc cmul(dsc a, dsc b) {
  return mk_dsc(ds_mul_sub(a.x, b.x, a.y, b.y), ds_mul_add(a.x, b.y, a.y, b.x));
}
__device__ __forceinline__ dsc mul_i(dsc a) { return mk_dsc(-a.y, a.x); }
__device__ __forceinline__ dsc cconj(dsc a) { return mk_dsc(a.x, -a.y); }
__device__ __forceinline__ dsc cfma(dsf s, dsc a, dsc c) {  // s*a + c
  return mk_dsc(fma(s, a.x, c.x), fma(s, a.y, c.y));
}

// ---------------------------------------------- conversions (integer only)
// double -> double-single: h is d truncated to 24 significant bits, l the
// next 24 bits of the remainder (truncated), so h + l carries 48 bits of d
// (relative error below 2^-47).  FP64 values below the FP32 normal range
// give zero, beyond it infinity (never reached by this method's fields);
// NaN stays NaN.
__device__ __forceinline__ dsf ds_from_double(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const uint32_t hi = (uint32_t)(u >> 32);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FF);
  const int ef = e - 1023 + 127;
  if (e == 0x7FF) {
    const bool nan = (u & 0x000FFFFFFFFFFFFFull) != 0;
    return dsf(__uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u)), 0.f);
  }
  if (ef <= 0) return dsf(__uint_as_float(sign), 0.f);
  if (ef >= 255) return dsf(__uint_as_float(sign | 0x7F800000u), 0.f);
  const float h = __uint_as_float(sign | ((uint32_t)ef << 23) | (uint32_t)((u >> 29) & 0x7FFFFFu));
  // remainder: the low 29 mantissa bits, worth rem * 2^(e - 1075)
  const uint32_t rem = (uint32_t)(u & 0x1FFFFFFFu);
  if (rem == 0u) return dsf(h, 0.f);
  const int p = 31 - __clz((int)rem);            // leading bit of rem, 0..28
  const int el = p + e - 1075 + 127;             // FP32 exponent field of l
  if (el <= 0) return dsf(h, 0.f);
  const uint32_t m = (p <= 23) ? (rem << (23 - p)) : (rem >> (p - 23));
  return dsf(h, __uint_as_float(sign | ((uint32_t)el << 23) | (m & 0x7FFFFFu)));
}
// FP32 -> FP64 by integer operations (exact for normal values; zero and
// subnormals give a signed zero, infinities stay, NaN is NaN)
__device__ __forceinline__ double ds_f32_to_f64(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  unsigned long long r;
  if (e == 0u) r = (unsigned long long)sign << 32;
  else if (e == 255u) r = ((unsigned long long)(sign | 0x7FF00000u | (m ? 0x80000u : 0u))) << 32;
  else r = ((unsigned long long)(sign | ((e + 896u) << 20) | (m >> 3)) << 32) | ((unsigned long long)(m & 7u) << 29);
  return __longlong_as_double((long long)r);
}
// double-single -> double: h and l converted exactly, one FP64 addition
__device__ __forceinline__ double ds_to_double(dsf a) { return ds_f32_to_f64(a.h) + ds_f32_to_f64(a.l); }

__device__ __forceinline__ dsc dsc_from_double2(double2 v) {
  return mk_dsc(ds_from_double(v.x), ds_from_double(v.y));
}
__device__ __forceinline__ double2 dsc_to_double2(dsc v) {
  return make_double2(ds_to_double(v.x), ds_to_double(v.y));
}

__device__ __forceinline__ dsc shfl_down2(dsc v, int o) {
  dsc r;
  r.x.h = __shfl_down_sync(0xffffffffu, v.x.h, o);
  r.x.l = __shfl_down_sync(0xffffffffu, v.x.l, o);
  r.y.h = __shfl_down_sync(0xffffffffu, v.y.h, o);
  r.y.l = __shfl_down_sync(0xffffffffu, v.y.l, o);
  return r;
}

}  // namespace
// a host-computed constant (a per-block parameter) in double-single
template <> __host__ __device__ __forceinline__ dsf as_prec<dsf>(double d, float) { return dsf(d); }

}  // namespace ptt
