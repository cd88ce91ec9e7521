// Double-float ("df64") arithmetic: a value is the unevaluated sum hi + lo
// of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits.
// GB300 runs FP32 at 64 times its FP64 rate, so the plan's factorisation
// uses these on the FP32 pipe.  The building blocks are the classical
// error-free transformations:
//   two_sum        s + e = a + b exactly (Knuth, TAOCP vol. 2, 4.2.2)
//   fast_two_sum   the same when |a| >= |b| (Dekker 1971)
//   two_prod       p + e = a * b exactly, with one fused multiply-add
// Addition is the "sloppy" double-length add (one renormalisation): its error
// is below about 2^-44 (|a| + |b|), which the well-conditioned Gram blocks
// (cond(mu I + G) <= 1 + ||G|| / mu) keep far below the FP32 rounding the
// result gets.  Square root and reciprocal take the FP32 value and one
// Newton correction computed in double length (Karp & Markstein 1997).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace recon {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float a) { return {a, 0.f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return {s, (a - (s - v)) + (b - v)};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}

// acc + a * b with one renormalisation of the product and one of the sum
__device__ __forceinline__ df df_fma(df acc, df a, df b) {
  df p = two_prod(a.hi, b.hi);
  const float pl = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  df s = two_sum(acc.hi, p.hi);
  return fast_two_sum(s.hi, s.lo + (acc.lo + pl));
}

// acc + a * b for FP32 a, b (the product is exact in double length)
__device__ __forceinline__ df df_fma_ff(df acc, float a, float b) {
  df p = two_prod(a, b);
  df s = two_sum(acc.hi, p.hi);
  return fast_two_sum(s.hi, s.lo + (acc.lo + p.lo));
}

// sqrt(a) for a > 0: s = sqrt(hi) rounded, then s + (a - s^2) / (2 s)
__device__ __forceinline__ df df_sqrt(df a) {
  const float s = __fsqrt_rn(a.hi);
  df p = two_prod(s, s);
  const float r = ((a.hi - p.hi) - p.lo + a.lo) * (0.5f / s);
  return fast_two_sum(s, r);
}

// 1 / a: q = 1/hi rounded, then q + q (1 - a q)
__device__ __forceinline__ df df_rcp(df a) {
  const float q = __frcp_rn(a.hi);
  df p = two_prod(a.hi, q);
  const float r = ((1.f - p.hi) - p.lo) - a.lo * q;
  return fast_two_sum(q, r * q);
}

__device__ __forceinline__ df df_from_double(double a) {
  const float h = (float)a;
  return {h, (float)(a - (double)h)};
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// complex double-float (16 bytes: one float4 in memory)
struct __align__(16) dc {
  df re, im;
};

__device__ __forceinline__ float4 dc_pack(dc a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ dc dc_unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

// The complex operations under the names the templated FFT and operator
// kernels use for float2 and double2, so they run unchanged in double-float.
__device__ __forceinline__ dc c_add(dc a, dc b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dc c_sub(dc a, dc b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dc c_mul(dc a, dc b) {
  return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
__device__ __forceinline__ void c_fma(dc& acc, dc a, dc b) { acc = c_add(acc, c_mul(a, b)); }
// acc += conj(a) b
__device__ __forceinline__ void c_fmac(dc& acc, dc a, dc b) {
  acc.re = df_add(acc.re, df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)));
  acc.im = df_add(acc.im, df_sub(df_mul(a.re, b.im), df_mul(a.im, b.re)));
}
// scaling by an FP32 number (a power of two in practice: exact) or by an
// FP64 one (1/sqrt(n), taken to double length first)
__device__ __forceinline__ dc c_scale(dc a, float s) { return {df_mul(a.re, df_make(s)), df_mul(a.im, df_make(s))}; }
__device__ __forceinline__ dc c_scale(dc a, double s) {
  const df f = df_from_double(s);
  return {df_mul(a.re, f), df_mul(a.im, f)};
}
template <> __device__ __forceinline__ dc c_zero<dc>() { return {{0.f, 0.f}, {0.f, 0.f}}; }
template <> __device__ __forceinline__ dc from_f2<dc>(float2 v) { return {{v.x, 0.f}, {v.y, 0.f}}; }
// one rounding of the double-length value to FP32 (|lo| <= ulp(hi)/2)
__device__ __forceinline__ float2 to_f2(dc z) { return make_float2(z.re.hi + z.re.lo, z.im.hi + z.im.lo); }
__device__ __forceinline__ double c_abs2d(dc a) {
  const double r = df_to_double(a.re), i = df_to_double(a.im);
  return r * r + i * i;
}

}  // namespace recon
