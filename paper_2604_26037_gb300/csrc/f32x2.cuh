// Pair-of-FP32 ("double-float") arithmetic for the FP64-class step 2 on the
// FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2 once normalised, about 48 significant bits.  GB300 issues
// 64 FP32 FMAs for every FP64 FMA, so an operation that costs 12-14 FP32
// instructions still runs about 5x faster than the FP64 instruction it
// replaces.  Building blocks, each an error-free transformation from the
// floating-point literature:
//   two_sum      (Knuth, TAOCP vol. 2, 4.2.2): s + e == a + b exactly, any a, b;
//   fast_two_sum (Dekker 1971): the same in three operations when |a| >= |b|;
//   two_prod     (FMA form, Ogita-Rump-Oishi 2005): p + e == a * b exactly.
// The operations below combine them as in Dekker's double-length arithmetic:
// products drop only lo * lo (relative 2^-48); sums keep the rounding error of
// the high parts exactly and round the low parts (relative about 2^-47).
// Every step uses the explicitly rounded intrinsics, so the compiler neither
// contracts nor reorders them.
#pragma once

#include <cuda_runtime.h>

namespace pawfe {

struct alignas(8) f32x2 {
  float hi, lo;
};

__device__ __forceinline__ f32x2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ f32x2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// nearest pair to an FP64 value (exact for |x| in the FP32 normal range up to
// the 2^-48 truncation of the second half)
__device__ __forceinline__ f32x2 x2_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}

__device__ __forceinline__ double x2_to(f32x2 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ f32x2 x2_norm(f32x2 a) { return two_sum(a.hi, a.lo); }

// a + b, normalised: the high parts error-free, the low parts rounded, then
// Dekker's renormalisation.  After a cancellation of the high parts (|s.hi| <
// |lo| is then possible) fast_two_sum still returns fl(s.hi + lo) and an
// estimate of its error, so the absolute error stays at about 2^-47 (|a| + |b|)
// (the "sloppy" double-word sum of the QD library, Hida-Li-Bailey 2001).
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
  const f32x2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) { return x2_add(a, f32x2{-b.hi, -b.lo}); }

// a * b, normalised
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// acc + a * b for a running sum: the high parts are added error-free, the
// errors gather in lo; the result is left unnormalised (|lo| may reach a few
// ulp(hi) after a cancellation) and is normalised by x2_norm / x2_add before
// it is used as a factor.
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 acc) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const f32x2 s = two_sum(acc.hi, p);
  return {s.hi, __fadd_rn(s.lo, __fadd_rn(acc.lo, e))};
}

// One interface over both number types, so that a kernel template serves the
// FP64 form and the pair-of-FP32 form: Ar<R>::fma(a, b, acc) = acc + a b,
// add, sub, mul, norm (make a running sum usable as a factor), from / to FP64.
template <typename R>
struct Ar;

template <>
struct Ar<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double norm(double a) { return a; }
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double to(double a) { return a; }
};

template <>
struct Ar<f32x2> {
  static __device__ __forceinline__ f32x2 zero() { return {0.0f, 0.0f}; }
  static __device__ __forceinline__ f32x2 fma(f32x2 a, f32x2 b, f32x2 c) { return x2_fma(a, b, c); }
  static __device__ __forceinline__ f32x2 add(f32x2 a, f32x2 b) { return x2_add(a, b); }
  static __device__ __forceinline__ f32x2 sub(f32x2 a, f32x2 b) { return x2_sub(a, b); }
  static __device__ __forceinline__ f32x2 mul(f32x2 a, f32x2 b) { return x2_mul(a, b); }
  static __device__ __forceinline__ f32x2 norm(f32x2 a) { return x2_norm(a); }
  static __device__ __forceinline__ f32x2 from(double x) { return x2_from(x); }
  static __device__ __forceinline__ double to(f32x2 a) { return x2_to(a); }
};

}  // namespace pawfe
