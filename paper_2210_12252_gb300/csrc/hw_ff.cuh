// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2, about 48 significant bits.  It runs on the FP32 pipe, which on this GPU
// issues 64 times the FP64 rate, for the transforms whose FP64 results the mixed-precision
// solver needs only to ~1e-13 relative.
//   sum:     Knuth's TwoSum gives the rounding error of hi_a + hi_b exactly; the low parts are
//            added to it and the pair renormalised with Dekker's FastTwoSum (the "sloppy"
//            double-float sum: its error is a few ulps of the larger operand's low part, which
//            is what the FFT's per-stage error analysis needs).
//   product: the FMA gives the exact error of hi_a hi_b (Dekker's TwoProduct without the
//            splitting), plus the cross terms hi_a lo_b + lo_a hi_b, renormalised.
// FP64 values convert exactly to the nearest pair (hi = the FP32 rounding, lo = the FP32
// rounding of the remainder); the pair converts back as hi + lo in FP64.
#pragma once

#include <cuda_runtime.h>

#include "hw_common.cuh"

namespace hw {

struct ff {
  float hi, lo;
  ff() = default;
  __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
  // constants: the FP32 rounding of x and of its remainder (x is a double literal, so the pair
  // carries its 53 bits to within the pair's 48)
  __host__ __device__ constexpr ff(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ constexpr ff(int x) : hi((float)x), lo(0.f) {}
};

struct ffc {
  ff x, y;
};

__host__ __device__ constexpr ff operator-(ff a) { return ff(-a.hi, -a.lo); }

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));   // a.hi + b.hi - s exactly
  return ff_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);   // a.hi b.hi - p exactly
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
// times +-1 (the transform's direction sign)
__device__ __forceinline__ ff operator*(int s, ff a) { return s > 0 ? a : -a; }

__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }

__device__ __forceinline__ ff ff_from(double x) {
  const float h = d2f(x);
  return ff(h, __double2float_rn(x - f2d(h)));
}
__device__ __forceinline__ double ff_to(ff a) { return f2d(a.hi) + f2d(a.lo); }

__device__ __forceinline__ ff shfl_xor(ff v, int m) {
  return ff(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}
__device__ __forceinline__ float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

// arithmetic type R of a slab kernel <-> storage type T of its global arrays
template <typename R> struct RcOf;
template <> struct RcOf<float> { using t = float2; };
template <> struct RcOf<double> { using t = double2; };
template <> struct RcOf<ff> { using t = ffc; };
template <typename R> using rc_t = typename RcOf<R>::t;

template <typename R>
__device__ __forceinline__ rc_t<R> mkr(R x, R y) {
  rc_t<R> r;
  r.x = x;
  r.y = y;
  return r;
}

template <typename R, typename T> __device__ __forceinline__ R to_r(T x) { return (R)x; }
template <> __device__ __forceinline__ ff to_r<ff, double>(double x) { return ff_from(x); }
template <typename T, typename R> __device__ __forceinline__ T from_r(R x) { return (T)x; }
template <> __device__ __forceinline__ double from_r<double, ff>(ff x) { return ff_to(x); }

}  // namespace hw
