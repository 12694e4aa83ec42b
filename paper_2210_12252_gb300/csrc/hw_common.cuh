// Device-side helpers shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace hw {

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

template <typename T> using cplx_t = typename C2<T>::t;

template <typename T>
__device__ __forceinline__ cplx_t<T> mk(T x, T y) {
  cplx_t<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V>
__device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename V>
__device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
// multiply by +i (s > 0) or -i (s < 0)
template <typename V>
__device__ __forceinline__ V cmul_i(V a, int s) {
  V r;
  if (s > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

}  // namespace hw
