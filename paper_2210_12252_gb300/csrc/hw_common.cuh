// Device-side helpers shared by the library's CUDA translation units.
#pragma once

#include <utility>
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

// Programmatic dependent launch.  A kernel launched with the programmatic-serialisation
// attribute may start while the kernel before it in the stream is still running; it touches
// nothing that kernel writes or reads, and allocates no tensor memory, before griddep_wait(),
// which returns once that kernel has completed and its writes are visible (at once in a launch
// without the attribute).  griddep_launch() lets the next such kernel start its CTAs early, as
// this grid's resources free up.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }
// Both, as a kernel's first statement: the kernel touches nothing before the kernel ahead of it
// has completed (the same order as a plain launch), and the next kernel may start its CTAs once
// every CTA of this one has got this far, which hides most of a launch's latency (a chain of
// short dependent kernels on this GPU: 4.1 -> 1.4 us per kernel).
__device__ __forceinline__ void griddep_entry() {
  griddep_wait();
  griddep_launch();
}

#ifdef __CUDACC__
// Launch k on stream st with programmatic stream serialisation; k starts with griddep_entry()
// (or reads nothing an earlier kernel writes before griddep_wait()).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(cudaStream_t st, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
// The same for a kernel given by address with its argument array (as cudaLaunchKernel takes).
inline cudaError_t launch_dep_c(cudaStream_t st, const void* k, dim3 grid, dim3 block, size_t smem, void** args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, k, args);
}
#endif

// FP64 <-> FP32 by integer bit operations.  This GPU executes the hardware conversions on its
// FP64 pipe (1/64 of the FP32 rate), which otherwise bounds kernels that convert every operand.
// d2f: round to nearest, ties to even (as a cast); magnitudes below 2^-126 flush to zero,
// overflow to infinity, NaN stays NaN (quiet, sign kept).  f2d: exact for normal numbers, zero,
// infinities and NaN (subnormal floats flush to zero).
__device__ __forceinline__ float d2f(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(u >> 32) & 0x80000000u;
  const unsigned long long v = u & 0x7FFFFFFFFFFFFFFFull;
  if (v > 0x7FF0000000000000ull) return __uint_as_float(sign | 0x7FC00000u);
  // drop 29 mantissa bits: add just under half an ulp, plus one when the kept last bit is odd
  const unsigned long long r = (v + 0x0FFFFFFFull + ((v >> 29) & 1ull)) >> 29;   // exponent | 23 bits
  const unsigned long long lo = 897ull << 23, hi = 1151ull << 23;
  const unsigned int bits = r < lo ? 0u : (r >= hi ? 0x7F800000u : (unsigned int)(r - (896ull << 23)));
  return __uint_as_float(bits | sign);
}
__device__ __forceinline__ double f2d(float x) {
  const unsigned int u = __float_as_uint(x);
  const unsigned int e = (u >> 23) & 0xFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  if (e == 0u) return __longlong_as_double((long long)sign);
  const unsigned long long e64 = e == 255u ? 2047ull : (unsigned long long)e + 896ull;
  return __longlong_as_double((long long)(sign | (e64 << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}
__device__ __forceinline__ float2 d2f(double2 x) { return make_float2(d2f(x.x), d2f(x.y)); }
__device__ __forceinline__ double2 f2d(float2 x) { return make_double2(f2d(x.x), f2d(x.y)); }

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

}  // namespace hw
