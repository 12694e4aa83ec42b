// H X for the helical-wave discretisation (arXiv 2210.12252, Algorithm 5), as three kernels:
//
//   k_radial_inv   gather of the kept coefficients + inverse radial transform
//                  G_{m,n}(r_p) = sum_k xi_{n,k}(r_p) X_{m,n,k}        (Algorithm 1, first loop)
//   k_slab         per radial node and column: inverse angular DFT of the kept (m, n) band,
//                  pointwise multiply by V(theta1, theta2, r_p), forward angular DFT cropped
//                  back to the band                                   (Algorithms 2 and 4)
//   k_radial_fwd   forward radial quadrature + reciprocal-space diagonal + scatter to the
//                  compact order
//                  Y_{m,n,k} = d_{m,n,k} X_{m,n,k} + sum_p O_n[k,p] H_{m,n}(r_p)
//                                                                      (Algorithm 3, Alg. 5)
//
// The intermediates G and H are stored as [column][r_p][pair] with pairs = the (m, n) angular
// pairs kept at any k-point, grouped by |n| so that pairs sharing a radial table are adjacent.
// The forward angular DFT is unnormalised; its 1/(N_th1 N_th2) and the quadrature factor
// 2 pi tau / Ncyc * w_p are folded into the forward radial table.
//
// The angular DFTs are mixed-radix (4, 3, 2) Stockham FFTs in shared memory.  The inverse
// transform is pruned to the kept band: the theta2 pass runs only over the m rows that carry
// kept pairs, the theta1 pass inserts those rows into otherwise-zero columns, and the forward
// pass extracts only the kept bins.  T is double (FP64 path) or float (mixed path); the
// diagonal term is always applied in FP64.
#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <vector>

#include "hw_common.cuh"
#include "hw_ctx.h"
#include "hw_ff.cuh"

namespace hw {

// --------------------------------------------------------------------------- shared FFT
struct FftDev {
  int n, nst;
  int rad[16];
};

// Batched Stockham FFT of `nb` transforms of length `n` stored with row stride n, ping-ponging
// between src and dst; returns the buffer that holds the result.  sign = -1 forward
// (e^{-2 pi i jk/n}), +1 inverse (unnormalised).  tw[t] = e^{-2 pi i t/n}.  Ends with a barrier.
template <typename T>
__device__ cplx_t<T>* fft_batch(cplx_t<T>* src, cplx_t<T>* dst, const FftDev& pl, int nb,
                                const cplx_t<T>* __restrict__ tw, int sign) {
  using V = cplx_t<T>;
  const int n = pl.n;
  int Ns = 1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.rad[s];
    const int nbf = n / R;
    const int tstride = n / (Ns * R);
    for (int idx = threadIdx.x; idx < nb * nbf; idx += blockDim.x) {
      const int b = idx / nbf, j = idx - b * nbf;
      const V* in = src + b * n;
      V* out = dst + b * n;
      const int k = j % Ns;
      V v0 = in[j], v1 = in[j + nbf], v2, v3;
      if (R >= 3) v2 = in[j + 2 * nbf];
      if (R == 4) v3 = in[j + 3 * nbf];
      if (k) {
        V w = tw[k * tstride];
        if (sign > 0) w = cconj(w);
        v1 = cmul(v1, w);
        if (R >= 3) {
          V w2 = tw[2 * k * tstride];
          if (sign > 0) w2 = cconj(w2);
          v2 = cmul(v2, w2);
        }
        if (R == 4) {
          V w3 = tw[3 * k * tstride];
          if (sign > 0) w3 = cconj(w3);
          v3 = cmul(v3, w3);
        }
      }
      const int base = (j / Ns) * Ns * R + k;
      if (R == 2) {
        out[base] = cadd(v0, v1);
        out[base + Ns] = csub(v0, v1);
      } else if (R == 4) {
        V s02 = cadd(v0, v2), d02 = csub(v0, v2);
        V s13 = cadd(v1, v3), d13 = csub(v1, v3);
        V t = cmul_i(d13, sign);  // sign*i*(v1 - v3)
        out[base] = cadd(s02, s13);
        out[base + Ns] = cadd(d02, t);
        out[base + 2 * Ns] = csub(s02, s13);
        out[base + 3 * Ns] = csub(d02, t);
      } else {  // R == 3
        const T h = T(0.86602540378443864676);  // sqrt(3)/2
        V s12 = cadd(v1, v2), d12 = csub(v1, v2);
        V t;
        t.x = v0.x - T(0.5) * s12.x;
        t.y = v0.y - T(0.5) * s12.y;
        V u = cmul_i(d12, sign);  // sign*i*(v1 - v2)
        u.x *= h;
        u.y *= h;
        out[base] = cadd(v0, s12);
        out[base + Ns] = cadd(t, u);
        out[base + 2 * Ns] = csub(t, u);
      }
    }
    __syncthreads();
    V* tmp = src;
    src = dst;
    dst = tmp;
    Ns *= R;
  }
  return src;
}

// The same Stockham passes with the length known at compile time (radix 4 while possible, then
// 3, then 2): divisions, strides and twiddle indices fold to constants, which matters because
// the slab kernel is bound by instruction issue.  Same arithmetic as fft_batch.
// shared-memory index map of the specialised slab's FFT buffers: one pad element after every
// 16, so the strided Stockham reads and writes spread over the banks
__device__ __forceinline__ int pd(int i) { return i + (i >> 4); }
__host__ __device__ inline int pd_size(int n) { return n + (n >> 4) + 1; }

template <typename T, int N, int Ns, bool PAD>
__device__ __forceinline__ void fft_ct_stages(cplx_t<T>*& src, cplx_t<T>*& dst, int nb,
                                              const cplx_t<T>* __restrict__ tw, int sign) {
  using V = cplx_t<T>;
  auto pd = [](int i) { return PAD ? i + (i >> 4) : i; };
  if constexpr (Ns < N) {
    constexpr int Rem = N / Ns;
    constexpr int R = (Rem % 4 == 0) ? 4 : ((Rem % 3 == 0) ? 3 : 2);
    constexpr int nbf = N / R;
    constexpr int tstride = N / (Ns * R);
    for (int idx = threadIdx.x; idx < nb * nbf; idx += blockDim.x) {
      const int b = idx / nbf, j = idx - b * nbf;
      const int ib = b * N;
      const int k = j % Ns;
      V v0 = src[pd(ib + j)], v1 = src[pd(ib + j + nbf)], v2, v3;
      if (R >= 3) v2 = src[pd(ib + j + 2 * nbf)];
      if (R == 4) v3 = src[pd(ib + j + 3 * nbf)];
      if (Ns > 1 && k) {
        V w = tw[k * tstride];
        if (sign > 0) w = cconj(w);
        v1 = cmul(v1, w);
        if (R >= 3) {
          V w2 = tw[2 * k * tstride];
          if (sign > 0) w2 = cconj(w2);
          v2 = cmul(v2, w2);
        }
        if (R == 4) {
          V w3 = tw[3 * k * tstride];
          if (sign > 0) w3 = cconj(w3);
          v3 = cmul(v3, w3);
        }
      }
      const int base = ib + (j / Ns) * Ns * R + k;
      if (R == 2) {
        dst[pd(base)] = cadd(v0, v1);
        dst[pd(base + Ns)] = csub(v0, v1);
      } else if (R == 4) {
        V s02 = cadd(v0, v2), d02 = csub(v0, v2);
        V s13 = cadd(v1, v3), d13 = csub(v1, v3);
        V t = cmul_i(d13, sign);
        dst[pd(base)] = cadd(s02, s13);
        dst[pd(base + Ns)] = cadd(d02, t);
        dst[pd(base + 2 * Ns)] = csub(s02, s13);
        dst[pd(base + 3 * Ns)] = csub(d02, t);
      } else {
        const T h = T(0.86602540378443864676);
        V s12 = cadd(v1, v2), d12 = csub(v1, v2);
        V t;
        t.x = v0.x - T(0.5) * s12.x;
        t.y = v0.y - T(0.5) * s12.y;
        V u = cmul_i(d12, sign);
        u.x *= h;
        u.y *= h;
        dst[pd(base)] = cadd(v0, s12);
        dst[pd(base + Ns)] = cadd(t, u);
        dst[pd(base + 2 * Ns)] = csub(t, u);
      }
    }
    __syncthreads();
    V* tmp = src;
    src = dst;
    dst = tmp;
    fft_ct_stages<T, N, Ns * R, PAD>(src, dst, nb, tw, sign);
  }
}

// length N at compile time when N > 0, else the runtime plan; PAD: buffers addressed through pd
template <typename T, int N, bool PAD>
__device__ __forceinline__ cplx_t<T>* fft_any(cplx_t<T>* src, cplx_t<T>* dst, const FftDev& pl, int nb,
                                              const cplx_t<T>* __restrict__ tw, int sign) {
  if constexpr (N > 0) {
    fft_ct_stages<T, N, 1, PAD>(src, dst, nb, tw, sign);
    return src;
  } else {
    return fft_batch<T>(src, dst, pl, nb, tw, sign);
  }
}

// --------------------------------------------------------------------------- radial inverse
template <typename T>
struct RadArgs {
  int Nr, K, nA, ncols, ns, c0;   // ncols columns of this pass start at global column c0;
                                  // global column c belongs to block c / ns, column c % ns
  const int* group_start;     // [N+2] pair range of each |n| group
  const int* off;             // [nk][nA]
  const int* Ka;              // [nk][nA]
  int64_t ld;
  const T* rtab;              // inverse [(N+1)][Nr][K] or forward [(N+1)][K][Nr]
  const double* ke;           // concatenated shifted kinetic energies (forward only)
  int64_t keoff[MAXSLOT];     // start of each block's k-point in ke
  // nu != 0 terms (forward only): qtab [(N+1)][K][K] = <F_k', F_k / r^2>, the signed order n
  // of every pair, the cyclic order and each block's nu
  const T* qtab;
  const int* pair_n;
  int ncyc;
  int any_nu;                 // some block of this launch has nu != 0
  double nu[MAXSLOT];
  // forward only: a fused recurrence step (y = al (H x - c x) - be y), or none
  int step;
  ChebStep cs;
  // inverse only: coefficients multiplied by i 2 pi m (scale_mode 1) or i 2 pi n Ncyc (2)
  // before the transform (the theta derivatives of Appendix C); 0: as they are
  int scale_mode;
  const int* pair_mrow;
  const int* mrow_m;
  cplx_t<T>* gh;              // G (inverse output) or H (forward input)
  Blocks blk;
};

constexpr int RAD_Q = 64;   // (column, pair) items per CTA
constexpr int RAD_THREADS = 256;

// table rows padded to a multiple of 4 entries (zeros), so that 4 consecutive entries load as
// one (FP32) or two (FP64) 16-byte shared-memory words
__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }

__device__ __forceinline__ void ld4(const float* p, float& a, float& b, float& c, float& d) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = v.x;
  b = v.y;
  c = v.z;
  d = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c, double& d) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
  a = v0.x;
  b = v0.y;
  c = v1.x;
  d = v1.y;
}

// dynamic shared memory of k_radial_inv / k_radial_fwd
inline size_t rad_inv_smem(int Nr, int K, size_t tsz) {
  return (((size_t)Nr * pad4(K) * tsz + 15) & ~size_t(15)) + (size_t)pad4(K) * RAD_Q * 2 * tsz;
}
inline size_t rad_fwd_smem(int Nr, int K, size_t tsz) {
  return (((size_t)K * pad4(Nr) * tsz + 15) & ~size_t(15)) + 32 * RAD_Q * 2 * tsz + (size_t)RAD_Q * (K + 1) * 2 * tsz;
}

// grid: x = tile of items within group g, y = g.  Items of group g are (c, a) with
// a in [gs, ge), flattened as c * na + (a - gs).  Each thread keeps the values of a block of
// radial nodes of one item in registers; the table rows are read 4 entries at a time (the same
// row for every lane of a warp: one broadcast word), the item's coefficients 4 at a time.
template <typename T>
__global__ void __launch_bounds__(RAD_THREADS, sizeof(T) == 4 ? 2 : 1) k_radial_inv(RadArgs<T> A) {
  griddep_entry();
  using V = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = blockIdx.y;
  const int gs = A.group_start[g], na = A.group_start[g + 1] - gs;
  const long nitems = (long)na * A.ncols;
  const long q0 = (long)blockIdx.x * RAD_Q;
  if (na == 0 || q0 >= nitems) return;
  const int K = A.K, Nr = A.Nr, Kp = pad4(K);
  T* Rs = reinterpret_cast<T*>(smem_raw);                 // [Nr][Kp]
  V* Xs = reinterpret_cast<V*>(smem_raw + (((size_t)Nr * Kp * sizeof(T) + 15) & ~size_t(15)));  // [Kp][RAD_Q]
  const T* tab = A.rtab + (size_t)g * Nr * K;
  for (int i = threadIdx.x; i < Nr * Kp; i += blockDim.x) {
    const int p = i / Kp, k = i - p * Kp;
    Rs[i] = k < K ? tab[(size_t)p * K + k] : T(0);
  }
  // per item: where its kept coefficients start, how many there are, and the derivative scale
  // (one thread per item, so the element loop below has no dependent index loads)
  __shared__ const double* s_x[RAD_Q];
  __shared__ int s_ka[RAD_Q];
  __shared__ T s_sc[RAD_Q];
  if (threadIdx.x < RAD_Q) {
    const int q = threadIdx.x;
    const long item = q0 + q;
    const double* xp = nullptr;
    int ka = 0;
    T sc = T(0);
    if (item < nitems) {
      const int c = (int)(item / na), a = gs + (int)(item - (long)c * na);
      const int cg = A.c0 + c;
      const int slot = cg / A.ns, sl = cg - slot * A.ns;
      const int kb = A.blk.kb[slot];
      ka = A.Ka[(size_t)kb * A.nA + a];
      xp = A.blk.x[slot] + 2 * ((size_t)A.off[(size_t)kb * A.nA + a] + (size_t)sl * A.ld);
      if (A.scale_mode != 0)
        sc = T(6.283185307179586 * (A.scale_mode == 1 ? (double)A.mrow_m[A.pair_mrow[a]]
                                                       : (double)A.pair_n[a] * A.ncyc));
    }
    s_x[q] = xp;
    s_ka[q] = ka;
    s_sc[q] = sc;
  }
  __syncthreads();
  // gather the kept coefficients of each item (zero beyond Ka); independent loads, unrolled
#pragma unroll 4
  for (int i = threadIdx.x; i < RAD_Q * Kp; i += blockDim.x) {
    const int q = i / Kp, k = i - q * Kp;
    V v = mk<T>(T(0), T(0));
    if (k < s_ka[q]) {
      const double* x = s_x[q] + 2 * k;
      if constexpr (sizeof(T) == 4)
        v = mk<T>(d2f(x[0]), d2f(x[1]));
      else
        v = mk<T>(x[0], x[1]);
      if (A.scale_mode != 0) {   // times i s
        const T sc = s_sc[q];
        v = mk<T>(-sc * v.y, sc * v.x);
      }
    }
    Xs[k * RAD_Q + q] = v;
  }
  __syncthreads();
  const int q = threadIdx.x % RAD_Q;
  const long item = q0 + q;
  if (item >= nitems) return;
  const int c = (int)(item / na), a = gs + (int)(item - (long)c * na);
  V* out = A.gh + ((size_t)c * Nr) * A.nA + a;
  constexpr int PG = RAD_THREADS / RAD_Q;            // node groups
  if constexpr (sizeof(T) == 8) {
    // FP64: bound by the FP64 pipe; one node at a time keeps more CTAs resident
    for (int p = threadIdx.x / RAD_Q; p < Nr; p += PG) {
      T ax = 0, ay = 0;
      const T* rr = Rs + (size_t)p * Kp;
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        const V xv = Xs[k * RAD_Q + q];
        ax += rr[k] * xv.x;
        ay += rr[k] * xv.y;
      }
      out[(size_t)p * A.nA] = mk<T>(ax, ay);
    }
    return;
  }
  constexpr int PP = 12;                             // nodes per register block
  for (int pb = (threadIdx.x / RAD_Q) * PP; pb < Nr; pb += PG * PP) {
    T ax[PP], ay[PP];
#pragma unroll
    for (int i = 0; i < PP; ++i) ax[i] = ay[i] = T(0);
    for (int k0 = 0; k0 < Kp; k0 += 4) {
      const V x0 = Xs[k0 * RAD_Q + q], x1 = Xs[(k0 + 1) * RAD_Q + q];
      const V x2 = Xs[(k0 + 2) * RAD_Q + q], x3 = Xs[(k0 + 3) * RAD_Q + q];
#pragma unroll
      for (int i = 0; i < PP; ++i) {
        const int p = min(pb + i, Nr - 1);   // nodes past Nr are computed, not stored
        T r0, r1, r2, r3;
        ld4(Rs + (size_t)p * Kp + k0, r0, r1, r2, r3);
        ax[i] += r0 * x0.x + r1 * x1.x + r2 * x2.x + r3 * x3.x;
        ay[i] += r0 * x0.y + r1 * x1.y + r2 * x2.y + r3 * x3.y;
      }
    }
#pragma unroll
    for (int i = 0; i < PP; ++i)
      if (pb + i < Nr) out[(size_t)(pb + i) * A.nA] = mk<T>(ax[i], ay[i]);
  }
}

// store H x (hx, hy) for one coefficient, or the fused recurrence step of A.step
template <typename T>
__device__ __forceinline__ void step_store(const RadArgs<T>& A, int slot, double* y, double x0, double x1,
                                           double hx, double hy) {
  if (A.step) {
    const double al = A.cs.al[slot], c = A.cs.c[slot], be = A.cs.be[slot];
    hx = al * (hx - c * x0);
    hy = al * (hy - c * x1);
    if (be != 0.0) {
      hx -= be * y[0];
      hy -= be * y[1];
    }
  }
  y[0] = hx;
  y[1] = hy;
}

// forward radial quadrature + diagonal term + scatter
template <typename T>
__global__ void __launch_bounds__(RAD_THREADS, sizeof(T) == 4 ? 2 : 1) k_radial_fwd(RadArgs<T> A) {
  griddep_entry();
  using V = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = blockIdx.y;
  const int gs = A.group_start[g], na = A.group_start[g + 1] - gs;
  const long nitems = (long)na * A.ncols;
  const long q0 = (long)blockIdx.x * RAD_Q;
  if (na == 0 || q0 >= nitems) return;
  const int K = A.K, Nr = A.Nr, Nrp = pad4(Nr);
  constexpr int PC = 32;                                   // radial nodes per chunk
  T* Rs = reinterpret_cast<T*>(smem_raw);                  // [K][Nrp]
  size_t o = (((size_t)K * Nrp * sizeof(T)) + 15) & ~size_t(15);
  V* Hs = reinterpret_cast<V*>(smem_raw + o);              // [PC][RAD_Q]
  o += (size_t)PC * RAD_Q * sizeof(V);
  V* Ys = reinterpret_cast<V*>(smem_raw + o);              // [RAD_Q][K+1]
  const T* tab = A.rtab + (size_t)g * K * Nr;
  for (int i = threadIdx.x; i < K * Nrp; i += blockDim.x) {
    const int k = i / Nrp, pp = i - k * Nrp;
    Rs[i] = pp < Nr ? tab[(size_t)k * Nr + pp] : T(0);
  }
  // per item: its H column (the (r, pair) intermediate at r_0), its coefficient offset in X / Y,
  // block slot and kept count (one thread per item; the loops below index these from shared
  // memory instead of chains of dependent global loads)
  __shared__ const V* s_h[RAD_Q];
  __shared__ int64_t s_o[RAD_Q], s_cs[RAD_Q];
  __shared__ int s_ka[RAD_Q], s_slot[RAD_Q];
  if (threadIdx.x < RAD_Q) {
    const int qq = threadIdx.x;
    const long it = q0 + qq;
    const V* hp = nullptr;
    int64_t o = 0, cs = 0;
    int ka = 0, slot = 0, aa = gs;
    if (it < nitems) {
      const int cc = (int)(it / na);
      aa = gs + (int)(it - (long)cc * na);
      const int cg = A.c0 + cc;
      slot = cg / A.ns;
      const int sl = cg - slot * A.ns;
      const int kb = A.blk.kb[slot];
      ka = A.Ka[(size_t)kb * A.nA + aa];
      o = (int64_t)A.off[(size_t)kb * A.nA + aa];
      cs = (int64_t)sl * A.ld;
      hp = A.gh + (size_t)cc * Nr * A.nA + aa;
    }
    s_h[qq] = hp;
    s_o[qq] = o;
    s_cs[qq] = cs;
    s_ka[qq] = ka;
    s_slot[qq] = slot;
  }
  __syncthreads();
  const int q = threadIdx.x % RAD_Q;
  const int kg = threadIdx.x / RAD_Q;                      // 4 groups of k
  constexpr int KG = RAD_THREADS / RAD_Q;
  const long item = q0 + q;
  int c = 0, a = gs;
  if (item < nitems) {
    c = (int)(item / na);
    a = gs + (int)(item - (long)c * na);
  }
  T acc[2 * 16];  // up to 16 k per thread: K <= 64
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = 0;
  const int kper = (K + KG - 1) / KG;
  for (int p0 = 0; p0 < Nr; p0 += PC) {
    const int pc = min(PC, Nr - p0);
    __syncthreads();
#pragma unroll 4
    for (int i = threadIdx.x; i < PC * RAD_Q; i += blockDim.x) {   // zero past pc
      const int pp = i / RAD_Q, qq = i - pp * RAD_Q;
      V v = mk<T>(T(0), T(0));
      const V* hp = s_h[qq];
      if (hp && pp < pc) v = hp[(size_t)(p0 + pp) * A.nA];
      Hs[pp * RAD_Q + qq] = v;
    }
    __syncthreads();
    if constexpr (sizeof(T) == 8) {   // FP64: one node at a time (bound by the FP64 pipe)
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int k = kg + j * KG;
        if (j < kper && k < K) {
          T ax = acc[2 * j], ay = acc[2 * j + 1];
          const T* rr = Rs + (size_t)k * Nrp + p0;
          for (int pp = 0; pp < pc; ++pp) {
            const V hv = Hs[pp * RAD_Q + q];
            ax += rr[pp] * hv.x;
            ay += rr[pp] * hv.y;
          }
          acc[2 * j] = ax;
          acc[2 * j + 1] = ay;
        }
      }
      continue;
    }
    // 4 nodes at a time: the item's 4 values once, each table row's 4 entries as one word
    for (int pp = 0; pp < pc; pp += 4) {
      const V h0 = Hs[pp * RAD_Q + q], h1 = Hs[(pp + 1) * RAD_Q + q];
      const V h2 = Hs[(pp + 2) * RAD_Q + q], h3 = Hs[(pp + 3) * RAD_Q + q];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int k = kg + j * KG;
        if (j < kper && k < K) {
          T r0, r1, r2, r3;
          ld4(Rs + (size_t)k * Nrp + p0 + pp, r0, r1, r2, r3);
          acc[2 * j] += r0 * h0.x + r1 * h1.x + r2 * h2.x + r3 * h3.x;
          acc[2 * j + 1] += r0 * h0.y + r1 * h1.y + r2 * h2.y + r3 * h3.y;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int k = kg + j * KG;
    if (j < kper && k < K) Ys[q * (K + 1) + k] = mk<T>(acc[2 * j], acc[2 * j + 1]);
  }
  __syncthreads();
  if (!A.any_nu) {
    // scatter without nu terms: (item, k) pairs over all threads, several independent global
    // round trips in flight per thread
#pragma unroll 4
    for (int idx = threadIdx.x; idx < RAD_Q * K; idx += RAD_THREADS) {
      const int qq = idx / K, k = idx - qq * K;
      if (k >= s_ka[qq]) continue;
      const int slot = s_slot[qq];
      const int64_t o = s_o[qq] + k;   // compact index of coefficient k of the item
      const double* x = A.blk.x[slot] + 2 * (o + s_cs[qq]);   // 8-byte aligned (ABI)
      double* y = A.blk.y[slot] + 2 * (o + s_cs[qq]);
      const double d = A.ke[A.keoff[slot] + o];
      const V h = Ys[qq * (K + 1) + k];
      const double x0 = x[0], x1 = x[1];
      double y0 = d * x0 + double(h.x), y1 = d * x1 + double(h.y);
      if (A.step) {
        const double al = A.cs.al[slot], cc2 = A.cs.c[slot], be = A.cs.be[slot];
        y0 = al * (y0 - cc2 * x0);
        y1 = al * (y1 - cc2 * x1);
        if (be != 0.0) {
          y0 -= be * y[0];
          y1 -= be * y[1];
        }
      }
      y[0] = y0;
      y[1] = y1;
    }
    return;
  }
  // scatter: one warp per item, lanes over k (contiguous in the compact order)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int qq = warp; qq < RAD_Q; qq += RAD_THREADS / 32) {
    const long it = q0 + qq;
    if (it >= nitems) break;
    const int cc = (int)(it / na), aa = gs + (int)(it - (long)cc * na);
    const int cg = A.c0 + cc;
    const int slot = cg / A.ns, s = cg - slot * A.ns;
    const int kb = A.blk.kb[slot];
    const int ka = A.Ka[(size_t)kb * A.nA + aa];
    const size_t o0 = (size_t)A.off[(size_t)kb * A.nA + aa];
    const double* x = A.blk.x[slot] + 2 * (o0 + (size_t)s * A.ld);
    double* y = A.blk.y[slot] + 2 * (o0 + (size_t)s * A.ld);
    const double* ke = A.ke + A.keoff[slot] + o0;
    const double nu = A.nu[slot];
    if (nu == 0.0) {
      for (int k = lane; k < ka; k += 32) {
        const V h = Ys[qq * (K + 1) + k];
        const double d = ke[k];
        step_store(A, slot, y + 2 * k, x[2 * k], x[2 * k + 1], d * x[2 * k] + double(h.x),
                   d * x[2 * k + 1] + double(h.y));
      }
      continue;
    }
    // nu != 0: the 1/r^2 terms of the I_n loop of Algorithm 5, which combine to
    // (nu^2 - 2 nu n Ncyc)/2 <F_k', F_k / r^2> within the pair (m, n): lanes hold the pair's
    // coefficients k = lane, lane + 32 (ka <= K <= 64) and broadcast them by shuffles
    const T cf = T(0.5 * nu * (nu - 2.0 * (double)A.pair_n[aa] * A.ncyc));
    const T* qt = A.qtab + (size_t)g * K * K;
    V x0 = mk<T>(T(0), T(0)), x1 = mk<T>(T(0), T(0));
    if (lane < ka) x0 = mk<T>(T(x[2 * lane]), T(x[2 * lane + 1]));
    if (lane + 32 < ka) x1 = mk<T>(T(x[2 * (lane + 32)]), T(x[2 * (lane + 32) + 1]));
    for (int kb = 0; kb < ka; kb += 32) {
      const int k = kb + lane;
      const T* qr = qt + (size_t)(k < ka ? k : 0) * K;
      T sx = 0, sy = 0;
      for (int j = 0; j < ka; ++j) {
        const V xj = j < 32 ? x0 : x1;
        const T vx = __shfl_sync(0xffffffffu, xj.x, j & 31);
        const T vy = __shfl_sync(0xffffffffu, xj.y, j & 31);
        const T qv = qr[j];
        sx += qv * vx;
        sy += qv * vy;
      }
      if (k < ka) {
        const V h = Ys[qq * (K + 1) + k];
        const double d = ke[k];
        step_store(A, slot, y + 2 * k, x[2 * k], x[2 * k + 1], d * x[2 * k] + double(h.x + cf * sx),
                   d * x[2 * k + 1] + double(h.y + cf * sy));
      }
    }
  }
}

// ------------------------------------------------------------ radial transforms, double-float
// The FP64 H X of a mixed-precision solve in double-float arithmetic (the angular kernel's
// `ff`), nu = 0: the tables as FP32 pairs, the G / H intermediates stored as pairs (the same 16
// bytes per complex value as complex128), X read and Y written in FP64 with the diagonal term
// in FP64.  Item and table layout as k_radial_inv / k_radial_fwd; one node per thread at a time.
__global__ void __launch_bounds__(RAD_THREADS, 2) k_radial_inv_ff(RadArgs<double> A, const ff* __restrict__ tabff) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = blockIdx.y;
  const int gs = A.group_start[g], na = A.group_start[g + 1] - gs;
  const long nitems = (long)na * A.ncols;
  const long q0 = (long)blockIdx.x * RAD_Q;
  if (na == 0 || q0 >= nitems) return;
  const int K = A.K, Nr = A.Nr, Kp = pad4(K);
  ff* Rs = reinterpret_cast<ff*>(smem_raw);   // [Nr][Kp]
  ffc* Xs = reinterpret_cast<ffc*>(smem_raw + (((size_t)Nr * Kp * sizeof(ff) + 15) & ~size_t(15)));   // [Kp][RAD_Q]
  const ff* tab = tabff + (size_t)g * Nr * K;
  for (int i = threadIdx.x; i < Nr * Kp; i += blockDim.x) {
    const int p = i / Kp, k = i - p * Kp;
    Rs[i] = k < K ? tab[(size_t)p * K + k] : ff(0);
  }
  __shared__ const double* s_x[RAD_Q];
  __shared__ int s_ka[RAD_Q];
  if (threadIdx.x < RAD_Q) {
    const int q = threadIdx.x;
    const long item = q0 + q;
    const double* xp = nullptr;
    int ka = 0;
    if (item < nitems) {
      const int c = (int)(item / na), a = gs + (int)(item - (long)c * na);
      const int cg = A.c0 + c;
      const int slot = cg / A.ns, sl = cg - slot * A.ns;
      const int kb = A.blk.kb[slot];
      ka = A.Ka[(size_t)kb * A.nA + a];
      xp = A.blk.x[slot] + 2 * ((size_t)A.off[(size_t)kb * A.nA + a] + (size_t)sl * A.ld);
    }
    s_x[q] = xp;
    s_ka[q] = ka;
  }
  __syncthreads();
#pragma unroll 4
  for (int i = threadIdx.x; i < RAD_Q * Kp; i += blockDim.x) {
    const int q = i / Kp, k = i - q * Kp;
    ffc v;
    v.x = ff(0);
    v.y = ff(0);
    if (k < s_ka[q]) {
      const double* x = s_x[q] + 2 * k;
      v.x = ff_from(x[0]);
      v.y = ff_from(x[1]);
    }
    Xs[k * RAD_Q + q] = v;
  }
  __syncthreads();
  const int q = threadIdx.x % RAD_Q;
  const long item = q0 + q;
  if (item >= nitems) return;
  const int c = (int)(item / na), a = gs + (int)(item - (long)c * na);
  ffc* out = reinterpret_cast<ffc*>(A.gh) + ((size_t)c * Nr) * A.nA + a;
  constexpr int PG = RAD_THREADS / RAD_Q;
  for (int p = threadIdx.x / RAD_Q; p < Nr; p += PG) {
    ff ax = ff(0), ay = ff(0);
    const ff* rr = Rs + (size_t)p * Kp;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
      const ffc xv = Xs[k * RAD_Q + q];
      ax += rr[k] * xv.x;
      ay += rr[k] * xv.y;
    }
    ffc o;
    o.x = ax;
    o.y = ay;
    out[(size_t)p * A.nA] = o;
  }
}

__global__ void __launch_bounds__(RAD_THREADS, 2) k_radial_fwd_ff(RadArgs<double> A, const ff* __restrict__ tabff) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = blockIdx.y;
  const int gs = A.group_start[g], na = A.group_start[g + 1] - gs;
  const long nitems = (long)na * A.ncols;
  const long q0 = (long)blockIdx.x * RAD_Q;
  if (na == 0 || q0 >= nitems) return;
  const int K = A.K, Nr = A.Nr, Nrp = pad4(Nr);
  constexpr int PC = 32;
  ff* Rs = reinterpret_cast<ff*>(smem_raw);                // [K][Nrp]
  size_t o = (((size_t)K * Nrp * sizeof(ff)) + 15) & ~size_t(15);
  ffc* Hs = reinterpret_cast<ffc*>(smem_raw + o);          // [PC][RAD_Q]
  o += (size_t)PC * RAD_Q * sizeof(ffc);
  ffc* Ys = reinterpret_cast<ffc*>(smem_raw + o);          // [RAD_Q][K+1]
  const ff* tab = tabff + (size_t)g * K * Nr;
  for (int i = threadIdx.x; i < K * Nrp; i += blockDim.x) {
    const int k = i / Nrp, pp = i - k * Nrp;
    Rs[i] = pp < Nr ? tab[(size_t)k * Nr + pp] : ff(0);
  }
  __shared__ const ffc* s_h[RAD_Q];
  __shared__ int64_t s_o[RAD_Q], s_cs[RAD_Q];
  __shared__ int s_ka[RAD_Q], s_slot[RAD_Q];
  if (threadIdx.x < RAD_Q) {
    const int qq = threadIdx.x;
    const long it = q0 + qq;
    const ffc* hp = nullptr;
    int64_t oo = 0, cs = 0;
    int ka = 0, slot = 0;
    if (it < nitems) {
      const int cc = (int)(it / na), aa = gs + (int)(it - (long)cc * na);
      const int cg = A.c0 + cc;
      slot = cg / A.ns;
      const int sl = cg - slot * A.ns;
      const int kb = A.blk.kb[slot];
      ka = A.Ka[(size_t)kb * A.nA + aa];
      oo = (int64_t)A.off[(size_t)kb * A.nA + aa];
      cs = (int64_t)sl * A.ld;
      hp = reinterpret_cast<const ffc*>(A.gh) + (size_t)cc * Nr * A.nA + aa;
    }
    s_h[qq] = hp;
    s_o[qq] = oo;
    s_cs[qq] = cs;
    s_ka[qq] = ka;
    s_slot[qq] = slot;
  }
  __syncthreads();
  const int q = threadIdx.x % RAD_Q;
  const int kg = threadIdx.x / RAD_Q;
  constexpr int KG = RAD_THREADS / RAD_Q;
  ff acc[2 * 16];   // up to 16 k per thread: K <= 64
#pragma unroll
  for (int i = 0; i < 32; ++i) acc[i] = ff(0);
  const int kper = (K + KG - 1) / KG;
  for (int p0 = 0; p0 < Nr; p0 += PC) {
    const int pc = min(PC, Nr - p0);
    __syncthreads();
#pragma unroll 4
    for (int i = threadIdx.x; i < PC * RAD_Q; i += blockDim.x) {
      const int pp = i / RAD_Q, qq = i - pp * RAD_Q;
      ffc v;
      v.x = ff(0);
      v.y = ff(0);
      const ffc* hp = s_h[qq];
      if (hp && pp < pc) v = hp[(size_t)(p0 + pp) * A.nA];
      Hs[pp * RAD_Q + qq] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = kg + j * KG;
      if (j < kper && k < K) {
        ff ax = acc[2 * j], ay = acc[2 * j + 1];
        const ff* rr = Rs + (size_t)k * Nrp + p0;
        for (int pp = 0; pp < pc; ++pp) {
          const ffc hv = Hs[pp * RAD_Q + q];
          ax += rr[pp] * hv.x;
          ay += rr[pp] * hv.y;
        }
        acc[2 * j] = ax;
        acc[2 * j + 1] = ay;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int k = kg + j * KG;
    if (j < kper && k < K) {
      ffc v;
      v.x = acc[2 * j];
      v.y = acc[2 * j + 1];
      Ys[q * (K + 1) + k] = v;
    }
  }
  __syncthreads();
#pragma unroll 4
  for (int idx = threadIdx.x; idx < RAD_Q * K; idx += RAD_THREADS) {
    const int qq = idx / K, k = idx - qq * K;
    if (k >= s_ka[qq]) continue;
    const int slot = s_slot[qq];
    const int64_t oo = s_o[qq] + k;
    const double* x = A.blk.x[slot] + 2 * (oo + s_cs[qq]);
    double* y = A.blk.y[slot] + 2 * (oo + s_cs[qq]);
    const double d = A.ke[A.keoff[slot] + oo];
    const ffc h = Ys[qq * (K + 1) + k];
    const double x0 = x[0], x1 = x[1];
    double y0 = d * x0 + ff_to(h.x), y1 = d * x1 + ff_to(h.y);
    if (A.step) {
      const double al = A.cs.al[slot], cc2 = A.cs.c[slot], be = A.cs.be[slot];
      y0 = al * (y0 - cc2 * x0);
      y1 = al * (y1 - cc2 * x1);
      if (be != 0.0) {
        y0 -= be * y[0];
        y1 -= be * y[1];
      }
    }
    y[0] = y0;
    y[1] = y1;
  }
}

// --------------------------------------------------------------------------- slab
template <typename T>
struct SlabArgs {
  int Nr, Nth1, Nth2, nA, nmr, ncols, Jc;
  FftDev p1, p2;
  const int* pair_n;
  const int* pair_mrow;
  const int* mrow_m;
  const int* slot_pair;   // [nmr][Nth2]: pair index or -1 (the lane-split slab only)
  const T* V;        // [Nr][Nth2][Nth1]
  const cplx_t<T>* tw1;
  const cplx_t<T>* tw2;
  const cplx_t<T>* G;
  cplx_t<T>* H;
};

constexpr int SLAB_THREADS = 256;

// grid: x = column, y = radial node.  N1, N2 > 0: grid sizes fixed at compile time (the
// kernel is then specialised for them); 0: taken from A.
template <typename T, int N1 = 0, int N2 = 0>
__global__ void __launch_bounds__(SLAB_THREADS) k_slab(SlabArgs<T> A) {
  griddep_entry();
  using V = cplx_t<T>;
  // the specialised FP32 FFTs address their buffers through pd (16-byte FP64 elements spread
  // over the banks already; padding them measured slower)
  constexpr bool PAD = N1 > 0 && sizeof(T) == sizeof(float);
  auto ix = [](int i) { return PAD ? pd(i) : i; };
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x, p = blockIdx.y;
  const int n1 = N1 > 0 ? N1 : A.Nth1, n2 = N2 > 0 ? N2 : A.Nth2, nmr = A.nmr;
  const int n2p = PAD ? n2 + 1 : n2;   // row stride of Tb
  const int wsz = PAD ? pd_size(max(nmr * n2, A.Jc * n1)) : max(nmr * n2, A.Jc * n1);
  V* Tb = reinterpret_cast<V*>(smem_raw);     // [nmr][n2p]
  V* W0 = Tb + nmr * n2p;
  V* W1 = W0 + wsz;
  const V zero = mk<T>(T(0), T(0));
  const V* Gc = A.G + ((size_t)c * A.Nr + p) * A.nA;
  V* Hc = A.H + ((size_t)c * A.Nr + p) * A.nA;
  // theta2 inverse pass over the kept m rows
  for (int i = threadIdx.x; i < nmr * n2; i += blockDim.x) W0[ix(i)] = zero;
  __syncthreads();
  for (int a = threadIdx.x; a < A.nA; a += blockDim.x)
    W0[ix(A.pair_mrow[a] * n2 + pmod(A.pair_n[a], n2))] = Gc[a];
  __syncthreads();
  V* r = fft_any<T, N2, PAD>(W0, W1, A.p2, nmr, A.tw2, +1);
  for (int i = threadIdx.x; i < nmr * n2; i += blockDim.x) {
    const int rr = i / n2, jj = i - rr * n2;
    Tb[rr * n2p + jj] = r[ix(i)];
  }
  __syncthreads();
  // theta1 pass per theta2 column chunk: insert rows, inverse FFT, x V, forward FFT, extract
  const T* Vp = A.V + (size_t)p * n2 * n1;
  for (int j0 = 0; j0 < n2; j0 += A.Jc) {
    const int jn = min(A.Jc, n2 - j0);
    for (int i = threadIdx.x; i < jn * n1; i += blockDim.x) W0[ix(i)] = zero;
    __syncthreads();
    for (int i = threadIdx.x; i < jn * nmr; i += blockDim.x) {
      const int jj = i / nmr, rr = i - jj * nmr;
      W0[ix(jj * n1 + pmod(A.mrow_m[rr], n1))] = Tb[rr * n2p + j0 + jj];
    }
    __syncthreads();
    V* u = fft_any<T, N1, PAD>(W0, W1, A.p1, jn, A.tw1, +1);
    for (int i = threadIdx.x; i < jn * n1; i += blockDim.x) {
      const T v = Vp[(size_t)j0 * n1 + i];
      V x = u[ix(i)];
      x.x *= v;
      x.y *= v;
      u[ix(i)] = x;
    }
    __syncthreads();
    V* w = fft_any<T, N1, PAD>(u, u == W0 ? W1 : W0, A.p1, jn, A.tw1, -1);
    for (int i = threadIdx.x; i < jn * nmr; i += blockDim.x) {
      const int jj = i / nmr, rr = i - jj * nmr;
      Tb[rr * n2p + j0 + jj] = w[ix(jj * n1 + pmod(A.mrow_m[rr], n1))];
    }
    __syncthreads();
  }
  // theta2 forward pass, extract the kept pairs
  for (int i = threadIdx.x; i < nmr * n2; i += blockDim.x) {
    const int rr = i / n2, jj = i - rr * n2;
    W0[ix(i)] = Tb[rr * n2p + jj];
  }
  __syncthreads();
  r = fft_any<T, N2, PAD>(W0, W1, A.p2, nmr, A.tw2, -1);
  for (int a = threadIdx.x; a < A.nA; a += blockDim.x)
    Hc[a] = r[ix(A.pair_mrow[a] * n2 + pmod(A.pair_n[a], n2))];
}

// 16-point DFT in registers, X[k] = sum_n x[n] W^(S n k), W = e^{2 pi i / 16}, as two radix-4
// passes (n = 4 n1 + n2, k = k1 + 4 k2) with the twiddles W^(S n2 k1) between them
template <int S, typename R>
__device__ __forceinline__ void dft16(R (&xr)[16], R (&xi)[16]) {
  constexpr R C8 = R(0.923879532511286756128183189396788933), S8 = R(0.382683432365089771728459984030398866);
  constexpr R R2 = R(0.707106781186547524400844362104849039);
  // W^e for e = 0..9 (cos, sin); forward (S = -1) takes the conjugates
  constexpr R wc[10] = {R(1), C8, R2, S8, R(0), -S8, -R2, -C8, R(-1), -C8};
  constexpr R ws[10] = {R(0), S8, R2, C8, R(1), C8, R2, S8, R(0), -S8};
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {   // 4-point DFTs over n1
    const R a0r = xr[n2], a0i = xi[n2], a1r = xr[4 + n2], a1i = xi[4 + n2];
    const R a2r = xr[8 + n2], a2i = xi[8 + n2], a3r = xr[12 + n2], a3i = xi[12 + n2];
    const R t0r = a0r + a2r, t0i = a0i + a2i, t1r = a0r - a2r, t1i = a0i - a2i;
    const R t2r = a1r + a3r, t2i = a1i + a3i;
    const R dr = a1r - a3r, di = a1i - a3i;
    const R t3r = -S * di, t3i = S * dr;   // (a1 - a3) (S i)
    xr[n2] = t0r + t2r;
    xi[n2] = t0i + t2i;
    xr[4 + n2] = t1r + t3r;
    xi[4 + n2] = t1i + t3i;
    xr[8 + n2] = t0r - t2r;
    xi[8 + n2] = t0i - t2i;
    xr[12 + n2] = t1r - t3r;
    xi[12 + n2] = t1i - t3i;
  }
#pragma unroll
  for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2) {   // twiddle W^(S n2 k1)
      const int e = n2 * k1;
      const R c = wc[e], sn = S * ws[e];
      const R r = xr[4 * k1 + n2], i = xi[4 * k1 + n2];
      xr[4 * k1 + n2] = r * c - i * sn;
      xi[4 * k1 + n2] = r * sn + i * c;
    }
  R orr[16], oi[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {   // 4-point DFTs over n2
    const R a0r = xr[4 * k1], a0i = xi[4 * k1], a1r = xr[4 * k1 + 1], a1i = xi[4 * k1 + 1];
    const R a2r = xr[4 * k1 + 2], a2i = xi[4 * k1 + 2], a3r = xr[4 * k1 + 3], a3i = xi[4 * k1 + 3];
    const R t0r = a0r + a2r, t0i = a0i + a2i, t1r = a0r - a2r, t1i = a0i - a2i;
    const R t2r = a1r + a3r, t2i = a1i + a3i;
    const R dr = a1r - a3r, di = a1i - a3i;
    const R t3r = -S * di, t3i = S * dr;
    orr[k1] = t0r + t2r;
    oi[k1] = t0i + t2i;
    orr[k1 + 4] = t1r + t3r;
    oi[k1 + 4] = t1i + t3i;
    orr[k1 + 8] = t0r - t2r;
    oi[k1 + 8] = t0i - t2i;
    orr[k1 + 12] = t1r - t3r;
    oi[k1 + 12] = t1i - t3i;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    xr[k] = orr[k];
    xi[k] = oi[k];
  }
}

// Slab for the 64 x 48 angular grid with the theta1 transforms split 64 = 4 x 16 over the
// 4 lanes of a theta2 row: lane q owns the points i = 4 t + q (t = 0..15).  With omega =
// e^{2 pi i / 64} and W = omega^4, a kept row m contributes T_m omega^(m q) W^(m t) to point
// 4 t + q, so the inverse transform is, per lane, the 16-point inverse DFT of the bins
// b = m mod 16 filled with T_m omega^(m q) (rows sharing a bin add, which is exact); after the
// potential multiply the forward value of row m is sum_q omega^(-m q) D_q[m mod 16], D_q the
// lane's 16-point forward DFT, summed over the row's 4 lanes by shuffles.  No barrier or table
// of the 64-point transform is involved; the theta2 passes are k_slab's FFTs, and the theta1
// pass works in place on the inverse theta2 pass's output buffer.
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(SLAB_THREADS) k_slab_r16(SlabArgs<T> A) {
  griddep_entry();
  static_assert(N1 == 64 && (4 * N2) % 32 == 0 && 4 * N2 <= SLAB_THREADS, "4 lanes of 16 points per theta2 row");
  using V = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x, p = blockIdx.y;
  constexpr int n1 = N1, n2 = N2, CS = 17;   // CS: padded 16-bin row per lane
  const int nmr = A.nmr;
  constexpr bool PADW = sizeof(T) == sizeof(float);
  const int wsz = PADW ? pd_size(nmr * n2) : nmr * n2;
  auto ix = [](int i) { return PADW ? pd(i) : i; };
  V* W0 = reinterpret_cast<V*>(smem_raw);   // the theta2 FFT buffers, [nmr][n2] each
  V* W1 = W0 + wsz;
  V* E4 = W1 + wsz;                         // [nmr][4]: omega^(m q)
  V* Cs = E4 + 4 * nmr;                     // [4 N2][CS]: one lane's 16 bins
  const V zero = mk<T>(T(0), T(0));
  const V* Gc = A.G + ((size_t)c * A.Nr + p) * A.nA;
  V* Hc = A.H + ((size_t)c * A.Nr + p) * A.nA;
  for (int t = threadIdx.x; t < 4 * nmr; t += blockDim.x) {
    const int r = t >> 2, q = t & 3;
    const V w = A.tw1[pmod(A.mrow_m[r] * q, n1)];   // e^{-2 pi i m q / 64}
    E4[t] = mk<T>(w.x, -w.y);
  }
  // theta2 inverse pass over the kept m rows.  Its first radix-4 Stockham pass (stride 1, no
  // twiddles) reads G through the (row, point) -> pair table, zero where no pair is kept, and
  // writes W1; the remaining passes start at stride 4.
  static_assert(N2 % 4 == 0, "first theta2 pass radix 4");
  {
    constexpr int nbf = N2 / 4;
    for (int idx = threadIdx.x; idx < nmr * nbf; idx += blockDim.x) {
      const int b = idx / nbf, j = idx - b * nbf;
      const int* sp = A.slot_pair + b * n2 + j;
      V v[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int a = sp[t * nbf];
        v[t] = a >= 0 ? Gc[a] : zero;
      }
      const V s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
      const V s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
      const V t = cmul_i(d13, +1);
      const int base = b * n2 + 4 * j;
      W1[ix(base)] = cadd(s02, s13);
      W1[ix(base + 1)] = cadd(d02, t);
      W1[ix(base + 2)] = csub(s02, s13);
      W1[ix(base + 3)] = csub(d02, t);
    }
    __syncthreads();
  }
  // Tb: the rows at the theta2 points, updated in place by the theta1 pass (the 4 lanes that
  // read and write the point j of every row are one warp's)
  V* Tb = W1;
  {
    V* dst = W0;
    fft_ct_stages<T, N2, 4, PADW>(Tb, dst, nmr, A.tw2, +1);
  }
  if (threadIdx.x < 4 * n2) {
    const int j = threadIdx.x >> 2, q = threadIdx.x & 3;
    V* cs = Cs + threadIdx.x * CS;
#pragma unroll
    for (int b = 0; b < 16; ++b) cs[b] = zero;
    for (int r = 0; r < nmr; ++r) {   // bins of this lane (its own row of Cs: no other writer)
      const V t = Tb[ix(r * n2 + j)], e = E4[4 * r + q];
      const int b = A.mrow_m[r] & 15;
      V v = cs[b];
      v.x += t.x * e.x - t.y * e.y;
      v.y += t.x * e.y + t.y * e.x;
      cs[b] = v;
    }
    T xr[16], xi[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      xr[b] = cs[b].x;
      xi[b] = cs[b].y;
    }
    dft16<+1, T>(xr, xi);   // xr[t] + i xi[t] = u(theta1 = 4 t + q)
    const T* Vrow = A.V + ((size_t)p * n2 + j) * n1 + q;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const T v = Vrow[4 * t];
      xr[t] *= v;
      xi[t] *= v;
    }
    dft16<-1, T>(xr, xi);
#pragma unroll
    for (int b = 0; b < 16; ++b) cs[b] = mk<T>(xr[b], xi[b]);
    __syncwarp();   // every lane of this point has read its column of Tb
    for (int r = 0; r < nmr; ++r) {
      const V d = cs[A.mrow_m[r] & 15], e = E4[4 * r + q];   // times conj(omega^(m q))
      T sr = d.x * e.x + d.y * e.y, si = d.y * e.x - d.x * e.y;
      sr += __shfl_xor_sync(0xffffffffu, sr, 1);
      si += __shfl_xor_sync(0xffffffffu, si, 1);
      sr += __shfl_xor_sync(0xffffffffu, sr, 2);
      si += __shfl_xor_sync(0xffffffffu, si, 2);
      if (q == (r & 3)) Tb[ix(r * n2 + j)] = mk<T>(sr, si);
    }
  }
  __syncthreads();
  // theta2 forward pass from Tb, extract the kept pairs
  V* r2 = fft_any<T, N2, PADW>(Tb, Tb == W0 ? W1 : W0, A.p2, nmr, A.tw2, -1);
  for (int a = threadIdx.x; a < A.nA; a += blockDim.x)
    Hc[a] = r2[ix(A.pair_mrow[a] * n2 + pmod(A.pair_n[a], n2))];
}

// 12-point DFT in registers, X[k] = sum_n x[n] e^(S 2 pi i n k / 12), as 4-point DFTs over n1
// (n = 3 n1 + n2), the twiddles e^(S 2 pi i n2 k1 / 12), then 3-point DFTs over n2 (k = k1 + 4 k2)
template <int S, typename R>
__device__ __forceinline__ void dft12(R (&xr)[12], R (&xi)[12]) {
  constexpr R H3 = R(0.866025403784438646763723170752936183);   // sin(pi / 3)
  // e^(2 pi i e / 12) for e = 0..6 (cos, sin); the sign S is applied to the sine
  constexpr R wc[7] = {R(1), H3, R(0.5), R(0), R(-0.5), -H3, R(-1)};
  constexpr R ws[7] = {R(0), R(0.5), H3, R(1), H3, R(0.5), R(0)};
  R ar[12], ai[12];   // a[4 n2 + k1]
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
    const R x0r = xr[n2], x0i = xi[n2], x1r = xr[3 + n2], x1i = xi[3 + n2];
    const R x2r = xr[6 + n2], x2i = xi[6 + n2], x3r = xr[9 + n2], x3i = xi[9 + n2];
    const R t0r = x0r + x2r, t0i = x0i + x2i, t1r = x0r - x2r, t1i = x0i - x2i;
    const R t2r = x1r + x3r, t2i = x1i + x3i;
    const R dr = x1r - x3r, di = x1i - x3i;
    const R t3r = -S * di, t3i = S * dr;   // (x1 - x3) (S i)
    ar[4 * n2] = t0r + t2r;
    ai[4 * n2] = t0i + t2i;
    ar[4 * n2 + 1] = t1r + t3r;
    ai[4 * n2 + 1] = t1i + t3i;
    ar[4 * n2 + 2] = t0r - t2r;
    ai[4 * n2 + 2] = t0i - t2i;
    ar[4 * n2 + 3] = t1r - t3r;
    ai[4 * n2 + 3] = t1i - t3i;
  }
#pragma unroll
  for (int n2 = 1; n2 < 3; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) {
      const int e = n2 * k1;
      const R c = wc[e], sn = S * ws[e];
      const R r = ar[4 * n2 + k1], i = ai[4 * n2 + k1];
      ar[4 * n2 + k1] = r * c - i * sn;
      ai[4 * n2 + k1] = r * sn + i * c;
    }
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    const R a0r = ar[k1], a0i = ai[k1];
    const R sr = ar[4 + k1] + ar[8 + k1], si = ai[4 + k1] + ai[8 + k1];
    const R dr = ar[4 + k1] - ar[8 + k1], di = ai[4 + k1] - ai[8 + k1];
    const R tr = a0r - R(0.5) * sr, ti = a0i - R(0.5) * si;
    const R ur = -S * H3 * di, ui = S * H3 * dr;   // (a1 - a2) S i sin(pi / 3)
    xr[k1] = a0r + sr;
    xi[k1] = a0i + si;
    xr[k1 + 4] = tr + ur;
    xi[k1 + 4] = ti + ui;
    xr[k1 + 8] = tr - ur;
    xi[k1 + 8] = ti - ui;
  }
}

// 4-point DFT across the 4 lanes q = q0 + 2 q1 of an aligned quad, X[d] = sum_q v_q (S i)^(q d),
// as two radix-2 steps over the lane bits; lane q ends with X[q1 + 2 q0]
template <int S, typename R>
__device__ __forceinline__ void quad_dft(R& vr, R& vi, int q) {
  R pr = shfl_xor(vr, 2), pi = shfl_xor(vi, 2);
  if (q & 2) {
    vr = pr - vr;
    vi = pi - vi;
  } else {
    vr += pr;
    vi += pi;
  }
  if (q == 3) {   // (S i)^(q0 d0) with q0 = d0 = 1
    const R t = vr;
    vr = -S * vi;
    vi = S * t;
  }
  pr = shfl_xor(vr, 1);
  pi = shfl_xor(vi, 1);
  if (q & 1) {
    vr = pr - vr;
    vi = pi - vi;
  } else {
    vr += pr;
    vi += pi;
  }
}

// Slab kernel for the 64 x 48 grid with every transform in registers, SQ slabs (the columns
// blockIdx.x * SQ .. of the radial node blockIdx.y) per CTA and two block barriers per CTA.
//   theta2 (48 = 12 x 4): the 4 lanes of a (slab, kept row) quad hold the points n = 4 a + q
//     (inverse: read from G through the (row, point) -> pair table) or j = c + 12 q (forward);
//     a lane's 12-point DFT, the twiddles e^(+-2 pi i q c / 48) and a 4-point DFT across the
//     quad by shuffles make the 48-point transform.
//   theta1 (64 = 16 x 4): as in k_slab_r16, lane q of a (slab, theta2 point) quad owns the
//     points 4 t + q; with the kept rows m_r = m_0 + r (r < nmr <= 16) the row values
//     T_r omega^(m_r q) sit in DFT slot r: the inverse DFT then misses the factor W^(m_0 t) of
//     the true bins m_r mod 16, and the forward DFT of row r, taken at slot r, misses
//     W^(-m_0 t) -- the two cancel through the (real) potential multiply, so no bin table
//     or shared-memory bins are needed; the 4 lanes' row sums are a reduce-scatter of 16
//     values by shuffles (lane q ends with the rows 4 q .. 4 q + 3).
// Tb[s][r][j]: the rows at the theta2 points, row stride SQ_RS = 49 (odd multiple of 16 + 1:
// the quads' accesses spread over the banks).
constexpr int SQ_RS = 49;

// T: the storage type of G, H, the tables and the potential; R: the arithmetic type (T itself,
// or double-float `ff` for T = double, with the potential given as FP32 pairs in Vr).
// FP32: three CTAs per SM (80 registers, a few spilled: 60.6 us per 64-column launch against
// 65.9 at two CTAs and 112 registers, 63.9 at four and 64).  Double-float: two CTAs per SM
// (128 registers, none spilled: 557 us per 76-column launch against 816 at one CTA and 193
// registers; three CTAs spill 420 bytes).
template <typename T, typename R = T>
__global__ void __launch_bounds__(SLAB_THREADS, sizeof(R) == 4 ? 3 : (std::is_same<T, R>::value ? 1 : 2))
    k_slab_q(SlabArgs<T> A, const R* __restrict__ Vr, int SQ) {
  using V = cplx_t<T>;
  using C = rc_t<R>;
  constexpr int n1 = 64, n2 = 48;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nmr = A.nmr, p = blockIdx.y, c0 = blockIdx.x * SQ;
  C* Tb = reinterpret_cast<C*>(smem_raw);   // [SQ][nmr][SQ_RS]
  C* E4 = Tb + (size_t)SQ * nmr * SQ_RS;    // [16][4]: omega^(m_r q), zero past nmr
  C* T48 = E4 + 64;                         // [48]: e^(-2 pi i t / 48)
  const R zr = R(0);
  for (int t = threadIdx.x; t < 64; t += blockDim.x) {
    const int r = t >> 2, q = t & 3;
    C e = mkr<R>(zr, zr);
    if (r < nmr) {
      const V w = A.tw1[pmod(A.mrow_m[r] * q, n1)];   // e^{-2 pi i m q / 64}
      e = mkr<R>(to_r<R>(w.x), to_r<R>(-w.y));
    }
    E4[t] = e;
  }
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const V w = A.tw2[t];
    T48[t] = mkr<R>(to_r<R>(w.x), to_r<R>(w.y));
  }
  griddep_wait();   // G is the radial inverse's output (the tables above are the basis's)
  __syncthreads();
  const int lane = threadIdx.x & 31, q = lane & 3;
  const int nq2 = SQ * nmr * 4;   // theta2 lanes
  // ---- inverse theta2: G -> Tb
  if (threadIdx.x - lane < nq2) {
    const int t = threadIdx.x, sr = t >> 2, s = sr / nmr, r = sr - s * nmr;
    const int c = c0 + s;
    const bool valid = t < nq2 && c < A.ncols;
    const V* Gc = A.G + ((size_t)(valid ? c : 0) * A.Nr + p) * A.nA;
    const int* sp = A.slot_pair + (size_t)(valid ? r : 0) * n2 + q;
    R xr[12], xi[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      const int pa = valid ? sp[4 * a] : -1;
      if constexpr (std::is_same<R, ff>::value) {   // G holds double-float pairs
        ffc v;
        v.x = ff(0);
        v.y = ff(0);
        if (pa >= 0) v = reinterpret_cast<const ffc*>(Gc)[pa];
        xr[a] = v.x;
        xi[a] = v.y;
      } else {
        V v = mk<T>(T(0), T(0));
        if (pa >= 0) v = Gc[pa];
        xr[a] = to_r<R>(v.x);
        xi[a] = to_r<R>(v.y);
      }
    }
    dft12<+1, R>(xr, xi);
    C* row = Tb + ((size_t)s * nmr + r) * SQ_RS + 12 * ((q >> 1) + 2 * (q & 1));
#pragma unroll
    for (int cc = 0; cc < 12; ++cc) {
      const C w = T48[q * cc];   // times e^{+2 pi i q c / 48}
      R vr = xr[cc] * w.x + xi[cc] * w.y, vi = xi[cc] * w.x - xr[cc] * w.y;
      quad_dft<+1, R>(vr, vi, q);
      if (valid) row[cc] = mkr<R>(vr, vi);
    }
  }
  __syncthreads();
  // ---- theta1 inverse, x V, theta1 forward, in place on Tb
  const R* Vp = Vr + (size_t)p * n2 * n1;
  for (int t = threadIdx.x; t < SQ * n2 * 4; t += blockDim.x) {
    const int sj = t >> 2, s = sj / n2, j = sj - s * n2;
    C* col = Tb + (size_t)s * nmr * SQ_RS + j;
    R xr[16], xi[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      xr[r] = zr;
      xi[r] = zr;
      if (r < nmr) {
        const C u = col[r * SQ_RS], e = E4[4 * r + q];
        xr[r] = u.x * e.x - u.y * e.y;
        xi[r] = u.x * e.y + u.y * e.x;
      }
    }
    dft16<+1, R>(xr, xi);   // the points 4 t + q, up to W^(m_0 t)
    const R* Vrow = Vp + (size_t)j * n1 + q;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const R v = Vrow[4 * k];
      xr[k] *= v;
      xi[k] *= v;
    }
    dft16<-1, R>(xr, xi);   // slot r: this lane's share of row r, up to omega^(-m_r q)
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const C e = E4[4 * r + q];   // times conj(omega^(m_r q))
      const R vr = xr[r] * e.x + xi[r] * e.y, vi = xi[r] * e.x - xr[r] * e.y;
      xr[r] = vr;
      xi[r] = vi;
    }
    // reduce-scatter over the quad: rows 8 h .. 8 h + 7 (h = q >> 1), then 4 q .. 4 q + 3
    const bool h = q & 2, l = q & 1;
    R kr[8], ki[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const R sr = h ? xr[i] : xr[8 + i], si = h ? xi[i] : xi[8 + i];
      kr[i] = (h ? xr[8 + i] : xr[i]) + shfl_xor(sr, 2);
      ki[i] = (h ? xi[8 + i] : xi[i]) + shfl_xor(si, 2);
    }
    __syncwarp();   // every lane of the quad has read its column of Tb
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const R sr = l ? kr[i] : kr[4 + i], si = l ? ki[i] : ki[4 + i];
      const R vr = (l ? kr[4 + i] : kr[i]) + shfl_xor(sr, 1);
      const R vi = (l ? ki[4 + i] : ki[i]) + shfl_xor(si, 1);
      const int r = 4 * q + i;
      if (r < nmr) col[r * SQ_RS] = mkr<R>(vr, vi);
    }
  }
  griddep_launch();   // only the forward theta2 pass is left: the next kernel's CTAs may start
  __syncthreads();
  // ---- forward theta2: Tb -> H (kept pairs only)
  if (threadIdx.x - lane < nq2) {
    const int t = threadIdx.x, sr = t >> 2, s = sr / nmr, r = sr - s * nmr;
    const int c = c0 + s;
    const bool valid = t < nq2 && c < A.ncols;
    const C* row = Tb + ((size_t)(valid ? s * nmr + r : 0)) * SQ_RS + 12 * q;
    const int b = (q >> 1) + 2 * (q & 1);   // this lane's n mod 4 after the quad DFT
    R xr[12], xi[12];
#pragma unroll
    for (int cc = 0; cc < 12; ++cc) {
      const C u = row[cc];
      R vr = u.x, vi = u.y;
      quad_dft<-1, R>(vr, vi, q);
      const C w = T48[b * cc];   // times e^{-2 pi i b c / 48}
      xr[cc] = vr * w.x - vi * w.y;
      xi[cc] = vr * w.y + vi * w.x;
    }
    dft12<-1, R>(xr, xi);   // F[4 a + b]
    if (valid) {
      V* Hc = A.H + ((size_t)c * A.Nr + p) * A.nA;
      const int* sp = A.slot_pair + (size_t)r * n2 + b;
#pragma unroll
      for (int a = 0; a < 12; ++a) {
        const int pa = sp[4 * a];
        if constexpr (std::is_same<R, ff>::value) {   // H holds double-float pairs
          if (pa >= 0) {
            ffc v;
            v.x = xr[a];
            v.y = xi[a];
            reinterpret_cast<ffc*>(Hc)[pa] = v;
          }
        } else {
          if (pa >= 0) Hc[pa] = mk<T>(from_r<T>(xr[a]), from_r<T>(xi[a]));
        }
      }
    }
  }
}

// slabs per CTA of k_slab_q: as many (slab, row) quads as fit the CTA's threads, at most 8
static int slab_q_per_cta(int nmr) { return std::max(1, std::min(8, SLAB_THREADS / (4 * std::max(nmr, 1)))); }
static size_t slab_q_smem_bytes(int nmr, size_t elem) {
  return elem * ((size_t)slab_q_per_cta(nmr) * nmr * SQ_RS + 64 + 48);
}

static size_t slab_r16_smem_bytes(int nmr, int n2, size_t elem) {
  const size_t w = elem == sizeof(float2) ? (size_t)pd_size(nmr * n2) : (size_t)nmr * n2;
  return elem * (2 * w + 4 * (size_t)nmr + (size_t)4 * n2 * 17);
}

// the 64 x 48 grid: the 4 x 16 theta1 variant (unless HW_OPT_SLAB_KERNEL selects the Stockham
// FFTs)
static bool use_slab_r16(const hw_ctx* ctx, size_t elem) {
  (void)elem;
  return ctx->slab_r16 && ctx->hb.prm.Nth1 == 64 && ctx->hb.prm.Nth2 == 48;
}

// the all-register variant (HW_OPT_SLAB_KERNEL = 2: FP32 only, the FP64 transforms stay on
// k_slab_r16, whose FP64-pipe work the register variant does not lower; 3: both precisions):
// 64 x 48 grid, at most 16 kept m rows, and those consecutive (m_r = m_0 + r)
static bool slab_q_shape(const hw_ctx* ctx) {
  const auto& mm = ctx->hb.mrow_m;
  if (ctx->hb.prm.Nth1 != 64 || ctx->hb.prm.Nth2 != 48 || mm.empty() || mm.size() > 16) return false;
  for (size_t r = 1; r < mm.size(); ++r)
    if (mm[r] != mm[0] + (int)r) return false;
  return true;
}
static bool use_slab_q(const hw_ctx* ctx, size_t elem) {
  const bool want = ctx->slab_r16 == 3 || (ctx->slab_r16 == 2 && elem == sizeof(float2));
  return want && slab_q_shape(ctx);
}


// --------------------------------------------------------------------------- host launcher
// the slab kernel for this basis's angular grid: specialised for the grids in use, generic
// otherwise
template <typename T>
static void* slab_kernel(int n1, int n2) {
  if (n1 == 64 && n2 == 48) return (void*)k_slab<T, 64, 48>;
  if (n1 == 192 && n2 == 96) return (void*)k_slab<T, 192, 96>;
  return (void*)k_slab<T, 0, 0>;
}

// ffp: the double-float FP64 path (G and H hold FP32 pairs)
template <typename T>
static cudaError_t launch_slab(const hw_ctx* ctx, dim3 grid, size_t smem, const SlabArgs<T>& sa, bool ffp = false) {
  if (ffp || use_slab_q(ctx, sizeof(cplx_t<T>))) {
    const int sq = slab_q_per_cta(sa.nmr);
    const dim3 g((grid.x + sq - 1) / sq, grid.y);
    if constexpr (sizeof(T) == sizeof(double)) {
      if (ffp) {
        return launch_dep(ctx->stream, k_slab_q<double, ff>, g, dim3(SLAB_THREADS), smem, sa,
                          reinterpret_cast<const ff*>(ctx->db.vff), sq);
      }
    }
    // the FP32 slab between the tensor-core radial kernels starts while the inverse drains
    return launch_ex(ctx, sizeof(T) == 4 && ctx->overlap_launch != 0, k_slab_q<T, T>, g, dim3(SLAB_THREADS), smem, sa,
                     sa.V, sq);
  }
  void* f = use_slab_r16(ctx, sizeof(cplx_t<T>)) ? (void*)k_slab_r16<T, 64, 48> : slab_kernel<T>(sa.Nth1, sa.Nth2);
  void* args[] = {(void*)&sa};
  return launch_dep_c(ctx->stream, f, grid, dim3(SLAB_THREADS), smem, args);
}

static FftDev to_dev(const FftPlan& p) {
  FftDev d;
  d.n = p.n;
  d.nst = p.nst;
  for (int i = 0; i < 16; ++i) d.rad[i] = p.rad[i];
  return d;
}

size_t slab_smem_bytes(const hw_ctx* ctx, size_t elem, int Jc) {
  const auto& hb = ctx->hb;
  const int nmr = (int)hb.mrow_m.size();
  const int n1 = hb.prm.Nth1, n2 = hb.prm.Nth2;
  if (use_slab_q(ctx, elem)) return slab_q_smem_bytes(nmr, elem);   // no theta2 chunks
  if (use_slab_r16(ctx, elem)) return slab_r16_smem_bytes(nmr, n2, elem);
  // padded layout: the FP32 kernels specialised for the grid (k_slab's PAD)
  const bool pad = elem == sizeof(float2) && slab_kernel<float>(n1, n2) != (void*)k_slab<float, 0, 0>;
  const int w = std::max(nmr * n2, Jc * n1);
  const size_t wsz = (size_t)(pad ? pd_size(w) : w);
  return elem * ((size_t)nmr * (n2 + (pad ? 1 : 0)) + 2 * wsz);
}

int slab_pick_jc(const hw_ctx* ctx, size_t elem) {
  // halve the column chunk while the slab's shared memory is above 110 KB (two CTAs per SM)
  // and halving still shrinks it (the theta2 rows set a floor)
  int Jc = ctx->hb.prm.Nth2;
  while (Jc > 1 && slab_smem_bytes(ctx, elem, Jc) > 110 * 1024 &&
         slab_smem_bytes(ctx, elem, (Jc + 1) / 2) < slab_smem_bytes(ctx, elem, Jc))
    Jc = (Jc + 1) / 2;
  return Jc;
}

// nu != 0 arguments of the forward radial kernel
template <typename T>
static void set_nu_args(const hw_ctx* ctx, const Blocks& blk, const DevTables<T>& tb, RadArgs<T>& ra) {
  ra.qtab = tb.qtab;
  ra.pair_n = ctx->db.pair_n;
  ra.ncyc = ctx->hb.prm.ncyc;
  ra.any_nu = 0;
  for (int i = 0; i < MAXSLOT; ++i) {
    ra.nu[i] = i < blk.nslot ? ctx->hb.nu[blk.kb[i]] : 0.0;
    if (ra.nu[i] != 0.0) ra.any_nu = 1;
  }
  ra.scale_mode = 0;
  ra.step = 0;
  ra.pair_mrow = ctx->db.pair_mrow;
  ra.mrow_m = ctx->db.mrow_m;
}

// Launch the three kernels for the column blocks `blk` (ns columns each) with the G / H
// intermediates in `gbuf` / `hbuf`, which hold `cols` columns each; columns are processed in
// passes of at most that many (fewer when the autotuner chose a narrower pass).  Every pass
// writes each intermediate value before reading it, so the buffers need no initialisation.
template <typename T>
static cudaError_t launch_hx_bufs(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, const ChebStep* step,
                                  void* gbuf, void* hbuf, int cols) {
  auto& hb = ctx->hb;
  auto& db = ctx->db;
  const DevTables<T>& tb = *reinterpret_cast<const DevTables<T>*>(
      sizeof(T) == 8 ? (const void*)&db.t64 : (const void*)&db.t32);
  const int ncols_total = blk.nslot * ns;
  const int ti = sizeof(T) == 8 ? 0 : 1;
  int chunk = cols;
  if (ctx->ws.pass_cols[ti] > 0) chunk = std::min(chunk, ctx->ws.pass_cols[ti]);
  if (chunk <= 0 || blk.nslot > MAXSLOT) return cudaErrorInvalidValue;
  const int Nr = hb.prm.Nr, K = hb.K;
  int maxna = 0;
  for (int g = 0; g <= hb.N; ++g) maxna = std::max(maxna, hb.group_start[g + 1] - hb.group_start[g]);
  const int Jc = ctx->ws.jc[ti] > 0 ? ctx->ws.jc[ti] : slab_pick_jc(ctx, sizeof(cplx_t<T>));
  for (int c0 = 0; c0 < ncols_total; c0 += chunk) {
    const int nc = std::min(chunk, ncols_total - c0);
    RadArgs<T> ra;
    ra.Nr = Nr;
    ra.K = K;
    ra.nA = hb.nA;
    ra.ncols = nc;
    ra.ns = ns;
    ra.c0 = c0;
    ra.group_start = db.group_start;
    ra.off = db.off;
    ra.Ka = db.Ka;
    ra.ld = ld;
    ra.ke = db.ke;
    for (int i = 0; i < blk.nslot; ++i) ra.keoff[i] = db.ke_off[blk.kb[i]];
    set_nu_args(ctx, blk, tb, ra);
    ra.blk = blk;
    ra.gh = reinterpret_cast<cplx_t<T>*>(gbuf);
    ra.rtab = tb.rinv;
    // FP64 H X in double-float (a mixed solve's, or HW_FP64_DF): all three kernels, which pass
    // FP32 pairs through G and H, on the register slab's shape and without nu != 0 terms
    const bool ffp = sizeof(T) == 8 && ctx->ff_now && slab_q_shape(ctx) && !ra.any_nu;
    dim3 grid((unsigned)(((long)maxna * nc + RAD_Q - 1) / RAD_Q), hb.N + 1);
    const size_t sm_inv = rad_inv_smem(Nr, K, sizeof(T));
    const bool tc = sizeof(T) == 4 && ctx->radial_tc && db.rt_ok;
    {
      ProfScope ps(ctx, HW_PH_RADIAL_INV);
      if (tc) {
        const cudaError_t e = launch_rinv_tc(ctx, blk, ns, ld, nc, c0, gbuf, 0);
        if (e != cudaSuccess) return e;
      } else if (ffp) {
        if constexpr (sizeof(T) == 8)
          launch_dep(ctx->stream, k_radial_inv_ff, grid, RAD_THREADS, sm_inv, ra, reinterpret_cast<const ff*>(db.ff_rinv));
      } else {
        launch_dep(ctx->stream, k_radial_inv<T>, grid, RAD_THREADS, sm_inv, ra);
      }
      ctx->launches++;
    }
    SlabArgs<T> sa;
    sa.Nr = Nr;
    sa.Nth1 = hb.prm.Nth1;
    sa.Nth2 = hb.prm.Nth2;
    sa.nA = hb.nA;
    sa.nmr = (int)hb.mrow_m.size();
    sa.ncols = nc;
    sa.Jc = Jc;
    sa.p1 = to_dev(ctx->plan1);
    sa.p2 = to_dev(ctx->plan2);
    sa.pair_n = db.pair_n;
    sa.pair_mrow = db.pair_mrow;
    sa.mrow_m = db.mrow_m;
    sa.slot_pair = db.slot_pair;
    sa.V = tb.V;
    sa.tw1 = reinterpret_cast<const cplx_t<T>*>(tb.tw1);
    sa.tw2 = reinterpret_cast<const cplx_t<T>*>(tb.tw2);
    sa.G = reinterpret_cast<const cplx_t<T>*>(gbuf);
    sa.H = reinterpret_cast<cplx_t<T>*>(hbuf);
    const size_t sm_slab = ffp ? slab_q_smem_bytes(sa.nmr, sizeof(double2)) : slab_smem_bytes(ctx, sizeof(cplx_t<T>), Jc);
    {
      ProfScope ps(ctx, HW_PH_SLAB);
      launch_slab<T>(ctx, dim3(nc, Nr), sm_slab, sa, ffp);
      ctx->launches++;
    }
    ra.gh = reinterpret_cast<cplx_t<T>*>(hbuf);
    ra.rtab = tb.rfwd;
    if (step) {
      ra.step = 1;
      ra.cs = *step;
    }
    const size_t sm_fwd = rad_fwd_smem(Nr, K, sizeof(T));
    {
      ProfScope ps(ctx, HW_PH_RADIAL_FWD);
      if (tc && !ra.any_nu) {
        const cudaError_t e = launch_rfwd_tc(ctx, blk, ns, ld, nc, c0, hbuf, step);
        if (e != cudaSuccess) return e;
      } else if (ffp) {
        if constexpr (sizeof(T) == 8)
          launch_dep(ctx->stream, k_radial_fwd_ff, grid, RAD_THREADS, sm_fwd, ra, reinterpret_cast<const ff*>(db.ff_rfwd));
      } else {
        launch_dep(ctx->stream, k_radial_fwd<T>, grid, RAD_THREADS, sm_fwd, ra);
      }
      ctx->launches++;
    }
  }
  return cudaGetLastError();
}

// H X with the intermediates in the context's workspace.
template <typename T>
cudaError_t launch_hx(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, const ChebStep* step) {
  return launch_hx_bufs<T>(ctx, blk, ns, ld, step, ctx->ws.gbuf, ctx->ws.hbuf, (int)ctx->ws.cols);
}

// H X with caller-chosen G / H buffers of `cols` columns each (the entry point that
// allocates nothing); the same launch configuration as launch_hx.
template <typename T>
cudaError_t launch_hx_into(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, void* gbuf, void* hbuf, int cols) {
  return launch_hx_bufs<T>(ctx, blk, ns, ld, nullptr, gbuf, hbuf, cols);
}

template cudaError_t launch_hx_into<double>(hw_ctx*, const Blocks&, int, int64_t, void*, void*, int);
template cudaError_t launch_hx_into<float>(hw_ctx*, const Blocks&, int, int64_t, void*, void*, int);

// --------------------------------------------------------------------------- electron density
// rho(theta1, theta2, r) += w_c |phi_c|^2 over columns (states) c (Sec. "Convergence Studies",
// the electron-density equation): the inverse radial transform is k_radial_inv; this kernel
// takes each column's (r_p, pair) values through the same inverse angular passes as k_slab
// and accumulates w_c |u|^2 for its radial node in shared memory, then adds the slab into rho
// ([i][j][p] order, like the potential handed to hw_set_potential).
template <typename T>
struct DensArgs {
  int Nr, Nth1, Nth2, nA, nmr, ncols, Jc, cpg;   // cpg: columns per CTA (blockIdx.y groups)
  FftDev p1, p2;
  const int* pair_n;
  const int* pair_mrow;
  const int* mrow_m;
  const cplx_t<T>* tw1;
  const cplx_t<T>* tw2;
  const cplx_t<T>* G;     // [column][r_p][pair] of this pass
  const double* wcol;     // [column] weight of each column of this pass
  double* rho;            // [N_th1][N_th2][N_r]
};

__host__ __device__ inline size_t dens_acc_bytes(int n1, int n2, size_t tsz) {
  return ((size_t)n1 * n2 * tsz + 15) & ~size_t(15);
}

template <typename T, int N1 = 0, int N2 = 0>
__global__ void __launch_bounds__(SLAB_THREADS) k_density(DensArgs<T> A) {
  griddep_entry();
  using V = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x, grp = blockIdx.y;
  const int n1 = N1 > 0 ? N1 : A.Nth1, n2 = N2 > 0 ? N2 : A.Nth2, nmr = A.nmr;
  T* acc = reinterpret_cast<T*>(smem_raw);                                      // [n2][n1]
  V* Tb = reinterpret_cast<V*>(smem_raw + dens_acc_bytes(n1, n2, sizeof(T)));   // [nmr][n2]
  const int wsz = max(nmr * n2, A.Jc * n1);
  V* W0 = Tb + nmr * n2;
  V* W1 = W0 + wsz;
  const V zero = mk<T>(T(0), T(0));
  for (int i = threadIdx.x; i < n1 * n2; i += blockDim.x) acc[i] = T(0);
  const int cbeg = grp * A.cpg, cend = min(A.ncols, cbeg + A.cpg);
  for (int c = cbeg; c < cend; ++c) {
    const T wc = (T)A.wcol[c];
    if (wc == T(0)) continue;   // uniform over the CTA
    const V* Gc = A.G + ((size_t)c * A.Nr + p) * A.nA;
    __syncthreads();
    for (int i = threadIdx.x; i < nmr * n2; i += blockDim.x) W0[i] = zero;
    __syncthreads();
    for (int a = threadIdx.x; a < A.nA; a += blockDim.x)
      W0[A.pair_mrow[a] * n2 + pmod(A.pair_n[a], n2)] = Gc[a];
    __syncthreads();
    V* r = fft_any<T, N2, false>(W0, W1, A.p2, nmr, A.tw2, +1);
    for (int i = threadIdx.x; i < nmr * n2; i += blockDim.x) Tb[i] = r[i];
    __syncthreads();
    for (int j0 = 0; j0 < n2; j0 += A.Jc) {
      const int jn = min(A.Jc, n2 - j0);
      for (int i = threadIdx.x; i < jn * n1; i += blockDim.x) W0[i] = zero;
      __syncthreads();
      for (int i = threadIdx.x; i < jn * nmr; i += blockDim.x) {
        const int jj = i / nmr, rr = i - jj * nmr;
        W0[jj * n1 + pmod(A.mrow_m[rr], n1)] = Tb[rr * n2 + j0 + jj];
      }
      __syncthreads();
      V* u = fft_any<T, N1, false>(W0, W1, A.p1, jn, A.tw1, +1);
      for (int i = threadIdx.x; i < jn * n1; i += blockDim.x) {
        const V x = u[i];
        acc[j0 * n1 + i] += wc * (x.x * x.x + x.y * x.y);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n1 * n2; t += blockDim.x) {
    const int j = t / n1, i = t - j * n1;
    atomicAdd(&A.rho[((size_t)i * n2 + j) * A.Nr + p], (double)acc[t]);
  }
}

template <typename T>
static void* density_kernel(int n1, int n2) {
  if (n1 == 64 && n2 == 48) return (void*)k_density<T, 64, 48>;
  if (n1 == 192 && n2 == 96) return (void*)k_density<T, 192, 96>;
  return (void*)k_density<T, 0, 0>;
}

static size_t density_smem_bytes(const hw_ctx* ctx, size_t tsz, int Jc) {
  const auto& hb = ctx->hb;
  const int nmr = (int)hb.mrow_m.size(), n1 = hb.prm.Nth1, n2 = hb.prm.Nth2;
  const size_t w = (size_t)std::max(nmr * n2, Jc * n1);
  return dens_acc_bytes(n1, n2, tsz) + 2 * tsz * ((size_t)nmr * n2 + 2 * w);
}

// whether the density kernel's shared memory fits for this basis (arithmetic of size tsz)
bool density_fits(const hw_ctx* ctx, size_t tsz) { return density_smem_bytes(ctx, tsz, 1) <= 200 * 1024; }

// rho += sum over the columns of blk (ns per block) of wcol[column] |phi_column|^2; wcol is a
// device array of blk.nslot * ns weights; rho must hold N_th1 N_th2 N_r doubles.
template <typename T>
cudaError_t launch_density(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, const double* wcol, double* rho) {
  auto& hb = ctx->hb;
  auto& db = ctx->db;
  const DevTables<T>& tb = *reinterpret_cast<const DevTables<T>*>(
      sizeof(T) == 8 ? (const void*)&db.t64 : (const void*)&db.t32);
  const int ncols_total = blk.nslot * ns;
  const int chunk = (int)ctx->ws.cols;
  if (chunk <= 0 || blk.nslot > MAXSLOT) return cudaErrorInvalidValue;
  const int Nr = hb.prm.Nr, K = hb.K;
  int Jc = hb.prm.Nth2;
  while (Jc > 1 && density_smem_bytes(ctx, sizeof(T), Jc) > 200 * 1024 &&
         density_smem_bytes(ctx, sizeof(T), (Jc + 1) / 2) < density_smem_bytes(ctx, sizeof(T), Jc))
    Jc = (Jc + 1) / 2;
  const size_t sm = density_smem_bytes(ctx, sizeof(T), Jc);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  int maxna = 0;
  for (int g = 0; g <= hb.N; ++g) maxna = std::max(maxna, hb.group_start[g + 1] - hb.group_start[g]);
  void* kf = density_kernel<T>(hb.prm.Nth1, hb.prm.Nth2);
  cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  for (int c0 = 0; c0 < ncols_total; c0 += chunk) {
    const int nc = std::min(chunk, ncols_total - c0);
    RadArgs<T> ra;
    ra.Nr = Nr;
    ra.K = K;
    ra.nA = hb.nA;
    ra.ncols = nc;
    ra.ns = ns;
    ra.c0 = c0;
    ra.group_start = db.group_start;
    ra.off = db.off;
    ra.Ka = db.Ka;
    ra.ld = ld;
    ra.ke = db.ke;
    for (int i = 0; i < blk.nslot; ++i) ra.keoff[i] = db.ke_off[blk.kb[i]];
    set_nu_args(ctx, blk, tb, ra);
    ra.blk = blk;
    ra.gh = reinterpret_cast<cplx_t<T>*>(ctx->ws.gbuf);
    ra.rtab = tb.rinv;
    dim3 grid((unsigned)(((long)maxna * nc + RAD_Q - 1) / RAD_Q), hb.N + 1);
    const size_t sm_inv = rad_inv_smem(Nr, K, sizeof(T));
    {
      ProfScope ps(ctx, HW_PH_RADIAL_INV);
      launch_dep(ctx->stream, k_radial_inv<T>, grid, RAD_THREADS, sm_inv, ra);
      ctx->launches++;
    }
    DensArgs<T> da;
    da.Nr = Nr;
    da.Nth1 = hb.prm.Nth1;
    da.Nth2 = hb.prm.Nth2;
    da.nA = hb.nA;
    da.nmr = (int)hb.mrow_m.size();
    da.ncols = nc;
    da.Jc = Jc;
    const int ncg = std::max(1, std::min(nc, (2 * 152 + Nr - 1) / Nr));
    da.cpg = (nc + ncg - 1) / ncg;
    da.p1 = to_dev(ctx->plan1);
    da.p2 = to_dev(ctx->plan2);
    da.pair_n = db.pair_n;
    da.pair_mrow = db.pair_mrow;
    da.mrow_m = db.mrow_m;
    da.tw1 = reinterpret_cast<const cplx_t<T>*>(tb.tw1);
    da.tw2 = reinterpret_cast<const cplx_t<T>*>(tb.tw2);
    da.G = reinterpret_cast<const cplx_t<T>*>(ctx->ws.gbuf);
    da.wcol = wcol + c0;
    da.rho = rho;
    void* args[] = {(void*)&da};
    {
      ProfScope ps(ctx, HW_PH_DENSITY);
      e = launch_dep_c(ctx->stream, kf, dim3(Nr, (nc + da.cpg - 1) / da.cpg), dim3(SLAB_THREADS), sm, args);
      ctx->launches++;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}
template cudaError_t launch_density<double>(hw_ctx*, const Blocks&, int, int64_t, const double*, double*);
template cudaError_t launch_density<float>(hw_ctx*, const Blocks&, int, int64_t, const double*, double*);

// --------------------------------------------------------------------------- gradients
// Cartesian gradient of E = sum Ehat F on the grid (Appendix C): k_radial_inv gives the
// (r_p, pair) values of E_r (radial table d xi / dr), E_theta2 (coefficients times i 2 pi n Ncyc)
// and E_theta1 (times i 2 pi m) in three regions of G; this kernel takes each through the
// inverse angular passes of k_slab and applies the chain rule of eq. Cartesian_Derivatives,
//   E_x = -sin(v)/(2 pi r) E_theta2 + cos(v) E_r,  E_y = cos(v)/(2 pi r) E_theta2 + sin(v) E_r,
//   E_z = (E_theta1 - alpha E_theta2)/tau,          v = 2 pi (alpha theta1 + theta2),
// writing D[column][component][i][j][p] (FP64).  The three sources are taken one after the
// other; each CTA owns its (column, r_p) outputs, so the later sources update them in place.
template <typename T>
struct GradArgs {
  int Nr, Nth1, Nth2, nA, nmr, ncols, Jc, cpg, ncyc;
  double alpha, tau;
  FftDev p1, p2;
  const int* pair_n;
  const int* pair_mrow;
  const int* mrow_m;
  const cplx_t<T>* tw1;
  const cplx_t<T>* tw2;
  const cplx_t<T>* G;      // [3][column][r_p][pair]: E_r, E_theta2, E_theta1
  const double* rnodes;    // [Nr]
  double2* D;              // [column][3][N_th1][N_th2][N_r] of this pass
};

template <typename T, int N1 = 0, int N2 = 0>
__global__ void __launch_bounds__(SLAB_THREADS) k_grad(GradArgs<T> A) {
  griddep_entry();
  using V = cplx_t<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = blockIdx.x, grp = blockIdx.y;
  const int n1 = N1 > 0 ? N1 : A.Nth1, n2 = N2 > 0 ? N2 : A.Nth2, nmr = A.nmr;
  V* Tb = reinterpret_cast<V*>(smem_raw);   // [nmr][n2]
  const int wsz = max(nmr * n2, A.Jc * n1);
  V* W0 = Tb + nmr * n2;
  V* W1 = W0 + wsz;
  const V zero = mk<T>(T(0), T(0));
  const double r = A.rnodes[p];
  const double inv2pir = 1.0 / (6.283185307179586 * r);
  const size_t grid = (size_t)n1 * n2 * A.Nr;
  const int cbeg = grp * A.cpg, cend = min(A.ncols, cbeg + A.cpg);
  for (int c = cbeg; c < cend; ++c) {
    double2* Dc = A.D + (size_t)c * 3 * grid;
    for (int src = 0; src < 3; ++src) {
      const V* Gc = A.G + (((size_t)src * A.ncols + c) * A.Nr + p) * A.nA;
      __syncthreads();
      for (int i = threadIdx.x; i < nmr * n2; i += blockDim.x) W0[i] = zero;
      __syncthreads();
      for (int a = threadIdx.x; a < A.nA; a += blockDim.x)
        W0[A.pair_mrow[a] * n2 + pmod(A.pair_n[a], n2)] = Gc[a];
      __syncthreads();
      V* rr = fft_any<T, N2, false>(W0, W1, A.p2, nmr, A.tw2, +1);
      for (int i = threadIdx.x; i < nmr * n2; i += blockDim.x) Tb[i] = rr[i];
      __syncthreads();
      for (int j0 = 0; j0 < n2; j0 += A.Jc) {
        const int jn = min(A.Jc, n2 - j0);
        for (int i = threadIdx.x; i < jn * n1; i += blockDim.x) W0[i] = zero;
        __syncthreads();
        for (int i = threadIdx.x; i < jn * nmr; i += blockDim.x) {
          const int jj = i / nmr, q = i - jj * nmr;
          W0[jj * n1 + pmod(A.mrow_m[q], n1)] = Tb[q * n2 + j0 + jj];
        }
        __syncthreads();
        V* u = fft_any<T, N1, false>(W0, W1, A.p1, jn, A.tw1, +1);
        for (int t = threadIdx.x; t < jn * n1; t += blockDim.x) {
          const int jj = t / n1, i = t - jj * n1, j = j0 + jj;
          const double2 x = make_double2((double)u[t].x, (double)u[t].y);
          const size_t o = ((size_t)i * n2 + j) * A.Nr + p;
          if (src == 2) {   // E_theta1
            double2 z = Dc[2 * grid + o];
            z.x += x.x / A.tau;
            z.y += x.y / A.tau;
            Dc[2 * grid + o] = z;
            continue;
          }
          // v / pi = 2 (alpha theta1 + theta2), theta1 = i / N_th1, theta2 = j / (Ncyc N_th2)
          double sv, cv;
          sincospi(2.0 * (A.alpha * i / n1 + (double)j / ((double)A.ncyc * n2)), &sv, &cv);
          if (src == 0) {   // E_r
            Dc[o] = make_double2(cv * x.x, cv * x.y);
            Dc[grid + o] = make_double2(sv * x.x, sv * x.y);
            Dc[2 * grid + o] = make_double2(0.0, 0.0);
          } else {          // E_theta2
            const double fx = -sv * inv2pir, fy = cv * inv2pir, fz = -A.alpha / A.tau;
            double2 a0 = Dc[o], a1 = Dc[grid + o], a2 = Dc[2 * grid + o];
            a0.x += fx * x.x;
            a0.y += fx * x.y;
            a1.x += fy * x.x;
            a1.y += fy * x.y;
            a2.x += fz * x.x;
            a2.y += fz * x.y;
            Dc[o] = a0;
            Dc[grid + o] = a1;
            Dc[2 * grid + o] = a2;
          }
        }
        __syncthreads();
      }
    }
  }
}

template <typename T>
static void* grad_kernel(int n1, int n2) {
  if (n1 == 64 && n2 == 48) return (void*)k_grad<T, 64, 48>;
  if (n1 == 192 && n2 == 96) return (void*)k_grad<T, 192, 96>;
  return (void*)k_grad<T, 0, 0>;
}

static size_t grad_smem_bytes(const hw_ctx* ctx, size_t csz, int Jc) {
  const auto& hb = ctx->hb;
  const int nmr = (int)hb.mrow_m.size(), n1 = hb.prm.Nth1, n2 = hb.prm.Nth2;
  const size_t w = (size_t)std::max(nmr * n2, Jc * n1);
  return csz * ((size_t)nmr * n2 + 2 * w);
}

// whether the gradient kernel's shared memory fits (complex element size csz)
bool gradient_fits(const hw_ctx* ctx, size_t csz) { return grad_smem_bytes(ctx, csz, 1) <= 200 * 1024; }

// D = Cartesian gradient of the ns columns of blk (one k-point slot); D holds ns * 3 *
// N_th1 N_th2 N_r complex128
template <typename T>
cudaError_t launch_gradient(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, double* D) {
  auto& hb = ctx->hb;
  auto& db = ctx->db;
  const DevTables<T>& tb = *reinterpret_cast<const DevTables<T>*>(
      sizeof(T) == 8 ? (const void*)&db.t64 : (const void*)&db.t32);
  if (blk.nslot != 1) return cudaErrorInvalidValue;
  const int chunk = (int)(ctx->ws.cols / 3);
  if (chunk <= 0) return cudaErrorInvalidValue;
  const int Nr = hb.prm.Nr, K = hb.K;
  int Jc = hb.prm.Nth2;
  const size_t csz = sizeof(cplx_t<T>);
  while (Jc > 1 && grad_smem_bytes(ctx, csz, Jc) > 200 * 1024 &&
         grad_smem_bytes(ctx, csz, (Jc + 1) / 2) < grad_smem_bytes(ctx, csz, Jc))
    Jc = (Jc + 1) / 2;
  const size_t sm = grad_smem_bytes(ctx, csz, Jc);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  int maxna = 0;
  for (int g = 0; g <= hb.N; ++g) maxna = std::max(maxna, hb.group_start[g + 1] - hb.group_start[g]);
  void* kf = grad_kernel<T>(hb.prm.Nth1, hb.prm.Nth2);
  cudaError_t e = cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  const size_t grid_pts = (size_t)hb.prm.Nth1 * hb.prm.Nth2 * Nr;
  for (int c0 = 0; c0 < ns; c0 += chunk) {
    const int nc = std::min(chunk, ns - c0);
    RadArgs<T> ra;
    ra.Nr = Nr;
    ra.K = K;
    ra.nA = hb.nA;
    ra.ncols = nc;
    ra.ns = ns;
    ra.c0 = c0;
    ra.group_start = db.group_start;
    ra.off = db.off;
    ra.Ka = db.Ka;
    ra.ld = ld;
    ra.ke = db.ke;
    ra.keoff[0] = db.ke_off[blk.kb[0]];
    set_nu_args(ctx, blk, tb, ra);
    ra.blk = blk;
    dim3 grid((unsigned)(((long)maxna * nc + RAD_Q - 1) / RAD_Q), hb.N + 1);
    const size_t sm_inv = rad_inv_smem(Nr, K, sizeof(T));
    cplx_t<T>* g0 = reinterpret_cast<cplx_t<T>*>(ctx->ws.gbuf);
    const size_t region = (size_t)nc * Nr * hb.nA;
    for (int src = 0; src < 3; ++src) {
      ra.gh = g0 + (size_t)src * region;
      ra.rtab = src == 0 ? tb.rder : tb.rinv;
      ra.scale_mode = src == 0 ? 0 : (src == 1 ? 2 : 1);
      ProfScope ps(ctx, HW_PH_RADIAL_INV);
      launch_dep(ctx->stream, k_radial_inv<T>, grid, RAD_THREADS, sm_inv, ra);
      ctx->launches++;
    }
    GradArgs<T> ga;
    ga.Nr = Nr;
    ga.Nth1 = hb.prm.Nth1;
    ga.Nth2 = hb.prm.Nth2;
    ga.nA = hb.nA;
    ga.nmr = (int)hb.mrow_m.size();
    ga.ncols = nc;
    ga.Jc = Jc;
    const int ncg = std::max(1, std::min(nc, (2 * 152 + Nr - 1) / Nr));
    ga.cpg = (nc + ncg - 1) / ncg;
    ga.ncyc = hb.prm.ncyc;
    ga.alpha = hb.prm.alpha;
    ga.tau = hb.prm.tau;
    ga.p1 = to_dev(ctx->plan1);
    ga.p2 = to_dev(ctx->plan2);
    ga.pair_n = db.pair_n;
    ga.pair_mrow = db.pair_mrow;
    ga.mrow_m = db.mrow_m;
    ga.tw1 = reinterpret_cast<const cplx_t<T>*>(tb.tw1);
    ga.tw2 = reinterpret_cast<const cplx_t<T>*>(tb.tw2);
    ga.G = g0;
    ga.rnodes = db.rnodes;
    ga.D = reinterpret_cast<double2*>(D) + (size_t)c0 * 3 * grid_pts;
    void* args[] = {(void*)&ga};
    {
      ProfScope ps(ctx, HW_PH_GRADIENT);
      // a plain launch: overlapped with the radial kernels before it (200 KB of shared memory
      // per CTA, one CTA per SM) the 16-column mixed gradient measured 1.27 -> 1.67 ms per call
      e = cudaLaunchKernel(kf, dim3(Nr, (nc + ga.cpg - 1) / ga.cpg), dim3(SLAB_THREADS), args, sm, ctx->stream);
      ctx->launches++;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}
template cudaError_t launch_gradient<double>(hw_ctx*, const Blocks&, int, int64_t, double*);
template cudaError_t launch_gradient<float>(hw_ctx*, const Blocks&, int, int64_t, double*);

// opt in to large dynamic shared memory for every instantiation (called once at setup)
cudaError_t hx_configure(hw_ctx* ctx) {
  cudaError_t e = cudaSuccess;
  const int big = 200 * 1024;
  e = cudaFuncSetAttribute(k_radial_inv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radial_inv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radial_fwd<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radial_fwd<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radial_inv_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_radial_fwd_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  for (void* f : {(void*)k_slab<double, 0, 0>, (void*)k_slab<float, 0, 0>, (void*)k_slab<double, 64, 48>,
                  (void*)k_slab<float, 64, 48>, (void*)k_slab<double, 192, 96>, (void*)k_slab<float, 192, 96>,
                  (void*)k_slab_r16<float, 64, 48>, (void*)k_slab_r16<double, 64, 48>, (void*)k_slab_q<float>,
                  (void*)k_slab_q<double>, (void*)k_slab_q<double, ff>})
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  (void)ctx;
  return e;
}

// ---------------------------------------------------------------------------- autotuner
// Times the H X pipeline on `ns` random-free columns (zeros are enough: the kernels' work does
// not depend on the values) for candidate slab theta2 chunks and column-pass widths and keeps
// the fastest per precision.
template <typename T>
static float time_hx(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, cudaEvent_t e0, cudaEvent_t e1) {
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, ctx->stream);
    if (launch_hx<T>(ctx, blk, ns, ld) != cudaSuccess) return 1e30f;
    cudaEventRecord(e1, ctx->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  return best;
}

template <typename T>
static void tune_one(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, cudaEvent_t e0, cudaEvent_t e1,
                     std::vector<float>& log) {
  const int ti = sizeof(T) == 8 ? 0 : 1;
  const auto& hb = ctx->hb;
  std::vector<int> jcs;
  for (int j = hb.prm.Nth2; j >= 1; j = (j > 1 ? (j + 1) / 2 : 0)) {
    if (slab_smem_bytes(ctx, sizeof(cplx_t<T>), j) <= 200 * 1024) jcs.push_back(j);
    if (j == 1) break;
  }
  float best = 1e30f;
  int bj = 0, bc = 0;
  const int cap = (int)ctx->ws.cols;
  const int passes[4] = {cap, std::min(cap, 512), std::min(cap, 128), std::min(cap, 32)};
  for (int jc : jcs) {
    if (jcs.size() > 4 && jc < 4) continue;
    for (int pc : passes) {
      ctx->ws.jc[ti] = jc;
      ctx->ws.pass_cols[ti] = pc;
      const float t = time_hx<T>(ctx, blk, ns, ld, e0, e1);
      log.push_back((float)ti);
      log.push_back((float)jc);
      log.push_back((float)pc);
      log.push_back(t);
      if (t < best) {
        best = t;
        bj = jc;
        bc = pc;
      }
    }
  }
  ctx->ws.jc[ti] = bj;
  ctx->ws.pass_cols[ti] = bc;
}

cudaError_t hx_autotune(hw_ctx* ctx, int k, int ns, std::vector<float>& log) {
  const int64_t L = ctx->hb.L[k];
  double2* X = nullptr;
  double2* Y = nullptr;
  cudaError_t e = cudaMalloc((void**)&X, (size_t)L * ns * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&Y, (size_t)L * ns * sizeof(double2));
  if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, (size_t)L * ns * sizeof(double2), ctx->stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    Blocks blk;
    blk.nslot = 1;
    blk.x[0] = reinterpret_cast<const double*>(X);
    blk.y[0] = reinterpret_cast<double*>(Y);
    blk.kb[0] = k;
    tune_one<double>(ctx, blk, ns, L, e0, e1, log);
    tune_one<float>(ctx, blk, ns, L, e0, e1, log);
    e = cudaStreamSynchronize(ctx->stream);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (X) cudaFree(X);
  if (Y) cudaFree(Y);
  return e;
}

template cudaError_t launch_hx<double>(hw_ctx*, const Blocks&, int, int64_t, const ChebStep*);
template cudaError_t launch_hx<float>(hw_ctx*, const Blocks&, int, int64_t, const ChebStep*);

}  // namespace hw
