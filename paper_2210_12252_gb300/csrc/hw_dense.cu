// Small dense FP64 linear algebra for the block eigensolver, batched over k-points:
//
//   k_chol        in-place Cholesky G = L L^H of a Hermitian positive definite n x n matrix
//                 (Cholesky-QR of the search directions); one CTA per problem, the matrix
//                 staged in shared memory.  A non-positive pivot sets the problem's fail flag.
//   k_trinv       L^{-1} of a lower-triangular matrix, written as the upper-triangular U^{-1}
//                 with U = L^H, so that W U^{-1} is a plain GEMM.
//   k_jacobi      all eigenpairs of nprob Hermitian n x n matrices by the parallel cyclic
//                 two-sided Jacobi method (round-robin pairing, n/2 disjoint rotations per
//                 step, one grid barrier per step); cooperative launch, bounded barrier waits.
//   k_eig_sort    ascending eigenvalues with eigenvector columns permuted accordingly.
//
// Problems carry a "valid size" nv <= n: entries beyond it are padding.  Gram matrices get an
// identity there (so Cholesky passes through), Rayleigh-Ritz matrices a huge diagonal (so the
// padding sorts last).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "hw_common.cuh"
#include "hw_ctx.h"

namespace hw {

// ---------------------------------------------------------------------- padding helpers
// G[b] (n x n, column-major, stride sG): zero rows/cols >= nv[b], diagonal = diagval (+ index)
__global__ void k_pad_square(double2* G, int n, int64_t sG, const int* nv, double diagval, int ramp) {
  griddep_entry();
  const int b = blockIdx.y;
  double2* g = G + (size_t)b * sG;
  const int v = nv[b];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
    const int i = t % n, j = t / n;
    if (i >= v || j >= v) {
      double2 z;
      z.x = (i == j) ? diagval + (ramp ? double(i) : 0.0) : 0.0;
      z.y = 0.0;
      g[t] = z;
    }
  }
}

// A = (A + A^H) / 2 in place
__global__ void k_hermitize(double2* A, int n, int64_t sA) {
  griddep_entry();
  const int b = blockIdx.y;
  double2* a = A + (size_t)b * sA;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
    const int i = t % n, j = t / n;
    if (i > j) continue;
    const double2 x = a[i + (size_t)j * n], y = a[j + (size_t)i * n];
    double2 m;
    m.x = 0.5 * (x.x + y.x);
    m.y = 0.5 * (x.y - y.y);
    if (i == j) m.y = 0.0;
    a[i + (size_t)j * n] = m;
    double2 mc = m;
    mc.y = -m.y;
    a[j + (size_t)i * n] = mc;
  }
}

// ---------------------------------------------------------------------- Cholesky
constexpr int CHOL_THREADS = 1024;

template <typename T> struct Cx;
template <> struct Cx<double> { using t = double2; };
template <> struct Cx<float> { using t = float2; };

// lower Cholesky in place (upper triangle zeroed); fail[b] = 1 + column of a bad pivot.
// Blocked right-looking with CHOL_NB-column panels, three block barriers per panel: warp 0
// factors the diagonal block (warp-synchronous), one thread per row solves the panel below
// it with the row held in registers, and all warps apply the rank-CHOL_NB update to the
// trailing lower triangle (a warp per column, lanes over rows: contiguous shared-memory reads).
// T is the arithmetic type.  T = double: the factor overwrites G (complex128).  T = float (the
// FP32-product phase): G is read as complex128 and the factor is written as complex64 into
// the first n*n*8 bytes of each problem's slot, which is what the FP32 triangular solve reads.
constexpr int CHOL_NB = 16;

template <typename T> __device__ __forceinline__ typename Cx<T>::t ld_c(const double2& x);
template <> __device__ __forceinline__ double2 ld_c<double>(const double2& x) { return x; }
template <> __device__ __forceinline__ float2 ld_c<float>(const double2& x) { return d2f(x); }

template <typename T>
__global__ void __launch_bounds__(CHOL_THREADS) k_chol(double2* G, int n, int64_t sG, int* fail, int use_smem) {
  griddep_entry();
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  double2* g = G + (size_t)b * sG;
  C* a = use_smem ? reinterpret_cast<C*>(smem_raw) : reinterpret_cast<C*>(g);   // global only for T = double
  __shared__ int bad;
  __shared__ T rdiag[CHOL_NB];
  if (threadIdx.x == 0) bad = 0;
  if (use_smem)
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) a[t] = ld_c<T>(g[t]);
  __syncthreads();
  for (int jb = 0; jb < n; jb += CHOL_NB) {
    const int nb = min(CHOL_NB, n - jb);
    // (1) diagonal block, warp 0
    if (warp == 0) {
      for (int c = 0; c < nb; ++c) {
        const int col = jb + c;
        T d = a[col + (size_t)col * n].x;
        const bool ok = d > (T)0 && isfinite(d);
        if (!ok) {
          if (lane == 0) bad = col + 1;
          break;   // warp-uniform
        }
        const T sq = sqrt(d), inv = (T)1 / sq;
        if (lane == 0) rdiag[c] = inv;
        if (lane == c) a[col + (size_t)col * n] = C{sq, (T)0};
        if (lane > c && lane < nb) {
          C v = a[jb + lane + (size_t)col * n];
          v.x *= inv;
          v.y *= inv;
          a[jb + lane + (size_t)col * n] = v;
        }
        __syncwarp();
        // update the rest of the diagonal block: a[i][k] -= l[i][c] conj(l[k][c]), c < k <= i < nb
        for (int t = lane; t < CHOL_NB * CHOL_NB; t += 32) {
          const int i = t % CHOL_NB, k = t / CHOL_NB;
          if (k > c && k <= i && i < nb) {
            const C li = a[jb + i + (size_t)col * n], lk = a[jb + k + (size_t)col * n];
            C v = a[jb + i + (size_t)(jb + k) * n];
            v.x -= li.x * lk.x + li.y * lk.y;
            v.y -= li.y * lk.x - li.x * lk.y;
            a[jb + i + (size_t)(jb + k) * n] = v;
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (bad) break;
    // (2) panel: row i >= jb + nb solves x L_d^H = a (row in registers):
    //     x_c = (a_c - sum_{cc<c} x_cc conj(L_d[c][cc])) / L_d[c][c]
    for (int i = jb + nb + threadIdx.x; i < n; i += blockDim.x) {
      C x[CHOL_NB];
#pragma unroll
      for (int c = 0; c < CHOL_NB; ++c) x[c] = c < nb ? a[i + (size_t)(jb + c) * n] : C{(T)0, (T)0};
#pragma unroll
      for (int c = 0; c < CHOL_NB; ++c) {
        if (c < nb) {
          C v = x[c];
#pragma unroll
          for (int cc = 0; cc < c; ++cc) {
            const C l = a[jb + c + (size_t)(jb + cc) * n];
            v.x -= x[cc].x * l.x + x[cc].y * l.y;
            v.y -= x[cc].y * l.x - x[cc].x * l.y;
          }
          v.x *= rdiag[c];
          v.y *= rdiag[c];
          x[c] = v;
        }
      }
#pragma unroll
      for (int c = 0; c < CHOL_NB; ++c)
        if (c < nb) a[i + (size_t)(jb + c) * n] = x[c];
    }
    __syncthreads();
    // (3) trailing update of the lower triangle: a[i][k] -= sum_c l[i][c] conj(l[k][c])
    for (int k = jb + nb + warp; k < n; k += nwarp) {
      for (int i = k + lane; i < n; i += 32) {
        C v = a[i + (size_t)k * n];
        for (int c = 0; c < nb; ++c) {
          const C li = a[i + (size_t)(jb + c) * n], lk = a[k + (size_t)(jb + c) * n];
          v.x -= li.x * lk.x + li.y * lk.y;
          v.y -= li.y * lk.x - li.x * lk.y;
        }
        a[i + (size_t)k * n] = v;
      }
    }
    __syncthreads();
  }
  // zero the strict upper triangle
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t % n, k = t / n;
    if (k > i) a[t].x = a[t].y = (T)0;
  }
  __syncthreads();
  if (use_smem) {
    if (sizeof(T) == sizeof(float)) {
      float2* gf = reinterpret_cast<float2*>(g);
      for (int t = threadIdx.x; t < n * n; t += blockDim.x) gf[t] = make_float2((float)a[t].x, (float)a[t].y);
    } else {
      for (int t = threadIdx.x; t < n * n; t += blockDim.x) g[t] = make_double2((double)a[t].x, (double)a[t].y);
    }
  }
  if (threadIdx.x == 0) fail[b] = bad;
}

// Unblocked right-looking Cholesky for the solver's block sizes (n <= CHS_NMAX), one CTA of
// CHS_THREADS per problem, one barrier per column: the lower triangle sits row-major in shared
// memory with an odd row pitch (n | 1: a warp's reads down a column fall in distinct banks);
// every thread reads the pivot d = a[c][c] itself and applies
//   a[i][k] -= a[i][c] conj(a[k][c]) / d,   c < k <= i,
// a warp per trailing row i (round robin), its lanes across k; the columns are scaled by
// 1 / sqrt(d) at the end.  Same input, output and fail[] contract as k_chol (a pivot that is
// not positive and finite stops the factorisation: fail = 1 + its column).
constexpr int CHS_THREADS = 512;
constexpr int CHS_NMAX = 112;

template <typename T>
__global__ void __launch_bounds__(CHS_THREADS) k_chol_small(double2* G, int n, int64_t sG, int* fail) {
  griddep_entry();
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* a = reinterpret_cast<C*>(smem_raw);
  const int b = blockIdx.x, ld = n | 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  double2* g = G + (size_t)b * sG;
  for (int k = warp; k < n; k += nwarp)   // column k of the source (column-major), rows i >= k
    for (int i = k + lane; i < n; i += 32) a[i * ld + k] = ld_c<T>(g[i + (size_t)k * n]);
  __syncthreads();
  int bad = 0;
  for (int c = 0; c < n; ++c) {
    const T d = a[c * ld + c].x;   // the same value for every thread: a uniform stop
    if (!(d > (T)0) || !isfinite(d)) {
      bad = c + 1;
      break;
    }
    const T id = (T)1 / d;
    for (int i = c + 1 + warp; i < n; i += nwarp) {
      const C li = a[i * ld + c];
      for (int k = c + 1 + lane; k <= i; k += 32) {
        const C lk = a[k * ld + c];
        C v = a[i * ld + k];
        v.x -= (li.x * lk.x + li.y * lk.y) * id;
        v.y -= (li.y * lk.x - li.x * lk.y) * id;
        a[i * ld + k] = v;
      }
    }
    __syncthreads();
  }
  if (!bad) {   // (uniform) scale: L[i][c] = a[i][c] / sqrt(a[c][c]), the roots taken first
    T* sq = reinterpret_cast<T*>(a + (size_t)n * ld);   // [n]
    for (int c = threadIdx.x; c < n; c += blockDim.x) sq[c] = sqrt(a[c * ld + c].x);
    __syncthreads();
    for (int i = warp; i < n; i += nwarp)
      for (int c = lane; c <= i; c += 32) {
        C v = a[i * ld + c];
        if (i == c) {
          v.x = sq[c];
          v.y = (T)0;
        } else {
          v.x /= sq[c];
          v.y /= sq[c];
        }
        a[i * ld + c] = v;
      }
  }
  __syncthreads();
  // out: column-major, zeros above the diagonal; complex64 into the first n*n*8 bytes of the
  // problem's slot for T = float (what the FP32 triangular solve reads), complex128 otherwise
  for (int k = warp; k < n; k += nwarp)
    for (int i = lane; i < n; i += 32) {
      const C v = i >= k ? a[i * ld + k] : C{(T)0, (T)0};
      const size_t t = i + (size_t)k * n;
      if (sizeof(T) == sizeof(float))
        reinterpret_cast<float2*>(g)[t] = make_float2((float)v.x, (float)v.y);
      else
        g[t] = make_double2((double)v.x, (double)v.y);
    }
  if (threadIdx.x == 0) fail[b] = bad;
}

// Given lower L (n x n), write Uinv = (L^H)^{-1} (upper triangular) into Ui.  Column j of
// L^{-1} by forward substitution (one thread per column); Uinv = (L^{-1})^H.
__global__ void k_trinv(const double2* L, int64_t sL, double2* Ui, int64_t sU, int n) {
  griddep_entry();
  const int b = blockIdx.y;
  const double2* l = L + (size_t)b * sL;
  double2* u = Ui + (size_t)b * sU;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  // x = L^{-1} e_j: x[i] = 0 for i < j; then store conj(x[i]) at u[j][i] (row j, column i)
  for (int i = 0; i < n; ++i) u[j + (size_t)i * n] = make_double2(0.0, 0.0);
  for (int i = j; i < n; ++i) {
    double sr = (i == j) ? 1.0 : 0.0, si = 0.0;
    for (int k = j; k < i; ++k) {
      const double2 lik = l[i + (size_t)k * n];
      const double2 xk = u[j + (size_t)k * n];   // conj(x[k]) stored
      // s -= l[i][k] * x[k]  with x[k] = conj(xk)
      sr -= lik.x * xk.x + lik.y * xk.y;
      si -= lik.y * xk.x - lik.x * xk.y;
    }
    const double2 lii = l[i + (size_t)i * n];      // real positive
    const double inv = 1.0 / lii.x;
    u[j + (size_t)i * n] = make_double2(sr * inv, -si * inv);
  }
}

// ---------------------------------------------------------------------- grid barrier
struct GridBar {
  unsigned int count;
  unsigned int gen;
  int abort;
  int pad;
};

// Default bound of a barrier wait: 2^24 polls with 100 ns sleeps, about 2 s.
constexpr long GRID_SPIN_LIMIT = 1L << 24;

// returns false when the barrier gave up (error flag set; the caller leaves the kernel).  A
// CTA that waits more than spin_limit polls sets bar->abort and *status = HW_ETIMEOUT; the
// CTAs still waiting see the abort and leave too.
__device__ bool grid_sync(GridBar* bar, int* status, long spin_limit = GRID_SPIN_LIMIT) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = &bar->gen;
    volatile int* vab = &bar->abort;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == gridDim.x - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long spins = 0;
      while (*vgen == g) {
        if (*vab) { ok = 0; break; }
        if (++spins > spin_limit) {
          atomicExch(&bar->abort, 1);
          atomicExch(status, HW_ETIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// ---------------------------------------------------------------------- Jacobi
struct JacArgs {
  int nprob, n, maxsweep;
  double tol;           // rotation threshold relative to ||A||_F
  double2* A0;          // [nprob][n*n] input (destroyed)
  double2* A1;          // [nprob][n*n] scratch
  double2* V;           // [nprob][n*n] eigenvectors (columns)
  int* rotated;         // [maxsweep+1] rotations applied per sweep (zeroed by the host)
  double* fro;          // [nprob] ||A||_F^2 (zeroed by the host)
  GridBar* bar;
  int* status;
  int* sweeps_done;
};

__device__ __forceinline__ int rr_index(int pos, int t, int n) {
  return pos == 0 ? 0 : 1 + (pos - 1 + t) % (n - 1);
}

// one rotation of the current step: pair (p < q), cos/sin, phase e = c/|c|, and the new
// diagonal entries of the pair
struct Rot {
  int p, q;
  double cs, sn, er, ei;
  double app, aqq;
};

// The rotation angle is computed in FP32 (no FP64 division or square root, which are slow
// on this GPU); the cosine/sine pair and the phase are then renormalised in FP64 by one
// Newton step for 1/sqrt(x) about 1, so the applied rotation is unitary to FP64 rounding.
// An inexact angle only leaves a residual coupling ~1e-7 |c| that later sweeps remove.
__device__ __forceinline__ double renorm(double x2) {   // ~1/sqrt(x2) for x2 = 1 + O(1e-7)
  const double d = x2 - 1.0;
  return 1.0 - 0.5 * d + 0.375 * d * d;
}

__device__ __forceinline__ Rot make_rot(const double2* a, int n, int p, int q, double thr) {
  Rot r;
  r.p = p;
  r.q = q;
  const double app = a[p + (size_t)p * n].x, aqq = a[q + (size_t)q * n].x;
  const double2 c = a[p + (size_t)q * n];
  const double c2 = c.x * c.x + c.y * c.y;
  r.app = app;
  r.aqq = aqq;
  if (!(c2 > thr * thr)) {   // negligible coupling: no rotation (keeps padding exactly decoupled)
    r.cs = 1.0; r.sn = 0.0; r.er = 1.0; r.ei = 0.0;
    return r;
  }
  const float acf = sqrtf((float)c2);
  const float zeta = (float)(aqq - app) / (2.0f * acf);
  const float t = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
  const float csf = rsqrtf(1.0f + t * t);
  double cs = csf, sn = (double)(t * csf);
  double sc = renorm(cs * cs + sn * sn);
  r.cs = cs * sc;
  r.sn = sn * sc;
  const float inv = 1.0f / acf;
  double er = (double)((float)c.x * inv), ei = (double)((float)c.y * inv);
  sc = renorm(er * er + ei * ei);
  r.er = er * sc;
  r.ei = ei * sc;
  return r;
}

// Grid-stride over (problem, block I, block J) and (problem, row, block I).  Every CTA first
// computes the step's rotations of all problems into shared memory (cheap, one per thread),
// then applies them; one grid barrier per step.  A sweep without any rotation above the
// threshold ends the iteration.
__global__ void __launch_bounds__(256) k_jacobi(JacArgs J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Rot* rot = reinterpret_cast<Rot*>(smem_raw);   // [nprob][n/2]
  __shared__ double thr_s[64];
  const int n = J.n, h = n / 2;
  const long nAh = (long)h * (h + 1) / 2;   // lower-triangle blocks per problem
  const long nA = (long)J.nprob * nAh;
  const long nV = (long)J.nprob * n * h;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long nth = (long)gridDim.x * blockDim.x;
  for (long t = tid; t < (long)J.nprob * n * n; t += nth) {
    const int b = (int)(t / ((long)n * n));
    const double2 v = J.A0[t];
    const double m2 = v.x * v.x + v.y * v.y;
    if (m2 < 1e18) atomicAdd(&J.fro[b], m2);   // padding entries (>= 1e9) do not count
  }
  if (!grid_sync(J.bar, J.status)) return;
  for (int b = threadIdx.x; b < J.nprob && b < 64; b += blockDim.x)
    thr_s[b] = J.tol * sqrt(J.fro[b]) + 1e-300;
  __syncthreads();
  double2* Acur = J.A0;
  double2* Anext = J.A1;
  int sweep = 0;
  for (; sweep < J.maxsweep; ++sweep) {
    int nrot = 0;
    for (int step = 0; step < n - 1; ++step) {
      // rotations of this step (identical in every CTA)
      for (int i = threadIdx.x; i < J.nprob * h; i += blockDim.x) {
        const int b = i / h, I = i - b * h;
        const int pI = rr_index(I, step, n), qI = rr_index(n - 1 - I, step, n);
        const Rot r = make_rot(Acur + (size_t)b * n * n, n, min(pI, qI), max(pI, qI), thr_s[b < 64 ? b : 63]);
        rot[i] = r;
        if (blockIdx.x == 0 && r.sn != 0.0) nrot = 1;
      }
      __syncthreads();
      for (long t = tid; t < nA + nV; t += nth) {
        if (t < nA) {
          const int b = (int)(t / nAh);
          const int rem = (int)(t - (long)b * nAh);
          // rem -> (I, Jb) with I >= Jb (row-major lower triangle of the h x h block grid)
          int I = (int)((sqrtf(8.0f * rem + 1.0f) - 1.0f) * 0.5f);
          while ((I + 1) * (I + 2) / 2 <= rem) ++I;
          while (I * (I + 1) / 2 > rem) --I;
          const int Jb = rem - I * (I + 1) / 2;
          const double2* a = Acur + (size_t)b * n * n;
          double2* an = Anext + (size_t)b * n * n;
          const Rot r1 = rot[b * h + I];
          const Rot r2 = rot[b * h + Jb];
          const int p1 = r1.p, q1 = r1.q, p2 = r2.p, q2 = r2.q;
          const double2 A_pp = a[p1 + (size_t)p2 * n], A_pq = a[p1 + (size_t)q2 * n];
          const double2 A_qp = a[q1 + (size_t)p2 * n], A_qq = a[q1 + (size_t)q2 * n];
          // M = J1^H A_blk: row p = cs A[p,:] - sn e1 A[q,:];  row q = sn A[p,:] + cs e1 A[q,:]
          const double2 eq_p = make_double2(r1.er * A_qp.x - r1.ei * A_qp.y, r1.er * A_qp.y + r1.ei * A_qp.x);
          const double2 eq_q = make_double2(r1.er * A_qq.x - r1.ei * A_qq.y, r1.er * A_qq.y + r1.ei * A_qq.x);
          const double2 M_pp = make_double2(r1.cs * A_pp.x - r1.sn * eq_p.x, r1.cs * A_pp.y - r1.sn * eq_p.y);
          const double2 M_pq = make_double2(r1.cs * A_pq.x - r1.sn * eq_q.x, r1.cs * A_pq.y - r1.sn * eq_q.y);
          const double2 M_qp = make_double2(r1.sn * A_pp.x + r1.cs * eq_p.x, r1.sn * A_pp.y + r1.cs * eq_p.y);
          const double2 M_qq = make_double2(r1.sn * A_pq.x + r1.cs * eq_q.x, r1.sn * A_pq.y + r1.cs * eq_q.y);
          // M J2: col p = cs M[:,p] - sn conj(e2) M[:,q];  col q = sn M[:,p] + cs conj(e2) M[:,q]
          const double2 cq_p = make_double2(r2.er * M_pq.x + r2.ei * M_pq.y, r2.er * M_pq.y - r2.ei * M_pq.x);
          const double2 cq_q = make_double2(r2.er * M_qq.x + r2.ei * M_qq.y, r2.er * M_qq.y - r2.ei * M_qq.x);
          const double2 o_pp = make_double2(r2.cs * M_pp.x - r2.sn * cq_p.x, r2.cs * M_pp.y - r2.sn * cq_p.y);
          const double2 o_qp = make_double2(r2.cs * M_qp.x - r2.sn * cq_q.x, r2.cs * M_qp.y - r2.sn * cq_q.y);
          const double2 o_pq = make_double2(r2.sn * M_pp.x + r2.cs * cq_p.x, r2.sn * M_pp.y + r2.cs * cq_p.y);
          const double2 o_qq = make_double2(r2.sn * M_qp.x + r2.cs * cq_q.x, r2.sn * M_qp.y + r2.cs * cq_q.y);
          if (I == Jb) {   // diagonal block: Hermitian by construction, keep it exactly so
            an[p1 + (size_t)p1 * n] = make_double2(o_pp.x, 0.0);
            an[q1 + (size_t)q1 * n] = make_double2(o_qq.x, 0.0);
            const double2 m = make_double2(0.5 * (o_pq.x + o_qp.x), 0.5 * (o_pq.y - o_qp.y));
            an[p1 + (size_t)q1 * n] = m;
            an[q1 + (size_t)p1 * n] = make_double2(m.x, -m.y);
            continue;
          }
          an[p1 + (size_t)p2 * n] = o_pp;
          an[q1 + (size_t)p2 * n] = o_qp;
          an[p1 + (size_t)q2 * n] = o_pq;
          an[q1 + (size_t)q2 * n] = o_qq;
          // mirrored block (J, I) = conjugate transpose
          an[p2 + (size_t)p1 * n] = make_double2(o_pp.x, -o_pp.y);
          an[p2 + (size_t)q1 * n] = make_double2(o_qp.x, -o_qp.y);
          an[q2 + (size_t)p1 * n] = make_double2(o_pq.x, -o_pq.y);
          an[q2 + (size_t)q1 * n] = make_double2(o_qq.x, -o_qq.y);
        } else {
          const long u = t - nA;
          const int b = (int)(u / ((long)n * h));
          const int rem = (int)(u - (long)b * n * h);
          const int row = rem % n, I = rem / n;
          const Rot r = rot[b * h + I];
          if (r.sn == 0.0) continue;
          double2* v = J.V + (size_t)b * n * n;
          const double2 vp = v[row + (size_t)r.p * n], vq = v[row + (size_t)r.q * n];
          // V' col p = cs vp - sn conj(e) vq;  col q = sn vp + cs conj(e) vq
          const double2 cv = make_double2(r.er * vq.x + r.ei * vq.y, r.er * vq.y - r.ei * vq.x);
          v[row + (size_t)r.p * n] = make_double2(r.cs * vp.x - r.sn * cv.x, r.cs * vp.y - r.sn * cv.y);
          v[row + (size_t)r.q * n] = make_double2(r.sn * vp.x + r.cs * cv.x, r.sn * vp.y + r.cs * cv.y);
        }
      }
      if (!grid_sync(J.bar, J.status)) return;
      double2* tmp = Acur;
      Acur = Anext;
      Anext = tmp;
    }
    // CTA 0 reports whether this sweep rotated anything (visible after the next barrier)
    if (blockIdx.x == 0) {
      nrot = __syncthreads_or(nrot);
      if (threadIdx.x == 0) J.rotated[sweep] = nrot;
    }
    if (!grid_sync(J.bar, J.status)) return;
    if (*((volatile int*)&J.rotated[sweep]) == 0) {
      ++sweep;
      break;
    }
  }
  // make sure the result sits in A0
  if (Acur != J.A0) {
    for (long t = tid; t < (long)J.nprob * n * n; t += nth) J.A0[t] = Acur[t];
  }
  if (tid == 0) *J.sweeps_done = sweep;
}

// eigenvalues ascending: w[b][i], vectors Z[b] columns permuted (Z may not alias V)
__global__ void k_eig_sort(const double2* A, const double2* V, int n, double* w, double2* Z) {
  griddep_entry();
  const int b = blockIdx.x;
  const double2* a = A + (size_t)b * n * n;
  const double2* v = V + (size_t)b * n * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = a[i + (size_t)i * n].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = a[j + (size_t)j * n].x;
      rank += (dj < di) || (dj == di && j < i);
    }
    w[(size_t)b * n + rank] = di;
    for (int r = 0; r < n; ++r) Z[(size_t)b * n * n + r + (size_t)rank * n] = v[r + (size_t)i * n];
  }
}

__global__ void k_identity(double2* V, int n, int nprob) {
  griddep_entry();
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < (long)nprob * n * n;
       t += (long)gridDim.x * blockDim.x) {
    const int r = (int)(t % n), c = (int)((t / n) % n);
    V[t] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  }
}

// ---------------------------------------------------------------------- host wrappers
struct DenseWork {
  double2* A1 = nullptr;
  double2* V = nullptr;
  int* rotated = nullptr;
  double* fro = nullptr;
  GridBar* bar = nullptr;
  int* sweeps = nullptr;
  size_t cap = 0;       // elements of A1 / V
  int maxsweep = 40;
  int coop_blocks = 0;
};


cudaError_t dense_alloc(DenseWork*& dw, size_t cap_elems, int maxnprob) {
  if (!dw) dw = new DenseWork();
  if (dw->cap >= cap_elems && dw->A1) return cudaSuccess;
  if (dw->A1) cudaFree(dw->A1);
  if (dw->V) cudaFree(dw->V);
  if (dw->rotated) cudaFree(dw->rotated);
  if (dw->fro) cudaFree(dw->fro);
  if (dw->bar) cudaFree(dw->bar);
  if (dw->sweeps) cudaFree(dw->sweeps);
  cudaError_t e = cudaMalloc((void**)&dw->A1, cap_elems * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw->V, cap_elems * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw->rotated, (size_t)(dw->maxsweep + 1) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw->fro, (size_t)maxnprob * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw->bar, sizeof(GridBar));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dw->sweeps, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(dw->bar, 0, sizeof(GridBar));
  dw->cap = cap_elems;
  if (e == cudaSuccess) {
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jacobi, 256, 200 * 1024);
    dw->coop_blocks = nsm * std::max(1, std::min(occ, 1));
  }
  return e;
}

void dense_free(DenseWork*& dw) {
  if (!dw) return;
  for (void* p : {(void*)dw->A1, (void*)dw->V, (void*)dw->rotated, (void*)dw->fro, (void*)dw->bar,
                  (void*)dw->sweeps})
    if (p) cudaFree(p);
  delete dw;
  dw = nullptr;
}

// Self-test of the bounded barrier wait: `rounds` grid barriers over the grid; the CTA
// `skip_block` (if >= 0) leaves before the first one, so the others can never be released and
// must give up after spin_limit polls with HW_ETIMEOUT in *status.
__global__ void k_barrier_selftest(GridBar* bar, int* status, long spin_limit, int skip_block, int rounds) {
  if ((int)blockIdx.x == skip_block) return;
  for (int r = 0; r < rounds; ++r)
    if (!grid_sync(bar, status, spin_limit)) return;
}

// Runs k_barrier_selftest as a cooperative launch (all CTAs co-resident) of nblocks CTAs on
// `st`, waits for it, and returns the device status word (HW_OK or HW_ETIMEOUT) in *wait_status.
cudaError_t dense_barrier_selftest(cudaStream_t st, int nblocks, long spin_limit, int skip_block,
                                   int* wait_status) {
  GridBar* bar = nullptr;
  int* status = nullptr;
  cudaError_t e = cudaMalloc((void**)&bar, sizeof(GridBar));
  if (e == cudaSuccess) e = cudaMalloc((void**)&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, sizeof(GridBar), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  int rounds = 3;
  void* args[] = {&bar, &status, &spin_limit, &skip_block, &rounds};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((void*)k_barrier_selftest, dim3(nblocks), dim3(128), args, 0, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(wait_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (bar) cudaFree(bar);
  if (status) cudaFree(status);
  return e;
}

// Eigen-decomposition of nprob Hermitian n x n matrices A (contiguous, n*n each; destroyed):
// w [nprob][n] ascending, Z [nprob][n*n] eigenvector columns.  status: device int (HW_*).
cudaError_t dense_heev(DenseWork* dw, cudaStream_t st, double2* A, int n, int nprob, double* w,
                       double2* Z, int* status, double tol) {
  const size_t elems = (size_t)nprob * n * n;
  if (elems > dw->cap || (n & 1)) return cudaErrorInvalidValue;
  launch_dep(st, k_identity, 256, 256, 0, dw->V, n, nprob);
  cudaMemsetAsync(dw->rotated, 0, (size_t)(dw->maxsweep + 1) * sizeof(int), st);
  cudaMemsetAsync(dw->fro, 0, (size_t)nprob * sizeof(double), st);
  cudaMemsetAsync(dw->bar, 0, sizeof(GridBar), st);
  JacArgs ja;
  ja.nprob = nprob;
  ja.n = n;
  ja.maxsweep = dw->maxsweep;
  ja.tol = tol;
  ja.A0 = A;
  ja.A1 = dw->A1;
  ja.V = dw->V;
  ja.rotated = dw->rotated;
  ja.fro = dw->fro;
  ja.bar = dw->bar;
  ja.status = status;
  ja.sweeps_done = dw->sweeps;
  void* args[] = {&ja};
  const size_t smem = (size_t)nprob * (n / 2) * sizeof(Rot);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  // grid: enough CTAs for ~2 items per thread, at most the co-resident count
  const long items = (long)nprob * (n / 2) * (n / 2 + 1) / 2 + (long)nprob * n * (n / 2);
  int blocks = (int)std::min<long>(dw->coop_blocks, std::max<long>(8, (items + 511) / 512));
  cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_jacobi, dim3(blocks), dim3(256), args, smem, st);
  if (e != cudaSuccess) return e;
  launch_dep(st, k_eig_sort, nprob, 256, 0, A, dw->V, n, w, Z);
  return cudaGetLastError();
}

static size_t chol_small_smem(int n, size_t elem) { return (size_t)n * (n | 1) * elem + (size_t)n * (elem / 2); }

cudaError_t dense_chol(cudaStream_t st, double2* G, int n, int nprob, int* fail, bool fp32) {
  if (n <= CHS_NMAX) {   // the solver's block sizes: the unblocked kernel
    if (fp32) {
      cudaFuncSetAttribute(k_chol_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      launch_dep(st, k_chol_small<float>, nprob, CHS_THREADS, chol_small_smem(n, sizeof(float2)), G, n, (int64_t)n * n, fail);
    } else {
      cudaFuncSetAttribute(k_chol_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
      launch_dep(st, k_chol_small<double>, nprob, CHS_THREADS, chol_small_smem(n, sizeof(double2)), G, n, (int64_t)n * n,
                                                                                             fail);
    }
    return cudaGetLastError();
  }
  if (fp32) {
    const size_t bytes = (size_t)n * n * sizeof(float2);
    if (bytes > 200 * 1024) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(k_chol<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    launch_dep(st, k_chol<float>, nprob, CHOL_THREADS, bytes, G, n, (int64_t)n * n, fail, 1);
    return cudaGetLastError();
  }
  const size_t bytes = (size_t)n * n * sizeof(double2);
  const int use_smem = bytes <= 200 * 1024;
  if (use_smem) cudaFuncSetAttribute(k_chol<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  launch_dep(st, k_chol<double>, nprob, CHOL_THREADS, use_smem ? bytes : 0, G, n, (int64_t)n * n, fail, use_smem);
  return cudaGetLastError();
}

cudaError_t dense_trinv(cudaStream_t st, const double2* L, double2* Ui, int n, int nprob) {
  launch_dep(st, k_trinv, dim3((n + 63) / 64, nprob), 64, 0, L, (int64_t)n * n, Ui, (int64_t)n * n, n);
  return cudaGetLastError();
}

cudaError_t dense_pad(cudaStream_t st, double2* G, int n, int nprob, const int* nv, double diag, int ramp) {
  launch_dep(st, k_pad_square, dim3(32, nprob), 256, 0, G, n, (int64_t)n * n, nv, diag, ramp);
  return cudaGetLastError();
}

cudaError_t dense_hermitize(cudaStream_t st, double2* A, int n, int nprob) {
  launch_dep(st, k_hermitize, dim3(32, nprob), 256, 0, A, n, (int64_t)n * n);
  return cudaGetLastError();
}

}  // namespace hw

// ===================================================================== FP32 Jacobi, one CTA
// Used while the eigensolver's residuals are large: the Rayleigh-Ritz matrix (shifted by the
// mean of its valid diagonal) is packed as a lower triangle in shared memory (n(n+1)/2
// complex FP32 values) and diagonalised by the same round-robin Jacobi as above without any
// grid barrier.  Rotations are logged to global memory; k_jac32_vectors replays the log on
// rows of the identity to form the eigenvectors.  Accuracy ~1e-7 relative; the caller
// re-orthonormalises the wanted vectors in FP64.
namespace hw {

struct Rot32 {
  float cs, sn, er, ei;
};

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }   // i >= j

__device__ __forceinline__ float2 tget(const float2* A, int r, int c) {
  if (r >= c) return A[tri(r, c)];
  const float2 v = A[tri(c, r)];
  return make_float2(v.x, -v.y);
}
__device__ __forceinline__ void tput(float2* A, int r, int c, float2 v) {
  if (r >= c) A[tri(r, c)] = v;
  else A[tri(c, r)] = make_float2(v.x, -v.y);
}

constexpr int J32_THREADS = 1024;

// grid: one CTA per problem.  A: [nprob][n*n] FP64 (read only).  shift: [nprob] output.
// log: [nprob][maxsweep][n-1][n/2] rotations.  w: [nprob][n] eigenvalues (unsorted, FP64).
__global__ void __launch_bounds__(J32_THREADS) k_jac32(const double2* A, int n, int maxsweep, double* shift,
                                                      Rot32* log, double* w, int* sweeps) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int h = n / 2;
  float2* S = reinterpret_cast<float2*>(smem_raw);
  Rot32* rot = reinterpret_cast<Rot32*>(smem_raw + (((size_t)n * (n + 1) / 2 * sizeof(float2) + 15) & ~size_t(15)));
  __shared__ double red[32];
  __shared__ float thr_s;
  __shared__ int any_s;
  const int b = blockIdx.x;
  const double2* a = A + (size_t)b * n * n;
  // shift = mean of the valid diagonal (padding entries are >= 1e9)
  double sd = 0.0, cnt = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = a[i + (size_t)i * n].x;
    if (fabs(d) < 1e9) { sd += d; cnt += 1.0; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = sd; }
  __syncthreads();
  __shared__ double mu_s;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    mu_s = t;
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    mu_s = t > 0.0 ? mu_s / t : 0.0;
    shift[b] = mu_s;
  }
  __syncthreads();
  const double mu = mu_s;
  float dmax = 0.f;
  for (int t = threadIdx.x; t < n * (n + 1) / 2; t += blockDim.x) {
    int i = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    const int j = t - i * (i + 1) / 2;
    double2 v = a[i + (size_t)j * n];
    if (i == j) {
      v.x = fabs(v.x) < 1e9 ? v.x - mu : v.x;
      v.y = 0.0;
      if (fabs(v.x) < 1e9) dmax = fmaxf(dmax, fabsf((float)v.x));
    }
    S[t] = make_float2((float)v.x, (float)v.y);
  }
  for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, (float)red[i]);
    thr_s = 2e-6f * fmaxf(m, 1e-30f);
  }
  __syncthreads();
  const float thr = thr_s;
  const int nblk = h * (h + 1) / 2;
  int sweep = 0;
  for (; sweep < maxsweep; ++sweep) {
    if (threadIdx.x == 0) any_s = 0;
    __syncthreads();
    for (int step = 0; step < n - 1; ++step) {
      for (int I = threadIdx.x; I < h; I += blockDim.x) {
        int p = rr_index(I, step, n), q = rr_index(n - 1 - I, step, n);
        if (p > q) { const int tt = p; p = q; q = tt; }
        const float app = S[tri(p, p)].x, aqq = S[tri(q, q)].x;
        const float2 c = tget(S, p, q);
        const float ac = sqrtf(c.x * c.x + c.y * c.y);
        Rot32 r;
        if (!(ac > thr)) {
          r.cs = 1.f; r.sn = 0.f; r.er = 1.f; r.ei = 0.f;
        } else {
          const float zeta = (aqq - app) / (2.0f * ac);
          const float t = copysignf(1.0f, zeta) / (fabsf(zeta) + sqrtf(1.0f + zeta * zeta));
          r.cs = rsqrtf(1.0f + t * t);
          r.sn = t * r.cs;
          r.er = c.x / ac;
          r.ei = c.y / ac;
          any_s = 1;
        }
        rot[I] = r;
        log[(((size_t)b * maxsweep + sweep) * (n - 1) + step) * h + I] = r;
      }
      __syncthreads();
      for (int it = threadIdx.x; it < nblk; it += blockDim.x) {
        int I = (int)((sqrtf(8.0f * it + 1.0f) - 1.0f) * 0.5f);
        while ((I + 1) * (I + 2) / 2 <= it) ++I;
        while (I * (I + 1) / 2 > it) --I;
        const int Jb = it - I * (I + 1) / 2;
        const Rot32 r1 = rot[I], r2 = rot[Jb];
        if (r1.sn == 0.f && r2.sn == 0.f) continue;
        int p1 = rr_index(I, step, n), q1 = rr_index(n - 1 - I, step, n);
        if (p1 > q1) { const int tt = p1; p1 = q1; q1 = tt; }
        int p2 = rr_index(Jb, step, n), q2 = rr_index(n - 1 - Jb, step, n);
        if (p2 > q2) { const int tt = p2; p2 = q2; q2 = tt; }
        const float2 A_pp = tget(S, p1, p2), A_pq = tget(S, p1, q2), A_qp = tget(S, q1, p2), A_qq = tget(S, q1, q2);
        const float2 eq_p = make_float2(r1.er * A_qp.x - r1.ei * A_qp.y, r1.er * A_qp.y + r1.ei * A_qp.x);
        const float2 eq_q = make_float2(r1.er * A_qq.x - r1.ei * A_qq.y, r1.er * A_qq.y + r1.ei * A_qq.x);
        const float2 M_pp = make_float2(r1.cs * A_pp.x - r1.sn * eq_p.x, r1.cs * A_pp.y - r1.sn * eq_p.y);
        const float2 M_pq = make_float2(r1.cs * A_pq.x - r1.sn * eq_q.x, r1.cs * A_pq.y - r1.sn * eq_q.y);
        const float2 M_qp = make_float2(r1.sn * A_pp.x + r1.cs * eq_p.x, r1.sn * A_pp.y + r1.cs * eq_p.y);
        const float2 M_qq = make_float2(r1.sn * A_pq.x + r1.cs * eq_q.x, r1.sn * A_pq.y + r1.cs * eq_q.y);
        const float2 cq_p = make_float2(r2.er * M_pq.x + r2.ei * M_pq.y, r2.er * M_pq.y - r2.ei * M_pq.x);
        const float2 cq_q = make_float2(r2.er * M_qq.x + r2.ei * M_qq.y, r2.er * M_qq.y - r2.ei * M_qq.x);
        const float2 o_pp = make_float2(r2.cs * M_pp.x - r2.sn * cq_p.x, r2.cs * M_pp.y - r2.sn * cq_p.y);
        const float2 o_qp = make_float2(r2.cs * M_qp.x - r2.sn * cq_q.x, r2.cs * M_qp.y - r2.sn * cq_q.y);
        const float2 o_pq = make_float2(r2.sn * M_pp.x + r2.cs * cq_p.x, r2.sn * M_pp.y + r2.cs * cq_p.y);
        const float2 o_qq = make_float2(r2.sn * M_qp.x + r2.cs * cq_q.x, r2.sn * M_qp.y + r2.cs * cq_q.y);
        if (I == Jb) {
          S[tri(p1, p1)] = make_float2(o_pp.x, 0.f);
          S[tri(q1, q1)] = make_float2(o_qq.x, 0.f);
          S[tri(q1, p1)] = make_float2(0.5f * (o_qp.x + o_pq.x), 0.5f * (o_qp.y - o_pq.y));
        } else {
          tput(S, p1, p2, o_pp);
          tput(S, p1, q2, o_pq);
          tput(S, q1, p2, o_qp);
          tput(S, q1, q2, o_qq);
        }
      }
      __syncthreads();
    }
    const int any = any_s;
    __syncthreads();
    if (!any) {
      ++sweep;
      break;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = S[tri(i, i)].x;
    w[(size_t)b * n + i] = fabsf(d) < 1e9f ? (double)d + mu : (double)d;
  }
  if (threadIdx.x == 0) sweeps[b] = sweep;
}

// replay the rotation log on rows [r0, r0 + RB) of the identity; Z[b] gets the eigenvectors
// in the column order of the log (unsorted), FP64.  grid (row blocks, nprob)
constexpr int JV_ROWS = 8;
__global__ void __launch_bounds__(256) k_jac32_vectors(const Rot32* log, int n, int maxsweep, const int* sweeps,
                                                       double2* Z) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* V = reinterpret_cast<float2*>(smem_raw);   // [JV_ROWS][n]
  const int b = blockIdx.y, r0 = blockIdx.x * JV_ROWS;
  const int h = n / 2;
  const int nr = min(JV_ROWS, n - r0);
  for (int t = threadIdx.x; t < JV_ROWS * n; t += blockDim.x) {
    const int rr = t / n, c = t - rr * n;
    V[t] = make_float2((r0 + rr) == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  const int ns = sweeps[b];
  for (int sw = 0; sw < ns; ++sw)
    for (int step = 0; step < n - 1; ++step) {
      const Rot32* rs = log + (((size_t)b * maxsweep + sw) * (n - 1) + step) * h;
      for (int t = threadIdx.x; t < nr * h; t += blockDim.x) {
        const int rr = t / h, I = t - rr * h;
        const Rot32 r = rs[I];
        if (r.sn == 0.f) continue;
        int p = rr_index(I, step, n), q = rr_index(n - 1 - I, step, n);
        if (p > q) { const int tt = p; p = q; q = tt; }
        float2* v = V + rr * n;
        const float2 vp = v[p], vq = v[q];
        const float2 cv = make_float2(r.er * vq.x + r.ei * vq.y, r.er * vq.y - r.ei * vq.x);
        v[p] = make_float2(r.cs * vp.x - r.sn * cv.x, r.cs * vp.y - r.sn * cv.y);
        v[q] = make_float2(r.sn * vp.x + r.cs * cv.x, r.sn * vp.y + r.cs * cv.y);
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < nr * n; t += blockDim.x) {
    const int rr = t / n, c = t - rr * n;
    Z[(size_t)b * n * n + (r0 + rr) + (size_t)c * n] = make_double2(V[t].x, V[t].y);
  }
}

// sort eigenvalues ascending and permute the eigenvector columns; grid nprob
__global__ void k_sort_pairs(const double* w_in, const double2* Zin, int n, double* w_out, double2* Zout) {
  griddep_entry();
  const int b = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = w_in[(size_t)b * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = w_in[(size_t)b * n + j];
      rank += (dj < di) || (dj == di && j < i);
    }
    w_out[(size_t)b * n + rank] = di;
    for (int r = 0; r < n; ++r) Zout[(size_t)b * n * n + r + (size_t)rank * n] = Zin[(size_t)b * n * n + r + (size_t)i * n];
  }
}

size_t jac32_smem(int n) {
  return (((size_t)n * (n + 1) / 2 * sizeof(float2) + 15) & ~size_t(15)) + (size_t)(n / 2) * sizeof(Rot32);
}

// FP32 eigen-decomposition of nprob Hermitian n x n FP64 matrices (A read only): w ascending,
// Z eigenvector columns (FP64 storage, FP32 accuracy).  scratch: log and unsorted copies.
cudaError_t dense_heev32(cudaStream_t st, const double2* A, int n, int nprob, double* w, double2* Z,
                         void* scratch, size_t scratch_bytes, int maxsweep) {
  const size_t smem = jac32_smem(n);
  if (smem > 226 * 1024 || (n & 1)) return cudaErrorInvalidValue;
  const size_t logb = (size_t)nprob * maxsweep * (n - 1) * (n / 2) * sizeof(Rot32);
  const size_t need = logb + (size_t)nprob * (n * 2 + 8) * sizeof(double) + (size_t)nprob * n * n * sizeof(double2) + 1024;
  if (need > scratch_bytes) return cudaErrorInvalidValue;
  unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
  Rot32* log = reinterpret_cast<Rot32*>(p);
  p += (logb + 255) & ~size_t(255);
  double* wu = reinterpret_cast<double*>(p);
  p += (((size_t)nprob * n * sizeof(double)) + 255) & ~size_t(255);
  double* shift = reinterpret_cast<double*>(p);
  p += (((size_t)nprob * sizeof(double)) + 255) & ~size_t(255);
  int* sweeps = reinterpret_cast<int*>(p);
  p += (((size_t)nprob * sizeof(int)) + 255) & ~size_t(255);
  double2* Zu = reinterpret_cast<double2*>(p);
  cudaFuncSetAttribute(k_jac32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  launch_dep(st, k_jac32, nprob, J32_THREADS, smem, A, n, maxsweep, shift, log, wu, sweeps);
  launch_dep(st, k_jac32_vectors, dim3((n + JV_ROWS - 1) / JV_ROWS, nprob), 256, JV_ROWS * n * sizeof(float2), 
      log, n, maxsweep, sweeps, Zu);
  launch_dep(st, k_sort_pairs, nprob, 256, 0, wu, Zu, n, w, Z);
  return cudaGetLastError();
}

size_t heev32_scratch_bytes(int n, int nprob, int maxsweep) {
  return (size_t)nprob * maxsweep * (n - 1) * (n / 2) * sizeof(Rot32) + (size_t)nprob * (n * 2 + 8) * sizeof(double) +
         (size_t)nprob * n * n * sizeof(double2) + 4096;
}

}  // namespace hw

// ===================================================================== Householder eigensolver
// For the Rayleigh-Ritz step only the lowest `nw` eigenpairs are needed.  Stages:
//   k_hh_tridiag  one CTA per problem: the matrix (shifted by the mean of its valid diagonal)
//                 packed as a lower triangle in shared memory, reduced to Hermitian tridiagonal
//                 form by n-2 Householder reflections in FP32; reflectors kept in global memory
//   k_tri_eig     one warp per wanted pair: the tridiagonal made real by a diagonal phase
//                 matrix, its j-th eigenvalue by Sturm multisection and the vector by inverse
//                 iteration (FP32)
//   k_tri_gs      one CTA per problem: Gram-Schmidt inside near-degenerate groups, phases
//   k_hh_back     one warp per wanted vector: Z = Q D Y (reflectors applied in reverse) in FP32
//                 registers, FP64 out
// followed (host side) by an FP64 refinement of the wanted vectors (Ogita-Aishima style
// first-order correction against all FP32 vectors, then Rayleigh-Ritz inside groups).
namespace hw {

struct HhArgs {
  int n, nw;
  const double2* A;    // [nprob][n*n] FP64 input (read only)
  float2* vq;          // [nprob][n][n] reflector k stored in column k (compacted rows k+1..nv-1)
  float* beta;         // [nprob][n]
  float* d;            // [nprob][n] diagonal of T (first nv entries)
  float2* e;           // [nprob][n] sub-diagonal of T (e[k] = T[k+1][k])
  float2* ph;          // [nprob][n] phases D with T = D Tr D^H, Tr real
  int* map;            // [nprob][n] compacted index -> original index (valid first, then padding)
  int* nv;             // [nprob] number of valid indices
  double* shift;       // [nprob]
  float* lam;          // [nprob][nw] eigenvalues of the shifted T (ascending)
  double* lam64;       // [nprob][n stride] the same plus the shift (FP64 storage), may be null
  float* Y;            // [nprob][nw][n] eigenvectors of Tr (compacted coordinates)
  float* work;         // [nprob][nw][2n] inverse-iteration factors
  double2* Z;          // output vectors, problem b at Z + b * zstride (column-major n x nw), original
  int64_t zstride;     // coordinates
};

constexpr int HH_THREADS = 512;   // measured: 1024 and 256 threads 8-10% slower on n = 72 ... 216

// block-wide sum, returned to every thread (warp shuffles, one partial per warp in red)
__device__ __forceinline__ float block_sum_f(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// Padding rows (diagonal >= 1e9, zero off the diagonal) are decoupled: they are moved out of
// the reduction (compacted index map) and come back as exact unit eigenvectors.
__global__ void __launch_bounds__(HH_THREADS) k_hh_tridiag(HhArgs H) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = H.n, b = blockIdx.x;
  float2* S = reinterpret_cast<float2*>(smem_raw);                       // packed lower triangle
  float2* v = S + ((size_t)n * (n + 1) / 2 + 1);                          // [n]
  float2* p = v + n;                                                      // [n]
  int* mp = reinterpret_cast<int*>(p + n);                                // [n]
  __shared__ float red[32];
  __shared__ int nv_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const double2* a = H.A + (size_t)b * n * n;
  // the diagonal into shared memory by all threads (in the v buffer, free until the first
  // reflection), then thread 0 builds the index map from it: no serial global loads
  double* dg = reinterpret_cast<double*>(v);
  for (int i = threadIdx.x; i < n; i += blockDim.x) dg[i] = a[i + (size_t)i * n].x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int c = 0;
    for (int i = 0; i < n; ++i)
      if (fabs(dg[i]) < 1e9) mp[c++] = i;
    const int nvalid = c;
    for (int i = 0; i < n; ++i) {   // padding after, ascending by diagonal value
      const double x = dg[i];
      if (fabs(x) < 1e9) continue;
      int q = c++;
      while (q > nvalid && dg[mp[q - 1]] > x) {
        mp[q] = mp[q - 1];
        --q;
      }
      mp[q] = i;
    }
    nv_s = nvalid;
    H.nv[b] = nvalid;
  }
  __syncthreads();
  const int nv = nv_s;
  for (int i = threadIdx.x; i < n; i += blockDim.x) H.map[(size_t)b * n + i] = mp[i];
  // shift = mean of the valid diagonal
  float sd = 0.f;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) sd += (float)dg[mp[i]];
  sd = block_sum_f(sd, red);
  const double mu = nv > 0 ? (double)(sd / (float)nv) : 0.0;
  // load the valid lower triangle, FP64 -> FP32, shifted: row i of the lower triangle is the
  // conjugate of column i above the diagonal (contiguous reads)
  for (int i = warp; i < nv; i += nwarp) {
    const double2* col = a + (size_t)mp[i] * n;
    for (int j = lane; j <= i; j += 32) {
      const double2 x = col[mp[j]];
      S[tri(i, j)] = i == j ? make_float2(d2f(x.x - mu), 0.f) : make_float2(d2f(x.x), -d2f(x.y));
    }
  }
  __syncthreads();
  float2* vq = H.vq + (size_t)b * n * n;
  // Three block barriers per reflection: the squared norm of the next column below the diagonal
  // is summed per warp during the rank-2 update (red_s), v^H p per warp during the product
  // (red_k), and w = p - K v is formed on the fly in the update.
  __shared__ float red_s[32], red_k[32];
  {
    float s0 = 0.f;
    for (int i = threadIdx.x; i < nv - 1; i += blockDim.x) {
      const float2 x = S[tri(1 + i, 0)];
      s0 += x.x * x.x + x.y * x.y;
    }
    for (int o = 16; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    if (lane == 0) red_s[warp] = s0;
  }
  __syncthreads();
  for (int k = 0; k < nv - 2; ++k) {
    const int m = nv - k - 1;   // length of the column below the diagonal
    // the per-warp partials summed by a shuffle tree in every warp (lane w holds warp w's)
    float s = lane < nwarp ? red_s[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    // every thread forms the reflector scalars from the same values (no broadcast barrier)
    float bet;
    float2 alpha;
    {
      const float2 x0 = S[tri(k + 1, k)];
      const float ax0 = sqrtf(x0.x * x0.x + x0.y * x0.y);
      const float tail = s - ax0 * ax0;
      if (!(tail > 1e-30f * fmaxf(s, 1e-30f)) || s == 0.f) {
        bet = 0.f;             // already reduced
        alpha = x0;
      } else {
        const float sq = sqrtf(s);
        const float2 ph = ax0 > 0.f ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.f, 0.f);
        alpha = make_float2(-ph.x * sq, -ph.y * sq);
        bet = 1.0f / (sq * (sq + ax0));   // 2 / ||v||^2
      }
    }
    if (threadIdx.x == 0) {
      H.beta[(size_t)b * n + k] = bet;
      H.e[(size_t)b * n + k] = alpha;
      H.d[(size_t)b * n + k] = S[tri(k, k)].x;
    }
    if (bet == 0.f) {   // (uniform) nothing to reflect; the next column's norm directly
      for (int i = threadIdx.x; i < m; i += blockDim.x) vq[(size_t)k * n + k + 1 + i] = make_float2(0.f, 0.f);
      __syncthreads();   // every thread has read red_s
      float s1 = 0.f;
      for (int i = threadIdx.x; i < m - 1; i += blockDim.x) {
        const float2 x = S[tri(k + 2 + i, k + 1)];
        s1 += x.x * x.x + x.y * x.y;
      }
      for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      if (lane == 0) red_s[warp] = s1;
      __syncthreads();
      continue;
    }
    // v = x - alpha e1
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      float2 x = S[tri(k + 1 + i, k)];
      if (i == 0) { x.x -= alpha.x; x.y -= alpha.y; }
      v[i] = x;
      vq[(size_t)k * n + k + 1 + i] = x;
    }
    __syncthreads();   // B1: v published (and every thread past its reads of red_s)
    // p = beta A' v   (A' = A[k+1:, k+1:]); 4 threads per row, uniform shuffles; v^H p per warp
    float kkp = 0.f;
    for (int t0 = 0; t0 < 4 * m; t0 += blockDim.x) {
      const int t = t0 + threadIdx.x;
      const bool act = t < 4 * m;
      const int i = t >> 2, part = t & 3;
      float pr = 0.f, pi = 0.f;
      if (act) {
        const int r = k + 1 + i;
        // j <= i: row r of the packed lower triangle (contiguous)
        const float2* row = S + tri(r, k + 1);
        int j = part;
        float qr = 0.f, qi = 0.f;   // a second accumulator: two independent chains
#pragma unroll 4
        for (; j + 4 <= i; j += 8) {
          const float2 a0 = row[j], a1 = row[j + 4];
          const float2 v0 = v[j], v1 = v[j + 4];
          pr += a0.x * v0.x - a0.y * v0.y;
          pi += a0.x * v0.y + a0.y * v0.x;
          qr += a1.x * v1.x - a1.y * v1.y;
          qi += a1.x * v1.y + a1.y * v1.x;
        }
        for (; j <= i; j += 4) {
          const float2 aij = row[j];
          const float2 vj = v[j];
          pr += aij.x * vj.x - aij.y * vj.y;
          pi += aij.x * vj.y + aij.y * vj.x;
        }
        // j > i: conj(A[c][r]) with c = k + 1 + j, packed index tri(c, r) advanced incrementally
        int c = k + 1 + j;
        int idx = tri(c, r);
#pragma unroll 4
        for (; j + 4 < m; j += 8) {
          const float2 a0 = S[idx], a1 = S[idx + 4 * c + 10];
          const float2 v0 = v[j], v1 = v[j + 4];
          pr += a0.x * v0.x + a0.y * v0.y;
          pi += a0.x * v0.y - a0.y * v0.x;
          qr += a1.x * v1.x + a1.y * v1.y;
          qi += a1.x * v1.y - a1.y * v1.x;
          idx += 8 * c + 36;   // tri(c + 8, r) - tri(c, r)
          c += 8;
        }
        for (; j < m; j += 4) {
          const float2 a = S[idx];
          const float2 vj = v[j];
          pr += a.x * vj.x + a.y * vj.y;
          pi += a.x * vj.y - a.y * vj.x;
          idx += 4 * c + 10;
          c += 4;
        }
        pr += qr;
        pi += qi;
      }
      pr += __shfl_xor_sync(0xffffffffu, pr, 1);
      pi += __shfl_xor_sync(0xffffffffu, pi, 1);
      pr += __shfl_xor_sync(0xffffffffu, pr, 2);
      pi += __shfl_xor_sync(0xffffffffu, pi, 2);
      if (act && part == 0) {
        const float2 pv = make_float2(bet * pr, bet * pi);
        p[i] = pv;
        kkp += v[i].x * pv.x + v[i].y * pv.y;
      }
    }
    for (int o = 16; o > 0; o >>= 1) kkp += __shfl_xor_sync(0xffffffffu, kkp, o);
    if (lane == 0) red_k[warp] = kkp;
    __syncthreads();   // B2: p and the v^H p partials published
    // K = (beta / 2) v^H p (real for Hermitian A'); A' -= v w^H + w v^H, w = p - K v, on the
    // lower triangle, one warp per row; lane 0 (column k + 1) sums the next column's norm
    float kk = lane < nwarp ? red_k[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
    kk *= 0.5f * bet;
    float s1 = 0.f;
    for (int i = warp; i < m; i += nwarp) {
      const float2 vi = v[i], pi2 = p[i];
      const float2 wi = make_float2(pi2.x - kk * vi.x, pi2.y - kk * vi.y);
      float2* row = S + tri(k + 1 + i, k + 1);
      for (int j = lane; j <= i; j += 32) {
        const float2 vj = v[j], pj = p[j];
        const float2 wj = make_float2(pj.x - kk * vj.x, pj.y - kk * vj.y);
        float2 x = row[j];
        x.x -= (vi.x * wj.x + vi.y * wj.y) + (wi.x * vj.x + wi.y * vj.y);
        x.y -= (vi.y * wj.x - vi.x * wj.y) + (wi.y * vj.x - wi.x * vj.y);
        if (i == j) x.y = 0.f;
        row[j] = x;
        if (j == 0 && i >= 1) s1 += x.x * x.x + x.y * x.y;
      }
    }
    if (lane == 0) red_s[warp] = s1;   // only lane 0 ever sees column k + 1 (j = 0)
    __syncthreads();   // B3: the trailing matrix and the next norm partials published
  }
  if (threadIdx.x == 0) {
    if (nv >= 2) {
      H.d[(size_t)b * n + nv - 2] = S[tri(nv - 2, nv - 2)].x;
      H.d[(size_t)b * n + nv - 1] = S[tri(nv - 1, nv - 1)].x;
      H.e[(size_t)b * n + nv - 2] = S[tri(nv - 1, nv - 2)];
      H.beta[(size_t)b * n + nv - 2] = 0.f;
      H.beta[(size_t)b * n + nv - 1] = 0.f;
    } else if (nv == 1) {
      H.d[(size_t)b * n] = S[0].x;
      H.beta[(size_t)b * n] = 0.f;
    }
    H.shift[b] = mu;
  }
}

// deterministic pseudo-random value in [-1, 1] for (problem, vector, entry, attempt)
__device__ __forceinline__ float hash_unit(int b, int j, int i, int a) {
  unsigned int x = (unsigned int)(b * 73856093) ^ (unsigned int)(j * 19349663) ^ (unsigned int)(i * 83492791) ^
                   (unsigned int)(a * 2654435761u);
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return (float)(x & 0xFFFFFF) * (2.0f / 16777215.0f) - 1.0f;
}

// eigenvalues count below x of the real tridiagonal (diag dd, off-diagonal magnitudes ee)
__device__ __forceinline__ int sturm32(const float* dd, const float* ee2, int n, float x, float pivmin) {
  int c = 0;
  float q = dd[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  if (q < 0.f) ++c;
  for (int i = 1; i < n; ++i) {
    q = dd[i] - x - __fdividef(ee2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++c;
  }
  return c;
}

// spectrum scale of the valid tridiagonal (Gershgorin), shared by the eigenvalue and the
// grouping kernels
__device__ __forceinline__ void tri_bounds(const float* dd, const float* ee, int nv, float& lo, float& hi) {
  lo = 1e30f;
  hi = -1e30f;
  for (int i = 0; i < nv; ++i) {
    const float r = (i > 0 ? ee[i - 1] : 0.f) + (i < nv - 1 ? ee[i] : 0.f);
    lo = fminf(lo, dd[i] - r);
    hi = fmaxf(hi, dd[i] + r);
  }
  if (nv == 0) lo = hi = 0.f;
}

constexpr int TRI_WARPS = 8;

// eigenvalue j by Sturm multisection (the 32 lanes of warp j test 32 interior points of the
// bracket, which shrinks 33-fold per round) and its vector by inverse iteration (lane 0 runs
// the recurrences with reciprocal pivots, the warp normalises); grid (ceil(nw / 8), nprob).
// Padding pairs (j >= nv) take their diagonal value.
__global__ void __launch_bounds__(32 * TRI_WARPS) k_tri_eig(HhArgs H) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = H.n, nw = H.nw, b = blockIdx.y;
  const int nv = H.nv[b];
  float* dd = reinterpret_cast<float*>(smem_raw);   // [n]
  float* ee = dd + n;                               // [n] |e|
  float* ee2 = ee + n;                              // [n] |e|^2
  __shared__ float bnd[2];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    dd[i] = H.d[(size_t)b * n + i];
    const float2 e = i < nv - 1 ? H.e[(size_t)b * n + i] : make_float2(0.f, 0.f);
    ee[i] = sqrtf(e.x * e.x + e.y * e.y);
    ee2[i] = e.x * e.x + e.y * e.y;
  }
  __syncthreads();
  if (threadIdx.x == 0) tri_bounds(dd, ee, nv, bnd[0], bnd[1]);
  __syncthreads();
  const float lo = bnd[0], hi = bnd[1];
  const float scale = fmaxf(fmaxf(fabsf(lo), fabsf(hi)), 1e-6f);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * TRI_WARPS + warp;
  if (j >= nw) return;
  if (j >= nv) {
    if (lane == 0) {
      const int src = H.map[(size_t)b * n + j];
      const double x = H.A[(size_t)b * n * n + src + (size_t)src * n].x;
      H.lam[(size_t)b * nw + j] = (float)(x - H.shift[b]);
      if (H.lam64) H.lam64[(size_t)b * n + j] = x;
    }
    return;
  }
  float a0 = lo, b0 = hi;
  for (int round = 0; round < 12 && b0 - a0 > 2e-7f * scale; ++round) {
    const float h = (b0 - a0) * (1.0f / 33.0f);
    const int cnt = sturm32(dd, ee2, nv, a0 + h * (float)(lane + 1), 1e-30f);
    const unsigned above = __ballot_sync(0xffffffffu, cnt > j);
    const int first = above ? __ffs(above) - 1 : 32;   // first test point with more than j below it
    const float na = first > 0 ? a0 + h * (float)first : a0;
    const float nb = first < 32 ? a0 + h * (float)(first + 1) : b0;
    a0 = na;
    b0 = nb;
  }
  const float lamj = 0.5f * (a0 + b0);
  // the warp's vector, reciprocal pivots and multipliers in shared memory (the factorisation
  // and the two solves below are serial recurrences on lane 0)
  float* __restrict__ y = ee2 + n + (size_t)warp * 3 * n;
  float* __restrict__ ru = y + n;   // reciprocal pivots
  float* __restrict__ l = ru + n;   // multipliers
  for (int i = lane; i < nv; i += 32) y[i] = hash_unit(b, j, i, 0);
  if (lane == 0) {
    H.lam[(size_t)b * nw + j] = lamj;
    if (H.lam64) H.lam64[(size_t)b * n + j] = (double)lamj + H.shift[b];
  }
  __syncwarp();
  const float guard = 1e-7f * scale;
  // perturb the shift slightly so equal eigenvalues give different vectors
  const float sh = lamj + (float)(j % 7) * 1e-7f * scale;
  if (lane == 0) {
    float up = dd[0] - sh;
    if (fabsf(up) < guard) up = guard;
    ru[0] = 1.0f / up;
    for (int i = 1; i < nv; ++i) {
      const float li = ee[i - 1] * ru[i - 1];
      l[i] = li;
      up = dd[i] - sh - li * ee[i - 1];
      if (fabsf(up) < guard) up = copysignf(guard, up == 0.f ? 1.f : up);
      ru[i] = 1.0f / up;
    }
  }
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    if (lane == 0) {
      float prev = y[0];
      for (int i = 1; i < nv; ++i) {
        prev = y[i] - l[i] * prev;
        y[i] = prev;
      }
      float nxt = y[nv - 1] * ru[nv - 1];
      y[nv - 1] = nxt;
      for (int i = nv - 2; i >= 0; --i) {
        nxt = (y[i] - ee[i] * nxt) * ru[i];
        y[i] = nxt;
      }
    }
    __syncwarp();
    float s = 0.f;
    for (int i = lane; i < nv; i += 32) s += y[i] * y[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    s = rsqrtf(fmaxf(s, 1e-30f));
    for (int i = lane; i < nv; i += 32) y[i] *= s;
    __syncwarp();
  }
  float* yg = H.Y + ((size_t)b * nw + j) * n;
  for (int i = lane; i < nv; i += 32) yg[i] = y[i];
}

// Gram-Schmidt inside groups of near-equal eigenvalues (gap < 1e-4 * scale, at most 32), one
// thread per group start; thread 0 first writes the phase chain d_0 = 1, d_{k+1} = d_k e_k/|e_k|.
// grid nprob
__global__ void __launch_bounds__(256) k_tri_gs(HhArgs H) {
  griddep_entry();
  const int n = H.n, nw = H.nw, b = blockIdx.x;
  const int nv = H.nv[b];
  const float* lam = H.lam + (size_t)b * nw;
  // |e_k| and the unit phases e_k / |e_k| into shared memory by all threads (the chain below and
  // the spectrum scale then read no global memory serially)
  extern __shared__ float tgs[];   // [n] |e| then [2n] unit phases
  float* ae_s = tgs;
  float2* u_s = reinterpret_cast<float2*>(tgs + ((n + 1) & ~1));
  for (int i = threadIdx.x; i < nv - 1; i += blockDim.x) {
    const float2 ek = H.e[(size_t)b * n + i];
    const float ae = sqrtf(ek.x * ek.x + ek.y * ek.y);
    ae_s[i] = ae;
    u_s[i] = ae > 0.f ? make_float2(ek.x / ae, ek.y / ae) : make_float2(1.f, 0.f);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float2 ph = make_float2(1.f, 0.f);
    float2* out = H.ph + (size_t)b * n;
    for (int i = 0; i < nv; ++i) {
      out[i] = ph;
      if (i < nv - 1) {
        const float2 u = u_s[i];
        ph = make_float2(ph.x * u.x - ph.y * u.y, ph.x * u.y + ph.y * u.x);
      }
    }
  }
  // scale of the valid spectrum
  float scale = 0.f;
  const int nvw = nv < nw ? nv : nw;
  for (int i = 0; i < nvw; ++i) scale = fmaxf(scale, fabsf(lam[i]));
  for (int i = 0; i < nv - 1; ++i) scale = fmaxf(scale, ae_s[i]);
  scale = fmaxf(scale, 1e-6f);
  for (int j = threadIdx.x; j < nvw; j += blockDim.x) {
    if (j > 0 && lam[j] - lam[j - 1] < 1e-4f * scale) continue;   // not a group start
    int end = j + 1;
    while (end < nvw && lam[end] - lam[end - 1] < 1e-4f * scale && end - j < 32) ++end;
    for (int c = j + 1; c < end; ++c) {
      float* yc = H.Y + ((size_t)b * nw + c) * n;
      // if the group's earlier vectors absorb almost all of this one (exactly degenerate,
      // decoupled eigenvalues give parallel inverse-iteration vectors), restart from a fresh
      // random vector on the group's support
      for (int attempt = 0; attempt < 4; ++attempt) {
        for (int pass = 0; pass < 2; ++pass)
          for (int q = j; q < c; ++q) {
            const float* yq = H.Y + ((size_t)b * nw + q) * n;
            float dot = 0.f;
            for (int i = 0; i < nv; ++i) dot += yq[i] * yc[i];
            for (int i = 0; i < nv; ++i) yc[i] -= dot * yq[i];
          }
        float s = 0.f;
        for (int i = 0; i < nv; ++i) s += yc[i] * yc[i];
        if (s > 1e-4f) {
          s = rsqrtf(s);
          for (int i = 0; i < nv; ++i) yc[i] *= s;
          break;
        }
        for (int i = 0; i < nv; ++i) {
          float t = 0.f;
          for (int q = j; q < c; ++q) t += fabsf((H.Y + ((size_t)b * nw + q) * n)[i]);
          yc[i] = hash_unit(b, c, i, attempt + 1) * (t > 0.f ? 1.f : 0.05f);
        }
        float s2 = 0.f;
        for (int i = 0; i < nv; ++i) s2 += yc[i] * yc[i];
        s2 = rsqrtf(fmaxf(s2, 1e-30f));
        for (int i = 0; i < nv; ++i) yc[i] *= s2;
      }
    }
  }
}

constexpr int HB_PER = 8;   // n <= 256 entries per vector, 8 per lane
constexpr int HB_RC = 16;   // reflectors staged in shared memory per round

// Z[:, j] = Q D y_j in FP32 registers, one warp per wanted vector, scattered back to the
// original indices (padding pairs: unit vectors); the CTA stages HB_RC reflectors at a time in
// shared memory (coalesced loads shared by its 8 vectors).  grid (ceil(nw / 8), nprob), 256
// threads, dynamic smem HB_RC * n complex64
__global__ void __launch_bounds__(256) k_hh_back(HhArgs H) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* vs = reinterpret_cast<float2*>(smem_raw);   // [HB_RC][n]
  __shared__ float bs[HB_RC];
  const int n = H.n, nw = H.nw, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + warp;
  const bool has = j < nw;
  const int nv = H.nv[b];
  const int* mp = H.map + (size_t)b * n;
  double2* z = H.Z + (size_t)b * H.zstride + (size_t)(has ? j : 0) * n;
  const bool pad = has && j >= nv;
  if (pad) {
    const int src = mp[j];
    for (int i = lane; i < n; i += 32) z[i] = make_double2(i == src ? 1.0 : 0.0, 0.0);
  }
  const bool work = has && !pad;   // warp-uniform
  float2 zr[HB_PER];
  if (work) {
    const float* y = H.Y + ((size_t)b * nw + j) * n;
    const float2* ph = H.ph + (size_t)b * n;
#pragma unroll
    for (int c = 0; c < HB_PER; ++c) {
      const int i = lane + 32 * c;
      if (i < nv) {
        const float yi = y[i];
        const float2 d = ph[i];
        zr[c] = make_float2(d.x * yi, d.y * yi);
      } else {
        zr[c] = make_float2(0.f, 0.f);
      }
    }
  }
  const float2* vq = H.vq + (size_t)b * n * n;
  const float* beta = H.beta + (size_t)b * n;
  for (int khi = nv - 3; khi >= 0; khi -= HB_RC) {
    const int klo = max(0, khi - HB_RC + 1);
    const int cnt = khi - klo + 1;
    __syncthreads();   // previous round's readers are done
    for (int t = threadIdx.x; t < cnt * nv; t += blockDim.x) {
      const int r = t / nv, i = t - r * nv;
      const int k = khi - r;
      vs[(size_t)r * n + i] = i > k ? vq[(size_t)k * n + i] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x < cnt) bs[threadIdx.x] = beta[khi - threadIdx.x];
    __syncthreads();
    if (!work) continue;
    for (int r = 0; r < cnt; ++r) {
      const float bet = bs[r];
      if (bet == 0.f) continue;
      const float2* v = vs + (size_t)r * n;
      float sr = 0.f, si = 0.f;   // s = v^H z
#pragma unroll
      for (int c = 0; c < HB_PER; ++c) {
        const int i = lane + 32 * c;
        if (i < nv) {
          const float2 vi = v[i];
          sr += vi.x * zr[c].x + vi.y * zr[c].y;
          si += vi.x * zr[c].y - vi.y * zr[c].x;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      sr *= bet;
      si *= bet;
#pragma unroll
      for (int c = 0; c < HB_PER; ++c) {
        const int i = lane + 32 * c;
        if (i < nv) {
          const float2 vi = v[i];
          zr[c].x -= vi.x * sr - vi.y * si;
          zr[c].y -= vi.x * si + vi.y * sr;
        }
      }
    }
  }
  if (!work) return;
#pragma unroll
  for (int c = 0; c < HB_PER; ++c) {
    const int i = lane + 32 * c;
    if (i < nv) z[mp[i]] = f2d(zr[c]);
  }
  for (int t = nv + lane; t < n; t += 32) z[mp[t]] = make_double2(0.0, 0.0);
}

size_t hh_smem(int n) {
  return ((size_t)n * (n + 1) / 2 + 1 + 2 * (size_t)n) * sizeof(float2) + (size_t)n * sizeof(int);
}

size_t hh_scratch_bytes(int n, int nw, int nprob) {
  const size_t per = (size_t)n * n * sizeof(float2) + 2 * n * sizeof(float) + 2 * n * sizeof(float2) +
                     n * sizeof(int) + sizeof(int) + sizeof(double) + nw * sizeof(float) +
                     (size_t)nw * n * sizeof(float) * 3;
  return (size_t)nprob * per + 16 * 256 + 4096;
}

// FP32 stage: Z (FP64 storage, problem b at Z + b * zstride, n x nw) holds approximate
// eigenvectors of the lowest nw eigenvalues of each A (read only), lam64 their eigenvalues
// (shift added back, stride n).  stage: 1 the reduction only, 2 the rest (same scratch), 3 both.
cudaError_t dense_heev_hh32(cudaStream_t st, const double2* A, int n, int nw, int nprob, double2* Z,
                            int64_t zstride, void* scratch, size_t scratch_bytes, double* lam64, int stage) {
  if (n > 32 * HB_PER || hh_smem(n) > 226 * 1024 || nw > n || nw < 1) return cudaErrorInvalidValue;
  if (hh_scratch_bytes(n, nw, nprob) > scratch_bytes) return cudaErrorInvalidValue;
  unsigned char* p = reinterpret_cast<unsigned char*>(scratch);
  auto take = [&](size_t bytes) {
    void* r = p;
    p += (bytes + 255) & ~size_t(255);
    return r;
  };
  HhArgs H;
  H.n = n;
  H.nw = nw;
  H.A = A;
  H.vq = (float2*)take((size_t)nprob * n * n * sizeof(float2));
  H.beta = (float*)take((size_t)nprob * n * sizeof(float));
  H.d = (float*)take((size_t)nprob * n * sizeof(float));
  H.e = (float2*)take((size_t)nprob * n * sizeof(float2));
  H.ph = (float2*)take((size_t)nprob * n * sizeof(float2));
  H.map = (int*)take((size_t)nprob * n * sizeof(int));
  H.nv = (int*)take((size_t)nprob * sizeof(int));
  H.shift = (double*)take((size_t)nprob * sizeof(double));
  H.lam = (float*)take((size_t)nprob * nw * sizeof(float));
  H.Y = (float*)take((size_t)nprob * nw * n * sizeof(float));
  H.work = (float*)take((size_t)nprob * nw * 2 * n * sizeof(float));
  H.Z = Z;
  H.zstride = zstride;
  H.lam64 = lam64;
  if (stage & 1) {
    cudaFuncSetAttribute(k_hh_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hh_smem(n));
    launch_dep(st, k_hh_tridiag, nprob, HH_THREADS, hh_smem(n), H);
  }
  if (!(stage & 2)) return cudaGetLastError();
  launch_dep(st, k_tri_eig, dim3((nw + TRI_WARPS - 1) / TRI_WARPS, nprob), 32 * TRI_WARPS, (3 + 3 * TRI_WARPS) * n * sizeof(float), H);
  launch_dep(st, k_tri_gs, nprob, 256, (size_t)(((n + 1) & ~1) + 2 * n) * sizeof(float), H);
  launch_dep(st, k_hh_back, dim3((nw + 7) / 8, nprob), 256, (size_t)HB_RC * n * sizeof(float2), H);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- FP64 refinement kernels
// First-order correction of the nw wanted vectors against all n vectors of Z:
// R = Z^H Z_w (n x nw), S = Z^H A Z_w (n x nw), lamall [n] estimates of every eigenvalue.
// E (n x nw): E_jj = (1 - R_jj)/2; E_ij = (S_ij - lam_j R_ij)/(lam_j - lam_i) (i != j) when that
// is below 0.1 in size, else the orthogonality fix -R_ij/2 (near-degenerate pair).  Adds the
// identity in rows < nw so that Z_w <- Z E is one GEMM.  grid (blocks, nprob)
__global__ void k_oa_correction(const double2* R, const double2* S, int n, int nw, const double* lamall, double2* E) {
  griddep_entry();
  const int b = blockIdx.y;
  const double2* r = R + (size_t)b * n * nw;
  const double2* s = S + (size_t)b * n * nw;
  double2* e = E + (size_t)b * n * nw;
  const double* la = lamall + (size_t)b * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * nw; t += gridDim.x * blockDim.x) {
    const int i = t % n, j = t / n;
    const double2 rij = r[t];
    const double lj = s[j + (size_t)j * n].x / r[j + (size_t)j * n].x;
    if (i == j) {
      e[t] = make_double2(1.0 + 0.5 * (1.0 - rij.x), 0.0);
      continue;
    }
    const double2 sij = s[t];
    const double li = i < nw ? s[i + (size_t)i * n].x / r[i + (size_t)i * n].x : la[i];
    const double num_r = sij.x - lj * rij.x, num_i = sij.y - lj * rij.y;
    double mag = sqrt(num_r * num_r + num_i * num_i);
    if (i < nw) {   // the decision must be the same for (i, j) and (j, i)
      const double2 sji = s[j + (size_t)i * n], rji = r[j + (size_t)i * n];
      const double mr = sji.x - li * rji.x, mi = sji.y - li * rji.y;
      mag = fmax(mag, sqrt(mr * mr + mi * mi));
    }
    const double den = lj - li;
    const double tau = 1e-8 * (1.0 + fmax(fabs(li), fabs(lj)));
    if (fabs(den) > tau && fabs(den) > 10.0 * mag) e[t] = make_double2(num_r / den, num_i / den);
    else e[t] = make_double2(-0.5 * rij.x, -0.5 * rij.y);
  }
}

// Final Rayleigh-Ritz of the wanted block from S_w = Z_w^H A Z_w (nw x nw, Z_w orthonormal):
// consecutive vectors whose coupling is not small against their gap (> 1e-7 of it) or whose
// gap is below 1e-8 (1 + |lambda|) form a group, diagonalised exactly by a serial FP64 Jacobi
// (one thread per group, groups of up to 16); couplings between groups get the first-order
// rotation S_ij / (lambda_j - lambda_i), unitary to O(1e-14).

// grp[j] = 1 joins j and j+1: some vector at or before j couples strongly to one after j
// (pairs at most 15 apart).  The strong-link bits of all such pairs are formed first, from
// the diagonal in shared memory.  grid nprob, dynamic smem nw doubles + nw 16-bit masks
__global__ void k_group_links(const double2* S, int nw, int* grp) {
  griddep_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* dg = reinterpret_cast<double*>(smem_raw);
  unsigned short* lk = reinterpret_cast<unsigned short*>(dg + nw);   // bit d-1: a links to a+d
  const int b = blockIdx.x;
  const double2* s = S + (size_t)b * nw * nw;
  for (int j = threadIdx.x; j < nw; j += blockDim.x) {
    dg[j] = s[j + (size_t)j * nw].x;
    lk[j] = 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nw * 15; t += blockDim.x) {
    const int a = t / 15, d = t % 15 + 1, k = a + d;
    if (k >= nw) continue;
    const double dj = dg[a], dk = dg[k];
    const double2 c = s[a + (size_t)k * nw];
    const double gap = fabs(dk - dj);
    if (gap < 1e-8 * (1.0 + fabs(dj) + fabs(dk)) || sqrt(c.x * c.x + c.y * c.y) > 1e-7 * gap)
      atomicOr(reinterpret_cast<unsigned int*>(lk + (a & ~1)), 1u << (d - 1 + 16 * (a & 1)));
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nw; j += blockDim.x) {
    int link = 0;
    for (int a = max(0, j - 14); a <= j && !link; ++a) {
      // a links to some k with j < k <= a + 15
      const unsigned int bits = lk[a];
      const int dmin = j + 1 - a;   // k = a + d > j
      link = (bits >> (dmin - 1)) != 0;
    }
    grp[(size_t)b * nw + j] = link;
  }
}

// Rayleigh-Ritz inside groups of consecutive vectors flagged by k_oa_correction: S (nw x nw,
// FP64) restricted to a group is diagonalised by a serial cyclic Jacobi (one thread per group);
// the group's rotation U is written into E (identity elsewhere) and the eigenvalues into lam.
__global__ void k_group_rr(const double2* S, int nw, const int* grp, double* lam, int lstride, double2* U) {
  griddep_entry();
  const int b = blockIdx.x;
  const double2* s = S + (size_t)b * nw * nw;
  double2* u = U + (size_t)b * nw * nw;
  double* l = lam + (size_t)b * lstride;
  const int* g = grp + (size_t)b * nw;
  // identity (the group rotations overwrite their blocks)
  for (int t = threadIdx.x; t < nw * nw; t += blockDim.x) {
    const int i = t % nw, j = t / nw;
    u[t] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int j0 = threadIdx.x; j0 < nw; j0 += blockDim.x) {
    if (j0 > 0 && g[j0 - 1]) continue;          // not a group start
    int end = j0 + 1;                            // group = [j0, end)
    while (end < nw && g[end - 1]) ++end;
    const int m = end - j0;
    if (m == 1) {
      l[j0] = s[j0 + (size_t)j0 * nw].x;
      continue;
    }
    if (m > 16) {   // larger groups keep the first-order result
      for (int c = 0; c < m; ++c) l[j0 + c] = s[(j0 + c) + (size_t)(j0 + c) * nw].x;
      continue;
    }
    double2 a[16][16], v[16][16];
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < m; ++k) {
        a[i][k] = s[(j0 + i) + (size_t)(j0 + k) * nw];
        v[i][k] = make_double2(i == k ? 1.0 : 0.0, 0.0);
      }
    for (int sweep = 0; sweep < 30; ++sweep) {
      double off = 0.0;
      for (int p = 0; p < m; ++p)
        for (int q = p + 1; q < m; ++q) off += a[p][q].x * a[p][q].x + a[p][q].y * a[p][q].y;
      if (off < 1e-30) break;
      for (int p = 0; p < m; ++p)
        for (int q = p + 1; q < m; ++q) {
          const double2 c = a[p][q];
          const double ac = hypot(c.x, c.y);
          if (ac < 1e-300) continue;
          const double zeta = (a[q][q].x - a[p][p].x) / (2.0 * ac);
          const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
          const double er = c.x / ac, ei = c.y / ac;
          // rows: p' = cs a_p - sn e a_q ; q' = sn a_p + cs e a_q  (J^H A)
          for (int k = 0; k < m; ++k) {
            const double2 ap = a[p][k], aq = a[q][k];
            const double2 eq = make_double2(er * aq.x - ei * aq.y, er * aq.y + ei * aq.x);
            a[p][k] = make_double2(cs * ap.x - sn * eq.x, cs * ap.y - sn * eq.y);
            a[q][k] = make_double2(sn * ap.x + cs * eq.x, sn * ap.y + cs * eq.y);
          }
          // cols: p' = cs a_p - sn conj(e) a_q ; q' = sn a_p + cs conj(e) a_q  (A J), same for V
          for (int k = 0; k < m; ++k) {
            const double2 ap = a[k][p], aq = a[k][q];
            const double2 cq = make_double2(er * aq.x + ei * aq.y, er * aq.y - ei * aq.x);
            a[k][p] = make_double2(cs * ap.x - sn * cq.x, cs * ap.y - sn * cq.y);
            a[k][q] = make_double2(sn * ap.x + cs * cq.x, sn * ap.y + cs * cq.y);
            const double2 vp = v[k][p], vq = v[k][q];
            const double2 cv = make_double2(er * vq.x + ei * vq.y, er * vq.y - ei * vq.x);
            v[k][p] = make_double2(cs * vp.x - sn * cv.x, cs * vp.y - sn * cv.y);
            v[k][q] = make_double2(sn * vp.x + cs * cv.x, sn * vp.y + cs * cv.y);
          }
        }
    }
    // sort the group ascending (selection) and write U, lam
    int ord[16];
    for (int i = 0; i < m; ++i) ord[i] = i;
    for (int i = 0; i < m; ++i)
      for (int k = i + 1; k < m; ++k)
        if (a[ord[k]][ord[k]].x < a[ord[i]][ord[i]].x) { const int tt = ord[i]; ord[i] = ord[k]; ord[k] = tt; }
    for (int c = 0; c < m; ++c) {
      l[j0 + c] = a[ord[c]][ord[c]].x;
      for (int i = 0; i < m; ++i) u[(j0 + i) + (size_t)(j0 + c) * nw] = v[i][ord[c]];
    }
  }
}

cudaError_t launch_oa_correction(cudaStream_t st, const double2* R, const double2* S, int n, int nw, int nprob,
                                 const double* lamall, double2* E) {
  launch_dep(st, k_oa_correction, dim3(16, nprob), 256, 0, R, S, n, nw, lamall, E);
  return cudaGetLastError();
}

// F = I + first-order rotation between groups, from S' = V_g^H S_w V_g (already rotated inside
// groups, so only between-group entries remain): F_ij = S'_ij / (lambda_j - lambda_i)
__global__ void k_first_order(const double2* Sp, int nw, const int* grp, double2* F) {
  griddep_entry();
  const int b = blockIdx.x;
  const double2* s = Sp + (size_t)b * nw * nw;
  double2* f = F + (size_t)b * nw * nw;
  const int* g = grp + (size_t)b * nw;
  extern __shared__ int gid[];   // [nw] the group flags, then in place the group starts
  for (int j = threadIdx.x; j < nw; j += blockDim.x) gid[j] = g[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    int cur = 0, prev = 0;
    for (int j = 0; j < nw; ++j) {
      const int flag = gid[j];
      if (j > 0 && !prev) cur = j;
      gid[j] = cur;
      prev = flag;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nw * nw; t += blockDim.x) {
    const int i = t % nw, j = t / nw;
    if (i == j) {
      f[t] = make_double2(1.0, 0.0);
    } else if (gid[i] == gid[j]) {
      f[t] = make_double2(0.0, 0.0);
    } else {
      const double den = s[j + (size_t)j * nw].x - s[i + (size_t)i * nw].x;
      const double2 c = s[t];
      f[t] = den != 0.0 ? make_double2(c.x / den, c.y / den) : make_double2(0.0, 0.0);
    }
  }
}

cudaError_t launch_first_order(cudaStream_t st, const double2* Sp, int nw, int nprob, const int* grp, double2* F) {
  launch_dep(st, k_first_order, nprob, 512, nw * sizeof(int), Sp, nw, grp, F);
  return cudaGetLastError();
}

// order the wanted pairs by eigenvalue: column rank(j) of Uout = column j of U
__global__ void k_sort_wanted(const double* lam_in, int lstride, const double2* U, int nw, double* lam_out,
                              double2* Uout) {
  griddep_entry();
  const int b = blockIdx.x;
  const double* l = lam_in + (size_t)b * lstride;
  for (int j = threadIdx.x; j < nw; j += blockDim.x) {
    const double dj = l[j];
    int rank = 0;
    for (int i = 0; i < nw; ++i) rank += (l[i] < dj) || (l[i] == dj && i < j);
    lam_out[(size_t)b * lstride + rank] = dj;
    for (int r = 0; r < nw; ++r) Uout[(size_t)b * nw * nw + r + (size_t)rank * nw] = U[(size_t)b * nw * nw + r + (size_t)j * nw];
  }
}

// group links and exact group rotations: Ug (identity outside groups), lam (unsorted)
cudaError_t launch_group_rr(cudaStream_t st, const double2* Sw, int nw, int nprob, int* grp, double* lam,
                            int lstride, double2* Ug) {
  launch_dep(st, k_group_links, nprob, 256, nw * sizeof(double) + ((nw + 1) / 2) * 4 + 16, Sw, nw, grp);
  launch_dep(st, k_group_rr, nprob, 64, 0, Sw, nw, grp, lam, lstride, Ug);
  return cudaGetLastError();
}

cudaError_t launch_sort_wanted(cudaStream_t st, const double* lam_in, int lstride, const double2* U, int nw, int nprob,
                               double* lam_out, double2* Uout) {
  launch_dep(st, k_sort_wanted, nprob, 128, 0, lam_in, lstride, U, nw, lam_out, Uout);
  return cudaGetLastError();
}

}  // namespace hw

// ===================================================================== Cholesky-QR apply
// W <- W (L^H)^{-1} for each k-point (skipped where skip[b] != 0): row w of W solves y L^H = w, i.e.
// y_j = (w_j - sum_{i<j} conj(L_ji) y_i) / L_jj, in place.  One warp per row: lane q keeps
// the columns j = q (mod 32) in registers; at step j the owner finishes y_j and broadcasts it,
// and every lane subtracts conj(L_kj) y_j from its columns k > j (right-looking order, same
// arithmetic).  L (m x m, lower, from k_chol) is read through the L1 cache (coalesced along a
// column), the reciprocal diagonal from shared memory.  W: rows x m block with leading
// dimension ld, batch stride sW.
namespace hw {
constexpr int TRSM_THREADS = 128;   // 4 rows per block, one warp per row

template <typename T, int NPER>
__global__ void __launch_bounds__(TRSM_THREADS) k_trsm_lh(const double2* __restrict__ L, int m, double2* W,
                                                          int64_t rows, int64_t ld, int64_t sW, const int* skip) {
  griddep_entry();
  using C = typename Cx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* dinv = reinterpret_cast<T*>(smem_raw);
  const int b = blockIdx.y;
  if (skip && skip[b]) return;   // failed factorisation: W left as it was
  // the factor: complex128 for T = double, complex64 (written by k_chol<float>) for T = float
  const C* l = reinterpret_cast<const C*>(L + (size_t)b * m * m);
  for (int j = threadIdx.x; j < m; j += blockDim.x) dinv[j] = (T)1 / l[j + (size_t)j * m].x;
  __syncthreads();
  const int q = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (TRSM_THREADS / 32) + (threadIdx.x >> 5);
  if (r >= rows) return;   // whole warp (one row per warp)
  double2* w = W + (size_t)b * sW + r;
  // acc[c] holds column q + 32 (cb + c) of the current window; after each group of 32 steps
  // the finished column acc[0] is stored and the window shifts (static register indices only)
  C acc[NPER];
#pragma unroll
  for (int c = 0; c < NPER; ++c) {
    const int j = q + 32 * c;
    acc[c] = ld_c<T>(j < m ? w[(size_t)j * ld] : make_double2(0.0, 0.0));
  }
  const int ncb = (m + 31) / 32;
  for (int cb = 0; cb < ncb; ++cb) {
    const int jend = min(32, m - 32 * cb);
    for (int o = 0; o < jend; ++o) {
      const int j = 32 * cb + o;
      T yx = (T)0, yy = (T)0;
      if (q == o) {
        const T di = dinv[j];
        yx = acc[0].x * di;
        yy = acc[0].y * di;
        acc[0].x = yx;
        acc[0].y = yy;
      }
      yx = __shfl_sync(0xffffffffu, yx, o);
      yy = __shfl_sync(0xffffffffu, yy, o);
      const C* lj = l + (size_t)j * m;
#pragma unroll
      for (int c = 0; c < NPER; ++c) {
        const int k = q + 32 * (cb + c);
        if (k > j && k < m) {
          const C lkj = lj[k];   // L[k][j]; acc -= conj(lkj) y
          acc[c].x -= lkj.x * yx + lkj.y * yy;
          acc[c].y -= lkj.x * yy - lkj.y * yx;
        }
      }
    }
    const int jf = q + 32 * cb;   // finished column of this lane
    if (jf < m) {
      if (sizeof(T) == sizeof(float))
        w[(size_t)jf * ld] = f2d(make_float2((float)acc[0].x, (float)acc[0].y));
      else
        w[(size_t)jf * ld] = make_double2((double)acc[0].x, (double)acc[0].y);
    }
#pragma unroll
    for (int c = 0; c + 1 < NPER; ++c) acc[c] = acc[c + 1];
    acc[NPER - 1].x = acc[NPER - 1].y = (T)0;
  }
}

template <typename T, int NPER>
static cudaError_t trsm_launch(cudaStream_t st, const double2* L, int m, int nprob, double2* W, int64_t rows,
                               int64_t ld, int64_t sW, const int* skip) {
  const int rpb = TRSM_THREADS / 32;
  launch_dep(st, k_trsm_lh<T, NPER>, dim3((unsigned)((rows + rpb - 1) / rpb), nprob), TRSM_THREADS, m * sizeof(T), 
      L, m, W, rows, ld, sW, skip);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t trsm_dispatch(cudaStream_t st, const double2* L, int m, int nprob, double2* W, int64_t rows,
                                 int64_t ld, int64_t sW, const int* skip) {
  const int nper = (m + 31) / 32;
  if (nper <= 1) return trsm_launch<T, 1>(st, L, m, nprob, W, rows, ld, sW, skip);
  if (nper <= 2) return trsm_launch<T, 2>(st, L, m, nprob, W, rows, ld, sW, skip);
  if (nper <= 3) return trsm_launch<T, 3>(st, L, m, nprob, W, rows, ld, sW, skip);
  return trsm_launch<T, 4>(st, L, m, nprob, W, rows, ld, sW, skip);
}

cudaError_t dense_trsm_lh(cudaStream_t st, const double2* L, int m, int nprob, double2* W, int64_t rows, int64_t ld,
                          int64_t sW, bool fp32, const int* skip) {
  if (m > 128) return cudaErrorInvalidValue;
  if (rows <= 0) return cudaSuccess;
  return fp32 ? trsm_dispatch<float>(st, L, m, nprob, W, rows, ld, sW, skip)
              : trsm_dispatch<double>(st, L, m, nprob, W, rows, ld, sW, skip);
}
}  // namespace hw
