// Tall-skinny complex Gram products C = alpha A^H B + beta C of the eigensolver's mixed form
// (Gram matrices of the Rayleigh-Ritz step, projections and Cholesky-QR: A, B are K x m and
// K x n blocks over the basis dimension K, with m, n at most a few hundred).
//
// GB300's FP64 rate is 1/64 of its FP32 rate, so the products are formed in FP32 (inputs
// rounded to nearest FP32 by integer bit operations, not by the FP64 conversion unit) and
// accumulated in FP32 over 32 rows only; every 32-row partial sum is added into an FP64
// accumulator.  Each CTA owns a 32 x 32 output tile and one K-chunk; the FP64 chunk results go
// to a workspace and a second kernel adds the chunks in a fixed order (deterministic).
//
// Error (entries of A^H B): input rounding 2^-24 per factor plus FP32 accumulation over 32
// terms, both random in sign: about 1e-8 of sum_k |a_k||b_k| in the worst observed cases, far
// below FP32 GEMM accumulation over K = 5066 (the reason FP32 products stall near a residual
// of 1e-5).  The FP64 method path does not use this kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "hw_common.cuh"

namespace hw {

namespace {

constexpr int GT = 32;        // output tile (rows and columns)
constexpr int GK = 32;        // rows per FP32 partial sum
constexpr int G_THREADS = 256;

// round-to-nearest double -> float by bit operations (values far from the float range limits;
// zero, tiny values and underflow map to zero)
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long v = u & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long r = ((v >> 28) + 1ull) >> 1;   // exponent | 23-bit mantissa, rounded
  const unsigned long long bias = 896ull << 23;            // (1023 - 127) << 23
  unsigned int bits = r > bias ? (unsigned int)(r - bias) : 0u;
  bits |= (unsigned int)(u >> 32) & 0x80000000u;
  return __uint_as_float(bits);
}

// grid (tiles_m * tiles_n, nchunk, batch); part[b][chunk][j * m + i] (FP64 complex)
__global__ void __launch_bounds__(G_THREADS) k_gram(const double2* __restrict__ A, int64_t lda, int64_t sA,
                                                    const double2* __restrict__ B, int64_t ldb, int64_t sB, int m,
                                                    int n, int K, int kc, double2* __restrict__ part) {
  griddep_entry();
  __shared__ float2 As[GK][GT + 1];
  __shared__ float2 Bs[GK][GT + 1];
  const int tiles_m = (m + GT - 1) / GT;
  const int i0 = (blockIdx.x % tiles_m) * GT, j0 = (blockIdx.x / tiles_m) * GT;
  const int chunk = blockIdx.y, nchunk = gridDim.y, b = blockIdx.z;
  const int kbeg = chunk * kc, kend = min(K, kbeg + kc);
  const double2* a = A + (size_t)b * sA;
  const double2* bb = B + (size_t)b * sB;
  const int t = threadIdx.x;
  const int ti = t & 15, tj = t >> 4;   // 2 x 2 outputs: rows i0 + 2ti + {0,1}, cols j0 + 2tj + {0,1}
  const int lk = t & 31, lc = t >> 5;   // loader: row kk = lk, columns lc + 8 q
  double acc64[2][2][2] = {};
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    const int k = k0 + lk;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lc + 8 * q;
      float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
      if (k < kend) {
        if (i0 + c < m) {
          const double2 x = a[(size_t)(i0 + c) * lda + k];
          va = make_float2(d2f_rn(x.x), d2f_rn(x.y));
        }
        if (j0 + c < n) {
          const double2 y = bb[(size_t)(j0 + c) * ldb + k];
          vb = make_float2(d2f_rn(y.x), d2f_rn(y.y));
        }
      }
      As[lk][c] = va;
      Bs[lk][c] = vb;
    }
    __syncthreads();
    float acc[2][2][2] = {};
#pragma unroll 8
    for (int kk = 0; kk < GK; ++kk) {
      const float2 a0 = As[kk][2 * ti], a1 = As[kk][2 * ti + 1];
      const float2 b0 = Bs[kk][2 * tj], b1 = Bs[kk][2 * tj + 1];
      // conj(a) * b
      acc[0][0][0] += a0.x * b0.x + a0.y * b0.y;
      acc[0][0][1] += a0.x * b0.y - a0.y * b0.x;
      acc[0][1][0] += a0.x * b1.x + a0.y * b1.y;
      acc[0][1][1] += a0.x * b1.y - a0.y * b1.x;
      acc[1][0][0] += a1.x * b0.x + a1.y * b0.y;
      acc[1][0][1] += a1.x * b0.y - a1.y * b0.x;
      acc[1][1][0] += a1.x * b1.x + a1.y * b1.y;
      acc[1][1][1] += a1.x * b1.y - a1.y * b1.x;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        acc64[p][r][0] += (double)acc[p][r][0];
        acc64[p][r][1] += (double)acc[p][r][1];
      }
    __syncthreads();
  }
  double2* out = part + ((size_t)b * nchunk + chunk) * (size_t)m * n;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int i = i0 + 2 * ti + p, j = j0 + 2 * tj + r;
      if (i < m && j < n) out[(size_t)j * m + i] = make_double2(acc64[p][r][0], acc64[p][r][1]);
    }
}

// C[b] = alpha sum_chunks part[b][chunk] + beta C[b]
__global__ void k_gram_reduce(const double2* __restrict__ part, int m, int n, int nchunk, int batch, double alpha,
                              double beta, double2* C, int64_t ldc, int64_t sC) {
  griddep_entry();
  const int64_t per = (int64_t)m * n, tot = per * batch;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / per, q = t - b * per;
    const int64_t j = q / m, i = q - j * m;
    double sx = 0.0, sy = 0.0;
    const double2* p = part + (size_t)b * nchunk * per + q;
    for (int c = 0; c < nchunk; ++c) {
      const double2 v = p[(size_t)c * per];
      sx += v.x;
      sy += v.y;
    }
    double2* cc = C + (size_t)b * sC + (size_t)j * ldc + i;
    double2 r = make_double2(alpha * sx, alpha * sy);
    if (beta != 0.0) {
      const double2 o = *cc;
      r.x += beta * o.x;
      r.y += beta * o.y;
    }
    *cc = r;
  }
}

}  // namespace

// workspace bytes needed by gram_cf for these sizes
size_t gram_work_bytes(int m, int n, int K, int batch) {
  const int tiles = ((m + GT - 1) / GT) * ((n + GT - 1) / GT);
  int nchunk = (2 * 152 + tiles * batch - 1) / (tiles * batch);
  const int maxc = (K + 255) / 256;
  nchunk = nchunk < 1 ? 1 : (nchunk > maxc ? maxc : nchunk);
  return (size_t)batch * nchunk * m * n * sizeof(double2);
}

// C = alpha A^H B + beta C for batch problems; returns cudaErrorInvalidValue when the workspace
// is too small
cudaError_t gram_cf(cudaStream_t st, int m, int n, int K, double alpha, const double2* A, int64_t lda, int64_t sA,
                    const double2* B, int64_t ldb, int64_t sB, double beta, double2* C, int64_t ldc, int64_t sC,
                    int batch, void* work, size_t work_bytes, int* launches) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (gram_work_bytes(m, n, K, batch) > work_bytes) return cudaErrorInvalidValue;
  const int tiles = ((m + GT - 1) / GT) * ((n + GT - 1) / GT);
  int nchunk = (2 * 152 + tiles * batch - 1) / (tiles * batch);
  const int maxc = (K + 255) / 256;
  nchunk = nchunk < 1 ? 1 : (nchunk > maxc ? maxc : nchunk);
  int kc = (K + nchunk - 1) / nchunk;
  kc = (kc + GK - 1) / GK * GK;
  nchunk = (K + kc - 1) / kc;
  if (nchunk < 1) nchunk = 1;
  double2* part = reinterpret_cast<double2*>(work);
  launch_dep(st, k_gram, dim3(tiles, nchunk, batch), G_THREADS, 0, A, lda, sA, B, ldb, sB, m, n, K, kc, part);
  const int64_t tot = (int64_t)m * n * batch;
  const int grid = (int)((tot + 255) / 256 < 152 * 8 ? (tot + 255) / 256 : 152 * 8);
  launch_dep(st, k_gram_reduce, grid, 256, 0, part, m, n, nchunk, batch, alpha, beta, C, ldc, sC);
  if (launches) *launches += 2;
  return cudaGetLastError();
}

}  // namespace hw
