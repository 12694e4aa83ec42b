// Complex block products of the eigensolver on the tensor cores (tcgen05, TMA, TMEM).
//
// The LOBPCG / Chebyshev steps of Sec. "Eigensolvers and Preconditioning" need, per iteration,
// products over the basis dimension L (Gram matrices S^H S and S^H H S, projections, the block
// updates [X P] = S Z): C = alpha op(A) B + beta C with op(A) = A^H (the reduction runs over L)
// or op(A) = A (the rows of C run over L), complex FP64 operands.  This GPU's FP64 rate is 1/64
// of its FP32 rate, while its tensor cores run at ~1-2 PFLOP/s; the products are computed there
// from split operands, in two accuracy classes:
//
// FP64 class (the FP64 phases): "digit planes" in the manner of Ozaki et al.  Every real row x of
//   an operand (complex entries as interleaved real pairs) is scaled by a power of two 2^-e so
//   that |x| < 1/2 and cut into S = 8 balanced base-2^7 digits,
//   x 2^-e = sum_{q=1..8} d_q 2^{-7 q} + eps, |d_q| <= 64, |eps| <= 2^-57;
//   the digits are small integers, exact in BF16.  A product sum_k x_k y_k is the sum over digit
//   pairs (p, q) with p + q <= 9 of 2^{-7 (p+q)} sum_k d_p,k d'_q,k; the pairs with p + q = t
//   form "group" t.  The tensor cores sum a group's integer products in FP32, exactly while the
//   sum stays below 2^24: every group's sum is drained from TMEM every 512 reduction elements
//   and added exactly to a 64-bit fixed-point accumulator.
// FP32 class (the FP32-product phase of the mixed form): "3 x TF32".  Every real entry x is
//   split as x = hi + lo + r with hi, lo TF32 numbers (hi = x rounded to 11 significant bits,
//   lo = x - hi rounded likewise; |r| <= 2^-22 |x|), and sum_k x_k y_k is taken as
//   hi hi' + hi lo' + lo hi' by three tcgen05 TF32 MMAs into one FP32 accumulator: per-entry
//   exponents, the accuracy of an FP32 product.
//
// Real forms (K = 2 x complex length, interleaved re/im):
//   op = ^H : D[i][j]     = sum_l a_il^re b_lj^re + a_il^im b_lj^im     = Re (A^H B)_ij
//             D[i][n + j] = sum_l a_il^re b_lj^im - a_il^im b_lj^re     = Im (A^H B)_ij
//             A-side rows: columns of A as (re, im); B-side rows j: (re, im), n + j: (im, -re)
//   op = N  : D[l][j]     = sum_c a_lc^re b_cj^re - a_lc^im b_cj^im     = Re (A B)_lj
//             D[l][n + j] = sum_c a_lc^re b_cj^im + a_lc^im b_cj^re     = Im (A B)_lj
//             A-side rows: rows of A as (re, im); B-side rows j: (re, -im), n + j: (im, re)
//
// Kernels: k_colmax / k_rowmax (FP64 class: the rows' largest magnitudes), k_split_cols /
// k_split_rows (the split planes [batch][plane][row][Kp], K contiguous, zero-padded to Kp),
// k_mma_digits / k_mma_tf32 (one CTA per 128 x BN output tile and K range: a TMA producer warp,
// an MMA warp issuing tcgen05.mma from shared memory into TMEM, eight epilogue warps draining
// TMEM), writing per-split partial sums [split][column][row]; k_zgemm_out adds the splits in a
// fixed order (deterministic) and applies the scales, alpha and beta.
// Every wait on an mbarrier is bounded; a wait that runs out sets HW_ETIMEOUT in the status word
// and the CTA leaves after its in-flight copies and tensor-core work have completed (or their
// own bounded waits ran out).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "hw_common.cuh"
#include "hw_ctx.h"
#include "hw_tc.cuh"
#include "hw_ff.cuh"

namespace hw {

// ----------------------------------------------------------------------------- configuration
template <int CLS> struct ZCfg;
template <> struct ZCfg<0> {      // FP64 class: BF16 digit planes, exact group sums
  static constexpr int S = 8, BITS = 7, BN = 64, SWZ = 64, STAGES = 2, WINDOW = 512;
};
constexpr int TF_PLANES = 2, TF_BN_MAX = 256, TF_STAGES = 2;   // FP32 class: TF32 hi / lo planes
constexpr int ZG_BM = 128;          // output rows per CTA (TMEM lanes)
constexpr int ZG_KALIGN = 64;       // Kp: reduction length padded to a multiple of this
// fixed point of the FP64 class: unit 2^-U with U = 61 - ceil(log2 Kp) (at most 56): the sum of
// Kp products of two numbers below 1/2 stays below 2^59 units, inside a signed 64-bit integer
inline int zg_fix_unit(int64_t Kp) {
  int l = 0;
  while ((int64_t(1) << l) < Kp) ++l;
  return std::min(56, 61 - l);
}
constexpr int ZG_THREADS = 320;     // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue (2 per TMEM lane quadrant)

template <int CLS>
constexpr size_t zg_stage_bytes() {
  return (size_t)ZCfg<CLS>::S * (ZG_BM + ZCfg<CLS>::BN) * ZCfg<CLS>::SWZ;
}
template <int CLS>
constexpr size_t zg_smem_bytes() {
  return (size_t)ZCfg<CLS>::STAGES * zg_stage_bytes<CLS>() + 1024;   // + alignment slack
}
__host__ __device__ constexpr size_t tf_stage_bytes() { return (size_t)TF_PLANES * (ZG_BM + TF_BN_MAX) * 128; }
__host__ __device__ constexpr size_t tf_smem_bytes() { return (size_t)TF_STAGES * tf_stage_bytes() + 1024; }

// ----------------------------------------------------------------------------- digit planes
// |x| as the ordered bit pattern of the magnitude (max of non-negative doubles = max of bits);
// zero for subnormals and zero (they take no part in the row scale)
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  return (u >> 52) == 0 ? 0ull : u;
}
// the row exponent e with max|x| 2^-e < 1/2 (e = E + 2 for max|x| in [2^E, 2^(E+1)))
__device__ __forceinline__ int row_exponent(unsigned long long mb) {
  return mb == 0 ? 0 : (int)(mb >> 52) - 1023 + 2;
}
// x 2^(bits s - e) rounded to the nearest integer (ties to even), exactly, by integer arithmetic
// on the FP64 encoding; |result| < 2^(bits s - 1) because |x| 2^-e < 1/2
template <int BITS, int S>
__device__ __forceinline__ long long fixed_of(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  if (E == 0) return 0;                                  // zero / subnormal
  const long long m = (long long)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  const int sh = E - 1075 - e + BITS * S;                // value = m 2^sh
  long long N;
  if (sh >= 0) {
    N = m << sh;
  } else {
    const int r = -sh;
    if (r > 62) {
      N = 0;
    } else {
      const long long q = m >> r, rem = m - (q << r), half = 1LL << (r - 1);
      N = q + ((rem > half || (rem == half && (q & 1))) ? 1 : 0);
    }
  }
  return (long long)(u >> 63) ? -N : N;
}
// balanced base-2^BITS digits of N, most significant first: d[0] 2^(BITS (S-1)) + ... + d[S-1]
template <int BITS, int S>
__device__ __forceinline__ void digits_of(long long N, float (&d)[S]) {
  constexpr long long B = 1LL << BITS, H = B >> 1;
#pragma unroll
  for (int q = S - 1; q >= 0; --q) {
    const long long r = ((N + H) & (B - 1)) - H;
    d[q] = (float)r;
    N = (N - r) >> BITS;
  }
  d[0] += (float)(N << BITS);   // N is zero here for |x| 2^-e < 1/2; kept for exactness
}

// x = hi + lo + r, |r| <= 2^-22 |x| (FP64 -> FP32 by bit operations, one FP64 subtraction)
__device__ __forceinline__ void tf32_split(double x, float& hi, float& lo) {
  hi = tf32_rn(d2f(x));
  lo = tf32_rn(d2f(x - f2d(hi)));
}

// ----------------------------------------------------------------------------- split planes
struct SplitArgs {
  const double2* X;      // source matrix, column-major complex, leading dimension ld
  int64_t ld, sX;        // leading dimension, batch stride (complex elements)
  int rows, cols;        // source shape (complex rows x columns)
  int mode;              // column sides: 0 out row c = (re, im) of column c; 1 rows c, cols+c =
                         // (re, im), (im, -re); 2 rows c, cols+c = (re, -im), (im, re)
                         // (row side: out row l = row l of X as (re, im))
  int nrow_out;          // rows of each output plane
  int64_t Kp;            // padded reduction length (real)
  void* P;               // planes [batch][plane][nrow_out][Kp] (BF16 digits or TF32 in FP32)
  const unsigned long long* mb;   // FP64 class: largest magnitude bits per source column / row
  int* ex;               // FP64 class: the exponents used, per output scale row [batch][cols or rows]
};

// |x| bits of every column's entries -> atomicMax into mb[batch][col]; grid (segments, cols, batch)
__global__ void k_colmax(const double2* X, int64_t ld, int64_t sX, int rows, int cols, unsigned long long* mb) {
  griddep_entry();
  const int c = blockIdx.y, b = blockIdx.z;
  const double2* x = X + (size_t)b * sX + (size_t)c * ld;
  unsigned long long m = 0;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < rows; l += gridDim.x * blockDim.x) {
    const double2 v = x[l];
    m = max(m, max(mag_bits(v.x), mag_bits(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(mb + (size_t)b * cols + c, m);
}

// |x| bits of every row's entries (rows of a column-major matrix): block (32 rows, 8 column
// groups), grid (row blocks, batch)
__global__ void __launch_bounds__(256) k_rowmax(const double2* X, int64_t ld, int64_t sX, int rows, int cols,
                                                unsigned long long* mb) {
  griddep_entry();
  __shared__ unsigned long long red[8][32];
  const int b = blockIdx.y, tx = threadIdx.x, ty = threadIdx.y;
  const int l = blockIdx.x * 32 + tx;
  unsigned long long m = 0;
  if (l < rows) {
    const double2* x = X + (size_t)b * sX + l;
    for (int c = ty; c < cols; c += 8) {
      const double2 v = x[(size_t)c * ld];
      m = max(m, max(mag_bits(v.x), mag_bits(v.y)));
    }
  }
  red[ty][tx] = m;
  __syncthreads();
  if (ty == 0 && l < rows) {
    for (int g = 1; g < 8; ++g) m = max(m, red[g][tx]);
    mb[(size_t)b * rows + l] = m;
  }
}

// Column sides: one thread per complex entry (grid (entry blocks over Kp/2, cols, batch)).
// CLS 0 writes S BF16 digit planes with the column's exponent, CLS 1 the TF32 hi / lo planes.
template <int CLS>
__global__ void __launch_bounds__(256) k_split_cols(SplitArgs a) {
  griddep_entry();
  const int c = blockIdx.y, b = blockIdx.z;
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= (int)(a.Kp >> 1)) return;
  double2 v = make_double2(0.0, 0.0);
  if (l < a.rows) v = a.X[(size_t)b * a.sX + (size_t)c * a.ld + l];
  const size_t plane = (size_t)a.nrow_out * a.Kp;
  const size_t r0 = (size_t)c * a.Kp, r1 = (size_t)(a.cols + c) * a.Kp;
  if constexpr (CLS == 0) {
    constexpr int S = ZCfg<0>::S, BITS = ZCfg<0>::BITS;
    const int e = row_exponent(a.mb[(size_t)b * a.cols + c]);
    if (l == 0) a.ex[(size_t)b * a.cols + c] = e;
    float dr[S], di[S];
    digits_of<BITS, S>(fixed_of<BITS, S>(v.x, e), dr);
    digits_of<BITS, S>(fixed_of<BITS, S>(v.y, e), di);
    __nv_bfloat16* P = reinterpret_cast<__nv_bfloat16*>(a.P) + (size_t)b * S * plane;
#pragma unroll
    for (int q = 0; q < S; ++q) {
      __nv_bfloat162* p0 = reinterpret_cast<__nv_bfloat162*>(P + q * plane + r0) + l;
      __nv_bfloat162* p1 = reinterpret_cast<__nv_bfloat162*>(P + q * plane + r1) + l;
      if (a.mode == 0) {
        *p0 = __floats2bfloat162_rn(dr[q], di[q]);
      } else if (a.mode == 1) {
        *p0 = __floats2bfloat162_rn(dr[q], di[q]);
        *p1 = __floats2bfloat162_rn(di[q], -dr[q]);
      } else {
        *p0 = __floats2bfloat162_rn(dr[q], -di[q]);
        *p1 = __floats2bfloat162_rn(di[q], dr[q]);
      }
    }
  } else {
    float hr, lr, hi_, li;
    tf32_split(v.x, hr, lr);
    tf32_split(v.y, hi_, li);
    float* P = reinterpret_cast<float*>(a.P) + (size_t)b * TF_PLANES * plane;
    float2* h0 = reinterpret_cast<float2*>(P + r0) + l;
    float2* q0 = reinterpret_cast<float2*>(P + plane + r0) + l;
    float2* h1 = reinterpret_cast<float2*>(P + r1) + l;
    float2* q1 = reinterpret_cast<float2*>(P + plane + r1) + l;
    if (a.mode == 0) {
      *h0 = make_float2(hr, hi_);
      *q0 = make_float2(lr, li);
    } else if (a.mode == 1) {
      *h0 = make_float2(hr, hi_);
      *q0 = make_float2(lr, li);
      *h1 = make_float2(hi_, -hr);
      *q1 = make_float2(li, -lr);
    } else {
      *h0 = make_float2(hr, -hi_);
      *q0 = make_float2(lr, -li);
      *h1 = make_float2(hi_, hr);
      *q1 = make_float2(li, lr);
    }
  }
}

// Row side (rows of a column-major matrix become K-major rows): a 32 x 32 tile of complex
// entries through shared memory, read along the rows' index, written along K.
// Block (32, 8); grid (row tiles, column tiles over Kp/2, batch).
template <int CLS>
__global__ void __launch_bounds__(256) k_split_rows(SplitArgs a) {
  griddep_entry();
  __shared__ double2 T[32][33];
  const int b = blockIdx.z, l0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const double2* X = a.X + (size_t)b * a.sX;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = c0 + ty + 8 * j, l = l0 + tx;
    T[ty + 8 * j][tx] = (l < a.rows && c < a.cols) ? X[(size_t)c * a.ld + l] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const size_t plane = (size_t)a.nrow_out * a.Kp;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int l = l0 + ty + 8 * j, c = c0 + tx;
    if (l >= a.rows || c >= (int)(a.Kp >> 1)) continue;
    const double2 v = T[tx][ty + 8 * j];
    if constexpr (CLS == 0) {
      constexpr int S = ZCfg<0>::S, BITS = ZCfg<0>::BITS;
      const int e = row_exponent(a.mb[(size_t)b * a.rows + l]);
      if (c == 0) a.ex[(size_t)b * a.rows + l] = e;
      float dr[S], di[S];
      digits_of<BITS, S>(fixed_of<BITS, S>(v.x, e), dr);
      digits_of<BITS, S>(fixed_of<BITS, S>(v.y, e), di);
      __nv_bfloat16* P = reinterpret_cast<__nv_bfloat16*>(a.P) + (size_t)b * S * plane + (size_t)l * a.Kp;
#pragma unroll
      for (int q = 0; q < S; ++q)
        reinterpret_cast<__nv_bfloat162*>(P + q * plane)[c] = __floats2bfloat162_rn(dr[q], di[q]);
    } else {
      float hr, lr, hi_, li;
      tf32_split(v.x, hr, lr);
      tf32_split(v.y, hi_, li);
      float* P = reinterpret_cast<float*>(a.P) + (size_t)b * TF_PLANES * plane + (size_t)l * a.Kp;
      reinterpret_cast<float2*>(P)[c] = make_float2(hr, hi_);
      reinterpret_cast<float2*>(P + plane)[c] = make_float2(lr, li);
    }
  }
}

struct MmaArgs {
  int Mr, Nr;            // real output rows / columns (D = A_r B_r^T)
  int kchunks;           // reduction chunks (of KC) in total
  int chunks_per_split;  // chunks handled by one CTA (the last split may have fewer)
  int nsplit;
  int BN;                // output columns per CTA (the TF32 kernel: a multiple of 32, <= 256)
  int64_t ldp;           // partial column pitch (elements; partials are [column][row])
  int64_t split_stride;  // partial elements per split (Nr_pad * ldp)
  int64_t batch_stride;  // partial elements per batch entry (nsplit * split_stride)
  void* part;            // int64 (FP64 class) or float (FP32 class) partials
  int fix_unit;          // FP64 class: fixed-point unit 2^-fix_unit
  int* status;
};

// group t = p + q (digits p, q numbered from 1) has weight 2^(-BITS t); for the FP64 class it
// enters the fixed point with unit 2^-U as g << (U - BITS t), or rounded g >> (BITS t - U)
__device__ __forceinline__ long long fix_add(long long acc, int g, int sh) {
  if (sh >= 0) return acc + ((long long)g << sh);
  const int r = -sh;
  return acc + (long long)((g + (1 << (r - 1))) >> r);
}

// add group T's FP32 sums (exact integers) of this thread's HB columns to the fixed point 2^-U
template <int BITS, int T, int S, int BN, int HB>
__device__ __forceinline__ void drain_group(uint32_t tl, long long (&acc)[HB], int U) {
  if constexpr (T <= S + 1) {
    const int sh = U - BITS * T;
#pragma unroll
    for (int c0 = 0; c0 < HB; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(tl + (uint32_t)((T - 2) * BN + c0), v);
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[c0 + j] = fix_add(acc[c0 + j], __float2int_rn(__uint_as_float(v[j])), sh);
    }
  }
}

// FP64 class: digit-plane products with exact group sums (see the head of this file)
__global__ void __launch_bounds__(ZG_THREADS, 1)
    k_mma_digits(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, MmaArgs a) {
  griddep_entry();
  using Cfg = ZCfg<0>;
  constexpr int S = Cfg::S, BITS = Cfg::BITS, BN = Cfg::BN, SWZ = Cfg::SWZ, STAGES = Cfg::STAGES;
  constexpr int KC = SWZ / 2;                             // reduction elements per stage
  constexpr int NG = S;                                   // groups t = 2 .. S + 1
  constexpr uint32_t TMEM_COLS = (NG * BN <= 256) ? ((NG * BN <= 128) ? 128 : 256) : 512;
  static_assert(NG * BN <= 512, "TMEM holds every group's accumulator");
  constexpr int WCH = Cfg::WINDOW / KC;                  // chunks per drain window
  constexpr uint32_t A_BYTES = S * ZG_BM * SWZ, B_BYTES = S * BN * SWZ;

  extern __shared__ __align__(1024) unsigned char zsm_raw[];
  unsigned char* zsm = (unsigned char*)(((uintptr_t)zsm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES], bar_acc_full, bar_acc_empty, bar_done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = blockIdx.x, tn = blockIdx.y;
  const int split = blockIdx.z % a.nsplit, batch = blockIdx.z / a.nsplit;
  const int c_begin = split * a.chunks_per_split;
  const int c_end = min(a.kchunks, c_begin + a.chunks_per_split);
  const int nch = max(0, c_end - c_begin);
  const int nwin = nch == 0 ? 0 : (nch + WCH - 1) / WCH;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    mbar_init(&bar_acc_full, 1);
    mbar_init(&bar_acc_empty, 256);
    mbar_init(&bar_done, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  auto fail = [&](int where) {
    abort_s = 1;
    atomicExch(a.status, HW_ETIMEOUT);
    (void)where;
  };

  if (warp == 0) {
    // ------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t in_flight = 0, parity = 0;       // per stage: a load was issued; its phase parity
      for (int it = 0; it < nch; ++it) {
        const int st = it % STAGES;
        const uint32_t ph = (uint32_t)((it / STAGES) & 1);
        if (*(volatile int*)&abort_s) break;
        if (!mbar_wait(&bar_empty[st], ph ^ 1u)) {
          fail(1);
          break;
        }
        unsigned char* sA = zsm + (size_t)st * (A_BYTES + B_BYTES);
        unsigned char* sB = sA + A_BYTES;
        mbar_expect_tx(&bar_full[st], A_BYTES + B_BYTES);
        const int k0 = (c_begin + it) * KC;
        tma_load_3d(sA, &tmA, k0, tm * ZG_BM, batch * S, &bar_full[st]);
        tma_load_3d(sB, &tmB, k0, tn * BN, batch * S, &bar_full[st]);
        in_flight |= 1u << st;
        parity = (parity & ~(1u << st)) | (ph << st);
      }
      // the copies this thread issued must land before the CTA may leave
      for (int s = 0; s < STAGES; ++s)
        if (((in_flight >> s) & 1u) && !mbar_wait(&bar_full[s], (parity >> s) & 1u)) fail(2);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = umma_idesc_bf16(BN);
      int it = 0;
      bool issued_any = false;
      for (int w = 0; w < nwin && !*(volatile int*)&abort_s; ++w) {
        if (w > 0 && !mbar_wait(&bar_acc_empty, (uint32_t)((w - 1) & 1))) {
          fail(3);
          break;
        }
        tc_fence_after();
        const int wend = min(nch, (w + 1) * WCH);
        bool first = true;
        for (; it < wend; ++it) {
          const int st = it % STAGES;
          if (!mbar_wait(&bar_full[st], (uint32_t)((it / STAGES) & 1))) {
            fail(4);
            break;
          }
          tc_fence_after();
          const uint32_t aBase = smem_u32(zsm + (size_t)st * (A_BYTES + B_BYTES));
          const uint32_t bBase = aBase + A_BYTES;
#pragma unroll 1
          for (int t = 2; t <= S + 1; ++t) {
            const uint32_t dt = tmem + (uint32_t)((t - 2) * BN);
            bool first_t = first;
#pragma unroll 1
            for (int p = max(1, t - S); p <= min(S, t - 1); ++p) {
              const int q = t - p;
              const uint64_t da = umma_desc<SWZ>(aBase + (uint32_t)((p - 1) * ZG_BM * SWZ));
              const uint64_t db = umma_desc<SWZ>(bBase + (uint32_t)((q - 1) * BN * SWZ));
#pragma unroll
              for (int kk = 0; kk < KC / 16; ++kk) {
                umma_bf16(dt, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc, first_t ? 0u : 1u);
                first_t = false;
              }
            }
          }
          issued_any = true;
          first = false;
          umma_commit(&bar_empty[st]);   // frees the stage once these MMAs have read it
        }
        if (*(volatile int*)&abort_s) break;
        umma_commit(&bar_acc_full);      // the window's sums are complete in TMEM
      }
      // no tensor-core work may be in flight when TMEM is released
      if (issued_any) {
        umma_commit(&bar_done);
        if (!mbar_wait(&bar_done, 0)) fail(5);
      }
    }
  } else {
    // ------------------------------------------------------------- epilogue (warps 2-9)
    constexpr int HB = BN / 2;                 // columns per epilogue thread
    const int quad = warp & 3;                 // TMEM lanes 32 quad .. 32 quad + 31
    const int hc = ((warp - 2) >> 2) * HB;     // first column of this warp's half
    const int row = quad * 32 + lane;          // output row within the tile
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)hc;
    const int grow = tm * ZG_BM + row;
    const int gcol = tn * BN + hc;
    long long acc[HB];
#pragma unroll
    for (int c = 0; c < HB; ++c) acc[c] = 0;
    bool ok = true;
    for (int w = 0; w < nwin; ++w) {
      if (!mbar_wait(&bar_acc_full, (uint32_t)(w & 1))) {
        fail(6);
        ok = false;
        break;
      }
      tc_fence_after();
      // group t's column block [(t - 2) BN, (t - 1) BN)
      drain_group<BITS, 2, S, BN, HB>(tl, acc, a.fix_unit);
      drain_group<BITS, 3, S, BN, HB>(tl, acc, a.fix_unit);
      drain_group<BITS, 4, S, BN, HB>(tl, acc, a.fix_unit);
      drain_group<BITS, 5, S, BN, HB>(tl, acc, a.fix_unit);
      drain_group<BITS, 6, S, BN, HB>(tl, acc, a.fix_unit);
      drain_group<BITS, 7, S, BN, HB>(tl, acc, a.fix_unit);
      drain_group<BITS, 8, S, BN, HB>(tl, acc, a.fix_unit);
      drain_group<BITS, 9, S, BN, HB>(tl, acc, a.fix_unit);
      tc_fence_before();
      mbar_arrive(&bar_acc_empty);
    }
    if (ok && !*(volatile int*)&abort_s && grow < a.Mr) {
      long long* P = reinterpret_cast<long long*>(a.part) + (size_t)batch * a.batch_stride +
                     (size_t)split * a.split_stride + (size_t)gcol * a.ldp + grow;
#pragma unroll
      for (int c = 0; c < HB; ++c)
        if (gcol + c < a.Nr) P[(size_t)c * a.ldp] = acc[c];
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// FP32 class: per stage the hi / lo TF32 planes of a 128 x 32 tile of A and a BN x 32 tile of B
// (128-byte swizzled rows); hi hi' + hi lo' + lo hi' accumulate into one FP32 tile in TMEM
// (BN columns); the epilogue writes the tile's FP32 partial sums.
__global__ void __launch_bounds__(ZG_THREADS, 1)
    k_mma_tf32(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, MmaArgs a) {
  griddep_entry();
  constexpr int KC = 32;                                  // FP32 entries per 128-byte row
  constexpr uint32_t TMEM_COLS = TF_BN_MAX;
  const int BN = a.BN;
  const uint32_t A_BYTES = TF_PLANES * ZG_BM * 128, B_BYTES = (uint32_t)(TF_PLANES * BN * 128);
  const uint32_t STAGE = (uint32_t)tf_stage_bytes();

  extern __shared__ __align__(1024) unsigned char zsm_raw[];
  unsigned char* zsm = (unsigned char*)(((uintptr_t)zsm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bar_full[TF_STAGES], bar_empty[TF_STAGES], bar_acc_full, bar_done;
  __shared__ uint32_t tmem_base_s;
  __shared__ int abort_s;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tm = blockIdx.x, tn = blockIdx.y;
  const int split = blockIdx.z % a.nsplit, batch = blockIdx.z / a.nsplit;
  const int c_begin = split * a.chunks_per_split;
  const int c_end = min(a.kchunks, c_begin + a.chunks_per_split);
  const int nch = max(0, c_end - c_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < TF_STAGES; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    mbar_init(&bar_acc_full, 1);
    mbar_init(&bar_done, 1);
    abort_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base_s;

  auto fail = [&]() {
    abort_s = 1;
    atomicExch(a.status, HW_ETIMEOUT);
  };

  if (warp == 0) {
    // ------------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t in_flight = 0, parity = 0;
      for (int it = 0; it < nch; ++it) {
        const int st = it % TF_STAGES;
        const uint32_t ph = (uint32_t)((it / TF_STAGES) & 1);
        if (*(volatile int*)&abort_s) break;
        if (!mbar_wait(&bar_empty[st], ph ^ 1u)) {
          fail();
          break;
        }
        unsigned char* sA = zsm + (size_t)st * STAGE;
        unsigned char* sB = sA + A_BYTES;
        mbar_expect_tx(&bar_full[st], A_BYTES + B_BYTES);
        const int k0 = (c_begin + it) * KC;
        tma_load_3d(sA, &tmA, k0, tm * ZG_BM, batch * TF_PLANES, &bar_full[st]);
        tma_load_3d(sB, &tmB, k0, tn * BN, batch * TF_PLANES, &bar_full[st]);
        in_flight |= 1u << st;
        parity = (parity & ~(1u << st)) | (ph << st);
      }
      for (int s = 0; s < TF_STAGES; ++s)
        if (((in_flight >> s) & 1u) && !mbar_wait(&bar_full[s], (parity >> s) & 1u)) fail();
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = umma_idesc_tf32(BN);
      bool issued_any = false;
      for (int it = 0; it < nch; ++it) {
        const int st = it % TF_STAGES;
        if (*(volatile int*)&abort_s) break;
        if (!mbar_wait(&bar_full[st], (uint32_t)((it / TF_STAGES) & 1))) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t aHi = smem_u32(zsm + (size_t)st * STAGE), aLo = aHi + ZG_BM * 128;
        const uint32_t bHi = aHi + A_BYTES, bLo = bHi + (uint32_t)(BN * 128);
#pragma unroll
        for (int kk = 0; kk < KC / 8; ++kk) {
          const uint64_t o = (uint64_t)(kk * 2);   // 8 TF32 entries = 32 bytes
          umma_tf32(tmem, umma_desc<128>(aHi) + o, umma_desc<128>(bHi) + o, idesc, (it | kk) ? 1u : 0u);
          umma_tf32(tmem, umma_desc<128>(aHi) + o, umma_desc<128>(bLo) + o, idesc, 1u);
          umma_tf32(tmem, umma_desc<128>(aLo) + o, umma_desc<128>(bHi) + o, idesc, 1u);
        }
        issued_any = true;
        umma_commit(&bar_empty[st]);
      }
      if (issued_any) {
        if (!*(volatile int*)&abort_s) umma_commit(&bar_acc_full);
        umma_commit(&bar_done);
        if (!mbar_wait(&bar_done, 0)) fail();
      }
    }
  } else {
    // ------------------------------------------------------------- epilogue (warps 2-9)
    const int HB = BN / 2;                     // a multiple of 16
    const int quad = warp & 3;
    const int hc = ((warp - 2) >> 2) * HB;
    const int row = quad * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)hc;
    const int grow = tm * ZG_BM + row;
    const int gcol = tn * BN + hc;
    bool ok = nch > 0 && mbar_wait(&bar_acc_full, 0u);
    if (nch > 0 && !ok) fail();
    tc_fence_after();
    float* P = reinterpret_cast<float*>(a.part) + (size_t)batch * a.batch_stride + (size_t)split * a.split_stride +
               (size_t)gcol * a.ldp + grow;
    const bool store = grow < a.Mr && !*(volatile int*)&abort_s;
    for (int c0 = 0; c0 < HB; c0 += 16) {
      uint32_t v[16];
      if (ok) tmem_ld16(tl + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (store && gcol + c0 + j < a.Nr) P[(size_t)(c0 + j) * a.ldp] = ok ? __uint_as_float(v[j]) : 0.f;
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// ----------------------------------------------------------------------------- reduction + output
struct OutArgs {
  int m, n, nsplit, cls, fix_unit;
  const void* part;
  int64_t ldp, split_stride, batch_stride;
  const int* exA;        // FP64 class: [batch][m]
  const int* exB;        // FP64 class: [batch][n]
  double alpha, beta;
  double2* C;
  int64_t ldc, sC;
};

// 2^e for the exponents that occur here (a normal FP64 number)
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(1023 + e) << 52); }

// C_ij = alpha (Re + i Im) scale + beta C_ij.  Block (64 rows, 4 thread groups), grid (row
// blocks, n or n / 4, batch).  With four or more splits group g adds the splits g, g + 4, ...
// of one column and the four group sums are added in the order g = 0..3; otherwise each group
// adds every split of its own column.  Deterministic (the FP64 class's 64-bit integer sums are
// exact in any order).  Partial reads ([split][column][row]) and writes of C are coalesced.
template <typename T, typename Acc>
__device__ __forceinline__ void sum_splits(const T* P, int nsplit, int g, int step, int64_t split_stride, size_t oR,
                                           size_t oI, Acc& re, Acc& im) {
  Acc r0 = 0, r1 = 0, i0 = 0, i1 = 0;
  int s = g;
  for (; s + step < nsplit; s += 2 * step) {
    const size_t o0 = (size_t)s * split_stride, o1 = o0 + (size_t)step * split_stride;
    r0 += (Acc)P[o0 + oR];
    i0 += (Acc)P[o0 + oI];
    r1 += (Acc)P[o1 + oR];
    i1 += (Acc)P[o1 + oI];
  }
  if (s < nsplit) {
    r0 += (Acc)P[(size_t)s * split_stride + oR];
    i0 += (Acc)P[(size_t)s * split_stride + oI];
  }
  re = r0 + r1;
  im = i0 + i1;
}

__global__ void __launch_bounds__(256) k_zgemm_out(OutArgs a) {
  griddep_entry();
  __shared__ double sre[4][64], sim[4][64];
  __shared__ long long ire[4][64], iim[4][64];
  const int b = blockIdx.z, r = threadIdx.x, g = threadIdx.y;
  const int i = blockIdx.x * 64 + r;
  // four or more splits: the four thread groups share one column's splits; fewer: each group
  // takes its own column (four columns per CTA) and all of its splits
  const bool by_split = a.nsplit >= 4;
  const int j = by_split ? blockIdx.y : blockIdx.y * 4 + g;
  const int gs = by_split ? g : 0, gstep = by_split ? 4 : 1;
  if (!by_split && j >= a.n) return;
  const size_t oR = (size_t)j * a.ldp, oI = (size_t)(a.n + j) * a.ldp;
  long long ir = 0, ii = 0;
  double dr = 0.0, di = 0.0;
  if (i < a.m) {
    if (a.cls == 0)
      sum_splits(reinterpret_cast<const long long*>(a.part) + (size_t)b * a.batch_stride + i, a.nsplit, gs, gstep,
                 a.split_stride, oR, oI, ir, ii);
    else
      sum_splits(reinterpret_cast<const float*>(a.part) + (size_t)b * a.batch_stride + i, a.nsplit, gs, gstep,
                 a.split_stride, oR, oI, dr, di);
  }
  if (by_split) {
    ire[g][r] = ir;
    iim[g][r] = ii;
    sre[g][r] = dr;
    sim[g][r] = di;
    __syncthreads();
    if (g != 0) return;
    ir = ire[0][r] + ire[1][r] + ire[2][r] + ire[3][r];
    ii = iim[0][r] + iim[1][r] + iim[2][r] + iim[3][r];
    dr = ((sre[0][r] + sre[1][r]) + sre[2][r]) + sre[3][r];
    di = ((sim[0][r] + sim[1][r]) + sim[2][r]) + sim[3][r];
  }
  if (i >= a.m) return;
  double re, im, sc;
  if (a.cls == 0) {
    re = (double)ir;
    im = (double)ii;
    sc = a.alpha * pow2(a.exA[(size_t)b * a.m + i] + a.exB[(size_t)b * a.n + j] - a.fix_unit);
  } else {
    re = dr;
    im = di;
    sc = a.alpha;
  }
  double2* c = a.C + (size_t)b * a.sC + (size_t)j * a.ldc + i;
  double2 v = make_double2(sc * re, sc * im);
  if (a.beta != 0.0) {
    const double2 o = *c;
    v.x += a.beta * o.x;
    v.y += a.beta * o.y;
  }
  *c = v;
}

// ----------------------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 3-D map over planes [planes][rows][Kp], box {swz / esz, box_rows, box_planes}
bool make_plane_map(CUtensorMap* m, const void* base, bool fp32, int64_t Kp, int rows, int planes,
                           int box_rows, int box_planes, int swz) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const int esz = fp32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * esz, (cuuint64_t)Kp * esz * rows};
  cuuint32_t box[3] = {(cuuint32_t)(swz / esz), (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base),
             dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             swz == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct ZgemmWork {
  void* buf = nullptr;   // planes A | planes B | partials | exponents | magnitude bits
  size_t cap = 0;
  int* status = nullptr;
  int nsm = 0;
  bool attr_set = false;
};

void zgemm_free(ZgemmWork*& w) {
  if (!w) return;
  if (w->buf) cudaFree(w->buf);
  if (w->status) cudaFree(w->status);
  delete w;
  w = nullptr;
}

static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

static cudaError_t zgemm_run(ZgemmWork* w, cudaStream_t st, int cls, bool transA, int m, int n, int k, double alpha,
                             const double2* A, int64_t lda, int64_t sA, const double2* B, int64_t ldb, int64_t sB,
                             double beta, double2* C, int64_t ldc, int64_t sC, int batch, int* launches) {
  const bool fp64 = cls == 0;
  const int planes = fp64 ? ZCfg<0>::S : TF_PLANES;
  const size_t esz = fp64 ? 2 : 4;
  const int Mr = m, Nr = 2 * n;
  const int64_t Kp = ((int64_t)2 * k + ZG_KALIGN - 1) / ZG_KALIGN * ZG_KALIGN;
  const int BN = fp64 ? ZCfg<0>::BN : std::min(TF_BN_MAX, (Nr + 31) / 32 * 32);
  const int KC = 32;   // reduction entries per stage in both classes
  const int mt = (Mr + ZG_BM - 1) / ZG_BM, nt = (Nr + BN - 1) / BN;
  const int kchunks = (int)(Kp / KC);
  // reduction splits: about one wave of CTAs, each at least 4 chunks, at most 32 splits
  const int tiles = mt * nt * batch;
  int nsplit = std::max(1, std::min({32, std::max(1, kchunks / 4), (w->nsm + tiles - 1) / tiles}));
  const int cps = (kchunks + nsplit - 1) / nsplit;
  nsplit = (kchunks + cps - 1) / cps;
  const int64_t ldp = (int64_t)mt * ZG_BM;
  const int64_t split_stride = (int64_t)nt * BN * ldp;
  const int64_t batch_stride = split_stride * nsplit;
  const size_t elem_part = fp64 ? 8 : 4;
  // per batch entry
  const size_t bytesA = (size_t)planes * Mr * Kp * esz, bytesB = (size_t)planes * Nr * Kp * esz;
  const size_t bytesP = (size_t)batch_stride * elem_part;
  const size_t bytesE = (size_t)(m + n) * sizeof(int), bytesM = (size_t)(m + n) * 8;
  const size_t per = al256(bytesA) + al256(bytesB) + al256(bytesP) + al256(bytesE) + al256(bytesM) + 5 * 256;
  // process the batch in chunks that fit the workspace (grown up to 1 GiB)
  const size_t limit = size_t(1) << 30;
  const int bchunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)batch, limit / per));
  const size_t need = per * bchunk;
  if (need > w->cap) {
    if (w->buf) cudaFree(w->buf);
    w->buf = nullptr;
    w->cap = 0;
    cudaError_t e = cudaMalloc(&w->buf, need);
    if (e != cudaSuccess) return e;
    w->cap = need;
  }
  if (!w->attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_mma_digits, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)zg_smem_bytes<0>());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_mma_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tf_smem_bytes());
    if (e != cudaSuccess) return e;
    w->attr_set = true;
  }
  for (int b0 = 0; b0 < batch; b0 += bchunk) {
    const int nb = std::min(bchunk, batch - b0);
    unsigned char* p = static_cast<unsigned char*>(w->buf);
    void* PA = p;
    p += al256(bytesA * nb);
    void* PB = p;
    p += al256(bytesB * nb);
    void* part = p;
    p += al256(bytesP * nb);
    int* exA = reinterpret_cast<int*>(p);
    int* exB = exA + (size_t)nb * m;
    p += al256(bytesE * nb);
    unsigned long long* mbA = reinterpret_cast<unsigned long long*>(p);
    unsigned long long* mbB = mbA + (size_t)nb * m;
    // split planes of the A side (columns of A for op = ^H, rows of A otherwise)
    SplitArgs sa;
    sa.X = A + (size_t)b0 * sA;
    sa.ld = lda;
    sa.sX = sA;
    sa.rows = transA ? k : m;
    sa.cols = transA ? m : k;
    sa.mode = 0;
    sa.nrow_out = Mr;
    sa.Kp = Kp;
    sa.P = PA;
    sa.mb = mbA;
    sa.ex = exA;
    SplitArgs sb;
    sb.X = B + (size_t)b0 * sB;
    sb.ld = ldb;
    sb.sX = sB;
    sb.rows = k;
    sb.cols = n;
    sb.mode = transA ? 1 : 2;
    sb.nrow_out = Nr;
    sb.Kp = Kp;
    sb.P = PB;
    sb.mb = mbB;
    sb.ex = exB;
    const int kh = (int)(Kp >> 1);
    if (fp64) {
      cudaMemsetAsync(mbA, 0, bytesM * nb, st);
      const int segs = std::max(1, std::min(64, (k + 2047) / 2048));
      if (transA)
        launch_dep(st, k_colmax, dim3(segs, m, nb), 256, 0, sa.X, lda, sA, k, m, mbA);
      else
        launch_dep(st, k_rowmax, dim3((m + 31) / 32, nb), dim3(32, 8), 0, sa.X, lda, sA, m, k, mbA);
      launch_dep(st, k_colmax, dim3(segs, n, nb), 256, 0, sb.X, ldb, sB, k, n, mbB);
      *launches += 2;
    }
    if (transA) {
      if (fp64)
        launch_dep(st, k_split_cols<0>, dim3((kh + 255) / 256, m, nb), 256, 0, sa);
      else
        launch_dep(st, k_split_cols<1>, dim3((kh + 255) / 256, m, nb), 256, 0, sa);
    } else {
      const dim3 g((m + 31) / 32, (kh + 31) / 32, nb);
      if (fp64)
        launch_dep(st, k_split_rows<0>, g, dim3(32, 8), 0, sa);
      else
        launch_dep(st, k_split_rows<1>, g, dim3(32, 8), 0, sa);
    }
    if (fp64)
      launch_dep(st, k_split_cols<0>, dim3((kh + 255) / 256, n, nb), 256, 0, sb);
    else
      launch_dep(st, k_split_cols<1>, dim3((kh + 255) / 256, n, nb), 256, 0, sb);
    CUtensorMap mA, mB;
    const int swz = fp64 ? ZCfg<0>::SWZ : 128;
    if (!make_plane_map(&mA, PA, !fp64, Kp, Mr, planes * nb, ZG_BM, planes, swz) ||
        !make_plane_map(&mB, PB, !fp64, Kp, Nr, planes * nb, BN, planes, swz))
      return cudaErrorInvalidValue;
    MmaArgs ma;
    ma.Mr = Mr;
    ma.Nr = Nr;
    ma.kchunks = kchunks;
    ma.chunks_per_split = cps;
    ma.nsplit = nsplit;
    ma.BN = BN;
    ma.ldp = ldp;
    ma.split_stride = split_stride;
    ma.batch_stride = batch_stride;
    ma.part = part;
    ma.fix_unit = zg_fix_unit(Kp);
    ma.status = w->status;
    const dim3 grid(mt, nt, nsplit * nb);
    if (fp64)
      launch_dep(st, k_mma_digits, grid, ZG_THREADS, zg_smem_bytes<0>(), mA, mB, ma);
    else
      launch_dep(st, k_mma_tf32, grid, ZG_THREADS, tf_smem_bytes(), mA, mB, ma);
    OutArgs oa;
    oa.m = m;
    oa.n = n;
    oa.nsplit = nsplit;
    oa.cls = cls;
    oa.fix_unit = zg_fix_unit(Kp);
    oa.part = part;
    oa.ldp = ldp;
    oa.split_stride = split_stride;
    oa.batch_stride = batch_stride;
    oa.exA = exA;
    oa.exB = exB;
    oa.alpha = alpha;
    oa.beta = beta;
    oa.C = C + (size_t)b0 * sC;
    oa.ldc = ldc;
    oa.sC = sC;
    launch_dep(st, k_zgemm_out, dim3((m + 63) / 64, nsplit >= 4 ? n : (n + 3) / 4, nb), dim3(64, 4), 0, oa);
    *launches += 4;
  }
  return cudaGetLastError();
}

cudaError_t zgemm_tc(ZgemmWork*& w, cudaStream_t st, int cls, bool transA, int m, int n, int k, double alpha,
                     const double2* A, int64_t lda, int64_t sA, const double2* B, int64_t ldb, int64_t sB,
                     double beta, double2* C, int64_t ldc, int64_t sC, int batch, int* launches) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (k <= 0 || (cls != 0 && cls != 1)) return cudaErrorInvalidValue;
  if (!w) {
    w = new ZgemmWork();
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&w->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaMalloc((void**)&w->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(w->status, 0, sizeof(int));
    if (e != cudaSuccess) return e;
  }
  return zgemm_run(w, st, cls, transA, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch, launches);
}

// ----------------------------------------------------------------------------- small products
// C_b = alpha op(A_b) B_b + beta C_b for the Rayleigh-Ritz step's small products (every extent
// below ZS_MAX), on the FP32 pipe: R = float for the FP32 class, double-float `ff` (~48-bit
// significands) for the FP64 class.  Operands are read in FP64 and rounded to R while they are
// staged; one CTA of 256 threads per 8 x 8 output tile, each output's reduction split four ways
// (k = part mod 4 within each 32-deep chunk) and the four partial sums added in a fixed order.
constexpr int ZS_T = 8, ZS_KC = 32, ZS_MAX = 1024;

template <typename R>
__global__ void __launch_bounds__(256) k_zgemm_small(int transA, int m, int n, int k, double alpha, const double2* A,
                                                      int64_t lda, int64_t sA, const double2* B, int64_t ldb,
                                                      int64_t sB, double beta, double2* C, int64_t ldc, int64_t sC) {
  griddep_entry();
  using Cr = rc_t<R>;
  __shared__ Cr As[ZS_T][ZS_KC + 1];   // op(A) rows of the tile, a chunk of the reduction
  __shared__ Cr Bs[ZS_KC][ZS_T];       // B rows (reduction index) x the tile's columns
  __shared__ Cr part_s[3][ZS_T * ZS_T];
  const int b = blockIdx.z;
  const int i0 = blockIdx.x * ZS_T, j0 = blockIdx.y * ZS_T;
  const int t = threadIdx.x, o = t & 63, p = t >> 6;   // output (tx, ty) = (o % 8, o / 8), reduction part p
  const int tx = o & 7, ty = o >> 3;
  const double2* a = A + (size_t)b * sA;
  const double2* bb = B + (size_t)b * sB;
  const R zr = R(0);
  R accr = zr, acci = zr;
  for (int k0 = 0; k0 < k; k0 += ZS_KC) {
    {   // one op(A) and one B element per thread, rounded to R
      // A tile: row r (0..7), reduction kk (0..31); consecutive threads along the operand's
      // contiguous index (the reduction for op = ^H, the rows otherwise)
      const int r = transA ? t >> 5 : t & 7, kk = transA ? t & 31 : t >> 3;
      const int gi = i0 + r, gk = k0 + kk;
      double2 x = make_double2(0.0, 0.0);
      if (gi < m && gk < k) {
        if (transA) {   // op(A)[i][k] = conj(A[k + i lda])
          x = a[gk + (size_t)gi * lda];
          x.y = -x.y;
        } else {
          x = a[gi + (size_t)gk * lda];
        }
      }
      As[r][kk] = mkr<R>(to_r<R>(x.x), to_r<R>(x.y));
      const int kb = t & 31, c = t >> 5;   // B tile: reduction kb, column c
      const int gkb = k0 + kb, gj = j0 + c;
      double2 y = make_double2(0.0, 0.0);
      if (gkb < k && gj < n) y = bb[gkb + (size_t)gj * ldb];
      Bs[kb][c] = mkr<R>(to_r<R>(y.x), to_r<R>(y.y));
    }
    __syncthreads();
#pragma unroll
    for (int kk = p; kk < ZS_KC; kk += 4) {
      const Cr x = As[tx][kk], y = Bs[kk][ty];
      accr += x.x * y.x - x.y * y.y;
      acci += x.x * y.y + x.y * y.x;
    }
    __syncthreads();
  }
  if (p > 0) part_s[p - 1][o] = mkr<R>(accr, acci);
  __syncthreads();
  if (p == 0) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {   // fixed order: part 0 + 1 + 2 + 3
      accr += part_s[q][o].x;
      acci += part_s[q][o].y;
    }
    const int gi = i0 + tx, gj = j0 + ty;
    if (gi < m && gj < n) {
      double2* c = C + (size_t)b * sC + gi + (size_t)gj * ldc;
      double2 v = make_double2(alpha * from_r<double>(accr), alpha * from_r<double>(acci));
      if (beta != 0.0) {   // C is not read when beta = 0
        const double2 c0 = *c;
        v.x += beta * c0.x;
        v.y += beta * c0.y;
      }
      *c = v;
    }
  }
}

// cls 0: FP64 class (double-float), 1: FP32 class
cudaError_t zgemm_small(cudaStream_t st, int cls, bool transA, int m, int n, int k, double alpha, const double2* A,
                        int64_t lda, int64_t sA, const double2* B, int64_t ldb, int64_t sB, double beta, double2* C,
                        int64_t ldc, int64_t sC, int batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  if (k <= 0 || m >= ZS_MAX || n >= ZS_MAX || k >= ZS_MAX || batch > 65535 || (cls != 0 && cls != 1))
    return cudaErrorInvalidValue;
  const dim3 grid((m + ZS_T - 1) / ZS_T, (n + ZS_T - 1) / ZS_T, batch);
  if (cls == 0)
    launch_dep(st, k_zgemm_small<ff>, grid, 256, 0, transA, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  else
    launch_dep(st, k_zgemm_small<float>, grid, 256, 0, transA, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  return cudaGetLastError();
}

int* zgemm_status_ptr(ZgemmWork* w) { return w ? w->status : nullptr; }

// status word of the tensor-core kernels (HW_OK, or HW_ETIMEOUT after a wait ran out); reset
int zgemm_status(ZgemmWork* w, cudaStream_t st, bool reset) {
  if (!w || !w->status) return HW_OK;
  int v = 0;
  cudaMemcpyAsync(&v, w->status, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  if (reset && v != 0) cudaMemsetAsync(w->status, 0, sizeof(int), st);
  return v;
}

}  // namespace hw

using namespace hw;

extern "C" hw_status hw_block_product(hw_ctx* ctx, int transA, int m, int n, int k, double alpha, const double* A,
                                      int64_t lda, int64_t sA, const double* B, int64_t ldb, int64_t sB, double beta,
                                      double* C, int64_t ldc, int64_t sC, int batch, int cls) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if ((transA != 0 && transA != 1) || cls < 0 || cls > 3 || m < 1 || n < 1 || k < 1 || batch < 1 || !A || !B || !C)
    return hw_fail(ctx, HW_EINVAL, "hw_block_product: bad arguments");
  if (cls >= 2 && (m >= 1024 || n >= 1024 || k >= 1024))
    return hw_fail(ctx, HW_EINVAL, "hw_block_product: the small-product classes take extents below 1024");
  if (lda < (transA ? k : m) || ldb < k || ldc < m || (batch > 1 && (sA < 0 || sB < 0 || sC < 0)))
    return hw_fail(ctx, HW_EINVAL, "hw_block_product: bad leading dimensions or strides");
  if ((int64_t)m > (1 << 20) || (int64_t)n > 4096 || (int64_t)k > (1 << 20))
    return hw_fail(ctx, HW_EINVAL, "hw_block_product: sizes out of range");
  cudaSetDevice(ctx->device);
  if (cls >= 2) {
    const cudaError_t e = zgemm_small(ctx->stream, cls - 2, transA != 0, m, n, k, alpha,
                                      reinterpret_cast<const double2*>(A), lda, sA, reinterpret_cast<const double2*>(B),
                                      ldb, sB, beta, reinterpret_cast<double2*>(C), ldc, sC, batch);
    ctx->launches++;
    if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("hw_block_product: ") + cudaGetErrorString(e));
    return HW_OK;
  }
  int nl = 0;
  cudaError_t e = zgemm_tc(ctx->zg, ctx->stream, cls, transA != 0, m, n, k, alpha,
                           reinterpret_cast<const double2*>(A), lda, sA, reinterpret_cast<const double2*>(B), ldb,
                           sB, beta, reinterpret_cast<double2*>(C), ldc, sC, batch, &nl);
  ctx->launches += nl;
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("hw_block_product: ") + cudaGetErrorString(e));
  return HW_OK;
}
