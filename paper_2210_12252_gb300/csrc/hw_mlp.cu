// Learned per-mode preconditioner: a 6 -> 64 -> 64 -> 1 network (SiLU) with BF16 weights and
// FP32 arithmetic, its inference inside the eigensolver and its training kernels.
//
// Not from the paper: it refines the paper's Teter-Payne-Allan diagonal (Sec. "Eigensolvers
// and Preconditioning").  For mode i of a column with Ritz value theta:
//   x_i = [KE_i/E0, (m-eta)/M, (n Ncyc - nu)/N, k/K, theta/E0, Vd_i/E0],  E0 = 10 Ha
//   o_i = w3 . silu(W2 silu(W1 x_i + b1) + b2) + b3,   s_i = tpa_i exp(o_i),   z_i = s_i r_i
// with tpa_i the TPA factor of the column and Vd_i the potential's diagonal in mode i
// (angular mean of V, integrated against xi_{n,k}^2).  A zero last layer reproduces TPA.
// Training loss per column (scale invariant, as LOBPCG is): 1 - |<z,e>|^2 / (|z|^2 |e|^2),
// e the target correction direction.  Gradients by hand-written backward kernels; Adam.
//
// Parameter layout (FP32, 4673 values): W1[64][6] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "hw_common.cuh"
#include "hw_ctx.h"

namespace hw {

constexpr int MH = 64, MIN_ = 6;
constexpr int OFF_W1 = 0, OFF_B1 = 384, OFF_W2 = 448, OFF_B2 = 4544, OFF_W3 = 4608, OFF_B3 = 4672;
constexpr int NPARAM = 4673;
constexpr float E0 = 10.0f;
constexpr int ROWVEC = MIN_ + 4 * MH + 1;   // per-row training scratch: x, h1, da1, h2, da2, do

struct MlpState {
  float* p32 = nullptr;       // FP32 master parameters
  float* m = nullptr;         // Adam moments
  float* v = nullptr;
  float* grad = nullptr;      // [NPARAM]
  int64_t adam_t = 0;
  double* vdiag = nullptr;    // concatenated per-k potential diagonal (same layout as ke)
  int* mnk = nullptr;         // concatenated per-k (m, n, k)
  double* colstat = nullptr;  // [cols][4]: ke_res, then A.re, A.im, B, C for training
  float* s_row = nullptr;     // [rows]
  float* rowbuf = nullptr;    // [rows][ROWVEC]
  double* ritz = nullptr;     // [cols]
  int64_t cap_rows = 0, cap_cols = 0;
  bool have_vdiag = false;
};

__device__ __forceinline__ float silu_f(float x) { return x / (1.0f + __expf(-x)); }
__device__ __forceinline__ float dsilu_f(float x) {
  const float sg = 1.0f / (1.0f + __expf(-x));
  return sg * (1.0f + x * (1.0f - sg));
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ------------------------------------------------------------------------ potential diagonal
// sum of V over the angular grid at each radial node
__global__ void k_vsum(const double* V, int n12, double* vsum) {
  griddep_entry();
  __shared__ double red[8];
  const int p = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n12; i += blockDim.x) s += V[(size_t)p * n12 + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    vsum[p] = t;
  }
}

// Vd_i = sum_p rfwd[n][k][p] rinv[n][p][k] vsum[p]  (rfwd carries 2 pi tau/Ncyc w_p/(N1 N2))
__global__ void k_vdiag(const int* mnk, int64_t nmode, const double* rinv, const double* rfwd,
                        const double* vsum, int Nr, int K, double* vd) {
  griddep_entry();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nmode; i += (int64_t)gridDim.x * blockDim.x) {
    const int n = abs(mnk[3 * i + 1]), k = mnk[3 * i + 2];
    const double* rf = rfwd + ((size_t)n * K + k) * Nr;
    const double* ri = rinv + (size_t)n * Nr * K + k;
    double s = 0.0;
    for (int p = 0; p < Nr; ++p) s += rf[p] * ri[(size_t)p * K] * vsum[p];
    vd[i] = s;
  }
}

// ------------------------------------------------------------------------ shared network code
struct MlpArgs {
  int ns;
  int64_t ld;
  int M, N, K, ncyc;
  const double* ke;
  const double* vd;
  const int* mnk;
  int64_t off[MAXSLOT];     // start of each block's k-point in ke / mnk
  int64_t vdoff[MAXSLOT];   // start of each block's k-point in vd
  int64_t L[MAXSLOT];
  double eta[MAXSLOT], nu[MAXSLOT];
  Blocks blk;               // x = R, y = Z (inference) or E (training)
  const double* ritz;       // [nslot][ns]
  const float* params;      // FP32 master
  double* colstat;          // [nslot*ns][5]
  float* s_row;             // [nslot*ns*Lmax]
  float* rowbuf;
  int64_t Lmax;
  float* grad;
};

__device__ __forceinline__ void load_params_bf16(const float* g, float* s) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) s[i] = bf16r(g[i]);
  __syncthreads();
}

__device__ __forceinline__ void features(const MlpArgs& A, int slot, int64_t i, double theta, float* x) {
  const int64_t o = A.off[slot] + i;
  const int m = A.mnk[3 * o], n = A.mnk[3 * o + 1], k = A.mnk[3 * o + 2];
  x[0] = (float)(A.ke[o] / E0);
  x[1] = (float)((m - A.eta[slot]) / (double)max(A.M, 1));
  x[2] = (float)((n * A.ncyc - A.nu[slot]) / (double)max(A.N, 1));
  x[3] = (float)(k / (double)max(A.K, 1));
  x[4] = (float)(theta / E0);
  x[5] = (float)(A.vd[A.vdoff[slot] + i] / E0);
}

// forward for one row; keeps a1 and h1 in registers, returns o (and h2 / a2 via callback)
__device__ __forceinline__ float net_forward(const float* P, const float* x, float* a1, float* h1) {
#pragma unroll
  for (int h = 0; h < MH; ++h) {
    float s = P[OFF_B1 + h];
#pragma unroll
    for (int i = 0; i < MIN_; ++i) s += P[OFF_W1 + h * MIN_ + i] * x[i];
    a1[h] = s;
    h1[h] = silu_f(s);
  }
  float o = P[OFF_B3];
  for (int h2 = 0; h2 < MH; ++h2) {
    float s = P[OFF_B2 + h2];
#pragma unroll
    for (int h = 0; h < MH; ++h) s += P[OFF_W2 + h2 * MH + h] * h1[h];
    o += P[OFF_W3 + h2] * silu_f(s);
  }
  return o;
}

__device__ __forceinline__ double tpa_of(double g) {
  const double P = 27.0 + g * (18.0 + g * (12.0 + g * 8.0));
  const double g2 = g * g;
  return P / (P + 16.0 * g2 * g2);
}

// per column: KE_res of the residual (the TPA statistic); grid (ns, nslot)
__global__ void k_col_keres(MlpArgs A) {
  griddep_entry();
  __shared__ double red[2][8];
  const int slot = blockIdx.y, s = blockIdx.x;
  const double2* r = reinterpret_cast<const double2*>(A.blk.x[slot]) + (size_t)s * A.ld;
  const double* ke = A.ke + A.off[slot];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = threadIdx.x; i < A.L[slot]; i += blockDim.x) {
    const double2 v = r[i];
    const double w = v.x * v.x + v.y * v.y;
    s0 += w;
    s1 += w * ke[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s0;
    red[1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      t0 += red[0][i];
      t1 += red[1][i];
    }
    double* cs = A.colstat + 5 * ((size_t)slot * A.ns + s);
    cs[0] = t0 > 0.0 ? t1 / t0 : 1.0;
    cs[1] = cs[2] = cs[3] = cs[4] = 0.0;
  }
}

// inference: Z = s R, all in FP32 (features, TPA factor, network, exp; FP64 <-> FP32 by bit
// operations, since this GPU's FP64 pipe would otherwise cost as much as the network);
// grid (row chunks, ns, nslot)
__global__ void __launch_bounds__(128) k_mlp_apply(MlpArgs A) {
  griddep_entry();
  extern __shared__ __align__(16) float Ps[];
  load_params_bf16(A.params, Ps);
  const int slot = blockIdx.z, s = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= A.L[slot]) return;
  const size_t col = (size_t)slot * A.ns + s;
  const float rkeres = 1.0f / d2f(A.colstat[5 * col]);
  const float theta = d2f(A.ritz[col]);
  const int64_t o = A.off[slot] + i;
  const int m = A.mnk[3 * o], n = A.mnk[3 * o + 1], k = A.mnk[3 * o + 2];
  const float ke = d2f(A.ke[o]);
  const float rE0 = (float)(1.0 / E0);
  float x[MIN_], a1[MH], h1[MH];
  x[0] = ke * rE0;
  x[1] = ((float)m - d2f(A.eta[slot])) / (float)max(A.M, 1);
  x[2] = ((float)(n * A.ncyc) - d2f(A.nu[slot])) / (float)max(A.N, 1);
  x[3] = (float)k / (float)max(A.K, 1);
  x[4] = theta * rE0;
  x[5] = d2f(A.vd[A.vdoff[slot] + i]) * rE0;
  const float out = net_forward(Ps, x, a1, h1);
  const float g = ke * rkeres;
  const float P = 27.0f + g * (18.0f + g * (12.0f + g * 8.0f));
  const float g2 = g * g;
  const float f = P / (P + 16.0f * g2 * g2) * expf(fminf(fmaxf(out, -30.f), 30.f));
  const float2 r = d2f(reinterpret_cast<const double2*>(A.blk.x[slot])[(size_t)s * A.ld + i]);
  reinterpret_cast<double2*>(A.blk.y[slot])[(size_t)s * A.ld + i] = f2d(make_float2(f * r.x, f * r.y));
}

// training forward: s_i per row and column sums A = <z,e>, B = |z|^2, C = |e|^2
__global__ void __launch_bounds__(128) k_mlp_fwd_train(MlpArgs A) {
  griddep_entry();
  extern __shared__ __align__(16) float Ps[];
  __shared__ double red[5][4];
  load_params_bf16(A.params, Ps);
  const int slot = blockIdx.z, s = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double vA_re = 0, vA_im = 0, vB = 0, vC = 0;
  const size_t col = (size_t)slot * A.ns + s;
  if (i < A.L[slot]) {
    const double keres = A.colstat[5 * col];
    const double theta = A.ritz[col];
    float x[MIN_], a1[MH], h1[MH];
    features(A, slot, i, theta, x);
    const float o = net_forward(Ps, x, a1, h1);
    const double sv = tpa_of(A.ke[A.off[slot] + i] / keres) * exp((double)fminf(fmaxf(o, -30.f), 30.f));
    A.s_row[col * A.Lmax + i] = (float)sv;
    const double2 r = reinterpret_cast<const double2*>(A.blk.x[slot])[(size_t)s * A.ld + i];
    const double2 e = reinterpret_cast<const double2*>(A.blk.y[slot])[(size_t)s * A.ld + i];
    // s conj(r) e
    vA_re = sv * (r.x * e.x + r.y * e.y);
    vA_im = sv * (r.x * e.y - r.y * e.x);
    vB = sv * sv * (r.x * r.x + r.y * r.y);
    vC = e.x * e.x + e.y * e.y;
  }
  double v[4] = {vA_re, vA_im, vB, vC};
#pragma unroll
  for (int c = 0; c < 4; ++c)
    for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
  if ((threadIdx.x & 31) == 0)
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x >> 5] = v[c];
  __syncthreads();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
    atomicAdd(&A.colstat[5 * col + 1 + threadIdx.x], t);
  }
}

// training backward per row: writes x, h1, da1, h2, da2, do to the row buffer
__global__ void __launch_bounds__(128) k_mlp_bwd_rows(MlpArgs A, int ncols_total) {
  griddep_entry();
  extern __shared__ __align__(16) float Ps[];
  load_params_bf16(A.params, Ps);
  const int slot = blockIdx.z, s = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const size_t col = (size_t)slot * A.ns + s;
  if (i >= A.Lmax) return;
  float* rb = A.rowbuf + (col * A.Lmax + i) * ROWVEC;
  if (i >= A.L[slot]) {
    for (int c = 0; c < ROWVEC; ++c) rb[c] = 0.f;
    return;
  }
  const double* cs = A.colstat + 5 * col;
  const double Are = cs[1], Aim = cs[2], B = cs[3], C = cs[4];
  const double sv = A.s_row[col * A.Lmax + i];
  const double2 r = reinterpret_cast<const double2*>(A.blk.x[slot])[(size_t)s * A.ld + i];
  const double2 e = reinterpret_cast<const double2*>(A.blk.y[slot])[(size_t)s * A.ld + i];
  // d loss / d s = -(2 Re(conj(A) conj(r) e) B - |A|^2 2 s |r|^2) / (B^2 C), loss averaged over columns
  const double cre = r.x * e.x + r.y * e.y, cim = r.x * e.y - r.y * e.x;   // conj(r) e
  const double dA2 = 2.0 * (Are * cre + Aim * cim);
  const double A2 = Are * Are + Aim * Aim;
  const double r2 = r.x * r.x + r.y * r.y;
  double ds = 0.0;
  if (B > 0.0 && C > 0.0) ds = -(dA2 * B - A2 * 2.0 * sv * r2) / (B * B * C) / ncols_total;
  const float dout = (float)(ds * sv);
  const double keres = cs[0];
  (void)keres;
  const double theta = A.ritz[col];
  float x[MIN_], a1[MH], h1[MH];
  features(A, slot, i, theta, x);
  net_forward(Ps, x, a1, h1);
  for (int c = 0; c < MIN_; ++c) rb[c] = x[c];
  for (int h = 0; h < MH; ++h) rb[MIN_ + h] = h1[h];
  float dh1[MH];
#pragma unroll
  for (int h = 0; h < MH; ++h) dh1[h] = 0.f;
  for (int h2 = 0; h2 < MH; ++h2) {
    float a2 = Ps[OFF_B2 + h2];
#pragma unroll
    for (int h = 0; h < MH; ++h) a2 += Ps[OFF_W2 + h2 * MH + h] * h1[h];
    const float hv = silu_f(a2);
    const float da2 = dout * Ps[OFF_W3 + h2] * dsilu_f(a2);
    rb[MIN_ + 2 * MH + h2] = hv;
    rb[MIN_ + 3 * MH + h2] = da2;
#pragma unroll
    for (int h = 0; h < MH; ++h) dh1[h] += Ps[OFF_W2 + h2 * MH + h] * da2;
  }
  for (int h = 0; h < MH; ++h) rb[MIN_ + MH + h] = dh1[h] * dsilu_f(a1[h]);
  rb[MIN_ + 4 * MH] = dout;
}

// weight gradients as sums over rows of outer products (split over row chunks, atomics)
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float* rowbuf, int64_t rows, float* grad) {
  griddep_entry();
  constexpr int CH = 32;
  __shared__ float rv[CH][ROWVEC];
  float acc[(NPARAM + 255) / 256];
#pragma unroll
  for (int j = 0; j < (NPARAM + 255) / 256; ++j) acc[j] = 0.f;
  const int64_t r0 = (int64_t)blockIdx.x * 1024;
  const int64_t r1 = (rows < r0 + 1024) ? rows : r0 + 1024;
  for (int64_t rb = r0; rb < r1; rb += CH) {
    const int nr = (int)((r1 - rb) < (int64_t)CH ? (r1 - rb) : (int64_t)CH);
    __syncthreads();
    for (int t = threadIdx.x; t < nr * ROWVEC; t += blockDim.x) rv[t / ROWVEC][t % ROWVEC] = rowbuf[(rb + t / ROWVEC) * ROWVEC + t % ROWVEC];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < (NPARAM + 255) / 256; ++j) {
      const int q = threadIdx.x + 256 * j;
      if (q >= NPARAM) break;
      float a = acc[j];
      for (int r = 0; r < nr; ++r) {
        const float* v = rv[r];
        const float* x = v;
        const float* h1 = v + MIN_;
        const float* da1 = v + MIN_ + MH;
        const float* h2 = v + MIN_ + 2 * MH;
        const float* da2 = v + MIN_ + 3 * MH;
        const float dout = v[MIN_ + 4 * MH];
        float g;
        if (q < OFF_B1) g = da1[q / MIN_] * x[q % MIN_];
        else if (q < OFF_W2) g = da1[q - OFF_B1];
        else if (q < OFF_B2) g = da2[(q - OFF_W2) / MH] * h1[(q - OFF_W2) % MH];
        else if (q < OFF_W3) g = da2[q - OFF_B2];
        else if (q < OFF_B3) g = dout * h2[q - OFF_W3];
        else g = dout;
        a += g;
      }
      acc[j] = a;
    }
  }
#pragma unroll
  for (int j = 0; j < (NPARAM + 255) / 256; ++j) {
    const int q = threadIdx.x + 256 * j;
    if (q < NPARAM && acc[j] != 0.f) atomicAdd(&grad[q], acc[j]);
  }
}

__global__ void k_loss(const double* colstat, int ncols, double* loss) {
  griddep_entry();
  double s = 0.0;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    const double* cs = colstat + 5 * c;
    const double A2 = cs[1] * cs[1] + cs[2] * cs[2];
    if (cs[3] > 0.0 && cs[4] > 0.0) s += 1.0 - A2 / (cs[3] * cs[4]);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *loss = t / ncols;
  }
}

__global__ void k_adam(float* p, float* m, float* v, const float* g, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  griddep_entry();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------------ host side
static cudaError_t mlp_fill_args(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, MlpArgs& a) {
  MlpState* st = ctx->mlp;
  const auto& hb = ctx->hb;
  a.ns = ns;
  a.ld = ld;
  a.M = hb.M;
  a.N = hb.N;
  a.K = hb.K;
  a.ncyc = hb.prm.ncyc;
  a.ke = ctx->db.ke;
  a.vd = st->vdiag;
  a.mnk = st->mnk;
  a.Lmax = 0;
  for (int i = 0; i < blk.nslot; ++i) {
    const int kb = blk.kb[i];
    a.off[i] = ctx->db.ke_off[kb];
    a.vdoff[i] = ctx->db.ke_off[kb];
    a.L[i] = hb.L[kb];
    a.eta[i] = hb.eta[kb];
    a.nu[i] = hb.nu[kb];
    a.Lmax = std::max(a.Lmax, a.L[i]);
  }
  a.blk = blk;
  a.ritz = st->ritz;
  a.params = st->p32;
  a.colstat = st->colstat;
  a.s_row = st->s_row;
  a.rowbuf = st->rowbuf;
  a.grad = st->grad;
  return cudaSuccess;
}

static cudaError_t mlp_reserve(hw_ctx* ctx, int64_t cols, int64_t rows) {
  MlpState* st = ctx->mlp;
  cudaError_t e = cudaSuccess;
  if (cols > st->cap_cols) {
    if (st->colstat) cudaFree(st->colstat);
    if (st->ritz) cudaFree(st->ritz);
    e = cudaMalloc((void**)&st->colstat, cols * 5 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&st->ritz, cols * sizeof(double));
    st->cap_cols = cols;
  }
  if (e == cudaSuccess && rows > st->cap_rows) {
    if (st->s_row) cudaFree(st->s_row);
    if (st->rowbuf) cudaFree(st->rowbuf);
    e = cudaMalloc((void**)&st->s_row, rows * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&st->rowbuf, rows * ROWVEC * sizeof(float));
    st->cap_rows = rows;
  }
  return e;
}

// called after hw_setup_basis / hw_set_potential: potential diagonal and index maps
cudaError_t mlp_refresh_potential(hw_ctx* ctx) {
  MlpState* st = ctx->mlp;
  if (!st || !ctx->have_basis || !ctx->have_V) return cudaSuccess;
  const auto& hb = ctx->hb;
  const int64_t nmode = ctx->db.ke_off[hb.nk];
  cudaError_t e = cudaSuccess;
  if (!st->mnk) {
    std::vector<int> all;
    all.reserve(3 * nmode);
    for (int b = 0; b < hb.nk; ++b) all.insert(all.end(), hb.mnk[b].begin(), hb.mnk[b].end());
    e = cudaMalloc((void**)&st->mnk, all.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(st->mnk, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void**)&st->vdiag, nmode * sizeof(double));
  }
  double* vsum = nullptr;
  if (e == cudaSuccess) e = cudaMalloc((void**)&vsum, hb.prm.Nr * sizeof(double));
  if (e != cudaSuccess) return e;
  launch_dep(ctx->stream, k_vsum, hb.prm.Nr, 256, 0, ctx->db.t64.V, hb.prm.Nth1 * hb.prm.Nth2, vsum);
  launch_dep(ctx->stream, k_vdiag, 256, 256, 0, st->mnk, nmode, ctx->db.t64.rinv, ctx->db.t64.rfwd, vsum, hb.prm.Nr,
                                        hb.K, st->vdiag);
  ctx->launches += 2;
  e = cudaStreamSynchronize(ctx->stream);
  cudaFree(vsum);
  st->have_vdiag = (e == cudaSuccess);
  return e;
}

void mlp_free_basis(hw_ctx* ctx) {
  MlpState* st = ctx->mlp;
  if (!st) return;
  if (st->mnk) cudaFree(st->mnk);
  if (st->vdiag) cudaFree(st->vdiag);
  st->mnk = nullptr;
  st->vdiag = nullptr;
  st->have_vdiag = false;
}

void mlp_free(hw_ctx* ctx) {
  MlpState* st = ctx->mlp;
  if (!st) return;
  mlp_free_basis(ctx);
  for (void* p : {(void*)st->p32, (void*)st->m, (void*)st->v, (void*)st->grad,
                  (void*)st->colstat, (void*)st->s_row, (void*)st->rowbuf, (void*)st->ritz})
    if (p) cudaFree(p);
  delete st;
  ctx->mlp = nullptr;
}

cudaError_t launch_precond_learned(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld,
                                   const double* const* ritz) {
  MlpState* st = ctx->mlp;
  if (!st || !st->have_vdiag) return cudaErrorNotReady;
  cudaError_t e = mlp_reserve(ctx, (int64_t)blk.nslot * ns, 0);
  if (e != cudaSuccess) return e;
  for (int b = 0; b < blk.nslot; ++b)
    cudaMemcpyAsync(st->ritz + (size_t)b * ns, ritz[b], ns * sizeof(double), cudaMemcpyDefault, ctx->stream);
  MlpArgs a;
  mlp_fill_args(ctx, blk, ns, ld, a);
  ProfScope ps(ctx, HW_PH_MLP);
  launch_dep(ctx->stream, k_col_keres, dim3(ns, blk.nslot), 256, 0, a);
  const int rb = 128;
  launch_dep(ctx->stream, k_mlp_apply, dim3((unsigned)((a.Lmax + rb - 1) / rb), ns, blk.nslot), rb, NPARAM * sizeof(float), a);
  ctx->launches += 2;
  return cudaGetLastError();
}

// forward + backward over one batch; gradient (averaged over columns) left in st->grad
static cudaError_t mlp_grad(hw_ctx* ctx, int k, const double* R, const double* E, const double* ritz_host,
                            int ns, int64_t ld, const double* vdiag_override, double* loss_dev) {
  MlpState* st = ctx->mlp;
  const int64_t L = ctx->hb.L[k];
  cudaError_t e = mlp_reserve(ctx, ns, (int64_t)ns * L);
  if (e != cudaSuccess) return e;
  cudaMemcpyAsync(st->ritz, ritz_host, ns * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  Blocks blk;
  blk.nslot = 1;
  blk.x[0] = R;
  blk.y[0] = const_cast<double*>(E);
  blk.kb[0] = k;
  MlpArgs a;
  mlp_fill_args(ctx, blk, ns, ld, a);
  if (vdiag_override) {
    a.vd = vdiag_override;
    a.vdoff[0] = 0;
  }
  ProfScope ps(ctx, HW_PH_MLP);
  cudaMemsetAsync(st->grad, 0, NPARAM * sizeof(float), ctx->stream);
  launch_dep(ctx->stream, k_col_keres, dim3(ns, 1), 256, 0, a);
  const int rb = 128;
  const dim3 g((unsigned)((L + rb - 1) / rb), ns, 1);
  launch_dep(ctx->stream, k_mlp_fwd_train, g, rb, NPARAM * sizeof(float), a);
  launch_dep(ctx->stream, k_mlp_bwd_rows, g, rb, NPARAM * sizeof(float), a, ns);
  const int64_t rows = (int64_t)ns * L;
  launch_dep(ctx->stream, k_mlp_wgrad, (unsigned)((rows + 1023) / 1024), 256, 0, st->rowbuf, rows, st->grad);
  launch_dep(ctx->stream, k_loss, 1, 256, 0, st->colstat, ns, loss_dev);
  ctx->launches += 5;
  return cudaGetLastError();
}

}  // namespace hw

using namespace hw;

static hw_status mlp_check(hw_ctx* ctx) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (!ctx->have_basis) return hw_fail(ctx, HW_ESTATE, "hw_setup_basis has not been called");
  return HW_OK;
}

extern "C" {

hw_status hw_set_mlp(hw_ctx* ctx, const float* params, int64_t n) {
  hw_status s = mlp_check(ctx);
  if (s != HW_OK) return s;
  if (!params || n != NPARAM) return hw_fail(ctx, HW_EINVAL, "the network has 4673 parameters");
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(params[i])) return hw_fail(ctx, HW_EINVAL, "non-finite network parameter");
  if (!ctx->mlp) {
    ctx->mlp = new MlpState();
    MlpState* st = ctx->mlp;
    cudaError_t e = cudaMalloc((void**)&st->p32, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&st->m, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&st->v, NPARAM * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&st->grad, NPARAM * sizeof(float));
    if (e != cudaSuccess) return hw_fail(ctx, HW_ENOMEM, "network state");
  }
  MlpState* st = ctx->mlp;
  cudaMemcpy(st->p32, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemset(st->m, 0, NPARAM * sizeof(float));
  cudaMemset(st->v, 0, NPARAM * sizeof(float));
  st->adam_t = 0;
  if (!st->have_vdiag && ctx->have_V) {
    cudaError_t e = mlp_refresh_potential(ctx);
    if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
  }
  return HW_OK;
}

hw_status hw_get_mlp(hw_ctx* ctx, float* params, int64_t n) {
  if (!ctx || !ctx->mlp) return hw_fail(ctx, HW_ESTATE, "no network installed");
  if (!params || n != NPARAM) return hw_fail(ctx, HW_EINVAL, "the network has 4673 parameters");
  cudaError_t e = cudaMemcpy(params, ctx->mlp->p32, NPARAM * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? HW_OK : hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
}

hw_status hw_get_potential_diagonal(hw_ctx* ctx, int k, double* vd) {
  hw_status s = mlp_check(ctx);
  if (s != HW_OK) return s;
  if (!ctx->mlp || !ctx->mlp->have_vdiag) return hw_fail(ctx, HW_ESTATE, "install a network and a potential first");
  if (k < 0 || k >= ctx->hb.nk || !vd) return hw_fail(ctx, HW_EINVAL, "bad k-point");
  cudaError_t e = cudaMemcpy(vd, ctx->mlp->vdiag + ctx->db.ke_off[k], ctx->hb.L[k] * sizeof(double),
                             cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? HW_OK : hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
}

hw_status hw_mlp_loss_grad(hw_ctx* ctx, int k, const double* R, const double* E, const double* ritz, int ns,
                           int64_t ld, const double* vdiag, double* loss, float* grad) {
  hw_status s = mlp_check(ctx);
  if (s != HW_OK) return s;
  if (!ctx->mlp || !ctx->mlp->have_vdiag) return hw_fail(ctx, HW_ESTATE, "install a network and a potential first");
  if (k < 0 || k >= ctx->hb.nk || !R || !E || !ritz || ns < 1 || ld < ctx->hb.L[k])
    return hw_fail(ctx, HW_EINVAL, "bad batch arguments");
  double* dloss = reinterpret_cast<double*>(ctx->dflag + 8);
  cudaError_t e = mlp_grad(ctx, k, R, E, ritz, ns, ld, vdiag, dloss);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, ctx->mlp->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return e == cudaSuccess ? HW_OK : hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
}

hw_status hw_mlp_train_step(hw_ctx* ctx, int k, const double* R, const double* E, const double* ritz, int ns,
                            int64_t ld, const double* vdiag, float lr, double* loss) {
  hw_status s = mlp_check(ctx);
  if (s != HW_OK) return s;
  if (!ctx->mlp || !ctx->mlp->have_vdiag) return hw_fail(ctx, HW_ESTATE, "install a network and a potential first");
  if (k < 0 || k >= ctx->hb.nk || !R || !E || !ritz || ns < 1 || ld < ctx->hb.L[k] || !(lr > 0))
    return hw_fail(ctx, HW_EINVAL, "bad batch arguments");
  MlpState* st = ctx->mlp;
  double* dloss = reinterpret_cast<double*>(ctx->dflag + 8);
  cudaError_t e = mlp_grad(ctx, k, R, E, ritz, ns, ld, vdiag, dloss);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
  st->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)st->adam_t), c2 = 1.f - std::pow(b2, (float)st->adam_t);
  {
    ProfScope ps(ctx, HW_PH_MLP);
    launch_dep(ctx->stream, k_adam, (NPARAM + 255) / 256, 256, 0, st->p32, st->m, st->v, st->grad, lr, b1, b2, 1e-8f, c1, c2);
    ctx->launches++;
  }
  if (loss) e = cudaMemcpyAsync(loss, dloss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return e == cudaSuccess ? HW_OK : hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
