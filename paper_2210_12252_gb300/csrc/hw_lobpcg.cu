// Block LOBPCG for the helical-wave Hamiltonian (arXiv 2210.12252, Sec. "Eigensolvers and
// Preconditioning": LOBPCG with the Teter-Payne-Allan preconditioner), batched over k-points
// that iterate in lockstep.
//
// Per iteration and k-point (X: nb Ritz vectors, P: previous search directions, W: new ones):
//   R = H X - X Theta, residual norms (FP64); columns with ||r|| <= tol are soft-locked
//   W = K R[:, active]                      preconditioner (TPA or learned)
//   W -= [X P]([X P]^H W), twice            projection (classical Gram-Schmidt, repeated)
//   W = W U^{-1}, W^H W = U^H U, twice      Cholesky-QR
//   HW = H W                                the matrix-free product of Algorithm 5
//   A = S^H (H S), S = [X P W] orthonormal  Rayleigh-Ritz projection, FP64
//   A = Z diag(lambda) Z^H                  dense Hermitian eigensolver (Jacobi)
//   X = S Z[:, :nb], HX = HS Z[:, :nb]
//   P = S Y, HP = HS Y with Y = the W/P part of Z[:, active], orthogonalised against Z[:, :nb]
//        and orthonormalised in the small space (so [X P] stays orthonormal)
// Padding: k-points share the block layout; columns beyond a k-point's valid counts are zero
// and their Gram / Rayleigh-Ritz rows are padded (identity / huge diagonal).
//
// Precision: HW_FP64 runs every product in FP64.  HW_MIXED applies H in FP32 (the transforms)
// while Gram, Cholesky, Rayleigh-Ritz and the residuals stay FP64; HX is refreshed with an FP64
// product when the residuals first fall below 1e-3, and every convergence claim is verified by
// an FP64 recomputation of HX before it is accepted.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hw_common.cuh"
#include "hw_ctx.h"

namespace hw {

struct DenseWork;
cudaError_t dense_alloc(DenseWork*& dw, size_t cap_elems, int maxnprob);
void dense_free(DenseWork*& dw);
cudaError_t dense_heev(DenseWork* dw, cudaStream_t st, double2* A, int n, int nprob, double* w,
                       double2* Z, int* status, double tol);
cudaError_t dense_chol(cudaStream_t st, double2* G, int n, int nprob, int* fail, bool fp32 = false);
cudaError_t dense_barrier_selftest(cudaStream_t st, int nblocks, long spin_limit, int skip_block, int* wait_status);
size_t gram_work_bytes(int m, int n, int K, int batch);
cudaError_t gram_cf(cudaStream_t st, int m, int n, int K, double alpha, const double2* A, int64_t lda, int64_t sA,
                    const double2* B, int64_t ldb, int64_t sB, double beta, double2* C, int64_t ldc, int64_t sC,
                    int batch, void* work, size_t work_bytes, int* launches);
cudaError_t dense_trinv(cudaStream_t st, const double2* L, double2* Ui, int n, int nprob);
cudaError_t dense_hermitize(cudaStream_t st, double2* A, int n, int nprob);
cudaError_t dense_heev32(cudaStream_t st, const double2* A, int n, int nprob, double* w, double2* Z,
                         void* scratch, size_t scratch_bytes, int maxsweep);
size_t heev32_scratch_bytes(int n, int nprob, int maxsweep);
size_t jac32_smem(int n);
size_t hh_smem(int n);
cudaError_t dense_trsm_lh(cudaStream_t st, const double2* L, int m, int nprob, double2* W, int64_t rows, int64_t ld,
                          int64_t sW, bool fp32 = false, const int* skip = nullptr);
size_t hh_scratch_bytes(int n, int nw, int nprob);
cudaError_t dense_heev_hh32(cudaStream_t st, const double2* A, int n, int nw, int nprob, double2* Z, int64_t zstride,
                            void* scratch, size_t scratch_bytes, double* lam64, int stage = 3);
cudaError_t launch_oa_correction(cudaStream_t st, const double2* R, const double2* S, int n, int nw, int nprob,
                                 const double* lamall, double2* E);
cudaError_t launch_group_rr(cudaStream_t st, const double2* Sw, int nw, int nprob, int* grp, double* lam,
                            int lstride, double2* Ug);
cudaError_t launch_first_order(cudaStream_t st, const double2* Sp, int nw, int nprob, const int* grp, double2* F);
cudaError_t launch_sort_wanted(cudaStream_t st, const double* lam_in, int lstride, const double2* U, int nw, int nprob,
                               double* lam_out, double2* Uout);
constexpr int J32_SWEEPS = 12;
// Rayleigh-Ritz in FP32 while residuals exceed this.  Measured on the tube workload the FP32
// phase raised the iteration count (60 -> 71) without lowering the eigensolver time (the
// single-CTA FP32 Jacobi is instruction-bound on one SM), so it is off.
constexpr double FP32_RR_ABOVE = 1e300;
cudaError_t launch_precond_learned(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld,
                                   const double* const* ritz);

struct LobpcgWork {
  int nk = 0, nb = 0, ne = 0;   // ne: even Rayleigh-Ritz size bound >= 3 nb
  int64_t Lpad = 0;
  double2* SB[2] = {nullptr, nullptr};
  double2* HSB[2] = {nullptr, nullptr};
  double2* R = nullptr;
  double2* A = nullptr;     // [nk][ne*ne]
  double2* Z = nullptr;     // [nk][ne*ne]
  double* w = nullptr;      // [nk][ne]
  double2* G = nullptr;     // [nk][nb*nb] Gram / Cholesky factor
  double2* Ui = nullptr;    // [nk][nb*nb]
  double2* C = nullptr;     // [nk][2nb*nb] projection coefficients
  double2* Y = nullptr;     // [nk][ne*nb]
  double2* Y2 = nullptr;    // [nk][ne*nb]
  double* res = nullptr;    // [nk][nb]
  double* theta = nullptr;  // [nk][nb]
  int* iact = nullptr;      // [nk][nb] active column indices (-1 = padding)
  int* fail = nullptr;      // [nk]
  int* status = nullptr;
  DenseWork* dw = nullptr;
  void* j32 = nullptr;      // FP32 Jacobi scratch (rotation log, unsorted pairs)
  size_t j32_bytes = 0;
  void* hh = nullptr;       // Householder eigensolver scratch
  size_t hh_bytes = 0;
  double2* B1 = nullptr;    // [nk][ne*nb] refinement buffers
  double2* B2 = nullptr;
  double2* B3 = nullptr;
  int* grp = nullptr;       // [nk][nb]
  double2* Abak = nullptr;  // [nk][ne*ne] copy of the Rayleigh-Ritz matrix (Jacobi retry)
  void* gwork = nullptr;                          // gram_cf chunk partials
  size_t gbytes = 0;
  float2* F32[3] = {nullptr, nullptr, nullptr};   // FP32 operand copies for low-precision products
  size_t f32_ab = 0, f32_c = 0;                   // their sizes (elements)
};

void lobpcg_free(hw_ctx* ctx) {
  LobpcgWork* w = ctx->lw;
  if (!w) return;
  for (void* p : {(void*)w->SB[0], (void*)w->SB[1], (void*)w->HSB[0], (void*)w->HSB[1], (void*)w->R,
                  (void*)w->A, (void*)w->Z, (void*)w->w, (void*)w->G, (void*)w->Ui, (void*)w->C,
                  (void*)w->Y, (void*)w->Y2, (void*)w->res, (void*)w->theta, (void*)w->iact,
                  (void*)w->fail, (void*)w->status, w->j32, w->hh, (void*)w->B1, (void*)w->B2,
                  (void*)w->B3, (void*)w->grp, (void*)w->Abak, (void*)w->F32[0], (void*)w->F32[1],
                  (void*)w->F32[2], w->gwork})
    if (p) cudaFree(p);
  dense_free(w->dw);
  delete w;
  ctx->lw = nullptr;
}

namespace {

// ------------------------------------------------------------------------ small kernels
// R = HX - X theta and ||r_j||_2 (FP64); grid (nb, nk)
__global__ void k_residual(const double2* S, const double2* HS, int64_t Lpad, int64_t sK,
                           const double* theta, int nb, double2* R, double* res) {
  griddep_entry();
  __shared__ double red[8];
  const int j = blockIdx.x, b = blockIdx.y;
  const double2* x = S + (size_t)b * sK + (size_t)j * Lpad;
  const double2* hx = HS + (size_t)b * sK + (size_t)j * Lpad;
  double2* r = R + (size_t)b * Lpad * nb + (size_t)j * Lpad;
  const double th = theta[(size_t)b * nb + j];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < Lpad; i += blockDim.x) {
    const double2 a = hx[i], v = x[i];
    double2 q;
    q.x = a.x - th * v.x;
    q.y = a.y - th * v.y;
    r[i] = q;
    s += q.x * q.x + q.y * q.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    res[(size_t)b * nb + j] = sqrt(t);
  }
}

// W[:, i] = R[:, iact[b][i]] (zero for -1); W lives in S at column offset woff; grid (na, nk)
__global__ void k_gather_w(const double2* R, int nb, int64_t Lpad, const int* iact, int na, double2* S,
                           int64_t sK, int woff) {
  griddep_entry();
  const int i = blockIdx.x, b = blockIdx.y;
  const int src = iact[(size_t)b * nb + i];
  double2* w = S + (size_t)b * sK + (size_t)(woff + i) * Lpad;
  const double2* r = R + (size_t)b * Lpad * nb + (size_t)(src < 0 ? 0 : src) * Lpad;
  for (int64_t t = threadIdx.x; t < Lpad; t += blockDim.x) w[t] = src < 0 ? make_double2(0.0, 0.0) : r[t];
}

// pad an n x n Gram matrix: rows/cols i >= nv[b] become identity
__global__ void k_pad_gram(double2* G, int n, const int* nv) {
  griddep_entry();
  const int b = blockIdx.y;
  double2* g = G + (size_t)b * n * n;
  const int v = nv[b];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
    const int i = t % n, j = t / n;
    if (i >= v || j >= v) g[t] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
}

// pad the Rayleigh-Ritz matrix: index j of S = [X(nb) P(np) W(na)] is valid iff j < nb, or
// j in the P block below npv[b], or j in the W block below nav[b]; invalid rows/cols get a
// huge distinct diagonal so they sort last.  n may exceed nb+np+na by one (even size).
__global__ void k_pad_rr(double2* A, int n, int nb, int np, int na, const int* npv, const int* nav) {
  griddep_entry();
  const int b = blockIdx.y;
  double2* a = A + (size_t)b * n * n;
  auto valid = [&](int j) {
    if (j < nb) return true;
    if (j < nb + np) return j - nb < npv[b];
    if (j < nb + np + na) return j - nb - np < nav[b];
    return false;
  };
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x) {
    const int i = t % n, j = t / n;
    if (!valid(i) || !valid(j)) a[t] = make_double2(i == j ? 1e10 * (1.0 + 1e-3 * i) : 0.0, 0.0);
  }
}

// Y[:, i] = Z[:, iact[b][i]] with the X rows (< nb) zeroed; zero column for padding; grid (na, nk)
__global__ void k_build_y(const double2* Z, int ne, int nb, const int* iact, int na, double2* Y) {
  griddep_entry();
  const int i = blockIdx.x, b = blockIdx.y;
  const int src = iact[(size_t)b * nb + i];
  double2* y = Y + (size_t)b * ne * na + (size_t)i * ne;
  const double2* z = Z + (size_t)b * ne * ne + (size_t)(src < 0 ? 0 : src) * ne;
  for (int r = threadIdx.x; r < ne; r += blockDim.x)
    y[r] = (src < 0 || r < nb) ? make_double2(0.0, 0.0) : z[r];
}

// C = 1.5 I - 0.5 G (one Newton-Schulz step towards orthonormal columns); grid (8, nk)
__global__ void k_ns_coef(const double2* G, int m, double2* C) {
  griddep_entry();
  const int b = blockIdx.y;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * m; t += gridDim.x * blockDim.x) {
    const int i = t % m, j = t / m;
    const double2 g = G[(size_t)b * m * m + t];
    C[(size_t)b * m * m + t] = make_double2((i == j ? 1.5 : 0.0) - 0.5 * g.x, -0.5 * g.y);
  }
}

// w[b][j] = Re(z_j^H t_j) for the first m columns (Z and T with leading dimension n); grid (m, nk)
__global__ void k_rq_diag(const double2* Z, const double2* T, int n, int64_t sZ, int64_t sT, double* w, int64_t sw) {
  griddep_entry();
  __shared__ double red[8];
  const int j = blockIdx.x, b = blockIdx.y;
  const double2* z = Z + (size_t)b * sZ + (size_t)j * n;
  const double2* t = T + (size_t)b * sT + (size_t)j * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += z[i].x * t[i].x + z[i].y * t[i].y;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
    w[(size_t)b * sw + j] = a;
  }
}

// check of the Householder route's wanted block: fail[b] = 1 when an entry of Z_w^H Z_w - I
// (G, m x m) exceeds tol in modulus or an eigenvalue is not finite; grid nk
__global__ void k_check_gram(const double2* G, int m, const double* w, int wstride, double tol, int* fail) {
  griddep_entry();
  __shared__ int bad;
  const int b = blockIdx.x;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  int mine = 0;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    const int i = t % m, j = t / m;
    const double2 g = G[(size_t)b * m * m + t];
    const double dx = g.x - (i == j ? 1.0 : 0.0);
    if (!(dx * dx + g.y * g.y < tol * tol)) mine = 1;
  }
  for (int j = threadIdx.x; j < m; j += blockDim.x)
    if (!isfinite(w[(size_t)b * wstride + j])) mine = 1;
  if (mine) bad = 1;
  __syncthreads();
  if (threadIdx.x == 0) fail[b] = bad;
}

// A[i][j] = conj(A[j][i]) for rows i in [nb, nS) and columns j < nb (the X rows of the
// Rayleigh-Ritz matrix are formed in FP64; their mirror image replaces the lower-left blocks).
// grid (8, nk)
__global__ void k_mirror_xrows(double2* A, int n, int nb, int nS) {
  griddep_entry();
  const int b = blockIdx.y;
  double2* a = A + (size_t)b * n * n;
  const int rows = nS - nb;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < rows * nb; t += gridDim.x * blockDim.x) {
    const int i = nb + t % rows, j = t / rows;
    const double2 v = a[j + (size_t)i * n];
    a[i + (size_t)j * n] = make_double2(v.x, -v.y);
  }
}

// Gaussian start block from a counter-based generator (splitmix64 + Box-Muller); grid (nb, nk)
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void k_random_start(double2* S, int64_t Lpad, int64_t sK, const int64_t* L, int nb, uint64_t seed) {
  griddep_entry();
  const int j = blockIdx.x, b = blockIdx.y;
  double2* x = S + (size_t)b * sK + (size_t)j * Lpad;
  for (int64_t i = threadIdx.x; i < Lpad; i += blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (i < L[b]) {
      const uint64_t c = ((uint64_t)b << 48) ^ ((uint64_t)j << 32) ^ (uint64_t)i;
      const uint64_t u1 = splitmix64(seed ^ (2 * c)), u2 = splitmix64(seed ^ (2 * c + 1));
      const double a = ((u1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      const double t = ((u2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
      const double rr = sqrt(-log(a));   // complex Gaussian with E|z|^2 = 1
      v.x = rr * cos(6.283185307179586 * t);
      v.y = rr * sin(6.283185307179586 * t);
    }
    x[i] = v;
  }
}

// ------------------------------------------------------------------ Chebyshev filter kernels
// Per-k-point scalars of one step of the scaled three-term recurrence.
struct ChebScal {
  double al[MAXSLOT], c[MAXSLOT], be[MAXSLOT];
};

// One recurrence step on column blocks of S (block q = columns q nb .. q nb + nb - 1):
//   S[dst] = al_b (HS[src] - c_b S[src]) - be_b S[dst]      (be_b = 0: S[dst] is not read)
// i.e. Y_i = al (H Y_{i-1} - c Y_{i-1}) - be Y_{i-2} with Y_{i-2} in the destination block;
// columns j0 .. j0 + gridDim.x - 1 of each block; grid (columns, nk); src != dst
__global__ void k_cheb(double2* S, const double2* HS, int64_t Lpad, int64_t sK, int nb, int src, int dst, int j0,
                       ChebScal sc) {
  griddep_entry();
  const int j = j0 + blockIdx.x, b = blockIdx.y;
  const double al = sc.al[b], c = sc.c[b], be = sc.be[b];
  const size_t o = (size_t)b * sK;
  const double2* x = S + o + (size_t)(src * nb + j) * Lpad;
  const double2* hx = HS + o + (size_t)(src * nb + j) * Lpad;
  double2* y = S + o + (size_t)(dst * nb + j) * Lpad;
  for (int64_t i = threadIdx.x; i < Lpad; i += blockDim.x) {
    const double2 v = x[i], h = hx[i];
    double2 r = make_double2(al * (h.x - c * v.x), al * (h.y - c * v.y));
    if (be != 0.0) {
      const double2 yo = y[i];
      r.x -= be * yo.x;
      r.y -= be * yo.y;
    }
    y[i] = r;
  }
}

// scale columns j0 .. j0 + gridDim.x - 1 of block q to unit 2-norm (zero columns stay zero);
// grid (columns, nk)
__global__ void k_colnorm(double2* S, int64_t Lpad, int64_t sK, int nb, int q, int j0) {
  griddep_entry();
  __shared__ double red[32];
  __shared__ double scale;
  const int j = j0 + blockIdx.x, b = blockIdx.y;
  double2* y = S + (size_t)b * sK + (size_t)(q * nb + j) * Lpad;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < Lpad; i += blockDim.x) {
    const double2 v = y[i];
    s += v.x * v.x + v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    scale = t > 0.0 ? 1.0 / sqrt(t) : 1.0;
  }
  __syncthreads();
  const double f = scale;
  for (int64_t i = threadIdx.x; i < Lpad; i += blockDim.x) {
    double2 v = y[i];
    v.x *= f;
    v.y *= f;
    y[i] = v;
  }
}

// out[0] = max_i V[i]; one CTA
__global__ void k_vmax(const double* V, int64_t n, double* out) {
  griddep_entry();
  __shared__ double red[32];
  double m = -1e300;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, V[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = fmax(t, red[i]);
    out[0] = t;
  }
}

// copy the user's start block (L_b x nb, ld L_b) into S; grid (nb, nk)
struct PtrArr {
  const double* p[MAXSLOT];
};
__global__ void k_copy_start(PtrArr src, double2* S, int64_t Lpad, int64_t sK, const int64_t* L) {
  griddep_entry();
  const int j = blockIdx.x, b = blockIdx.y;
  const double2* s = reinterpret_cast<const double2*>(src.p[b]) + (size_t)j * L[b];
  double2* x = S + (size_t)b * sK + (size_t)j * Lpad;
  for (int64_t i = threadIdx.x; i < Lpad; i += blockDim.x) x[i] = i < L[b] ? s[i] : make_double2(0.0, 0.0);
}

// ------------------------------------------------------------------------ cuBLAS helper
// dst[b][c][r] = src[b][c*ld + r] (FP64 -> FP32 complex, packed columns); grid-stride
__global__ void k_cvt_d2f(const double2* __restrict__ src, int64_t ld, int rows, int cols, int64_t sSrc,
                          float2* __restrict__ dst, int batch) {
  griddep_entry();
  const int64_t per = (int64_t)rows * cols, tot = per * batch;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / per, q = t - b * per, c = q / rows, r = q - c * rows;
    dst[t] = d2f(src[b * sSrc + c * ld + r]);
  }
}

// dst[b][c*ld + r] = src[b][c][r] (FP32 -> FP64)
__global__ void k_cvt_f2d(const float2* __restrict__ src, int rows, int cols, double2* __restrict__ dst, int64_t ld,
                          int64_t sDst, int batch) {
  griddep_entry();
  const int64_t per = (int64_t)rows * cols, tot = per * batch;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / per, q = t - b * per, c = q / rows, r = q - c * rows;
    dst[b * sDst + c * ld + r] = f2d(src[t]);
  }
}

// Batched complex GEMM.  With `lowp` set (the early, large-residual iterations of the mixed
// form) products A^H B over the basis dimension go to gram_cf (FP32 products, FP64
// accumulation every 32 rows) when `gram` is on, the other products to cuBLAS CGEMM on FP32
// copies of the operands; otherwise everything is FP64 (cuBLAS ZGEMM).
struct Gemm {
  hw_ctx* ctx;
  cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
  cudaError_t ce = cudaSuccess;
  bool gram = false;          // mixed form: A^H B over the basis dimension by gram_cf
  void* gwork = nullptr;
  size_t gbytes = 0;
  bool lowp = false;
  float2* a32 = nullptr;
  float2* b32 = nullptr;
  float2* c32 = nullptr;
  size_t cap_ab = 0, cap_c = 0;   // elements
  void cvt_in(const double2* src, int64_t ld, int rows, int cols, int64_t s, float2* dst, int batch) {
    const int64_t tot = (int64_t)rows * cols * batch;
    const int grid = (int)std::min<int64_t>((tot + 255) / 256, 152 * 16);
    launch_dep(ctx->stream, k_cvt_d2f, grid, 256, 0, src, ld, rows, cols, s, dst, batch);
    ctx->launches++;
  }
  void operator()(cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double alpha,
                  const double2* A, int64_t lda, int64_t sA, const double2* B, int64_t ldb, int64_t sB,
                  double beta, double2* C, int64_t ldc, int64_t sC, int batch) {
    if (st != CUBLAS_STATUS_SUCCESS || m <= 0 || n <= 0) return;
    if (k <= 0) {  // C = beta C
      if (beta == 1.0) return;
    }
    ProfScope ps(ctx, HW_PH_GEMM);
    // the tensor-core kernel: products over the basis dimension (or all, option 2)
    if (ctx->tc_gemm && k >= 1 && tb == CUBLAS_OP_N && (ta == CUBLAS_OP_C || ta == CUBLAS_OP_N) &&
        (ctx->tc_gemm == 2 || (ta == CUBLAS_OP_C ? k : m) >= 1024) && n <= 4096) {
      int nl = 0;
      const cudaError_t e = zgemm_tc(ctx->zg, ctx->stream, lowp ? 1 : 0, ta == CUBLAS_OP_C, m, n, k, alpha, A, lda,
                                     sA, B, ldb, sB, beta, C, ldc, sC, batch, &nl);
      ctx->launches += nl;
      if (e != cudaSuccess && ce == cudaSuccess) ce = e;
      return;
    }
    // the small products (every extent below 1024: the Rayleigh-Ritz step) on the FP32 pipe
    // (HW_OPT_SMALL_GEMM): the FP32 class always; the FP64 class in double-float inside
    // mixed-precision solves (the FP64 refinement divides its products' errors by eigenvalue
    // gaps: double-float's ~1e-14 leaves the refined vectors orthonormal to ~1e-11, within the
    // mixed solver's 1e-9 check; FP64 solves and hw_heev keep FP64 products)
    if (ctx->small_gemm && (lowp || ctx->mixed_solve || ctx->small_gemm == 2) && k >= 1 && tb == CUBLAS_OP_N &&
        (ta == CUBLAS_OP_C || ta == CUBLAS_OP_N) && m < 1024 && n < 1024 && k < 1024 && batch <= 65535) {
      const cudaError_t e = zgemm_small(ctx->stream, lowp ? 1 : 0, ta == CUBLAS_OP_C, m, n, k, alpha, A, lda, sA, B,
                                        ldb, sB, beta, C, ldc, sC, batch);
      ctx->launches++;
      if (e != cudaSuccess && ce == cudaSuccess) ce = e;
      return;
    }
    if (gram && lowp && ta == CUBLAS_OP_C && tb == CUBLAS_OP_N && k >= 256 &&
        gram_work_bytes(m, n, k, batch) <= gbytes) {
      int nl = 0;
      const cudaError_t e = gram_cf(ctx->stream, m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch,
                                    gwork, gbytes, &nl);
      ctx->launches += nl;
      if (e != cudaSuccess && ce == cudaSuccess) ce = e;
      return;
    }
    const int ra = ta == CUBLAS_OP_N ? m : k, ca = ta == CUBLAS_OP_N ? k : m;
    const int rb = tb == CUBLAS_OP_N ? k : n, cb = tb == CUBLAS_OP_N ? n : k;
    if (lowp && k >= 16 && (size_t)ra * ca * batch <= cap_ab &&
        (size_t)rb * cb * batch <= cap_ab && (size_t)m * n * batch <= cap_c) {
      cvt_in(A, lda, ra, ca, sA, a32, batch);
      const bool same = A == B && lda == ldb && sA == sB && ra == rb && ca == cb;
      if (!same) cvt_in(B, ldb, rb, cb, sB, b32, batch);
      if (beta != 0.0) cvt_in(C, ldc, m, n, sC, c32, batch);
      const cuComplex al = make_cuComplex((float)alpha, 0.f), be = make_cuComplex((float)beta, 0.f);
      st = cublasCgemmStridedBatched(ctx->cublas, ta, tb, m, n, k, &al, reinterpret_cast<const cuComplex*>(a32), ra,
                                     (int64_t)ra * ca, reinterpret_cast<const cuComplex*>(same ? a32 : b32), rb,
                                     (int64_t)rb * cb, &be, reinterpret_cast<cuComplex*>(c32), m, (int64_t)m * n,
                                     batch);
      const int64_t tot = (int64_t)m * n * batch;
      const int grid = (int)std::min<int64_t>((tot + 255) / 256, 152 * 16);
      launch_dep(ctx->stream, k_cvt_f2d, grid, 256, 0, c32, m, n, C, ldc, sC, batch);
      ctx->launches++;
      return;
    }
    const cuDoubleComplex al = make_cuDoubleComplex(alpha, 0.0), be = make_cuDoubleComplex(beta, 0.0);
    st = cublasZgemmStridedBatched(ctx->cublas, ta, tb, m, n, std::max(k, 1), &al,
                                   reinterpret_cast<const cuDoubleComplex*>(A), (int)lda, sA,
                                   reinterpret_cast<const cuDoubleComplex*>(B), (int)ldb, sB, &be,
                                   reinterpret_cast<cuDoubleComplex*>(C), (int)ldc, sC, batch);
  }
};

}  // namespace

// append one iteration's largest wanted residual of k-point kidx to the context's history
static void hist_push(hw_ctx* ctx, int kidx, int phase, double res) {
  size_t slot = 0;
  while (slot < ctx->hist_k.size() && ctx->hist_k[slot] != kidx) ++slot;
  if (slot == ctx->hist_k.size()) {
    ctx->hist_k.push_back(kidx);
    ctx->hist_phase.emplace_back();
    ctx->hist_res.emplace_back();
  }
  ctx->hist_phase[slot].push_back(phase);
  ctx->hist_res[slot].push_back(res);
}

// Orthonormalise `ncol` columns of S at column offset c0 for every k-point by Cholesky-QR
// (Gram, Cholesky, triangular inverse, GEMM), `passes` times.  nv[b]: valid columns of k-point
// b (device).  On a failed factorisation the k-point's fail flag is set.
static hw_status cholqr(hw_ctx* ctx, LobpcgWork* w, Gemm& gemm, double2* S, int c0, int ncol,
                        const int* d_nv, int passes, std::vector<int>& failed) {
  const int nk = w->nk;
  const int64_t Lpad = w->Lpad, sK = Lpad * 3 * w->nb;
  double2* Wb = S + (size_t)c0 * Lpad;
  failed.assign(nk, 0);
  for (int pass = 0; pass < passes; ++pass) {
    // FP32 factor in the FP32-product phase; a k-point whose FP32 factorisation fails keeps its
    // block untouched and is factored again in FP64
    for (int attempt = gemm.lowp ? 0 : 1; attempt < 2; ++attempt) {
      const bool fp32 = attempt == 0;
      const bool keep = gemm.lowp;
      gemm.lowp = fp32;
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, ncol, ncol, (int)Lpad, 1.0, Wb, Lpad, sK, Wb, Lpad, sK, 0.0, w->G, ncol,
           (int64_t)ncol * ncol, nk);
      gemm.lowp = keep;
      {
        ProfScope ps_(ctx, HW_PH_OTHER);
        launch_dep(ctx->stream, k_pad_gram, dim3(8, nk), 256, 0, w->G, ncol, d_nv);
        ctx->launches++;
      }
      {
        ProfScope ps_(ctx, HW_PH_CHOL,
                      nk * ((8.0 / 3.0) * ncol * (double)ncol * ncol + 4.0 * (double)Lpad * ncol * ncol));
        dense_hermitize(ctx->stream, w->G, ncol, nk);
        dense_chol(ctx->stream, w->G, ncol, nk, w->fail, fp32);
        const cudaError_t te = dense_trsm_lh(ctx->stream, w->G, ncol, nk, Wb, Lpad, Lpad, sK, fp32, w->fail);
        if (te != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("cholqr: ") + cudaGetErrorString(te));
        ctx->launches += 3;
      }
      std::vector<int> f(nk);
      cudaMemcpyAsync(f.data(), w->fail, nk * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("cholqr: ") + cudaGetErrorString(e));
      bool anyf = false;
      for (int b = 0; b < nk; ++b) anyf = anyf || f[b];
      if (!anyf) break;
      if (!fp32)
        for (int b = 0; b < nk; ++b)
          if (f[b]) failed[b] = 1;
    }
  }
  return gemm.st == CUBLAS_STATUS_SUCCESS ? HW_OK : hw_fail(ctx, HW_ECUDA, "cuBLAS failure in Cholesky-QR");
}

// Orthonormalise `ncol` nearly orthonormal columns of S at column offset c0 (all valid, every
// k-point) by `passes` Newton-Schulz steps X <- X (3 I - X^H X) / 2 in FP64 products: the
// deviation from orthonormality E = X^H X - I goes to (3/4) E^2 + O(E^3) per step, so two steps
// take the FP32 phase's 1e-6 to the products' rounding.  The product X C goes through w->R
// (free here: the caller recomputes the residuals).  ok = false, with S untouched, when some
// k-point's Gram is more than 0.1 from the identity in an entry: the caller then uses
// Cholesky-QR.
static hw_status ns_orth(hw_ctx* ctx, LobpcgWork* w, Gemm& gemm, double2* S, int c0, int ncol, int passes,
                         bool& ok) {
  const int nk = w->nk;
  const int64_t Lpad = w->Lpad, sK = Lpad * 3 * w->nb;
  double2* Xb = S + (size_t)c0 * Lpad;
  cudaStream_t st = ctx->stream;
  ok = true;
  for (int pass = 0; pass < passes; ++pass) {
    gemm(CUBLAS_OP_C, CUBLAS_OP_N, ncol, ncol, (int)Lpad, 1.0, Xb, Lpad, sK, Xb, Lpad, sK, 0.0, w->G, ncol,
         (int64_t)ncol * ncol, nk);
    if (pass == 0) {
      std::vector<double2> g((size_t)nk * ncol * ncol);
      cudaMemcpyAsync(g.data(), w->G, g.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("Newton-Schulz: ") + cudaGetErrorString(e));
      double dev = 0.0;
      for (size_t t = 0; t < g.size(); ++t) {
        const int i = (int)(t % ncol), j = (int)((t / ncol) % ncol);
        dev = std::max(dev, std::hypot(g[t].x - (i == j ? 1.0 : 0.0), g[t].y));
      }
      if (!(dev <= 0.1)) {
        ok = false;
        return HW_OK;
      }
    }
    {
      ProfScope ps_(ctx, HW_PH_CHOL);
      launch_dep(st, k_ns_coef, dim3(8, nk), 256, 0, w->G, ncol, w->Ui);
      ctx->launches++;
    }
    gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, ncol, ncol, 1.0, Xb, Lpad, sK, w->Ui, ncol, (int64_t)ncol * ncol, 0.0,
         w->R, Lpad, Lpad * w->nb, nk);
    cudaMemcpy2DAsync(Xb, (size_t)sK * sizeof(double2), w->R, (size_t)Lpad * w->nb * sizeof(double2),
                      (size_t)Lpad * ncol * sizeof(double2), nk, cudaMemcpyDeviceToDevice, st);
  }
  return gemm.st == CUBLAS_STATUS_SUCCESS ? HW_OK : hw_fail(ctx, HW_ECUDA, "cuBLAS failure in Newton-Schulz");
}

// Rayleigh-Ritz eigenpairs of the nk matrices w->A (n x n, padded, Hermitian): w->w ascending,
// w->Z eigenvector columns.  fp32: FP32 Jacobi, then the first nb vectors are made orthonormal
// in FP64 (two Newton-Schulz steps) and their Rayleigh quotients recomputed in FP64; else the
// FP64 Jacobi.
// Householder route: FP32 tridiagonalisation, bisection, inverse iteration and back-transform
// for all n vectors, then two FP64 first-order corrections of the wanted nb vectors against
// all n, then FP64 Rayleigh-Ritz inside groups of near-degenerate wanted vectors.
static cudaError_t rr_eig_hh(hw_ctx* ctx, LobpcgWork* w, Gemm& gemm, int n, int nb, bool lite) {
  cudaStream_t st = ctx->stream;
  const int nk = w->nk;
  cudaError_t e;
  {
    ProfScope ps_(ctx, HW_PH_EIG);
    dense_hermitize(st, w->A, n, nk);
    ctx->launches++;
  }
  {
    ProfScope ps_(ctx, HW_PH_TRIDIAG, (16.0 / 3.0) * n * (double)n * n * nk);
    e = dense_heev_hh32(st, w->A, n, lite ? nb : n, nk, w->Z, (int64_t)n * n, w->hh, w->hh_bytes, w->w, 1);
    ctx->launches++;
  }
  if (e != cudaSuccess) return e;
  {
    ProfScope ps_(ctx, HW_PH_EIG);
    e = dense_heev_hh32(st, w->A, n, lite ? nb : n, nk, w->Z, (int64_t)n * n, w->hh, w->hh_bytes, w->w, 2);
    ctx->launches += 3;
  }
  if (e != cudaSuccess) return e;
  const int64_t sZ = (int64_t)n * n, sB = (int64_t)n * nb;
  if (lite) {
    // FP32-product phase: the FP32 pairs, made orthonormal by two Newton-Schulz steps
    for (int pass = 0; pass < 2; ++pass) {
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, n, 1.0, w->Z, n, sZ, w->Z, n, sZ, 0.0, w->G, nb, (int64_t)nb * nb, nk);
      {
        ProfScope ps_(ctx, HW_PH_EIG);
        launch_dep(st, k_ns_coef, dim3(8, nk), 256, 0, w->G, nb, w->Ui);
        ctx->launches++;
      }
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, nb, 1.0, w->Z, n, sZ, w->Ui, nb, (int64_t)nb * nb, 0.0, w->B2, n, sB, nk);
      cudaMemcpy2DAsync(w->Z, (size_t)sZ * 16, w->B2, (size_t)sB * 16, (size_t)sB * 16, nk, cudaMemcpyDeviceToDevice, st);
    }
    return cudaGetLastError();
  }
  for (int it = 0; it < 2; ++it) {
    gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, n, 1.0, w->A, n, sZ, w->Z, n, sZ, 0.0, w->B1, n, sB, nk);   // A Z_w
    gemm(CUBLAS_OP_C, CUBLAS_OP_N, n, nb, n, 1.0, w->Z, n, sZ, w->B1, n, sB, 0.0, w->B2, n, sB, nk);  // Z^H A Z_w
    gemm(CUBLAS_OP_C, CUBLAS_OP_N, n, nb, n, 1.0, w->Z, n, sZ, w->Z, n, sZ, 0.0, w->B3, n, sB, nk);   // Z^H Z_w
    {
      ProfScope ps_(ctx, HW_PH_EIG);
      e = launch_oa_correction(st, w->B3, w->B2, n, nb, nk, w->w, w->B1);
      ctx->launches++;
    }
    if (e != cudaSuccess) return e;
    gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, n, 1.0, w->Z, n, sZ, w->B1, n, sB, 0.0, w->B2, n, sB, nk);   // Z E
    cudaMemcpy2DAsync(w->Z, (size_t)sZ * 16, w->B2, (size_t)sB * 16, (size_t)sB * 16, nk, cudaMemcpyDeviceToDevice, st);
  }
  // orthonormalise the wanted block (two Newton-Schulz steps)
  for (int pass = 0; pass < 2; ++pass) {
    gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, n, 1.0, w->Z, n, sZ, w->Z, n, sZ, 0.0, w->G, nb, (int64_t)nb * nb, nk);
    {
      ProfScope ps_(ctx, HW_PH_EIG);
      launch_dep(st, k_ns_coef, dim3(8, nk), 256, 0, w->G, nb, w->Ui);
      ctx->launches++;
    }
    gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, nb, 1.0, w->Z, n, sZ, w->Ui, nb, (int64_t)nb * nb, 0.0, w->B2, n, sB, nk);
    cudaMemcpy2DAsync(w->Z, (size_t)sZ * 16, w->B2, (size_t)sB * 16, (size_t)sB * 16, nk, cudaMemcpyDeviceToDevice, st);
  }
  gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, n, 1.0, w->A, n, sZ, w->Z, n, sZ, 0.0, w->B1, n, sB, nk);
  gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, n, 1.0, w->Z, n, sZ, w->B1, n, sB, 0.0, w->G, nb, (int64_t)nb * nb, nk);
  {
    ProfScope ps_(ctx, HW_PH_EIG);
    // exact rotations inside groups of near-degenerate vectors: Ug in B3, eigenvalues (unsorted)
    // in B2 viewed as doubles
    e = launch_group_rr(st, w->G, nb, nk, w->grp, reinterpret_cast<double*>(w->B2), n, w->B3);
    ctx->launches += 2;
  }
  if (e != cudaSuccess) return e;
  // S' = Ug^H S_w Ug, then U = Ug (I + F) with F the first-order rotation between groups
  const int64_t s2 = (int64_t)nb * nb;
  gemm(CUBLAS_OP_N, CUBLAS_OP_N, nb, nb, nb, 1.0, w->G, nb, s2, w->B3, nb, s2, 0.0, w->C, nb, (int64_t)2 * nb * nb, nk);
  gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, nb, 1.0, w->B3, nb, s2, w->C, nb, (int64_t)2 * nb * nb, 0.0, w->G, nb, s2, nk);
  {
    ProfScope ps_(ctx, HW_PH_EIG);
    e = launch_first_order(st, w->G, nb, nk, w->grp, w->Ui);
    ctx->launches++;
  }
  if (e != cudaSuccess) return e;
  gemm(CUBLAS_OP_N, CUBLAS_OP_N, nb, nb, nb, 1.0, w->B3, nb, s2, w->Ui, nb, s2, 0.0, w->C, nb, s2, nk);   // contiguous
  {
    ProfScope ps_(ctx, HW_PH_EIG);
    e = launch_sort_wanted(st, reinterpret_cast<double*>(w->B2), n, w->C, nb, nk, w->w, w->Ui);
    ctx->launches++;
  }
  if (e != cudaSuccess) return e;
  gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, nb, 1.0, w->Z, n, sZ, w->Ui, nb, (int64_t)nb * nb, 0.0, w->B2, n, sB, nk);
  cudaMemcpy2DAsync(w->Z, (size_t)sZ * 16, w->B2, (size_t)sB * 16, (size_t)sB * 16, nk, cudaMemcpyDeviceToDevice, st);
  return cudaGetLastError();
}

static cudaError_t rr_eig(hw_ctx* ctx, LobpcgWork* w, Gemm& gemm, int n, int nb, bool fp32, bool lite = false) {
  cudaStream_t st = ctx->stream;
  const int nk = w->nk;
  cudaError_t e;
  if (ctx->rr_method == 0 && w->hh && hh_smem(n) <= 226 * 1024) {
    // the Householder route is checked (orthonormal wanted block, finite eigenvalues); a
    // problem that fails the check is solved again by the FP64 Jacobi from a saved copy
    cudaMemcpyAsync(w->Abak, w->A, (size_t)nk * n * n * 16, cudaMemcpyDeviceToDevice, st);
    e = rr_eig_hh(ctx, w, gemm, n, nb, lite);
    if (e != cudaSuccess) return e;
    gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, n, 1.0, w->Z, n, (int64_t)n * n, w->Z, n, (int64_t)n * n, 0.0, w->G, nb,
         (int64_t)nb * nb, nk);
    {
      ProfScope ps_(ctx, HW_PH_EIG);
      // FP64 route: orthonormal to 1e-9; FP32-product phase: to 1e-5
      launch_dep(st, k_check_gram, nk, 256, 0, w->G, nb, w->w, n, lite ? 1e-5 : 1e-9, w->fail);
      ctx->launches++;
    }
    std::vector<int> f(nk);
    cudaMemcpyAsync(f.data(), w->fail, nk * sizeof(int), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    bool any = false;
    for (int b = 0; b < nk; ++b) any = any || f[b];
    if (!any) return cudaSuccess;
    ctx->rr_fallbacks++;
    cudaMemcpyAsync(w->A, w->Abak, (size_t)nk * n * n * 16, cudaMemcpyDeviceToDevice, st);
  }
  if (fp32 && w->j32 && jac32_smem(n) <= 226 * 1024) {
    {
      ProfScope ps_(ctx, HW_PH_EIG);
      dense_hermitize(st, w->A, n, nk);
      e = dense_heev32(st, w->A, n, nk, w->w, w->Z, w->j32, w->j32_bytes, J32_SWEEPS);
      ctx->launches += 4;
    }
    if (e != cudaSuccess) return e;
    const int64_t sZ = (int64_t)n * n;
    for (int pass = 0; pass < 2; ++pass) {
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, n, 1.0, w->Z, n, sZ, w->Z, n, sZ, 0.0, w->G, nb, (int64_t)nb * nb, nk);
      {
        ProfScope ps_(ctx, HW_PH_OTHER);
        launch_dep(st, k_ns_coef, dim3(8, nk), 256, 0, w->G, nb, w->Ui);
        ctx->launches++;
      }
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, nb, 1.0, w->Z, n, sZ, w->Ui, nb, (int64_t)nb * nb, 0.0, w->Y2, n,
           (int64_t)n * nb, nk);
      // each k-point's n x nb block back into the first nb columns of its n x n Z
      cudaMemcpy2DAsync(w->Z, (size_t)n * n * 16, w->Y2, (size_t)n * nb * 16, (size_t)n * nb * 16, nk,
                        cudaMemcpyDeviceToDevice, st);
    }
    gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, nb, n, 1.0, w->A, n, sZ, w->Z, n, sZ, 0.0, w->Y2, n, (int64_t)n * nb, nk);
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_rq_diag, dim3(nb, nk), 256, 0, w->Z, w->Y2, n, sZ, (int64_t)n * nb, w->w, n);
      ctx->launches++;
    }
    return cudaGetLastError();
  }
  {
    ProfScope ps_(ctx, HW_PH_EIG);
    dense_hermitize(st, w->A, n, nk);
    e = dense_heev(w->dw, st, w->A, n, nk, w->w, w->Z, w->status, 1e-14);
    ctx->launches += 4;
  }
  return e;
}

// apply H to `ncol` columns of S at column offset c0, result at the same offset of HS; or, with
// `step` (per k-point scalars) and dst, the fused recurrence step
//   S[:, dst ..] = al (H S[:, c0 ..] - c S[:, c0 ..]) - be S[:, dst ..]
static hw_status apply_block(hw_ctx* ctx, LobpcgWork* w, const std::vector<int>& kidx, double2* S, double2* HS,
                             int c0, int ncol, bool fp64, const std::vector<int>* only = nullptr,
                             const ChebStep* step = nullptr, int dst = 0) {
  if (ncol <= 0) return HW_OK;
  const int64_t sK = w->Lpad * 3 * w->nb;
  Blocks blk;
  blk.nslot = 0;
  ChebStep cs;
  for (int b = 0; b < w->nk; ++b) {
    if (only && !(*only)[b]) continue;
    blk.x[blk.nslot] = reinterpret_cast<const double*>(S + (size_t)b * sK + (size_t)c0 * w->Lpad);
    blk.y[blk.nslot] = step ? reinterpret_cast<double*>(S + (size_t)b * sK + (size_t)dst * w->Lpad)
                            : reinterpret_cast<double*>(HS + (size_t)b * sK + (size_t)c0 * w->Lpad);
    blk.kb[blk.nslot] = kidx[b];
    if (step) {
      cs.al[blk.nslot] = step->al[b];
      cs.c[blk.nslot] = step->c[b];
      cs.be[blk.nslot] = step->be[b];
    }
    ++blk.nslot;
  }
  if (blk.nslot == 0) return HW_OK;
  const ChebStep* sp = step ? &cs : nullptr;
  ctx->ff_now = fp64 && ctx->ff_solve;   // a mixed solve's FP64 H X: double-float angular transforms
  cudaError_t e = fp64 ? launch_hx<double>(ctx, blk, ncol, w->Lpad, sp) : launch_hx<float>(ctx, blk, ncol, w->Lpad, sp);
  ctx->ff_now = false;
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("apply_H: ") + cudaGetErrorString(e));
  return HW_OK;
}

static hw_status ensure_work(hw_ctx* ctx, int nk, int nb, int64_t Lpad) {
  LobpcgWork* w = ctx->lw;
  if (w && w->nk == nk && w->nb == nb && w->Lpad == Lpad) return HW_OK;
  lobpcg_free(ctx);
  w = new LobpcgWork();
  ctx->lw = w;
  w->nk = nk;
  w->nb = nb;
  w->Lpad = Lpad;
  w->ne = 3 * nb + ((3 * nb) & 1);
  const size_t sK = (size_t)Lpad * 3 * nb;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) e = cudaMemset(*p, 0, std::max<size_t>(bytes, 16));
  };
  for (int i = 0; i < 2; ++i) {
    A((void**)&w->SB[i], nk * sK * sizeof(double2));
    A((void**)&w->HSB[i], nk * sK * sizeof(double2));
  }
  A((void**)&w->R, (size_t)nk * Lpad * nb * sizeof(double2));
  const size_t ne2 = (size_t)w->ne * w->ne;
  A((void**)&w->A, nk * ne2 * sizeof(double2));
  A((void**)&w->Z, nk * ne2 * sizeof(double2));
  A((void**)&w->w, (size_t)nk * w->ne * sizeof(double));
  A((void**)&w->G, (size_t)nk * nb * nb * sizeof(double2));
  A((void**)&w->Ui, (size_t)nk * nb * nb * sizeof(double2));
  A((void**)&w->C, (size_t)nk * 2 * nb * nb * sizeof(double2));
  A((void**)&w->Y, (size_t)nk * w->ne * nb * sizeof(double2));
  A((void**)&w->Y2, (size_t)nk * w->ne * nb * sizeof(double2));
  A((void**)&w->res, (size_t)nk * nb * sizeof(double));
  A((void**)&w->theta, (size_t)nk * nb * sizeof(double));
  A((void**)&w->iact, (size_t)nk * nb * sizeof(int));
  A((void**)&w->fail, (size_t)nk * sizeof(int));
  A((void**)&w->status, sizeof(int));
  if (e == cudaSuccess) e = dense_alloc(w->dw, nk * ne2, nk);
  w->gbytes = gram_work_bytes(w->ne, w->ne, (int)Lpad, nk);
  A(&w->gwork, w->gbytes);
  // the Householder route wherever one of the Rayleigh-Ritz sizes fits a CTA's shared memory
  // (nb: a filter cycle's; 2 nb: [X W]; 3 nb: [X W P]); rr_eig checks the size of each call,
  // so a block whose 3 nb does not fit (above 78 columns) still takes it for the smaller ones
  if (e == cudaSuccess && hh_smem(nb) <= 226 * 1024) {
    w->hh_bytes = hh_scratch_bytes(w->ne, w->ne, nk);
    e = cudaMalloc(&w->hh, w->hh_bytes);
    A((void**)&w->B1, (size_t)nk * w->ne * nb * sizeof(double2));
    A((void**)&w->B2, (size_t)nk * w->ne * nb * sizeof(double2));
    A((void**)&w->B3, (size_t)nk * w->ne * nb * sizeof(double2));
    A((void**)&w->grp, (size_t)nk * nb * sizeof(int));
    A((void**)&w->Abak, nk * ne2 * sizeof(double2));
  }
  if (e == cudaSuccess && jac32_smem(w->ne) <= 226 * 1024) {
    w->j32_bytes = heev32_scratch_bytes(w->ne, nk, J32_SWEEPS);
    e = cudaMalloc(&w->j32, w->j32_bytes);
  }
  if (e != cudaSuccess) {
    lobpcg_free(ctx);
    return hw_fail(ctx, HW_ENOMEM, std::string("eigensolver workspace: ") + cudaGetErrorString(e));
  }
  return HW_OK;
}

}  // namespace hw

using namespace hw;

namespace {
// Training-data recorder of hw_solve_eigs_traced (single k-point).
struct Trace {
  int n_rec;
  const int* rec_iters;
  double* rec_R;       // device [n_rec][nb][ld]
  double* rec_E;       // device [n_rec][nb][ld]: the recorded X block until the end, then E
  double* rec_theta;   // host [n_rec][nb]
  double* rec_res;     // host [n_rec][nb]
  int64_t ld;
  std::vector<char> got;
};
}  // namespace

// Rayleigh-Ritz on the nb columns of column block q of SB[from] (H times them in the same
// block of HSB[from]): the Ritz vectors and their H products go to block 0 of SB[to] /
// HSB[to] (to != from), the Ritz values to w->theta.  dnv: the device count array (its P and
// W counts are zeroed).
static hw_status rr_subspace(hw_ctx* ctx, LobpcgWork* w, Gemm& gemm, int* dnv, int from, int q, int to) {
  const int nk = w->nk, nb = w->nb;
  const int64_t Lpad = w->Lpad, sK = Lpad * 3 * nb;
  cudaStream_t st = ctx->stream;
  const int n = nb + (nb & 1);
  const double2* Y = w->SB[from] + (size_t)q * nb * Lpad;
  const double2* HY = w->HSB[from] + (size_t)q * nb * Lpad;
  gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, (int)Lpad, 1.0, Y, Lpad, sK, HY, Lpad, sK, 0.0, w->A, n, (int64_t)n * n,
       nk);
  std::vector<int> z(nk, 0);
  cudaMemcpyAsync(dnv + nk, z.data(), nk * sizeof(int), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dnv + 2 * nk, z.data(), nk * sizeof(int), cudaMemcpyHostToDevice, st);
  {
    ProfScope ps_(ctx, HW_PH_OTHER);
    launch_dep(st, k_pad_rr, dim3(8, nk), 256, 0, w->A, n, nb, 0, 0, dnv + nk, dnv + 2 * nk);
    ctx->launches++;
  }
  cudaError_t e = rr_eig(ctx, w, gemm, n, nb, false, gemm.lowp);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("eigensolver: ") + cudaGetErrorString(e));
  gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, nb, nb, 1.0, Y, Lpad, sK, w->Z, n, (int64_t)n * n, 0.0, w->SB[to],
       Lpad, sK, nk);
  gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, nb, nb, 1.0, HY, Lpad, sK, w->Z, n, (int64_t)n * n, 0.0, w->HSB[to],
       Lpad, sK, nk);
  for (int b = 0; b < nk; ++b)
    cudaMemcpyAsync(w->theta + (size_t)b * nb, w->w + (size_t)b * n, nb * sizeof(double), cudaMemcpyDeviceToDevice, st);
  return HW_OK;
}

// Arguments and buffers shared by the block eigensolvers.
struct SolveSetup {
  std::vector<int> kidx;
  std::vector<int64_t> Lb;   // basis size of each k-point
  int nb = 0;
  int64_t Lpad = 0, sK = 0;
  int64_t* dL = nullptr;     // device copy of Lb
  int* dnv = nullptr;        // device [3][nk]: valid column counts (CholQR / P / W)
  ~SolveSetup() {
    cudaFree(dL);
    cudaFree(dnv);
  }
};

// Validate the arguments common to the eigensolvers, size the workspace, point `gemm` at the
// FP32 product buffers of the mixed form, and copy the per-k-point sizes to the device.
static hw_status solve_setup(hw_ctx* ctx, int nk, const int* kidx_in, int n_eig, int block, double tol,
                             int maxit, hw_prec prec, const double* evals, const double* const* evecs,
                             int64_t ld_evecs, SolveSetup& su, Gemm& gemm, bool cheb = false) {
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (!ctx->have_basis) return hw_fail(ctx, HW_ESTATE, "hw_setup_basis has not been called");
  if (!ctx->have_V) return hw_fail(ctx, HW_ESTATE, "no potential installed");
  if (nk < 1 || nk > MAXSLOT || !kidx_in || !evals) return hw_fail(ctx, HW_EINVAL, "bad k-point list");
  if (n_eig < 1 || !(tol > 0) || maxit < 1) return hw_fail(ctx, HW_EINVAL, "bad n_eig / tol / maxit");
  if (prec != HW_FP64 && prec != HW_MIXED) return hw_fail(ctx, HW_EINVAL, "bad precision");
  su.kidx.assign(kidx_in, kidx_in + nk);
  int64_t Lmax = 0, Lmin = INT64_MAX;
  for (int b = 0; b < nk; ++b) {
    if (su.kidx[b] < 0 || su.kidx[b] >= ctx->hb.nk) return hw_fail(ctx, HW_EINVAL, "k-point index out of range");
    Lmax = std::max(Lmax, ctx->hb.L[su.kidx[b]]);
    Lmin = std::min(Lmin, ctx->hb.L[su.kidx[b]]);
  }
  // default buffer: LOBPCG n_eig / 8 (at least 4); the Chebyshev solver 3 n_eig / 16 (at least 8),
  // the wider buffer speeding up the filter on the columns near the top of the wanted set
  // (measured on the tube, 64 eigenpairs over 24 start blocks: block 76 against 72, 32.1 against
  // 34.6 ms per chosen-form solve; 74 and 78 slower than both)
  const int nb = block > 0 ? block : n_eig + (cheb ? std::max(8, 3 * n_eig / 16) : std::max(4, n_eig / 8));
  if (nb < n_eig) return hw_fail(ctx, HW_EINVAL, "block < n_eig");
  if (nb > 112) return hw_fail(ctx, HW_EINVAL, "block > 112");
  if (3 * (int64_t)nb > Lmin) return hw_fail(ctx, HW_EINVAL, "block too large for the basis (3*block > L)");
  if (evecs && ld_evecs < Lmax) return hw_fail(ctx, HW_EINVAL, "ld_evecs < L");
  su.nb = nb;
  su.Lpad = (Lmax + 7) / 8 * 8;
  su.sK = su.Lpad * 3 * nb;
  const int64_t Lpad = su.Lpad;
  cudaSetDevice(ctx->device);
  hw_status hs = ensure_work(ctx, nk, nb, Lpad);
  if (hs != HW_OK) return hs;
  LobpcgWork* w = ctx->lw;
  // mixed form: products over the basis dimension in complex FP32 until the residuals fall
  // below 10^-lowp_exp, then FP64
  if (prec == HW_MIXED && ctx->lowp_exp > 0) {
    const size_t ab = (size_t)nk * Lpad * 3 * nb;
    const size_t cc = std::max((size_t)nk * Lpad * 2 * nb, (size_t)nk * w->ne * w->ne);
    if (w->f32_ab < ab || w->f32_c < cc) {
      for (auto& p : w->F32) {
        if (p) cudaFree(p);
        p = nullptr;
      }
      cudaError_t e0 = cudaMalloc((void**)&w->F32[0], ab * sizeof(float2));
      if (e0 == cudaSuccess) e0 = cudaMalloc((void**)&w->F32[1], ab * sizeof(float2));
      if (e0 == cudaSuccess) e0 = cudaMalloc((void**)&w->F32[2], cc * sizeof(float2));
      if (e0 != cudaSuccess) {
        for (auto& p : w->F32) {
          if (p) cudaFree(p);
          p = nullptr;
        }
        w->f32_ab = w->f32_c = 0;
        return hw_fail(ctx, HW_ENOMEM, "FP32 product buffers");
      }
      w->f32_ab = ab;
      w->f32_c = cc;
    }
    gemm.a32 = w->F32[0];
    gemm.b32 = w->F32[1];
    gemm.c32 = w->F32[2];
    gemm.cap_ab = w->f32_ab;
    gemm.cap_c = w->f32_c;
    gemm.lowp = true;
  }
  if (prec == HW_MIXED && ctx->gram_mixed) {
    gemm.gram = true;
    gemm.gwork = w->gwork;
    gemm.gbytes = w->gbytes;
  }
  su.Lb.resize(nk);
  for (int b = 0; b < nk; ++b) su.Lb[b] = ctx->hb.L[su.kidx[b]];
  if (cudaMalloc((void**)&su.dL, nk * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc((void**)&su.dnv, 3 * nk * sizeof(int)) != cudaSuccess)
    return hw_fail(ctx, HW_ENOMEM, "eigensolver size arrays");
  cudaMemcpy(su.dL, su.Lb.data(), nk * sizeof(int64_t), cudaMemcpyHostToDevice);
  cudaMemsetAsync(w->status, 0, sizeof(int), ctx->stream);
  return HW_OK;
}

// Deflation of a windowed solve: the eigenvectors the earlier windows converged (per k-point
// at Q[b], leading dimension ld, the first nq columns), against which a window's start block and
// new search directions are projected.
struct Deflate {
  int nq = 0;
  const double2* Q[MAXSLOT] = {};
  int64_t ld = 0;
  double2* C = nullptr;   // scratch: nq x (at most 112) coefficients
};

// columns c0 .. c0 + ncol - 1 of every k-point's block in S (rows Lb[b], leading dimension
// Lpad, k-point stride sK) minus their components along Q[b]: X -= Q (Q^H X), twice, in FP64,
// or (fp32) with complex FP32 products, which round the columns to FP32 as well: for search
// directions only, whose FP32-level traces along Q enter the Ritz vectors scaled by their
// coefficients (of the order of the residuals)
static void deflate_cols(Gemm& gemm, const Deflate* df, const std::vector<int64_t>& Lb, double2* S, int64_t Lpad,
                         int64_t sK, int c0, int ncol, bool fp32 = false) {
  if (!df || df->nq == 0 || ncol <= 0) return;
  const bool keep = gemm.lowp;
  gemm.lowp = fp32;
  for (int pass = 0; pass < 2; ++pass)
    for (size_t b = 0; b < Lb.size(); ++b) {
      double2* X = S + (size_t)b * sK + (size_t)c0 * Lpad;
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, df->nq, ncol, (int)Lb[b], 1.0, df->Q[b], df->ld, 0, X, Lpad, 0, 0.0, df->C,
           df->nq, 0, 1);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lb[b], ncol, df->nq, -1.0, df->Q[b], df->ld, 0, df->C, df->nq, 0, 1.0, X,
           Lpad, 0, 1);
    }
  gemm.lowp = keep;
}

// Start block in the first nb columns of SB[0]: the caller's X0 (L_b x nb, ld L_b, zero padded),
// a seeded complex Gaussian block, or (keep) the block already there; projected against the
// deflation set (if any); then Cholesky-QR twice.
static hw_status start_block(hw_ctx* ctx, SolveSetup& su, Gemm& gemm, const double* const* X0, bool keep = false,
                             const Deflate* df = nullptr) {
  LobpcgWork* w = ctx->lw;
  const int nk = w->nk, nb = su.nb;
  cudaStream_t st = ctx->stream;
  if (keep) {
    // the caller filled SB[0]
  } else if (X0) {
    PtrArr pa;
    for (int b = 0; b < nk; ++b) {
      if (!X0[b]) return hw_fail(ctx, HW_EINVAL, "null start block");
      pa.p[b] = X0[b];
    }
    ProfScope ps_(ctx, HW_PH_OTHER);
    launch_dep(st, k_copy_start, dim3(nb, nk), 256, 0, pa, w->SB[0], su.Lpad, su.sK, su.dL);
    ctx->launches++;
  } else {
    ProfScope ps_(ctx, HW_PH_OTHER);
    launch_dep(st, k_random_start, dim3(nb, nk), 256, 0, w->SB[0], su.Lpad, su.sK, su.dL, nb, 0x5eed1234abcdULL);
    ctx->launches++;
  }
  deflate_cols(gemm, df, su.Lb, w->SB[0], su.Lpad, su.sK, 0, nb);
  std::vector<int> nvh(3 * nk, nb);
  cudaMemcpy(su.dnv, nvh.data(), 3 * nk * sizeof(int), cudaMemcpyHostToDevice);
  std::vector<int> failed;
  hw_status hs = cholqr(ctx, w, gemm, w->SB[0], 0, nb, su.dnv, 2, failed);
  if (hs != HW_OK) return hs;
  for (int b = 0; b < nk; ++b)
    if (failed[b]) return hw_fail(ctx, HW_EINVAL, "start block is rank deficient");
  return HW_OK;
}

static hw_status solve_impl(hw_ctx* ctx, int nk, const int* kidx_in, int n_eig, int block,
                            double tol, int maxit, hw_prec prec, int precond_kind,
                            const double* const* X0, double* evals, double* const* evecs,
                            int64_t ld_evecs, int* iters, double* resid, Trace* trace,
                            bool keep_start = false, bool no_p = false, const Deflate* df = nullptr,
                            double tol_accept = 0.0) {
  if (!ctx) return HW_EINVAL;
  if (precond_kind != HW_PRECOND_TPA && precond_kind != HW_PRECOND_NONE &&
      !(precond_kind == HW_PRECOND_LEARNED && ctx->mlp))
    return hw_fail(ctx, HW_EINVAL, "bad preconditioner kind (learned needs hw_set_mlp)");
  Gemm gemm{ctx};
  SolveSetup su;
  hw_status hs = solve_setup(ctx, nk, kidx_in, n_eig, block, tol, maxit, prec, evals, evecs, ld_evecs, su, gemm);
  if (hs != HW_OK) return hs;
  const std::vector<int>& kidx = su.kidx;
  const std::vector<int64_t>& Lb = su.Lb;
  const int nb = su.nb;
  const int64_t Lpad = su.Lpad, sK = su.sK;
  int* dnv = su.dnv;
  LobpcgWork* w = ctx->lw;
  cudaStream_t st = ctx->stream;
  const double lowp_thr = (prec == HW_MIXED && ctx->lowp_exp > 0) ? std::pow(10.0, -ctx->lowp_exp) : 0.0;
  std::vector<int> failed;
  int cur = 0;
  hs = start_block(ctx, su, gemm, X0, keep_start, df);
  if (hs != HW_OK) return hs;
  const bool mixed = prec == HW_MIXED;
  bool fp64_products = !mixed;
  hs = apply_block(ctx, w, kidx, w->SB[0], w->HSB[0], 0, nb, fp64_products);
  if (hs != HW_OK) return hs;
  // Rayleigh-Ritz on X alone: SB[from] -> SB[1 - from]
  auto rr_on_x = [&](int from) -> hw_status {
    const hw_status h = rr_subspace(ctx, w, gemm, dnv, from, 0, 1 - from);
    if (h == HW_OK) cur = 1 - from;
    return h;
  };
  hs = rr_on_x(0);
  if (hs != HW_OK) return hs;
  int np = 0;                                  // P block width (uniform)
  std::vector<int> npv(nk, 0);                 // valid P columns per k-point
  std::vector<char> done(nk, 0);
  std::vector<int> it_done(nk, maxit);
  std::vector<double> resh((size_t)nk * nb), thh((size_t)nk * nb);
  bool refreshed = !mixed;
  double lowp_best = 1e300;
  int lowp_best_it = 0;
  bool hyb_on = ctx->hybrid != 0;
  double hyb_best = 1e300;
  int hyb_best_it = 0;
  int it = 0;
  // no_p: start without conjugate directions; they are switched on for good once an iteration
  // fails to halve the largest wanted residual
  bool p_off = no_p;
  double p_prev = 1e300;
  int p_it = -1;
  double acc_best = 1e300;   // best largest residual since the FP32 phase (tol_accept)
  int acc_best_it = 0;
  hw_status final_status = HW_ENOTCONV;
  for (it = 0; it <= maxit; ++it) {
    double2* S = w->SB[cur];
    double2* HS = w->HSB[cur];
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_residual, dim3(nb, nk), 256, 0, S, HS, Lpad, sK, w->theta, nb, w->R, w->res);
      ctx->launches++;
    }
    cudaMemcpyAsync(resh.data(), w->res, resh.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(thh.data(), w->theta, thh.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    int dstat = 0, zstat = 0;
    cudaMemcpyAsync(&dstat, w->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ctx->zg) cudaMemcpyAsync(&zstat, zgemm_status_ptr(ctx->zg), sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("eigensolver: ") + cudaGetErrorString(e));
    if (dstat == HW_ETIMEOUT) return hw_fail(ctx, HW_ETIMEOUT, "dense eigensolver barrier timed out");
    if (zstat == HW_ETIMEOUT) {
      zgemm_status(ctx->zg, st, true);
      return hw_fail(ctx, HW_ETIMEOUT, "a wait in the tensor-core block product timed out");
    }
    if (gemm.st != CUBLAS_STATUS_SUCCESS) return hw_fail(ctx, HW_ECUDA, "cuBLAS failure");
    if (gemm.ce != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("Gram kernel: ") + cudaGetErrorString(gemm.ce));
    if (trace) {
      for (int r = 0; r < trace->n_rec; ++r) {
        if (trace->rec_iters[r] != it || trace->got[r]) continue;
        trace->got[r] = 1;
        const size_t nbytes = (size_t)Lb[0] * 16;
        cudaMemcpy2DAsync(trace->rec_R + 2 * (size_t)r * nb * trace->ld, trace->ld * 16, w->R, Lpad * 16, nbytes,
                          nb, cudaMemcpyDeviceToDevice, st);
        cudaMemcpy2DAsync(trace->rec_E + 2 * (size_t)r * nb * trace->ld, trace->ld * 16, S, Lpad * 16, nbytes, nb,
                          cudaMemcpyDeviceToDevice, st);
        for (int j = 0; j < nb; ++j) {
          trace->rec_theta[(size_t)r * nb + j] = thh[j];
          trace->rec_res[(size_t)r * nb + j] = resh[j];
        }
      }
    }
    // mixed: refresh HX in FP64 once the residuals are small, and before accepting convergence
    // tol_accept > tol (a window of a windowed solve): tol is the target, and once the largest
    // residual has stopped falling (past the FP32 phase, no 30% drop in 8 iterations: the
    // precision's floor) a k-point whose residuals are at most tol_accept is accepted
    const double thr = (tol_accept > tol && !gemm.lowp && it - acc_best_it >= 8) ? tol_accept : tol;
    double maxres = 0.0;
    std::vector<int> claim(nk, 0);
    int nclaim = 0;
    for (int b = 0; b < nk; ++b) {
      if (done[b]) continue;
      double mr = 0.0;
      for (int j = 0; j < n_eig; ++j) mr = std::max(mr, resh[(size_t)b * nb + j]);
      maxres = std::max(maxres, mr);
      hist_push(ctx, kidx[b], gemm.lowp ? HW_HIST_LOBPCG_FP32 : (mixed && hyb_on ? HW_HIST_LOBPCG_HYBRID
                                                                                   : HW_HIST_LOBPCG_FP64), mr);
      if (mr <= thr) {
        claim[b] = 1;
        ++nclaim;
      }
    }
    if (gemm.lowp || maxres < 0.7 * acc_best) {
      acc_best = maxres;
      acc_best_it = it;
    }
    // FP32 products stall near residual 1e-5: leave them also when the best residual has not
    // dropped by 30% in 4 iterations
    if (gemm.lowp) {
      if (maxres < 0.7 * lowp_best) {
        lowp_best = maxres;
        lowp_best_it = it;
      }
    }
    // the hybrid FP64 phase stalls near residual 3e-7: it hands over to all-FP64 products when
    // the best residual has not dropped by 30% in 4 iterations
    if (p_off) {   // (a repeated check of the same iteration, after a precision switch, only updates)
      if (it > p_it && p_it >= 0 && maxres > 0.5 * p_prev) p_off = false;
      p_prev = maxres;
      p_it = it;
    }
    bool hyb_stall = false;
    if (mixed && !gemm.lowp && hyb_on) {
      if (maxres < 0.7 * hyb_best) {
        hyb_best = maxres;
        hyb_best_it = it;
      } else if (it - hyb_best_it >= 4 && nclaim == 0) {
        hyb_on = false;
        hyb_stall = true;
      }
    }
    if (hyb_stall || (gemm.lowp && (maxres < lowp_thr || nclaim > 0 || it - lowp_best_it >= 4))) {
      // leave the FP32 (or hybrid) products: X re-orthonormalised and its H X recomputed in
      // FP64; the conjugate directions P kept, orthogonalised against the new X and
      // orthonormalised in FP64 (H P transformed alongside); a Rayleigh-Ritz step on X alone;
      // then this iteration starts over from the residuals (no step is lost)
      gemm.lowp = false;
      hyb_best = 1e300;
      hyb_best_it = it;
      std::vector<int> nbv(nk, nb);
      cudaMemcpyAsync(dnv, nbv.data(), nk * sizeof(int), cudaMemcpyHostToDevice, st);
      deflate_cols(gemm, df, Lb, S, Lpad, sK, 0, nb);   // FP32 rounding leaves traces along Q
      bool ns_ok = false;
      hs = ns_orth(ctx, w, gemm, S, 0, nb, 2, ns_ok);
      if (hs == HW_OK && !ns_ok) hs = cholqr(ctx, w, gemm, S, 0, nb, dnv, 2, failed);
      if (hs != HW_OK) return hs;
      hs = apply_block(ctx, w, kidx, S, HS, 0, nb, true);
      if (hs != HW_OK) return hs;
      if (np > 0) {
        double2* P = S + (size_t)nb * Lpad;
        double2* HP = HS + (size_t)nb * Lpad;
        gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, np, (int)Lpad, 1.0, S, Lpad, sK, P, Lpad, sK, 0.0, w->C, nb,
             (int64_t)2 * nb * nb, nk);
        gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, np, nb, -1.0, S, Lpad, sK, w->C, nb, (int64_t)2 * nb * nb, 1.0, P,
             Lpad, sK, nk);
        gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, np, nb, -1.0, HS, Lpad, sK, w->C, nb, (int64_t)2 * nb * nb, 1.0,
             HP, Lpad, sK, nk);
        cudaMemcpyAsync(dnv, npv.data(), nk * sizeof(int), cudaMemcpyHostToDevice, st);
        gemm(CUBLAS_OP_C, CUBLAS_OP_N, np, np, (int)Lpad, 1.0, P, Lpad, sK, P, Lpad, sK, 0.0, w->G, np,
             (int64_t)np * np, nk);
        {
          ProfScope ps_(ctx, HW_PH_OTHER);
          launch_dep(st, k_pad_gram, dim3(8, nk), 256, 0, w->G, np, dnv);
          ctx->launches++;
        }
        {
          ProfScope ps_(ctx, HW_PH_CHOL, nk * ((8.0 / 3.0) * np * (double)np * np + 8.0 * (double)Lpad * np * np));
          dense_hermitize(st, w->G, np, nk);
          dense_chol(st, w->G, np, nk, w->fail, false);
          cudaError_t te = dense_trsm_lh(st, w->G, np, nk, P, Lpad, Lpad, sK, false, w->fail);
          if (te == cudaSuccess) te = dense_trsm_lh(st, w->G, np, nk, HP, Lpad, Lpad, sK, false, w->fail);
          if (te != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("P at the switch: ") + cudaGetErrorString(te));
          ctx->launches += 4;
        }
        std::vector<int> f(nk);
        cudaMemcpyAsync(f.data(), w->fail, nk * sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        bool pf = false;
        for (int b = 0; b < nk; ++b) pf = pf || (f[b] && npv[b] > 0);
        if (pf) {
          np = 0;   // P not usable: restart the conjugate directions
          std::fill(npv.begin(), npv.end(), 0);
        }
      }
      hs = rr_on_x(cur);   // X, H X into the other buffer
      if (hs != HW_OK) return hs;
      if (np > 0) {         // P, H P follow them
        const int from = 1 - cur;
        cudaMemcpy2DAsync(w->SB[cur] + (size_t)nb * Lpad, (size_t)sK * 16, w->SB[from] + (size_t)nb * Lpad,
                          (size_t)sK * 16, (size_t)Lpad * np * 16, nk, cudaMemcpyDeviceToDevice, st);
        cudaMemcpy2DAsync(w->HSB[cur] + (size_t)nb * Lpad, (size_t)sK * 16, w->HSB[from] + (size_t)nb * Lpad,
                          (size_t)sK * 16, (size_t)Lpad * np * 16, nk, cudaMemcpyDeviceToDevice, st);
      }
      refreshed = true;
      --it;   // the same iteration, from the residuals of the new X
      continue;
    }
    if (mixed && ((!refreshed && maxres < 1e-3) || nclaim > 0)) {
      std::vector<int> which(nk, 0);
      for (int b = 0; b < nk; ++b) which[b] = !done[b] && (!refreshed || claim[b]);
      hs = apply_block(ctx, w, kidx, S, HS, 0, nb, true, &which);
      if (hs != HW_OK) return hs;
      refreshed = true;
      {
        ProfScope ps_(ctx, HW_PH_OTHER);
        launch_dep(st, k_residual, dim3(nb, nk), 256, 0, S, HS, Lpad, sK, w->theta, nb, w->R, w->res);
        ctx->launches++;
      }
      cudaMemcpyAsync(resh.data(), w->res, resh.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("eigensolver: ") + cudaGetErrorString(e));
      for (int b = 0; b < nk; ++b) {
        claim[b] = 0;
        if (done[b]) continue;
        double mr = 0.0;
        for (int j = 0; j < n_eig; ++j) mr = std::max(mr, resh[(size_t)b * nb + j]);
        claim[b] = mr <= thr;
      }
    } else if (!mixed) {
      // FP64 products: residuals are already exact
    }
    for (int b = 0; b < nk; ++b) {
      if (done[b] || !claim[b]) continue;
      done[b] = 1;
      it_done[b] = it;
      for (int j = 0; j < n_eig; ++j) {
        evals[(size_t)b * n_eig + j] = thh[(size_t)b * nb + j];
        if (resid) resid[(size_t)b * n_eig + j] = resh[(size_t)b * nb + j];
      }
      if (evecs && evecs[b])
        cudaMemcpy2DAsync(evecs[b], ld_evecs * 16, S + (size_t)b * sK, Lpad * 16, Lb[b] * 16, n_eig,
                          cudaMemcpyDeviceToDevice, st);
    }
    bool all = true;
    for (int b = 0; b < nk; ++b) all = all && done[b];
    if (all) {
      final_status = HW_OK;
      break;
    }
    if (it == maxit) break;
    // ---- active sets (soft locking)
    std::vector<int> act((size_t)nk * nb, -1);
    std::vector<int> nav(nk, 0);
    int na = 0;
    for (int b = 0; b < nk; ++b) {
      if (done[b]) continue;
      for (int j = 0; j < nb; ++j)
        if (resh[(size_t)b * nb + j] > tol) act[(size_t)b * nb + nav[b]++] = j;
      na = std::max(na, nav[b]);
    }
    if (na == 0) na = 1;  // converged residuals but claim not verified yet: keep one direction
    cudaMemcpyAsync(w->iact, act.data(), act.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    std::vector<int> nvall(3 * nk);
    for (int b = 0; b < nk; ++b) {
      nvall[b] = nav[b];
      nvall[nk + b] = npv[b];
      nvall[2 * nk + b] = nav[b];
    }
    cudaMemcpyAsync(dnv, nvall.data(), 3 * nk * sizeof(int), cudaMemcpyHostToDevice, st);
    const int woff = nb + np;
    // ---- W = K R[:, act]
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_gather_w, dim3(na, nk), 256, 0, w->R, nb, Lpad, w->iact, na, S, sK, woff);
      ctx->launches++;
    }
    {
      Blocks blk;
      blk.nslot = nk;
      for (int b = 0; b < nk; ++b) {
        blk.x[b] = reinterpret_cast<const double*>(S + (size_t)b * sK + (size_t)woff * Lpad);
        blk.y[b] = reinterpret_cast<double*>(S + (size_t)b * sK + (size_t)woff * Lpad);
        blk.kb[b] = kidx[b];
      }
      if (precond_kind == HW_PRECOND_TPA) {
        e = launch_tpa(ctx, blk, na, Lpad);
      } else if (precond_kind == HW_PRECOND_LEARNED) {
        // Ritz value of each W column: theta of its source column
        std::vector<double> rz((size_t)nk * na, 0.0);
        for (int b = 0; b < nk; ++b)
          for (int i = 0; i < nav[b]; ++i) rz[(size_t)b * na + i] = thh[(size_t)b * nb + act[(size_t)b * nb + i]];
        cudaMemcpyAsync(w->C, rz.data(), rz.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        std::vector<const double*> rp(nk);
        for (int b = 0; b < nk; ++b) rp[b] = reinterpret_cast<const double*>(w->C) + (size_t)b * na;
        e = launch_precond_learned(ctx, blk, na, Lpad, rp.data());
        cudaStreamSynchronize(st);
      } else {
        e = cudaSuccess;
      }
      if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("precond: ") + cudaGetErrorString(e));
    }
    // FP64 phase of the mixed form ("hybrid"): only the products that involve X stay FP64 (its
    // rows of the Rayleigh-Ritz matrix, its share of the X / H X update, and one projection of
    // W and of P against X, which keeps the basis orthonormal to FP64 accuracy where it
    // matters).  W and P enter the Ritz vectors with weights of the order of the residuals, so
    // their mutual orthogonalisation, their Gram block and the P update are formed in FP32.
    const bool hyb = mixed && !gemm.lowp && hyb_on;
    const bool lowp_now = gemm.lowp;
    deflate_cols(gemm, df, Lb, S, Lpad, sK, woff, na, lowp_now || hyb);   // W against the earlier windows
    gemm.lowp = lowp_now || hyb;
    // ---- project out [X P], twice
    for (int pass = 0; pass < 2; ++pass) {
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb + np, na, (int)Lpad, 1.0, S, Lpad, sK, S + (size_t)woff * Lpad, Lpad, sK,
           0.0, w->C, nb + np, (int64_t)2 * nb * nb, nk);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, na, nb + np, -1.0, S, Lpad, sK, w->C, nb + np,
           (int64_t)2 * nb * nb, 1.0, S + (size_t)woff * Lpad, Lpad, sK, nk);
    }
    // ---- Cholesky-QR of W (twice)
    hs = cholqr(ctx, w, gemm, S, woff, na, dnv, 2, failed);
    gemm.lowp = lowp_now;
    if (hs != HW_OK) return hs;
    if (hyb) {
      // W orthogonal to X to FP64 accuracy: one FP64 projection pass against X alone
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, na, (int)Lpad, 1.0, S, Lpad, sK, S + (size_t)woff * Lpad, Lpad, sK, 0.0,
           w->C, nb, (int64_t)2 * nb * nb, nk);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, na, nb, -1.0, S, Lpad, sK, w->C, nb, (int64_t)2 * nb * nb, 1.0,
           S + (size_t)woff * Lpad, Lpad, sK, nk);
    }
    bool anyfail = false;
    for (int b = 0; b < nk; ++b)
      if (failed[b] && nav[b] > 0) {
        anyfail = true;
        nav[b] = 0;   // drop this k-point's search directions for this iteration
      }
    if (anyfail) {
      for (int b = 0; b < nk; ++b) nvall[2 * nk + b] = nav[b];
      for (int b = 0; b < nk; ++b)
        if (nav[b] == 0)
          cudaMemsetAsync(S + (size_t)b * sK + (size_t)woff * Lpad, 0, (size_t)Lpad * na * sizeof(double2), st);
      cudaMemcpyAsync(dnv, nvall.data(), 3 * nk * sizeof(int), cudaMemcpyHostToDevice, st);
    }
    // ---- HW
    hs = apply_block(ctx, w, kidx, S, HS, woff, na, fp64_products);
    if (hs != HW_OK) return hs;
    // ---- Rayleigh-Ritz on S = [X P W]
    const int nS = nb + np + na;
    const int n = nS + (nS & 1);
    if (hyb && nS > nb) {
      // X rows in FP64, the [P W] block in FP32, the lower-left blocks mirrored
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nS, (int)Lpad, 1.0, S, Lpad, sK, HS, Lpad, sK, 0.0, w->A, n, (int64_t)n * n,
           nk);
      gemm.lowp = true;
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nS - nb, nS - nb, (int)Lpad, 1.0, S + (size_t)nb * Lpad, Lpad, sK,
           HS + (size_t)nb * Lpad, Lpad, sK, 0.0, w->A + nb + (size_t)nb * n, n, (int64_t)n * n, nk);
      gemm.lowp = false;
      {
        ProfScope ps_(ctx, HW_PH_OTHER);
        launch_dep(st, k_mirror_xrows, dim3(8, nk), 256, 0, w->A, n, nb, nS);
        ctx->launches++;
      }
    } else {
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nS, nS, (int)Lpad, 1.0, S, Lpad, sK, HS, Lpad, sK, 0.0, w->A, n, (int64_t)n * n,
           nk);
    }
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_pad_rr, dim3(8, nk), 256, 0, w->A, n, nb, np, na, dnv + nk, dnv + 2 * nk);
      ctx->launches++;
    }
    e = rr_eig(ctx, w, gemm, n, nb, maxres > FP32_RR_ABOVE, gemm.lowp);
    if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("eigensolver: ") + cudaGetErrorString(e));
    const int nxt = 1 - cur;
    double2* S2 = w->SB[nxt];
    double2* HS2 = w->HSB[nxt];
    // the P basis in the small space: FP32 in the hybrid phase as well
    gemm.lowp = lowp_now || hyb;
    for (int b = 0; b < nk; ++b)
      cudaMemcpyAsync(w->theta + (size_t)b * nb, w->w + (size_t)b * n, nb * sizeof(double), cudaMemcpyDeviceToDevice, st);
    bool pfail = p_off;   // p_off: no conjugate directions this iteration (subspace [X W])
    if (!p_off) {
    // ---- P = S Y (active columns), Y orthogonal to Z[:, :nb] and orthonormal
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_build_y, dim3(na, nk), 128, 0, w->Z, n, nb, w->iact, na, w->Y);
      ctx->launches++;
    }
    for (int pass = 0; pass < 2; ++pass) {
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, na, n, 1.0, w->Z, n, (int64_t)n * n, w->Y, n, (int64_t)n * na, 0.0, w->C, nb,
           (int64_t)2 * nb * nb, nk);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, n, na, nb, -1.0, w->Z, n, (int64_t)n * n, w->C, nb, (int64_t)2 * nb * nb, 1.0,
           w->Y, n, (int64_t)n * na, nk);
    }
    // small-space Cholesky-QR of Y (FP32 factor in the FP32-product phase, FP64 retry)
    for (int pass = 0; pass < 2; ++pass) {
      for (int attempt = gemm.lowp ? 0 : 1; attempt < 2; ++attempt) {
        const bool fp32 = attempt == 0;
        const bool keep = gemm.lowp;
        gemm.lowp = fp32;
        gemm(CUBLAS_OP_C, CUBLAS_OP_N, na, na, n, 1.0, w->Y, n, (int64_t)n * na, w->Y, n, (int64_t)n * na, 0.0, w->G,
             na, (int64_t)na * na, nk);
        gemm.lowp = keep;
        {
          ProfScope ps_(ctx, HW_PH_OTHER);
          launch_dep(st, k_pad_gram, dim3(8, nk), 256, 0, w->G, na, dnv + 2 * nk);
          ctx->launches++;
        }
        {
          ProfScope ps_(ctx, HW_PH_CHOL, nk * ((8.0 / 3.0) * na * (double)na * na + 4.0 * (double)n * na * na));
          dense_hermitize(st, w->G, na, nk);
          dense_chol(st, w->G, na, nk, w->fail, fp32);
          const cudaError_t te = dense_trsm_lh(st, w->G, na, nk, w->Y, n, n, (int64_t)n * na, fp32, w->fail);
          if (te != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("P basis: ") + cudaGetErrorString(te));
          ctx->launches += 3;
        }
        std::vector<int> f(nk);
        cudaMemcpyAsync(f.data(), w->fail, nk * sizeof(int), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        bool anyf = false;
        for (int b = 0; b < nk; ++b) anyf = anyf || (f[b] && nav[b] > 0);
        if (!anyf) break;
        if (!fp32) pfail = true;
      }
    }
    }
    if (pfail) {
      np = 0;   // restart the conjugate directions everywhere
      std::fill(npv.begin(), npv.end(), 0);
    } else {
      np = na;
      npv = nav;
    }
    gemm.lowp = lowp_now;
    // ---- block updates [X P]_new = S [Z_w Y], [HX HP]_new = HS [Z_w Y] (Y copied next to Z_w)
    const int ncols = nb + (pfail ? 0 : na);
    if (!pfail && na > 0)
      cudaMemcpy2DAsync(w->Z + (size_t)nb * n, (size_t)n * n * 16, w->Y, (size_t)n * na * 16, (size_t)n * na * 16, nk,
                        cudaMemcpyDeviceToDevice, st);
    if (hyb && nS > nb) {
      // [P W] rows of the coefficients in FP32, X rows in FP64 (accumulated in FP64)
      gemm.lowp = true;
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, ncols, nS - nb, 1.0, S + (size_t)nb * Lpad, Lpad, sK, w->Z + nb, n,
           (int64_t)n * n, 0.0, S2, Lpad, sK, nk);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, ncols, nS - nb, 1.0, HS + (size_t)nb * Lpad, Lpad, sK, w->Z + nb,
           n, (int64_t)n * n, 0.0, HS2, Lpad, sK, nk);
      gemm.lowp = false;
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, ncols, nb, 1.0, S, Lpad, sK, w->Z, n, (int64_t)n * n, 1.0, S2, Lpad,
           sK, nk);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, ncols, nb, 1.0, HS, Lpad, sK, w->Z, n, (int64_t)n * n, 1.0, HS2,
           Lpad, sK, nk);
      if (!pfail && na > 0) {
        // P orthogonal to the new X to FP64 accuracy (H P corrected alongside)
        gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, na, (int)Lpad, 1.0, S2, Lpad, sK, S2 + (size_t)nb * Lpad, Lpad, sK, 0.0,
             w->C, nb, (int64_t)2 * nb * nb, nk);
        gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, na, nb, -1.0, S2, Lpad, sK, w->C, nb, (int64_t)2 * nb * nb, 1.0,
             S2 + (size_t)nb * Lpad, Lpad, sK, nk);
        gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, na, nb, -1.0, HS2, Lpad, sK, w->C, nb, (int64_t)2 * nb * nb, 1.0,
             HS2 + (size_t)nb * Lpad, Lpad, sK, nk);
      }
    } else {
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, ncols, nS, 1.0, S, Lpad, sK, w->Z, n, (int64_t)n * n, 0.0, S2, Lpad,
           sK, nk);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, ncols, nS, 1.0, HS, Lpad, sK, w->Z, n, (int64_t)n * n, 0.0, HS2,
           Lpad, sK, nk);
    }
    gemm.lowp = lowp_now;
    cur = nxt;
  }
  // k-points that never converged: report the last Ritz values
  for (int b = 0; b < nk; ++b) {
    if (!done[b]) {
      for (int j = 0; j < n_eig; ++j) {
        evals[(size_t)b * n_eig + j] = thh[(size_t)b * nb + j];
        if (resid) resid[(size_t)b * n_eig + j] = resh[(size_t)b * nb + j];
      }
      if (evecs && evecs[b])
        cudaMemcpy2DAsync(evecs[b], ld_evecs * 16, w->SB[cur] + (size_t)b * sK, Lpad * 16, Lb[b] * 16, n_eig,
                          cudaMemcpyDeviceToDevice, st);
    }
    if (iters) iters[b] = it_done[b];
  }
  if (trace && final_status == HW_OK) {
    // e_j = (I - X X^H) X* X*^H x_j with X* the converged n_eig vectors (first columns of S)
    const double2* Xs = w->SB[cur];
    const int64_t ld = trace->ld;
    for (int r = 0; r < trace->n_rec; ++r) {
      if (!trace->got[r]) continue;
      double2* Xr = reinterpret_cast<double2*>(trace->rec_E) + (size_t)r * nb * ld;
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, n_eig, nb, (int)Lb[0], 1.0, Xs, Lpad, sK, Xr, ld, 0, 0.0, w->C, n_eig, 0, 1);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lb[0], nb, n_eig, 1.0, Xs, Lpad, sK, w->C, n_eig, 0, 0.0, w->R, Lpad, 0, 1);
      gemm(CUBLAS_OP_C, CUBLAS_OP_N, nb, nb, (int)Lb[0], 1.0, Xr, ld, 0, w->R, Lpad, 0, 0.0, w->C, nb, 0, 1);
      gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lb[0], nb, nb, -1.0, Xr, ld, 0, w->C, nb, 0, 1.0, w->R, Lpad, 0, 1);
      cudaMemcpy2DAsync(Xr, ld * 16, w->R, Lpad * 16, (size_t)Lb[0] * 16, nb, cudaMemcpyDeviceToDevice, st);
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("eigensolver: ") + cudaGetErrorString(e));
  if (gemm.st != CUBLAS_STATUS_SUCCESS) return hw_fail(ctx, HW_ECUDA, "cuBLAS failure");
  if (final_status != HW_OK) return hw_fail(ctx, HW_ENOTCONV, "maxit reached before convergence");
  return HW_OK;
}

// Chebyshev-filtered subspace iteration (the alternative eigensolver the paper leaves to future
// work, Sec. "Eigensolvers and Preconditioning"; the filter is the scaled three-term Chebyshev
// recurrence of Zhou and Saad's filtered subspace iteration).  Per cycle and k-point, with Ritz
// values theta_0 <= ... <= theta_{nb-1} of the current block X:
//   damped interval [a, b]: a = theta_{nb-1}, b = an upper bound of the spectrum,
//   e = (b - a)/2, c = (b + a)/2, sigma_1 = e/(theta_0 - c), tau = 2/sigma_1,
//   Y_0 = X, Y_1 = (sigma_1/e)(H X - c X),
//   Y_i = (2 sigma_i/e)(H Y_{i-1} - c Y_{i-1}) - sigma_{i-1} sigma_i Y_{i-2},
//     sigma_i = 1/(tau - sigma_{i-1}),  i = 2 .. m,
// so that p_m(theta_0) = 1 and the wanted end of the spectrum is amplified relative to [a, b];
// then the columns of Y_m are normalised, orthonormalised (Cholesky-QR twice), multiplied by H,
// and a Rayleigh-Ritz step on them gives the next X.  H X of the current X comes from the
// Rayleigh-Ritz step, so a cycle costs m products H Y.
// Upper bound: b = max KE + max V (+ the largest positive 1/r^2 term for nu != 0): H is the
// diagonal KE plus B^H W diag(V) B (an orthogonal projection of V, so bounded by max V) plus
// the nu terms, bounded by their coefficient times the row-sum norm of the I_n table.
// Mixed form: the filter's H products, the Gram matrices and the Rayleigh-Ritz products are
// FP32 until the residuals fall below 10^-lowp_exp (or stop falling); then LOBPCG's mixed form
// (with the given preconditioner; by default without conjugate directions, HW_OPT_TAIL_NO_P)
// finishes from the filtered Ritz block.  FP64 form: filter cycles to the end.
static hw_status chfsi_impl(hw_ctx* ctx, int nk, const int* kidx_in, int n_eig, int block, double tol, int maxit,
                            hw_prec prec, int precond_kind, const double* const* X0, double* evals,
                            double* const* evecs, int64_t ld_evecs, int* iters, double* resid,
                            const Deflate* df = nullptr, double tol_accept = 0.0) {
  if (!ctx) return HW_EINVAL;
  Gemm gemm{ctx};
  SolveSetup su;
  // the filter converges the top wanted columns at the rate of the gap to the first unwanted
  // one: a default buffer of at least 8 columns (measured on the Ncyc = 3 tube, 32 eigenpairs:
  // block 36 1.71 s, block 40 0.50 s)
  hw_status hs = solve_setup(ctx, nk, kidx_in, n_eig, block, tol, maxit, prec, evals, evecs, ld_evecs, su, gemm, true);
  if (hs != HW_OK) return hs;
  const std::vector<int>& kidx = su.kidx;
  const int nb = su.nb, mmax = ctx->cheb_degree;
  const int64_t Lpad = su.Lpad, sK = su.sK;
  int* dnv = su.dnv;
  LobpcgWork* w = ctx->lw;
  cudaStream_t st = ctx->stream;
  const bool mixed = prec == HW_MIXED;
  const double lowp_thr = (mixed && ctx->lowp_exp > 0) ? std::pow(10.0, -ctx->lowp_exp) : 0.0;
  // ---- upper bounds of the spectra
  double vmax = 0.0;
  {
    const auto& pr = ctx->hb.prm;
    const int64_t grid = (int64_t)pr.Nth1 * pr.Nth2 * pr.Nr;
    ProfScope ps_(ctx, HW_PH_OTHER);
    launch_dep(st, k_vmax, 1, 1024, 0, ctx->db.t64.V, grid, w->res);
    ctx->launches++;
    cudaMemcpyAsync(&vmax, w->res, sizeof(double), cudaMemcpyDeviceToHost, st);
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("spectral bound: ") + cudaGetErrorString(e));
  }
  std::vector<double> bup(nk);
  {
    const auto& hb = ctx->hb;
    const int K = hb.K;
    std::vector<double> qnorm(hb.N + 1, 0.0);   // row-sum norm of each |n| table
    for (int g = 0; g <= hb.N; ++g)
      for (int k = 0; k < K; ++k) {
        double r = 0.0;
        for (int kk = 0; kk < K; ++kk) r += std::fabs(hb.qtab[((size_t)g * K + k) * K + kk]);
        qnorm[g] = std::max(qnorm[g], r);
      }
    for (int b = 0; b < nk; ++b) {
      const auto& ke = hb.ke[kidx[b]];
      double kmax = -1e300;
      for (double v : ke) kmax = std::max(kmax, v);
      const double nu = hb.nu[kidx[b]];
      double extra = 0.0;
      if (nu != 0.0)
        for (int n = -hb.N; n <= hb.N; ++n)
          extra = std::max(extra, 0.5 * nu * (nu - 2.0 * n * hb.prm.ncyc) * qnorm[std::abs(n)]);
      const double bound = kmax + vmax + extra;
      bup[b] = bound + 1e-3 * std::fabs(bound) + 1e-3;
    }
  }
  hs = start_block(ctx, su, gemm, X0, false, df);
  if (hs != HW_OK) return hs;
  bool lowp = gemm.lowp;   // FP32 phase of the mixed form
  hs = apply_block(ctx, w, kidx, w->SB[0], w->HSB[0], 0, nb, !lowp);
  if (hs != HW_OK) return hs;
  hs = rr_subspace(ctx, w, gemm, dnv, 0, 0, 1);
  if (hs != HW_OK) return hs;
  int cur = 1;
  std::vector<char> done(nk, 0);
  std::vector<int> it_done(nk, maxit);
  std::vector<double> resh((size_t)nk * nb), thh((size_t)nk * nb);
  double lowp_best = 1e300, lowp_prev = 1e300;
  int lowp_best_it = 0;
  hw_status final_status = HW_ENOTCONV;
  std::vector<int> failed;
  int it = 0;
  for (it = 0; it <= maxit; ++it) {
    double2* S = w->SB[cur];
    double2* HS = w->HSB[cur];
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_residual, dim3(nb, nk), 256, 0, S, HS, Lpad, sK, w->theta, nb, w->R, w->res);
      ctx->launches++;
    }
    cudaMemcpyAsync(resh.data(), w->res, resh.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(thh.data(), w->theta, thh.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    int dstat = 0, zstat = 0;
    cudaMemcpyAsync(&dstat, w->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ctx->zg) cudaMemcpyAsync(&zstat, zgemm_status_ptr(ctx->zg), sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("eigensolver: ") + cudaGetErrorString(e));
    if (dstat == HW_ETIMEOUT) return hw_fail(ctx, HW_ETIMEOUT, "dense eigensolver barrier timed out");
    if (zstat == HW_ETIMEOUT) {
      zgemm_status(ctx->zg, st, true);
      return hw_fail(ctx, HW_ETIMEOUT, "a wait in the tensor-core block product timed out");
    }
    if (gemm.st != CUBLAS_STATUS_SUCCESS) return hw_fail(ctx, HW_ECUDA, "cuBLAS failure");
    if (gemm.ce != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("Gram kernel: ") + cudaGetErrorString(gemm.ce));
    double maxres = 0.0;
    std::vector<int> claim(nk, 0);
    int nclaim = 0;
    for (int b = 0; b < nk; ++b) {
      if (done[b]) continue;
      double mr = 0.0;
      for (int j = 0; j < n_eig; ++j) mr = std::max(mr, resh[(size_t)b * nb + j]);
      maxres = std::max(maxres, mr);
      hist_push(ctx, kidx[b], lowp ? HW_HIST_FILTER_FP32 : HW_HIST_FILTER_FP64, mr);
      if (mr <= tol) {
        claim[b] = 1;
        ++nclaim;
      }
    }
    if (lowp) {
      if (maxres < 0.7 * lowp_best) {
        lowp_best = maxres;
        lowp_best_it = it;
      }
      // a filter cycle shrinks the residuals by an order of magnitude or more until the FP32
      // rounding floor; less than a halving means the floor is reached
      const bool stalled = maxres > 0.5 * lowp_prev;
      lowp_prev = maxres;
      if (maxres < lowp_thr || nclaim > 0 || stalled || it - lowp_best_it >= 3) {
        // leave the FP32 phase.  A further filter cycle would need FP64 H products (FP32 noise
        // in a filtered block leaves residuals near ||H|| 1e-7); the end phase is handed to
        // LOBPCG's mixed form instead (its corrections tolerate FP32 H products and every claim
        // is an FP64 residual), started from the filtered Ritz block
        if (cur != 0)
          cudaMemcpy2DAsync(w->SB[0], (size_t)sK * 16, w->SB[cur], (size_t)sK * 16, (size_t)Lpad * nb * 16, nk,
                            cudaMemcpyDeviceToDevice, st);
        std::vector<int> itl(nk, 0);
        hs = solve_impl(ctx, nk, kidx_in, n_eig, nb, tol, std::max(1, maxit - it), prec, precond_kind, nullptr,
                        evals, evecs, ld_evecs, itl.data(), resid, nullptr, true, ctx->tail_no_p != 0, df,
                        tol_accept);
        if (iters)
          for (int b = 0; b < nk; ++b) iters[b] = it + itl[b];
        return hs;
      }
      nclaim = 0;
      std::fill(claim.begin(), claim.end(), 0);
    }
    for (int b = 0; b < nk; ++b) {
      if (done[b] || !claim[b]) continue;
      done[b] = 1;
      it_done[b] = it;
      for (int j = 0; j < n_eig; ++j) {
        evals[(size_t)b * n_eig + j] = thh[(size_t)b * nb + j];
        if (resid) resid[(size_t)b * n_eig + j] = resh[(size_t)b * nb + j];
      }
      if (evecs && evecs[b])
        cudaMemcpy2DAsync(evecs[b], ld_evecs * 16, S + (size_t)b * sK, Lpad * 16, su.Lb[b] * 16, n_eig,
                          cudaMemcpyDeviceToDevice, st);
    }
    bool all = true;
    for (int b = 0; b < nk; ++b) all = all && done[b];
    if (all) {
      final_status = HW_OK;
      break;
    }
    if (it == maxit) break;
    // ---- the filter: Y_m = p_m(H) X in the column blocks of S (block i mod 2 holds Y_i; the
    //      step writing Y_i reads Y_{i-2} from the same block, element by element)
    // (k-points already done are filtered along with the rest: their blocks stay well defined)
    ChebScal sc;
    std::vector<double> sig(nk), tau(nk), ee(nk);
    for (int b = 0; b < MAXSLOT; ++b) sc.al[b] = sc.c[b] = sc.be[b] = 0.0;
    for (int b = 0; b < nk; ++b) {
      const double a0 = thh[(size_t)b * nb], a = thh[(size_t)b * nb + nb - 1];
      double bb = bup[b];
      if (!(bb > a + 1e-8)) bb = a + std::max(1.0, std::fabs(a));   // bound below the block: widen
      ee[b] = 0.5 * (bb - a);
      sc.c[b] = 0.5 * (bb + a);
      double den = a0 - sc.c[b];
      if (!(den < -1e-12 * ee[b])) den = -ee[b];   // degenerate block (all Ritz values equal)
      sig[b] = ee[b] / den;
      tau[b] = 2.0 / sig[b];
      sc.al[b] = sig[b] / ee[b];
    }
    // degree of this cycle: the largest degree the option allows, or (adaptive, FP64 cycles)
    // the smallest that reduces every unconverged wanted residual to tol, taking one cycle to
    // shrink column j's error by the factor 1/T_m(|xi_j|), xi_j = (theta_j - c)/e (the filter's
    // gain on theta_j over the damped interval).  FP32 cycles keep the full degree: their phase
    // ends at a fixed residual anyway, and fewer products per cycle only add cycles there.
    int m = mmax;
    if (ctx->cheb_adapt && !lowp) {
      const double target = tol;
      int need = 2;
      for (int b = 0; b < nk; ++b) {
        if (done[b]) continue;
        for (int j = 0; j < n_eig; ++j) {
          const double rj = resh[(size_t)b * nb + j];
          if (rj <= 0.5 * target) continue;
          const double xi = std::fabs((thh[(size_t)b * nb + j] - sc.c[b]) / ee[b]);
          if (!(xi > 1.0 + 1e-9)) {
            need = mmax;
            continue;
          }
          need = std::max(need, (int)std::ceil(std::acosh(2.0 * rj / target) / std::acosh(xi)));
        }
      }
      m = std::max(2, std::min(mmax, need));
    }
    // soft locking: the leading Ritz columns whose residuals are already below half the
    // phase's target (1e-5 level in the FP32 phase, tol after it) are not filtered; they keep
    // their place (and H X) in the block and take part in the Rayleigh-Ritz step.  The count is
    // the smallest over the k-points still running (the batch filters one column range).
    int nl = n_eig;
    {
      const double lthr = 0.5 * (lowp ? std::max(lowp_thr, tol) : tol);
      for (int b = 0; b < nk; ++b) {
        if (done[b]) continue;
        int cnt = 0;
        while (cnt < n_eig && resh[(size_t)b * nb + cnt] <= lthr) ++cnt;
        nl = std::min(nl, cnt);
      }
      if (!ctx->cheb_lock) nl = 0;
    }
    const int na = nb - nl;   // filtered columns nl .. nb-1 (na >= nb - n_eig >= 1)
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_cheb, dim3(na, nk), 256, 0, S, HS, Lpad, sK, nb, 0, 1, nl, sc);
      ctx->launches++;
    }
    for (int i = 2; i <= m; ++i) {   // each step fused into the H Y launch
      const int src = (i - 1) % 2, dst = i % 2;
      ChebStep step;
      for (int b = 0; b < nk; ++b) {
        const double sn = 1.0 / (tau[b] - sig[b]);
        step.al[b] = 2.0 * sn / ee[b];
        step.c[b] = sc.c[b];
        step.be[b] = sig[b] * sn;
        sig[b] = sn;
      }
      hs = apply_block(ctx, w, kidx, S, HS, src * nb + nl, na, !lowp, nullptr, &step, dst * nb + nl);
      if (hs != HW_OK) return hs;
    }
    const int q = m % 2;
    {
      ProfScope ps_(ctx, HW_PH_OTHER);
      launch_dep(st, k_colnorm, dim3(na, nk), 256, 0, S, Lpad, sK, nb, q, nl);
      ctx->launches++;
    }
    double2* Yq = S + (size_t)q * nb * Lpad;    // the filtered block: [X_locked | Y_active]
    double2* HYq = HS + (size_t)q * nb * Lpad;
    // windowed solve: the filter amplifies the earlier windows' eigenvectors most (their
    // eigenvalues lie below the block's), so the traces of them that rounding leaves are
    // projected out before the orthonormalisation
    deflate_cols(gemm, df, su.Lb, S, Lpad, sK, q * nb + nl, na, lowp);
    if (nl > 0) {
      if (q != 0) {   // the locked columns and their H products live in block 0
        cudaMemcpy2DAsync(Yq, (size_t)sK * 16, S, (size_t)sK * 16, (size_t)nl * Lpad * 16, nk,
                          cudaMemcpyDeviceToDevice, st);
        cudaMemcpy2DAsync(HYq, (size_t)sK * 16, HS, (size_t)sK * 16, (size_t)nl * Lpad * 16, nk,
                          cudaMemcpyDeviceToDevice, st);
      }
      // the active columns orthogonal to the locked ones (twice)
      for (int pass = 0; pass < 2; ++pass) {
        gemm(CUBLAS_OP_C, CUBLAS_OP_N, nl, na, (int)Lpad, 1.0, Yq, Lpad, sK, Yq + (size_t)nl * Lpad, Lpad, sK,
             0.0, w->C, nl, (int64_t)2 * nb * nb, nk);
        gemm(CUBLAS_OP_N, CUBLAS_OP_N, (int)Lpad, na, nl, -1.0, Yq, Lpad, sK, w->C, nl, (int64_t)2 * nb * nb,
             1.0, Yq + (size_t)nl * Lpad, Lpad, sK, nk);
      }
    }
    std::vector<int> nav(nk, na);
    cudaMemcpyAsync(dnv, nav.data(), nk * sizeof(int), cudaMemcpyHostToDevice, st);
    hs = cholqr(ctx, w, gemm, S, q * nb + nl, na, dnv, 2, failed);
    if (hs != HW_OK) return hs;
    for (int b = 0; b < nk; ++b)
      if (failed[b] && !done[b])
        return hw_fail(ctx, HW_ENOTCONV, "Chebyshev filter: the filtered block lost rank (lower the degree)");
    hs = apply_block(ctx, w, kidx, S, HS, q * nb + nl, na, !lowp);
    if (hs != HW_OK) return hs;
    hs = rr_subspace(ctx, w, gemm, dnv, cur, q, 1 - cur);
    if (hs != HW_OK) return hs;
    cur = 1 - cur;
  }
  for (int b = 0; b < nk; ++b) {
    if (!done[b]) {
      for (int j = 0; j < n_eig; ++j) {
        evals[(size_t)b * n_eig + j] = thh[(size_t)b * nb + j];
        if (resid) resid[(size_t)b * n_eig + j] = resh[(size_t)b * nb + j];
      }
      if (evecs && evecs[b])
        cudaMemcpy2DAsync(evecs[b], ld_evecs * 16, w->SB[cur] + (size_t)b * sK, Lpad * 16, su.Lb[b] * 16, n_eig,
                          cudaMemcpyDeviceToDevice, st);
    }
    if (iters) iters[b] = it_done[b];
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("eigensolver: ") + cudaGetErrorString(e));
  if (gemm.st != CUBLAS_STATUS_SUCCESS) return hw_fail(ctx, HW_ECUDA, "cuBLAS failure");
  if (final_status != HW_OK) return hw_fail(ctx, HW_ENOTCONV, "maxit reached before convergence");
  return HW_OK;
}

extern "C" hw_status hw_gram(hw_ctx* ctx, int m, int n, int K, int nprob, const double* A, int64_t lda, int64_t sA,
                              const double* B, int64_t ldb, int64_t sB, double* C, int64_t ldc, int64_t sC) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (m < 1 || n < 1 || m > 512 || n > 512 || K < 1 || nprob < 1 || nprob > MAXSLOT || !A || !B || !C ||
      lda < K || ldb < K || ldc < m)
    return hw_fail(ctx, HW_EINVAL, "hw_gram: bad sizes");
  cudaSetDevice(ctx->device);
  const size_t need = gram_work_bytes(m, n, K, nprob);
  void* work = nullptr;
  if (cudaMalloc(&work, need) != cudaSuccess) return hw_fail(ctx, HW_ENOMEM, "hw_gram workspace");
  int nl = 0;
  cudaError_t e = gram_cf(ctx->stream, m, n, K, 1.0, reinterpret_cast<const double2*>(A), lda, sA,
                          reinterpret_cast<const double2*>(B), ldb, sB, 0.0, reinterpret_cast<double2*>(C), ldc, sC,
                          nprob, work, need, &nl);
  ctx->launches += nl;
  const cudaError_t e2 = cudaStreamSynchronize(ctx->stream);
  cudaFree(work);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("hw_gram: ") + cudaGetErrorString(e));
  return HW_OK;
}

extern "C" hw_status hw_heev(hw_ctx* ctx, int n, int nprob, int nw, const double* A, double* w, double* Z,
                              int method) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (n < 2 || (n & 1) || nprob < 1 || nprob > MAXSLOT || nw < 1 || nw > n || !A || !w || !Z)
    return hw_fail(ctx, HW_EINVAL, "need even n >= 2, 1 <= nprob <= 64, 1 <= nw <= n");
  if (method != 0 && method != 1) return hw_fail(ctx, HW_EINVAL, "method 0 (Jacobi) or 1 (Householder)");
  const int nbw = std::max(nw, (n + 2) / 3);
  if (3 * nbw + ((3 * nbw) & 1) < n) return hw_fail(ctx, HW_EINVAL, "size");
  cudaSetDevice(ctx->device);
  hw_status hs = ensure_work(ctx, nprob, nbw, 8);
  if (hs != HW_OK) return hs;
  LobpcgWork* wk = ctx->lw;
  if (method == 1 && !(wk->hh && hh_smem(n) <= 226 * 1024))
    return hw_fail(ctx, HW_EINVAL, "n too large for the Householder route (shared-memory bound)");
  cudaStream_t st = ctx->stream;
  cudaMemcpyAsync(wk->A, A, (size_t)nprob * n * n * 16, cudaMemcpyDeviceToDevice, st);
  Gemm gemm{ctx};
  cudaError_t e;
  if (method == 1) {
    e = rr_eig_hh(ctx, wk, gemm, n, nw, false);
  } else {
    ProfScope ps_(ctx, HW_PH_EIG);
    dense_hermitize(st, wk->A, n, nprob);
    e = dense_heev(wk->dw, st, wk->A, n, nprob, wk->w, wk->Z, wk->status, 1e-14);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(w, wk->w, (size_t)nprob * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Z, wk->Z, (size_t)nprob * n * n * 16, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("heev: ") + cudaGetErrorString(e));
  if (gemm.st != CUBLAS_STATUS_SUCCESS) return hw_fail(ctx, HW_ECUDA, "cuBLAS failure in heev");
  return HW_OK;
}

// complex64 factors in the first n*n*8 bytes of each n*n*16-byte slot -> complex128 in dst
__global__ void k_factor_c64_to_c128(const double2* slots, double2* dst, int n) {
  griddep_entry();
  const float2* f = reinterpret_cast<const float2*>(slots + (size_t)blockIdx.y * n * n);
  double2* d = dst + (size_t)blockIdx.y * n * n;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n * n; t += gridDim.x * blockDim.x)
    d[t] = make_double2((double)f[t].x, (double)f[t].y);
}

extern "C" hw_status hw_cholesky(hw_ctx* ctx, int n, int nprob, double* G, double* L, int* fail, hw_prec prec) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (n < 1 || nprob < 1 || nprob > MAXSLOT || !G || !L || !fail || G == L)
    return hw_fail(ctx, HW_EINVAL, "need n >= 1, 1 <= nprob <= 64, distinct G and L, a fail array");
  if (prec != HW_FP64 && prec != HW_MIXED) return hw_fail(ctx, HW_EINVAL, "precision HW_FP64 or HW_MIXED");
  if (prec == HW_MIXED && (size_t)n * n * sizeof(float2) > 200 * 1024)
    return hw_fail(ctx, HW_EINVAL, "n too large for the FP32 factorisation (shared-memory bound, n <= 160)");
  cudaSetDevice(ctx->device);
  hw_status hs = ensure_work(ctx, nprob, 4, 8);
  if (hs != HW_OK) return hs;
  cudaStream_t st = ctx->stream;
  const size_t bytes = (size_t)nprob * n * n * sizeof(double2);
  double2* g = reinterpret_cast<double2*>(G);
  double2* l = reinterpret_cast<double2*>(L);
  cudaError_t e = cudaMemcpyAsync(l, g, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    ProfScope ps_(ctx, HW_PH_CHOL);
    e = dense_chol(st, l, n, nprob, ctx->lw->fail, prec == HW_MIXED);
    ctx->launches++;
  }
  if (e == cudaSuccess && prec == HW_MIXED) {   // the FP32 factor, widened through G
    launch_dep(st, k_factor_c64_to_c128, dim3(16, nprob), 256, 0, l, g, n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(l, g, bytes, cudaMemcpyDeviceToDevice, st);
    ctx->launches++;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(fail, ctx->lw->fail, (size_t)nprob * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("cholesky: ") + cudaGetErrorString(e));
  return HW_OK;
}

extern "C" hw_status hw_selftest_barrier(hw_ctx* ctx, int nblocks, long long spin_limit, int skip_block,
                                         int* wait_status) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  int nsm = 0;
  cudaSetDevice(ctx->device);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (nblocks < 2 || nblocks > nsm || spin_limit < 1 || spin_limit > (1LL << 24) || skip_block < -1 ||
      skip_block >= nblocks || !wait_status)
    return hw_fail(ctx, HW_EINVAL, "need 2 <= nblocks <= SM count, 1 <= spin_limit <= 2^24, -1 <= skip_block < nblocks");
  int ws = -1;
  const cudaError_t e = dense_barrier_selftest(ctx->stream, nblocks, (long)spin_limit, skip_block, &ws);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("barrier self-test: ") + cudaGetErrorString(e));
  *wait_status = ws;
  return HW_OK;
}

extern "C" hw_status hw_get_residual_history(hw_ctx* ctx, int k, int* phase, double* res, int max_n, int* n_out) {
  if (!ctx || !n_out) return HW_EINVAL;
  size_t slot = 0;
  while (slot < ctx->hist_k.size() && ctx->hist_k[slot] != k) ++slot;
  if (slot == ctx->hist_k.size()) {
    *n_out = 0;
    return HW_OK;
  }
  const int n = (int)ctx->hist_res[slot].size();
  *n_out = n;
  for (int i = 0; i < std::min(n, max_n); ++i) {
    if (phase) phase[i] = ctx->hist_phase[slot][i];
    if (res) res[i] = ctx->hist_res[slot][i];
  }
  return HW_OK;
}

// marks a mixed-precision solve: its FP64 H X takes the double-float angular kernel
// (HW_OPT_FP64_HX) and its small FP64-class products the double-float kernel (HW_OPT_SMALL_GEMM)
struct FfSolveScope {
  hw_ctx* c;
  FfSolveScope(hw_ctx* ctx, hw_prec prec) : c(ctx) {
    c->ff_solve = prec == HW_MIXED && c->fp64_hx_ff;
    c->mixed_solve = prec == HW_MIXED;
  }
  ~FfSolveScope() { c->ff_solve = c->mixed_solve = false; }
};

static hw_status solve_window(hw_ctx* ctx, int nk, const int* kidx, int n_eig, int block, double tol, int maxit,
                              hw_prec prec, int precond_kind, const double* const* X0, double* evals,
                              double* const* evecs, int64_t ld_evecs, int* iters, double* resid, const Deflate* df,
                              double tol_accept = 0.0) {
  FfSolveScope ffs(ctx, prec);
  if (ctx->eigensolver == 1)
    return chfsi_impl(ctx, nk, kidx, n_eig, block, tol, maxit, prec, precond_kind, X0, evals, evecs, ld_evecs, iters,
                      resid, df, tol_accept);
  return solve_impl(ctx, nk, kidx, n_eig, block, tol, maxit, prec, precond_kind, X0, evals, evecs, ld_evecs,
                    iters, resid, nullptr, false, false, df, tol_accept);
}

extern "C" hw_status hw_solve_eigs(hw_ctx* ctx, int nk, const int* kidx, int n_eig, int block, double tol,
                                   int maxit, hw_prec prec, int precond_kind, const double* const* X0,
                                   double* evals, double* const* evecs, int64_t ld_evecs, int* iters,
                                   double* resid) {
  if (!ctx) return HW_EINVAL;
  ctx->hist_k.clear();
  ctx->hist_phase.clear();
  ctx->hist_res.clear();
  const int wmax = ctx->window > 0 ? ctx->window : 80;
  if (n_eig <= wmax)
    return solve_window(ctx, nk, kidx, n_eig, block, tol, maxit, prec, precond_kind, X0, evals, evecs, ld_evecs,
                        iters, resid, nullptr);
  // windows of equal size, each solved in the complement of the ones before
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (!ctx->have_basis) return hw_fail(ctx, HW_ESTATE, "hw_setup_basis has not been called");
  if (nk < 1 || nk > MAXSLOT || !kidx || !evals) return hw_fail(ctx, HW_EINVAL, "bad k-point list");
  if (X0) return hw_fail(ctx, HW_EINVAL, "a windowed solve takes no start block (X0 must be NULL)");
  int64_t Lmax = 0, Lmin = INT64_MAX;
  for (int b = 0; b < nk; ++b) {
    if (kidx[b] < 0 || kidx[b] >= ctx->hb.nk) return hw_fail(ctx, HW_EINVAL, "k-point index out of range");
    Lmax = std::max(Lmax, ctx->hb.L[kidx[b]]);
    Lmin = std::min(Lmin, ctx->hb.L[kidx[b]]);
  }
  if (evecs) {
    if (ld_evecs < Lmax) return hw_fail(ctx, HW_EINVAL, "ld_evecs < L");
    for (int b = 0; b < nk; ++b)
      if (!evecs[b]) return hw_fail(ctx, HW_EINVAL, "null eigenvector block");
  }
  const int nwin = (n_eig + wmax - 1) / wmax;
  const int wsz = (n_eig + nwin - 1) / nwin;
  cudaSetDevice(ctx->device);
  // the converged vectors: the caller's evecs, or a scratch block when the caller wants none
  const int64_t ldq = evecs ? ld_evecs : Lmax;
  double2* own = nullptr;
  if (!evecs && cudaMalloc((void**)&own, (size_t)nk * ldq * n_eig * sizeof(double2)) != cudaSuccess)
    return hw_fail(ctx, HW_ENOMEM, "windowed solve: eigenvector scratch");
  Deflate df;
  df.ld = ldq;
  if (cudaMalloc((void**)&df.C, (size_t)n_eig * 112 * sizeof(double2)) != cudaSuccess) {
    cudaFree(own);
    return hw_fail(ctx, HW_ENOMEM, "windowed solve: projection scratch");
  }
  std::vector<double2*> Qp(nk);
  for (int b = 0; b < nk; ++b) {
    Qp[b] = evecs ? reinterpret_cast<double2*>(evecs[b]) : own + (size_t)b * ldq * n_eig;
    df.Q[b] = Qp[b];
  }
  std::vector<double> ev((size_t)nk * wsz), rs((size_t)nk * wsz);
  std::vector<int> itw(nk, 0);
  for (size_t i = 0; i < (size_t)nk * n_eig; ++i) {
    evals[i] = std::nan("");
    if (resid) resid[i] = std::nan("");
  }
  if (iters)
    for (int b = 0; b < nk; ++b) iters[b] = 0;
  hw_status result = HW_OK;
  for (int w0 = 0; w0 < n_eig; w0 += wsz) {
    const int nw = std::min(wsz, n_eig - w0);
    df.nq = w0;
    std::vector<double*> out(nk);
    for (int b = 0; b < nk; ++b) out[b] = reinterpret_cast<double*>(Qp[b] + (size_t)w0 * ldq);
    // default block: a wide buffer (the top columns of a window converge at the rate of the gap
    // to the first column outside the block), at most 112 columns and what the basis allows
    int bw = block;
    if (bw <= 0) {
      bw = (int)std::min<int64_t>(std::min(112, nw + std::max(32, nw / 2)), Lmin / 3);
      if (bw < nw) bw = 0;   // the solver's own default (and its error if that does not fit)
    }
    // a locked eigenvector's residual r_i is orthogonal to its own window's block and points
    // mostly at the first eigenvectors beyond it, which later windows solve for in the
    // complement of the locked set: an eigenvector y there keeps the true residual
    // ||R^H y|| whatever the window does.  Windows before the last therefore aim at tol / 2,
    // which keeps that floor below tol; where the precision's own floor stops them above it
    // (the mixed form's FP32 products), they are accepted at tol.
    const bool last = w0 + nw >= n_eig;
    const double tw = last ? tol : std::max(0.5 * tol, std::min(tol, 1e-11));
    const hw_status hs = solve_window(ctx, nk, kidx, nw, bw, tw, maxit, prec, precond_kind, nullptr, ev.data(),
                                      out.data(), ldq, itw.data(), rs.data(), &df, last ? 0.0 : tol);
    if (hs == HW_OK || hs == HW_ENOTCONV) {
      for (int b = 0; b < nk; ++b) {
        for (int j = 0; j < nw; ++j) {
          evals[(size_t)b * n_eig + w0 + j] = ev[(size_t)b * nw + j];
          if (resid) resid[(size_t)b * n_eig + w0 + j] = rs[(size_t)b * nw + j];
        }
        if (iters) iters[b] += itw[b];
      }
    }
    if (hs != HW_OK) {   // a window that did not converge ends the solve (its message is kept)
      result = hs;
      break;
    }
  }
  cudaStreamSynchronize(ctx->stream);
  cudaFree(df.C);
  cudaFree(own);
  return result;
}

extern "C" hw_status hw_solve_eigs_traced(hw_ctx* ctx, int k, int n_eig, int block, double tol, int maxit,
                                          hw_prec prec, int precond_kind, const double* X0, int n_rec,
                                          const int* rec_iters, double* rec_R, double* rec_E,
                                          double* rec_theta, double* rec_res, int64_t ld, double* evals,
                                          int* iters) {
  if (!ctx) return HW_EINVAL;
  if (n_rec < 0 || (n_rec > 0 && (!rec_iters || !rec_R || !rec_E || !rec_theta || !rec_res)))
    return hw_fail(ctx, HW_EINVAL, "bad trace buffers");
  if (ctx->have_basis && (k < 0 || k >= ctx->hb.nk || ld < ctx->hb.L[k]))
    return hw_fail(ctx, HW_EINVAL, "bad k-point or ld");
  Trace tr{n_rec, rec_iters, rec_R, rec_E, rec_theta, rec_res, ld, std::vector<char>(std::max(n_rec, 0), 0)};
  const double* x0[1] = {X0};
  FfSolveScope ffs(ctx, prec);
  return solve_impl(ctx, 1, &k, n_eig, block, tol, maxit, prec, precond_kind, X0 ? x0 : nullptr, evals, nullptr,
                    0, iters, nullptr, &tr);
}
