// Teter-Payne-Allan diagonal preconditioner (arXiv 2210.12252, Sec. "Eigensolvers and
// Preconditioning"):  Z_i = P(g_i) / (P(g_i) + 16 g_i^4) R_i,  P(g) = 27 + 18g + 12g^2 + 8g^3,
// g_i = KE_i / KE_res, with KE_res the |R_i|^2-weighted mean of the shifted kinetic energies
// KE_i over the column (the "kinetic energy of the residual vector").
//
// One CTA per column: a reduction pass and an apply pass over the column, both 128-bit
// (one complex128 per thread per step) coalesced streams.
#include "hw_common.cuh"
#include "hw_ctx.h"

namespace hw {

constexpr int TPA_THREADS = 256;

struct TpaArgs {
  int ns;
  int64_t ld;
  const double* ke;
  int64_t keoff[MAXSLOT];
  int64_t L[MAXSLOT];
  Blocks blk;      // x = R, y = Z
};

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

// grid: x = column within block, y = block slot
__global__ void __launch_bounds__(TPA_THREADS) k_tpa(TpaArgs A) {
  griddep_entry();
  __shared__ double red[TPA_THREADS / 32];
  const int slot = blockIdx.y, s = blockIdx.x;
  const int64_t L = A.L[slot];
  const double2* r = reinterpret_cast<const double2*>(A.blk.x[slot]) + (size_t)s * A.ld;
  double2* z = reinterpret_cast<double2*>(A.blk.y[slot]) + (size_t)s * A.ld;
  const double* ke = A.ke + A.keoff[slot];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
    const double2 v = r[i];
    const double w = v.x * v.x + v.y * v.y;
    s0 += w;
    s1 += w * ke[i];
  }
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  const double ke_res = s0 > 0.0 ? s1 / s0 : 1.0;
  const double inv = ke_res > 0.0 ? 1.0 / ke_res : 0.0;
  for (int64_t i = threadIdx.x; i < L; i += blockDim.x) {
    const double g = ke[i] * inv;
    const double P = 27.0 + g * (18.0 + g * (12.0 + g * 8.0));
    const double g2 = g * g;
    const double f = P / (P + 16.0 * g2 * g2);
    double2 v = r[i];
    v.x *= f;
    v.y *= f;
    z[i] = v;
  }
}

cudaError_t launch_tpa(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld) {
  if (blk.nslot > MAXSLOT || blk.nslot < 1 || ns < 1) return cudaErrorInvalidValue;
  TpaArgs a;
  a.ns = ns;
  a.ld = ld;
  a.ke = ctx->db.ke;
  for (int i = 0; i < blk.nslot; ++i) {
    a.keoff[i] = ctx->db.ke_off[blk.kb[i]];
    a.L[i] = ctx->hb.L[blk.kb[i]];
  }
  a.blk = blk;
  ProfScope ps(ctx, HW_PH_PRECOND);
  launch_dep(ctx->stream, k_tpa, dim3(ns, blk.nslot), TPA_THREADS, 0, a);
  ctx->launches++;
  return cudaGetLastError();
}

}  // namespace hw
