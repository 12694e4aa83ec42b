// C ABI of the helical-wave library (declarations and argument contracts: include/helicwave.h).
// Context lifetime, basis setup and upload, potential installation, H X and preconditioner
// entry points.  The block eigensolver lives in hw_lobpcg.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hw_common.cuh"
#include "hw_ctx.h"

hw_status hw_fail(hw_ctx* ctx, hw_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

namespace hw {

void free_basis(hw_ctx* ctx);
void lobpcg_free(hw_ctx* ctx);

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (dev >= 0 && cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// V[i][j][p] (eq. wavefun_storage_real) -> Vd[p][j][i] in FP64 and FP32
__global__ void k_v_relayout(const double* __restrict__ V, double* __restrict__ V64,
                             float* __restrict__ V32, float2* __restrict__ Vff, int n1, int n2, int nr) {
  griddep_entry();
  const long total = (long)n1 * n2 * nr;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n1);
    const long rest = t / n1;
    const int j = (int)(rest % n2);
    const int p = (int)(rest / n2);
    const double v = V[((size_t)i * n2 + j) * nr + p];
    V64[t] = v;
    const float h = (float)v;
    V32[t] = h;
    Vff[t] = make_float2(h, (float)(v - (double)h));   // the pair hi + lo (double-float)
  }
}

std::vector<double> twiddles(int n) {
  std::vector<double> t(2 * n);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < n; ++k) {
    const long double a = -2.0L * pi * k / n;
    t[2 * k] = (double)cosl(a);
    t[2 * k + 1] = (double)sinl(a);
  }
  return t;
}

hw_status cuda_fail(hw_ctx* ctx, cudaError_t e, const char* what) {
  return hw_fail(ctx, HW_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

hw_status check_device_call(hw_ctx* ctx) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (!ctx->have_basis) return hw_fail(ctx, HW_ESTATE, "hw_setup_basis has not been called");
  return HW_OK;
}

}  // namespace

void free_basis(hw_ctx* ctx) {
  auto& db = ctx->db;
  dfree(db.group_start);
  dfree(db.pair_n);
  dfree(db.pair_mrow);
  dfree(db.mrow_m);
  dfree(db.slot_pair);
  dfree(db.off);
  dfree(db.Ka);
  dfree(db.ke);
  dfree(db.vscratch);
  dfree(db.vff);
  dfree(db.ff_rinv);
  dfree(db.ff_rfwd);
  db.ke_off.clear();
  for (auto* t : {&db.t64.rinv, &db.t64.rfwd, &db.t64.qtab, &db.t64.rder, &db.t64.V, &db.t64.tw1, &db.t64.tw2})
    dfree(*t);
  for (auto* t : {&db.t32.rinv, &db.t32.rfwd, &db.t32.qtab, &db.t32.rder, &db.t32.V, &db.t32.tw1, &db.t32.tw2})
    dfree(*t);
  dfree(db.rnodes);
  dfree(db.rt_inv);
  dfree(db.rt_fwd);
  db.rt_ok = false;
  dfree(ctx->ws.gbuf);
  dfree(ctx->ws.hbuf);
  ctx->ws.cols = 0;
  lobpcg_free(ctx);
  mlp_free_basis(ctx);
  ctx->have_basis = false;
  ctx->have_V = false;
}

}  // namespace hw

using namespace hw;

extern "C" {

hw_status hw_create(hw_ctx** out, int device, void* cuda_stream) {
  if (!out) return HW_EINVAL;
  *out = nullptr;
  hw_ctx* ctx = new (std::nothrow) hw_ctx();
  if (!ctx) return HW_ENOMEM;
  ctx->device = device;
  if (device >= 0) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device >= n) {
      delete ctx;
      return HW_ECUDA;
    }
    DeviceGuard g(device);
    cudaSetDevice(device);
    ctx->stream = (cudaStream_t)cuda_stream;
    if (cublasCreate(&ctx->cublas) != CUBLAS_STATUS_SUCCESS) {
      delete ctx;
      return HW_ECUDA;
    }
    cublasSetStream(ctx->cublas, ctx->stream);
    cublasSetPointerMode(ctx->cublas, CUBLAS_POINTER_MODE_HOST);
    if (cudaMalloc((void**)&ctx->dflag, 64 * sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->dflag, 0, 64 * sizeof(int)) != cudaSuccess) {
      cublasDestroy(ctx->cublas);
      delete ctx;
      return HW_ECUDA;
    }
    if (hx_configure(ctx) != cudaSuccess) {
      cudaFree(ctx->dflag);
      cublasDestroy(ctx->cublas);
      delete ctx;
      return HW_ECUDA;
    }
  }
  *out = ctx;
  return HW_OK;
}

void hw_destroy(hw_ctx* ctx) {
  if (!ctx) return;
  if (ctx->device >= 0) {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_basis(ctx);
    mlp_free(ctx);
    if (ctx->dflag) cudaFree(ctx->dflag);
    if (ctx->dens_w) cudaFree(ctx->dens_w);
    zgemm_free(ctx->zg);
    if (ctx->cublas) cublasDestroy(ctx->cublas);
  }
  delete ctx;
}

const char* hw_last_error(const hw_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

hw_status hw_setup_basis(hw_ctx* ctx, const hw_basis_params* params, int nk, const double* eta,
                         const double* nu, const double* ecut_per_k, int64_t* L_out) {
  if (!ctx || !params) return hw_fail(ctx, HW_EINVAL, "null argument");
  HostBasis hb;
  std::string msg = build_host_basis(*params, nk, eta, nu, ecut_per_k, hb);
  if (!msg.empty()) return hw_fail(ctx, HW_EINVAL, msg);
  if (hb.K > 64) return hw_fail(ctx, HW_EINVAL, "K = Nr/oversample must be <= 64");
  FftPlan p1, p2;
  if (!make_fft_plan(params->Nth1, p1) || !make_fft_plan(params->Nth2, p2))
    return hw_fail(ctx, HW_EINVAL, "angular grid sizes must factor into 2 and 3");
  if (ctx->device >= 0) {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_basis(ctx);
    auto& db = ctx->db;
    cudaError_t e = cudaSuccess;
    const int Nr = params->Nr, K = hb.K, N = hb.N;
    // radial tables
    std::vector<double> rinv((size_t)(N + 1) * Nr * K), rfwd((size_t)(N + 1) * K * Nr);
    const double pi = 3.14159265358979323846;
    const double scale = 2.0 * pi * params->tau / params->ncyc / (double(params->Nth1) * params->Nth2);
    for (int n = 0; n <= N; ++n)
      for (int p = 0; p < Nr; ++p)
        for (int k = 0; k < K; ++k) {
          const double x = hb.xi[((size_t)n * Nr + p) * K + k];
          rinv[((size_t)n * Nr + p) * K + k] = x;
          rfwd[((size_t)n * K + k) * Nr + p] = scale * hb.wr[p] * x;
        }
    std::vector<float> rinv32(rinv.begin(), rinv.end()), rfwd32(rfwd.begin(), rfwd.end());
    // the radial tables as double-float pairs (hi = FP32 rounding, lo = FP32 rounding of the rest)
    auto pairs = [](const std::vector<double>& v) {
      std::vector<float2> o(v.size());
      for (size_t i = 0; i < v.size(); ++i) {
        const float h = (float)v[i];
        o[i] = make_float2(h, (float)(v[i] - (double)h));
      }
      return o;
    };
    const std::vector<float2> rinvff = pairs(rinv), rfwdff = pairs(rfwd);
    std::vector<float> qtab32(hb.qtab.begin(), hb.qtab.end());
    std::vector<float> rder32(hb.xid.begin(), hb.xid.end());
    std::vector<double> tw1 = twiddles(params->Nth1), tw2 = twiddles(params->Nth2);
    std::vector<float> tw1f(tw1.begin(), tw1.end()), tw2f(tw2.begin(), tw2.end());
    std::vector<double> keall;
    db.ke_off.assign(nk + 1, 0);
    for (int b = 0; b < nk; ++b) {
      db.ke_off[b] = (int64_t)keall.size();
      keall.insert(keall.end(), hb.ke[b].begin(), hb.ke[b].end());
    }
    db.ke_off[nk] = (int64_t)keall.size();
    const size_t grid = (size_t)params->Nth1 * params->Nth2 * Nr;
#define UP(dst, vec)                                            \
  if (e == cudaSuccess) e = upload(&(dst), (vec).data(), (vec).size());
    UP(db.group_start, hb.group_start);
    UP(db.pair_n, hb.pair_n);
    UP(db.pair_mrow, hb.pair_mrow);
    UP(db.mrow_m, hb.mrow_m);
    UP(db.slot_pair, hb.slot_pair);
    UP(db.off, hb.off);
    UP(db.Ka, hb.Ka);
    UP(db.ke, keall);
    UP(db.t64.rinv, rinv);
    UP(db.t64.rfwd, rfwd);
    UP(db.t64.qtab, hb.qtab);
    UP(db.t32.qtab, qtab32);
    UP(db.t64.rder, hb.xid);
    UP(db.t32.rder, rder32);
    UP(db.rnodes, hb.r);
    UP(db.t64.tw1, tw1);
    UP(db.t64.tw2, tw2);
    UP(db.ff_rinv, rinvff);
    UP(db.ff_rfwd, rfwdff);
    UP(db.t32.rinv, rinv32);
    UP(db.t32.rfwd, rfwd32);
    UP(db.t32.tw1, tw1f);
    UP(db.t32.tw2, tw2f);
#undef UP
    if (e == cudaSuccess) e = cudaMalloc((void**)&db.t64.V, grid * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&db.t32.V, grid * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void**)&db.vscratch, grid * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&db.vff, grid * sizeof(float2));
    if (e == cudaSuccess) e = radial_tc_setup(ctx, hb, rinv, rfwd);
    // G / H workspace: passes of up to `cols` columns, ~1 GiB for both buffers
    const size_t per_col = 2 * (size_t)Nr * hb.nA * sizeof(double2);
    size_t cols = std::max<size_t>(16, std::min<size_t>(2048, (size_t(1) << 30) / per_col));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ws.gbuf, cols * per_col / 2);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->ws.hbuf, cols * per_col / 2);
    if (e != cudaSuccess) {
      free_basis(ctx);
      return hw_fail(ctx, e == cudaErrorMemoryAllocation ? HW_ENOMEM : HW_ECUDA,
                     std::string("setup upload: ") + cudaGetErrorString(e));
    }
    ctx->ws.cols = cols;
  }
  ctx->hb = std::move(hb);
  ctx->plan1 = p1;
  ctx->plan2 = p2;
  ctx->have_basis = true;
  ctx->have_V = false;
  if (L_out)
    for (int b = 0; b < nk; ++b) L_out[b] = ctx->hb.L[b];
  return HW_OK;
}

hw_status hw_get_sizes(const hw_ctx* ctx, int* M, int* N, int* K, int64_t* grid_points,
                       int* n_pairs) {
  if (!ctx) return HW_EINVAL;
  if (!ctx->have_basis) return HW_ESTATE;
  const auto& hb = ctx->hb;
  if (M) *M = hb.M;
  if (N) *N = hb.N;
  if (K) *K = hb.K;
  if (grid_points) *grid_points = (int64_t)hb.prm.Nth1 * hb.prm.Nth2 * hb.prm.Nr;
  if (n_pairs) *n_pairs = hb.nA;
  return HW_OK;
}

hw_status hw_get_grid(const hw_ctx* ctx, double* r_nodes, double* r_weights) {
  if (!ctx) return HW_EINVAL;
  if (!ctx->have_basis) return HW_ESTATE;
  if (r_nodes) std::memcpy(r_nodes, ctx->hb.r.data(), ctx->hb.r.size() * sizeof(double));
  if (r_weights) std::memcpy(r_weights, ctx->hb.wr.data(), ctx->hb.wr.size() * sizeof(double));
  return HW_OK;
}

hw_status hw_get_index_map(const hw_ctx* ctx, int k, int32_t* mnk) {
  if (!ctx || !mnk) return HW_EINVAL;
  if (!ctx->have_basis) return HW_ESTATE;
  if (k < 0 || k >= ctx->hb.nk) return HW_EINVAL;
  std::memcpy(mnk, ctx->hb.mnk[k].data(), ctx->hb.mnk[k].size() * sizeof(int32_t));
  return HW_OK;
}

hw_status hw_get_kinetic(const hw_ctx* ctx, int k, double* ke) {
  if (!ctx || !ke) return HW_EINVAL;
  if (!ctx->have_basis) return HW_ESTATE;
  if (k < 0 || k >= ctx->hb.nk) return HW_EINVAL;
  std::memcpy(ke, ctx->hb.ke[k].data(), ctx->hb.ke[k].size() * sizeof(double));
  return HW_OK;
}

hw_status hw_get_radial_table(const hw_ctx* ctx, int n, double* table) {
  if (!ctx || !table) return HW_EINVAL;
  if (!ctx->have_basis) return HW_ESTATE;
  const auto& hb = ctx->hb;
  if (n < -hb.N || n > hb.N) return HW_EINVAL;
  const size_t sz = (size_t)hb.prm.Nr * hb.K;
  std::memcpy(table, hb.xi.data() + (size_t)std::abs(n) * sz, sz * sizeof(double));
  return HW_OK;
}

hw_status hw_get_itable(const hw_ctx* ctx, int n, double* table) {
  if (!ctx || !table) return HW_EINVAL;
  if (!ctx->have_basis) return HW_ESTATE;
  const auto& hb = ctx->hb;
  if (n < -hb.N || n > hb.N) return HW_EINVAL;
  const size_t sz = (size_t)hb.K * hb.K;
  const double s = 0.5 * hb.prm.R * hb.prm.R;   // I = (R^2 / 2) <F_k', F_k / r^2>
  const double* q = hb.qtab.data() + (size_t)std::abs(n) * sz;
  for (size_t i = 0; i < sz; ++i) table[i] = s * q[i];
  return HW_OK;
}

hw_status hw_set_potential(hw_ctx* ctx, const double* V, int on_device) {
  hw_status st = check_device_call(ctx);
  if (st != HW_OK) return st;
  if (!V) return hw_fail(ctx, HW_EINVAL, "null potential");
  DeviceGuard g(ctx->device);
  const auto& p = ctx->hb.prm;
  const size_t grid = (size_t)p.Nth1 * p.Nth2 * p.Nr;
  cudaError_t e;
  if (on_device) {
    e = cudaMemcpyAsync(ctx->db.vscratch, V, grid * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
  } else {
    for (size_t i = 0; i < grid; ++i)
      if (!std::isfinite(V[i])) return hw_fail(ctx, HW_EINVAL, "potential has a non-finite entry");
    e = cudaMemcpyAsync(ctx->db.vscratch, V, grid * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "set_potential copy");
  launch_dep(ctx->stream, k_v_relayout, 1024, 256, 0, ctx->db.vscratch, ctx->db.t64.V, ctx->db.t32.V, ctx->db.vff,
                                              p.Nth1, p.Nth2, p.Nr);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "set_potential relayout");
  ctx->launches++;
  ctx->have_V = true;
  if (ctx->mlp) {
    e = mlp_refresh_potential(ctx);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "potential diagonal");
  }
  return HW_OK;
}

hw_status hw_build_potential(hw_ctx* ctx, int n_atoms, const double* atoms, double* V_out) {
  if (!ctx) return HW_EINVAL;
  if (!ctx->have_basis) return hw_fail(ctx, HW_ESTATE, "hw_setup_basis has not been called");
  if (n_atoms < 0 || (n_atoms > 0 && !atoms)) return hw_fail(ctx, HW_EINVAL, "bad atom list");
  for (int a = 0; a < n_atoms; ++a) {
    for (int c = 0; c < 5; ++c)
      if (!std::isfinite(atoms[5 * a + c])) return hw_fail(ctx, HW_EINVAL, "non-finite atom entry");
    if (!(atoms[5 * a + 4] > 0)) return hw_fail(ctx, HW_EINVAL, "sigma must be > 0");
    if (atoms[5 * a] < 0) return hw_fail(ctx, HW_EINVAL, "atom radius must be >= 0");
  }
  std::vector<double> V;
  build_gaussian_potential(ctx->hb, n_atoms, atoms, V);
  if (V_out) std::memcpy(V_out, V.data(), V.size() * sizeof(double));
  if (ctx->device < 0) return HW_OK;
  return hw_set_potential(ctx, V.data(), 0);
}

static hw_status apply_common(hw_ctx* ctx, int nk, const int* kidx, const double* const* X,
                              double* const* Y, int ns, int64_t ld, hw_prec prec) {
  hw_status st = check_device_call(ctx);
  if (st != HW_OK) return st;
  if (!ctx->have_V) return hw_fail(ctx, HW_ESTATE, "no potential installed");
  if (nk < 1 || ns < 1 || !kidx || !X || !Y) return hw_fail(ctx, HW_EINVAL, "bad block arguments");
  if (prec != HW_FP64 && prec != HW_MIXED && prec != HW_FP64_DF) return hw_fail(ctx, HW_EINVAL, "bad precision");
  int64_t maxL = 0;
  for (int b = 0; b < nk; ++b) {
    if (kidx[b] < 0 || kidx[b] >= ctx->hb.nk) return hw_fail(ctx, HW_EINVAL, "k-point index out of range");
    if (!X[b] || !Y[b]) return hw_fail(ctx, HW_EINVAL, "null block pointer");
    if (X[b] == Y[b]) return hw_fail(ctx, HW_EINVAL, "X and Y must not overlap");
    maxL = std::max(maxL, ctx->hb.L[kidx[b]]);
  }
  if (ld < maxL) return hw_fail(ctx, HW_EINVAL, "ld < L");
  DeviceGuard g(ctx->device);
  for (int b0 = 0; b0 < nk; b0 += MAXSLOT) {
    Blocks blk;
    blk.nslot = std::min(MAXSLOT, nk - b0);
    for (int i = 0; i < blk.nslot; ++i) {
      blk.x[i] = X[b0 + i];
      blk.y[i] = Y[b0 + i];
      blk.kb[i] = kidx[b0 + i];
    }
    ctx->ff_now = prec == HW_FP64_DF;
    cudaError_t e = prec == HW_MIXED ? launch_hx<float>(ctx, blk, ns, ld) : launch_hx<double>(ctx, blk, ns, ld);
    ctx->ff_now = false;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "apply_H launch");
  }
  return HW_OK;
}

hw_status hw_apply_H(hw_ctx* ctx, int k, const double* X, double* Y, int ns, int64_t ld,
                     hw_prec prec) {
  return apply_common(ctx, 1, &k, &X, &Y, ns, ld, prec);
}

hw_status hw_apply_H_batched(hw_ctx* ctx, int nk, const int* kidx, const double* const* X,
                             double* const* Y, int ns, int64_t ld, hw_prec prec) {
  return apply_common(ctx, nk, kidx, X, Y, ns, ld, prec);
}

hw_status hw_density(hw_ctx* ctx, int nk, const int* kidx, const double* const* X, int ns, int64_t ld,
                     const double* occ, const double* w, double* rho, hw_prec prec) {
  hw_status st = check_device_call(ctx);
  if (st != HW_OK) return st;
  if (nk < 1 || ns < 1 || !kidx || !X || !occ || !w || !rho) return hw_fail(ctx, HW_EINVAL, "bad density arguments");
  if (prec != HW_FP64 && prec != HW_MIXED && prec != HW_FP64_DF) return hw_fail(ctx, HW_EINVAL, "bad precision");
  int64_t maxL = 0;
  for (int b = 0; b < nk; ++b) {
    if (kidx[b] < 0 || kidx[b] >= ctx->hb.nk) return hw_fail(ctx, HW_EINVAL, "k-point index out of range");
    if (!X[b]) return hw_fail(ctx, HW_EINVAL, "null block pointer");
    maxL = std::max(maxL, ctx->hb.L[kidx[b]]);
  }
  if (ld < maxL) return hw_fail(ctx, HW_EINVAL, "ld < L");
  if (!density_fits(ctx, prec == HW_FP64 ? sizeof(double) : sizeof(float)))
    return hw_fail(ctx, HW_EINVAL, "angular grid too large for the density kernel at this precision");
  DeviceGuard g(ctx->device);
  const size_t ncol = (size_t)nk * ns;
  if (ctx->dens_w_n < ncol) {
    if (ctx->dens_w) cudaFree(ctx->dens_w);
    ctx->dens_w = nullptr;
    ctx->dens_w_n = 0;
    if (cudaMalloc((void**)&ctx->dens_w, ncol * sizeof(double)) != cudaSuccess)
      return hw_fail(ctx, HW_ENOMEM, "density weights");
    ctx->dens_w_n = ncol;
  }
  // column weight (2 / Ncyc) w_b occ_{b,j}
  std::vector<double> wc(ncol);
  const double f = 2.0 / ctx->hb.prm.ncyc;
  for (int b = 0; b < nk; ++b)
    for (int j = 0; j < ns; ++j) wc[(size_t)b * ns + j] = f * w[b] * occ[(size_t)b * ns + j];
  cudaError_t e = cudaMemcpyAsync(ctx->dens_w, wc.data(), ncol * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  const size_t G = (size_t)ctx->hb.prm.Nth1 * ctx->hb.prm.Nth2 * ctx->hb.prm.Nr;
  if (e == cudaSuccess) e = cudaMemsetAsync(rho, 0, G * sizeof(double), ctx->stream);
  for (int b0 = 0; b0 < nk && e == cudaSuccess; b0 += MAXSLOT) {
    Blocks blk;
    blk.nslot = std::min(MAXSLOT, nk - b0);
    for (int i = 0; i < blk.nslot; ++i) {
      blk.x[i] = X[b0 + i];
      blk.y[i] = nullptr;
      blk.kb[i] = kidx[b0 + i];
    }
    const double* wb = ctx->dens_w + (size_t)b0 * ns;
    e = prec == HW_FP64 ? launch_density<double>(ctx, blk, ns, ld, wb, rho)
                        : launch_density<float>(ctx, blk, ns, ld, wb, rho);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);   // wc must outlive the copy
  if (e != cudaSuccess) return cuda_fail(ctx, e, "density");
  return HW_OK;
}

hw_status hw_gradient(hw_ctx* ctx, int k, const double* X, int ns, int64_t ld, double* D, hw_prec prec) {
  hw_status st = check_device_call(ctx);
  if (st != HW_OK) return st;
  if (k < 0 || k >= ctx->hb.nk) return hw_fail(ctx, HW_EINVAL, "k-point index out of range");
  if (!X || !D || ns < 1 || ld < ctx->hb.L[k]) return hw_fail(ctx, HW_EINVAL, "bad gradient arguments");
  if (prec != HW_FP64 && prec != HW_MIXED) return hw_fail(ctx, HW_EINVAL, "bad precision");
  if (!gradient_fits(ctx, prec == HW_FP64 ? sizeof(double2) : sizeof(float2)))
    return hw_fail(ctx, HW_EINVAL, "angular grid too large for the gradient kernel at this precision");
  DeviceGuard g(ctx->device);
  Blocks blk;
  blk.nslot = 1;
  blk.x[0] = X;
  blk.y[0] = nullptr;
  blk.kb[0] = k;
  const cudaError_t e = prec == HW_FP64 ? launch_gradient<double>(ctx, blk, ns, ld, D)
                                        : launch_gradient<float>(ctx, blk, ns, ld, D);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gradient");
  return HW_OK;
}

hw_status hw_apply_precond(hw_ctx* ctx, int k, const double* R, double* Z, int ns, int64_t ld,
                           const double* ritz, int kind) {
  hw_status st = check_device_call(ctx);
  if (st != HW_OK) return st;
  if (k < 0 || k >= ctx->hb.nk) return hw_fail(ctx, HW_EINVAL, "k-point index out of range");
  if (!R || !Z || ns < 1 || ld < ctx->hb.L[k]) return hw_fail(ctx, HW_EINVAL, "bad block arguments");
  DeviceGuard g(ctx->device);
  Blocks blk;
  blk.nslot = 1;
  blk.x[0] = R;
  blk.y[0] = Z;
  blk.kb[0] = k;
  cudaError_t e;
  if (kind == HW_PRECOND_TPA) {
    e = launch_tpa(ctx, blk, ns, ld);
  } else if (kind == HW_PRECOND_NONE) {
    e = (R == Z) ? cudaSuccess
                 : cudaMemcpy2DAsync(Z, ld * 16, R, ld * 16, ctx->hb.L[k] * 16, ns, cudaMemcpyDeviceToDevice,
                                     ctx->stream);
  } else if (kind == HW_PRECOND_LEARNED) {
    if (!ctx->mlp) return hw_fail(ctx, HW_ESTATE, "no network installed (hw_set_mlp)");
    if (!ctx->have_V) return hw_fail(ctx, HW_ESTATE, "no potential installed");
    if (!ritz) return hw_fail(ctx, HW_EINVAL, "the learned preconditioner needs the Ritz values");
    e = launch_precond_learned(ctx, blk, ns, ld, &ritz);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  } else {
    return hw_fail(ctx, HW_EINVAL, "unknown preconditioner kind");
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "apply_precond");
  return HW_OK;
}

hw_status hw_autotune(hw_ctx* ctx, int k, int ns, float* results, int max_results, int* n_results) {
  hw_status st = check_device_call(ctx);
  if (st != HW_OK) return st;
  if (!ctx->have_V) return hw_fail(ctx, HW_ESTATE, "no potential installed");
  if (k < 0 || k >= ctx->hb.nk || ns < 1) return hw_fail(ctx, HW_EINVAL, "bad k-point or column count");
  DeviceGuard g(ctx->device);
  std::vector<float> log;
  cudaError_t e = hx_autotune(ctx, k, ns, log);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
  const int nr = (int)(log.size() / 4);
  if (results)
    for (int i = 0; i < std::min(nr, max_results); ++i)
      for (int c = 0; c < 4; ++c) results[4 * i + c] = log[4 * i + c];
  if (n_results) *n_results = nr;
  return HW_OK;
}

hw_status hw_set_option(hw_ctx* ctx, int option, int value) {
  if (!ctx) return HW_EINVAL;
  if (option == HW_OPT_RR_METHOD) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "RR method 0 (auto) or 1 (Jacobi)");
    ctx->rr_method = value;
    return HW_OK;
  }
  if (option == HW_OPT_LOWP_SWITCH) {
    if (value < 0 || value > 12) return hw_fail(ctx, HW_EINVAL, "low-precision switch exponent 0..12");
    ctx->lowp_exp = value;
    return HW_OK;
  }
  if (option == HW_OPT_GRAM_KERNEL) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "Gram kernel option 0 or 1");
    ctx->gram_mixed = value;
    return HW_OK;
  }
  if (option == HW_OPT_HYBRID) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "hybrid option 0 or 1");
    ctx->hybrid = value;
    return HW_OK;
  }
  if (option == HW_OPT_EIGENSOLVER) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "eigensolver 0 (LOBPCG) or 1 (Chebyshev filtering)");
    ctx->eigensolver = value;
    return HW_OK;
  }
  if (option == HW_OPT_CHEB_DEGREE) {
    if (value < 2 || value > 64) return hw_fail(ctx, HW_EINVAL, "Chebyshev degree 2..64");
    ctx->cheb_degree = value;
    return HW_OK;
  }
  if (option == HW_OPT_CHEB_ADAPT) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "adaptive Chebyshev degree option 0 or 1");
    ctx->cheb_adapt = value;
    return HW_OK;
  }
  if (option == HW_OPT_TAIL_NO_P) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "end-phase option 0 or 1");
    ctx->tail_no_p = value;
    return HW_OK;
  }
  if (option == HW_OPT_CHEB_LOCK) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "Chebyshev locking option 0 or 1");
    ctx->cheb_lock = value;
    return HW_OK;
  }
  if (option == HW_OPT_SLAB_KERNEL) {
    if (value < 0 || value > 3)
      return hw_fail(ctx, HW_EINVAL,
                     "slab kernel option 0 (FFT), 1 (4 x 16), 2 (registers, FP32) or 3 (registers, both)");
    ctx->slab_r16 = value;
    return HW_OK;
  }
  if (option == HW_OPT_WINDOW) {
    if (value < 0 || value > 100) return hw_fail(ctx, HW_EINVAL, "window 0 (100) or 1..100 eigenpairs");
    ctx->window = value;
    return HW_OK;
  }
  if (option == HW_OPT_TC_GEMM) {
    if (value < 0 || value > 2) return hw_fail(ctx, HW_EINVAL, "block-product option 0, 1 or 2");
    ctx->tc_gemm = value;
    return HW_OK;
  }
  if (option == HW_OPT_RADIAL_KERNEL) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "radial kernel option 0 (SIMT) or 1 (tensor cores)");
    ctx->radial_tc = value;
    return HW_OK;
  }
  if (option == HW_OPT_FP64_HX) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "FP64 H X option 0 (FP64) or 1 (double-float)");
    ctx->fp64_hx_ff = value;
    return HW_OK;
  }
  if (option == HW_OPT_SMALL_GEMM) {
    if (value < 0 || value > 2)
      return hw_fail(ctx, HW_EINVAL, "small-product option 0 (cuBLAS), 1 (SIMT kernel, FP32 class) or 2 (both classes)");
    ctx->small_gemm = value;
    return HW_OK;
  }
  if (option == HW_OPT_OVERLAP_LAUNCH) {
    if (value != 0 && value != 1) return hw_fail(ctx, HW_EINVAL, "overlapped-launch option 0 or 1");
    ctx->overlap_launch = value;
    return HW_OK;
  }
  return hw_fail(ctx, HW_EINVAL, "unknown or read-only option");
}

hw_status hw_get_option(hw_ctx* ctx, int option, long long* value) {
  if (!ctx || !value) return HW_EINVAL;
  if (option == HW_OPT_RR_METHOD) { *value = ctx->rr_method; return HW_OK; }
  if (option == HW_OPT_RR_FALLBACKS) { *value = ctx->rr_fallbacks; return HW_OK; }
  if (option == HW_OPT_LOWP_SWITCH) { *value = ctx->lowp_exp; return HW_OK; }
  if (option == HW_OPT_GRAM_KERNEL) { *value = ctx->gram_mixed; return HW_OK; }
  if (option == HW_OPT_HYBRID) { *value = ctx->hybrid; return HW_OK; }
  if (option == HW_OPT_EIGENSOLVER) { *value = ctx->eigensolver; return HW_OK; }
  if (option == HW_OPT_CHEB_DEGREE) { *value = ctx->cheb_degree; return HW_OK; }
  if (option == HW_OPT_CHEB_ADAPT) { *value = ctx->cheb_adapt; return HW_OK; }
  if (option == HW_OPT_CHEB_LOCK) { *value = ctx->cheb_lock; return HW_OK; }
  if (option == HW_OPT_TAIL_NO_P) { *value = ctx->tail_no_p; return HW_OK; }
  if (option == HW_OPT_SLAB_KERNEL) { *value = ctx->slab_r16; return HW_OK; }
  if (option == HW_OPT_WINDOW) { *value = ctx->window; return HW_OK; }
  if (option == HW_OPT_TC_GEMM) { *value = ctx->tc_gemm; return HW_OK; }
  if (option == HW_OPT_RADIAL_KERNEL) { *value = ctx->radial_tc; return HW_OK; }
  if (option == HW_OPT_FP64_HX) { *value = ctx->fp64_hx_ff; return HW_OK; }
  if (option == HW_OPT_SMALL_GEMM) { *value = ctx->small_gemm; return HW_OK; }
  if (option == HW_OPT_OVERLAP_LAUNCH) { *value = ctx->overlap_launch; return HW_OK; }
  return hw_fail(ctx, HW_EINVAL, "unknown option");
}

hw_status hw_synchronize(hw_ctx* ctx) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return HW_OK;
  DeviceGuard g(ctx->device);
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronize");
  return HW_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------ profiling
namespace hw {

ProfScope::ProfScope(hw_ctx* ctx, int ph, double work) : ctx_(ctx), ph_(ph), work_(work) {
  if (!ctx_ || !ctx_->prof.on) return;
  auto& p = ctx_->prof;
  if (p.pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    p.pool.push_back(e);
  }
  a_ = p.pool.back();
  p.pool.pop_back();
  cudaEventRecord(a_, ctx_->stream);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  auto& p = ctx_->prof;
  cudaEvent_t b;
  if (p.pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) {
      p.pool.push_back(a_);
      return;
    }
  } else {
    b = p.pool.back();
    p.pool.pop_back();
  }
  cudaEventRecord(b, ctx_->stream);
  p.pending.push_back({ph_, a_, b, work_});
}

static void prof_collect(hw_ctx* ctx) {
  auto& p = ctx->prof;
  for (auto& r : p.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      p.ms[r.ph] += ms;
      p.cnt[r.ph] += 1;
      p.work[r.ph] += r.work;
    }
    p.pool.push_back(r.a);
    p.pool.push_back(r.b);
  }
  p.pending.clear();
}

}  // namespace hw

extern "C" {

hw_status hw_profile(hw_ctx* ctx, int enable) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  cudaStreamSynchronize(ctx->stream);
  hw::prof_collect(ctx);
  for (int i = 0; i < HW_NPHASE; ++i) {
    ctx->prof.ms[i] = 0.0;
    ctx->prof.cnt[i] = 0;
    ctx->prof.work[i] = 0.0;
  }
  ctx->prof.on = enable != 0;
  return HW_OK;
}

hw_status hw_profile_read(hw_ctx* ctx, double* ms, int64_t* count) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
  hw::prof_collect(ctx);
  for (int i = 0; i < HW_NPHASE; ++i) {
    if (ms) ms[i] = ctx->prof.ms[i];
    if (count) count[i] = ctx->prof.cnt[i];
  }
  return HW_OK;
}

hw_status hw_profile_work(hw_ctx* ctx, double* work) {
  if (!ctx || !work) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, cudaGetErrorString(e));
  hw::prof_collect(ctx);
  for (int i = 0; i < HW_NPHASE; ++i) work[i] = ctx->prof.work[i];
  return HW_OK;
}

int64_t hw_launch_count(const hw_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
