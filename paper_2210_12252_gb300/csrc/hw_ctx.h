// The library context and device-side data (CUDA translation units only).
#pragma once

#include <cublas_v2.h>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "hw_internal.h"

namespace hw {

constexpr int MAXSLOT = 64;   // column blocks (k-points) per launch

template <typename T>
struct DevTables {
  T* rinv = nullptr;   // [(N+1)][Nr][K]      xi_{n,k}(r_p)
  T* rfwd = nullptr;   // [(N+1)][K][Nr]      (2 pi tau / Ncyc) w_p xi_{n,k}(r_p) / (Nth1 Nth2)
  T* qtab = nullptr;   // [(N+1)][K][K]       <F_{m,n,k'}, F_{m,n,k} / r^2> (symmetric)
  T* rder = nullptr;   // [(N+1)][Nr][K]      d xi_{n,k} / dr at r_p (Appendix C's B_n)
  T* V = nullptr;      // [Nr][Nth2][Nth1]    potential, slab layout
  T* tw1 = nullptr;    // [2*Nth1]            e^{-2 pi i t / Nth1} as (re, im)
  T* tw2 = nullptr;    // [2*Nth2]
};

struct DevBasis {
  int* group_start = nullptr;  // [N+2]
  int* pair_n = nullptr;       // [nA]
  int* pair_mrow = nullptr;    // [nA]
  int* mrow_m = nullptr;       // [nmr]
  int* slot_pair = nullptr;    // [nmr][Nth2]: pair index or -1
  int* off = nullptr;          // [nk][nA]
  int* Ka = nullptr;           // [nk][nA]
  double* ke = nullptr;        // concatenated [sum L_b] shifted kinetic energies
  double* rnodes = nullptr;    // [Nr] radial nodes r_p
  std::vector<int64_t> ke_off; // host: start of k-point b in ke
  double* vscratch = nullptr;  // [grid] staging for set_potential
  float2* vff = nullptr;       // [Nr][Nth2][Nth1] the potential as FP32 pairs (hi, lo), slab layout
  float2* ff_rinv = nullptr;   // the radial tables of DevTables as FP32 pairs (hi, lo)
  float2* ff_rfwd = nullptr;
  DevTables<double> t64;
  DevTables<float> t32;
  // tensor-core radial transforms of the FP32 H X: BF16 three-part tables per |n| group
  __nv_bfloat16* rt_inv = nullptr;   // [(N+1)][3][rt_npad][rt_kb * 32]   xi rows p, columns k
  __nv_bfloat16* rt_fwd = nullptr;   // [(N+1)][3][rt_kpad][rt_kbp * 32]  O rows k, columns p
  int rt_npad = 0, rt_kb = 0, rt_kpad = 0, rt_kbp = 0;
  bool rt_ok = false;          // the shapes fit the kernels (N_r <= 256, K <= 64)
  // TMA maps over the two tables: 3-D {32-column block, rows, group x part}, 64-byte swizzle
  CUtensorMap rt_map_inv, rt_map_fwd;
};

// G / H intermediates for `cols` columns per pass, [column][r_p][pair] complex FP64-sized
struct Workspace {
  void* gbuf = nullptr;
  void* hbuf = nullptr;
  size_t cols = 0;        // capacity of gbuf / hbuf in FP64 columns
  int pass_cols[2] = {0, 0};   // autotuned columns per pass (FP64, FP32); 0 = capacity
  int jc[2] = {0, 0};          // autotuned slab theta2 chunk (FP64, FP32); 0 = heuristic
};

// per-launch column blocks, passed by value to the kernels
struct Blocks {
  const double* x[MAXSLOT];
  double* y[MAXSLOT];
  int kb[MAXSLOT];
  int nslot;
};

// One step of a three-term recurrence fused into an H X launch: the forward radial kernel
// writes y = al_b (H x - c_b x) - be_b y (y's old content read only when be_b != 0) instead of
// H x, per column block b (the scaled Chebyshev filter).
struct ChebStep {
  double al[MAXSLOT], c[MAXSLOT], be[MAXSLOT];
};

struct LobpcgWork;
struct MlpState;
struct ZgemmWork;

// Per-phase timing with CUDA events on the context's stream (enabled by hw_profile).
struct Prof {
  bool on = false;
  struct Rec {
    int ph;
    cudaEvent_t a, b;
    double work;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> pending;
  double ms[HW_NPHASE] = {0};
  int64_t cnt[HW_NPHASE] = {0};
  double work[HW_NPHASE] = {0};
};

}  // namespace hw

struct hw_ctx {
  int device = -1;
  cudaStream_t stream = nullptr;
  cublasHandle_t cublas = nullptr;
  std::string err;
  bool have_basis = false;
  bool have_V = false;
  hw::HostBasis hb;
  hw::FftPlan plan1, plan2;
  hw::DevBasis db;
  hw::Workspace ws;
  hw::LobpcgWork* lw = nullptr;
  hw::MlpState* mlp = nullptr;
  hw::ZgemmWork* zg = nullptr;   // workspace of the tensor-core block products
  int tc_gemm = 1;             // HW_OPT_TC_GEMM
  int* dflag = nullptr;        // device status word for bounded waits
  int64_t launches = 0;        // kernels of this library launched on the stream
  double* dens_w = nullptr;    // column weights of hw_density (grown when needed)
  size_t dens_w_n = 0;
  int rr_method = 0;           // HW_OPT_RR_METHOD
  int lowp_exp = 5;            // HW_OPT_LOWP_SWITCH
  int gram_mixed = 0;          // HW_OPT_GRAM_KERNEL
  int hybrid = 1;              // HW_OPT_HYBRID
  int eigensolver = 0;         // HW_OPT_EIGENSOLVER
  int cheb_degree = 24;        // HW_OPT_CHEB_DEGREE
  int cheb_adapt = 1;          // HW_OPT_CHEB_ADAPT
  int cheb_lock = 1;           // HW_OPT_CHEB_LOCK
  int tail_no_p = 0;           // HW_OPT_TAIL_NO_P
  int window = 0;              // HW_OPT_WINDOW (0: 100)
  int slab_r16 = 2;            // HW_OPT_SLAB_KERNEL
  int fp64_hx_ff = 1;          // HW_OPT_FP64_HX: the mixed solver's FP64 H X with double-float angular transforms
  int small_gemm = 1;          // HW_OPT_SMALL_GEMM: the solver's small products on the library's SIMT kernel
  bool ff_solve = false;       // a mixed-precision solve with fp64_hx_ff is running
  bool mixed_solve = false;    // a mixed-precision solve is running
  bool ff_now = false;         // the FP64 H X being launched uses the double-float angular kernel
  int radial_tc = 1;           // HW_OPT_RADIAL_KERNEL
  int overlap_launch = 1;      // HW_OPT_OVERLAP_LAUNCH: the FP32 H X chain by programmatic dependent launch
  int64_t rr_fallbacks = 0;    // Householder results rejected by the check (Jacobi used)
  // residual history of the last hw_solve_eigs: per k-point slot, per iteration (filter cycle
  // or LOBPCG iteration) the phase code (HW_HIST_*) and the largest wanted residual
  std::vector<std::vector<int>> hist_phase;
  std::vector<std::vector<double>> hist_res;
  std::vector<int> hist_k;     // k-point index of each slot
  hw::Prof prof;
};

// set the context's error message and return the status
hw_status hw_fail(hw_ctx* ctx, hw_status st, const std::string& msg);

namespace hw {
// Records [start, end) events of one phase on the context's stream when profiling is on.
class ProfScope {
 public:
  ProfScope(hw_ctx* ctx, int ph, double work = 0.0);
  ~ProfScope();
 private:
  hw_ctx* ctx_;
  int ph_;
  double work_;
  cudaEvent_t a_ = nullptr;
};
}  // namespace hw

#ifdef __CUDACC__
namespace hw {
// Launch k on the context's stream; overlap: with the programmatic-serialisation attribute (the
// kernel waits for its predecessor with griddep_wait before it touches that kernel's data).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(const hw_ctx* ctx, bool overlap, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                             Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = overlap ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}
}  // namespace hw
#endif

namespace hw {
template <typename T>
cudaError_t launch_hx(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, const ChebStep* step = nullptr);
cudaError_t hx_configure(hw_ctx* ctx);
bool density_fits(const hw_ctx* ctx, size_t tsz);
bool gradient_fits(const hw_ctx* ctx, size_t csz);
template <typename T>
cudaError_t launch_gradient(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, double* D);
template <typename T>
cudaError_t launch_density(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, const double* wcol, double* rho);
cudaError_t hx_autotune(hw_ctx* ctx, int k, int ns, std::vector<float>& log);
template <typename T>
cudaError_t launch_hx_into(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, void* gbuf, void* hbuf, int cols);
cudaError_t launch_tpa(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld);
// tensor-core radial transforms of the FP32 H X (hw_radial_tc.cu)
// 3-D TMA map over [planes][rows][Kp] BF16 (fp32 = false) or FP32 elements, box
// {swz / element size, box_rows, box_planes}, swz = 64 or 128-byte swizzle; false if the driver
// entry point is missing or the shape is rejected
bool make_plane_map(CUtensorMap* m, const void* base, bool fp32, int64_t Kp, int rows, int planes, int box_rows,
                    int box_planes, int swz);
// C_b = alpha op(A_b) B_b + beta C_b for small products (every extent below 1024) on the FP32
// pipe: cls 0 double-float (FP64 class), 1 FP32
cudaError_t zgemm_small(cudaStream_t st, int cls, bool transA, int m, int n, int k, double alpha, const double2* A,
                        int64_t lda, int64_t sA, const double2* B, int64_t ldb, int64_t sB, double beta, double2* C,
                        int64_t ldc, int64_t sC, int batch);
cudaError_t radial_tc_setup(hw_ctx* ctx, const HostBasis& hb, const std::vector<double>& rinv,
                            const std::vector<double>& rfwd);
cudaError_t launch_rinv_tc(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, int nc, int c0, void* gbuf,
                           int scale_mode);
cudaError_t launch_rfwd_tc(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld, int nc, int c0, void* hbuf,
                           const ChebStep* step);
// C = alpha op(A) B + beta C on the tensor cores (hw_zgemm.cu): cls 0 FP64 class, 1 FP32 class
cudaError_t zgemm_tc(ZgemmWork*& w, cudaStream_t st, int cls, bool transA, int m, int n, int k, double alpha,
                     const double2* A, int64_t lda, int64_t sA, const double2* B, int64_t ldb, int64_t sB,
                     double beta, double2* C, int64_t ldc, int64_t sC, int batch, int* launches);
void zgemm_free(ZgemmWork*& w);
int zgemm_status(ZgemmWork* w, cudaStream_t st, bool reset);
int* zgemm_status_ptr(ZgemmWork* w);
cudaError_t launch_precond_learned(hw_ctx* ctx, const Blocks& blk, int ns, int64_t ld,
                                   const double* const* ritz);
cudaError_t mlp_refresh_potential(hw_ctx* ctx);
void mlp_free_basis(hw_ctx* ctx);
void mlp_free(hw_ctx* ctx);
}  // namespace hw
