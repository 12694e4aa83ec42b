// H X for callers that cannot allocate device memory.
//
// Some callers must not allocate once they are running: code that keeps to a device-memory
// budget fixed at start-up, code that runs where cudaMalloc is not permitted or would
// synchronise the device at the wrong moment, or hosts whose allocator owns all device memory.
// hw_apply_H_noalloc gives them the H X product without any allocation: the G / H intermediates
// of the three H X kernels live in one file-scope device array of HW_NOALLOC_SCRATCH_BYTES
// (64 MiB), which every GPU that loads this library holds until the process exits.  Columns
// are processed in as many passes as that array requires.
//
// The array is shared by every call on a device and keeps the last call's contents; nothing in
// it needs to start at zero (each pass writes every intermediate value before reading it).
// Calls whose work overlaps on the GPU (different streams, or different contexts on one device)
// race on the array and must be ordered by the caller.  The array's device address is resolved
// once per device and kept for the life of the process (a device reset is not supported).
#include <cstdint>
#include <mutex>

#include "hw_ctx.h"

namespace hw {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_addr_mu;
void* g_addr[64] = {nullptr};   // device address of the array, per device

// host code must not use g_noalloc_scratch's name as an address: resolve it once per device,
// with that device current
cudaError_t scratch_address(int device, void** out) {
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[device]) {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}
}  // namespace

}  // namespace hw

using namespace hw;

extern "C" hw_status hw_apply_H_noalloc(hw_ctx* ctx, int k, const double* X, double* Y, int ns, int64_t ld,
                                        hw_prec prec) {
  if (!ctx) return HW_EINVAL;
  if (ctx->device < 0) return hw_fail(ctx, HW_ESTATE, "host-only context has no device");
  if (!ctx->have_basis) return hw_fail(ctx, HW_ESTATE, "hw_setup_basis has not been called");
  if (!ctx->have_V) return hw_fail(ctx, HW_ESTATE, "no potential installed");
  if (k < 0 || k >= ctx->hb.nk) return hw_fail(ctx, HW_EINVAL, "k-point index out of range");
  if (!X || !Y || ns < 1 || ld < ctx->hb.L[k]) return hw_fail(ctx, HW_EINVAL, "bad block arguments");
  {
    // the byte ranges the block arguments span, [p, p + 16 ((ns - 1) ld + L))
    const uintptr_t span = 16u * ((uintptr_t)(ns - 1) * (uintptr_t)ld + (uintptr_t)ctx->hb.L[k]);
    const uintptr_t x0 = (uintptr_t)X, y0 = (uintptr_t)Y;
    if (x0 < y0 + span && y0 < x0 + span) return hw_fail(ctx, HW_EINVAL, "X and Y must not overlap");
  }
  if (prec != HW_FP64 && prec != HW_MIXED) return hw_fail(ctx, HW_EINVAL, "bad precision");
  const size_t elem = prec == HW_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t per_buf = (size_t)ctx->hb.prm.Nr * ctx->hb.nA * elem;   // one column of G (or H)
  const size_t cols = NOALLOC_SCRATCH_BYTES / (2 * per_buf);
  if (cols < 1)
    return hw_fail(ctx, HW_EINVAL,
                   "basis too large for the fixed 64 MiB scratch: one column needs " +
                       std::to_string(2 * per_buf) + " bytes");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  void* base = nullptr;
  cudaError_t e = scratch_address(ctx->device, &base);
  if (e == cudaSuccess) {
    Blocks blk;
    blk.nslot = 1;
    blk.x[0] = X;
    blk.y[0] = Y;
    blk.kb[0] = k;
    void* g = base;
    void* h = static_cast<unsigned char*>(base) + cols * per_buf;
    e = prec == HW_FP64 ? launch_hx_into<double>(ctx, blk, ns, ld, g, h, (int)cols)
                        : launch_hx_into<float>(ctx, blk, ns, ld, g, h, (int)cols);
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return hw_fail(ctx, HW_ECUDA, std::string("apply_H_noalloc: ") + cudaGetErrorString(e));
  return HW_OK;
}
