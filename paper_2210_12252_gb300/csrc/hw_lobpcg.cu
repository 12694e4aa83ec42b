// Block LOBPCG (placeholder until the solver lands).
#include "hw_ctx.h"

namespace hw {
struct LobpcgWork {};
void lobpcg_free(hw_ctx* ctx) {
  delete ctx->lw;
  ctx->lw = nullptr;
}
}  // namespace hw

extern "C" hw_status hw_solve_eigs(hw_ctx* ctx, int, const int*, int, int, double, int, hw_prec, int,
                                   const double* const*, double*, double* const*, int64_t, int*, double*) {
  return hw_fail(ctx, HW_ESTATE, "solver not built yet");
}
