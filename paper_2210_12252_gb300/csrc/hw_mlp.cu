// Learned per-mode preconditioner (placeholder until the network kernels land).
#include "hw_ctx.h"

namespace hw {
struct MlpState {};
cudaError_t launch_precond_learned(hw_ctx*, const Blocks&, int, int64_t, const double* const*) {
  return cudaErrorNotSupported;
}
}  // namespace hw
