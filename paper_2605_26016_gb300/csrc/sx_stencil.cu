// Shared-memory halo stencil backend with the fused Heun step (placeholder until the kernel lands).
#include "sx_internal.h"

namespace sx {

int stencil_plan(sx_ctx *c) {
  (void)c;
  return set_error(SX_ERR_UNSUPPORTED, "stencil backend not built yet");
}
void stencil_free(sx_ctx *c) { c->stencil = nullptr; }
cudaError_t stencil_field(const sx_ctx *, const double *, double *, bool, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t stencil_heun_step(const sx_ctx *, const double *, double *, const HeunConst &, uint64_t, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace sx
