// stencil3d.cu -- 3D time-step kernels (placeholder until the 2.5D kernel lands).
#include "fwi_internal.cuh"

namespace fwi {
cudaError_t launch_step3d(bool, const CUtensorMap&, const Layout&, const Coef&, const StepParams&, int, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace fwi
