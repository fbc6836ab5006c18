// Adjoint of the imaging map (toi_degrid_backward); filled in by the
// differentiable-localisation path.
#include "toi_internal.cuh"

namespace toi {

cudaError_t launch_degrid_backward(toi_plan_s* p, Slot& s, const float* grad_image,
                                   float* grad_sample, float* grad_weight) {
  (void)p; (void)s; (void)grad_image; (void)grad_sample; (void)grad_weight;
  return cudaErrorNotSupported;
}

}  // namespace toi
