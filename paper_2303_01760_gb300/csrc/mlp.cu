// Learned weight predictor (placeholder until the predictor kernels land).
#include "common.cuh"

namespace hsm {

hsm_status compute_rbf_weights_learned(hsm_plan p, uint8_t*, int32_t*, int*) {
  return set_error(p, HSM_ESTATE, "no learned predictor attached");
}

}  // namespace hsm
