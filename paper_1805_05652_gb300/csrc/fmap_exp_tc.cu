// Tensor-core (tcgen05) contraction of the exponential window: placeholder
// until the sm_103a kernels land; the plan refuses these precisions.
#include "fmap_device.cuh"

namespace fmap {

bool exp_tc_available(fmap_precision) { return false; }

size_t exp_tc_operand_bytes(const fmap_grid&, int32_t, int32_t, fmap_precision) { return 0; }

cudaError_t launch_exp_tc(fmap_plan_s*, const fmap_atoms*, float*, cudaStream_t,
                          int64_t* tiles_used) {
  *tiles_used = 0;
  return cudaErrorNotSupported;
}

}  // namespace fmap
