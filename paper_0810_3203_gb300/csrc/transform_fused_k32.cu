// Persistent launches of the sub-transform kernel (job_kernel.cuh) for rings of thirty-two words
// per lane: one launch runs every job of a plan's fused form, claiming jobs in dependency order.
#include "job_kernel.cuh"

namespace tftgpu {

cudaError_t launch_fused_k32(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, cudaStream_t s,
                             const FusedArgs &fa, uint32_t *fault, const Launch *plain, const CellMaps *cm) {
  return launch_fused_as<32>(p, x, stride_limbs, s, fa, fault, plain, cm);
}

}  // namespace tftgpu
