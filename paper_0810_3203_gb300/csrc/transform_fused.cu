// Persistent launches of the sub-transform kernel (job_kernel.cuh) for rings of four to sixteen
// words per lane whose words fill all 32 lanes (N = 4096, 8192, 16384): one launch runs every job
// of a plan's fused form, claiming jobs in dependency order. Other rings get no fused form from
// the planner.
#include "job_kernel.cuh"

namespace tftgpu {

cudaError_t launch_fused_small(const TransformPlan &p, uint64_t *x, int64_t stride_limbs, cudaStream_t s,
                               const FusedArgs &fa, uint32_t *fault, const Launch *plain, const CellMaps *cm) {
  switch (p.ring.K) {
    case 4: return launch_fused_as<4>(p, x, stride_limbs, s, fa, fault, plain, cm);
    case 8: return launch_fused_as<8>(p, x, stride_limbs, s, fa, fault, plain, cm);
    case 16: return launch_fused_as<16>(p, x, stride_limbs, s, fa, fault, plain, cm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tftgpu
