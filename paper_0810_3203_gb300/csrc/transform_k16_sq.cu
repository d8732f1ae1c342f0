// Per-pass launches of the sub-transform kernel (job_kernel.cuh) for rings of sixteen words per lane (N = 9216 .. 16384), omega = sqrt2.
#include "job_kernel.cuh"

namespace tftgpu {

TFT_DEFINE_PLAIN(16, sq, true)

}  // namespace tftgpu
