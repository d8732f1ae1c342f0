// Per-pass launches of the sub-transform kernel (job_kernel.cuh) for rings of thirty-two words per lane (N = 17408 .. 32768), omega = 2.
#include "job_kernel.cuh"

namespace tftgpu {

TFT_DEFINE_PLAIN(32, w2, false)

}  // namespace tftgpu
