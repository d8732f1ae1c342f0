// Per-pass launches of the sub-transform kernel (job_kernel.cuh) for rings of one or two 32-bit words per lane (N <= 2048).
#include "job_kernel.cuh"

namespace tftgpu {

TFT_DEFINE_PLAIN(1, w2, false)
TFT_DEFINE_PLAIN(1, sq, true)
TFT_DEFINE_PLAIN(2, w2, false)
TFT_DEFINE_PLAIN(2, sq, true)

}  // namespace tftgpu
